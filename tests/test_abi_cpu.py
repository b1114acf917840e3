"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
function that include/bbp.h declares (no compute calls here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bbp.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\**\s+\**(bbp_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2301_05844_gb300 import build
    if not os.path.exists(build.LIB) or os.environ.get("BBP_REBUILD"):
        build.build()
    return build.LIB


def test_header_declares_the_boundary():
    fns = declared_functions()
    for f in ("bbp_create_lattice", "bbp_set_tensors", "bbp_sweep", "bbp_expect", "bbp_destroy", "bbp_last_error"):
        assert f in fns


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    missing = [f for f in declared_functions() if not hasattr(lib, f)]
    assert not missing
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    for f in declared_functions():
        assert re.search(rf"\bT {f}\b", out), f


def test_binding_has_no_fallback_and_null_handles_are_rejected(libpath):
    from paper_2301_05844_gb300 import binding as B
    L = B.lib()
    assert L.bbp_sweep(None, 1, None, None) == B.ERR_INVALID
    assert b"NULL" in L.bbp_last_error()
    L.bbp_destroy(None)  # no-op
    desc = B.make_desc(4, 4, 2, 2, 3, 2, 16)  # 3 does not divide 4
    h = ctypes.c_void_p()
    assert L.bbp_create_lattice(ctypes.byref(desc), ctypes.byref(h)) == B.ERR_INVALID


@pytest.mark.parametrize("cfg", [
    dict(Lx=4, Ly=4, d=2, D=2, bx=2, by=2, chi=16),
    dict(Lx=12, Ly=12, d=2, D=3, bx=3, by=3, chi=32),
    dict(Lx=2, Ly=2, d=2, D=4, bx=4, by=4, chi=64, boundary="infinite", dtype=3),
    dict(Lx=6, Ly=6, d=2, D=3, bx=3, by=2, chi=12, dtype=1),
    dict(Lx=4, Ly=4, d=2, D=2, bx=4, by=4, chi=16),
])
def test_sweep_plan_passes_the_bounds_check(libpath, cfg):
    """Planning and the host-side bounds check of every task run before any CUDA
    call: without a GPU creation stops at the arena allocation (OOM), never at an
    internal plan error."""
    from paper_2301_05844_gb300 import binding as B
    L = B.lib()
    desc = B.make_desc(**cfg)
    h = ctypes.c_void_p()
    rc = L.bbp_create_lattice(ctypes.byref(desc), ctypes.byref(h))
    msg = L.bbp_last_error().decode()
    assert rc in (B.OK, B.ERR_OOM), msg
    assert "internal" not in msg
    if rc == B.OK:
        L.bbp_destroy(h)


def test_library_generator_matches_the_oracle_definition(libpath):
    """The counter-based generator in the library equals the oracle's SplitMix64
    definition bit for bit (both sides draw the same initial fit states)."""
    import numpy as np
    from oracle import blockbp as ob
    L = ctypes.CDLL(libpath)
    L.bbp_selftest_rng.argtypes = [ctypes.c_ulonglong, ctypes.c_ulonglong, ctypes.c_longlong, ctypes.c_void_p]
    for seed, stream in [(0, 0), (7, ob.stream_id(0, 3, 17, 2, 4)), (2**63 + 5, ob.stream_id(1, 9, 1, 0, 3))]:
        out = np.zeros(257)
        assert L.bbp_selftest_rng(seed, stream, 257, out.ctypes.data) == 0
        assert np.array_equal(out, ob.uniform_pm1(seed, stream, 257))
