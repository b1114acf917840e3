"""The C-ABI library builds for sm_103a, loads without a GPU, and exports every
function that include/bbp.h declares (no compute calls here)."""
import ctypes
import os
import re
import subprocess

import numpy as np
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
    dict(Lx=6, Ly=6, d=1, D=3, bx=3, by=3, chi=8, single_layer=1, init_mode=1),
    dict(Lx=6, Ly=6, d=1, D=3, bx=3, by=3, chi=8, single_layer=1, prec="tf32x3", warm_start=1),
    dict(Lx=1, Ly=1, d=1, D=2, bx=4, by=4, chi=16, boundary="infinite", single_layer=1, prec="bf16"),
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


def test_footprint_is_planned_without_allocating(libpath):
    """bbp_lattice_footprint runs the planning only: it works without a GPU, grows
    with chi and with the lattice, and rejects what bbp_create_lattice rejects."""
    from paper_2301_05844_gb300 import binding as B
    f8 = B.footprint(Lx=12, Ly=12, d=2, D=3, bx=3, by=3, chi=8)
    f32 = B.footprint(Lx=12, Ly=12, d=2, D=3, bx=3, by=3, chi=32)
    big = B.footprint(Lx=24, Ly=24, d=2, D=3, bx=3, by=3, chi=8)
    assert 0 < f8 < f32 and f8 < big
    with pytest.raises(B.BBPError) as e:
        B.footprint(Lx=4, Ly=4, d=2, D=2, bx=3, by=2, chi=16)
    assert e.value.code == B.ERR_INVALID
    with pytest.raises(B.BBPError) as e:  # refused before any per-site host allocation
        B.footprint(Lx=8192, Ly=4, d=2, D=2, bx=2, by=2, chi=16)
    assert e.value.code == B.ERR_INVALID and "4096" in str(e.value)


def test_random_descriptions_plan_within_bounds(libpath):
    """Property test of the host planner: 500 seeded random descriptions (OBC and infinite,
    every precision, real, complex and single-layer tensors, blocks 1-15 sites a side,
    chi 1-79, fit and read-out options) all plan completely, and every task of every plan
    passes the host check of its operand ranges against the arena (bbp_lattice_footprint
    runs the planning and that check of bbp_create_lattice without allocating)."""
    from paper_2301_05844_gb300 import binding as B
    L = B.lib()
    rng = np.random.default_rng(2024)
    for _ in range(500):
        inf, single = rng.random() < 0.3, rng.random() < 0.25
        D, d = int(rng.integers(1, 6)), 1 if single else int(rng.integers(1, 4))
        if inf:
            Lx, Ly = int(rng.integers(1, 3)), int(rng.integers(1, 3))
            bx, by = Lx * int(rng.integers(1, 4)), Ly * int(rng.integers(1, 4))
        else:
            bx, by = int(rng.integers(1, 6)), int(rng.integers(1, 6))
            Lx, Ly = bx * int(rng.integers(1, 4)), by * int(rng.integers(1, 4))
        dtypes = [B.F64, B.F32] if single else [B.F64, B.C128, B.F32, B.C64]
        desc = B.make_desc(Lx, Ly, d, D, bx, by, int(rng.integers(1, 80)), boundary="infinite" if inf else "obc",
                           chi_exp=int(rng.integers(0, 40)), dtype=dtypes[int(rng.integers(0, len(dtypes)))],
                           prec=["fp64", "tf32", "bf16", "tf32x3"][int(rng.integers(0, 4))],
                           fit_max_sweeps=int(rng.integers(1, 11)), init_mode=int(rng.integers(0, 2)),
                           warm_start=int(rng.integers(0, 2)), hermitian_basis=int(rng.integers(0, 2)),
                           single_layer=int(single))
        nbytes = ctypes.c_size_t()
        rc = L.bbp_lattice_footprint(ctypes.byref(desc), ctypes.byref(nbytes))
        assert rc == B.OK and nbytes.value > 0, (rc, L.bbp_last_error().decode())


def test_shifted_partition_descriptions(libpath):
    """Shifted partitions: on infinite lattices 0 <= shift < unit cell (same footprint); with
    OBC 0 <= shift < block side, the blocks on the lattice edges narrower (a 4x4 lattice in
    2x2 blocks shifted by (1, 1) has 3 x 3 blocks and 24 messages instead of 8)."""
    from paper_2301_05844_gb300 import binding as B
    cell = dict(Lx=2, Ly=2, d=2, D=2, bx=4, by=4, chi=4, boundary="infinite")
    assert B.footprint(shift=(1, 1), **cell) == B.footprint(**cell)
    obc = dict(Lx=4, Ly=4, d=2, D=2, bx=2, by=2, chi=4)
    assert B.footprint(shift=(1, 1), **obc) > B.footprint(shift=(1, 0), **obc) > B.footprint(**obc)
    for bad in (dict(cell, shift=(2, 0)), dict(cell, shift=(0, -1)), dict(obc, shift=(2, 0)),
                dict(obc, shift=(0, -1))):
        with pytest.raises(B.BBPError) as e:
            B.footprint(**bad)
        assert e.value.code == B.ERR_INVALID


def test_single_layer_descriptions(libpath):
    """A single-layer network is planned with legs of dimension D (not D^2): it holds less
    than the PEPS of the same D, and it must have d = 1 and real tensors."""
    from paper_2301_05844_gb300 import binding as B
    cfg = dict(Lx=6, Ly=6, D=3, bx=3, by=3, chi=8)
    assert 0 < B.footprint(d=1, single_layer=1, **cfg) < B.footprint(d=2, **cfg)
    for bad in (dict(d=2, single_layer=1), dict(d=1, single_layer=1, dtype=B.C128), dict(d=1, single_layer=2)):
        with pytest.raises(B.BBPError) as e:
            B.footprint(**cfg, **bad)
        assert e.value.code == B.ERR_INVALID


def test_every_entry_point_catches_host_exceptions():
    """No C++ exception crosses the C boundary: every function the header declares
    (but bbp_last_error, which only returns a pointer) is defined with a
    function-try-block whose handler turns the exception into an error code."""
    csrc = os.path.join(ROOT, "paper_2301_05844_gb300", "csrc")
    src = "".join(open(os.path.join(csrc, f)).read() for f in sorted(os.listdir(csrc)) if f.endswith(".cu"))
    for f in declared_functions():
        if f == "bbp_last_error":
            continue
        m = re.search(rf"^(?:extern \"C\" )?(?:int|void) {f}\(([^)]*)\)\s*(try\s*)?\{{", src, flags=re.M)
        assert m, f"definition of {f} not found"
        assert m.group(2), f"{f} is not guarded by a function-try-block"
    assert src.count("abi_error();") >= len(declared_functions()) - 1


def test_server_host_logic_without_a_gpu(libpath):
    """Argument checks and admission run on the host: a request above the byte budget
    is refused at submission, bad descriptions and terms are rejected, and a request
    whose device allocation fails (no GPU here) finishes with that error code."""
    import numpy as np
    from paper_2301_05844_gb300 import binding as B
    from paper_2301_05844_gb300 import inputs
    L = B.lib()
    h = ctypes.c_void_p()
    assert L.bbp_server_create(0, 4, ctypes.byref(h)) == B.ERR_INVALID
    assert L.bbp_server_create(1 << 20, 0, ctypes.byref(h)) == B.ERR_INVALID
    cfg = dict(Lx=4, Ly=4, d=2, D=2, bx=2, by=2, chi=16)
    T = inputs.uniform_noise_peps(4, 4, 2, 2, seed=1)
    need = B.footprint(**cfg)
    srv = B.Server(max_bytes=need, max_active=2)
    try:
        with pytest.raises(B.BBPError) as e:
            srv.submit(T, **dict(cfg, Lx=8, Ly=8))  # refused before its tensors are read
        assert e.value.code == B.ERR_OOM
        with pytest.raises(B.BBPError) as e:
            srv.submit(T, **dict(cfg, bx=3))
        assert e.value.code == B.ERR_INVALID
        with pytest.raises(B.BBPError) as e:
            srv.submit(T, [[]], **cfg)  # a term on no site
        assert e.value.code == B.ERR_INVALID
        E = inputs.positive_network(4, 4, 2, seed=3)
        sl = dict(cfg, d=1, single_layer=1)
        with pytest.raises(B.BBPError) as e:  # an impurity at a site outside the lattice
            srv.submit(E, [[(16, np.ones((2, 2, 2, 2)))]], **sl)
        assert e.value.code == B.ERR_INVALID
        rid = srv.submit(T, [[(0, inputs.SIGMA_Z)]], **cfg)
        assert L.bbp_server_wait(srv.h, rid, -1.0) == B.ERR_INVALID
        assert L.bbp_server_wait(srv.h, rid, float("nan")) == B.ERR_INVALID
        assert L.bbp_server_wait(srv.h, rid, 60.0) in (B.ERR_OOM, B.ERR_CUDA)
        st = srv.poll(rid)
        assert st["state"] in (B.ERR_OOM, B.ERR_CUDA) and st["values"] is None
        s = srv.stats()
        assert s["submitted"] == 1 and s["done"] == 0 and s["bytes_in_use"] == 0
        assert L.bbp_server_poll(srv.h, 12345, None, None, None, None, None, None) == B.ERR_INVALID
    finally:
        srv.close()
