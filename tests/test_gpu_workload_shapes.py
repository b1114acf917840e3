"""GPU parity against the oracle at the shapes of the larger workloads.

* Infinite 2x2 complex unit cell, D=4, one 4x4 block messaging itself, chi=64 (the mixed-
  precision workload): the complex FP64 path against the complex oracle (same arithmetic
  sequence, 1e-10); the split tensor-core paths (TF32X3, BF16X3), which run complex tensors
  in the Hermitian basis, against the oracle in the same basis (1e-5, the bar the workload
  statement sets for reduced precision with FP64 truncation).  Plain TF32 / BF16 are held to
  ten times the unit roundoff of their operands (2^-11, 2^-8): they do not meet 1e-5.
* D=5, chi=96, 4x4 blocks (the 32x32 workload's tiles, bonds and truncation) on an 8x8
  lattice (4 blocks, 8 messages), tensors U[0,1] + 0.1 N(0,1) in FP32: FP64 against the
  oracle at 1e-10, TF32X3 and BF16X3 at 1e-5.
* The infinite D=4 case is ill-conditioned at one fit sweep per column: there FP64 parity is
  held to ten times the oracle's own response to a 1e-15 perturbation of its input.
* The fit stop rule active (App. A: std/|mean| of the losses below 1e-6, at most 10 fit
  sweeps) on the 12x12, D=3, chi=32 workload: the FP64 path runs exactly the oracle's
  number of fit sweeps in every message sweep and matches its <O> to 1e-10; the split paths
  (tolerance raised to 3e-5, the oracle likewise) match <O> to 1e-5.
Every run uses fixed message-sweep counts, so that both sides run the same steps."""
import numpy as np
import pytest

from _gpu import run_both
from oracle import blockbp as ob
from paper_2301_05844_gb300 import binding as B
from paper_2301_05844_gb300 import inputs as I

pytestmark = pytest.mark.gpu
SX, SY, SZ = I.SIGMA_X, I.SIGMA_Y, I.SIGMA_Z
TOL64, TOLMIX = 1e-10, 1e-5
UNIT_ROUNDOFF = {"tf32": 2.0 ** -11, "bf16": 2.0 ** -8}


def c3_terms():
    """sigma_a sigma_a (a = x, y, z) on the four nearest-neighbour bonds of the block's 2x2
    centre (the Heisenberg term is their sum / 4)."""
    ctr = [5, 6, 9, 10]
    bonds = [(ctr[0], ctr[1]), (ctr[2], ctr[3]), (ctr[0], ctr[2]), (ctr[1], ctr[3])]
    return [[(a, P), (b, P)] for a, b in bonds for P in (SX, SY, SZ)]


C3_KW = dict(Lx=2, Ly=2, d=2, D=4, bx=4, by=4, chi=64, boundary="infinite", fit_tol=0.0, fit_max_sweeps=1,
             seed=3, warm_start=True)
C3_SWEEPS = 2


def _c3_oracle(hb, tensors=None):
    cfg = I.config(3)
    T = [np.asarray(t) for t in cfg["tensors"]] if tensors is None else tensors
    k = dict(C3_KW)
    o = ob.Lattice(k["Lx"], k["Ly"], k["d"], k["D"], k["bx"], k["by"], T, boundary="infinite", chi=k["chi"],
                   fit_tol=k["fit_tol"], fit_max_sweeps=k["fit_max_sweeps"], seed=k["seed"],
                   warm_start=k["warm_start"], hermitian_basis=hb)
    res = [o.sweep() for _ in range(C3_SWEEPS)]
    return T, np.array(res), o.expect(c3_terms())


def _c3_gpu(T, prec, hb):
    g = B.Lattice(dtype=B.C64, prec=prec, hermitian_basis=hb, **C3_KW)
    g.set_tensors(T)
    res = [g.sweep(1)[0] for _ in range(C3_SWEEPS)]
    v = g.expect(c3_terms())
    g.close()
    return np.array(res), v


def test_c3_shape_complex_fp64_against_the_oracle():
    """The complex FP64 path against the complex oracle.  With N(0,1) complex tensors, chi=64
    truncates a flat spectrum and one fit sweep per column leaves the fits far from their
    optimum, so the result responds to rounding: the oracle itself, given tensors perturbed
    by 1e-15 relative, moves <O> by ~3e-7 (measured 2.6e-7).  The GPU is held to ten times
    that sensitivity, measured here, and to 1e-10 wherever the problem is better conditioned."""
    T, ores, ov = _c3_oracle(hb=False)
    rng = np.random.default_rng(0)
    Tp = [t.astype(np.complex128) * (1 + 1e-15 * rng.standard_normal(t.shape)) for t in T]
    _, pres, pv = _c3_oracle(hb=False, tensors=Tp)
    sens_o, sens_r = float(np.max(np.abs(pv - ov))), float(np.max(np.abs(pres - ores) / np.abs(ores)))
    gres, gv = _c3_gpu(T, "fp64", 0)
    assert np.max(np.abs(gres - ores) / np.abs(ores)) <= max(1e-9, 10 * sens_r), (gres, ores, sens_r)
    err = float(np.max(np.abs(gv - ov)))
    assert err <= max(TOL64, 10 * sens_o), (err, sens_o)


def test_c3_shape_tensor_core_paths_against_the_oracle():
    """Hermitian-basis oracle against the tensor-core paths; the plain complex oracle's
    difference from it (the basis changes how the truncated fits start) is not compared."""
    T, ores, ov = _c3_oracle(hb=True)
    err = {}
    for prec in ("tf32x3", "bf16x3", "tf32", "bf16"):
        gres, gv = _c3_gpu(T, prec, 1)
        err[prec] = float(np.max(np.abs(gv - ov)))
        assert gres[0] == pytest.approx(ores[0], rel=1e-2)
    assert err["tf32x3"] < TOLMIX and err["bf16x3"] < TOLMIX, err
    assert err["tf32"] < 10 * UNIT_ROUNDOFF["tf32"] and err["bf16"] < 10 * UNIT_ROUNDOFF["bf16"], err


def test_c4_shape_against_the_oracle():
    """D=5, chi=96, 4x4 blocks on an 8x8 lattice, 2 warm-started message sweeps of one fit
    sweep per column: <sigma_z>, <sigma_x> on the centre sites of every block."""
    L, D, chi = 8, 5, 96
    T = I.uniform_noise_peps(L, L, 2, D, seed=4, dtype=np.float32)
    T64 = [np.asarray(t, dtype=np.float64) for t in T]
    centres = [18, 19, 26, 27, 21, 22, 29, 30, 34, 35, 42, 43, 37, 38, 45, 46]
    terms = [[(s, P)] for s in centres for P in (SZ, SX)]
    kw = dict(fit_tol=0.0, fit_max_sweeps=1, seed=4, warm_start=True)
    o = ob.Lattice(L, L, 2, D, 4, 4, T64, chi=chi, **kw)
    ores = np.array([o.sweep() for _ in range(2)])
    ov = o.expect(terms)
    err = {}
    for prec in ("fp64", "tf32x3", "bf16x3"):
        g = B.Lattice(Lx=L, Ly=L, d=2, D=D, bx=4, by=4, chi=chi, dtype=B.F32, prec=prec, **kw)
        g.set_tensors(T)
        gres = np.array([g.sweep(1)[0] for _ in range(2)])
        gv = g.expect(terms)
        g.close()
        err[prec] = float(np.max(np.abs(gv - ov)))
        if prec == "fp64":
            assert np.allclose(gres, ores, rtol=1e-8, atol=1e-13), (gres, ores)
    assert err["fp64"] < TOL64 and err["tf32x3"] < TOLMIX and err["bf16x3"] < TOLMIX, err


def c2_terms():
    return [[(s, SZ)] for s in range(0, 144, 7)] + [[(s, SX)] for s in range(0, 144, 11)] + \
        [[(13, SZ), (14, SZ)], [(52, SZ), (64, SZ)], [(2, SX), (3, SX)]]


def test_active_fit_stop_rule_fp64_counts_and_values():
    """The fit loops stop by the App. A rule (1e-6, at most 10 sweeps): in every message
    sweep the FP64 path runs the oracle's number of fit sweeps, summed over all column fits,
    and ends at the oracle's <O>."""
    cfg = I.config(2)
    T = cfg["tensors"]
    g = B.Lattice(Lx=12, Ly=12, d=2, D=3, bx=3, by=3, chi=32, prec="fp64", fit_tol=1e-6, fit_max_sweeps=10, seed=7)
    g.set_tensors(T)
    o = ob.Lattice(12, 12, 2, 3, 3, 3, [np.asarray(t) for t in T], chi=32, fit_tol=1e-6, fit_max_sweeps=10, seed=7)
    gcounts, gres, ores = [], [], []
    prev = 0
    for _ in range(4):
        gres.append(g.sweep(1)[0])
        ores.append(o.sweep())
        fs = g.stats()["fit_sweeps"]
        gcounts.append(fs - prev)
        prev = fs
    nfits = 48 * 3
    assert gcounts == o.fit_sweeps, (gcounts, o.fit_sweeps)
    assert any(c > nfits for c in gcounts) and all(c < 10 * nfits for c in gcounts)  # the rule was active
    assert np.allclose(gres, ores, rtol=1e-8, atol=1e-14)
    gv, ov = g.expect(c2_terms()), o.expect(c2_terms())
    assert np.max(np.abs(gv - ov)) < TOL64, np.max(np.abs(gv - ov))


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_active_fit_stop_rule_split_paths(prec):
    """The split tensor-core paths under the same active stop rule (the paper's 1e-6, raised to
    the paths' 3e-5; the oracle at the same tolerances): <O> within 1e-5 of the oracle after 6
    sweeps."""
    cfg = I.config(2)
    g, o, gr, orr, gv, ov = run_both(cfg["tensors"], 12, 12, 2, 3, 3, 3, 32, c2_terms(), n_sweeps=6, fit_tol=1e-6,
                                     fit_max_sweeps=10, prec=prec, warm_start=True, oracle_fit_tol=3e-5,
                                     oracle_readout_fit_tol=3e-5)
    assert np.max(np.abs(gv - ov)) < TOLMIX, np.max(np.abs(gv - ov))
