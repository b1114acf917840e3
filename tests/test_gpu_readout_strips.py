"""Read-out closings shared per column strip (App. A read-out: <O> = N_O / N_I from the
block, its incoming messages and the environment columns): terms whose operators sit on
non-adjacent rows of one column, on diagonal sites of two columns, in two columns of one
block and across block edges.  FP64 closings are compared with the oracle at the FP64
tolerance; FP32 closings (tensor-core lattices) with the oracle at the split paths' bound
and with the same lattice's FP64 closings, also on 16-row blocks (every strip environment is
rescaled by a power of two as it is formed)."""
import numpy as np
import pytest

from _gpu import run_both
from paper_2301_05844_gb300 import inputs as I

pytestmark = pytest.mark.gpu
SZ, SX, SY = I.SIGMA_Z, I.SIGMA_X, I.SIGMA_Y
TOL64 = 1e-10
BOUND_SPLIT = 1e-5  # split paths (TF32X3, BF16X3) against the oracle


def strip_terms():
    # 6x6 OBC lattice, 3x3 blocks; site s = 6 * row + col
    return [
        [(14, SZ)], [(35, SX)], [(0, SZ)],
        [(0, SZ), (12, SZ)],    # column 0, rows 0 and 2 of block 0 (a plain row between them)
        [(1, SX), (13, SZ)],    # column 1, rows 0 and 2
        [(0, SX), (7, SX)],     # diagonal: rows 0 and 1 of columns 0 and 1
        [(3, SZ), (4, SX)],     # two columns of block 1
        [(19, SZ), (26, SZ)],   # diagonal in block 2
        [(12, SX), (18, SX)],   # vertical pair across the block row edge
        [(2, SZ), (3, SZ)],     # horizontal pair across the block column edge
    ]


def test_strip_geometries_fp64():
    T = I.uniform_noise_peps(6, 6, 2, 2, seed=41)
    g, o, gr, orr, gv, ov = run_both(T, 6, 6, 2, 2, 3, 3, 16, strip_terms(), n_sweeps=3, chi_exp=20)
    scale = max(1.0, float(np.max(np.abs(ov))))
    assert np.max(np.abs(gv - ov)) <= TOL64 * scale, np.max(np.abs(gv - ov))


def test_strip_geometries_complex_fp64():
    rng = np.random.default_rng(43)
    T = I.uniform_noise_peps(6, 6, 2, 2, seed=43)
    T = [t + 0.3j * rng.standard_normal(t.shape) for t in T]
    terms = strip_terms() + [[(2, SY), (14, SY)]]
    g, o, gr, orr, gv, ov = run_both(T, 6, 6, 2, 2, 3, 3, 16, terms, n_sweeps=3, chi_exp=20)
    scale = max(1.0, float(np.max(np.abs(ov))))
    assert np.max(np.abs(gv - ov)) <= TOL64 * scale, np.max(np.abs(gv - ov))


@pytest.mark.parametrize("prec", ["tf32x3", "bf16x3"])
def test_strip_geometries_fp32_closings(prec):
    T = I.uniform_noise_peps(6, 6, 2, 2, seed=42)
    terms = strip_terms()
    out = {}
    for keep in (0, 1):
        g, o, gr, orr, gv, ov = run_both(T, 6, 6, 2, 2, 3, 3, 16, terms, n_sweeps=4, chi_exp=20, prec=prec,
                                         oracle_fit_tol=3e-5, oracle_readout_fit_tol=3e-5, keep_fp64=keep)
        assert np.max(np.abs(gv - ov)) < BOUND_SPLIT, (keep, np.max(np.abs(gv - ov)))
        out[keep] = gv
        g.close()
    assert np.max(np.abs(out[0] - out[1])) < BOUND_SPLIT


def test_tall_blocks_fp32_closings():
    """4x16 OBC lattice, two 2x16 blocks (18-row strips), D=2."""
    T = I.uniform_noise_peps(4, 16, 2, 2, seed=44)
    terms = [[(s, SZ)] for s in (0, 5, 33, 62, 63)] + [[(s, SX)] for s in (2, 30, 61)] + \
        [[(8, SZ), (12, SZ)], [(1, SX), (2, SX)], [(40, SZ), (45, SZ)], [(20, SZ), (36, SZ)]]
    vals = {}
    for keep in (0, 1):
        g, o, gr, orr, gv, ov = run_both(T, 4, 16, 2, 2, 2, 16, 8, terms, n_sweeps=3, prec="tf32x3",
                                         oracle_fit_tol=3e-5, oracle_readout_fit_tol=3e-5, keep_fp64=keep)
        assert np.all(np.isfinite(gv))
        assert np.max(np.abs(gv - ov)) < BOUND_SPLIT, (keep, np.max(np.abs(gv - ov)))
        vals[keep] = gv
        g.close()
    assert np.max(np.abs(vals[0] - vals[1])) < BOUND_SPLIT
