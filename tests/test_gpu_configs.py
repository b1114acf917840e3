"""Workload-shape checks on the GPU beyond the oracle-sized cases.

C4 shape (D=5, chi=96, 4x4 blocks, TF32): the tensor-core path against the FP64 GPU path
on the same lattice, the same generator draws and the same fixed number of sweeps, so
that the difference is the contraction precision alone (the C4 statement compares TF32
with FP64 on the GPU).  An 8x8 lattice (4 blocks, 8 messages) keeps the FP64 run short;
the tiles, bonds and truncation are those of the 32x32 workload."""
import numpy as np
import pytest

from paper_2301_05844_gb300 import binding as B
from paper_2301_05844_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def test_c4_shape_tf32_against_fp64_on_gpu():
    L, D, chi = 8, 5, 96
    T = I.uniform_noise_peps(L, L, 2, D, seed=4, dtype=np.float32)
    terms = [[(s, P)] for s in (18, 19, 26, 27, 36, 45) for P in (I.SIGMA_Z, I.SIGMA_X)]
    vals = {}
    for prec in ("fp64", "tf32"):
        g = B.Lattice(Lx=L, Ly=L, d=2, D=D, bx=4, by=4, chi=chi, dtype=B.F32, prec=prec, fit_tol=1e-6,
                      fit_max_sweeps=3, seed=4, warm_start=1)
        g.set_tensors(T)
        r, k, _ = g.sweep(3)
        vals[prec] = (g.expect(terms), r)
        g.close()
    d = np.max(np.abs(vals["tf32"][0] - vals["fp64"][0]))
    assert d < 1e-4, d
    assert np.all(np.abs(vals["tf32"][0].imag) == 0)
