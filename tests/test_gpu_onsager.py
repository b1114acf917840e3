"""The infinite path on the GPU against the classical 2D Ising model: the PEPS whose norm is
the Ising partition function (inputs.ising_peps), one 4x4 block messaging itself.

FP64: the same arithmetic sequence as the oracle (fixed sweeps and fit sweeps, the same
generator draws for the random initial messages), 1e-10.  Tensor-core paths: run to
convergence, <sz> against Onsager's magnetisation deep in the ordered phase, where the
FP64 oracle is within 6.0e-5 of it at this block size."""
import math

import numpy as np
import pytest

from _gpu import run_both
from paper_2301_05844_gb300 import binding as B
from paper_2301_05844_gb300 import inputs as I

pytestmark = pytest.mark.gpu
BETA = 0.6


def onsager(beta):
    s = math.sinh(2 * beta)
    return (1 - s ** -4) ** 0.125 if s > 1 else 0.0


def test_ising_fp64_parity_with_oracle():
    T = [I.ising_peps(BETA, h=1e-6)]
    terms = [[(s, I.SIGMA_Z)] for s in (5, 6, 9, 10)] + [[(5, I.SIGMA_Z), (6, I.SIGMA_Z)]]
    g, o, gr, orr, gv, ov = run_both(T, 1, 1, 2, 2, 4, 4, 16, terms, 6, boundary="infinite", fit_tol=0.0,
                                     fit_max_sweeps=2, seed=3, init_mode=1)
    assert np.max(np.abs(gv - ov)) < 1e-10, np.max(np.abs(gv - ov))
    assert np.allclose(gr, orr, rtol=1e-6, atol=1e-14)


@pytest.mark.parametrize("prec,tol", [("tf32x3", 1.5e-4), ("bf16", 2e-3)])
def test_ising_tensor_cores_against_onsager(prec, tol):
    g = B.Lattice(Lx=1, Ly=1, d=2, D=2, bx=4, by=4, chi=16, boundary="infinite", prec=prec, fit_tol=1e-6,
                  fit_max_sweeps=10, seed=3, init_mode=1, warm_start=1)
    g.set_tensors([I.ising_peps(BETA, h=1e-6)])
    g.sweep(30)
    m = g.expect([[(5, I.SIGMA_Z)]])[0].real
    assert abs(m - onsager(BETA)) < tol, (m, onsager(BETA))
