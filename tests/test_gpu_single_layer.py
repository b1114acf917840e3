"""Single-layer networks on the GPU: the tensors are the network's own K-leg site tensors
(a 2D classical model's partition function, Sec. on the 2D Ising model), contracted as they
are, with impurity tensors for the read-out.

FP64: the same arithmetic sequence as the oracle (fixed sweeps and fit sweeps, the same
generator draws), 1e-10.  Tree block graphs: exact against the exact contraction.  The
classical Ising network on the infinite path: |<s>| against Onsager's magnetisation on the
FP64 and tensor-core paths (the FP64 oracle is within 6.0e-5 of it at this block size)."""
import math

import numpy as np
import pytest

import _exact as X
from _gpu import message_fidelity, run_both
from paper_2301_05844_gb300 import binding as B
from paper_2301_05844_gb300 import inputs as I

pytestmark = pytest.mark.gpu
BETA = 0.6


def onsager(beta):
    s = math.sinh(2 * beta)
    return (1 - s ** -4) ** 0.125 if s > 1 else 0.0


def _terms(E, seed, sites):
    """Terms with seeded random impurity tensors (each the shape of the site it replaces)."""
    rng = np.random.default_rng(seed)
    imp = {s: rng.uniform(-1.0, 1.0, np.shape(E[s])) for s in sorted({x for t in sites for x in t})}
    return [[(s, imp[s]) for s in t] for t in sites]


def test_single_layer_fp64_parity_truncating():
    """6x6 OBC network, K=3, 3x3 blocks (a loop of four blocks), chi=8 (the column MPS are
    truncated), uniform random initial messages; impurities inside a block, across a block
    edge and on the lattice corner."""
    E = I.positive_network(6, 6, 3, seed=21)
    terms = _terms(E, 4, [(7,), (0,), (14,), (7, 8), (8, 9), (2, 8), (20, 26), (35,)])
    g, o, gr, orr, gv, ov = run_both(E, 6, 6, 1, 3, 3, 3, 8, terms, n_sweeps=3, chi_exp=20, init_mode=1, seed=9,
                                     single_layer=True)
    assert np.allclose(gr, orr, rtol=1e-9, atol=1e-14), (gr, orr)
    assert message_fidelity(g, o) > 1 - 1e-10
    assert np.max(np.abs(gv - ov)) <= 1e-10 * max(1.0, np.max(np.abs(ov)))


@pytest.mark.parametrize("bx,by", [(4, 1), (1, 4), (4, 2)])
def test_single_layer_tree_strips_exact(bx, by):
    E = I.positive_network(4, 4, 2, seed=11)
    terms = _terms(E, 7, [(5,), (0,), (5, 6), (6, 10), (1, 2)])
    nblk = (4 // bx) * (4 // by)
    g, o, gr, orr, gv, ov = run_both(E, 4, 4, 1, 2, bx, by, 16, terms, n_sweeps=nblk + 1, chi_exp=18,
                                     single_layer=True)
    Z = X.network_value(E, 4, 4)
    exact = np.array([X.network_value(E, 4, 4, dict(t)) / Z for t in terms])
    assert np.max(np.abs(gv - exact)) < 1e-11
    assert np.max(np.abs(gv - ov)) < 1e-10


def test_single_layer_ising_fp64_parity_with_oracle():
    E, Ez = I.ising_network(BETA, h=1e-6)
    terms = [[(s, Ez)] for s in (5, 6, 9, 10)] + [[(5, Ez), (6, Ez)]]
    g, o, gr, orr, gv, ov = run_both([E], 1, 1, 1, 2, 4, 4, 16, terms, 6, boundary="infinite", fit_tol=0.0,
                                     fit_max_sweeps=2, seed=3, init_mode=1, single_layer=True)
    assert np.max(np.abs(gv - ov)) < 1e-10, np.max(np.abs(gv - ov))
    assert np.allclose(gr, orr, rtol=1e-6, atol=1e-14)


@pytest.mark.parametrize("prec,tol", [("fp64", 1.5e-4), ("tf32x3", 1.5e-4), ("bf16", 2e-3)])
def test_single_layer_ising_against_onsager(prec, tol):
    E, Ez = I.ising_network(BETA, h=1e-6)
    g = B.Lattice(Lx=1, Ly=1, d=1, D=2, bx=4, by=4, chi=16, boundary="infinite", prec=prec, fit_tol=1e-6,
                  fit_max_sweeps=10, seed=3, init_mode=1, warm_start=1, single_layer=1)
    g.set_tensors([E])
    g.sweep(30)
    m = g.expect([[(5, Ez)]])[0].real
    assert abs(abs(m) - onsager(BETA)) < tol, (m, onsager(BETA))


def test_single_layer_tensor_cores_against_fp64():
    """The truncating 6x6 network run to convergence on the split-TF32 path agrees with
    the FP64 path within the 1e-5 that the tensor-core paths are held to."""
    E = I.positive_network(6, 6, 3, seed=21)
    terms = _terms(E, 4, [(7,), (14,), (7, 8), (8, 9), (20, 26)])
    vals = {}
    for prec in ("fp64", "tf32x3"):
        g = B.Lattice(Lx=6, Ly=6, d=1, D=3, bx=3, by=3, chi=8, prec=prec, fit_tol=1e-6, fit_max_sweeps=10, seed=9,
                      init_mode=1, warm_start=1, single_layer=1)
        g.set_tensors(E)
        g.sweep(25)
        vals[prec] = g.expect(terms)
    assert np.max(np.abs(vals["tf32x3"] - vals["fp64"])) < 1e-5


def test_single_layer_served_solve_equals_solve_alone():
    """A single-layer solve through the request server returns exactly what the same solve
    returns alone (the server copies each impurity tensor at its site's shape)."""
    E = I.positive_network(4, 4, 2, seed=11)
    terms = _terms(E, 7, [(5,), (0,), (5, 6), (1, 2)])
    kw = dict(Lx=4, Ly=4, d=1, D=2, bx=2, by=2, chi=16, tol=1e-10, max_sweeps=30, seed=1, single_layer=1)
    srv = B.Server(max_bytes=1 << 30, max_active=2)
    try:
        out = srv.wait(srv.submit(E, terms, **kw), timeout_s=300.0)
    finally:
        srv.close()
    g = B.Lattice(**kw)
    g.set_tensors(E)
    g.sweep(0)
    assert np.array_equal(out["values"], g.expect(terms))
