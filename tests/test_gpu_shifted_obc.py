"""Shifted partitions of OBC lattices on the GPU (the paper covers every bond from a block
centre by partitions shifted against each other, Sec. "The blockBP algorithm"): block
boundaries at shift, shift + b, ..., the blocks on the lattice edges narrower.

* Parity with the oracle's shifted partition (FP64, 1e-10: residuals, messages, <O> inside
  blocks and across the moved block edges), on C1's lattice and on a truncating 6x6 D=3 case;
  the split-BF16 path within 1e-5 of the oracle there.
* Shifted strips form a chain of blocks (a tree): every observable equals brute force.
* Reading each term from the partition that holds it deepest inside a block
  (bbp_expect_centred); a bond on a block edge read from a partition that holds it inside a
  block is closer to brute force, the reason the paper gives for shifted partitions; the
  trace distance between the two-site RDMs of two partitions on the GPU equals the oracle's."""
import numpy as np
import pytest

import _exact as X
from _gpu import message_fidelity, run_both
from oracle import blockbp as ob
from paper_2301_05844_gb300 import binding as B
from paper_2301_05844_gb300 import inputs as I

pytestmark = pytest.mark.gpu
SZ, SX = I.SIGMA_Z, I.SIGMA_X


def close(a, b, tol=1e-10):
    a, b = np.asarray(a), np.asarray(b)
    return np.max(np.abs(a - b)) <= tol * max(1.0, np.max(np.abs(b)))


@pytest.mark.parametrize("shift", [(1, 1), (0, 1), (1, 0)])
def test_shifted_obc_parity_c1(shift):
    cfg = I.config(1)
    terms = I.standard_terms(4, 4)
    g, o, gr, orr, gv, ov = run_both(cfg["tensors"], 4, 4, 2, 2, 2, 2, 16, terms, n_sweeps=6, shift=shift)
    assert close(gr, orr, 1e-9), (gr, orr)
    assert message_fidelity(g, o) > 1 - 1e-10
    assert close(gv, ov)


def test_shifted_obc_truncating_and_split_bf16():
    """6x6, D=3, 3x3 blocks shifted by (1, 2): blocks of 1, 3, 2 columns and 2, 3, 1 rows,
    chi=12 (truncating)."""
    T = I.uniform_noise_peps(6, 6, 2, 3, seed=5)
    terms = [[(s, P)] for s in (0, 7, 14, 21, 28, 35) for P in (SZ, SX)] + \
        [[(7, SZ), (8, SZ)], [(8, SZ), (9, SZ)], [(14, SX), (20, SX)], [(20, SZ), (26, SZ)]]
    g, o, gr, orr, gv, ov = run_both(T, 6, 6, 2, 3, 3, 3, 12, terms, n_sweeps=3, chi_exp=20, shift=(1, 2))
    assert o.nbx == 3 and o.nby == 3
    assert close(gr, orr, 1e-9)
    assert close(gv, ov)
    g2, o2, gr2, orr2, gv2, ov2 = run_both(T, 6, 6, 2, 3, 3, 3, 12, terms, n_sweeps=3, chi_exp=20, shift=(1, 2),
                                           prec="bf16x3", oracle_fit_tol=3e-5, oracle_readout_fit_tol=3e-5)
    assert np.max(np.abs(gv2 - ov2)) < 1e-5, np.max(np.abs(gv2 - ov2))


@pytest.mark.parametrize("bx,by,shift", [(4, 2, (0, 1)), (2, 4, (1, 0)), (4, 1, (0, 0))])
def test_shifted_obc_strips_exact(bx, by, shift):
    T = I.uniform_noise_peps(4, 4, 2, 2, seed=1)
    terms = I.standard_terms(4, 4)
    g = B.Lattice(Lx=4, Ly=4, d=2, D=2, bx=bx, by=by, chi=16, chi_exp=18, fit_tol=0.0, fit_max_sweeps=2,
                  shift=shift)
    g.set_tensors(T)
    g.sweep(4)
    psi = X.state_vector(T, 4, 4)
    exact = np.array([X.exact_expect(psi, 16, 2, t) for t in terms])
    assert close(g.expect(terms), exact, 1e-11)


def test_centred_readout_and_rdm_trace_distance():
    """Four partitions of C1's lattice (shifts (0,0), (1,1), (0,1), (1,0)), converged: each
    term is read from a partition that holds it inside one block where one exists (the pair
    5-6 lies on a block edge unshifted, inside a block shifted by (1, 1): its error against
    brute force drops, 1.4e-4 -> 7.8e-5 in the oracle), and the values are those partitions'
    own read-outs.  (On this small lattice the shifted partitions' one-site edge blocks are
    poor elsewhere: the choice of partitions and block sizes is the caller's.)  The trace
    distance between the two-site RDMs of two partitions equals the oracle's."""
    cfg = I.config(1)
    T = cfg["tensors"]
    terms = I.standard_terms(4, 4)
    psi = X.state_vector(T, 4, 4)
    exact = np.array([X.exact_expect(psi, 16, 2, t) for t in terms])
    shifts = ((0, 0), (1, 1), (0, 1), (1, 0))
    lats, orc = [], []
    for sh in shifts:
        g = B.Lattice(Lx=4, Ly=4, d=2, D=2, bx=2, by=2, chi=16, fit_tol=1e-12, fit_max_sweeps=6, shift=sh)
        g.set_tensors(T)
        g.sweep(30)
        lats.append(g)
        o = ob.Lattice(4, 4, 2, 2, 2, 2, T, chi=16, fit_tol=1e-12, fit_max_sweeps=6, shift=sh)
        o.run(n_sweeps=30)
        orc.append(o)
    v, chosen = B.expect_centred(lats, terms)
    own = [lats[k].expect(terms) for k in range(len(lats))]
    assert close(v, np.array([own[k][i] for i, k in enumerate(chosen)]), 1e-12)
    assert close(v, np.array([orc[k].expect([t])[0] for t, k in zip(terms, chosen)]))
    for t, k in zip(terms, chosen):
        if len(t) == 2:
            rc = [divmod(s, 4) for s, _ in t]
            inside = [orc[j].block_of(*rc[0]) == orc[j].block_of(*rc[1]) for j in range(len(shifts))]
            assert inside[k] or not any(inside)
    i56 = next(i for i, t in enumerate(terms) if [s for s, _ in t] == [5, 6])
    assert chosen[i56] != 0 and abs(v[i56] - exact[i56]) < abs(own[0][i56] - exact[i56])
    for sites in ([5, 6], [9, 10]):
        dg = ob.trace_distance(lats[0].rdm(sites), lats[1].rdm(sites))
        do = ob.trace_distance(orc[0].rdm(sites), orc[1].rdm(sites))
        assert abs(dg - do) < 1e-10 and dg > 1e-8
