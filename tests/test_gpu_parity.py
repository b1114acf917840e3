"""GPU parity: the CUDA library (through the C ABI) against the FP64 oracle on the
same seeded inputs, same fit-sweep counts and same generator streams.  Compared are
gauge-invariant quantities only: residuals, <O>, and message overlaps.  FP64 path:
1e-10 relative (the tolerance the workload statement fixes for the FP64 path)."""
import math

import numpy as np
import pytest

import _exact as X
from _gpu import message_fidelity, run_both
from paper_2301_05844_gb300 import binding as B
from paper_2301_05844_gb300 import inputs as I

pytestmark = pytest.mark.gpu
SZ, SX, SY = I.SIGMA_Z, I.SIGMA_X, I.SIGMA_Y
TOL64 = 1e-10


def close(a, b, tol=TOL64):
    a, b = np.asarray(a), np.asarray(b)
    return np.max(np.abs(a - b)) <= tol * max(1.0, np.max(np.abs(b)))


def test_config1_fp64_parity_and_brute_force():
    """4x4 OBC, D=2, 2x2 blocks, chi=16: residual per sweep, messages and the 56
    standard observables match the oracle; error vs brute force is reported."""
    cfg = I.config(1)
    terms = I.standard_terms(4, 4)
    g, o, gr, orr, gv, ov = run_both(cfg["tensors"], 4, 4, 2, 2, 2, 2, 16, terms, n_sweeps=6)
    assert close(gr, orr, 1e-9), (gr, orr)
    assert message_fidelity(g, o) > 1 - 1e-10
    assert close(gv, ov)
    psi = X.state_vector(cfg["tensors"], 4, 4)
    ex = np.array([X.exact_expect(psi, 16, 2, t) for t in terms])
    err = np.max(np.abs(gv - ex))
    assert err < 1e-3  # blockBP approximation on a loop block graph (reported, not parity)


@pytest.mark.parametrize("bx,by", [(4, 1), (1, 4), (4, 2)])
def test_tree_strips_exact_on_gpu(bx, by):
    T = I.uniform_noise_peps(4, 4, 2, 2, seed=1)
    terms = I.standard_terms(4, 4)
    nblk = (4 // bx) * (4 // by)
    g, o, gr, orr, gv, ov = run_both(T, 4, 4, 2, 2, bx, by, 16, terms, n_sweeps=nblk + 1, chi_exp=18)
    psi = X.state_vector(T, 4, 4)
    ex = np.array([X.exact_expect(psi, 16, 2, t) for t in terms])
    assert close(gv, ex, 1e-11)
    assert close(gv, ov)


def test_complex_obc_ragged_tiles():
    """6x6 OBC, D=3 (K=9), 3x3 blocks, chi=12 (truncating): ragged 64-wide tiles, complex."""
    rng = np.random.default_rng(31)
    T = I.uniform_noise_peps(6, 6, 2, 3, seed=5)
    T = [t + 0.2j * rng.standard_normal(t.shape) for t in T]
    terms = [[(7, SZ)], [(14, SX)], [(7, SZ), (8, SZ)], [(8, SY), (9, SY)], [(2, SX), (8, SX)], [(20, SZ), (26, SZ)]]
    g, o, gr, orr, gv, ov = run_both(T, 6, 6, 2, 3, 3, 3, 12, terms, n_sweeps=3, chi_exp=20)
    assert close(gr, orr, 1e-9)
    assert message_fidelity(g, o) > 1 - 1e-10
    assert close(gv, ov)


def test_infinite_complex_cell():
    """Infinite 2x2 unit cell, complex, D=2, 2x2 block messaging itself."""
    T = I.complex_normal_cell(2, 2, 2, 2, seed=3)
    T = [t.astype(np.complex128) for t in T]
    terms = [[(0, SZ)], [(3, SX)], [(0, SZ), (1, SZ)], [(1, SX), (3, SX)]]
    g, o, gr, orr, gv, ov = run_both(T, 2, 2, 2, 2, 2, 2, 4, terms, n_sweeps=4, boundary="infinite")
    assert close(gr, orr, 1e-9)
    assert close(gv, ov)


def test_infinite_shifted_partition():
    """Infinite 2x2 complex cell, 4x4 block, the partition shifted by (1, 1): parity with the
    oracle's shifted partition, and bit for bit the run of the cell rolled by one site."""
    T = [t.astype(np.complex128) for t in I.complex_normal_cell(2, 2, 2, 2, seed=3)]
    terms = [[(0, SZ)], [(5, SX)], [(5, SZ), (6, SZ)], [(6, SX), (10, SX)]]
    g, o, gr, orr, gv, ov = run_both(T, 2, 2, 2, 2, 4, 4, 4, terms, n_sweeps=3, boundary="infinite",
                                     shift=(1, 1))
    assert close(gr, orr, 1e-9)
    assert close(gv, ov)
    rolled = [T[((r + 1) % 2) * 2 + (c + 1) % 2] for r in range(2) for c in range(2)]
    g2, o2, gr2, orr2, gv2, ov2 = run_both(rolled, 2, 2, 2, 2, 4, 4, 4, terms, n_sweeps=3, boundary="infinite")
    assert np.array_equal(gv, gv2)


def test_nonsquare_blocks_and_random_init():
    T = I.uniform_noise_peps(4, 4, 2, 2, seed=1)
    terms = I.standard_terms(4, 4)
    g, o, gr, orr, gv, ov = run_both(T, 4, 4, 2, 2, 2, 1, 8, terms, n_sweeps=3, init_mode=1, seed=11)
    assert close(gr, orr, 1e-9)
    assert close(gv, ov)


def test_single_block_no_messages():
    T = I.uniform_noise_peps(4, 4, 2, 2, seed=1)
    terms = I.standard_terms(4, 4)
    g = B.Lattice(Lx=4, Ly=4, d=2, D=2, bx=4, by=4, chi=16, chi_exp=64, fit_tol=0.0, fit_max_sweeps=2)
    g.set_tensors(T)
    r, k, rc = g.sweep(3)
    assert r == 0.0
    psi = X.state_vector(T, 4, 4)
    ex = np.array([X.exact_expect(psi, 16, 2, t) for t in terms])
    assert close(g.expect(terms), ex, 1e-11)


def test_error_paths():
    g = B.Lattice(Lx=4, Ly=4, d=2, D=2, bx=2, by=2, chi=16)
    with pytest.raises(B.BBPError) as e:
        g.sweep(1)
    assert e.value.code == B.ERR_STATE
    g.set_tensors(I.uniform_noise_peps(4, 4, 2, 2, seed=1))
    g.sweep(1)
    with pytest.raises(B.BBPError) as e:
        g.expect([[(0, SZ), (10, SZ)]])  # different blocks, not neighbours
    assert e.value.code == B.ERR_INVALID
    with pytest.raises(B.BBPError) as e:
        g.expect([[(99, SZ)]])
    assert e.value.code == B.ERR_INVALID


@pytest.mark.parametrize("chi", [16, 6])
def test_warm_start_parity(chi):
    """Fits started from the previous sweep's result, on both sides: same residuals,
    messages and <O>, with the full bond (16) and a truncating one (6)."""
    cfg = I.config(1)
    terms = I.standard_terms(4, 4)
    g, o, gr, orr, gv, ov = run_both(cfg["tensors"], 4, 4, 2, 2, 2, 2, chi, terms, n_sweeps=6, warm_start=True,
                                     fit_max_sweeps=2)
    assert close(gr, orr, 1e-9), (gr, orr)
    assert message_fidelity(g, o) > 1 - 1e-10
    assert close(gv, ov)


@pytest.mark.parametrize("chi", [16, 6])
def test_warm_start_readout_parity(chi):
    """Warm read-out (warm_start = 2) with chi_exp = chi: the read-out's environment columns of every one-block
    region start from the sweep's last fits in the same frame, on both sides (blocks at the
    lattice edge have no message toward it and start cold); same <O>."""
    cfg = I.config(1)
    terms = I.standard_terms(4, 4)
    g, o, gr, orr, gv, ov = run_both(cfg["tensors"], 4, 4, 2, 2, 2, 2, chi, terms, n_sweeps=4, warm_start=2,
                                     fit_max_sweeps=2, chi_exp=chi)
    assert close(gr, orr, 1e-9), (gr, orr)
    assert close(gv, ov)


def test_warm_start_readout_truncating_6x6():
    """6x6 OBC, D=3, 3x3 blocks, chi = chi_exp = 12 (truncating), warm read-out, one fit sweep per
    fit, six sweeps (the messages converge to a residual of ~1e-14, while a read-out fit started
    cold stays unconverged: warm and cold read-outs differ by 1.0e-7 here): interior frames'
    environment columns start from the sweep's fits; frames at the lattice edge and cross-block
    pairs (merged regions) start cold.  With one fit sweep per fit the fits never converge, so
    the roundoff of the two sides' QRs at the truncation stays in their results; the bound is
    1e-8, ten times below the warm/cold difference it has to resolve."""
    T = I.uniform_noise_peps(6, 6, 2, 3, seed=5)
    terms = [[(7, SZ)], [(14, SX)], [(7, SZ), (8, SZ)], [(2, SX), (3, SX)], [(14, SZ), (20, SZ)], [(21, SZ)]]
    g, o, gr, orr, gv, ov = run_both(T, 6, 6, 2, 3, 3, 3, 12, terms, n_sweeps=6, warm_start=2, fit_max_sweeps=1,
                                     chi_exp=12)
    assert close(gr, orr, 1e-9)
    assert np.max(np.abs(gv - ov)) < 1e-8, (np.max(np.abs(gv - ov)), 1 - message_fidelity(g, o))


def test_bonds_above_the_numerical_rank():
    """chi = 64 > the rank that the column MPS can carry next to an open edge: the fits
    meet QR columns beyond the numerical rank (tiny norms) and must still match the
    oracle (FP64, 1e-10)."""
    T = I.uniform_noise_peps(6, 6, 2, 3, seed=11)
    terms = I.standard_terms(6, 6)
    g, o, gres, ores, gv, ov = run_both(T, 6, 6, 2, 3, 3, 3, 64, terms, 3, fit_tol=0.0, fit_max_sweeps=2, seed=7)
    assert np.allclose(gres, ores, rtol=1e-8, atol=1e-14)
    assert np.max(np.abs(gv - ov)) < 1e-10


def test_rdm_parity_and_exact_on_trees():
    """bbp_rdm: 1- and 2-site reduced density matrices (inside a block, across a block
    edge) equal the oracle's on the loop block graph of C1 and the exact partial trace on
    a tree of strip blocks; Tr(rho O) = <O>; the trace distance of the C1 RDMs to the
    exact ones (the blockBP error on a loop) is stated, not pinned."""
    import _exact as Xe
    from oracle import blockbp as ob
    cfg = I.config(1)
    sites = ([5], [5, 6], [6, 10], [1, 2])
    g, o, gr, orr, gv, ov = run_both(cfg["tensors"], 4, 4, 2, 2, 2, 2, 16, [], n_sweeps=6)
    psi = Xe.state_vector(cfg["tensors"], 4, 4)
    for s in sites:
        rg = g.rdm(s)
        assert close(rg, o.rdm(s))
        assert abs(np.trace(rg) - 1) < 1e-12 and np.max(np.abs(rg - rg.conj().T)) < 1e-12
        assert ob.trace_distance(rg, Xe.exact_rdm(psi, 16, 2, s)) < 1e-2
    rho = g.rdm([5, 6])
    assert abs(np.trace(rho @ np.kron(SZ, SX)) - g.expect([[(5, SZ), (6, SX)]])[0]) < 1e-12
    T = I.uniform_noise_peps(4, 4, 2, 2, seed=1)
    g, o, gr, orr, gv, ov = run_both(T, 4, 4, 2, 2, 4, 2, 16, [], n_sweeps=3, chi_exp=18)
    psi = Xe.state_vector(T, 4, 4)
    for s in sites:
        assert np.max(np.abs(g.rdm(s) - Xe.exact_rdm(psi, 16, 2, s))) < 1e-11
