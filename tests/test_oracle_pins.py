"""Pins of the FP64 oracle against facts fixed by the paper and by the mathematics.

Each test would fail under a plausible mistake in the oracle: a wrong merge order
or misplaced conjugate in the double layer, a transposed MPO leg, a wrong frame
rotation, a dropped environment term, a wrong QR sign, a broken stop rule.
References are independent: brute-force state vectors, textbook site BP, dense
MPO x MPS products, closed-form product-state values.
"""
import math
import os

import numpy as np
import pytest

import _exact as X
from oracle import blockbp as ob
from paper_2301_05844_gb300 import inputs as I

SZ, SX, SY = I.SIGMA_Z, I.SIGMA_X, I.SIGMA_Y


def exact_values(T, Lx, Ly, terms):
    psi = X.state_vector(T, Lx, Ly)
    return np.array([X.exact_expect(psi, Lx * Ly, T[0].shape[0], t) for t in terms])


# -------------------------------------------------------------------------------------
def test_splitmix64_published_outputs():
    """SplitMix64 outputs from state 0 (Steele et al. 2014), stored in tests/golden."""
    path = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.txt")
    want = [int(l, 16) for l in open(path) if l.strip() and not l.startswith("#")]
    g = 0x9E3779B97F4A7C15
    got = ob.splitmix64(np.array([(k * g) % 2**64 for k in range(len(want))], dtype=np.uint64))
    assert [int(v) for v in got] == want
    u = ob.uniform_pm1(7, 3, 1000)
    assert u.min() >= -1.0 and u.max() < 1.0 and abs(u.mean()) < 0.1


def test_double_layer_contracts_to_norm_and_expectation():
    """The closed double-layer network equals <psi|psi>, and with O inserted <psi|O|psi>
    (Fig. 1(a,b)); complex tensors catch a misplaced conjugate or ket/bra swap."""
    rng = np.random.default_rng(11)
    Lx, Ly, d, D = 2, 2, 2, 2
    T = []
    for r in range(Ly):
        for c in range(Lx):
            shp = I.site_shape(r, c, Lx, Ly, d, D)
            T.append(rng.standard_normal(shp) + 1j * rng.standard_normal(shp))
    psi = X.state_vector(T, Lx, Ly)
    O = np.array([[0.3, 1.0 - 0.5j], [0.2 + 0.7j, -1.1]])  # not Hermitian on purpose
    for opsite in (None, 0, 3):
        E = [ob.double_layer(T[i], O if i == opsite else None) for i in range(4)]
        val = _closed_2x2(E)
        if opsite is None:
            ref = np.vdot(psi, psi)
        else:
            ref = X.exact_expect(psi, 4, 2, [(opsite, O)]) * np.vdot(psi, psi)
        assert abs(val - ref) < 1e-12 * abs(np.vdot(psi, psi))


def _closed_2x2(E):
    """Exact contraction of a 2x2 OBC double-layer network E[u,l,d,r]."""
    e0, e1, e2, e3 = E
    # bonds: e0.r-e1.l (a), e0.d-e2.u (b), e1.d-e3.u (c), e2.r-e3.l (e)
    return np.einsum("xyba,zacw,bvue,cesq->", e0, e1, e2, e3, optimize=True)


def test_qr_lq_factors():
    """Q orthonormal, Q^dagger M upper triangular with a real non-negative diagonal."""
    rng = np.random.default_rng(5)
    for cplx in (False, True):
        M = rng.standard_normal((12, 5)) + (1j * rng.standard_normal((12, 5)) if cplx else 0)
        Q = ob.qr_q(M)
        R = np.conj(Q.T) @ M
        assert np.allclose(np.conj(Q.T) @ Q, np.eye(5), atol=1e-13)
        assert np.allclose(np.tril(R, -1), 0, atol=1e-12)
        assert np.all(np.abs(np.diag(R).imag) < 1e-12) and np.all(np.diag(R).real > 0)
        assert np.allclose(Q @ R, M, atol=1e-12)
        Lq = ob.lq_q(M.T.copy())
        L = M.T @ np.conj(Lq.T)
        assert np.allclose(Lq @ np.conj(Lq.T), np.eye(5), atol=1e-13)
        assert np.allclose(np.triu(L, 1), 0, atol=1e-12) and np.all(np.diag(L).real > 0)


def _random_mpo_mps(rng, n, p, q, w, x, cplx=False):
    def rnd(*s):
        a = rng.standard_normal(s)
        return a + 1j * rng.standard_normal(s) if cplx else a
    ws = [1] + [w] * (n - 1) + [1]
    xs = [1] + [x] * (n - 1) + [1]
    O = [rnd(ws[i], p, q, ws[i + 1]) for i in range(n)]
    Xs = [rnd(xs[i], p, xs[i + 1]) for i in range(n)]
    return O, Xs


@pytest.mark.parametrize("cplx", [False, True])
def test_fit_full_rank_is_exact(cplx):
    """At full bond the variational fit reproduces O|X> exactly (App. A, Eq. distance = 0)."""
    rng = np.random.default_rng(3)
    O, Xs = _random_mpo_mps(rng, 4, 2, 3, 2, 2, cplx)
    dt = np.complex128 if cplx else np.float64
    Y, hist = ob.fit_mpo_mps(O, Xs, ob.FitOpts(chi=100, tol=0.0, max_sweeps=2),
                             lambda i, s: ob.random_site(1, i, s, dt), dt)
    assert np.allclose(X.dense_mps(Y), X.dense_mpo_apply(O, Xs), atol=1e-10)


@pytest.mark.parametrize("cplx", [False, True])
def test_fit_loss_identity_and_monotone(cplx):
    """-||Yt||^2 = ||Y - O X||^2 - <X|O^dag O|X> (App. A) and the loss never rises
    once the environments are canonical (from the first right-to-left update on)."""
    rng = np.random.default_rng(4)
    O, Xs = _random_mpo_mps(rng, 5, 2, 2, 3, 3, cplx)
    dt = np.complex128 if cplx else np.float64
    Y, hist = ob.fit_mpo_mps(O, Xs, ob.FitOpts(chi=3, tol=0.0, max_sweeps=6),
                             lambda i, s: ob.random_site(9, i, s, dt), dt)
    ox = X.dense_mpo_apply(O, Xs)
    y = X.dense_mps(Y)
    final_loss = -np.vdot(Y[0], Y[0]).real
    assert abs(np.linalg.norm(y - ox) ** 2 - np.linalg.norm(ox) ** 2 - final_loss) < 1e-9 * np.linalg.norm(ox) ** 2
    flat = [l for h in hist for l in h]
    n = len(Xs)
    tail = flat[n - 1:]
    assert all(b <= a + 1e-10 * abs(a) for a, b in zip(tail, tail[1:]))
    assert final_loss <= tail[-1] + 1e-10 * abs(tail[-1])


def test_fit_stop_rule():
    """std/|mean| of the losses of one sweep below tol ends the fit (App. A)."""
    rng = np.random.default_rng(8)
    O, Xs = _random_mpo_mps(rng, 4, 2, 2, 2, 2)
    _, hist = ob.fit_mpo_mps(O, Xs, ob.FitOpts(chi=100, tol=1e-6, max_sweeps=10),
                             lambda i, s: ob.random_site(2, i, s, np.float64), np.float64)
    last = np.array(hist[-1])
    assert len(hist) < 10 and np.std(last) / abs(np.mean(last)) < 1e-6


# -------------------------------------------------------------------------------------
@pytest.mark.parametrize("cplx", [False, True])
def test_single_block_equals_brute_force(cplx):
    """One block covering the lattice: no messages, the read-out at full chi_exp is the
    exact contraction (Fig. 1(e) with a trivial environment)."""
    rng = np.random.default_rng(21)
    T = I.uniform_noise_peps(4, 4, 2, 2, seed=1)
    if cplx:
        T = [t + 0.3j * rng.standard_normal(t.shape) for t in T]
    terms = I.standard_terms(4, 4) + [[(5, SY), (6, SY)], [(0, SX), (9, SZ)], [(1, SX), (13, SX)]]
    lat = ob.Lattice(4, 4, 2, 2, 4, 4, T, chi=16, chi_exp=64, fit_tol=0.0, fit_max_sweeps=2)
    assert not lat.msgs
    got = lat.expect(terms)
    assert np.max(np.abs(got - exact_values(T, 4, 4, terms))) < 1e-12


@pytest.mark.parametrize("bx,by", [(4, 1), (4, 2), (1, 4), (2, 4)])
def test_tree_block_graph_is_exact(bx, by):
    """Strip blocks form a chain (a tree): the BP fixed point is the exact environment
    (Sec. "The blockBP algorithm"), so every <O> equals brute force at full chi."""
    T = I.uniform_noise_peps(4, 4, 2, 2, seed=1)
    terms = I.standard_terms(4, 4)
    lat = ob.Lattice(4, 4, 2, 2, bx, by, T, chi=16, chi_exp=18, fit_tol=0.0, fit_max_sweeps=2)
    nblk = lat.nbx * lat.nby
    res, sweeps, _ = lat.run(n_sweeps=nblk + 1)
    assert abs(res) < 1e-12
    got = lat.expect(terms)
    assert np.max(np.abs(got - exact_values(T, 4, 4, terms))) < 1e-12


def test_product_state_D1_exact_after_one_sweep():
    """D=1: <O>_s = t_s^dag O t_s / t_s^dag t_s after one sweep; residual 0 from sweep 2."""
    rng = np.random.default_rng(2)
    vecs = [rng.standard_normal(2) + 1j * rng.standard_normal(2) for _ in range(36)]
    T = I.product_peps(6, 6, 2, 1, vecs)
    lat = ob.Lattice(6, 6, 2, 1, 3, 2, T, chi=4, fit_tol=0.0, fit_max_sweeps=1)
    lat.sweep()
    assert abs(lat.sweep()) < 1e-14
    terms = [[(s, SZ)] for s in range(36)] + [[(s, SX)] for s in range(36)]
    got = lat.expect(terms)
    want = [np.vdot(v, O @ v) / np.vdot(v, v) for O in (SZ, SX) for v in vecs]
    assert np.max(np.abs(got - np.array(want))) < 1e-13


@pytest.mark.parametrize("D,chi", [(2, 1), (2, 4), (3, 5)])
@pytest.mark.parametrize("h_limit", ["plus", "up"])
def test_tfim_limits_with_gauges(D, chi, h_limit):
    """Transverse-Ising limits: |+>^N (field -> infinity) and |up>^N (field 0), embedded
    at bond D and dressed with random bond gauges, are exact for any chi >= 1."""
    t = np.array([1.0, 1.0]) / math.sqrt(2) if h_limit == "plus" else np.array([1.0, 0.0])
    Lx = Ly = 4
    T = I.gauge_dress(I.product_peps(Lx, Ly, 2, D, [t] * 16), Lx, Ly, seed=D * 10 + chi)
    lat = ob.Lattice(Lx, Ly, 2, D, 2, 2, T, chi=chi, chi_exp=chi, fit_tol=0.0, fit_max_sweeps=2)
    lat.run(n_sweeps=3)
    terms = [[(5, SX)], [(5, SZ)], [(5, SZ), (6, SZ)], [(1, SZ), (2, SZ)], [(2, SX), (6, SX)]]
    want = [1, 0, 0, 0, 1] if h_limit == "plus" else [0, 1, 1, 1, 0]
    assert np.max(np.abs(lat.expect(terms) - np.array(want))) < 1e-10


def test_tfim_limit_infinite_gauged():
    """The same closed form on an infinite 2x2 unit cell with complex gauges."""
    t = np.array([1.0, 1.0]) / math.sqrt(2)
    T = I.gauge_dress(I.product_peps(2, 2, 2, 2, [t] * 4, boundary="infinite"), 2, 2, seed=3,
                      boundary="infinite", complex_gauge=True)
    lat = ob.Lattice(2, 2, 2, 2, 2, 2, T, boundary="infinite", chi=2, fit_tol=0.0, fit_max_sweeps=2)
    lat.run(n_sweeps=3)
    got = lat.expect([[(0, SX)], [(3, SZ)], [(0, SX), (1, SX)], [(1, SZ), (3, SZ)]])
    assert np.max(np.abs(got - np.array([1, 0, 1, 0]))) < 1e-10


@pytest.mark.parametrize("cplx", [False, True])
def test_block_size_one_equals_textbook_bp(cplx):
    """Blocks of one site reduce blockBP to plain BP (Sec. "The blockBP algorithm")."""
    T = I.uniform_noise_peps(4, 3, 2, 2, seed=1)
    if cplx:
        rng = np.random.default_rng(1)
        T = [t + 0.2j * rng.standard_normal(t.shape) for t in T]
    terms = I.standard_terms(4, 3)
    lat = ob.Lattice(4, 3, 2, 2, 1, 1, T, chi=4, fit_tol=0.0, fit_max_sweeps=1)
    lat.run(n_sweeps=60)
    got = lat.expect(terms)
    ref = X.textbook_bp(T, 4, 3, terms)
    assert np.max(np.abs(got - ref)) < 1e-12


def test_messages_unit_norm_hermitian_and_converge():
    """||m|| = 1, m(k,k') = conj m(k',k) as an operator (full rank, Hermitian init),
    residual -> 0 at the fixed point; Im<O> ~ 0 for Hermitian O."""
    rng = np.random.default_rng(6)
    T = I.uniform_noise_peps(4, 4, 2, 2, seed=1)
    T = [t + 0.3j * rng.standard_normal(t.shape) for t in T]
    lat = ob.Lattice(4, 4, 2, 2, 2, 2, T, chi=16, fit_tol=1e-12, fit_max_sweeps=6)
    res, sweeps, ok = lat.run(tol=1e-13, max_sweeps=15)
    assert ok and res < 1e-13
    for m in lat.msgs.values():
        assert abs(ob.mps_overlap(m, m) - 1) < 1e-13
        herm = [s.reshape(s.shape[0], 2, 2, s.shape[2]).transpose(0, 2, 1, 3).reshape(s.shape).conj() for s in m]
        assert abs(abs(ob.mps_overlap(m, herm)) - 1) < 1e-11
        assert abs(ob.identity_trace(m, 2).imag) < 1e-12 and ob.identity_trace(m, 2).real > 0
    vals = lat.expect(I.standard_terms(4, 4))
    assert np.max(np.abs(vals.imag)) < 1e-12


def test_gauge_invariance_full_rank():
    """Random invertible gauges on every bond leave <O> unchanged at full chi."""
    T = I.uniform_noise_peps(4, 4, 2, 2, seed=1)
    Tg = I.gauge_dress(T, 4, 4, seed=17)
    terms = I.standard_terms(4, 4)
    vals = []
    for TT in (T, Tg):
        lat = ob.Lattice(4, 4, 2, 2, 2, 2, TT, chi=16, fit_tol=1e-12, fit_max_sweeps=6)
        lat.run(n_sweeps=12)
        vals.append(lat.expect(terms))
    assert np.max(np.abs(vals[0] - vals[1])) < 1e-10


def test_relative_stop_rule_and_init_modes():
    """Relative criterion r_l / r_1 < tol (App. A) stops earlier than absolute 1e-16;
    random-MPDO init (App. A) reaches the same fixed point as the identity init."""
    T = I.uniform_noise_peps(4, 4, 2, 2, seed=1)
    terms = I.standard_terms(4, 4)
    a = ob.Lattice(4, 4, 2, 2, 2, 2, T, chi=16, fit_tol=1e-12, fit_max_sweeps=6)
    r, k, ok = a.run(tol=1e-5, max_sweeps=20, relative=True)
    assert ok and a.residuals[-1] / a.residuals[0] < 1e-5 and k < 10
    b = ob.Lattice(4, 4, 2, 2, 2, 2, T, chi=16, fit_tol=1e-12, fit_max_sweeps=6, init_mode=1, seed=5)
    b.run(n_sweeps=12)
    a.run(n_sweeps=12)
    assert np.max(np.abs(a.expect(terms) - b.expect(terms))) < 1e-10


def test_normalise_message_norm_and_phase():
    """Unit 2-norm and <I|m> real positive after normalisation, for an arbitrary
    complex MPS whose identity trace has a generic phase."""
    rng = np.random.default_rng(12)
    M = [rng.standard_normal(s) + 1j * rng.standard_normal(s) for s in [(1, 9, 3), (3, 9, 3), (3, 9, 1)]]
    N = ob.normalise_message(M, 3)
    assert abs(ob.mps_overlap(N, N) - 1) < 1e-13
    tau = ob.identity_trace(N, 3)
    assert abs(tau.imag) < 1e-13 * abs(tau) and tau.real > 0
    # same state up to the phase
    assert abs(abs(ob.mps_overlap(N, M)) ** 2 - ob.mps_overlap(M, M).real) < 1e-10 * ob.mps_overlap(M, M).real


def test_residual_is_mean_squared_message_distance():
    """r_l = mean over messages of ||m^l - m^{l-1}||^2 of the normalised messages
    (the mean-square reading of the stop rule), checked with dense vectors."""
    T = I.uniform_noise_peps(4, 4, 2, 2, seed=1)
    lat = ob.Lattice(4, 4, 2, 2, 2, 2, T, chi=16, fit_tol=0.0, fit_max_sweeps=2)
    lat.sweep()
    old = {k: X.dense_mps(v) for k, v in lat.msgs.items()}
    r = lat.sweep()
    new = {k: X.dense_mps(v) for k, v in lat.msgs.items()}
    want = np.mean([np.linalg.norm(new[k] - old[k]) ** 2 for k in old])
    assert abs(r - want) < 1e-13 and r > 1e-6


def test_warm_start_reaches_the_same_fixed_point():
    """Starting each fit from the previous sweep's fitted MPS (warm start) changes the
    path, not the fixed point: at full chi both runs agree on every <O>."""
    T = I.uniform_noise_peps(4, 4, 2, 2, seed=1)
    terms = I.standard_terms(4, 4)
    vals = []
    for warm in (False, True):
        lat = ob.Lattice(4, 4, 2, 2, 2, 2, T, chi=16, fit_tol=1e-12, fit_max_sweeps=6, warm_start=warm)
        lat.run(n_sweeps=12)
        vals.append(lat.expect(terms))
    assert np.max(np.abs(vals[0] - vals[1])) < 1e-10


def test_warm_readout_environments_change_nothing_at_full_rank():
    """warm_start = 2 also starts the read-out's environment columns of one-block regions
    from the sweep's last fits (chi_exp = chi).  Where those fits are exact (full rank) the
    starting point cannot move <O>: warm_start 2 agrees with 0 on every observable, one-block
    and two-block (cross-edge pair) regions alike."""
    T = I.uniform_noise_peps(4, 4, 2, 2, seed=5)
    terms = I.standard_terms(4, 4)
    vals = []
    for warm in (0, 2):
        lat = ob.Lattice(4, 4, 2, 2, 2, 2, T, chi=16, chi_exp=16, fit_tol=1e-12, fit_max_sweeps=6, warm_start=warm)
        lat.run(n_sweeps=6)
        vals.append(lat.expect(terms))
    assert np.max(np.abs(vals[0] - vals[1])) < 1e-10


def _onsager(beta):
    """Spontaneous magnetisation of the 2D square-lattice Ising model (Onsager, Yang):
    (1 - sinh(2 beta)^-4)^(1/8) below the critical temperature, 0 above it."""
    s = math.sinh(2 * beta)
    return (1 - s ** -4) ** 0.125 if s > 1 else 0.0


def _ising_m(beta, b, h, chi=16):
    T = I.ising_peps(beta, h=h)
    o = ob.Lattice(1, 1, 2, 2, b, b, [T], boundary="infinite", chi=chi, fit_tol=1e-10, fit_max_sweeps=20, seed=3,
                   init_mode=1)
    r, k, conv = o.run(tol=1e-12, max_sweeps=80)
    assert conv
    c = (b // 2) * b + b // 2 - 1  # a site next to the block centre
    return o.expect([[(c, I.SIGMA_Z)]])[0].real


def test_infinite_ising_magnetisation_against_onsager():
    """The infinite path on the PEPS whose norm is the classical Ising partition function
    (Sec. "The blockBP algorithm": one block messaging itself): deep in the ordered phase
    <sz> approaches Onsager's magnetisation, about tenfold closer per block-size step
    (measured 5.8e-4, 6.0e-5, 7.5e-6 for blocks 2, 4, 6 at beta = 0.6); in the disordered
    phase without a field <sz> vanishes.  The model is isotropic, so this does not tell
    the four directions apart (the gauge-dressed infinite cell pins that); it pins the
    feedback of the block's own messages on the infinite path, the fits and the read-out
    against the exact thermodynamics (a planted mistake that stops feeding the messages
    back fails it)."""
    beta = 0.6
    err = [abs(_ising_m(beta, b, 1e-6) - _onsager(beta)) for b in (2, 4, 6)]
    assert err[0] < 1e-3 and err[1] < 1.5e-4 and err[2] < 2e-5, err
    assert err[0] > err[1] > err[2]
    assert abs(_ising_m(0.7, 4, 1e-6) - _onsager(0.7)) < 1e-5
    assert abs(_ising_m(0.3, 4, 0.0)) < 1e-5


# ---- single-layer networks (K-leg site tensors used as they are, no double layer) ----

def _sl_terms(E, rng):
    imp = {s: rng.uniform(-1.0, 1.0, np.shape(E[s])) for s in (0, 1, 2, 5, 6, 10)}
    return [[(5, imp[5])], [(0, imp[0])], [(5, imp[5]), (6, imp[6])], [(6, imp[6]), (10, imp[10])],
            [(1, imp[1]), (2, imp[2])]]


def test_single_layer_single_block_and_tree_strips_exact():
    """A single-layer network (Sec. on the 2D Ising model: blockBP on a network given by its
    own K-leg tensors) read out with impurity tensors: one block covering the lattice, and
    strip blocks whose block graph is a chain (a tree, where the BP fixed point is exact,
    Sec. "The blockBP algorithm"), both equal the exact contraction ratio Z_imp / Z."""
    rng = np.random.default_rng(7)
    E = I.positive_network(4, 4, 2, seed=11)
    terms = _sl_terms(E, rng)
    Z = X.network_value(E, 4, 4)
    exact = np.array([X.network_value(E, 4, 4, dict(t)) / Z for t in terms])
    o = ob.Lattice(4, 4, 1, 2, 4, 4, E, chi=16, single_layer=True)
    assert np.max(np.abs(o.expect(terms).real - exact)) < 1e-12
    for bx, by in ((4, 1), (4, 2), (1, 4), (2, 4)):
        o = ob.Lattice(4, 4, 1, 2, bx, by, E, chi=16, single_layer=True, init_mode=1, seed=5)
        r, k, conv = o.run(tol=1e-14, max_sweeps=40)
        assert conv
        assert np.max(np.abs(o.expect(terms).real - exact)) < 1e-12, (bx, by)


def test_single_layer_equals_double_layer_path():
    """Feeding the double layers E = T (x) T* of a PEPS as a single-layer network (bond
    K = D^2, impurities E^O) reaches the same fixed point as the double-layer path: the
    two differ only in the initial messages and the phase reference of the normalisation."""
    T = I.uniform_noise_peps(4, 4, 2, 2, seed=1)
    od = ob.Lattice(4, 4, 2, 2, 2, 2, T, chi=16)
    od.run(tol=1e-14, max_sweeps=80)
    osl = ob.Lattice(4, 4, 1, 4, 2, 2, [ob.double_layer(t) for t in T], chi=16, single_layer=True)
    osl.run(tol=1e-14, max_sweeps=80)
    dterms = [[(5, I.SIGMA_Z)], [(0, I.SIGMA_X)], [(5, I.SIGMA_Z), (6, I.SIGMA_Z)], [(6, I.SIGMA_Z), (10, I.SIGMA_Z)]]
    sterms = [[(s, ob.double_layer(T[s], op)) for s, op in t] for t in dterms]
    assert np.max(np.abs(od.expect(dterms) - osl.expect(sterms))) < 1e-9


def _ising_network_m(beta, b, h, chi=16):
    E, Ez = I.ising_network(beta, h)
    o = ob.Lattice(1, 1, 1, 2, b, b, [E], boundary="infinite", chi=chi, fit_tol=1e-10, fit_max_sweeps=20, seed=3,
                   init_mode=1, single_layer=True)
    r, k, conv = o.run(tol=1e-12, max_sweeps=80)
    assert conv
    c = (b // 2) * b + b // 2 - 1  # a site next to the block centre
    return o.expect([[(c, Ez)]])[0].real


def test_single_layer_ising_against_onsager():
    """The classical 2D Ising model as its own single-layer network (bond 2, Sec. on the 2D
    Ising model), on the infinite path with uniform random initial messages: |<s>| approaches
    Onsager's magnetisation about tenfold per block-size step (measured 5.8e-4, 6.0e-5,
    7.4e-6 for blocks 2, 4, 6 at beta = 0.6; the random start may settle in either ordered
    state, so the magnitude is compared) and vanishes in the disordered phase."""
    beta = 0.6
    err = [abs(abs(_ising_network_m(beta, b, 1e-6)) - _onsager(beta)) for b in (2, 4, 6)]
    assert err[0] < 1e-3 and err[1] < 1.5e-4 and err[2] < 2e-5, err
    assert err[0] > err[1] > err[2]
    assert abs(abs(_ising_network_m(0.7, 4, 1e-6)) - _onsager(0.7)) < 1e-5
    assert abs(_ising_network_m(0.3, 4, 0.0)) < 1e-5


def test_single_layer_message_normalisation():
    """A single-layer message is normalised to unit 2-norm with <1|m> (all-ones vector on
    every site) real positive, and its initial messages are the all-ones product (mode 0)
    or positive uniform entries (mode 1)."""
    rng = np.random.default_rng(3)
    M = [rng.standard_normal((1, 3, 2)), rng.standard_normal((2, 3, 2)), rng.standard_normal((2, 3, 1))]
    N = ob.normalise_message(M, 0, single=True)
    assert abs(ob.mps_overlap(N, N) - 1.0) < 1e-13
    t = ob.ones_trace(N)
    assert t > 0 and abs(t * ob.mps_overlap(M, M) ** 0.5 - abs(ob.ones_trace(M))) < 1e-12
    for s in ob.ones_message(3, 4, np.float64):
        assert s.shape == (1, 4, 1) and np.all(s == 1.0)
    U = ob.uniform_message(3, 4, 9, ob.stream_id(2, 0, 5, 0, 0), np.float64)
    assert all(np.all((s >= 0.0) & (s < 1.0)) for s in U) and len({s.tobytes() for s in U}) == 3


# ---- reduced density matrices and their trace distance ----

def test_rdm_equals_partial_trace_and_trace_distance():
    """The read-out's RDMs (entries read as expectations of matrix units) on one block
    covering the lattice equal the state's partial trace; they are Hermitian with unit
    trace and give Tr(rho O) = <O>.  The trace distance is 1 for orthogonal pure states,
    0 for equal ones, and |p - q| for diagonal qubit states."""
    T = I.uniform_noise_peps(4, 4, 2, 2, seed=1)
    o = ob.Lattice(4, 4, 2, 2, 4, 4, T, chi=16, chi_exp=64)
    psi = X.state_vector(T, 4, 4)
    for sites in ([5], [5, 6], [6, 10], [0, 4]):
        rho = o.rdm(sites)
        assert np.max(np.abs(rho - X.exact_rdm(psi, 16, 2, sites))) < 1e-12
        assert abs(np.trace(rho) - 1) < 1e-12 and np.max(np.abs(rho - rho.conj().T)) < 1e-12
    rho = o.rdm([5, 6])
    O = np.kron(I.SIGMA_Z, I.SIGMA_X)
    assert abs(np.trace(rho @ O) - o.expect([[(5, I.SIGMA_Z), (6, I.SIGMA_X)]])[0]) < 1e-12
    up, down = np.diag([1.0, 0.0]), np.diag([0.0, 1.0])
    assert abs(ob.trace_distance(up, down) - 1.0) < 1e-15 and ob.trace_distance(up, up) == 0.0
    assert abs(ob.trace_distance(np.diag([0.7, 0.3]), np.diag([0.2, 0.8])) - 0.5) < 1e-15


def test_single_layer_gauge_invariance_full_rank():
    """Random invertible gauges G, G^-1 on every bond of a single-layer network (a loop of
    2x2 blocks) leave the network, and the blockBP read-out at full chi, unchanged.  The
    impurity tensors are dressed with the same gauges as the tensors they replace."""
    E = I.positive_network(4, 4, 2, seed=11)
    rng = np.random.default_rng(5)
    imp = {s: rng.uniform(-1.0, 1.0, np.shape(E[s])) for s in (0, 5, 6)}

    def dress(tensors):
        return [t[0] for t in I.gauge_dress([np.asarray(t)[None] for t in tensors], 4, 4, seed=17)]

    Eg = dress(E)
    assert abs(X.network_value(Eg, 4, 4) / X.network_value(E, 4, 4) - 1.0) < 1e-12
    sets = ([5], [0], [5, 6])
    terms, gterms = [], []
    for sites in sets:
        Es = list(E)
        for s in sites:
            Es[s] = imp[s]
        Ed = dress(Es)
        terms.append([(s, imp[s]) for s in sites])
        gterms.append([(s, Ed[s]) for s in sites])
    vals = []
    for tensors, tt in ((E, terms), (Eg, gterms)):
        lat = ob.Lattice(4, 4, 1, 2, 2, 2, tensors, chi=16, fit_tol=1e-12, fit_max_sweeps=6, single_layer=True)
        lat.run(n_sweeps=12)
        vals.append(lat.expect(tt))
    assert np.max(np.abs(vals[0] - vals[1])) < 1e-10


# ---- shifted partitions of an infinite lattice ----

@pytest.mark.parametrize("Lx,Ly,bx,by,shift", [(2, 2, 4, 4, (1, 0)), (2, 2, 4, 4, (0, 1)), (2, 2, 4, 4, (1, 1)),
                                              (3, 1, 3, 3, (1, 0)), (3, 1, 3, 3, (2, 0))])
def test_shifted_partition_maps_block_sites_to_the_shifted_cell(Lx, Ly, bx, by, shift):
    """A partition shifted by (sx, sy) puts lattice site (r + sy, c + sx) at block site (r, c).
    Pinned on a product state with a different state on every site of the cell, dressed with
    complex gauges (exact for any partition): <sz>, <sx> and <sz sz> at every block site equal
    the closed-form values of the shifted cell sites (the 3-site cell tells +1 from -1)."""
    n = Lx * Ly
    vecs = [np.array([math.cos(0.45 * i), math.sin(0.45 * i)]) for i in range(n)]
    T = I.gauge_dress(I.product_peps(Lx, Ly, 2, 2, vecs, boundary="infinite"), Lx, Ly, seed=3, boundary="infinite",
                      complex_gauge=True)
    sx, sy = shift
    lat = ob.Lattice(Lx, Ly, 2, 2, bx, by, T, boundary="infinite", chi=2, fit_tol=0.0, fit_max_sweeps=2,
                     shift=shift)
    lat.run(n_sweeps=3)

    def cell(r, c):
        return vecs[((r + sy) % Ly) * Lx + (c + sx) % Lx]

    def ev(v, O):
        return float(v @ O @ v) / float(v @ v)

    terms, want = [], []
    for r in range(by):
        for c in range(bx):
            s = r * bx + c
            terms += [[(s, SZ)], [(s, SX)]]
            want += [ev(cell(r, c), SZ), ev(cell(r, c), SX)]
            if c + 1 < bx:
                terms.append([(s, SZ), (s + 1, SZ)])
                want.append(ev(cell(r, c), SZ) * ev(cell(r, c + 1), SZ))
    assert np.max(np.abs(lat.expect(terms) - np.array(want))) < 1e-10


def test_shifted_partition_equals_the_rolled_cell():
    """Shifting the partition by (1, 1) is the same computation as rolling the unit cell by one
    site in each direction (bit-identical); shifts are taken within the unit cell."""
    T = I.complex_normal_cell(2, 2, 2, 2, seed=3)
    T = [t.astype(np.complex128) for t in T]
    terms = [[(0, SZ)], [(5, SX)], [(5, SZ), (6, SZ)], [(6, SX), (10, SX)]]
    kw = dict(boundary="infinite", chi=4, fit_tol=0.0, fit_max_sweeps=2, seed=5)
    a = ob.Lattice(2, 2, 2, 2, 4, 4, T, shift=(1, 1), **kw)
    rolled = [T[((r + 1) % 2) * 2 + (c + 1) % 2] for r in range(2) for c in range(2)]
    b = ob.Lattice(2, 2, 2, 2, 4, 4, rolled, **kw)
    d = ob.Lattice(2, 2, 2, 2, 4, 4, T, **kw)
    for lat in (a, b, d):
        lat.run(n_sweeps=3)
    assert np.array_equal(a.expect(terms), b.expect(terms))
    assert np.max(np.abs(a.expect(terms) - d.expect(terms))) > 1e-6  # the shift does change the partition
    with pytest.raises(AssertionError):
        ob.Lattice(2, 2, 2, 2, 4, 4, T, shift=(2, 0), **kw)


@pytest.mark.parametrize("bx,by,shift", [(4, 2, (0, 1)), (2, 4, (1, 0)), (4, 4, (0, 2)), (4, 4, (3, 0))])
def test_shifted_obc_strips_exact(bx, by, shift):
    """OBC partitions shifted by (sx, sy) move the block boundaries to sx, sx + bx, ... (and
    sy, sy + by, ...), leaving narrower blocks on the lattice edges.  Shifted strips are a
    chain of blocks (a tree, where the BP fixed point is exact), so every observable, also
    across the moved boundaries, equals brute force at full bond dimension."""
    T = I.uniform_noise_peps(4, 4, 2, 2, seed=1)
    terms = I.standard_terms(4, 4)
    lat = ob.Lattice(4, 4, 2, 2, bx, by, T, chi=16, chi_exp=18, fit_tol=0.0, fit_max_sweeps=2, shift=shift)
    assert lat.nbx * lat.nby == 3 or lat.nbx * lat.nby == 2
    lat.run(n_sweeps=4)
    psi = X.state_vector(T, 4, 4)
    exact = np.array([X.exact_expect(psi, 16, 2, t) for t in terms])
    assert np.max(np.abs(lat.expect(terms) - exact)) < 1e-11


def test_shifted_obc_partition_geometry_and_loops():
    """A 2x2-block partition of a 4x4 lattice shifted by (1, 1) has a 3 x 3 grid of blocks of
    sizes 1, 2, 1 per side; its messages converge and its observables stay within the blockBP
    error of brute force (a loop of blocks: stated, not exact)."""
    T = I.uniform_noise_peps(4, 4, 2, 2, seed=1)
    lat = ob.Lattice(4, 4, 2, 2, 2, 2, T, chi=16, fit_tol=1e-12, fit_max_sweeps=6, shift=(1, 1))
    assert (lat.xs, lat.ys) == ([0, 1, 3, 4], [0, 1, 3, 4])
    assert [lat.block_size(b) for b in range(9)] == [(1, 1), (1, 2), (1, 1), (2, 1), (2, 2), (2, 1), (1, 1),
                                                     (1, 2), (1, 1)]
    r, k, conv = lat.run(tol=1e-12, max_sweeps=60)
    assert conv
    terms = I.standard_terms(4, 4)
    psi = X.state_vector(T, 4, 4)
    exact = np.array([X.exact_expect(psi, 16, 2, t) for t in terms])
    assert np.max(np.abs(lat.expect(terms) - exact)) < 1e-2


# -------------------------------------------------------------------------------------
# The Hermitian-basis option: the same method after a fixed unitary change of basis on
# every merged leg (the basis of the library's real-arithmetic paths for complex tensors).
def _complex_peps(Lx, Ly, D, seed):
    re = I.uniform_noise_peps(Lx, Ly, 2, D, seed=seed)
    im = I.uniform_noise_peps(Lx, Ly, 2, D, seed=seed + 100)
    return [a + 0.4j * (b - 0.5) for a, b in zip(re, im)]


def test_hermitian_basis_matrix_and_real_double_layer():
    """V is unitary and V^T conj(V) = I (every bond keeps its value); the double layer of
    a complex tensor is real in the basis, and so is E^O for a Hermitian O but not for a
    non-Hermitian one; transforming the merged legs one by one equals the dense map."""
    for D in (1, 2, 3, 4):
        V = ob.hermitian_basis_matrix(D)
        assert np.allclose(V @ np.conj(V.T), np.eye(D * D), atol=1e-15)
        assert np.allclose(V.T @ np.conj(V), np.eye(D * D), atol=1e-15)
        # Hermitian (ket, bra) matrices map to real vectors, anti-Hermitian ones to i * real
        rng = np.random.default_rng(D)
        G = rng.standard_normal((D, D)) + 1j * rng.standard_normal((D, D))
        h = (G + np.conj(G.T)).reshape(-1)
        assert np.max(np.abs((V @ h).imag)) < 1e-14
        assert np.max(np.abs((V @ (G - np.conj(G.T)).reshape(-1)).real)) < 1e-14
    T = _complex_peps(3, 3, 2, seed=41)[4]  # interior site: every leg D = 2
    E = ob.double_layer(T)
    Eh = ob.to_hermitian_basis_E(E, T.shape[1:])
    assert np.max(np.abs(Eh.imag)) < 1e-13 * np.max(np.abs(Eh))
    V = ob.hermitian_basis_matrix(2)
    dense = np.einsum("Uu,Ll,Dd,Rr,uldr->ULDR", V, V, np.conj(V), np.conj(V), E, optimize=True)
    assert np.max(np.abs(Eh - dense)) < 1e-13
    Eo = ob.to_hermitian_basis_E(ob.double_layer(T, SY), T.shape[1:])
    assert np.max(np.abs(Eo.imag)) < 1e-13 * np.max(np.abs(Eo))
    Ep = ob.to_hermitian_basis_E(ob.double_layer(T, (SX + 1j * SY) / 2), T.shape[1:])
    assert np.max(np.abs(Ep.imag)) > 1e-3 * np.max(np.abs(Ep))


def test_hermitian_basis_single_block_and_trees_exact():
    """In the Hermitian basis a block covering the lattice, and strip blocks (a tree), still
    give the exact <O> of a complex PEPS, non-Hermitian operators included."""
    T = _complex_peps(4, 4, 2, seed=23)
    SP = (SX + 1j * SY) / 2
    terms = [[(s, SZ)] for s in range(16)] + [[(5, SY)], [(9, SP)], [(10, SY), (11, SY)], [(5, SP), (9, SZ)]]
    ex = exact_values(T, 4, 4, terms)
    one = ob.Lattice(4, 4, 2, 2, 4, 4, T, chi=16, chi_exp=64, fit_tol=0.0, fit_max_sweeps=2, hermitian_basis=True)
    assert np.max(np.abs(one.expect(terms) - ex)) < 1e-12
    for bx, by in ((4, 1), (2, 4)):
        lat = ob.Lattice(4, 4, 2, 2, bx, by, T, chi=16, chi_exp=18, fit_tol=0.0, fit_max_sweeps=2,
                         hermitian_basis=True)
        assert all(m[0].dtype == np.float64 for m in lat.msgs.values())
        lat.run(n_sweeps=lat.nbx * lat.nby + 1)
        assert np.max(np.abs(lat.expect(terms) - ex)) < 1e-11


@pytest.mark.parametrize("init_mode", [0, 1])
def test_hermitian_basis_equals_complex_at_full_rank(init_mode):
    """At full message rank the fixed point does not depend on how the fits start, so the
    real-arithmetic run agrees with the complex one: residuals, <O>, and every message
    equals the complex message mapped by V (conj(V) for messages sent right or down)."""
    T = _complex_peps(4, 4, 2, seed=21)
    terms = I.standard_terms(4, 4) + [[(5, SY), (6, SY)], [(9, (SX + 1j * SY) / 2)]]
    a = ob.Lattice(4, 4, 2, 2, 2, 2, T, chi=16, fit_tol=0.0, fit_max_sweeps=3, seed=7, init_mode=init_mode)
    b = ob.Lattice(4, 4, 2, 2, 2, 2, T, chi=16, fit_tol=0.0, fit_max_sweeps=3, seed=7, init_mode=init_mode,
                   hermitian_basis=True)
    ra = [a.sweep() for _ in range(6)]
    rb = [b.sweep() for _ in range(6)]
    assert np.allclose(ra, rb, rtol=1e-6, atol=1e-14)
    assert np.max(np.abs(a.expect(terms) - b.expect(terms))) < 1e-12
    for (bi, dr), m in a.msgs.items():
        mh = ob.to_hermitian_basis_mps(m, 2, conj_basis=dr in (ob.RIGHT, ob.DOWN))
        assert abs(abs(ob.mps_overlap(b.msgs[(bi, dr)], mh)) - 1.0) < 1e-12


def test_fit_sweep_counts():
    """fit_sweeps[l] sums, over the column fits of sweep l, the fit sweeps each ran: every fit
    runs fit_max_sweeps when the tolerance is 0, one when any tolerance is met at once, and
    with the paper's 1e-6 a number in between for each fit (App. A stop rule)."""
    T = I.uniform_noise_peps(6, 6, 2, 2, seed=3)
    nfits = 8 * 3  # 8 messages (2x2 blocks of 3x3 sites, 4 interior edges) x 3 frame columns
    for tol, mx, want in ((0.0, 3, nfits * 3), (10.0, 5, nfits)):
        lat = ob.Lattice(6, 6, 2, 2, 3, 3, T, chi=4, fit_tol=tol, fit_max_sweeps=mx, seed=2)
        lat.run(n_sweeps=2)
        assert lat.fit_sweeps == [want, want]
    lat = ob.Lattice(6, 6, 2, 2, 3, 3, T, chi=4, fit_tol=1e-6, fit_max_sweeps=10, seed=2)
    lat.run(n_sweeps=2)
    assert all(nfits < f < 10 * nfits for f in lat.fit_sweeps), lat.fit_sweeps
