"""Complex tensors in the Hermitian basis (real arithmetic on the FP64 and tensor-core
paths) against the complex FP64 oracle, and against closed forms.

At full message rank the blockBP fixed point does not depend on how the fits start,
so the real-arithmetic run and the oracle's complex run agree to rounding; with active
truncation both run their fits to convergence and agree to the fit tolerance."""
import numpy as np
import pytest

import _exact as X
from _gpu import message_fidelity_hb, run_both
from paper_2301_05844_gb300 import binding as B
from paper_2301_05844_gb300 import inputs as I

pytestmark = pytest.mark.gpu
SX, SY, SZ = I.SIGMA_X, I.SIGMA_Y, I.SIGMA_Z
SPLUS = (SX + 1j * SY) / 2  # not Hermitian: exercises the O = H + iA split of the read-out


def complex_obc(Lx, Ly, D, seed):
    re = I.uniform_noise_peps(Lx, Ly, 2, D, seed=seed)
    im = I.uniform_noise_peps(Lx, Ly, 2, D, seed=seed + 100)
    return [a + 0.4j * (b - 0.5) for a, b in zip(re, im)]


def terms_4x4():
    return [[(s, SZ)] for s in range(16)] + [[(5, SX)], [(6, SY)], [(9, SPLUS)], [(10, SY), (11, SY)],
                                             [(5, SPLUS), (9, SZ)], [(1, SX), (2, SY)]]


def test_full_rank_complex_obc_fp64_hermitian_basis():
    """4x4 OBC, D=2, 2x2 blocks, chi=16 (full rank: no truncation): Hermitian-basis FP64
    equals the complex oracle to 1e-10 on every <O> (incl. sigma_y and sigma_+), the
    residuals agree, and every message equals the oracle's in the rotated basis."""
    T = complex_obc(4, 4, 2, seed=21)
    terms = terms_4x4()
    g, o, gr, orr, gv, ov = run_both(T, 4, 4, 2, 2, 2, 2, 16, terms, 6, fit_tol=0.0, fit_max_sweeps=3,
                                     hermitian_basis=1)
    assert not g.complex_messages()
    assert np.max(np.abs(gv - ov)) < 1e-10, np.max(np.abs(gv - ov))
    assert np.allclose(gr, orr, rtol=1e-6, atol=1e-13)
    assert message_fidelity_hb(g, o, 2) > 1 - 1e-10


def test_brute_force_single_block_hermitian_basis():
    """One block covering a complex 4x4 lattice (no messages): the read-out in the
    Hermitian basis equals the exact state-vector expectation values to 1e-12."""
    T = complex_obc(4, 4, 2, seed=23)
    terms = terms_4x4()
    g = B.Lattice(Lx=4, Ly=4, d=2, D=2, bx=4, by=4, chi=16, dtype=B.C128, hermitian_basis=1, chi_exp=64)
    g.set_tensors(T)
    v = g.expect(terms)
    psi = X.state_vector(T, 4, 4)
    ex = np.array([X.exact_expect(psi, 16, 2, t) for t in terms])
    assert np.max(np.abs(v - ex)) < 1e-12, np.max(np.abs(v - ex))


def test_infinite_complex_cell_truncating():
    """Infinite 2x2 complex cell, D=2, one 4x4 block (column bonds truncated at chi=16),
    fits run to convergence.  Against the oracle in the Hermitian basis (same arithmetic
    sequence): FP64 to 1e-10, TF32X3 / BF16X3 to 1e-5, plain TF32 / BF16 to ten times their
    operands' unit roundoff; the oracle's sweeps use the fit tolerance each path raises
    1e-12 to (3e-5 / 3e-3 / 3e-2 for the split paths / TF32 / BF16), its read-out fits the
    tolerance of the path's read-out fits (3e-5 on the tensor cores for the split paths, else
    1e-12 in FP64).  The
    complex oracle's truncated fits start from complex draws and may settle in a different,
    equally valid truncated optimum: FP64 in the Hermitian basis stays within 1e-5 of it
    (measured 3.2e-6)."""
    from oracle import blockbp as ob
    T = [t.astype(np.complex128) for t in I.complex_normal_cell(2, 2, 2, 2, seed=3)]
    terms = [[(5, SZ)], [(6, SX)], [(9, SY)], [(10, SPLUS)], [(5, SZ), (6, SZ)], [(5, SX), (9, SX)],
             [(6, SY), (10, SY)]]
    # (sweep, read-out) fit tolerance of each path when 1e-12 is asked for
    floor = {"fp64": (1e-12, 1e-12), "tf32x3": (3e-5, 3e-5), "bf16x3": (3e-5, 3e-5), "tf32": (3e-3, 1e-12),
             "bf16": (3e-2, 1e-12)}
    bound = {"fp64": 1e-10, "tf32x3": 1e-5, "bf16x3": 1e-5, "tf32": 10 * 2.0 ** -11, "bf16": 10 * 2.0 ** -8}
    ref = {}
    for tol in sorted(set(floor.values())):
        o = ob.Lattice(2, 2, 2, 2, 4, 4, T, boundary="infinite", chi=16, fit_tol=tol[0], fit_max_sweeps=30, seed=7,
                       hermitian_basis=True, readout_fit_tol=tol[1])
        for _ in range(8):
            o.sweep()
        ref[tol] = o.expect(terms)
    oc = ob.Lattice(2, 2, 2, 2, 4, 4, T, boundary="infinite", chi=16, fit_tol=1e-12, fit_max_sweeps=30, seed=7)
    for _ in range(8):
        oc.sweep()
    ovc = oc.expect(terms)
    vals, err = {}, {}
    for prec in ("fp64", "tf32x3", "bf16x3", "tf32", "bf16"):
        g = B.Lattice(Lx=2, Ly=2, d=2, D=2, bx=4, by=4, chi=16, boundary="infinite", dtype=B.C128, prec=prec,
                      fit_tol=1e-12, fit_max_sweeps=30, seed=7, hermitian_basis=1)
        g.set_tensors(T)
        g.sweep(8)
        vals[prec] = g.expect(terms)
        g.close()
        err[prec] = float(np.max(np.abs(vals[prec] - ref[floor[prec]])))
    assert all(err[p] < bound[p] for p in err), err
    assert np.max(np.abs(vals["fp64"] - ovc)) < 1e-5
    # Hermitian operators read out exactly real in the real basis
    herm = [k for k, t in enumerate(terms) if all(np.allclose(P, P.conj().T) for _, P in t)]
    assert np.all(vals["fp64"][herm].imag == 0.0)


def test_gauge_dressed_complex_product_is_exact():
    """A complex product state dressed with complex gauges on every bond (dense
    tensors, same state): blockBP is exact for any chi; BF16 contractions in the
    Hermitian basis give the closed-form <sigma> within 1e-3."""
    rng = np.random.default_rng(31)
    vecs = []
    for _ in range(36):
        t = rng.standard_normal(2) + 1j * rng.standard_normal(2)
        vecs.append(t / np.linalg.norm(t))
    T = I.gauge_dress(I.product_peps(6, 6, 2, 3, vecs), 6, 6, seed=32, complex_gauge=True)
    terms = [[(s, P)] for s in (7, 14, 21, 28) for P in (SX, SY, SZ)] + [[(14, SZ), (15, SX)]]
    g = B.Lattice(Lx=6, Ly=6, d=2, D=3, bx=3, by=3, chi=8, dtype=B.C128, prec="bf16", fit_tol=1e-6,
                  fit_max_sweeps=10, seed=3)
    g.set_tensors(T)
    g.sweep(4)
    v = g.expect(terms)
    ex = []
    for t in terms:
        val = 1.0
        for s, P in t:
            val *= np.vdot(vecs[s], P @ vecs[s])
        ex.append(val)
    assert np.max(np.abs(v - np.array(ex))) < 1e-3, np.max(np.abs(v - np.array(ex)))
