"""Shared helpers for the GPU parity tests: run the CUDA library and the oracle on
the same seeded inputs with the same settings."""
import numpy as np

from oracle import blockbp as ob
from paper_2301_05844_gb300 import binding as B


def run_both(T, Lx, Ly, d, D, bx, by, chi, terms, n_sweeps, boundary="obc", chi_exp=0, fit_tol=0.0,
             fit_max_sweeps=2, seed=7, init_mode=0, dtype=None, prec="fp64", warm_start=False, hermitian_basis=0,
             single_layer=False, shift=(0, 0), oracle_hb=False, oracle_fit_tol=None, oracle_readout_fit_tol=None,
             keep_fp64=0):
    """oracle_hb: run the oracle in its Hermitian-basis option (the basis of the library's
    real-arithmetic paths for complex tensors).  oracle_fit_tol / oracle_readout_fit_tol: the
    fit tolerance of the oracle's message sweeps / read-out fits (default: fit_tol), set to
    what the library's path raises fit_tol to."""
    cplx = any(np.iscomplexobj(t) for t in T)
    if dtype is None:
        dtype = B.C128 if cplx else B.F64
    g = B.Lattice(Lx=Lx, Ly=Ly, d=d, D=D, bx=bx, by=by, chi=chi, boundary=boundary, chi_exp=chi_exp, dtype=dtype,
                  prec=prec, fit_tol=fit_tol, fit_max_sweeps=fit_max_sweeps, seed=seed, init_mode=init_mode,
                  warm_start=warm_start, hermitian_basis=hermitian_basis, single_layer=int(single_layer), shift=shift,
                  keep_fp64=keep_fp64)
    g.set_tensors(T)
    o = ob.Lattice(Lx, Ly, d, D, bx, by, [np.asarray(t) for t in T], boundary=boundary, chi=chi, chi_exp=chi_exp,
                   fit_tol=fit_tol if oracle_fit_tol is None else oracle_fit_tol, fit_max_sweeps=fit_max_sweeps,
                   seed=seed, init_mode=init_mode, warm_start=warm_start, single_layer=single_layer, shift=shift,
                   hermitian_basis=oracle_hb,
                   readout_fit_tol=fit_tol if oracle_readout_fit_tol is None else oracle_readout_fit_tol)
    gres, ores = [], []
    for _ in range(n_sweeps):
        gres.append(g.sweep(1)[0])
        ores.append(o.sweep())
    gv = g.expect(terms) if terms else None
    ov = o.expect(terms) if terms else None
    return g, o, np.array(gres), np.array(ores), gv, ov


def message_fidelity(g, o):
    """min over messages of |<m_gpu|m_oracle>| (both unit norm)."""
    worst = 1.0
    for (bi, dr), m in o.msgs.items():
        mg = g.get_message(bi, dr)
        ov = abs(ob.mps_overlap(mg, m))
        worst = min(worst, ov)
    return worst


def to_hermitian_basis(site, D, conj_basis=False):
    """Message site [a, k, b] (k = ket*D + bra) in the library's Hermitian basis:
    coordinate v_(x,x) at k = x*D + x, (v_(x,y) + v_(y,x))/sqrt 2 at k = x*D + y for x < y,
    (v_(y,x) - v_(x,y))/(i sqrt 2) at k = x*D + y for x > y (sign flipped in the conjugate
    basis, which the down and right legs use)."""
    out = np.zeros(site.shape, dtype=np.complex128)
    for x in range(D):
        for y in range(D):
            k, kt = x * D + y, y * D + x
            if x == y:
                out[:, k, :] = site[:, k, :]
            elif x < y:
                out[:, k, :] = (site[:, k, :] + site[:, kt, :]) / np.sqrt(2)
            else:
                out[:, k, :] = (site[:, kt, :] - site[:, k, :]) / (1j * np.sqrt(2)) * (-1 if conj_basis else 1)
    return out


def message_fidelity_hb(g, o, D):
    """min over messages of |<m_gpu|V m_oracle>| for a lattice run in the Hermitian basis."""
    worst = 1.0
    for (bi, dr), m in o.msgs.items():
        mg = g.get_message(bi, dr)
        # a message carries the legs of its side: right / down legs use the conjugate basis
        mo = [to_hermitian_basis(np.asarray(x), D, conj_basis=dr in (B.RIGHT, B.DOWN)) for x in m]
        worst = min(worst, abs(ob.mps_overlap(mg, mo)))
    return worst
