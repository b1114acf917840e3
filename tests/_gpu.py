"""Shared helpers for the GPU parity tests: run the CUDA library and the oracle on
the same seeded inputs with the same settings."""
import numpy as np

from oracle import blockbp as ob
from paper_2301_05844_gb300 import binding as B


def run_both(T, Lx, Ly, d, D, bx, by, chi, terms, n_sweeps, boundary="obc", chi_exp=0, fit_tol=0.0,
             fit_max_sweeps=2, seed=7, init_mode=0, dtype=None, prec="fp64", warm_start=False):
    cplx = any(np.iscomplexobj(t) for t in T)
    if dtype is None:
        dtype = B.C128 if cplx else B.F64
    g = B.Lattice(Lx=Lx, Ly=Ly, d=d, D=D, bx=bx, by=by, chi=chi, boundary=boundary, chi_exp=chi_exp, dtype=dtype,
                  prec=prec, fit_tol=fit_tol, fit_max_sweeps=fit_max_sweeps, seed=seed, init_mode=init_mode,
                  warm_start=warm_start)
    g.set_tensors(T)
    o = ob.Lattice(Lx, Ly, d, D, bx, by, [np.asarray(t) for t in T], boundary=boundary, chi=chi, chi_exp=chi_exp,
                   fit_tol=fit_tol, fit_max_sweeps=fit_max_sweeps, seed=seed, init_mode=init_mode,
                   warm_start=warm_start)
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
