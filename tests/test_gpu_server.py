"""Request server (continuous batching of whole solves): every solve served in a mix,
under a byte budget that forces queuing, returns exactly what the same solve returns
when run alone through bbp_create_lattice / bbp_sweep / bbp_expect, and a served FP64
solve agrees with the oracle run to the same stop rule."""
import numpy as np
import pytest

from paper_2301_05844_gb300 import binding as B
from paper_2301_05844_gb300 import inputs

pytestmark = pytest.mark.gpu


def _mix():
    """Requests of different sizes, block shapes, precisions and stop rules."""
    reqs = []

    def add(T, terms, **kw):
        reqs.append((T, terms, kw))

    T1 = inputs.uniform_noise_peps(4, 4, 2, 2, seed=1)
    add(T1, inputs.standard_terms(4, 4), Lx=4, Ly=4, d=2, D=2, bx=2, by=2, chi=16, tol=1e-10, max_sweeps=30, seed=1)
    T6 = inputs.uniform_noise_peps(6, 6, 2, 3, seed=11)
    add(T6, inputs.standard_terms(6, 6), Lx=6, Ly=6, d=2, D=3, bx=3, by=2, chi=12, tol=1e-8, max_sweeps=20,
        seed=2, fit_tol=1e-6, fit_max_sweeps=4)
    T12 = inputs.near_product_peps(12, 12, 2, 3, seed=2)
    add(T12, inputs.standard_terms(12, 12)[:40], Lx=12, Ly=12, d=2, D=3, bx=3, by=3, chi=32, dtype=B.F32,
        prec="tf32", tol=1e-8, max_sweeps=12, seed=3, fit_tol=1e-6, fit_max_sweeps=6, warm_start=1)
    T8 = inputs.uniform_noise_peps(8, 8, 2, 2, seed=12)
    add(T8, inputs.standard_terms(8, 8)[:30], Lx=8, Ly=8, d=2, D=2, bx=4, by=4, chi=16, prec="bf16", tol=1e-6,
        max_sweeps=10, seed=4, fit_tol=1e-6, fit_max_sweeps=4)
    Tc = inputs.complex_normal_cell(2, 2, 2, 2, seed=13, dtype=np.complex128)
    add(Tc, [[(0, inputs.SIGMA_Z)], [(5, inputs.SIGMA_X)], [(0, inputs.SIGMA_Z), (1, inputs.SIGMA_Z)]],
        Lx=2, Ly=2, d=2, D=2, bx=4, by=4, chi=16, boundary="infinite", dtype=B.C128, tol=1e-9, max_sweeps=25,
        seed=5, stop_relative=0)
    Ts = inputs.uniform_noise_peps(4, 4, 2, 2, seed=14)  # one block: no messages
    add(Ts, inputs.standard_terms(4, 4)[:8], Lx=4, Ly=4, d=2, D=2, bx=4, by=4, chi=16, seed=6)
    # repeats with other seeds, so that equal shapes share the device at once
    add(T1, inputs.standard_terms(4, 4)[:10], Lx=4, Ly=4, d=2, D=2, bx=2, by=2, chi=16, tol=1e-9, max_sweeps=30,
        seed=21)
    add(T6, inputs.standard_terms(6, 6)[:12], Lx=6, Ly=6, d=2, D=3, bx=3, by=2, chi=12, tol=1e-8, max_sweeps=20,
        seed=22, fit_tol=1e-6, fit_max_sweeps=4)
    return reqs


def _alone(T, terms, kw):
    g = B.Lattice(**kw)
    g.set_tensors(T)
    r, k, _ = g.sweep(0)
    v = g.expect(terms)
    g.close()
    return v, k, r


def test_served_mix_equals_solves_run_alone():
    reqs = _mix()
    feet = [B.footprint(**kw) for _, _, kw in reqs]
    budget = sorted(feet)[-1] + sorted(feet)[-2]  # at most the two largest at once: queuing happens
    srv = B.Server(max_bytes=budget, max_active=6)
    try:
        ids = [srv.submit(T, terms, **kw) for T, terms, kw in reqs]
        served = [srv.wait(i, timeout_s=300.0) for i in ids]
        st = srv.stats()
        assert st["done"] == len(reqs) and st["bytes_in_use"] == 0
    finally:
        srv.close()
    for (T, terms, kw), out in zip(reqs, served):
        v, k, r = _alone(T, terms, kw)
        assert out["state"] == B.Server.DONE
        assert out["sweeps"] == k, kw
        # same launches on the same data: bit-identical results
        assert np.array_equal(out["values"], v), (kw, np.max(np.abs(out["values"] - v)))
        assert out["residual"] == r
        assert out["latency_s"] > 0


def test_served_solve_matches_the_oracle():
    from oracle import blockbp as ob
    T = inputs.uniform_noise_peps(4, 4, 2, 2, seed=1)
    terms = inputs.standard_terms(4, 4)
    srv = B.Server(max_bytes=1 << 30, max_active=2)
    try:
        rid = srv.submit(T, terms, Lx=4, Ly=4, d=2, D=2, bx=2, by=2, chi=16, tol=1e-9, max_sweeps=30, seed=7,
                         fit_tol=0.0, fit_max_sweeps=2)
        out = srv.wait(rid, timeout_s=300.0)
    finally:
        srv.close()
    o = ob.Lattice(4, 4, 2, 2, 2, 2, T, chi=16, fit_tol=0.0, fit_max_sweeps=2, seed=7)
    r, k, conv = o.run(tol=1e-9, max_sweeps=30)
    assert conv and out["sweeps"] == k
    assert np.max(np.abs(out["values"] - o.expect(terms))) < 1e-10
