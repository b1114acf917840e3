"""Launch-shape autotuner (bbp_autotune): the chosen GEMM tiles and QR cluster sizes change
speed, never results."""
import numpy as np
import pytest

from paper_2301_05844_gb300 import binding as B
from paper_2301_05844_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _run(prec, tune):
    T = I.uniform_noise_peps(6, 6, 2, 3, seed=15)
    g = B.Lattice(Lx=6, Ly=6, d=2, D=3, bx=3, by=3, chi=24, prec=prec, fit_tol=1e-6, fit_max_sweeps=4, seed=5,
                  warm_start=1)
    g.set_tensors(T)
    info = g.autotune(2) if tune else None
    res = [g.sweep(1)[0] for _ in range(3)]
    v = g.expect(I.standard_terms(6, 6))
    msgs = [np.concatenate([x.ravel() for x in g.get_message(0, B.RIGHT)])]
    g.close()
    return np.array(res), v, msgs, info


@pytest.mark.parametrize("prec", ["tf32x3", "bf16", "fp64"])
def test_autotuned_tiles_give_identical_results(prec):
    r0, v0, m0, _ = _run(prec, False)
    r1, v1, m1, info = _run(prec, True)
    before, after, changed = info
    assert before > 0 and 0 < after <= before * 1.05
    assert np.array_equal(r0, r1)
    assert np.array_equal(v0, v1)
    assert all(np.array_equal(a, b) for a, b in zip(m0, m1))


def test_autotune_order_and_fp64_qr_only():
    T = I.uniform_noise_peps(4, 4, 2, 2, seed=1)
    g = B.Lattice(Lx=4, Ly=4, d=2, D=2, bx=2, by=2, chi=16, prec="tf32x3")
    with pytest.raises(B.BBPError) as e:
        g.autotune(1)  # no tensors yet
    assert e.value.code == B.ERR_STATE
    g.set_tensors(T)
    g.sweep(1)
    with pytest.raises(B.BBPError) as e:
        g.autotune(1)  # sweeps already ran
    assert e.value.code == B.ERR_STATE
    h = B.Lattice(Lx=4, Ly=4, d=2, D=2, bx=2, by=2, chi=16)
    h.set_tensors(T)
    before, after, changed = h.autotune(1)  # FP64 path: only the QR cluster sizes are tuned
    assert before > 0 and 0 < after <= before and changed >= 0
