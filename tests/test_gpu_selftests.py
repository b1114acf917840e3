"""Device self-tests that are not steps of the method.

* A bounded pipeline wait runs out: a tensor-core GEMM whose operand copies are withheld
  returns BBP_ERR_TIMEOUT (the wait gives up, the CTAs free their tensor memory and return),
  and the context stays usable (the same GEMM then runs normally).
* The QR's refined 1/sqrt(s) and 1/d (FP32 seeds, one third-order step in FP64) against
  the exact values (Python's decimal arithmetic at 60 digits) and CUDA's 1.0 / sqrt(x) and
  1.0 / x, over [2^-100, 2^100]: within 2 units in the last place."""
import decimal
import numpy as np
import pytest

from paper_2301_05844_gb300 import binding as B

pytestmark = pytest.mark.gpu


def test_gemm_wait_times_out_with_a_status():
    L = B.lib()
    assert L.bbp_selftest_gemm_timeout() == B.ERR_TIMEOUT
    assert b"timed out" in L.bbp_last_error()
    rng = np.random.default_rng(3)
    A = rng.standard_normal((256, 64)).astype(np.float32)
    Bm = rng.standard_normal((64, 64)).astype(np.float32)
    Cm = np.zeros((256, 64), np.float32)
    assert L.bbp_selftest_gemm(256, 64, 64, B.PREC_TF32, A.ctypes.data, Bm.ctypes.data, Cm.ctypes.data) == 0
    ref = A.astype(np.float64) @ Bm.astype(np.float64).T
    assert np.abs(Cm - ref).max() < 1e-2 * np.abs(ref).max()


def _ulps(got, exact):
    """|got - exact| in units of the spacing of doubles at exact."""
    return np.abs(got - exact) / np.spacing(np.abs(exact))


def test_refined_rsqrt_and_reciprocal_ulp_bound():
    import ctypes as C
    L = B.lib()
    rng = np.random.default_rng(11)
    e = rng.uniform(-100.0, 100.0, 4000)
    x = np.concatenate([np.exp2(e), np.exp2(np.arange(-100, 101, dtype=np.float64)),
                        [1.0, np.nextafter(1.0, 2.0), np.nextafter(1.0, 0.0), 2.0 ** 100, 2.0 ** -100,
                         np.nextafter(2.0 ** -100, 1.0), np.nextafter(2.0 ** 100, 0.0)]])
    x = np.clip(x, 2.0 ** -100, 2.0 ** 100)
    outs = [np.zeros_like(x) for _ in range(4)]
    p = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    L.bbp_selftest_scalar.argtypes = [C.c_longlong] + [C.POINTER(C.c_double)] * 5
    assert L.bbp_selftest_scalar(len(x), p(x), *[p(o) for o in outs]) == 0
    rs, rc, rs_cuda, rc_cuda = outs
    ctx = decimal.Context(prec=60)
    ex_rs = np.array([float(ctx.divide(1, ctx.sqrt(decimal.Decimal(float(v))))) for v in x])
    ex_rc = np.array([float(ctx.divide(1, decimal.Decimal(float(v)))) for v in x])
    assert np.all(rc_cuda == ex_rc)  # IEEE division is correctly rounded
    assert np.max(_ulps(rs_cuda, ex_rs)) <= 1.0  # two correctly rounded steps
    u_rs, u_rc = np.max(_ulps(rs, ex_rs)), np.max(_ulps(rc, ex_rc))
    assert u_rs <= 2.0 and u_rc <= 2.0, (u_rs, u_rc)
    assert np.max(np.abs(rs - rs_cuda) / np.spacing(rs_cuda)) <= 3.0
