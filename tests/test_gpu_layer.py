"""The layered pair contraction of the read-out's site rows (App. A read-out closings of real
double-layer lattices, contracted with the ket and the bra tensor in turn instead of with
E = sum_p Tk_p (x) Tb_p), through bbp_selftest_layer, against the definition written with
numpy: ragged pair counts (not a multiple of the CTA's 8 or 4 pairs), odd and unit legs,
d = 1..4, the largest legs the kernel takes (K1 K2 = N1 N2 = 32), FP64 and FP32 arithmetic."""
import ctypes as C

import numpy as np
import pytest

from paper_2301_05844_gb300 import binding as B

pytestmark = pytest.mark.gpu

SHAPES = [  # d, K1, K2, N1, N2, M1, M2
    (2, 5, 5, 5, 5, 2, 20),
    (3, 3, 2, 2, 3, 3, 13),
    (1, 1, 4, 4, 1, 1, 5),
    (2, 4, 8, 8, 4, 2, 9),
    (4, 2, 2, 3, 3, 2, 7),
    (2, 1, 1, 1, 32, 1, 3),
    (1, 32, 1, 1, 1, 2, 3),
]


def _run(f32, d, K1, K2, N1, N2, M1, M2, X, Tk, Tb):
    L = B.lib()
    L.bbp_selftest_layer.argtypes = [C.c_int] * 8 + [C.c_void_p] * 4
    Y = np.zeros((M1, M2, N1 * N1, N2 * N2))
    rc = L.bbp_selftest_layer(f32, d, K1, K2, N1, N2, M1, M2, X.ctypes.data, Tk.ctypes.data, Tb.ctypes.data,
                              Y.ctypes.data)
    return rc, Y


def _reference(X, Tk, Tb, K1, K2, M1, M2, N1, N2):
    """Y[m1][m2][(n1 n1')][(n2 n2')] = sum_p Tk[p,k1,k2,n1,n2] X[(k1 k1')][m1][(k2 k2')][m2]
    Tb[p,k1',k2',n1',n2'], and the same sum over absolute values (the rounding scale)."""
    X6 = X.reshape(K1, K1, M1, K2, K2, M2)
    spec = "pabcd,aembfn,pefgh->mncgdh"
    Y = np.einsum(spec, Tk, X6, Tb).reshape(M1, M2, N1 * N1, N2 * N2)
    S = np.einsum(spec, np.abs(Tk), np.abs(X6), np.abs(Tb)).reshape(M1, M2, N1 * N1, N2 * N2)
    return Y, S


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("f32", [0, 1])
def test_layer_pair_against_definition(shape, f32):
    d, K1, K2, N1, N2, M1, M2 = shape
    rng = np.random.default_rng(7 * d + K1 + 3 * N2 + M2)
    X = rng.standard_normal((K1 * K1, M1, K2 * K2, M2))
    Tk = rng.standard_normal((d, K1, K2, N1, N2))
    Tb = rng.standard_normal((d, K1, K2, N1, N2))
    rc, Y = _run(f32, d, K1, K2, N1, N2, M1, M2, X, Tk, Tb)
    assert rc == 0
    ref, scale = _reference(X, Tk, Tb, K1, K2, M1, M2, N1, N2)
    # FP64: rounding of sums of at most d K1 K2 (K1 K2 + 1) terms; FP32: operands and the
    # intermediate rounded to 2^-24, sums of at most d K1 K2 terms
    tol = 1e-5 if f32 else 1e-13
    assert np.all(np.abs(Y - ref) <= tol * scale), np.max(np.abs(Y - ref) / scale)


def test_layer_pair_same_tensor_and_rejected_shapes():
    """Ket and bra the same tensor (the rows without an operator): Y is symmetric under the
    joint swap of ket and bra on every leg when X is; legs beyond the kernel are refused."""
    d, K1, K2, N1, N2, M1, M2 = 2, 3, 3, 3, 3, 1, 6
    rng = np.random.default_rng(11)
    X = rng.standard_normal((K1, K1, M1, K2, K2, M2))
    X = 0.5 * (X + X.transpose(1, 0, 2, 4, 3, 5))  # symmetric under (k1 k1')(k2 k2') swaps
    X = X.reshape(K1 * K1, M1, K2 * K2, M2)
    T = rng.standard_normal((d, K1, K2, N1, N2))
    rc, Y = _run(0, d, K1, K2, N1, N2, M1, M2, X, T, T)
    assert rc == 0
    Y6 = Y.reshape(M1, M2, N1, N1, N2, N2)
    assert np.max(np.abs(Y6 - Y6.transpose(0, 1, 3, 2, 5, 4))) < 1e-12 * np.max(np.abs(Y6))
    big = np.zeros(36 * 36)
    rc, _ = _run(0, 2, 6, 6, 1, 1, 1, 1, big, np.zeros(2 * 36), np.zeros(2 * 36))
    assert rc < 0
