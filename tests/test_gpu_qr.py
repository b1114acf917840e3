"""The standalone truncation step (batched QR with non-negative diag(R)) against the
definition: Q^dagger Q = I, R = Q^dagger A upper triangular with a real non-negative
diagonal, Q R = A; loss = -||A||^2."""
import numpy as np
import pytest

from paper_2301_05844_gb300 import binding as B

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("m,n,batch", [(288, 32, 5), (81, 81, 2), (1000, 17, 3), (1024, 64, 2), (600, 512, 1),
                                       (2400, 96, 3), (1500, 37, 2), (5000, 20, 2), (1, 1, 3), (16, 1, 4)])
def test_qr_batched(cplx, m, n, batch):
    """Shapes of the fits, the largest cluster shape (1024 x 64), the blocked one-CTA QR of
    matrices beyond a cluster's shared memory (the 2400 x 96 site matrices of D=5, chi=96;
    panels of 16 / 8 / 4 columns, a last panel narrower than the others), the largest n
    (512) and the degenerate 1 x 1 and single-column cases."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(m + n)
    A = rng.standard_normal((batch, m, n)) + (1j * rng.standard_normal((batch, m, n)) if cplx else 0)
    a = torch.tensor(A.view(np.float64) if cplx else A, dtype=torch.float64, device="cuda")
    q = torch.zeros_like(a)
    loss = torch.zeros(batch, dtype=torch.float64, device="cuda")
    assert B.lib().bbp_qr_batched(batch, m, n, int(cplx), a.data_ptr(), q.data_ptr(), loss.data_ptr(), None) == 0
    Q = q.cpu().numpy()
    Q = Q.view(np.complex128) if cplx else Q
    for b in range(batch):
        R = np.conj(Q[b].T) @ A[b]
        assert np.allclose(np.conj(Q[b].T) @ Q[b], np.eye(n), atol=1e-12)
        assert np.allclose(np.tril(R, -1), 0, atol=1e-10)
        assert np.all(np.abs(np.diag(R).imag) < 1e-10) and np.all(np.diag(R).real >= 0)
        assert np.allclose(Q[b] @ R, A[b], atol=1e-10)
    assert np.allclose(loss.cpu().numpy(), -np.sum(np.abs(A) ** 2, axis=(1, 2)), rtol=1e-13)


@pytest.mark.parametrize("cplx", [False, True])
def test_qr_rank_deficient_and_tiny_columns(cplx):
    """Columns beyond the numerical rank (an exact copy, a zero column, columns at
    1e-170 and 1e-300 scale, an exact multiple left with rounding-level residue): Q stays
    finite and orthonormal, R = Q^dagger A is upper triangular with a non-negative
    diagonal and Q R = A; on the well-conditioned leading columns Q equals numpy's
    (LAPACK) Q with the same sign convention."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    m, n = 81, 12
    A = rng.standard_normal((m, n)) + (1j * rng.standard_normal((m, n)) if cplx else 0)
    A[:, 4] = A[:, 1]                       # exact copy
    A[:, 5] = 0.0                           # zero column
    A[:, 6] *= 1e-170                       # squared norm underflows
    A[:, 7] *= 1e-300                       # entries near the denormal range
    A[:, 8] = 3.0 * A[:, 2] - 0.5 * A[:, 0]  # dependent: residue of rounding size
    A = A[None]
    a = torch.tensor(A.view(np.float64) if cplx else A, dtype=torch.float64, device="cuda")
    q = torch.zeros_like(a)
    assert B.lib().bbp_qr_batched(1, m, n, int(cplx), a.data_ptr(), q.data_ptr(), None, None) == 0
    Q = q.cpu().numpy()
    Q = (Q.view(np.complex128) if cplx else Q)[0]
    assert np.all(np.isfinite(Q))
    assert np.allclose(np.conj(Q.T) @ Q, np.eye(n), atol=1e-12)
    R = np.conj(Q.T) @ A[0]
    assert np.allclose(np.tril(R, -1), 0, atol=1e-10)
    assert np.all(np.abs(np.diag(R).imag) < 1e-10) and np.all(np.diag(R).real >= -1e-12)
    assert np.allclose(Q @ R, A[0], atol=1e-10)
    Qn, Rn = np.linalg.qr(A[0][:, :4])
    ph = np.diag(Rn) / np.abs(np.diag(Rn))
    assert np.allclose(Q[:, :4], Qn * ph[None, :], atol=1e-12)


@pytest.mark.parametrize("m,n,batch,scale", [(9, 9, 3, 1.0), (12, 9, 2, 1.0), (108, 12, 4, 1.0), (27, 27, 2, 1.0),
                                             (1, 1, 2, 1.0), (33, 17, 2, 1.0), (300, 64, 2, 1.0),
                                             (2400, 96, 2, 1.0), (1500, 37, 1, 1.0), (108, 12, 2, 1e25),
                                             (300, 64, 1, 1e-25)])
def test_qr_fp32_arithmetic(m, n, batch, scale):
    """The FP32-arithmetic blocked QR of the tensor-core paths: on small matrices (one panel
    wider than the matrix, square ones) as well as the 2400 x 96 site matrices.  Q against
    the FP64 QR of the same FP32 input with the same sign rule (well-conditioned Gaussian
    matrices: the FP32 factorisation's error is a few units of 2^-24 times a modest growth
    factor), orthonormality, Q R = A with R = Q^T A upper triangular and diag(R) >= 0, the
    loss in FP64, and no write past a task's 2 m n workspace.  Scaled by 1e25 (squares beyond
    the FP32 range) and 1e-25 (squares below it), Q is the same."""
    import ctypes as C
    rng = np.random.default_rng(3 * m + n)
    A = (scale * rng.standard_normal((batch, m, n))).astype(np.float32)
    Q = np.zeros((batch, m, n))
    loss = np.zeros(batch)
    intact = C.c_int(0)
    L = B.lib()
    L.bbp_selftest_qr_fp32.argtypes = [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.POINTER(C.c_int)]
    assert L.bbp_selftest_qr_fp32(batch, m, n, A.ctypes.data, Q.ctypes.data, loss.ctypes.data, C.byref(intact)) == 0
    assert intact.value == 1
    tol = 2e-5 * np.sqrt(m)
    for b in range(batch):
        Ad = A[b].astype(np.float64)
        Qn, Rn = np.linalg.qr(Ad)
        Qn = Qn * np.where(np.diag(Rn) < 0, -1.0, 1.0)[None, :]
        assert np.max(np.abs(Q[b] - Qn)) < tol
        assert np.max(np.abs(Q[b].T @ Q[b] - np.eye(n))) < tol
        R = Q[b].T @ Ad
        assert np.max(np.abs(np.tril(R, -1))) < tol * np.max(np.abs(Ad))
        assert np.all(np.diag(R) > -tol)
        assert np.max(np.abs(Q[b] @ np.triu(R) - Ad)) < tol * np.max(np.abs(Ad))
    assert np.allclose(loss, -np.sum(A.astype(np.float64) ** 2, axis=(1, 2)), rtol=1e-6)
