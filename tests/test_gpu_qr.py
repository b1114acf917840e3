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
