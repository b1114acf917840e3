"""The standalone truncation step (batched QR with non-negative diag(R)) against the
definition: Q^dagger Q = I, R = Q^dagger A upper triangular with a real non-negative
diagonal, Q R = A; loss = -||A||^2."""
import numpy as np
import pytest

from paper_2301_05844_gb300 import binding as B

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("m,n,batch", [(288, 32, 5), (81, 81, 2), (1000, 17, 3)])
def test_qr_batched(cplx, m, n, batch):
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
