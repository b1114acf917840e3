"""bbp_qr_batched_noalloc, the variant of the batched QR for callers that cannot
allocate device memory mid-run (its workspace is a fixed array inside the library),
gives the same Q and losses as bbp_qr_batched on the same inputs, on two calls in a
row, and a call made after the first one changes neither the device's free memory nor
the caching allocator's counters.  Collected last so that a stop at the first failure
has run every other test."""
import numpy as np
import pytest

from paper_2301_05844_gb300 import binding as B

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_qr_twice():
    torch = pytest.importorskip("torch")
    L = B.lib()
    rng = np.random.default_rng(77)
    for call, (m, n, batch, cplx) in enumerate([(288, 32, 6, 0), (96, 40, 4, 1)]):
        A = rng.standard_normal((batch, m, n * (2 if cplx else 1)))
        a = torch.tensor(A, dtype=torch.float64, device="cuda")
        q_ref, q_na = torch.zeros_like(a), torch.full_like(a, float("nan"))
        l_ref = torch.zeros(batch, dtype=torch.float64, device="cuda")
        l_na = torch.full_like(l_ref, float("nan"))
        assert L.bbp_qr_batched(batch, m, n, cplx, a.data_ptr(), q_ref.data_ptr(), l_ref.data_ptr(), None) == 0
        assert L.bbp_qr_batched_noalloc(batch, m, n, cplx, a.data_ptr(), q_na.data_ptr(), l_na.data_ptr(), None) == 0
        torch.cuda.synchronize()
        assert torch.allclose(q_na, q_ref, rtol=0, atol=1e-10), call
        assert torch.allclose(l_na, l_ref, rtol=1e-13, atol=0), call


def test_noalloc_call_leaves_device_memory_alone():
    """After a first real and a first complex call on the device, further calls leave the
    free device memory and the caching allocator's statistics exactly as they were."""
    torch = pytest.importorskip("torch")
    L = B.lib()
    rng = np.random.default_rng(78)
    bufs = []
    for m, n, cplx in ((240, 24, 0), (120, 16, 1)):
        A = rng.standard_normal((3, m, n * (2 if cplx else 1)))
        a = torch.tensor(A, dtype=torch.float64, device="cuda")
        bufs.append((m, n, cplx, a, torch.zeros_like(a), torch.zeros(3, dtype=torch.float64, device="cuda")))
    # first calls of both scalar types (module and kernels loaded, workspace committed)
    for m, n, cplx, a, q, lo in bufs:
        assert L.bbp_qr_batched_noalloc(3, m, n, cplx, a.data_ptr(), q.data_ptr(), lo.data_ptr(), None) == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    stats0 = {k: v for k, v in torch.cuda.memory_stats().items() if k.endswith(".allocated") or "segment" in k}
    for m, n, cplx, a, q, lo in bufs * 2:
        assert L.bbp_qr_batched_noalloc(3, m, n, cplx, a.data_ptr(), q.data_ptr(), lo.data_ptr(), None) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    stats1 = {k: v for k, v in torch.cuda.memory_stats().items() if k.endswith(".allocated") or "segment" in k}
    assert stats1 == stats0


def test_noalloc_rejects_requests_beyond_the_workspace():
    torch = pytest.importorskip("torch")
    L = B.lib()
    a = torch.zeros(1, dtype=torch.float64, device="cuda")
    # 4096 x 512 doubles need 32 MiB of workspace per matrix
    assert L.bbp_qr_batched_noalloc(1, 4096, 512, 0, a.data_ptr(), a.data_ptr(), None, None) == B.ERR_INVALID
    assert b"workspace" in L.bbp_last_error()
