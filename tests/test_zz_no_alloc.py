"""The allocation-free QR entry point agrees with the allocating one.

tt_qr_device_noalloc is for callers that may not allocate device memory where
they need the factorisation (a pool that must not grow, an allocator owned by
another framework, a path that must not synchronise).  It runs the same QR
kernel with its workspace in a fixed device array.  This file is collected
last so that a run stopping at the first failure has run everything else; it
also passes alone in a fresh process.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_qr_matches_allocating_entry_point_twice():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2212_11973_gb300 import tantrg as tt
    tt.load_library()
    ctx = tt.Context()
    rng = np.random.default_rng(2212)
    for (m, n) in ((300, 130), (1100, 257)):  # two calls in a row, different sizes
        A = torch.from_numpy(rng.standard_normal((m, n))).cuda()
        Q_ref, R_ref = tt.qr_device(ctx, A)
        At = A.t().contiguous()                      # column-major m x n
        Q = torch.full((n, m), float("nan"), dtype=torch.float64, device="cuda")
        R = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
        tt.qr_device_noalloc(At, Q, R)
        torch.cuda.synchronize()
        assert torch.allclose(Q.t(), Q_ref, rtol=0, atol=1e-12)
        assert torch.allclose(R.t(), R_ref, rtol=0, atol=1e-11)
    # beyond the fixed scratch: rejected without touching the GPU
    big = torch.zeros((400, 4000), dtype=torch.float64, device="cuda")  # 2 m n + n^2 > 2^21 doubles
    with pytest.raises(tt.TTError):
        tt.qr_device_noalloc(big, torch.empty_like(big), torch.empty((400, 400), dtype=torch.float64, device="cuda"))
    ctx.close()
