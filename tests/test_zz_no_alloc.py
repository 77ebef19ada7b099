"""The allocation-free tensor-core GEMM (qtt_cgemm_noalloc), meant for callers
that may not allocate device memory, computes what the allocating entry point
(qtt_cgemm, tensor-core engine) computes, on two calls in a row that reuse its
fixed scratch array; sizes beyond that array are refused up front.

Collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_gemm_matches_allocating_entry_point_on_two_calls():
    import torch
    from paper_2512_07811_gb300 import qtt as Q
    ctx = Q.Context(0)
    stream = torch.cuda.Stream()
    for M, N, K in [(200, 150, 96), (320, 64, 256)]:
        rng = np.random.default_rng(M * N + K)
        A = (rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))).astype(np.complex64)
        B = (rng.standard_normal((K, N)) + 1j * rng.standard_normal((K, N))).astype(np.complex64)
        dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
        ref = torch.zeros((M, N), dtype=torch.complex64, device="cuda")
        out = torch.full((M, N), float("nan"), dtype=torch.complex64, device="cuda")
        torch.cuda.synchronize()
        Q.qtt_cgemm(ctx, M, N, K, dA.data_ptr(), dB.data_ptr(), ref.data_ptr(), 1)
        Q.qtt_cgemm_noalloc(stream.cuda_stream, M, N, K, dA.data_ptr(), dB.data_ptr(), out.data_ptr())
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.all(np.isfinite(o))
        assert np.linalg.norm(o - r) / np.linalg.norm(r) <= 1e-6
        exact = A.astype(np.complex128) @ B.astype(np.complex128)
        assert np.linalg.norm(o - exact) / np.linalg.norm(exact) < 1e-5 + 2.5e-8 * K


def test_noalloc_gemm_refuses_sizes_beyond_its_array():
    import torch
    from paper_2512_07811_gb300 import qtt as Q
    buf = torch.zeros(16, dtype=torch.complex64, device="cuda")
    with pytest.raises(Q.QTTError) as e:
        Q.qtt_cgemm_noalloc(0, 2048, 2048, 2048, buf.data_ptr(), buf.data_ptr(), buf.data_ptr())
    assert e.value.status == -3
