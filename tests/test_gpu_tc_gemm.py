"""The tensor-core (tcgen05, kind::tf32, three-term split) complex GEMM
against numpy in complex128 and against the CUDA-core GEMM, on sizes that
span several 128-wide tiles with ragged tails."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("M,N,K", [(128, 64, 32), (300, 200, 150), (512, 256, 1024), (37, 5, 3)])
def test_tc_gemm_matches_reference(M, N, K):
    import torch
    from paper_2512_07811_gb300 import qtt as Q
    ctx = Q.Context(0)
    rng = np.random.default_rng(M + N + K)
    A = (rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))).astype(np.complex64)
    B = (rng.standard_normal((K, N)) + 1j * rng.standard_normal((K, N))).astype(np.complex64)
    ref = A.astype(np.complex128) @ B.astype(np.complex128)
    dA, dB = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    out = {}
    for eng in (0, 1):
        dC = torch.zeros((M, N), dtype=torch.complex64, device="cuda")
        torch.cuda.synchronize()
        Q.qtt_cgemm(ctx, M, N, K, dA.data_ptr(), dB.data_ptr(), dC.data_ptr(), eng)
        out[eng] = dC.cpu().numpy().astype(np.complex128)
    scale = np.abs(A).max() * np.abs(B).max() * K
    rel = lambda x: np.linalg.norm(x - ref) / np.linalg.norm(ref)
    # CUDA cores: FP32 level
    assert np.abs(out[0] - ref).max() <= 2e-6 * scale
    assert rel(out[0]) < 2e-6
    # tensor cores, three-term TF32 split: measured about 2e-5 at K = 1024,
    # growing with K (the accumulation inside the tensor core)
    assert rel(out[1]) < 1e-5 + 2.5e-8 * K


def test_tc32_rounding_and_solver():
    """The tensor-core precision mode: the rounding bound at a tolerance above
    its contraction accuracy, agreement with the CUDA-core float path, and
    the laminate's exact 20/11 to 1e-4."""
    import math
    from oracle import tt as T
    from oracle import ms as MS
    from paper_2512_07811_gb300 import inputs as I
    from paper_2512_07811_gb300 import qtt as Q
    ctx = Q.Context(0)
    low = I.random_tt_cores(16, 2, 64, seed=51, dtype=np.complex128)
    noise = I.random_tt_cores(16, 2, 32, seed=52, dtype=np.complex128)
    x = T.tt_add(low, noise, 1.0, 1e-2)
    g = Q.TT.from_cores(ctx, x, Q.C64)
    y_tc, _ = Q.tt_round(ctx, g, 1e-3, prec=Q.PREC_TC32)
    y_f, _ = Q.tt_round(ctx, g, 1e-3, prec=Q.PREC_F32)
    yt = [c.astype(np.complex128) for c in y_tc.cores()]
    yf = [c.astype(np.complex128) for c in y_f.cores()]
    nx = T.tt_norm(x)
    assert T.tt_norm(T.tt_add(yt, x, 1.0, -1.0)) <= 1e-3 * nx * 1.01
    assert T.tt_norm(T.tt_add(yt, yf, 1.0, -1.0)) <= 1e-4 * nx
    pb = MS.scalar_problem(I.laminate_indicator(32), 1.0, 10.0)
    C, rep = Q.ms_homogenize(ctx, pb.indicator, "scalar", (1.0, 10.0), pb.C0, tol=1e-8, max_rank=64, eps=1e-6,
                             max_iter=6, prec=Q.PREC_TC32, load_mask=1)
    assert abs(C[0, 0] - 20.0 / 11.0) < 1e-4 * 20.0 / 11.0


def test_sketched_rounding_with_single_pass_tensor_core_sketch():
    """QTT_PREC_TF32S: the right partial contractions of the sketch on the
    tensor cores (batched, three-term TF32 split): the rounded Hadamard
    product (rank 128, inside the sketch width 144) keeps the float path's
    accuracy against the exact product, and differs from the float-sketch
    result in the last bits (the tensor-core route did run)."""
    from oracle import tt as T
    from paper_2512_07811_gb300 import inputs as I
    from paper_2512_07811_gb300 import qtt as Q
    ctx = Q.Context(0)
    d = 12
    x = I.random_tt_cores(d, 2, 8, seed=61, dtype=np.complex128)
    y = I.random_tt_cores(d, 2, 16, seed=62, dtype=np.complex128)
    exact = T.tt_full(T.tt_hadamard(x, y))
    sk, _ = I.sketch_cores(np.random.default_rng(63), d, [2] * d, 144)
    X = Q.TT.from_cores(ctx, x, Q.C64)
    Y = Q.TT.from_cores(ctx, y, Q.C64)
    S = Q.TT.from_cores(ctx, sk, Q.C64)
    DX = Q.qtt_mpo_diag(ctx, X)
    errs, fulls = {}, {}
    for name, p in [("f32", Q.PREC_F32), ("tf32s", Q.PREC_TF32S)]:
        z, info = Q.tt_round_sketched(ctx, [(1.0, DX, Y)], S, 1e-6, 0, prec=p)
        fulls[name] = T.tt_full([c.astype(np.complex128) for c in z.cores()])
        errs[name] = np.linalg.norm(fulls[name] - exact) / np.linalg.norm(exact)
    print("\nrelative error: float sketch %.2e, tensor-core sketch %.2e" % (errs["f32"], errs["tf32s"]))
    assert errs["f32"] < 2e-5 and errs["tf32s"] < 2e-5
    assert np.abs(fulls["f32"] - fulls["tf32s"]).max() > 0
