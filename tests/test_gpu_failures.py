"""Error paths on the GPU, every failure made on the host side (no GPU
fault): a non-finite input core must end a rounding with QTT_ERR_NAN, and an
injected allocation failure must return QTT_ERR_OOM with the context still
usable afterwards."""
import numpy as np
import pytest

from paper_2512_07811_gb300 import inputs as I

pytestmark = pytest.mark.gpu

QTT_ERR_OOM = -2
QTT_ERR_NAN = -6


@pytest.fixture(scope="module")
def Q():
    from paper_2512_07811_gb300 import qtt
    return qtt


@pytest.fixture(scope="module")
def ctx(Q):
    return Q.Context(0)


@pytest.mark.parametrize("dtype", ["c128", "c64"])
def test_nan_poisoned_core_returns_err_nan(Q, ctx, dtype):
    cores = I.random_tt_cores(10, 2, 8, seed=3, dtype=np.complex128)
    cores[4] = cores[4].copy()
    cores[4][0, 1, 0] = np.nan
    dt = Q.C128 if dtype == "c128" else Q.C64
    x = Q.TT.from_cores(ctx, cores, dtype=dt)
    with pytest.raises(Q.QTTError) as e:
        Q.tt_round(ctx, x, 1e-6)
    assert e.value.status == QTT_ERR_NAN
    # the same context still rounds a clean train
    y, info = Q.tt_round(ctx, Q.TT.from_cores(ctx, I.random_tt_cores(10, 2, 8, seed=4), dtype=dt), 1e-6)
    assert info.max_rank_out <= 8


def test_nan_poisoned_phase_image_returns_err_nan(Q, ctx):
    ind = np.zeros((8, 8, 8))
    ind[:4] = 1.0
    ind[2, 3, 1] = np.nan
    with pytest.raises(Q.QTTError) as e:
        Q.ms_homogenize(ctx, ind, "scalar", (1.0, 10.0), 5.5 * np.eye(3), tol=1e-8, max_rank=16, eps=1e-8)
    assert e.value.status == QTT_ERR_NAN


@pytest.mark.parametrize("after", [0, 3, 20])
def test_injected_allocation_failure_returns_err_oom(Q, ctx, after):
    import torch
    x = Q.TT.from_cores(ctx, I.random_tt_cores(12, 2, 16, seed=5))
    ref, _ = Q.tt_round(ctx, x, 1e-8)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    ctx.fail_alloc_after(after)
    try:
        with pytest.raises(Q.QTTError) as e:
            Q.tt_round(ctx, x, 1e-8)
        assert e.value.status == QTT_ERR_OOM
    finally:
        ctx.fail_alloc_after(-1)
    ctx.sync()
    y, _ = Q.tt_round(ctx, x, 1e-8)
    assert y.ranks == ref.ranks
    # nothing of the failed call is left allocated beyond the stream-ordered pool's slack
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)
