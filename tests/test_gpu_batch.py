"""Many RVEs solved together (concurrent streams) give exactly the results of
one-by-one solves, and finish sooner than the one-by-one loop."""
import time

import numpy as np
import pytest

from oracle import ms as MS
from paper_2512_07811_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    from paper_2512_07811_gb300 import qtt
    return qtt


def problems():
    out = []
    lam1, mu1 = I.lame_from_young(1.0, 0.3)
    for i, (nb, rng) in enumerate(I.batched_rve_set(count=3, seed=4, log2_min=3, log2_max=3)):
        ind, contrast = I.ellipsoid_rve(1 << nb, rng)
        pb = MS.scalar_problem(ind, 1.0, contrast)
        out.append((pb.indicator, "scalar", (1.0, contrast), pb.C0))
    pb = MS.scalar_problem(I.sphere_indicator(8, 0.2), 1.0, 10.0)
    out.append((pb.indicator, "scalar", (1.0, 10.0), pb.C0))
    lam2, mu2 = I.lame_from_young(10.0, 0.3)
    pe = MS.elastic_problem(I.box_indicator(8, 0.2), lam1, mu1, lam2, mu2)
    out.append((pe.indicator, "elastic", (lam1, mu1, lam2, mu2), pe.C0))
    return out


def test_batch_equals_sequential_and_is_faster(Q):
    ctx = Q.Context(0)
    probs = problems()
    kw = dict(tol=1e-6, max_rank=32, eps=1e-6, max_iter=6, min_iter=6, prec=Q.PREC_F32, load_mask=0x3)
    t0 = time.perf_counter()
    seq = [Q.ms_homogenize(ctx, ind, kind, mod, C0, **kw)[0] for ind, kind, mod, C0 in probs]
    t_seq = time.perf_counter() - t0
    t0 = time.perf_counter()
    bat, reps = Q.ms_homogenize_batch(ctx, probs, workers=8, **kw)
    t_bat = time.perf_counter() - t0
    print("\nsequential %.2f s, batched %.2f s" % (t_seq, t_bat))
    for a, b in zip(seq, bat):
        np.testing.assert_array_equal(a[:, :2], b[:, :2])
    assert all(r.iterations[0] == 6 for r in reps)
    assert t_bat < t_seq
