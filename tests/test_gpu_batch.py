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


def test_batch_equals_sequential(Q):
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


def _rank_limited(seed, d, n, K, k_true):
    """A train of bond ranks K whose true ranks are min(K, k_true): the last
    K - k_true slices of every inner bond are zero."""
    rng = np.random.default_rng(seed)
    ranks = [1] + [min(K, n ** min(k, d - k)) for k in range(1, d)] + [1]
    cores = []
    for k in range(d):
        c = (rng.standard_normal((ranks[k], n, ranks[k + 1]))
             + 1j * rng.standard_normal((ranks[k], n, ranks[k + 1]))) / np.sqrt(2 * K)
        if k < d - 1 and ranks[k + 1] > k_true:
            c[:, :, k_true:] = 0
        cores.append(c)
    return cores


@pytest.mark.parametrize("fp32", [False, True])
def test_round_batch_equals_one_by_one(Q, fp32):
    """Trains of one shape but different true ranks (so the lockstep path pads
    and crops) plus flat random trains truncated at 1e-3: every output has the
    ranks of its own tt_round and agrees with it (1e-10 FP64, 1e-5 FP32) and
    with the oracle's rounding."""
    from oracle import tt as T
    ctx = Q.Context(0)
    dt = Q.C64 if fp32 else Q.C128
    trains = []
    for b, kt in enumerate([3, 9, 16, 16, 5, 12]):
        base = _rank_limited(200 + b, 10, 2, 16, kt)
        trains.append(T.tt_add(base, base, 1.0, 0.75))
    rng_eps = 1e-6 if fp32 else 1e-10
    xs = [Q.TT.from_cores(ctx, c, dt) for c in trains]
    ys, infos = Q.tt_round_batch(ctx, xs, rng_eps)
    for b, (x, y, inf) in enumerate(zip(xs, ys, infos)):
        y1, inf1 = Q.tt_round(ctx, x, rng_eps)
        assert y.ranks == y1.ranks, (b, y.ranks, y1.ranks)
        assert abs(inf.norm - inf1.norm) <= 1e-12 * inf1.norm
        ref, _ = T.tt_round(trains[b], rng_eps)
        assert y.ranks == T.tt_ranks(ref)
        tol = 1e-5 if fp32 else 1e-10
        yc = [c.astype(np.complex128) for c in y.cores()]
        d1 = T.tt_norm(T.tt_add(yc, [c.astype(np.complex128) for c in y1.cores()], 1.0, -1.0)) / inf1.norm
        d2 = T.tt_norm(T.tt_add(yc, ref, 1.0, -1.0)) / T.tt_norm(ref)
        assert d1 < tol and d2 < tol, (b, d1, d2)
    # flat spectra, a real truncation at 1e-3: ranks may differ per train
    flat = [I.random_tt_cores(12, 2, 24, seed=300 + b, dtype=np.complex128) for b in range(4)]
    xs = [Q.TT.from_cores(ctx, c, dt) for c in flat]
    ys, _ = Q.tt_round_batch(ctx, xs, 1e-3)
    for x, y, c in zip(xs, ys, flat):
        y1, _ = Q.tt_round(ctx, x, 1e-3)
        assert y.ranks == y1.ranks
        yc = [a.astype(np.complex128) for a in y.cores()]
        assert T.tt_norm(T.tt_add(yc, c, 1.0, -1.0)) <= 1e-3 * T.tt_norm(c) * (1 + 1e-6)


def test_round_batch_bench_shape(Q):
    """The rank-128 sums of the TT-op workload (d = 30) in FP32, four at a
    time.  Their flat spectra truncate nothing at 1e-6, so the rounded train
    equals its input up to FP32 rounding: ranks of the one-by-one rounding,
    and both results within 5e-5 of the input (the batched GEMMs take other
    tiles and split-K than single ones, so the two FP32 results differ at
    that level -- 3.5e-5 measured -- but neither is closer to the input)."""
    from oracle import tt as T
    ctx = Q.Context(0)
    zs, zc = [], []
    for b in range(4):
        x = I.random_tt_cores(30, 2, 64, seed=400 + b, dtype=np.complex128)
        y = I.random_tt_cores(30, 2, 64, seed=500 + b, dtype=np.complex128)
        z = Q.tt_add(ctx, 1.0, Q.TT.from_cores(ctx, x, Q.C64), 1.0, Q.TT.from_cores(ctx, y, Q.C64))
        zs.append(z)
        zc.append([c.astype(np.complex128) for c in z.cores()])
    ys, infos = Q.tt_round_batch(ctx, zs, 1e-6)
    for z, c, y, inf in zip(zs, zc, ys, infos):
        y1, inf1 = Q.tt_round(ctx, z, 1e-6)
        assert y.ranks == y1.ranks
        nz = T.tt_norm(c)
        for out in (y, y1):
            a = [t.astype(np.complex128) for t in out.cores()]
            assert T.tt_norm(T.tt_add(a, c, 1.0, -1.0)) < 5e-5 * nz


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_concurrent_load_cases_equal_sequential(Q, prec):
    """The six load cases of an 8^3 elastic sphere solved at the same time on
    six streams (operators built once, shared read-only) give the same
    effective tensor bit for bit as one after another, and the timed region
    counts the iterations after the warm-up of every load case."""
    ctx = Q.Context(0)
    lam1, mu1 = I.lame_from_young(1.0, 0.3)
    lam2, mu2 = I.lame_from_young(10.0, 0.3)
    C0 = MS.iso_voigt(0.5 * (lam1 + lam2), 0.5 * (mu1 + mu2))
    geo = Q.Ellipsoids(I.sphere_rows(0.2), (8, 8, 8))
    p = Q.PREC_F64 if prec == "f64" else Q.PREC_F32
    kw = dict(tol=0.0, max_rank=64, eps=1e-6, prec=p, max_iter=5, min_iter=5, interleaved=False, warm_iter=2)
    Cs, rs = Q.ms_homogenize(ctx, geo, "elastic", (lam1, mu1, lam2, mu2), C0, lc_workers=1, **kw)
    Cc, rc = Q.ms_homogenize(ctx, geo, "elastic", (lam1, mu1, lam2, mu2), C0, lc_workers=6, **kw)
    np.testing.assert_array_equal(Cs, Cc)
    assert rc.timed_iter == 6 * 3 and rc.timed_ms > 0 and rc.timed_launches > 0
    assert list(rc.iterations) == [5] * 6


def test_setup_handle_reused_equals_one_call(Q):
    """Operator trains built once (ms_setup) and used by two solves of
    different precisions give the effective tensors of two ms_homogenize
    calls bit for bit."""
    ctx = Q.Context(0)
    geo = Q.Ellipsoids(I.sphere_rows(0.2), (8, 8, 8))
    kw = dict(tol=1e-6, max_rank=64, eps=1e-6, max_iter=20, interleaved=False, load_mask=0b11)
    ops = Q.ms_setup(ctx, geo, "scalar", (1.0, 10.0), 5.5 * np.eye(3), interleaved=False)
    g, p = ops.ranks
    assert g > 1 and p > 1
    for prec in [Q.PREC_F64, Q.PREC_F32]:
        Ca, ra = Q.ms_homogenize(ctx, geo, "scalar", (1.0, 10.0), 5.5 * np.eye(3), prec=prec, **kw)
        Cb, rb = Q.ms_homogenize(ctx, None, "scalar", None, None, prec=prec, ops=ops, **kw)
        np.testing.assert_array_equal(Ca, Cb)
        assert rb.setup_ms == 0 and ra.green_rank == rb.green_rank == g


def test_results_identical_across_processes():
    """The same solve in two fresh processes gives the same effective tensor
    bit for bit: the GEMM tile tuner, which each process runs by timing,
    chooses only between tile edges that sum in the same order."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = (
        "import sys; sys.path.insert(0, %r)\n"
        "import numpy as np\n"
        "from paper_2512_07811_gb300 import qtt as Q, inputs as I\n"
        "ctx = Q.Context(0)\n"
        "geo = Q.Ellipsoids(I.sphere_rows(0.2), (16, 16, 16))\n"
        "C, rep = Q.ms_homogenize(ctx, geo, 'scalar', (1.0, 10.0), 5.5 * np.eye(3), tol=0.0, max_rank=64,\n"
        "                         eps=1e-6, prec=Q.PREC_F32, max_iter=4, min_iter=4, interleaved=False)\n"
        "print(' '.join(float(v).hex() for v in C.ravel()))\n" % root)
    outs = [subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
            for _ in range(2)]
    for o in outs:
        assert o.returncode == 0, o.stderr[-2000:]
    assert outs[0].stdout.strip().splitlines()[-1] == outs[1].stdout.strip().splitlines()[-1]
