"""The tensor-core path: tcgen05 GEMM scores, the dense cutover and the
exhaustive scan, all against FP64."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GAMMA_TC = 2.0 ** -12     # accumulation-error allowance the library's bound uses
U_BF16 = 2.0 ** -8


@pytest.fixture(scope="module")
def gt():
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device: the GPU tests need a GB300")
    from paper_2311_02573_gb300 import gt as g
    g.load()
    return g


def bf16_value(bits):
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def bf16_rn(x):
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return ((b + 0x7FFF + ((b >> 16) & 1)) >> 16).astype(np.uint16)


def same_sets(res, ref):
    assert np.array_equal(res.offsets, ref.offsets), "neighbour counts differ"
    assert np.array_equal(res.ids, ref.ids), "neighbour ids differ"


@pytest.mark.parametrize("tile", [128, 256, 512, 1024])
@pytest.mark.parametrize("d,N,B", [(1000, 5000, 200), (512, 3000, 130), (64, 700, 129),
                                   (1000, 5000, 300)])
def test_dense_scores_against_fp64(gt, d, N, B, tile):
    ds = synth.generate(synth.Workload("t", N, d, B, (0.9,), "uniform:5", seed=d + N),
                        screen=False)
    t = gt.Tree(ds.F)
    t.set_tuning("bf16", tile=tile)
    qhat = bf16_value(bf16_rn(ds.Q))
    for h in sorted({0, 1, 3, t.levels - 1}):
        S = t.dense_scores(ds.Q, h)
        yhat = bf16_value(t.read_rows(h, "bf16"))
        ref = qhat @ yhat.T                     # exact products of the BF16 operands
        assert S.shape == ref.shape
        err = np.abs(S - ref)
        assert np.all(err <= GAMMA_TC * ref + 1e-30), f"level {h}: max rel {np.max(err / ref)}"
        # the bound the pruning uses holds against the exact FP64 pool score
        exact = ds.Q.astype(np.float64) @ oracle.pools_fp64(ds.F, h).T
        eh = h * 2.0 ** -24
        cu = (1 + GAMMA_TC) / ((1 - U_BF16) ** 2 * (1 - eh))
        cl = 1 / ((1 + GAMMA_TC) * (1 + U_BF16) ** 2)
        assert np.all(exact <= S * cu * (1 + 2e-6))
        if h == 0:
            assert np.all(exact >= S * cl * (1 - 2e-6))
    t.close()


@pytest.mark.parametrize("tile", [256, 1024])
def test_dense_scores_adversarial(gt, tile):
    # near-one-hot and flat vectors, many equal products: accumulation order
    d = 1024
    rng = np.random.default_rng(4)
    F = np.full((600, d), 1.0 / np.sqrt(d), dtype=np.float32)
    F[:300] = np.exp(-20 * rng.random((300, d))).astype(np.float32)
    F /= np.linalg.norm(F.astype(np.float64), axis=1, keepdims=True).astype(np.float32)
    Q = np.concatenate([F[:64], np.full((64, d), 1.0 / np.sqrt(d), np.float32)])
    t = gt.Tree(F)
    t.set_tuning("bf16", tile=tile)
    S = t.dense_scores(Q, 0)
    ref = bf16_value(bf16_rn(Q)) @ bf16_value(bf16_rn(F)).T
    assert np.all(np.abs(S - ref) <= GAMMA_TC * ref + 1e-30)
    t.close()


@pytest.mark.parametrize("rho", [0.8, 0.9, 0.95])
def test_cutover_parity(gt, rho):
    ds = synth.generate(synth.Workload("t", 40_000, 1000, 300, (rho,), "uniform:20",
                                       seed=int(rho * 100)))
    r = ds.rho_for(rho)
    ref = oracle.brute_force(ds.F, ds.Q, r)
    assert ref.ambiguous.sum() == 0
    t = gt.Tree(ds.F)
    L = t.levels - 1
    t.set_tuning("bf16", tile={0.8: 128, 0.9: 1024, 0.95: 512}[rho], inflight=10)
    for cut in (1, 4, 9, L):
        for dtype in ("bf16", "fp8", "f32"):
            res = t.query(ds.Q, r, dtype=dtype, cutover=cut)
            same_sets(res, ref)
            assert res.stats["cutover"] == cut
            assert res.stats["dense_tests"] == ds.Q.shape[0] * ((40_000 + (1 << cut) - 1) >> cut)
    same_sets(t.query(ds.Q, r, dtype="bf16"), ref)            # automatic cutover
    same_sets(t.exhaustive(ds.Q, r), ref)
    t.close()


def test_exhaustive_parity_and_rechecks(gt, small_ds):
    ds = small_ds
    r = ds.rho_for(0.9)
    ref = oracle.brute_force(ds.F, ds.Q, r)
    t = gt.Tree(ds.F)
    res = t.exhaustive(ds.Q, r)
    same_sets(res, ref)
    # near-threshold items are decided by the FP64 recheck
    rho = np.float32(0.8)
    x = np.array([rho + 2e-5, rho - 2e-5] * 40 + [0.1] * 100, dtype=np.float32)
    d = 16
    F = np.zeros((x.size, d), np.float32)
    F[:, 0] = x
    F[:, 1] = np.sqrt(1 - x.astype(np.float64) ** 2).astype(np.float32)
    q = np.zeros((1, d), np.float32)
    q[0, 0] = 1.0
    t2 = gt.Tree(F)
    res = t2.exhaustive(q, rho)
    same_sets(res, oracle.brute_force(F, q, rho))
    assert res.stats["rechecks"] >= 80
    for cut in range(1, t2.levels):
        same_sets(t2.query(q, rho, cutover=cut), oracle.brute_force(F, q, rho))
    t.close()
    t2.close()


def test_exhaustive_over_raw_database(gt, small_ds):
    """gt_exhaustive(F, N, d, Q, B, rho): the Exh comparator (Sec. 4) over the
    caller's rows, no tree: equal to the FP64 definition element by element."""
    ds = small_ds
    r = ds.rho_for(0.9)
    ref = oracle.brute_force(ds.F, ds.Q, r)
    assert ref.ambiguous.sum() == 0
    N, B = ds.F.shape[0], ds.Q.shape[0]
    Fd = torch.from_numpy(ds.F).cuda()
    Fp = torch.from_numpy(ds.F).pin_memory()
    # pageable host rows, device rows, page-locked host rows; device queries
    for F, Q in ((ds.F, ds.Q), (Fd, ds.Q), (Fp, torch.from_numpy(ds.Q).cuda()), (ds.F, ds.Q)):
        res = gt.exhaustive(F, Q, r)
        same_sets(res, ref)
        assert res.stats["dense_tests"] == N * B and res.stats["gathered_tests"] == 0
    res = gt.exhaustive(Fd, ds.Q, r, results_on_device=True, max_batch=37)
    assert res.on_device and res.stats["micro_batches"] == 3
    res.free()
    # a smaller database after a larger one (storage kept), then another width
    sub = np.ascontiguousarray(ds.F[:777])
    same_sets(gt.exhaustive(sub, ds.Q, r), oracle.brute_force(sub, ds.Q, r))
    small = synth.generate(synth.Workload("t", 3000, 64, 129, (0.9,), "uniform:5", seed=64),
                           screen=True)
    r64 = small.rho_for(0.9)
    same_sets(gt.exhaustive(small.F, small.Q, r64), oracle.brute_force(small.F, small.Q, r64))
    # rho given per query, one threshold differing
    r2 = r.copy()
    r2[::2] = np.float32(0.95)
    ref2 = oracle.brute_force(ds.F, ds.Q, r2)
    if ref2.ambiguous.sum() == 0:
        same_sets(gt.exhaustive(ds.F, ds.Q, r2), ref2)
    # a negative entry in F is refused, and the context still works afterwards
    bad = ds.F[:100].copy()
    bad[7, 3] = -1e-3
    with pytest.raises(gt.GTError) as e:
        gt.exhaustive(bad, ds.Q, r)
    assert e.value.status == 2
    same_sets(gt.exhaustive(ds.F, ds.Q, r), ref)


def test_exhaustive_raw_near_threshold_rechecks(gt):
    # items within 2e-5 of rho: every one settled by the FP64 recheck
    rho = np.float32(0.8)
    x = np.array([rho + 2e-5, rho - 2e-5] * 40 + [0.1] * 100, dtype=np.float32)
    d = 16
    F = np.zeros((x.size, d), np.float32)
    F[:, 0] = x
    F[:, 1] = np.sqrt(1 - x.astype(np.float64) ** 2).astype(np.float32)
    q = np.zeros((1, d), np.float32)
    q[0, 0] = 1.0
    res = gt.exhaustive(F, q, rho)
    same_sets(res, oracle.brute_force(F, q, rho))
    assert res.stats["rechecks"] >= 80 and res.stats["results"] == 40


def test_cutover_with_micro_batches(gt, small_ds):
    ds = small_ds
    r = ds.rho_for(0.9)
    ref = oracle.brute_force(ds.F, ds.Q, r)
    t = gt.Tree(ds.F)
    res = t.query(ds.Q, r, dtype="bf16", cutover=6, max_batch=33)
    same_sets(res, ref)
    assert res.stats["micro_batches"] == 4
    res = t.exhaustive(ds.Q, r, max_batch=50, scratch_bytes=1 << 16)
    same_sets(res, ref)
    t.close()


def test_autotune_choice_is_used_and_exact(gt, small_ds):
    ds = small_ds
    r = ds.rho_for(0.9)
    ref = oracle.brute_force(ds.F, ds.Q, r)
    t = gt.Tree(ds.F)
    for dtype in ("bf16", "fp8"):
        tune = t.autotune(ds.Q, r, dtype=dtype)
        assert 1 <= tune["cutover"] <= min(8, t.levels - 1) and tune["inflight"] in (0, 1, 2, 4, 9, 10, 12, 16, 32)
        assert tune["tile_n"] in (128, 256, 512, 1024)
        assert abs(tune["best_ms"] - min(tune["ms"].values())) < 1e-6
        res = t.query(ds.Q, r, dtype=dtype)               # automatic cutover = tuned
        assert res.stats["cutover"] == tune["cutover"]
        same_sets(res, ref)
    t.close()


def test_graph_capture_and_replay(gt, small_ds):
    ds = small_ds
    r = ds.rho_for(0.9)
    ref = oracle.brute_force(ds.F, ds.Q, r)
    t = gt.Tree(ds.F)
    Qd = torch.from_numpy(ds.Q).cuda()
    rd = torch.from_numpy(r).cuda()
    s = torch.cuda.Stream()
    for stream in (None, s):                       # legacy default stream and a user stream
        a = t.query(Qd, rd, dtype="bf16", cutover=3, stream=stream, timing=True)
        b = t.query(Qd, rd, dtype="bf16", cutover=3, stream=stream, timing=True)
        c = t.query(Qd, rd, dtype="bf16", cutover=3, stream=stream, graph=False)
        assert a.stats["graph_captures"] + a.stats["graph_replays"] == a.stats["micro_batches"]
        assert b.stats["graph_replays"] == b.stats["micro_batches"]
        assert c.stats["graph_captures"] == 0 and c.stats["graph_replays"] == 0
        for res in (a, b, c):
            same_sets(res, ref)
        assert b.stats["kernel_ms"]["dense"] > 0 and b.stats["kernel_ms"]["leaf"] > 0
    t.close()


@pytest.mark.parametrize("rho", [0.8, 0.9])
def test_subtraction_path_parity(gt, rho):
    # N not a power of two: some pools lack a right child
    ds = synth.generate(synth.Workload("t", 37_771, 1000, 200, (rho,), "uniform:20",
                                       seed=int(rho * 1000) + 3))
    r = ds.rho_for(rho)
    ref = oracle.brute_force(ds.F, ds.Q, r)
    t = gt.Tree(ds.F)
    t.set_tuning("bf16", tile=1024 if rho == 0.9 else 256)
    for cut in (2, 3, 5, 8):
        for dtype in ("bf16", "fp8", "f32"):
            sub = t.query(ds.Q, r, dtype=dtype, cutover=cut, subtract=1)
            same_sets(sub, ref)
            direct = t.query(ds.Q, r, dtype=dtype, cutover=cut, subtract=-1)
            same_sets(direct, ref)
            # the subtraction path gathers one child per surviving pool
            lv_s, lv_d = sub.stats["level_tests"], direct.stats["level_tests"]
            above = sum(lv_s[1:cut])
            assert above <= 0.75 * sum(lv_d[1:cut]) + 16
            # and at the items: a left item is gathered only when its upper
            # bound (the pool's minus its right sibling's) reaches rho and its
            # lower bound does not, so with BF16 or FP32 rows most left
            # neighbours are accepted without their rows
            frac = 0.9 if dtype == "fp8" else 0.7
            assert lv_s[0] <= frac * lv_d[0] + 16, (dtype, cut, lv_s[0], lv_d[0])
    t.close()


def test_subtraction_path_tiny_trees(gt):
    rng = np.random.default_rng(12)
    for N in (5, 7, 9, 17, 33, 100):
        d = 32
        F = np.exp(3 * rng.standard_normal((N, d)))
        F /= np.linalg.norm(F, axis=1, keepdims=True)
        F = F.astype(np.float32)
        Q = F[rng.integers(0, N, 5)] * np.exp(0.1 * rng.standard_normal((5, d)))
        Q = (Q / np.linalg.norm(Q, axis=1, keepdims=True)).astype(np.float32)
        t = gt.Tree(F)
        for cut in range(2, t.levels):
            for rho in (0.3, 0.8):
                same_sets(t.query(Q, rho, cutover=cut, subtract=1),
                          oracle.brute_force(F, Q, rho, margin=0.0))
        t.close()


@pytest.mark.parametrize("rho", [0.8, 0.9])
def test_ring_gather_parity(gt, rho):
    # rows fed through the shared-memory ring (tests-in-flight code 16), on
    # every level kernel: frontier, leaves, subtraction, root-down traversal
    ds = synth.generate(synth.Workload("t", 29_999, 1000, 150, (rho,), "uniform:20",
                                       seed=int(rho * 1000) + 11))
    r = ds.rho_for(rho)
    ref = oracle.brute_force(ds.F, ds.Q, r)
    t = gt.Tree(ds.F)
    for dtype in ("bf16", "fp8", "f32"):
        t.set_tuning(dtype, inflight=16)
        for cut, sub in ((-2, -1), (2, 1), (3, -1), (3, 1), (6, 1)):
            res = t.query(ds.Q, r, dtype=dtype, cutover=cut, subtract=sub)
            same_sets(res, ref)
        # micro-batches and a frontier budget that forces retries
        res = t.query(ds.Q, r, dtype=dtype, cutover=3, max_batch=37, scratch_bytes=1 << 20)
        same_sets(res, ref)
    t.close()


def test_ring_gather_tiny_lists(gt):
    # lists shorter than one block's chunk, and a single query
    ds = synth.generate(synth.Workload("t", 3_001, 64, 9, (0.9,), "uniform:3", seed=5))
    r = ds.rho_for(0.9)
    ref = oracle.brute_force(ds.F, ds.Q, r)
    t = gt.Tree(ds.F)
    for dtype in ("bf16", "fp8", "f32"):
        t.set_tuning(dtype, inflight=16)
        same_sets(t.query(ds.Q, r, dtype=dtype, cutover=-2), ref)
        same_sets(t.query(ds.Q, r, dtype=dtype, cutover=2, subtract=1), ref)
        one = t.query(ds.Q[:1], r[:1], dtype=dtype, cutover=-2)
        assert np.array_equal(one.neighbours(0), ref.neighbours(0))
    t.close()


@pytest.mark.parametrize("d", [16, 100, 513, 600, 800, 1000, 1024, 1040])
def test_ring_gather_widths(gt, d):
    # the ring-fed gather over row widths: rows of one to eight 16-byte
    # vectors per lane, the widest narrow rows (1024) and the first wide ones
    # (1040), and BF16 rows whose ring depth is odd (600, 800: 7 and 5 slots
    # per warp); frontier, leaves, subtraction levels and items, and retries
    ds = synth.generate(synth.Workload("t", 12_000, d, 90, (0.85,), "uniform:8", seed=d))
    r = ds.rho_for(0.85)
    ref = oracle.brute_force(ds.F, ds.Q, r)
    t = gt.Tree(ds.F)
    for dtype in ("bf16", "fp8", "f32"):
        t.set_tuning(dtype, inflight=16)
        for cut, sub in ((-2, -1), (2, 1), (3, -1), (3, 1), (5, 1)):
            same_sets(t.query(ds.Q, r, dtype=dtype, cutover=cut, subtract=sub), ref)
    same_sets(t.query(ds.Q, r, dtype="bf16", cutover=3, max_batch=7, scratch_bytes=1 << 19), ref)
    t.close()
    if d in (600, 800, 1000):
        # the prefix layout's splits take the same ring
        tp = gt.Tree(ds.F, layout="prefix", prefix_level=3)
        same_sets(tp.query(ds.Q, r, dtype="bf16"), ref)
        tp.close()


@pytest.mark.parametrize("inflight", [0, 4, 16])
def test_gather_thresholds_at_scores(gt, inflight):
    # every query's threshold is an item's exact score rounded to FP32, or
    # one FP32 step either side: the item sits inside every low-precision
    # bound, so only the FP32 refine and the FP64 recheck may decide it; the
    # sets must still be exact (default kernels, registers, ring)
    ds = synth.generate(synth.Workload("t", 20_000, 1000, 120, (0.9,), "uniform:10", seed=77),
                        screen=False)
    S = ds.Q.astype(np.float64) @ ds.F.astype(np.float64).T
    rng = np.random.default_rng(5)
    rho = np.empty(ds.Q.shape[0], dtype=np.float32)
    for q in range(ds.Q.shape[0]):
        top = np.argsort(-S[q])[:40]
        v = np.float32(S[q, top[rng.integers(0, 40)]])
        rho[q] = [np.nextafter(v, np.float32(0)), v, np.nextafter(v, np.float32(2))][q % 3]
    rho = np.clip(rho, np.float32(1e-3), np.float32(1.0))
    ref = oracle.brute_force(ds.F, ds.Q, rho, margin=0.0)
    t = gt.Tree(ds.F)
    for dtype in ("bf16", "fp8", "f32"):
        t.set_tuning(dtype, inflight=inflight)
        for cut, sub in ((-2, -1), (3, 1), (3, -1)):
            same_sets(t.query(ds.Q, rho, dtype=dtype, cutover=cut, subtract=sub), ref)
    t.close()


def test_graph_cache_eviction_with_timing(gt, small_ds):
    # more micro-batches in one call than the graph cache holds: graphs are
    # evicted while the call's timer still reads their events
    ds = small_ds
    r = ds.rho_for(0.9)
    Q = np.concatenate([ds.Q, ds.Q, ds.Q])[:300]
    rr = np.concatenate([r, r, r])[:300]
    ref = oracle.brute_force(ds.F, Q, rr)
    t = gt.Tree(ds.F)
    for _ in range(2):
        res = t.query(Q, rr, dtype="bf16", cutover=3, max_batch=4, timing=True)
        assert res.stats["micro_batches"] == 75
        assert res.stats["graph_captures"] + res.stats["graph_replays"] == 75
        assert res.stats["kernel_ms"]["dense"] > 0
        same_sets(res, ref)
    t.close()
