"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Neighbour sets must be identical (same ids, same counts) for every query in
every row format; the generator's 1e-5 margin makes the exact answer unique.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _require_gpu():
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device: the GPU tests need a GB300")


@pytest.fixture(scope="module")
def gt():
    _require_gpu()
    from paper_2311_02573_gb300 import gt as g
    g.load()
    return g


def same_sets(res, ref, B=None):
    B = len(ref.offsets) - 1 if B is None else B
    assert np.array_equal(res.offsets, ref.offsets), "neighbour counts differ"
    assert np.array_equal(res.ids, ref.ids), "neighbour ids differ"


def bf16_rn(x):
    """float32 -> bfloat16 bits, round to nearest even (finite inputs)."""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return ((b + 0x7FFF + ((b >> 16) & 1)) >> 16).astype(np.uint16)


def e4m3_value(codes):
    c = codes.astype(np.int32)
    e = (c >> 3) & 0xF
    m = c & 7
    sign = np.where(c >> 7, -1.0, 1.0)
    return sign * np.where(e == 0, m * 2.0 ** -9, (1 + m / 8.0) * 2.0 ** (e - 7.0))


# -- tree build: the pooled rows ----------------------------------------------

def test_tree_invariants(gt, small_ds):
    F = small_ds.F[:5000]
    t = gt.Tree(F)
    N, L = F.shape[0], t.levels - 1
    assert L == int(np.ceil(np.log2(N)))
    prev = t.read_rows(0)
    assert np.array_equal(prev, F)                       # level 0 = the items
    for h in range(1, L + 1):
        cur = t.read_rows(h)
        left = prev[0::2]
        right = prev[1::2]
        expect = left.copy()
        expect[: right.shape[0]] = left[: right.shape[0]] + right   # fl32(l + r)
        assert np.array_equal(cur, expect), f"level {h} is not the pairwise sum"
        exact = oracle.pools_fp64(F, h)
        rel = np.abs(cur - exact) / np.maximum(exact, 1e-30)
        assert rel.max() <= h * 2.0 ** -24 * 1.0001
        # BF16 copy = round-to-nearest of the FP32 row
        assert np.array_equal(t.read_rows(h, "bf16"), bf16_rn(cur))
        # FP8 copy: power-of-two scale, max/scale in (224, 448], error <= 2^-4 x + s 2^-10
        codes, sc = t.read_rows(h, "fp8")
        assert np.all(np.log2(sc) == np.round(np.log2(sc)))
        mx = cur.max(1)
        assert np.all(mx / sc <= 448) and np.all(mx / sc > 224)
        val = e4m3_value(codes) * sc[:, None]
        assert np.all(np.abs(val - cur) <= 2.0 ** -4 * cur + sc[:, None] * 2.0 ** -10)
        prev = cur
    # the root is the sum of all items
    root = t.read_rows(L)[0].astype(np.float64)
    assert np.allclose(root, F.astype(np.float64).sum(0), rtol=L * 2.0 ** -23)
    t.close()


def test_permuted_build_returns_original_ids(gt, small_ds):
    ds = small_ds
    N = 4096
    F = ds.F[:N]
    perm = np.random.default_rng(5).permutation(N)
    t = gt.Tree(F, perm=perm)
    assert np.array_equal(t.read_rows(0), F[perm])
    rho = ds.rho_for(0.9)
    ref = oracle.brute_force(F, ds.Q, rho)
    same_sets(t.query(ds.Q, rho, dtype="bf16", cutover=-2), ref)
    t.close()


# -- queries: exact sets in every format ----------------------------------------

@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
def test_query_parity_small(gt, small_ds, dtype):
    ds = small_ds
    rho = ds.rho_for(0.9)
    ref = oracle.brute_force(ds.F, ds.Q, rho)
    assert ref.ambiguous.sum() == 0
    t = gt.Tree(ds.F)
    res = t.query(ds.Q, rho, dtype=dtype, cutover=-2)
    same_sets(res, ref)
    assert res.stats["results"] == len(ref.ids)
    t.close()


@pytest.mark.parametrize("rho", [0.8, 0.95])
def test_query_parity_other_thresholds(gt, rho):
    ds = synth.generate(synth.WORKLOADS["softmax_n20k_d1000"].__class__(
        "t", 30_000, 1000, 64, (rho,), "uniform:10", seed=77))
    r = ds.rho_for(rho)
    ref = oracle.brute_force(ds.F, ds.Q, r)
    t = gt.Tree(ds.F)
    for dtype in ("f32", "bf16", "fp8"):
        same_sets(t.query(ds.Q, r, dtype=dtype, cutover=-2), ref)
    t.close()


def test_plain_counts_match_algorithm1(gt, small_ds):
    # N = 2^14: the splitting tree of Algorithm 1 and the power-of-two levels
    # coincide, so the level-wise traversal tests 2 (T - 1) + 1 pools where
    # Algorithm 1 makes T tests (one test per split, the left child derived),
    # up to pools whose score lies within the FP32 bound of rho (kept by the GPU)
    ds = small_ds
    F = ds.F[:16384]
    rho = ds.rho_for(0.9)
    a1 = oracle.alg1(F, ds.Q, rho)
    t = gt.Tree(F)
    res = t.query(ds.Q, rho, dtype="f32", cutover=-2)
    same_sets(res, a1)
    expect = int((2 * (a1.tests - 1) + 1).sum())
    got = res.stats["gathered_tests"]
    assert expect <= got <= expect * 1.01 + 8
    # per level: depth k of Algorithm 1 is level L - k; each depth-k test of
    # Algorithm 1 (k >= 1) stands for a pair of level L-k pools
    L = t.levels - 1
    lv = res.stats["level_tests"]
    assert lv[L] == ds.Q.shape[0]
    for k in range(1, L + 1):
        assert lv[L - k] >= 2 * a1.rounds[k]
    t.close()


def test_per_query_rho_served_workload(gt):
    ds = synth.generate("softmax_n1m_d512_served", n_queries=200, N=40_000)
    ref = oracle.brute_force(ds.F, ds.Q, ds.rho)
    t = gt.Tree(ds.F)
    for dtype in ("f32", "bf16", "fp8"):
        same_sets(t.query(ds.Q, ds.rho, dtype=dtype, cutover=-2), ref)
    t.close()


# -- edge cases -----------------------------------------------------------------

def _tiny(N, d=32, B=6, seed=0):
    rng = np.random.default_rng(seed)
    F = np.exp(3 * rng.standard_normal((N, d)))
    F /= np.linalg.norm(F, axis=1, keepdims=True)
    Q = F[rng.integers(0, N, B)] * np.exp(0.1 * rng.standard_normal((B, d)))
    Q /= np.linalg.norm(Q, axis=1, keepdims=True)
    return F.astype(np.float32), Q.astype(np.float32)


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 7, 8, 9, 16, 17, 63, 64, 65])
def test_tiny_enumeration(gt, N):
    F, Q = _tiny(N, seed=N)
    t = gt.Tree(F)
    for rho in (0.3, 0.7, 0.9):
        ref = oracle.brute_force(F, Q, rho, margin=0.0)
        for dtype in ("f32", "bf16", "fp8"):
            same_sets(t.query(Q, rho, dtype=dtype, cutover=-2), ref)
    t.close()


def test_degenerate_inputs(gt):
    d = 64
    # identical items: every pool positive down to the leaves
    f = np.zeros(d, np.float32)
    f[3] = 0.6
    f[9] = 0.8
    F = np.tile(f, (300, 1))
    t = gt.Tree(F)
    res = t.query(f[None], 0.999, dtype="fp8", cutover=-2)
    assert res.ids.tolist() == list(range(300))
    t.close()
    # one-hot items: cosines exactly 0 or 1, rho = 1 keeps only the match
    F = np.eye(d, dtype=np.float32)
    t = gt.Tree(F)
    for dtype in ("f32", "bf16", "fp8"):
        res = t.query(F[[5, 40]], 1.0, dtype=dtype, cutover=-2)
        assert res.neighbours(0).tolist() == [5] and res.neighbours(1).tolist() == [40]
    t.close()


def _two_hot_rows(x, d=16):
    F = np.zeros((x.size, d), np.float32)
    F[:, 0] = x
    F[:, 1] = np.sqrt(1 - x.astype(np.float64) ** 2).astype(np.float32)
    q = np.zeros((1, d), np.float32)
    q[0, 0] = 1.0                   # q.f_i = x_i exactly
    return F, q


def test_adversarial_near_threshold(gt):
    rho = np.float32(0.8)
    # rho +- 2e-5: inside the BF16 / FP8 bounds, outside the FP32 one, so the
    # in-warp FP32 refine settles them
    x = np.array([rho + 2e-5, rho - 2e-5] * 40 + [0.1] * 100, dtype=np.float32)
    F, q = _two_hot_rows(x)
    ref = oracle.brute_force(F, q, rho)
    t = gt.Tree(F)
    for dtype in ("f32", "bf16", "fp8"):
        res = t.query(q, rho, dtype=dtype, cutover=-2)
        same_sets(res, ref)
        if dtype != "f32":
            assert res.stats["refines"] >= 80
    t.close()
    # one FP32 ulp either side of rho (and rho itself): inside every bound, so
    # the FP64 recheck decides them
    up, dn = np.nextafter(rho, np.float32(2)), np.nextafter(rho, np.float32(0))
    x = np.array([up, dn, rho] * 30 + [0.1] * 60, dtype=np.float32)
    F, q = _two_hot_rows(x)
    ref = oracle.brute_force(F, q, rho, margin=0.0)
    assert len(ref.ids) == 60
    t = gt.Tree(F)
    for dtype in ("f32", "bf16", "fp8"):
        res = t.query(q, rho, dtype=dtype, cutover=-2)
        same_sets(res, ref)
        assert res.stats["rechecks"] >= 90
    t.close()


def test_empty_and_dimension_limits(gt):
    F, Q = _tiny(100, d=2048, B=3, seed=9)
    t = gt.Tree(F)
    res = t.query(Q[:0], np.zeros(0, np.float32), dtype="bf16", cutover=-2)
    assert res.offsets.tolist() == [0] and res.ids.size == 0
    same_sets(t.query(Q, 0.5, dtype="bf16", cutover=-2), oracle.brute_force(F, Q, 0.5, margin=0))
    t.close()
    F1, Q1 = _tiny(50, d=1, B=2, seed=1)          # d = 1: every cosine is 1
    t = gt.Tree(F1)
    assert t.query(Q1, 1.0, dtype="f32", cutover=-2).ids.size == 100
    t.close()


def test_stale_query_rows_do_not_leak(gt, small_ds):
    # a rejected batch (an infinite entry) leaves its rows in the query
    # workspace; the dense GEMM's last tile of a smaller batch after it spans
    # those rows, and none of them may reach the traversal
    ds = small_ds
    r = ds.rho_for(0.9)
    t = gt.Tree(ds.F)
    bad = ds.Q[:100].copy()
    bad[60:, :] = np.inf
    with pytest.raises(gt.GTError):
        t.query(bad, r[:100], dtype="bf16", cutover=3)
    ref = oracle.brute_force(ds.F, ds.Q[:50], r[:50])
    for cut, sub in ((3, 1), (3, -1), (0, -1)):
        res = t.query(ds.Q[:50], r[:50], dtype="bf16", cutover=cut, subtract=sub)
        assert np.array_equal(res.offsets, ref.offsets) and np.array_equal(res.ids, ref.ids)
    t.close()


def test_errors_are_reported_not_faulted(gt):
    F, Q = _tiny(64, seed=3)
    bad = F.copy()
    bad[7, 2] = -1e-3
    with pytest.raises(gt.GTError) as e:
        gt.Tree(bad)
    assert e.value.status == 2                                     # GT_EDOMAIN
    bad[7, 2] = np.nan
    with pytest.raises(gt.GTError):
        gt.Tree(bad)
    t = gt.Tree(F)
    with pytest.raises(gt.GTError) as e:
        t.query(Q, 0.0, cutover=-2)
    assert e.value.status == 1                                     # GT_EINVAL
    with pytest.raises(gt.GTError):
        t.query(Q, 1.5, cutover=-2)
    Qb = Q.copy()
    Qb[0, 0] = np.inf
    with pytest.raises(gt.GTError) as e:
        t.query(Qb, 0.5, cutover=-2)
    assert e.value.status == 2
    with pytest.raises(gt.GTError) as e:
        t.insert(bad[5:9])                                         # row 7 holds the NaN
    assert e.value.status == 2
    assert t.size == 64                                            # unchanged
    same_sets(t.query(Q, 0.5, cutover=-2), oracle.brute_force(F, Q, 0.5, margin=0))
    t.close()


def test_host_and_device_inputs_agree(gt, small_ds):
    ds = small_ds
    rho = ds.rho_for(0.9)
    Fd = torch.from_numpy(ds.F).cuda()
    Qd = torch.from_numpy(ds.Q).cuda()
    rd = torch.from_numpy(rho).cuda()
    t = gt.Tree(Fd)
    a = t.query(ds.Q, rho, dtype="bf16", cutover=-2)
    b = t.query(Qd, rd, dtype="bf16", cutover=-2)
    same_sets(a, b)
    c = t.query(Qd, rd, dtype="bf16", cutover=-2, results_on_device=True)
    assert c.on_device
    c.free()
    # page-locked host inputs are read in place by the preparation kernel;
    # pageable ones are staged: both give the device inputs' sets, on the
    # root-down and the dense-cutover paths, and through gt_query_into
    Qp = torch.from_numpy(ds.Q).pin_memory()
    rp = torch.from_numpy(rho).pin_memory()
    ref = oracle.brute_force(ds.F, ds.Q, rho)
    for cut in (-2, 3):
        same_sets(t.query(Qp, rp, dtype="bf16", cutover=cut), ref)
        same_sets(t.query(ds.Q, rho, dtype="bf16", cutover=cut), ref)
        same_sets(t.query(Qp, rho, dtype="bf16", cutover=cut), ref)
    offs = torch.empty(ds.Q.shape[0] + 1, dtype=torch.int64).pin_memory().numpy()
    ids = torch.empty(200_000, dtype=torch.int32).pin_memory().numpy()
    n = t.query_into(Qp, rp, offs, ids)
    assert np.array_equal(offs, ref.offsets) and np.array_equal(ids[:n], ref.ids)
    bad = Qp.clone()
    bad[3, 5] = -1.0
    with pytest.raises(gt.GTError):
        t.query(bad, rp, dtype="bf16")
    t.close()


def test_micro_batches_and_overflow_retries(gt, small_ds):
    ds = small_ds
    rho = ds.rho_for(0.9)
    ref = oracle.brute_force(ds.F, ds.Q, rho)
    t = gt.Tree(ds.F)
    res = t.query(ds.Q, rho, dtype="fp8", cutover=-2, max_batch=7)
    same_sets(res, ref)
    assert res.stats["micro_batches"] == -(-ds.Q.shape[0] // 7)
    # a scratch budget far below one batch's frontier forces split-and-retry
    res = t.query(ds.Q, rho, dtype="bf16", cutover=-2, scratch_bytes=1 << 16, max_batch=100)
    same_sets(res, ref)
    assert res.stats["retries"] >= 1
    t.close()


# -- streaming inserts ------------------------------------------------------------

def test_insert_equals_full_build(gt, small_ds):
    ds = small_ds
    F = ds.F[:6000]
    full = gt.Tree(F)
    t = gt.Tree(F[:3000], capacity=3500)          # forces a storage growth too
    t.insert(F[3000:3001])
    t.insert(F[3001:3100])
    t.insert(torch.from_numpy(F[3100:]).cuda())
    assert t.size == 6000 and t.levels == full.levels
    for h in range(full.levels):
        assert np.array_equal(t.read_rows(h), full.read_rows(h)), f"level {h}"
        assert np.array_equal(t.read_rows(h, "bf16"), full.read_rows(h, "bf16"))
        a, sa = t.read_rows(h, "fp8")
        b, sb = full.read_rows(h, "fp8")
        assert np.array_equal(a, b) and np.array_equal(sa, sb)
    rho = ds.rho_for(0.9)
    ref = oracle.brute_force(F, ds.Q, rho)
    for dtype in ("f32", "bf16", "fp8"):
        same_sets(t.query(ds.Q, rho, dtype=dtype, cutover=-2), ref)
    t.close()
    full.close()


@pytest.mark.parametrize("pooling", ["sum", "max"])
def test_short_appends_equal_full_build(gt, small_ds, pooling):
    # appends of 1 to 8 rows at every parity of the tree size (the short-append
    # path recomputes the levels from rows kept in shared memory): every level
    # stays bitwise equal to a full build of the same rows
    ds = small_ds
    F = ds.F[:3100]
    t = gt.Tree(F[:3000], capacity=3200, pooling=pooling)
    n = 3000
    for m in (1, 1, 2, 3, 1, 5, 8, 2, 7, 4, 1, 6, 3):
        t.insert(F[n:n + m])
        n += m
        if n in (3001, 3004, 3013, 3023, 3044):
            full = gt.Tree(F[:n], pooling=pooling)
            for h in range(full.levels):
                assert np.array_equal(t.read_rows(h), full.read_rows(h)), f"n {n} level {h}"
                assert np.array_equal(t.read_rows(h, "bf16"), full.read_rows(h, "bf16"))
                a, sa = t.read_rows(h, "fp8")
                b, sb = full.read_rows(h, "fp8")
                assert np.array_equal(a, b) and np.array_equal(sa, sb)
            full.close()
    assert n == 3044
    t.close()


def test_insert_crossing_power_of_two(gt):
    F, Q = _tiny(40, d=48, B=8, seed=11)
    t = gt.Tree(F[:8])
    for i in range(8, 40):
        t.insert(F[i:i + 1])
        if i + 1 in (9, 16, 17, 33):
            ref = oracle.brute_force(F[: i + 1], Q, 0.6, margin=0)
            same_sets(t.query(Q, 0.6, dtype="bf16", cutover=-2), ref)
    assert t.levels == 7
    t.close()


def test_long_neighbour_lists_sort_in_global_memory(gt):
    # > 4096 neighbours for one query: the CSR sort leaves shared memory
    d = 32
    rng = np.random.default_rng(21)
    base = np.zeros(d, np.float32)
    base[0] = 1.0
    F = np.tile(base, (9000, 1))
    F[:, 1] = rng.uniform(0.0, 0.05, 9000).astype(np.float32)
    F /= np.linalg.norm(F.astype(np.float64), axis=1, keepdims=True).astype(np.float32)
    F = F[rng.permutation(9000)]
    t = gt.Tree(F)
    q = base[None].copy()
    for dtype in ("f32", "bf16"):
        res = t.query(np.repeat(q, 3, 0), 0.9, dtype=dtype, cutover=-2)
        ref = oracle.brute_force(F, np.repeat(q, 3, 0), 0.9, margin=0.0)
        assert len(ref.neighbours(0)) > 4096
        same_sets(res, ref)
    t.close()


@pytest.mark.parametrize("n_hit", [255, 256, 257, 300, 511, 512, 513, 4096, 4097])
def test_neighbour_list_lengths_at_sort_boundaries(gt, n_hit):
    # lists on both sides of each CSR sort's capacity (256 and 512 ids per
    # warp, 4096 in shared memory), in one call with short lists beside them
    d = 32
    rng = np.random.default_rng(n_hit)
    N = 6000
    F = np.zeros((N, d), np.float32)
    F[:, 2:] = rng.uniform(0.5, 1.0, (N, d - 2)).astype(np.float32)
    hit = rng.choice(N, n_hit, replace=False)
    F[hit, 0] = 50.0                      # these score ~1 against e_0
    F[hit, 2:] = 0.0
    F /= np.linalg.norm(F.astype(np.float64), axis=1, keepdims=True).astype(np.float32)
    Q = np.zeros((3, d), np.float32)
    Q[0, 0] = 1.0                         # n_hit neighbours
    Q[1, 0] = 1.0
    Q[2] = F[hit[0]]                      # an item of the group: the same list
    t = gt.Tree(F)
    for dtype in ("bf16", "f32"):
        res = t.query(Q, 0.9, dtype=dtype, cutover=-2)
        ref = oracle.brute_force(F, Q, 0.9, margin=0.0)
        assert len(ref.neighbours(0)) == n_hit
        same_sets(res, ref)
    t.close()


def test_query_into_caller_buffers(gt, small_ds):
    ds = small_ds
    F = ds.F[:8000]
    rho = ds.rho_for(0.9)
    ref = oracle.brute_force(F, ds.Q, rho)
    t = gt.Tree(F)
    B = ds.Q.shape[0]
    n_ref = len(ref.ids)
    # host (pageable), host (pinned) and device buffers
    for kind in ("numpy", "pinned", "cuda"):
        if kind == "numpy":
            offs, ids = np.empty(B + 1, np.int64), np.empty(n_ref + 7, np.int32)
        elif kind == "pinned":
            offs = torch.empty(B + 1, dtype=torch.int64).pin_memory().numpy()
            ids = torch.empty(n_ref + 7, dtype=torch.int32).pin_memory().numpy()
        else:
            offs = torch.empty(B + 1, dtype=torch.int64, device="cuda")
            ids = torch.empty(n_ref + 7, dtype=torch.int32, device="cuda")
        n = t.query_into(ds.Q, rho, offs, ids, dtype="bf16")
        assert n == n_ref
        o = offs.cpu().numpy() if kind == "cuda" else offs
        i = ids.cpu().numpy() if kind == "cuda" else ids
        assert np.array_equal(o, ref.offsets) and np.array_equal(i[:n], ref.ids)
    # too small an ids buffer: an error, not a partial result
    with pytest.raises(gt.GTError, match="EOVERFLOW"):
        t.query_into(ds.Q, rho, np.empty(B + 1, np.int64), np.empty(max(0, n_ref - 1), np.int32))
    # a buffer of the wrong type is refused rather than copied
    with pytest.raises(TypeError):
        t.query_into(ds.Q, rho, np.empty(B + 1, np.int32), np.empty(n_ref, np.int32))
    t.close()


def test_sm_limit_side_by_side_calls(gt, small_ds):
    # two trees whose calls run on about half of the SMs each, from two host
    # threads on two streams: both answers exact
    import threading
    ds = small_ds
    r = ds.rho_for(0.9)
    ref = oracle.brute_force(ds.F, ds.Q, r)
    trees = [gt.Tree(ds.F), gt.Tree(ds.F)]
    for t_, n in zip(trees, (40, 112)):
        t_.set_sm_limit(n)
        t_.set_tuning("bf16", inflight=16)
    Qd = torch.from_numpy(ds.Q).cuda()
    rd = torch.from_numpy(r).cuda()
    out = [None, None]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]

    def run(i):
        out[i] = trees[i].query(Qd, rd, dtype="bf16", cutover=3, subtract=1, stream=streams[i])

    for _ in range(2):
        ths = [threading.Thread(target=run, args=(i,)) for i in (0, 1)]
        for th in ths:
            th.start()
        for th in ths:
            th.join()
        for res in out:
            same_sets(res, ref)
    trees[0].set_sm_limit(0)                      # all SMs again
    same_sets(trees[0].query(ds.Q, r, dtype="bf16", cutover=3, subtract=1), ref)
    with pytest.raises(gt.GTError):
        trees[0].set_sm_limit(1)
    for t_ in trees:
        t_.close()
