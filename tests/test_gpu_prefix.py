"""The prefix-sum layout (Eq. 1, cumulative sums restarted per block of 2^c
items): its stored rows against the oracle's FP64 block sums, and its query
path against the FP64 brute force."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def gt():
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device: the GPU tests need a GB300")
    from paper_2311_02573_gb300 import gt as g
    g.load()
    return g


def same_sets(res, ref):
    assert np.array_equal(res.offsets, ref.offsets), "neighbour counts differ"
    assert np.array_equal(res.ids, ref.ids), "neighbour ids differ"


def bf16_rn(x):
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return ((b + 0x7FFF + ((b >> 16) & 1)) >> 16).astype(np.uint16)


def block_ends(n, c):
    return np.minimum(np.arange(0, n, 1 << c) + (1 << c), n) - 1


@pytest.mark.parametrize("c", [1, 3, 5])
def test_prefix_rows_match_oracle(gt, small_ds, c):
    # N = 5003: the last block is partial.  The rows are FP64 sums in item
    # order rounded once to FP32 (BF16: round to nearest of that FP32 value),
    # so they equal the oracle's sums rounded the same way, bit for bit
    F = small_ds.F[:5003]
    t = gt.Tree(F, layout="prefix", prefix_level=c, formats=("bf16", "f32"))
    P = oracle.block_prefix_fp64(F, c).astype(np.float32)
    assert np.array_equal(t.read_rows(0, "f32"), F)
    assert np.array_equal(t.read_rows(-1, "f32"), P)
    assert np.array_equal(t.read_rows(-1, "bf16"), bf16_rn(P))
    assert np.array_equal(t.read_rows(c, "bf16"), bf16_rn(P[block_ends(F.shape[0], c)]))
    t.close()


@pytest.mark.parametrize("rho", [0.8, 0.9])
def test_prefix_query_parity(gt, rho):
    ds = synth.generate(synth.Workload("t", 30_001, 1000, 150, (rho,), "uniform:20",
                                       seed=int(rho * 100) + 77))
    r = ds.rho_for(rho)
    ref = oracle.brute_force(ds.F, ds.Q, r)
    assert ref.ambiguous.sum() == 0
    for c in (2, 3, 5):
        t = gt.Tree(ds.F, layout="prefix", prefix_level=c, formats=("bf16", "f32"))
        for dtype in ("bf16", "f32"):
            res = t.query(ds.Q, r, dtype=dtype)
            same_sets(res, ref)
            assert res.stats["cutover"] == c
            same_sets(t.query(ds.Q, r, dtype=dtype, cutover=c, graph=False), ref)
        # several micro-batches
        same_sets(t.query(ds.Q, r, dtype="bf16", max_batch=37), ref)
        t.close()


@pytest.mark.parametrize("N", [1, 2, 3, 7, 8, 9, 1000, 4097])
def test_prefix_small_and_ragged(gt, small_ds, N):
    ds = small_ds
    rho = ds.rho_for(0.8)
    F = ds.F[:N]
    ref = oracle.brute_force(F, ds.Q, rho)
    assert ref.ambiguous.sum() == 0
    for c in (1, 3):
        t = gt.Tree(F, layout="prefix", prefix_level=c)
        same_sets(t.query(ds.Q, rho, dtype="bf16"), ref)
        t.close()


def test_prefix_narrow_rows(gt):
    # d = 100 and d = 64: row widths below one 128-column chunk of the ring
    for d in (64, 100):
        ds = synth.generate(synth.Workload("t", 7_000, d, 64, (0.9,), "uniform:10", seed=d))
        r = ds.rho_for(0.9)
        ref = oracle.brute_force(ds.F, ds.Q, r)
        assert ref.ambiguous.sum() == 0
        t = gt.Tree(ds.F, layout="prefix", prefix_level=4, formats=("bf16", "f32"))
        for dtype in ("bf16", "f32"):
            same_sets(t.query(ds.Q, r, dtype=dtype), ref)
        t.close()


@pytest.mark.parametrize("dtype", ["bf16", "f32"])
def test_prefix_counts_bracket_exact_pools(gt, small_ds, dtype):
    # N = 2^14, c = 5: the GPU keeps every pool whose exact score reaches rho
    # (soundness) and none below rho by more than the bounds' slack, which is
    # under 2^-6 of the block's score for both row formats
    ds = small_ds
    F = ds.F[:16384]
    c = 5
    rho = ds.rho_for(0.9)
    t = gt.Tree(F, layout="prefix", prefix_level=c, formats=("bf16", "f32"))
    res = t.query(ds.Q, rho, dtype=dtype)
    same_sets(res, oracle.brute_force(F, ds.Q, rho))
    lv = res.stats["level_tests"]
    Qd = ds.Q.astype(np.float64)
    S_block = oracle.pools_fp64(F, c) @ Qd.T          # blocks x queries
    for l in range(1, c + 1):
        S = oracle.pools_fp64(F, l) @ Qd.T             # level-l pools x queries
        blk = S_block[np.arange(S.shape[0]) >> (c - l)]
        exact = int((S >= rho[None, :]).sum())
        slack = int((S >= rho[None, :] - 2.0 ** -6 * blk).sum())
        # slot l-1 holds the kept level-l pools (each split by one gather)
        assert exact <= lv[l - 1] <= slack, (l, exact, lv[l - 1], slack)
    t.close()


def test_prefix_inserts_match_build(gt, small_ds):
    ds = small_ds
    F = ds.F[:5001]
    full = gt.Tree(F, layout="prefix", prefix_level=3, formats=("bf16", "f32"))
    t = gt.Tree(F[:3000], capacity=3500, layout="prefix", prefix_level=3, formats=("bf16", "f32"))
    t.insert(F[3000:3001])   # inside the last partial block
    t.insert(F[3001:3003])
    t.insert(F[3003:])       # past the capacity: the storage grows
    assert t.size == 5001
    assert np.array_equal(t.read_rows(0, "f32"), full.read_rows(0, "f32"))
    for dt in ("f32", "bf16"):
        assert np.array_equal(t.read_rows(-1, dt), full.read_rows(-1, dt))
    assert np.array_equal(t.read_rows(3, "bf16"), full.read_rows(3, "bf16"))
    rho = ds.rho_for(0.8)
    same_sets(t.query(ds.Q, rho, dtype="bf16"), oracle.brute_force(F, ds.Q, rho))
    t.close()
    full.close()


def test_prefix_refusals(gt, small_ds):
    F = small_ds.F[:2048]
    Q, rho = small_ds.Q[:8], small_ds.rho_for(0.8)[:8]
    with pytest.raises(gt.GTError):
        gt.Tree(F, layout="prefix", formats=("bf16", "fp8"))
    with pytest.raises(gt.GTError):
        gt.Tree(F, layout="prefix", pooling="max")
    with pytest.raises(gt.GTError):
        gt.Tree(F, layout="prefix", prefix_level=13)
    t = gt.Tree(F, layout="prefix", prefix_level=3)   # BF16 prefix rows only
    with pytest.raises(gt.GTError):
        t.query(Q, rho, dtype="f32")
    with pytest.raises(gt.GTError):
        t.query(Q, rho, dtype="fp8")
    with pytest.raises(gt.GTError):
        t.query(Q, rho, dtype="bf16", cutover=4)
    with pytest.raises(gt.GTError):
        t.exhaustive(Q, rho)
    with pytest.raises(gt.GTError):
        gt.Server(t, cutover=4)                       # its dense level is prefix_level
    with pytest.raises(gt.GTError):
        t.set_tuning("bf16", inflight=2)              # splits always use the ring
    with pytest.raises(gt.GTError):
        t.pair_bounds(0, "bf16", Q, np.zeros((1, 2), dtype=np.int32))
    with pytest.raises(gt.GTError):
        t.read_rows(1, "bf16")
    Qd = torch.from_numpy(Q).cuda()
    rd = torch.from_numpy(rho).cuda()
    off = torch.zeros(9, dtype=torch.int64, device="cuda")
    ids = torch.zeros(64, dtype=torch.int32, device="cuda")
    with pytest.raises(gt.GTError):
        t.query_static(Qd, rd, off, ids)
    # the tree stays usable after the refusals
    same_sets(t.query(Q, rho, dtype="bf16"), oracle.brute_force(F, Q, rho))
    t.close()


def test_prefix_autotune_picks_a_tile(gt, small_ds):
    ds = small_ds
    F = ds.F[:12_000]
    rho = ds.rho_for(0.9)
    ref = oracle.brute_force(F, ds.Q, rho)
    assert ref.ambiguous.sum() == 0
    t = gt.Tree(F, layout="prefix", prefix_level=3)
    tune = t.autotune(ds.Q, rho)
    assert tune["cutover"] == 3 and tune["subtract"] == 0
    assert tune["tile_n"] in (128, 256, 512, 1024)
    assert abs(tune["best_ms"] - min(v for k, v in tune["ms"].items() if k.startswith("tile"))) < 1e-6
    res = t.query(ds.Q, rho, dtype="bf16")
    same_sets(res, ref)
    for tile in (128, 512, 1024):
        t.set_tuning("bf16", tile=tile)
        same_sets(t.query(ds.Q, rho, dtype="bf16"), ref)
    t.close()
