"""One persistent launch for every level below the cutover (k_drain, tests
in flight code 32): its warps drain the dense GEMM's list as a shared work
queue, each carrying the entries it claims down to the items.  Its answers
must equal the FP64 definition, and its per-level test counts those of the
per-level launches (the same tests, the same arithmetic)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

DRAIN, RING = 32, 16


@pytest.fixture(scope="module")
def gt():
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device: the GPU tests need a GB300")
    from paper_2311_02573_gb300 import gt as g
    g.load()
    return g


@pytest.fixture(scope="module")
def ds40k():
    return synth.generate(synth.Workload("t", 40_001, 1000, 300, (0.8,), "uniform:20", seed=77))


def same_sets(res, ref):
    assert np.array_equal(res.offsets, ref.offsets), "neighbour counts differ"
    assert np.array_equal(res.ids, ref.ids), "neighbour ids differ"


@pytest.mark.parametrize("dtype", ["f32", "bf16", "fp8"])
def test_drain_equals_definition_and_level_launches(gt, ds40k, dtype):
    ds = ds40k
    r = ds.rho_for(0.8)
    ref = oracle.brute_force(ds.F, ds.Q, r)
    assert ref.ambiguous.sum() == 0
    t = gt.Tree(ds.F)
    for cut in (2, 3, 4, 5):
        t.set_tuning(dtype, inflight=DRAIN)
        a = t.query(ds.Q, r, dtype=dtype, cutover=cut, subtract=1)
        same_sets(a, ref)
        t.set_tuning(dtype, inflight=RING)
        b = t.query(ds.Q, r, dtype=dtype, cutover=cut, subtract=1)
        same_sets(b, ref)
        assert a.stats["level_tests"] == b.stats["level_tests"], f"cutover {cut}"
        assert a.stats["rechecks"] == b.stats["rechecks"]
        assert a.stats["refines"] == b.stats["refines"]
        # one launch for the levels and the items instead of one per level,
        # the items and the left items
        assert a.stats["level_launches"] == 1 and a.stats["launches"] < b.stats["launches"]
    t.close()


def test_drain_small_and_ragged_trees(gt):
    # N from a handful of items to a few tiles, with odd tails at every level
    for N in (5, 17, 64, 65, 999, 4097):
        B = max(2, min(40, N // 8))
        ds = synth.generate(synth.Workload("t", N, 128, B, (0.9,), "uniform:1", seed=N))
        r = ds.rho_for(0.9)
        ref = oracle.brute_force(ds.F, ds.Q, r)
        assert ref.ambiguous.sum() == 0
        t = gt.Tree(ds.F)
        t.set_tuning("bf16", inflight=DRAIN)
        for cut in range(2, min(5, t.levels - 1) + 1):
            same_sets(t.query(ds.Q, r, dtype="bf16", cutover=cut, subtract=1), ref)
        t.close()


def test_drain_micro_batches_graphs_and_timeout(gt, ds40k):
    ds = ds40k
    r = ds.rho_for(0.8)
    ref = oracle.brute_force(ds.F, ds.Q, r)
    t = gt.Tree(ds.F)
    t.set_tuning("bf16", inflight=DRAIN)
    res = t.query(ds.Q, r, dtype="bf16", cutover=3, subtract=1, max_batch=70)
    same_sets(res, ref)
    assert res.stats["micro_batches"] == 5
    for _ in range(2):                        # captured once, then replayed
        res = t.query(ds.Q, r, dtype="bf16", cutover=3, subtract=1)
        same_sets(res, ref)
    assert res.stats["graph_replays"] >= 1
    t.set_wait_expiry(True)
    with pytest.raises(gt.GTError) as e:
        t.query(ds.Q, r, dtype="bf16", cutover=3, subtract=1)
    assert e.value.status == 5
    t.set_wait_expiry(False)
    same_sets(t.query(ds.Q, r, dtype="bf16", cutover=3, subtract=1), ref)
    t.close()


def test_drain_with_inserts_and_per_query_rho(gt):
    ds = synth.generate("softmax_n1m_d512_served", n_queries=200, N=30_000)
    t = gt.Tree(ds.F[:20_000], capacity=24_000)
    t.insert(ds.F[20_000:])                  # grows the storage
    t.set_tuning("bf16", inflight=DRAIN)
    ref = oracle.brute_force(ds.F, ds.Q, ds.rho)
    assert ref.ambiguous.sum() == 0
    for dtype in ("bf16", "fp8"):
        t.set_tuning(dtype, inflight=DRAIN)
        same_sets(t.query(ds.Q, ds.rho, dtype=dtype, cutover=3, subtract=1), ref)
    t.close()
