"""Descriptors with negative entries (Sec. 2: pools by element-wise maximum
and minimum): the GPU tree of split rows [max(f, 0), max(-f, 0)] under max
pooling, against the FP64 brute force (the sets) and the oracle's max/min
splitting tree (its rows and its dot-product counts)."""
import numpy as np
import pytest

import oracle
import oracle.signed
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


def workload(N, d, B, seed):
    # a query is its source item plus noise of norm about 0.35: cosine ~0.94
    return synth.signed_workload(N, d, B, noise=0.35 / np.sqrt(d), seed=seed)


def split(X):
    return np.concatenate([np.maximum(X, 0), np.maximum(-X, 0)], axis=1).astype(np.float32)


def test_signed_tree_rows_are_split_max_min_pools(gt):
    # N = 2^11: every GPU pool is a node of the oracle's splitting tree, whose
    # maximum row M and minimum row m give the pool [max(M, 0), max(-m, 0)]
    F, _ = workload(2048, 24, 4, seed=5)
    t = gt.Tree(F, pooling="maxmin")
    assert t.row_width == 48 and t.dim == 24
    prev = t.read_rows(0)
    assert np.array_equal(prev, split(F))
    ix = oracle.signed.MaxMinIndex(F)
    node = {(a, n): k for k, (a, n) in enumerate(zip(ix.first, ix.size))}
    for h in range(1, t.levels):
        cur = t.read_rows(h)
        assert np.array_equal(cur, np.maximum(prev[0::2], prev[1::2])), f"level {h}"
        for j in (0, cur.shape[0] // 2, cur.shape[0] - 1):
            k = node[(j << h, 1 << h)]
            want = np.concatenate([np.maximum(ix.M[k], 0), np.maximum(-ix.m[k], 0)])
            assert np.array_equal(cur[j], want.astype(np.float32)), f"level {h} row {j}"
        prev = cur
    t.close()


@pytest.mark.parametrize("N,d", [(3001, 32), (4096, 100), (20000, 256)])
def test_signed_query_parity(gt, N, d):
    F, Q = workload(N, d, 64, seed=N + d)
    rho = np.full(Q.shape[0], 0.8, dtype=np.float32)
    rho[1::3] = np.float32(0.7)                         # per-query thresholds
    ref = oracle.brute_force(F, Q, rho)
    assert ref.ambiguous.sum() == 0
    assert len(ref.ids) >= Q.shape[0] // 2              # most queries find their source
    t = gt.Tree(F, pooling="maxmin")
    L = t.levels - 1
    for dtype in ("f32", "bf16", "fp8"):
        for cut in sorted({-2, min(3, L), min(6, L)}):
            res = t.query(Q, rho, dtype=dtype, cutover=cut)
            same_sets(res, ref)
            # no item is accepted on a bound: every neighbour came from the
            # signed FP64 recheck
            assert res.stats["rechecks"] >= res.stats["results"]
    Qd, rd = torch.from_numpy(Q).cuda(), torch.from_numpy(rho).cuda()
    same_sets(t.query(Qd, rd, dtype="bf16"), ref)       # automatic cutover, device inputs
    t.close()


def test_signed_counts_match_oracle(gt):
    # N = 2^12, FP32 rows, root down: the GPU tests every node the oracle's
    # max/min splitting tests with the split-row bound U' (up to nodes within
    # the FP32 bound of rho), and rechecks every item whose U' reaches rho
    F, Q = workload(4096, 32, 40, seed=11)
    rho = 0.8
    ids, tests, amb = oracle.signed.maxmin_split(F, Q, rho, split=True)
    assert amb.sum() == 0
    Up = split(Q).astype(np.float64) @ split(F).astype(np.float64).T
    n_exact = int((Up >= rho).sum())        # each costs the oracle one more dot product
    nodes = int(tests.sum()) - n_exact
    t = gt.Tree(F, pooling="maxmin")
    res = t.query(Q, np.float32(rho), dtype="f32", cutover=-2)
    for q in range(Q.shape[0]):
        assert np.array_equal(res.neighbours(q), ids[q])
    assert nodes <= res.stats["gathered_tests"] <= nodes * 1.01 + 8
    assert n_exact <= res.stats["rechecks"] <= n_exact * 1.01 + 8
    t.close()


def test_signed_inserts_static_and_autotune(gt):
    F, Q = workload(5000, 48, 50, seed=21)
    rho = np.float32(0.8)
    ref = oracle.brute_force(F, Q, rho)
    assert ref.ambiguous.sum() == 0
    full = gt.Tree(F, pooling="maxmin")
    t = gt.Tree(F[:2000], capacity=2500, pooling="maxmin")
    t.insert(F[2000:2001])
    t.insert(F[2001:])                                  # grows the storage
    assert t.size == 5000 and t.levels == full.levels
    for h in range(full.levels):
        assert np.array_equal(t.read_rows(h), full.read_rows(h)), f"level {h}"
    for dtype in ("f32", "bf16", "fp8"):
        same_sets(t.query(Q, rho, dtype=dtype, cutover=4), ref)
    # the allocation-free query takes the same path from the root
    Qd = torch.from_numpy(Q).cuda()
    rd = torch.full((Q.shape[0],), float(rho), dtype=torch.float32, device="cuda")
    off = torch.zeros(Q.shape[0] + 1, dtype=torch.int64, device="cuda")
    out = torch.zeros(len(ref.ids) + 8, dtype=torch.int32, device="cuda")
    n = t.query_static(Qd, rd, off, out, dtype="bf16")
    assert n == len(ref.ids)
    assert np.array_equal(off.cpu().numpy(), ref.offsets)
    assert np.array_equal(out[:n].cpu().numpy(), ref.ids)
    tune = t.autotune(Q, rho, dtype="bf16")
    assert tune["subtract"] == 0 and tune["cutover"] >= 1
    same_sets(t.query(Q, rho, dtype="bf16"), ref)
    t.close()
    full.close()


def test_signed_domain_and_refusals(gt):
    F, Q = workload(600, 16, 8, seed=3)
    t = gt.Tree(F, pooling="maxmin")                     # negative entries are fine
    with pytest.raises(gt.GTError) as e:                 # items are decided by a recheck
        t.exhaustive(Q, 0.8)
    assert e.value.status == 1
    with pytest.raises(gt.GTError) as e:                 # so is a cutover at the items
        t.query(Q, 0.8, cutover=0)
    assert e.value.status == 1
    with pytest.raises(gt.GTError) as e:                 # no drain schedule (max pools)
        gt.Server(t, schedule="drain")
    assert e.value.status == 1
    bad = Q.copy()
    bad[2, 5] = np.nan
    with pytest.raises(gt.GTError) as e:
        t.query(bad, 0.8)
    assert e.value.status == 2
    Fb = F.copy()
    Fb[7, 1] = np.inf
    with pytest.raises(gt.GTError) as e:
        gt.Tree(Fb, pooling="maxmin")
    assert e.value.status == 2
    with pytest.raises(gt.GTError) as e:                 # rows are 2d wide: d <= 1024
        gt.Tree(np.zeros((4, 1025), np.float32), pooling="maxmin")
    assert e.value.status == 1
    with pytest.raises(gt.GTError) as e:                 # sum pools still refuse negatives
        gt.Tree(F)
    assert e.value.status == 2
    t.close()


def test_signed_served_exact_with_inserts(gt):
    # the continuous-batching server over split rows: queries and inserts of
    # d entries, one level per step, every answer the exact set over the
    # items present when its group was admitted
    F, Q = workload(6000, 48, 120, seed=31)
    rho = np.full(Q.shape[0], 0.8, dtype=np.float32)
    rho[::4] = np.float32(0.75)
    t = gt.Tree(F[:5000], capacity=5500, pooling="maxmin")
    srv = gt.Server(t, dtype="bf16", max_group=16)
    assert srv.stats()["schedule"] == 1
    done, nxt, ins, step = {}, 0, 5000, 0
    while len(done) < Q.shape[0]:
        if nxt < Q.shape[0]:
            srv.submit(Q[nxt:nxt + 10], rho[nxt:nxt + 10], np.arange(nxt, min(nxt + 10, Q.shape[0])))
            nxt += 10
        if step % 3 == 0 and ins < F.shape[0]:
            srv.insert(F[ins:ins + 100])                 # grows the storage past 5500
            ins += 100
        srv.step()
        for tag, ids, snap in srv.poll():
            done[tag] = (ids, snap)
        step += 1
        assert step < 2000
    srv.close()
    snaps = {}
    for tag, (ids, snap) in done.items():
        snaps.setdefault(snap, []).append(tag)
    assert len(snaps) >= 3
    for snap, tags in snaps.items():
        tags = np.array(sorted(tags))
        ref = oracle.brute_force(F[:snap], Q[tags], rho[tags])
        assert ref.ambiguous.sum() == 0
        for i, tag in enumerate(tags):
            assert np.array_equal(done[tag][0], ref.neighbours(i)), f"query {tag} (N={snap})"
    t.close()
