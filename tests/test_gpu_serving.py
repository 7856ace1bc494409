"""The continuous-batching server: exact answers in the mix, equal to alone."""
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


@pytest.fixture(scope="module")
def stream_ds():
    # per-query rho ~ U[0.8, 0.97]; the last 3000 rows arrive as inserts
    return synth.generate("softmax_n1m_d512_served", n_queries=700, N=43_000)


def _serve(gt, t, ds, n0, dtype, max_group, insert_every, schedule="auto"):
    srv = gt.Server(t, dtype=dtype, max_group=max_group, schedule=schedule)
    B = ds.Q.shape[0]
    rng = np.random.default_rng(3)
    arrivals = np.sort(rng.integers(0, 40, B))          # step at which each query arrives
    nxt, ins, done, step = 0, n0, {}, 0
    while len(done) < B:
        k = np.searchsorted(arrivals, step, side="right")
        if k > nxt:
            srv.submit(ds.Q[nxt:k], ds.rho[nxt:k], np.arange(nxt, k))
            nxt = k
        if insert_every and step % insert_every == 0 and ins < ds.F.shape[0]:
            m = min(250, ds.F.shape[0] - ins)
            srv.insert(ds.F[ins:ins + m])
            ins += m
        srv.step()
        for tag, ids, snap in srv.poll():
            done[tag] = (ids, snap)
        step += 1
        assert step < 10_000
    st = srv.stats()
    srv.close()
    return done, st


@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_served_results_exact_with_inserts(gt, stream_ds, dtype):
    # one level per step: several groups in flight at different levels
    ds = stream_ds
    n0 = 40_000
    t = gt.Tree(ds.F[:n0], capacity=ds.F.shape[0])
    done, st = _serve(gt, t, ds, n0, dtype, max_group=64, insert_every=3, schedule="levels")
    assert st["schedule"] == 1
    assert st["completed"] == ds.Q.shape[0] and st["inserted"] == ds.F.shape[0] - n0
    assert st["steps"] > st["completed"] / 64                # several groups in flight
    by_snap = {}
    for tag, (ids, snap) in done.items():
        by_snap.setdefault(snap, []).append(tag)
    assert len(by_snap) >= 3                                 # inserts landed between groups
    for snap, tags in by_snap.items():
        tags = np.array(sorted(tags))
        ref = oracle.brute_force(ds.F[:snap], ds.Q[tags], ds.rho[tags])
        assert ref.ambiguous.sum() == 0
        for i, tag in enumerate(tags):
            assert np.array_equal(done[tag][0], ref.neighbours(i)), f"query {tag} (N={snap})"
    t.close()


@pytest.mark.parametrize("dtype", ["bf16", "f32"])
def test_prefix_served_results_exact_with_inserts(gt, stream_ds, dtype):
    # the prefix layout (Eq. 1's cumulative sums restarted per block of 8
    # items) behind the same server: GEMM over the blocks' totals, one prefix
    # split per kept pool and step; inserts append items and extend the last
    # block, which leaves every prefix row a group admitted earlier reads as it was
    ds = stream_ds
    n0 = 40_000
    t = gt.Tree(ds.F[:n0], capacity=41_000, layout="prefix", prefix_level=3,
                formats=("bf16", "f32"))
    done, st = _serve(gt, t, ds, n0, dtype, max_group=64, insert_every=3)
    assert t.size == ds.F.shape[0]                           # grown past the capacity
    assert st["completed"] == ds.Q.shape[0] and st["cutover"] == 3
    by_snap = {}
    for tag, (ids, snap) in done.items():
        by_snap.setdefault(snap, []).append(tag)
    assert len(by_snap) >= 3
    for snap, tags in by_snap.items():
        tags = np.array(sorted(tags))
        ref = oracle.brute_force(ds.F[:snap], ds.Q[tags], ds.rho[tags])
        assert ref.ambiguous.sum() == 0
        for i, tag in enumerate(tags):
            assert np.array_equal(done[tag][0], ref.neighbours(i)), f"query {tag} (N={snap})"
    t.close()


def test_prefix_served_equals_alone(gt, stream_ds):
    ds = stream_ds
    n0 = 40_000
    t = gt.Tree(ds.F[:n0], capacity=ds.F.shape[0], layout="prefix", prefix_level=3)
    done, _ = _serve(gt, t, ds, n0, "bf16", max_group=128, insert_every=5)
    t.close()
    rng = np.random.default_rng(11)
    for tag in rng.choice(ds.Q.shape[0], 12, replace=False):
        ids, snap = done[int(tag)]
        alone = gt.Tree(ds.F[:snap], layout="prefix", prefix_level=3)
        res = alone.query(ds.Q[tag:tag + 1], ds.rho[tag:tag + 1], dtype="bf16")
        assert np.array_equal(res.neighbours(0), ids)
        alone.close()


@pytest.mark.parametrize("schedule", ["drain", "immediate"])
@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_drain_server_exact_with_inserts(gt, stream_ds, dtype, schedule):
    # tests in flight code 32: one launch takes a group through every level
    # below the cutover and its items, either the step after its admission
    # (drain: while the step admits the next group) or in the step that
    # admits it (immediate)
    ds = stream_ds
    n0 = 40_000
    t = gt.Tree(ds.F[:n0], capacity=ds.F.shape[0])
    done, st = _serve(gt, t, ds, n0, dtype, max_group=64, insert_every=3, schedule=schedule)
    assert st["schedule"] == {"drain": 2, "immediate": 3}[schedule]
    assert st["completed"] == ds.Q.shape[0] and st["inserted"] == ds.F.shape[0] - n0
    by_snap = {}
    for tag, (ids, snap) in done.items():
        by_snap.setdefault(snap, []).append(tag)
    assert len(by_snap) >= 3
    for snap, tags in by_snap.items():
        tags = np.array(sorted(tags))
        ref = oracle.brute_force(ds.F[:snap], ds.Q[tags], ds.rho[tags])
        assert ref.ambiguous.sum() == 0
        for i, tag in enumerate(tags):
            assert np.array_equal(done[tag][0], ref.neighbours(i)), f"query {tag} (N={snap})"
    # the same tests as the level-by-level server (one group at a time)
    srv_counts = {}
    for code in ("levels", schedule):
        srv = gt.Server(t, dtype=dtype, max_group=4096, schedule=code)
        srv.submit(ds.Q, ds.rho, np.arange(ds.Q.shape[0]))
        got = {}
        for _ in range(100):
            srv.step()
            for tag, ids, snap in srv.poll():
                got[tag] = ids
            if len(got) == ds.Q.shape[0]:
                break
        srv_counts[code] = srv.stats()
        srv.close()
        ref = oracle.brute_force(ds.F, ds.Q, ds.rho)
        for tag in range(ds.Q.shape[0]):
            assert np.array_equal(got[tag], ref.neighbours(tag))
    assert srv_counts[schedule]["gathered_tests"] == srv_counts["levels"]["gathered_tests"]
    assert srv_counts[schedule]["steps"] < srv_counts["levels"]["steps"]
    if schedule == "immediate":
        # the whole queue fits one group: answered by the first step
        assert srv_counts[schedule]["steps"] == 1
    t.close()


def test_insert_into_a_tail_sibling_keeps_the_left_bound(gt):
    # N0 = 3999: the last level-1 row (item 3998) is the right child of a
    # level-2 pool whose left child (items 3996, 3997) holds the query's
    # neighbour 3996.  The level-2 step bounds that pool from its row; then an
    # insert puts a copy of the query (item 3999) into the last level-1 row;
    # the level-1 step must not subtract the grown row's lower bound from the
    # pool's earlier bound (that would prune item 3996's pair).
    rng = np.random.default_rng(17)
    d, n0 = 64, 3999
    F = np.exp(3 * rng.standard_normal((n0 + 1, d)))
    F /= np.linalg.norm(F, axis=1, keepdims=True)
    F = F.astype(np.float32)
    F[n0] = F[3996]                      # the inserted item scores 1 like the neighbour
    q = F[3996:3997].copy()
    rho = np.array([0.9], np.float32)
    ref = oracle.brute_force(F[:n0], q, rho, margin=0.0)
    assert 3996 in ref.neighbours(0)
    t = gt.Tree(F[:n0], capacity=n0 + 16)
    srv = gt.Server(t, dtype="bf16", cutover=3, schedule="levels")
    srv.submit(q, rho, np.array([7]))
    srv.step()                           # admitted: the level-3 GEMM
    srv.step()                           # level 2: right children tested, left ones bounded
    srv.insert(F[n0:n0 + 1])             # applied at the start of the next step
    got = {}
    for _ in range(6):
        srv.step()
        for tag, ids, snap in srv.poll():
            got[tag] = (ids, snap)
    srv.close()
    ids, snap = got[7]
    assert snap == n0
    assert np.array_equal(ids, ref.neighbours(0))
    t.close()


@pytest.mark.parametrize("schedule", ["levels", "drain"])
def test_insert_into_a_tail_pool_gives_no_lower_bound(gt, schedule):
    # N0 = 3999: the last level-1 row holds item 3998 alone and is the right
    # child of a level-2 pool that survives (item 3996 is a copy of the
    # query).  After admission an insert puts another copy of the query
    # (item 3999) into that row.  When the grown row is gathered, its lower
    # bound covers the new item too, so it must not travel as the pool's
    # lower bound: item 3998 (scoring below rho) would be accepted without
    # its row as the pool's bound minus nothing (no right item in the view).
    # (The immediate schedule answers a group within the step that admits
    # it, before any later insert.)
    rng = np.random.default_rng(29)
    d, n0 = 64, 3999
    F = np.exp(3 * rng.standard_normal((n0 + 1, d)))
    F /= np.linalg.norm(F, axis=1, keepdims=True)
    F = F.astype(np.float32)
    F[3996] = F[n0]
    q = F[n0:n0 + 1].copy()
    rho = np.array([0.9], np.float32)
    ref = oracle.brute_force(F[:n0], q, rho, margin=0.0)
    assert 3996 in ref.neighbours(0) and 3998 not in ref.neighbours(0)
    assert float(F[3998].astype(np.float64) @ q[0].astype(np.float64)) < 0.8
    t = gt.Tree(F[:n0], capacity=n0 + 16)
    srv = gt.Server(t, dtype="bf16", cutover=3, schedule=schedule)
    srv.submit(q, rho, np.array([5]))
    srv.step()                           # admitted: the level-3 GEMM
    if schedule == "levels":
        srv.step()                       # level 2 (its right children gathered before the insert)
    srv.insert(F[n0:n0 + 1])             # applied at the start of the next step
    got = {}
    for _ in range(6):
        srv.step()
        for tag, ids, snap in srv.poll():
            got[tag] = (ids, snap)
    srv.close()
    ids, snap = got[5]
    assert snap == n0
    assert np.array_equal(ids, ref.neighbours(0))
    t.close()


@pytest.mark.parametrize("schedule", ["levels", "drain", "immediate"])
@pytest.mark.parametrize("dtype", ["bf16", "fp8"])
def test_served_recheck_decides_items_at_rho(gt, schedule, dtype):
    # items one FP32 ulp either side of rho, and rho itself, among 2048: every
    # bound straddles rho for them, so the FP64 recheck decides them, here in
    # the served steps of a group of 5 queries (the immediate schedule runs a
    # small group's recheck in the block that then assembles its CSR)
    rho = np.float32(0.8)
    up, dn = np.nextafter(rho, np.float32(2)), np.nextafter(rho, np.float32(0))
    rng = np.random.default_rng(3)
    x = np.array([up, dn, rho] * 30 + [0.1] * 1958, dtype=np.float32)[rng.permutation(2048)]
    F = np.zeros((x.size, 16), np.float32)
    F[:, 0] = x
    F[:, 1] = np.sqrt(1 - x.astype(np.float64) ** 2).astype(np.float32)
    Q = np.zeros((5, 16), np.float32)
    Q[:, 0] = 1.0                                   # q.f_i = x_i exactly
    ref = oracle.brute_force(F, Q[:1], np.array([rho]), margin=0.0)
    assert len(ref.ids) == 60
    t = gt.Tree(F)
    srv = gt.Server(t, dtype=dtype, schedule=schedule, max_group=5)
    srv.submit(Q, np.full(5, rho, np.float32), np.arange(5))
    got = {}
    for _ in range(40):
        srv.step()
        for tag, ids, snap in srv.poll():
            got[tag] = ids
        if len(got) == 5:
            break
    st = srv.stats()
    srv.close()
    t.close()
    assert sorted(got) == list(range(5))
    for i in range(5):
        assert np.array_equal(got[i], ref.neighbours(0))
    assert st["rechecks"] >= 5 * 90


def test_served_equals_alone(gt, stream_ds):
    ds = stream_ds
    n0 = 40_000
    t = gt.Tree(ds.F[:n0], capacity=ds.F.shape[0])
    done, st = _serve(gt, t, ds, n0, "bf16", max_group=128, insert_every=5)
    assert st["schedule"] == 3                               # the automatic choice here
    t.close()
    rng = np.random.default_rng(9)
    for tag in rng.choice(ds.Q.shape[0], 12, replace=False):
        ids, snap = done[int(tag)]
        alone = gt.Tree(ds.F[:snap])
        res = alone.query(ds.Q[tag:tag + 1], ds.rho[tag:tag + 1], dtype="bf16")
        assert np.array_equal(res.neighbours(0), ids)
        alone.close()


def test_server_refuses_bad_insert_rows_when_queued(gt, stream_ds):
    # rows are checked when they are queued (a step then applies them without
    # waiting for the device): a negative or non-finite entry is refused at
    # once and nothing of that call is queued
    ds = stream_ds
    t = gt.Tree(ds.F[:1000], capacity=2000)
    srv = gt.Server(t, dtype="bf16")
    for bad in (-1e-3, np.nan, np.inf):
        row = ds.F[1000:1002].copy()
        row[1, 5] = bad
        with pytest.raises(gt.GTError) as e:
            srv.insert(row)
        assert e.value.status == 2
    srv.insert(ds.F[1000:1002])
    srv.submit(ds.Q[:4], ds.rho[:4], np.arange(4))
    got = {}
    for _ in range(8):
        srv.step()
        for tag, ids, snap in srv.poll():
            got[tag] = (ids, snap)
    srv.close()
    ref = oracle.brute_force(ds.F[:1002], ds.Q[:4], ds.rho[:4])
    for i in range(4):
        assert got[i][1] == 1002
        assert np.array_equal(got[i][0], ref.neighbours(i))
    t.close()


def test_server_without_inserts_matches_batch_query(gt, stream_ds):
    ds = stream_ds
    t = gt.Tree(ds.F)
    done, st = _serve(gt, t, ds, ds.F.shape[0], "bf16", max_group=4096, insert_every=0)
    ref = t.query(ds.Q, ds.rho, dtype="bf16")
    for tag in range(ds.Q.shape[0]):
        assert np.array_equal(done[tag][0], ref.neighbours(tag))
    assert st["cutover"] == 3 and st["retries"] == 0
    t.close()


@pytest.mark.parametrize("schedule", ["levels", "immediate"])
def test_server_admission_backs_off_on_overflow(gt, stream_ds, schedule):
    ds = stream_ds
    t = gt.Tree(ds.F)
    # a frontier budget far below one full group's survivors: groups are cut
    # until they fit, and every answer is still exact (the immediate schedule
    # drops an overflowed group's answers and answers it again, smaller; its
    # GEMM list may fill the whole budget, so a lower rho makes it overflow)
    rho = ds.rho if schedule == "levels" else np.full(ds.Q.shape[0], 0.65, np.float32)
    srv = gt.Server(t, dtype="bf16", max_group=512, scratch_bytes=1 << 21, schedule=schedule)
    srv.submit(ds.Q, rho, np.arange(ds.Q.shape[0]))
    done = {}
    for _ in range(5000):
        srv.step()
        for tag, ids, snap in srv.poll():
            done[tag] = ids
        if len(done) == ds.Q.shape[0]:
            break
    st = srv.stats()
    srv.close()
    assert st["retries"] >= 1 and st["max_group"] < 512
    ref = t.query(ds.Q, rho, dtype="bf16")
    for tag in range(ds.Q.shape[0]):
        assert np.array_equal(done[tag], ref.neighbours(tag))
    t.close()


def test_streaming_setting_exact(gt):
    # Sec. 4's streaming setting in small: 80% of the database indexed, the
    # rest added 100 points at a time with one query after each addition;
    # every answer is the exact set over the items present at that moment
    ds = synth.generate(synth.Workload("t", 12_000, 1000, 40, (0.9,), "uniform:10", seed=21))
    N = ds.F.shape[0]
    n0 = int(0.8 * N)
    t = gt.Tree(ds.F[:n0], capacity=N)
    ref = oracle.brute_force(ds.F, ds.Q, ds.rho_for(0.9))
    assert ref.ambiguous.sum() == 0
    rho = np.full(1, 0.9, dtype=np.float32)
    n, k = n0, 0
    while n < N:
        m = min(100, N - n)
        t.insert(np.ascontiguousarray(ds.F[n:n + m]))
        n += m
        q = k % ds.Q.shape[0]
        res = t.query(np.ascontiguousarray(ds.Q[q:q + 1]), rho, dtype="bf16")
        want = ref.neighbours(q)
        assert np.array_equal(res.neighbours(0), want[want < n]), f"query {q} at N = {n}"
        k += 1
    assert t.size == N
    t.close()
