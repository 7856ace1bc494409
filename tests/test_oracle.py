"""Pins for the oracle: each checks it against something other than itself
(closed forms, hand-worked traces, a library product, the paper's Table 3)."""
import math
import os

import numpy as np
import pytest

import oracle
from oracle import count_model as cm

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _two_hot(scores, d=8):
    """Items f_i = (x_i, sqrt(1 - x_i^2), 0, ...): unit norm, non-negative, and
    q = e_0 scores each exactly x_i (as float32)."""
    x = np.asarray(scores, dtype=np.float32)
    F = np.zeros((x.size, d), dtype=np.float32)
    F[:, 0] = x
    F[:, 1] = np.sqrt(np.maximum(0.0, 1.0 - x.astype(np.float64) ** 2)).astype(np.float32)
    q = np.zeros((1, d), dtype=np.float32)
    q[0, 0] = 1.0
    return F, q


# -- brute force: the definition --------------------------------------------

def test_brute_force_closed_form_scores():
    rng = np.random.default_rng(0)
    x = rng.random(257).astype(np.float32)
    F, q = _two_hot(x)
    for rho in (0.1, 0.5, 0.9, float(x[17])):
        res = oracle.brute_force(F, q, rho)
        expect = np.nonzero(x >= np.float32(rho))[0]
        assert np.array_equal(res.neighbours(0), expect)


def test_brute_force_one_hot_and_identical():
    d = 16
    F = np.eye(d, dtype=np.float32)                   # cosines are 0 or 1 exactly
    Q = np.eye(d, dtype=np.float32)[[3, 7]]
    res = oracle.brute_force(F, Q, 0.5)
    assert res.neighbours(0).tolist() == [3] and res.neighbours(1).tolist() == [7]
    same = np.tile(F[5], (9, 1))                       # all identical items
    res = oracle.brute_force(same, F[5:6], 0.999)
    assert res.neighbours(0).tolist() == list(range(9))


def test_brute_force_matches_library_product(small_ds):
    ds = small_ds
    rho = ds.rho_for(0.9)
    S = ds.Q.astype(np.float64) @ ds.F.astype(np.float64).T
    res = oracle.brute_force(ds.F, ds.Q, rho)
    assert res.ambiguous.sum() == 0
    for q in range(ds.Q.shape[0]):
        assert np.array_equal(res.neighbours(q), np.nonzero(S[q] >= rho[q])[0])


def test_toy_pool_prune_rule():
    # Sec. 2 toy example: y = f1 + f2 + f3 + f4; q.y < rho implies every q.f_i < rho
    rng = np.random.default_rng(3)
    for _ in range(200):
        F = rng.random((4, 12)) ** 4
        F /= np.linalg.norm(F, axis=1, keepdims=True)
        q = rng.random(12) ** 4
        q /= np.linalg.norm(q)
        y = F.sum(0)
        rho = rng.uniform(0.05, 1.0)
        if q @ y < rho:
            assert np.all(F @ q < rho)
        res = oracle.alg1(F.astype(np.float32), q[None].astype(np.float32), rho)
        bf = oracle.brute_force(F.astype(np.float32), q[None].astype(np.float32), rho)
        assert np.array_equal(res.ids, bf.ids)


# -- Algorithm 1 --------------------------------------------------------------

def test_alg1_hand_worked_trace():
    # x = [0.1, 0.9, 0, 0, 0.3], rho = 0.5.  Root [1,5] scores 1.3 (test 1);
    # n = 5 -> right [3,5] tested: 0.3 (test 2); left [1,2] = 1.0.  Pop [1,2]:
    # n = 2 -> right item 2 tested: 0.9 (test 3), flagged; item 1 = 0.1, not.
    # Pop [3,5]: 0.3 < 0.5, pruned.  Three tests, one per depth, neighbour {2}.
    F, q = _two_hot([0.1, 0.9, 0.0, 0.0, 0.3])
    res = oracle.alg1(F, q, 0.5)
    assert res.neighbours(0).tolist() == [1]
    assert res.tests[0] == 3
    assert res.rounds[:4].tolist() == [1, 1, 1, 0]
    assert oracle.alg1_scores(np.array([0.1, 0.9, 0.0, 0.0, 0.3]), 0.5) == 3


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 7, 8, 9, 16, 17, 63, 64])
def test_alg1_counts_all_positive_and_none(N):
    # every pool positive: one test per internal node of the splitting tree
    # (N - 1 of them) plus the root test = N; nothing positive: the root only
    rng = np.random.default_rng(N)
    x = rng.uniform(0.2, 0.9, N).astype(np.float32)
    F, q = _two_hot(x)
    res = oracle.alg1(F, q, 0.1)
    assert res.tests[0] == N and res.neighbours(0).tolist() == list(range(N))
    res = oracle.alg1(F, q, float(x.astype(np.float64).sum()) + 1.0)
    assert res.tests[0] == 1 and res.neighbours(0).size == 0


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 7, 8, 9, 16, 17, 63, 64])
def test_alg1_equals_brute_force_tiny(N):
    rng = np.random.default_rng(100 + N)
    d = 32
    F = np.exp(3 * rng.standard_normal((N, d)))
    F /= np.linalg.norm(F, axis=1, keepdims=True)
    F = F.astype(np.float32)
    Q = F[rng.integers(0, N, 6)] * np.exp(0.1 * rng.standard_normal((6, d)))
    Q /= np.linalg.norm(Q, axis=1, keepdims=True)
    Q = Q.astype(np.float32)
    for rho in (0.3, 0.7, 0.9, 0.99):
        a = oracle.alg1(F, Q, rho)
        b = oracle.brute_force(F, Q, rho, margin=0.0)
        assert np.array_equal(a.offsets, b.offsets) and np.array_equal(a.ids, b.ids)
        assert a.ambiguous.sum() == 0


def test_alg1_adversarial_near_rho():
    # an item exactly 2e-5 above / below rho, identical items, one-hot items
    rho = np.float32(0.8)
    x = np.array([rho + 2e-5, rho - 2e-5, 0.0, 1.0, 1.0, 1.0, 0.5, rho + 2e-5],
                 dtype=np.float32)
    F, q = _two_hot(x)
    a = oracle.alg1(F, q, rho)
    b = oracle.brute_force(F, q, rho)
    assert a.ids.tolist() == b.ids.tolist() == [0, 3, 4, 5, 7]
    assert a.ambiguous.sum() == 0 and b.ambiguous.sum() == 0


def test_alg1_equals_brute_force_workload(small_ds):
    ds = small_ds
    rho = ds.rho_for(0.9)
    a = oracle.alg1(ds.F, ds.Q, rho)
    b = oracle.brute_force(ds.F, ds.Q, rho)
    assert a.ambiguous.sum() == 0 and b.ambiguous.sum() == 0
    assert np.array_equal(a.offsets, b.offsets) and np.array_equal(a.ids, b.ids)
    # every query finds at least its planted duplicates' worth of structure
    assert (np.diff(a.offsets) >= 0).all()
    assert a.tests.min() >= 1 and a.tests.max() <= ds.F.shape[0]


def test_alg1_bound_flags_a_tie_deep_in_the_array():
    # an item scoring exactly rho at position 3001 of 4096: its score is
    # derived from running sums with a nonzero error bound, so the decision
    # is counted as ambiguous (a bound of zero, or one dropping the running
    # sums' terms, would report none)
    rho = np.float32(0.8)
    x = np.full(4096, 0.1, np.float32)
    x[3001] = rho
    F, q = _two_hot(x)
    a = oracle.Index(F).query(q, rho, margin=0.0)
    assert a.ambiguous.sum() >= 1
    assert 3001 in a.neighbours(0).tolist()        # the FP64 sums here are exact


def test_alg1_bound_covers_large_running_sums():
    # 1000 items of about 1e9 first, then about a million items scoring
    # 0.01-0.1 (full FP32 mantissas): the running sums are about 1e12, so
    # every addition rounds by up to 6e-5, and items one FP32 ulp either side
    # of rho deep in the array get derived scores that can fall on the wrong
    # side of rho.  The bound's running-sum terms (about 0.1 there) flag each
    # of them; decisions on items far from rho stay exact.
    rng = np.random.default_rng(11)
    rho = np.float32(0.8)
    near = np.array([300_017, 555_555, 777_001, 999_983])
    x = np.concatenate([rng.uniform(1e9, 2e9, 1000),
                        rng.uniform(0.01, 0.1, 1_000_000)]).astype(np.float32)
    x[near[0::2]] = np.nextafter(rho, np.float32(2))
    x[near[1::2]] = np.nextafter(rho, np.float32(0))
    F = np.zeros((x.size, 2), np.float32)
    F[:, 0] = x
    q = np.array([[1.0, 0.0]], np.float32)
    a = oracle.Index(F).query(q, rho, margin=0.0)
    assert a.ambiguous.sum() >= near.size
    exact = np.nonzero(x >= rho)[0]                   # q.f_i = x_i exactly
    got = a.neighbours(0)
    assert np.array_equal(np.setdiff1d(got, near), np.setdiff1d(exact, near))


def test_alg1_bound_at_full_scale():
    # N = 1M, d = 1000 softmax features, rho = 0.8: the queries of the
    # benchmark's 1024-query sample on which a bound that adds the parent's
    # whole error at every subtraction (so that the running sums' errors grow
    # down a run of left halves) reported decisions it could not vouch for.
    # Their errors cancel at the shared end of a pool and its right half, so
    # every decision is vouched for, and the sets equal the brute force.
    import synth
    qs = np.array([216, 229, 350, 358, 1025, 1752, 1756, 2305, 4042, 4656, 5399, 6240,
                   6293, 6517, 7226, 7572, 8001, 8943, 8992, 9916])
    ds = synth.generate("softmax_n1m_d1000", screen=qs, device="cpu")
    rho = ds.rho_for(0.8)[qs]
    ix = oracle.Index(ds.F)
    a = ix.query(ds.Q[qs], rho)
    ix.close()
    b = oracle.brute_force(ds.F, ds.Q[qs], rho)
    assert b.ambiguous.sum() == 0
    assert a.ambiguous.sum() == 0
    assert np.array_equal(a.offsets, b.offsets) and np.array_equal(a.ids, b.ids)


# -- pooling by element-wise maximum (Sec. 2) --------------------------------------

def _split_path_depth(N, t):
    """Depth of item t in Algorithm 1's splitting tree (left half floor(n/2))."""
    si, ei, depth = 0, N - 1, 0
    while si < ei:
        h = (ei - si + 1) // 2
        if t < si + h:
            ei = si + h - 1
        else:
            si = si + h
        depth += 1
    return depth


@pytest.mark.parametrize("N", [1, 2, 3, 5, 8, 13, 16, 64, 100])
def test_maxpool_one_hot_closed_form(N):
    # one-hot items e_i and query e_t: a pool's maximum vector contains e_t
    # iff t is a member, so exactly the pools on t's path pass; each split
    # of a passing pool tests both halves: 1 + 2 depth(t) tests, answer {t}
    d = max(N, 8)
    F = np.zeros((N, d), dtype=np.float32)
    F[np.arange(N), np.arange(N)] = 1.0
    for t in {0, N // 2, N - 1}:
        q = np.zeros((1, d), dtype=np.float32)
        q[0, t] = 1.0
        res = oracle.maxpool(F, q, 0.5)
        assert res.neighbours(0).tolist() == [t]
        depth = _split_path_depth(N, t)
        assert res.tests[0] == 1 + 2 * depth
        assert res.rounds[0] == 1 and all(res.rounds[k] == 2 for k in range(1, depth + 1))
        assert res.ambiguous.sum() == 0


def test_maxpool_vectors_are_column_maxima():
    rng = np.random.default_rng(7)
    F = rng.random((37, 12)).astype(np.float32)
    ix = oracle.MaxIndex(F)
    assert np.array_equal(ix.vec(0, 37), F.max(axis=0))        # the root
    # walk a few nodes of the splitting tree: [first, first + n)
    for first, n in ((0, 18), (18, 19), (18, 9), (27, 10), (27, 5), (32, 5), (36, 1)):
        v = ix.vec(first, n)
        assert v is not None and np.array_equal(v, F[first:first + n].max(axis=0))
    assert ix.vec(1, 5) is None                                   # not a node
    ix.close()


@pytest.mark.parametrize("N", [1, 2, 3, 4, 5, 7, 8, 9, 16, 17, 63, 64, 1000, 3001])
def test_maxpool_equals_brute_force(N):
    rng = np.random.default_rng(300 + N)
    d = 32
    F = np.exp(3 * rng.standard_normal((N, d)))
    F /= np.linalg.norm(F, axis=1, keepdims=True)
    F = F.astype(np.float32)
    Q = F[rng.integers(0, N, 6)] * np.exp(0.1 * rng.standard_normal((6, d)))
    Q /= np.linalg.norm(Q, axis=1, keepdims=True)
    Q = Q.astype(np.float32)
    for rho in (0.3, 0.7, 0.9, 0.99):
        a = oracle.maxpool(F, Q, rho)
        b = oracle.brute_force(F, Q, rho, margin=0.0)
        assert np.array_equal(a.offsets, b.offsets) and np.array_equal(a.ids, b.ids)
        assert a.ambiguous.sum() == 0


def test_maxpool_prunes_where_sum_pools_do(small_ds):
    # q.max(pool) <= q.sum(pool) for non-negative entries, so every pool the
    # sum traversal prunes the max traversal prunes too: at every depth k >= 1
    # the max traversal tests at most two pools per split the sum one makes
    ds = small_ds
    F = ds.F[:8192]
    rho = ds.rho_for(0.9)
    a = oracle.alg1(F, ds.Q, rho)
    m = oracle.maxpool(F, ds.Q, rho)
    assert np.array_equal(a.ids, m.ids) and np.array_equal(a.offsets, m.offsets)
    for k in range(1, 14):
        assert m.rounds[k] <= 2 * a.rounds[k]


# -- block prefix sums (Eq. 1 restarted per block) ------------------------------

def test_block_prefix_against_pools_and_global_sums():
    rng = np.random.default_rng(5)
    F = rng.random((1000, 37)).astype(np.float32)
    for c in (0, 1, 3, 6, 12):
        P = oracle.block_prefix_fp64(F, c)
        size = 1 << c
        if c == 0:
            assert np.array_equal(P, F.astype(np.float64))
        # the last row of each block is the block's pool (tree level c)
        ends = np.minimum(np.arange(0, F.shape[0], size) + size, F.shape[0]) - 1
        assert np.allclose(P[ends], oracle.pools_fp64(F, c), rtol=1e-14, atol=0)
        # consecutive rows of a block differ by the item; a block's first row
        # is its first item
        starts = np.arange(F.shape[0]) % size == 0
        assert np.array_equal(P[starts], F[starts].astype(np.float64))
        inner = ~starts
        diff = P[inner] - P[np.flatnonzero(inner) - 1]
        assert np.allclose(diff, F[inner], rtol=1e-12, atol=1e-13)
        # Eq. 1's global cumulative sums, less the sum before the block
        C = np.cumsum(F.astype(np.float64), axis=0)
        before = np.vstack([np.zeros((1, F.shape[1])), C])[(np.arange(F.shape[0]) >> c) << c]
        assert np.allclose(P, C - before, rtol=1e-12, atol=1e-12)


# -- signed descriptors: pools with a maximum and a minimum row (Sec. 2) ---------

def _signed_case(seed, N=3000, d=32, B=40, noise=0.06):
    import synth
    F, Q = synth.signed_workload(N, d, B, noise=noise, seed=seed)
    return F, Q, np.full(B, 0.8, np.float32)


def test_signed_split_worked_example():
    # three items e1, e2, -e1 and q = e1, rho = 0.5.  Algorithm 1's tree: the
    # root [0, 3) (M = (1, 1), m = (-1, 0): U = 1, split), item 0 (U = q.f = 1,
    # accepted) and the pool [1, 3) (M = (0, 1), m = (-1, 0): U = 0, pruned):
    # 3 tests.  By the split-row bound the item costs one more test (its U' = 1
    # reaches rho, so q.f is computed): 4 tests
    from oracle import signed
    F = np.array([[1.0, 0.0], [0.0, 1.0], [-1.0, 0.0]], dtype=np.float32)
    Q = np.array([[1.0, 0.0]], dtype=np.float32)
    ids, tests, amb = signed.maxmin_split(F, Q, 0.5)
    assert ids[0].tolist() == [0] and tests.tolist() == [3] and amb.sum() == 0
    ids, tests, _ = signed.maxmin_split(F, Q, 0.5, split=True)
    assert ids[0].tolist() == [0] and tests.tolist() == [4]
    ix = signed.MaxMinIndex(F)
    assert ix.bound(0, Q[0].astype(np.float64)) == 1.0
    assert [ix.first[n] for n in range(len(ix.first))] == [0, 0, 1, 1, 2]


def test_signed_split_sets_equal_brute_force():
    from oracle import signed
    F, Q, rho = _signed_case(3)
    assert (F < 0).any() and (Q < 0).any()
    ref = oracle.brute_force(F, Q, rho)
    assert ref.ambiguous.sum() == 0
    ids, tests, amb = signed.maxmin_split(F, Q, rho)
    assert amb.sum() == 0
    assert sum(len(x) for x in ids) > 20          # the planted neighbours are found
    for i in range(Q.shape[0]):
        assert np.array_equal(ids[i], ref.neighbours(i)), i
    assert np.all(tests < 2 * F.shape[0])         # never more than every node of the tree
    # pruning by the looser split-row bound: the same sets, never fewer tests
    s_ids, s_tests, s_amb = signed.maxmin_split(F, Q, rho, split=True)
    assert s_amb.sum() == 0
    assert all(np.array_equal(x, y) for x, y in zip(ids, s_ids))
    assert np.all(s_tests >= tests)


def test_signed_split_reduces_to_max_pooling_on_nonnegative_data(small_ds):
    # with F >= 0 and q >= 0 the bound is q . M, the max-pool score: the same
    # sets and the same number of tested nodes as the max-pool oracle (C)
    from oracle import signed
    F, Q = small_ds.F[:3000], small_ds.Q[:24]
    rho = small_ds.rho_for(0.8)[:24]
    ids, tests, amb = signed.maxmin_split(F, Q, rho)
    m = oracle.maxpool(F, Q, rho)
    assert amb.sum() == 0 and m.ambiguous.sum() == 0
    assert np.array_equal(tests, m.tests)
    for i in range(Q.shape[0]):
        assert np.array_equal(ids[i], m.neighbours(i))


def test_signed_split_sign_symmetry_and_dominance():
    from oracle import signed
    F, Q, rho = _signed_case(8, N=1500)
    a_ids, a_tests, _ = signed.maxmin_split(F, Q, rho)
    b_ids, b_tests, _ = signed.maxmin_split(-F, -Q, rho)   # q.f unchanged, M and m swap roles
    assert np.array_equal(a_tests, b_tests)
    assert all(np.array_equal(x, y) for x, y in zip(a_ids, b_ids))
    # every node's bound is at least its best member's score, and equals the
    # item's score at the leaves
    ix = signed.MaxMinIndex(F)
    Fd = F.astype(np.float64)
    for q in Q[:5].astype(np.float64):
        s = Fd @ q
        for node in range(0, len(ix.first), 7):
            a, n = ix.first[node], ix.size[node]
            u = ix.bound(node, q)
            assert u >= s[a:a + n].max() - 1e-12
            if n == 1:
                assert abs(u - s[a]) <= 1e-12
            # the split-row bound (non-negative rows [f+, f-]) is looser, never tighter
            assert ix.split_bound(node, q) >= u - 1e-12


# -- the count model (Sec. 5) ---------------------------------------------------

def _table3():
    rows = []
    with open(os.path.join(GOLDEN, "table3_theoretical.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            db, N, lam, rho, E = line.split()
            rows.append((db, int(N), float(lam), float(rho), int(E)))
    return rows


@pytest.mark.parametrize("row", _table3(), ids=lambda r: f"{r[0]}-{r[3]}")
def test_count_model_reproduces_table3(row):
    db, N, lam, rho, E = row
    got = cm.expected_tests(N, rho, lam)
    if db == "IMDB-Wiki":
        # the text's lambda = 10 is evidently rounded: within 0.5%
        assert abs(got - E) / E < 5e-3
    else:
        assert round(got) == E


def _table3_max():
    rows = []
    with open(os.path.join(GOLDEN, "table3_max_upper.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            db, N, lam, c, rho, E = line.split()
            rows.append((db, int(N), float(lam), float(c), float(rho), int(E)))
    return rows


@pytest.mark.parametrize("row", _table3_max(), ids=lambda r: f"{r[0]}-{r[4]}")
def test_max_pool_bound_reproduces_table3(row):
    # the printed values are rounded from the paper's own arithmetic: within 2
    db, N, lam, c, rho, E = row
    assert abs(cm.expected_tests_max_upper(N, rho, lam, c) - E) <= 2


def test_max_pool_bound_closed_forms():
    # no pool ever pruned (F_X(rho / c) ~ 0): every node of the tree is
    # tested, 2N - 1 for N a power of two
    for m in (1, 5, 12, 20):
        N = 2 ** m
        got = cm.expected_tests_max_upper(N, 0.8, 34.0, 1e14)
        assert abs(got - (2 * N - 1)) <= 1e-6 * N
    # every pool pruned (rho / c >= 1, so F_X = 1): the root test alone
    for N in (2, 1000, 10 ** 6):
        assert cm.expected_tests_max_upper(N, 0.8, 34.0, 0.5) == 1.0
    # the bound falls as rho rises and grows with c
    for lam in (10.0, 34.0, 57.0):
        Es = [cm.expected_tests_max_upper(10 ** 6, r, lam, 10.0) for r in (0.5, 0.7, 0.8, 0.9)]
        assert all(a >= b for a, b in zip(Es, Es[1:]))
        Es = [cm.expected_tests_max_upper(10 ** 6, 0.8, lam, c) for c in (2.0, 5.0, 10.0, 20.0)]
        assert all(a <= b for a, b in zip(Es, Es[1:]))


def test_max_pool_bound_single_split_against_simulation():
    # N = 2 with a pool score equal to c times its largest member score: the
    # root is tested, and both items are tested when it is positive, so the
    # mean count is the bound itself (no 1/2 factor)
    rng = np.random.default_rng(11)
    for lam, c, rho in ((34.0, 10.0, 0.8), (10.0, 3.0, 0.7), (57.0, 7.0, 0.9)):
        x = cm.tne_ppf(rng.random((400_000, 2)), lam)
        count = 1.0 + 2.0 * (c * x.max(1) >= rho)
        want = cm.expected_tests_max_upper(2, rho, lam, c)
        assert abs(count.mean() - want) < 1e-2


def test_tne_moments_against_quadrature():
    from scipy.integrate import quad
    for lam in (10.0, 30.0, 34.0, 57.0, 84.0):
        Z = 1.0 - math.exp(-lam)
        m1 = quad(lambda x: x * lam * math.exp(-lam * x) / Z, 0, 1)[0]
        m2 = quad(lambda x: x * x * lam * math.exp(-lam * x) / Z, 0, 1)[0]
        assert abs(cm.tne_mean(lam) - m1) < 1e-12
        assert abs(cm.tne_var(lam) - (m2 - m1 * m1)) < 1e-12


def test_small_pool_law_against_monte_carlo():
    rng = np.random.default_rng(7)
    for lam in (10.0, 34.0):
        for L in (1, 2, 3, 5):
            x = cm.tne_ppf(rng.random((400_000, L)), lam).sum(1)
            for rho in (0.05, 0.2, 0.7):
                p = cm.p_prune(L, rho, lam)
                assert abs(p - (x <= rho).mean()) < 4e-3


def test_count_model_monotone():
    # p_L increases with lambda and decreases with L; E decreases with lambda
    for rho in (0.7, 0.9):
        for L in (8, 16, 32):
            ps = [cm.p_prune(L, rho, lam) for lam in (10, 20, 34, 57)]
            assert all(a <= b for a, b in zip(ps, ps[1:]))
        for lam in (10, 34):
            # within each of the model's two regimes (exact law below 6
            # members, CLT from 6 on; the switch itself is not monotone)
            for Ls in ((1, 2, 3, 4, 5), (6, 8, 16, 32)):
                ps = [cm.p_prune(L, rho, lam) for L in Ls]
                assert all(a >= b for a, b in zip(ps, ps[1:]))
        Es = [cm.expected_tests(10 ** 6, rho, lam) for lam in (10, 30, 34, 57)]
        assert all(a >= b for a, b in zip(Es, Es[1:]))


@pytest.mark.parametrize("lam,rho", [(34, 0.8), (57, 0.8), (30, 0.9), (57, 0.7)])
def test_traversal_count_matches_model(lam, rho):
    # Algorithm 1 run on i.i.d. TNE scores: the mean count is within 5% of
    # E(rho) (the model's CLT and independence approximations)
    rng = np.random.default_rng(lam * 10 + int(rho * 10))
    N = 1_000_000
    ts = [oracle.alg1_scores(cm.tne_ppf(rng.random(N), lam), rho) for _ in range(8)]
    E = cm.expected_tests(N, rho, lam)
    assert abs(np.mean(ts) - E) / E < 0.05
