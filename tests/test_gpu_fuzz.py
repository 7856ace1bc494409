"""Seeded random configurations against the definition.

Each case draws a database (softmax-like rows with near-duplicates of the
queries planted), a batch, rho, a row format, a layout or pooling, and the
traversal's knobs (cutover level, subtraction path, tests in flight per warp,
GEMM tile, micro-batch size), and compares the neighbour sets with the
oracle's FP64 brute force.  The draws cover row widths on both sides of the
ring's slot sizes (odd ring depths included), trees of one item to a few
thousand, and every kernel family the options select.
"""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

WIDTHS = [1, 7, 33, 100, 513, 600, 800, 1000, 1024, 1040, 1300]
INFLIGHT = [0, 1, 2, 4, 16, 32]
TILES = [0, 128, 256, 512, 1024]


@pytest.fixture(scope="module")
def gt():
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device: the GPU tests need a GB300")
    from paper_2311_02573_gb300 import gt as g
    g.load()
    return g


def draw(seed):
    rng = np.random.default_rng(1000 + seed)
    d = int(rng.choice(WIDTHS))
    N = int(rng.choice([1, 2, 3, 5, 8, 9, 31, 64, 65, 200, 777, 2048, 2049, 4100]))
    B = int(rng.integers(1, 70))
    F = np.exp(float(rng.uniform(1.0, 3.0)) * rng.standard_normal((N, d)))
    F /= np.linalg.norm(F, axis=1, keepdims=True)
    Q = F[rng.integers(0, N, B)] * np.exp(0.05 * rng.standard_normal((B, d)))
    # near-duplicates of some queries planted in the database
    k = min(N, int(rng.integers(0, 40)))
    if k:
        rows = rng.choice(N, k, replace=False)
        src = rng.integers(0, B, k)
        F[rows] = Q[src] * np.exp(0.03 * rng.standard_normal((k, d)))
        F[rows] /= np.linalg.norm(F[rows], axis=1, keepdims=True)
    Q /= np.linalg.norm(Q, axis=1, keepdims=True)
    rho = rng.uniform(0.3, 0.97, B).astype(np.float32)
    opts = dict(
        dtype=str(rng.choice(["f32", "bf16", "fp8"])),
        layout=str(rng.choice(["tree", "tree", "prefix"])),
        pooling=str(rng.choice(["sum", "sum", "max"])),
        cutover=int(rng.choice([-2, -1, 0, 1, 2, 3, 4, 5])),
        subtract=int(rng.choice([-1, 0, 1])),
        inflight=int(rng.choice(INFLIGHT)),
        tile=int(rng.choice(TILES)),
        max_batch=int(rng.choice([0, 0, 7, 16])),
    )
    return F.astype(np.float32), Q.astype(np.float32), rho, opts


@pytest.mark.parametrize("seed", range(120))
def test_random_configuration_equals_definition(gt, seed):
    F, Q, rho, o = draw(seed)
    N, d = F.shape
    ref = oracle.brute_force(F, Q, rho, margin=0.0)
    if o["layout"] == "prefix" and N >= 2:
        # (the prefix layout stores cumulative sums: sum pools only)
        t = gt.Tree(F, layout="prefix", prefix_level=int(min(3, max(1, (N - 1).bit_length() - 1))),
                    formats=("bf16", "f32") if o["dtype"] == "f32" else None)
        dtype = "f32" if o["dtype"] == "f32" else "bf16"
        res = t.query(Q, rho, dtype=dtype)
    else:
        t = gt.Tree(F, pooling=o["pooling"])
        if o["inflight"] or o["tile"]:
            t.set_tuning(o["dtype"], inflight=o["inflight"] or -1, tile=o["tile"] or -1)
        cut = o["cutover"]
        if cut >= t.levels:
            cut = -1
        res = t.query(Q, rho, dtype=o["dtype"], cutover=cut, subtract=o["subtract"],
                      max_batch=o["max_batch"])
    t.close()
    assert np.array_equal(res.offsets, ref.offsets), f"counts differ: {o}, N={N}, d={d}"
    assert np.array_equal(res.ids, ref.ids), f"ids differ: {o}, N={N}, d={d}"


@pytest.mark.parametrize("seed", range(24))
def test_random_served_configuration_equals_definition(gt, seed):
    # a server over a random tree: random schedule, group cap, row format,
    # arrivals in random chunks with inserts between them; every answer is
    # the definition over the items present when its group was admitted
    rng = np.random.default_rng(5000 + seed)
    d = int(rng.choice([33, 100, 600, 800, 1000]))
    N0 = int(rng.integers(600, 5000))
    n_ins = int(rng.integers(0, 400))
    B = int(rng.integers(20, 150))
    F = np.exp(2.5 * rng.standard_normal((N0 + n_ins, d)))
    F /= np.linalg.norm(F, axis=1, keepdims=True)
    Q = F[rng.integers(0, N0 + n_ins, B)] * np.exp(0.05 * rng.standard_normal((B, d)))
    Q /= np.linalg.norm(Q, axis=1, keepdims=True)
    F, Q = F.astype(np.float32), Q.astype(np.float32)
    rho = rng.uniform(0.5, 0.97, B).astype(np.float32)
    schedule = str(rng.choice(["auto", "levels", "drain", "immediate"]))
    dtype = str(rng.choice(["bf16", "fp8"]))
    t = gt.Tree(F[:N0], capacity=N0 + n_ins + 8)
    srv = gt.Server(t, dtype=dtype, max_group=int(rng.choice([1, 5, 32, 64, 100, 4096])),
                    schedule=schedule)
    sent, ins, done = 0, N0, {}
    for _ in range(20_000):
        if sent < B and rng.random() < 0.5:
            k = min(B, sent + int(rng.integers(1, 12)))
            srv.submit(Q[sent:k], rho[sent:k], np.arange(sent, k))
            sent = k
        if ins < N0 + n_ins and rng.random() < 0.3:
            m = min(N0 + n_ins - ins, int(rng.integers(1, 9)))
            srv.insert(F[ins:ins + m])
            ins += m
        srv.step()
        for tag, ids, snap in srv.poll():
            done[tag] = (ids, snap)
        if len(done) == B:
            break
    srv.close()
    t.close()
    assert len(done) == B
    for tag in range(B):
        ids, snap = done[tag]
        ref = oracle.brute_force(F[:snap], Q[tag:tag + 1], rho[tag:tag + 1], margin=0.0)
        assert np.array_equal(ids, ref.neighbours(0)), f"query {tag}, N={snap}, {schedule}, {dtype}"
