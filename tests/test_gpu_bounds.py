"""The traversal's per-test bounds against FP64 (gt_pair_bounds runs the
level kernels' own dot product and bound code on given (query, pool) pairs):
the upper bound that prunes is at or above the exact pool score and the lower
bound that accepts (or that the subtraction path takes) is at or below it, in
every row format, at every level, for sum and for max pools."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# how far above the exact score an upper bound may sit (relative, plus an
# absolute slack for FP8's subnormal term): the format's rounding on both
# sides, FP32 accumulation and pool rounding, with room to spare
LOOSE = {"f32": (2e-4, 0.0), "bf16": (0.02, 0.0), "fp8": (0.2, 1e-3)}


@pytest.fixture(scope="module")
def gt():
    if not torch.cuda.is_available():
        pytest.fail("no CUDA device: the GPU tests need a GB300")
    from paper_2311_02573_gb300 import gt as g
    g.load()
    return g


def max_pools(F, h):
    """Element-wise maxima of the power-of-two blocks of F's rows (exact)."""
    size = 1 << h
    starts = np.arange(0, F.shape[0], size)
    return np.maximum.reduceat(F.astype(np.float64), starts, axis=0)


def pairs_for(S, rng, k=40):
    """Each query against its k best pools (the ones near any threshold) and k
    random ones."""
    nq, nr = S.shape
    k = min(k, nr)
    out = []
    for q in range(nq):
        top = np.argsort(-S[q])[:k]
        rnd = rng.integers(0, nr, k)
        for j in np.concatenate([top, rnd]):
            out.append((q, j))
    return np.array(out, dtype=np.int32)


def check(out, exact, dtype, what):
    U, L = out[:, 1].astype(np.float64), out[:, 2].astype(np.float64)
    assert np.all(np.isfinite(out)), what
    bad = np.flatnonzero(U < exact)
    assert bad.size == 0, f"{what}: U below the exact score at {bad[:5]}: {U[bad[:5]]} < {exact[bad[:5]]}"
    bad = np.flatnonzero(L > exact)
    assert bad.size == 0, f"{what}: L above the exact score at {bad[:5]}: {L[bad[:5]]} > {exact[bad[:5]]}"
    rel, ab = LOOSE[dtype]
    assert np.all(U <= exact * (1 + rel) + ab), f"{what}: upper bound looser than the format allows"


@pytest.mark.parametrize("d", [1000, 100, 1040])
def test_pair_bounds_hold_against_fp64(gt, d):
    ds = synth.generate(synth.Workload("t", 6000, d, 48, (0.8,), "uniform:10", seed=d + 3),
                        screen=False)
    t = gt.Tree(ds.F)
    Q64 = ds.Q.astype(np.float64)
    rng = np.random.default_rng(d)
    for h in sorted({0, 1, 2, 5, t.levels - 1}):
        S = Q64 @ oracle.pools_fp64(ds.F, h).T      # exact: FP32 products, FP64 sums
        pairs = pairs_for(S, rng)
        exact = S[pairs[:, 0], pairs[:, 1]]
        for dtype in ("f32", "bf16", "fp8"):
            out = t.pair_bounds(h, dtype, ds.Q, pairs)
            check(out, exact, dtype, f"level {h} {dtype}")
    t.close()


def test_subtraction_bound_holds(gt):
    # the left child's bounds: U_parent - max(L_right, 0) (rounded up by the
    # kernels) is at or above its exact score, L_parent - U_right (rounded
    # down) at or below it
    ds = synth.generate(synth.Workload("t", 8192, 256, 40, (0.8,), "uniform:10", seed=9),
                        screen=False)
    t = gt.Tree(ds.F)
    Q64 = ds.Q.astype(np.float64)
    rng = np.random.default_rng(1)
    for h in (0, 1, 3):
        Sp = Q64 @ oracle.pools_fp64(ds.F, h + 1).T
        Sc = Q64 @ oracle.pools_fp64(ds.F, h).T
        pp = pairs_for(Sp, rng, 30)
        right = pp.copy()
        right[:, 1] = 2 * pp[:, 1] + 1
        left_exact = Sc[pp[:, 0], 2 * pp[:, 1]]
        for dtype in ("f32", "bf16", "fp8"):
            bp = t.pair_bounds(h + 1, dtype, ds.Q, pp).astype(np.float64)
            br = t.pair_bounds(h, dtype, ds.Q, right).astype(np.float64)
            Up, Lp = bp[:, 1], bp[:, 2]
            Ur, Lr = br[:, 1], br[:, 2]
            assert np.all(Up - np.maximum(Lr, 0.0) >= left_exact), f"level {h} {dtype}"
            assert np.all(Lp - Ur <= left_exact), f"level {h} {dtype}"
    t.close()


def test_max_pool_bounds_hold(gt):
    ds = synth.generate(synth.Workload("t", 5000, 300, 32, (0.8,), "uniform:10", seed=21),
                        screen=False)
    t = gt.Tree(ds.F, pooling="max")
    Q64 = ds.Q.astype(np.float64)
    rng = np.random.default_rng(2)
    for h in (1, 3, t.levels - 1):
        S = Q64 @ max_pools(ds.F, h).T
        pairs = pairs_for(S, rng)
        exact = S[pairs[:, 0], pairs[:, 1]]
        for dtype in ("f32", "bf16", "fp8"):
            check(t.pair_bounds(h, dtype, ds.Q, pairs), exact, dtype, f"max level {h} {dtype}")
    t.close()


def test_pair_bounds_adversarial_rows(gt):
    # near-one-hot and flat rows and queries, and rows whose entries span many
    # binades (FP8 subnormals): the bounds must still hold
    d = 512
    rng = np.random.default_rng(4)
    F = np.full((512, d), 1.0 / np.sqrt(d), dtype=np.float32)
    F[:256] = np.exp(-30 * rng.random((256, d))).astype(np.float32)
    F[256:300] = np.exp(-60 * rng.random((44, d))).astype(np.float32)
    F /= np.linalg.norm(F.astype(np.float64), axis=1, keepdims=True).astype(np.float32)
    Q = np.concatenate([F[:32], np.full((8, d), 1.0 / np.sqrt(d), np.float32)])
    t = gt.Tree(F)
    Q64 = Q.astype(np.float64)
    for h in (0, 2, 6):
        S = Q64 @ oracle.pools_fp64(F, h).T
        q, j = np.meshgrid(np.arange(S.shape[0]), np.arange(S.shape[1]), indexing="ij")
        pairs = np.stack([q.ravel(), j.ravel()], axis=1).astype(np.int32)
        exact = S.ravel()
        for dtype in ("f32", "bf16", "fp8"):
            check(t.pair_bounds(h, dtype, Q, pairs), exact, dtype, f"adversarial level {h} {dtype}")
    t.close()


def test_pair_bounds_arguments(gt, small_ds):
    t = gt.Tree(small_ds.F[:1000])
    Q = small_ds.Q[:4]
    out = t.pair_bounds(0, "bf16", Q, np.array([[0, 0], [4, 0], [0, 1000], [-1, 3]], np.int32))
    assert np.all(np.isfinite(out[0])) and np.all(np.isnan(out[1:]))
    with pytest.raises(gt.GTError):
        t.pair_bounds(t.levels, "bf16", Q, np.array([[0, 0]], np.int32))
    bad = Q.copy()
    bad[0, 0] = -1.0
    with pytest.raises(gt.GTError):
        t.pair_bounds(0, "bf16", bad, np.array([[0, 0]], np.int32))
    t.close()
