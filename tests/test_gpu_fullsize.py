"""Parity at the workloads' full sizes, in the launch configuration bench.py
uses, on sampled queries the oracle computes one by one (plus properties that
hold for every query)."""
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


def _check_sample(res, ds, rho, sample, F=None):
    F = ds.F if F is None else F
    ref = oracle.brute_force(F, ds.Q[sample], rho[sample])
    assert ref.ambiguous.sum() == 0
    for i, q in enumerate(sample):
        assert np.array_equal(res.neighbours(int(q)), ref.neighbours(i)), f"query {q}"


def _check_members(res, ds, rho, rng, n=20000):
    # every returned id scores >= rho in FP64 (a property of every query)
    lib = synth._load()
    counts = np.diff(res.offsets)
    qs = np.repeat(np.arange(len(counts)), counts)
    pick = rng.choice(qs.size, min(n, qs.size), replace=False)
    qi = np.ascontiguousarray(qs[pick].astype(np.int64))
    fi = np.ascontiguousarray(res.ids[pick].astype(np.int64))
    out = np.empty(qi.size)
    lib.syn_pair_dots(synth._p(ds.Q), synth._p(ds.F), ds.F.shape[1], qi.size, synth._p(qi),
                      synth._p(fi), synth._p(out))
    assert np.all(out >= rho[qi].astype(np.float64))


def test_paper_scale_1m(gt):
    ds = synth.generate("softmax_n1m_d1000")
    N, B = ds.F.shape[0], ds.Q.shape[0]
    Fd = torch.from_numpy(ds.F).cuda()
    t = gt.Tree(Fd)
    rng = np.random.default_rng(11)
    sample = np.sort(rng.choice(B, 48, replace=False))
    Qd = torch.from_numpy(ds.Q).cuda()
    for rho_v in ds.workload.rhos:
        rho = ds.rho_for(rho_v)
        rd = torch.from_numpy(rho).cuda()
        t.autotune(Qd[:2048], rd[:2048], dtype="bf16")
        for dtype in ("bf16", "fp8", "f32"):
            res = t.query(Qd, rd, dtype=dtype)
            _check_sample(res, ds, rho, sample)
            _check_members(res, ds, rho, rng)
            # planted near-duplicates with FP64 cosine >= rho are all found
            for q in sample:
                p = ds.planted[q]
                if len(p):
                    s = ds.F[p].astype(np.float64) @ ds.Q[q].astype(np.float64)
                    assert set(p[s >= rho[q]].tolist()) <= set(res.neighbours(int(q)).tolist())
        ex = t.exhaustive(Qd[sample], rd[sample])
        ref = oracle.brute_force(ds.F, ds.Q[sample], rho[sample])
        assert np.array_equal(ex.offsets, ref.offsets) and np.array_equal(ex.ids, ref.ids)
        # the Exh comparator over the raw rows (no tree), in the bench's form
        raw = gt.exhaustive(Fd, Qd[sample], rd[sample])
        assert np.array_equal(raw.offsets, ref.offsets) and np.array_equal(raw.ids, ref.ids)
    t.close()


def test_prefix_layout_paper_scale_1m(gt):
    # the prefix-sum layout (blocks of 8 items) at the headline workload, in
    # both prefix-row formats: sampled queries against the oracle, members of
    # every query's list checked in FP64
    ds = synth.generate("softmax_n1m_d1000")
    B = ds.Q.shape[0]
    t = gt.Tree(torch.from_numpy(ds.F).cuda(), layout="prefix", prefix_level=3,
                formats=("bf16", "f32"))
    rng = np.random.default_rng(13)
    sample = np.sort(rng.choice(B, 48, replace=False))
    Qd = torch.from_numpy(ds.Q).cuda()
    rho = ds.rho_for(0.8)
    rd = torch.from_numpy(rho).cuda()
    for dtype in ("bf16", "f32"):
        res = t.query(Qd, rd, dtype=dtype)
        assert res.stats["cutover"] == 3
        _check_sample(res, ds, rho, sample)
        _check_members(res, ds, rho, rng)
    t.close()


def test_large_10m_fp8_micro_batches(gt):
    free, _ = torch.cuda.mem_get_info()
    if free < 200e9:
        pytest.fail(f"the 10M workload needs ~200 GB of device memory, {free / 1e9:.0f} GB free")
    w = synth.WORKLOADS["softmax_n10m_d1000"]
    rng = np.random.default_rng(5)
    # screen the sampled queries (the margin is needed where the oracle looks);
    # include queries with the most planted duplicates
    counts = synth._plant_counts(w, w.n_queries)
    assert counts.max() > 300 and (counts == 0).mean() > 0.8        # heavy-tailed plants
    heavy = np.argsort(counts)[-8:]
    sample = np.union1d(np.sort(rng.choice(w.n_queries, 40, replace=False)), heavy)
    ds = synth.generate(w, screen=sample)
    Fd = torch.from_numpy(ds.F).cuda()
    t = gt.Tree(Fd, formats=("bf16", "fp8"))
    del Fd
    torch.cuda.empty_cache()
    rho = ds.rho_for(0.9)
    rd = torch.from_numpy(rho).cuda()
    Qd = torch.from_numpy(ds.Q).cuda()
    res = t.query(Qd, rd, dtype="fp8", max_batch=4096)
    assert res.stats["micro_batches"] == -(-ds.Q.shape[0] // 4096)
    _check_sample(res, ds, rho, sample)
    _check_members(res, ds, rho, rng)
    t.close()
