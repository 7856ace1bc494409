"""Checkpoint and resume of a tree (gt_save / gt_load): the reopened tree
holds the same rows at every level, bit for bit, and answers exactly; and an
allocation the device cannot satisfy is reported, not faulted."""
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


def _rows(t, kind):
    info = t.info()
    out = []
    if kind == "prefix":
        out.append(t.read_rows(0, "f32"))
        out.append(t.read_rows(info["prefix_level"], "bf16"))
        out.append(t.read_rows(-1, "bf16"))
        return out
    for h in range(info["levels"]):
        out.append(t.read_rows(h, "f32"))
        out.append(t.read_rows(h, "bf16"))
        out.extend(t.read_rows(h, "fp8"))
    return out


@pytest.mark.parametrize("kind", ["sum", "max", "maxmin", "prefix"])
def test_save_load_round_trip(gt, small_ds, tmp_path, kind):
    if kind == "maxmin":
        F, Q = synth.signed_workload(6000, 64, 60, noise=0.35 / 8.0, seed=4)
        rho = np.full(Q.shape[0], 0.8, dtype=np.float32)
        opts = dict(pooling="maxmin")
    else:
        F, Q, rho = small_ds.F[:6000], small_ds.Q, small_ds.rho_for(0.9)
        opts = dict(layout="prefix", prefix_level=3) if kind == "prefix" else dict(pooling=kind)
    perm = np.random.default_rng(2).permutation(4000) if kind == "sum" else None
    t = gt.Tree(F[:4000], perm=perm, capacity=4500, **opts)
    t.insert(F[4000:])                                   # grown past its capacity
    if kind != "prefix":
        t.set_tuning("bf16", cutover=3, inflight=16)
    path = str(tmp_path / f"tree_{kind}.gt")
    t.save(path)
    u = gt.Tree.load(path)
    assert u.info() == t.info()
    for a, b in zip(_rows(t, kind), _rows(u, kind)):
        assert np.array_equal(a, b)
    ref = oracle.brute_force(F, Q, rho)
    assert ref.ambiguous.sum() == 0
    for tree in (t, u):
        same_sets(tree.query(Q, rho, dtype="bf16"), ref)
    # both keep growing the same way
    more = F[:300] * np.float32(0.999)
    t.insert(more)
    u.insert(more)
    for a, b in zip(_rows(t, kind), _rows(u, kind)):
        assert np.array_equal(a, b)
    t.close()
    u.close()


def test_allocation_failure_is_reported(gt, small_ds):
    # storage for 2^31 - 2 rows of 2048 entries (tens of TB) cannot be had:
    # the build returns GT_ENOMEM and the device stays usable
    F = np.full((8, 2048), 1.0 / np.sqrt(2048), dtype=np.float32)
    with pytest.raises(gt.GTError) as e:
        gt.Tree(F, capacity=(1 << 31) - 2)
    assert e.value.status == 3
    ds = small_ds
    r = ds.rho_for(0.9)
    t = gt.Tree(ds.F)
    same_sets(t.query(ds.Q, r), oracle.brute_force(ds.F, ds.Q, r))
    t.close()
