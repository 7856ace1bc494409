"""Failure detection without a fault: the gather kernels' bounded waits.

Every wait of a ring-fed gather kernel on its bulk copies is bounded (1 s);
when one runs out the kernel raises a status word, lets the copies it started
land, and returns, and the call reports GT_ETIMEOUT.  gt_set_wait_expiry makes
the kernels start no copy, so their first wait runs out at once with nothing
in flight: the call must fail with GT_ETIMEOUT, and the tree must answer the
next query exactly."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

GT_ETIMEOUT = 5


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


def test_expired_wait_returns_timeout_and_tree_recovers(gt, small_ds):
    ds = small_ds
    r = ds.rho_for(0.9)
    ref = oracle.brute_force(ds.F, ds.Q, r)
    assert ref.ambiguous.sum() == 0
    t = gt.Tree(ds.F)
    for dtype in ("bf16", "fp8"):
        t.set_tuning(dtype, inflight=16)                 # ring-fed gathers at every level
    calls = [dict(cutover=3, subtract=1), dict(cutover=3, subtract=-1), dict(cutover=-2)]
    for kw in calls:                                     # graphs captured in the normal state
        same_sets(t.query(ds.Q, r, **kw), ref)
    t.set_wait_expiry(True)
    for kw in calls:
        for dtype in ("bf16", "fp8"):
            with pytest.raises(gt.GTError) as e:
                t.query(ds.Q, r, dtype=dtype, **kw)
            assert e.value.status == GT_ETIMEOUT, str(e.value)
    t.set_wait_expiry(False)
    for kw in calls:                                     # the same graphs, replayed
        for dtype in ("bf16", "fp8", "f32"):
            same_sets(t.query(ds.Q, r, dtype=dtype, **kw), ref)
    t.close()


def test_expired_wait_on_prefix_layout(gt, small_ds):
    ds = small_ds
    r = ds.rho_for(0.9)
    ref = oracle.brute_force(ds.F, ds.Q, r)
    p = gt.Tree(ds.F, layout="prefix", prefix_level=3)
    same_sets(p.query(ds.Q, r), ref)
    p.set_wait_expiry(True)
    with pytest.raises(gt.GTError) as e:
        p.query(ds.Q, r)
    assert e.value.status == GT_ETIMEOUT
    p.set_wait_expiry(False)
    same_sets(p.query(ds.Q, r), ref)
    p.close()
