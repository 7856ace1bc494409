"""gt_query_static, the allocation-free query, against the definition
(the oracle's FP64 brute force) and against gt_query.

Callers that cannot allocate device memory while they serve (cudaMalloc can
stall every stream on the device; some processes give all device memory to
another allocator) use gt_query_static, which keeps its scratch in one fixed
device array.  This file runs after every other test so that a failure here
leaves the rest of the suite already run.
"""
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


def test_static_query_matches_gt_query_twice(gt):
    ds = synth.generate("softmax_n20k_d1000", n_queries=200, N=20_000)
    rho = ds.rho_for(0.9)
    exact = oracle.brute_force(ds.F, ds.Q, rho)     # the definition, FP64
    assert exact.ambiguous.sum() == 0                  # the inputs keep their margin
    t = gt.Tree(torch.from_numpy(ds.F).cuda())
    Qd = torch.from_numpy(ds.Q).cuda()
    rd = torch.from_numpy(rho).cuda()
    for dtype in ("f32", "bf16", "fp8"):
        ref = t.query(ds.Q, rho, dtype=dtype, cutover=-2)
        for call in range(2):                        # the array keeps the last call's state
            offsets = torch.full((201,), -1, dtype=torch.int64, device="cuda")
            ids = torch.full((len(exact.ids) + 16,), -1, dtype=torch.int32, device="cuda")
            free_before = torch.cuda.mem_get_info()[0]
            n = t.query_static(Qd, rd, offsets, ids, dtype=dtype)
            torch.cuda.synchronize()
            if call == 1:
                # set-up is done: later calls leave the device's free memory as it was
                assert torch.cuda.mem_get_info()[0] == free_before
            got_off, got_ids = offsets.cpu().numpy(), ids[:n].cpu().numpy()
            # exact sets: equal to the FP64 definition, and to gt_query's
            assert n == len(exact.ids)
            assert np.array_equal(got_off, exact.offsets)
            assert np.array_equal(got_ids, exact.ids)
            assert np.array_equal(got_off, ref.offsets) and np.array_equal(got_ids, ref.ids)
    t.close()


def test_static_query_limits(gt):
    ds = synth.generate("softmax_n20k_d1000", n_queries=300, N=5_000, screen=False)
    t = gt.Tree(torch.from_numpy(ds.F).cuda())
    Qd = torch.from_numpy(ds.Q).cuda()
    rd = torch.full((300,), 0.9, dtype=torch.float32, device="cuda")
    offsets = torch.zeros(301, dtype=torch.int64, device="cuda")
    ids = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(gt.GTError) as e:                 # above the 256-query limit
        t.query_static(Qd, rd, offsets, ids)
    assert e.value.status == 1
    with pytest.raises(gt.GTError) as e:                 # ids buffer too small: count reported
        t.query_static(Qd[:50], rd[:50], offsets[:51], ids)
    assert e.value.status == 6 and e.value.n_results > 1
    with pytest.raises(TypeError):                       # host tensors are refused
        t.query_static(torch.from_numpy(ds.Q[:2]), rd[:2], offsets[:3], ids)
    with pytest.raises(TypeError):                       # so is a mistyped output
        t.query_static(Qd[:2], rd[:2], offsets[:3].to(torch.int32), ids)
    t.close()
