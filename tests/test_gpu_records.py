"""Exact node records through the C ABI: a run split into path ranges,
checkpointed to the host and resumed, or split across two record sets merged
on the host, finalises to the same bits as one pdd_estimate_nodes call."""
import numpy as np
import pytest

from paper_1512_02818_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_split_checkpoint_merge_equal_single_run():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1512_02818_gb300 import build, pdd
    build.build()
    ctx = pdd.Context(0)
    prob = pdd.Problem(ctx, pdd.PDD_PROBLEM_CFG0_2D)
    prob.set_control_grid(0, W.control_grid(0, 129, 1e-2))
    nodes = W.workload_nodes("c1")[::8]
    n = nodes.shape[0]
    cols = [torch.from_numpy(np.ascontiguousarray(nodes[:, j])).cuda() for j in range(2)]
    N, h = 900, 1e-3
    ref = prob.estimate(cols, N, h, grid_id=0, seed=77, stream_tag=3, kappa=1.0)
    ref = {k: v.cpu().numpy() for k, v in ref.items() if torch.is_tensor(v)}

    def same(res):
        for f in pdd.STAT_FIELDS + pdd.COUNT_FIELDS:
            assert np.array_equal(res[f].cpu().numpy(), ref[f], equal_nan=True), f

    rec = torch.zeros((n, pdd.PDD_RECORD_WORDS), dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    prob.accumulate(cols, 300, h, rec, path_offset=0, grid_id=0, seed=77, stream_tag=3)
    # checkpoint: records to the host, device copy wiped, then restored
    saved = rec.cpu().numpy().copy()
    rec.zero_()
    rec.copy_(torch.from_numpy(saved).cuda())
    torch.cuda.synchronize()
    prob.accumulate(cols, 400, h, rec, path_offset=300, grid_id=0, seed=77, stream_tag=3)
    prob.accumulate(cols, 200, h, rec, path_offset=700, grid_id=0, seed=77, stream_tag=3)
    same(ctx.finalize_records(rec))
    # two record sets (e.g. two GPUs) merged on the host
    r1 = torch.zeros_like(rec)
    r2 = torch.zeros_like(rec)
    torch.cuda.synchronize()
    prob.accumulate(cols, 450, h, r1, path_offset=0, grid_id=0, seed=77, stream_tag=3)
    prob.accumulate(cols, 450, h, r2, path_offset=450, grid_id=0, seed=77, stream_tag=3)
    a = r1.cpu().numpy().view(np.uint64).copy()
    b = r2.cpu().numpy().view(np.uint64).copy()
    pdd.pdd_records_merge(a.ctypes.data, b.ctypes.data, n)
    merged = torch.from_numpy(a.view(np.int64)).cuda()
    torch.cuda.synchronize()
    same(ctx.finalize_records(merged))
    with pytest.raises(pdd.PddError):
        prob.accumulate(cols, 10, h, rec, path_offset=2**32 - 5, grid_id=0)
    prob.close()
    ctx.close()
