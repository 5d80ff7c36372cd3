"""Failure handling without a GPU fault: the host stops work in flight.

A long estimate runs in one thread; another thread calls pdd_ctx_abort.  The
kernels take no further paths (nothing on the device waits), the estimate
returns PDD_ERR_CANCELLED well before its full duration with the statistics
of the paths that ran, and the context stays usable: the next call is not
affected and equals the same call on a fresh context, bit for bit.
"""
import threading
import time

import numpy as np
import pytest

from paper_1512_02818_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_abort_stops_work_in_flight():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1512_02818_gb300 import build, pdd
    build.build()
    ctx = pdd.Context(0)
    prob = pdd.Problem(ctx, pdd.PDD_PROBLEM_CFG0_2D)
    nodes = W.workload_nodes("c1")
    cols = [torch.from_numpy(np.ascontiguousarray(nodes[:, j])).cuda() for j in range(2)]
    prob.estimate(cols, 100, 1e-3)  # workspace and kernels loaded
    torch.cuda.synchronize()
    n_paths = 10_000_000  # ~2.7e12 path-steps: about 10 s if it ran to the end
    out = {}

    def run():
        t0 = time.perf_counter()
        try:
            out["res"] = prob.estimate(cols, n_paths, 1e-4, seed=5, stream_tag=3)
            out["status"] = out["res"]["status"]
        except pdd.PddError as e:
            out["status"] = e.status
        out["secs"] = time.perf_counter() - t0

    th = threading.Thread(target=run)
    th.start()
    time.sleep(0.5)
    t_abort = time.perf_counter()
    ctx.abort()
    out["abort_call_s"] = time.perf_counter() - t_abort
    th.join(timeout=60)
    assert not th.is_alive()
    assert out["status"] == pdd.PDD_ERR_CANCELLED, out
    assert out["secs"] < 4.0, out["secs"]
    # the context is usable and the next call is unaffected
    small = prob.estimate(cols, 500, 1e-3, seed=9, stream_tag=4)
    ctx2 = pdd.Context(0)
    prob2 = pdd.Problem(ctx2, pdd.PDD_PROBLEM_CFG0_2D)
    ref = prob2.estimate(cols, 500, 1e-3, seed=9, stream_tag=4)
    torch.cuda.synchronize()
    for f in pdd.STAT_FIELDS + pdd.COUNT_FIELDS:
        assert np.array_equal(small[f].cpu().numpy(), ref[f].cpu().numpy(), equal_nan=True), f
    # an abort with nothing in flight does not touch the next call either
    ctx.abort()
    again = prob.estimate(cols, 500, 1e-3, seed=9, stream_tag=4)
    torch.cuda.synchronize()
    assert np.array_equal(again["mean_phi"].cpu().numpy(), ref["mean_phi"].cpu().numpy())
    prob2.close()
    ctx2.close()
    prob.close()
    ctx.close()
