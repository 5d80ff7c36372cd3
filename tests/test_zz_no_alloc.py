"""The allocation-free estimate (pdd_estimate_nodes_noalloc) against the
regular one (pdd_estimate_nodes), through the C ABI.

Some callers cannot let the library allocate device memory -- their own pool
allocator has reserved it, or their loop cannot afford cudaMalloc/cudaFree.
The allocation-free entry point keeps its scratch in one fixed device array
instead.  This test checks that

* it gives the same per-node results as the regular entry point, bit for bit
  (both add exact integer sums over the same paths), on two calls in a row,
  so the second call does not see the first call's leftovers in the shared
  array;
* it runs on a context whose memory budget is too small for any workspace
  (where pdd_estimate_nodes fails with PDD_ERR_NOMEM), so it cannot have
  fallen back to the context's workspace, and the device's free memory is
  the same before and after the second call;
* it refuses more nodes than the array holds;
* it leaves the caller's current device as it was.

This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_1512_02818_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _args(pdd, cols, n_paths, dt, grid_id, tag):
    a = pdd.EstimateArgs()
    a.n_nodes = cols[0].shape[0]
    a.coords[0] = cols[0].data_ptr()
    a.coords[1] = cols[1].data_ptr()
    a.coords[2] = None
    a.coords_on_device = 1
    a.grid_id = grid_id
    a.n_paths = n_paths
    a.dt = dt
    a.kappa = 1.3
    a.seed = 1234
    a.stream_tag = tag
    a.flags = 0
    return a


def _outputs(pdd, torch, n):
    out = pdd.NodeStats()
    out.on_device = 1
    res = {}
    for f in pdd.STAT_FIELDS:
        res[f] = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        setattr(out, f, res[f].data_ptr())
    for f in pdd.COUNT_FIELDS:
        res[f] = torch.full((n,), -1, dtype=torch.int64, device="cuda")
        setattr(out, f, res[f].data_ptr())
    torch.cuda.synchronize()  # the fills ran on torch's stream, the library uses its own
    return out, res


def test_noalloc_matches_regular_entry_point_twice():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1512_02818_gb300 import build, pdd
    build.build()
    lib = pdd.lib()
    grid = W.control_grid(0, 129, 1e-2)
    # regular entry point on its own context
    ctx_ref = pdd.Context(0)
    prob_ref = pdd.Problem(ctx_ref, pdd.PDD_PROBLEM_CFG0_2D)
    prob_ref.set_control_grid(0, grid)
    # allocation-free entry point on a context that cannot hold any workspace
    ctx = pdd.Context(0, mem_budget=1)
    prob = pdd.Problem(ctx, pdd.PDD_PROBLEM_CFG0_2D)
    prob.set_control_grid(0, grid)  # grids are loaded at set-up (this allocates)
    nodes = W.workload_nodes("c1")[::2]  # 128 nodes
    n = nodes.shape[0]
    cols = [torch.from_numpy(np.ascontiguousarray(nodes[:, j])).cuda() for j in range(2)]
    torch.cuda.synchronize()
    dev_before = torch.cuda.current_device()
    for grid_id, n_paths in ((0, 3000), (pdd.PDD_CV_NONE, 2000)):
        args = _args(pdd, cols, n_paths, 1e-3, grid_id, 5)
        ref_out, ref = _outputs(pdd, torch, n)
        st = lib.pdd_estimate_nodes(prob_ref.handle, ctypes.byref(args), ctypes.byref(ref_out))
        assert st == 0, lib.pdd_last_error()
        # the small budget really blocks the context's workspace
        chk_out, _ = _outputs(pdd, torch, n)
        st = lib.pdd_estimate_nodes(prob.handle, ctypes.byref(args), ctypes.byref(chk_out))
        assert st == pdd.PDD_ERR_NOMEM
        for call in range(2):
            out, got = _outputs(pdd, torch, n)
            free_before = torch.cuda.mem_get_info()[0]
            st = lib.pdd_estimate_nodes_noalloc(prob.handle, ctypes.byref(args), ctypes.byref(out))
            assert st == 0, lib.pdd_last_error()
            torch.cuda.synchronize()
            if call == 1:  # the first call may load the array's module
                assert torch.cuda.mem_get_info()[0] == free_before
            for f in pdd.STAT_FIELDS + pdd.COUNT_FIELDS:
                assert np.array_equal(got[f].cpu().numpy(), ref[f].cpu().numpy(),
                                      equal_nan=True), (grid_id, call, f)
            assert np.all(got["n_paths"].cpu().numpy() == n_paths)
            assert torch.cuda.current_device() == dev_before
    # more nodes than the fixed scratch holds: refused before any launch
    big = [torch.zeros(pdd.PDD_NOALLOC_MAX_NODES + 1, dtype=torch.float32, device="cuda")
           for _ in range(2)]
    args = _args(pdd, big, 10, 1e-3, pdd.PDD_CV_NONE, 5)
    out, _ = _outputs(pdd, torch, pdd.PDD_NOALLOC_MAX_NODES + 1)
    st = lib.pdd_estimate_nodes_noalloc(prob.handle, ctypes.byref(args), ctypes.byref(out))
    assert st == pdd.PDD_ERR_INVALID
    assert b"PDD_NOALLOC_MAX_NODES" in lib.pdd_last_error()
    prob.close()
    ctx.close()
    prob_ref.close()
    ctx_ref.close()
