"""The allocation-free estimate (pdd_estimate_nodes_noalloc) against the
regular one (pdd_estimate_nodes), through the C ABI.

Some callers cannot let the library allocate device memory -- their own pool
allocator has reserved it, or their loop cannot afford cudaMalloc/cudaFree.
The allocation-free entry point keeps its scratch in one fixed device array
instead; this test checks that it gives the same per-node results as the
regular entry point on two calls in a row (the second call must not see the
first call's leftovers in the shared array), and that it refuses more nodes
than the array holds.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_1512_02818_gb300 import workloads as W
from parity import node_tolerance

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
    ctx = pdd.Context(0)
    prob = pdd.Problem(ctx, pdd.PDD_PROBLEM_CFG0_2D)
    prob.set_control_grid(0, W.control_grid(0, 129, 1e-2))
    nodes = W.workload_nodes("c1")[::2]  # 128 nodes
    n = nodes.shape[0]
    cols = [torch.from_numpy(np.ascontiguousarray(nodes[:, j])).cuda() for j in range(2)]
    torch.cuda.synchronize()
    for grid_id, n_paths in ((0, 3000), (pdd.PDD_CV_NONE, 2000)):
        args = _args(pdd, cols, n_paths, 1e-3, grid_id, 5)
        ref_out, ref = _outputs(pdd, torch, n)
        assert lib.pdd_estimate_nodes(prob.handle, ctypes.byref(args), ctypes.byref(ref_out)) == 0
        for call in range(2):
            out, got = _outputs(pdd, torch, n)
            st = lib.pdd_estimate_nodes_noalloc(prob.handle, ctypes.byref(args), ctypes.byref(out))
            assert st == 0, lib.pdd_last_error()
            torch.cuda.synchronize()
            for m, se in (("mean_phi", "se_phi"), ("mean_cv", "se_cv")):
                r, g = ref[m].cpu().numpy(), got[m].cpu().numpy()
                tol = node_tolerance(r, got[se].cpu().numpy(), ref[se].cpu().numpy())
                assert np.all(np.abs(g - r) <= tol), (call, m)
            for f in ("var_phi", "var_cv", "mean_steps"):
                assert np.allclose(got[f].cpu().numpy(), ref[f].cpu().numpy(), rtol=1e-12), f
            assert np.array_equal(got["n_paths"].cpu().numpy(), ref["n_paths"].cpu().numpy())
            assert np.all(got["n_paths"].cpu().numpy() == n_paths)
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
