"""Precision study of the anisotropic 2D workload (32x32 subdomains, 31,744
nodes, dt = 1e-4, eps = 1e-2 control grid on 513^2): on a 256-node subsample
both the FP32 and the FP64 paths are compared with the FP64 oracle on the
same streams, path by path (first 32 paths of every node), and their node
means with each other."""
import numpy as np
import pytest

from paper_1512_02818_gb300 import workloads as W
from parity import PATH_ATOL, PATH_FRAC

pytestmark = pytest.mark.gpu


def test_fp32_and_fp64_paths_against_the_oracle():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import oracle
    from paper_1512_02818_gb300 import build, pdd
    build.build()
    oracle.build()
    ctx = pdd.Context(0)
    v = W.control_grid(1, 513, 1e-2)
    sub = W.workload_nodes("c4")[::124][:256]
    n_paths, h, k = 2000, 1e-4, 32
    ni = np.repeat(np.arange(len(sub)), k)
    pi = np.tile(np.arange(k), len(sub))
    ref = oracle.sample_paths(oracle.ANISO_2D, sub, ni, pi, h, seed=1234, tag=0,
                              cv=oracle.CV_GRID, grad=oracle.build_gradient(2, v), grid_n=513)
    res = {}
    for name, prec in (("fp32", pdd.PDD_PATH_FP32), ("fp64", pdd.PDD_PATH_FP64)):
        prob = pdd.Problem(ctx, pdd.PDD_PROBLEM_ANISO_2D, precision=prec)
        prob.set_control_grid(0, v)
        r = prob.estimate(sub, n_paths, h, grid_id=0, emit_paths=True)
        torch.cuda.synchronize()
        res[name] = {f: t.cpu().numpy() for f, t in r.items() if torch.is_tensor(t)}
        prob.close()
        steps = res[name]["steps"][ni, pi]
        same = steps == ref["steps"]
        dphi = np.abs(res[name]["phi"][ni, pi].astype(np.float64) - ref["phi"])
        dxi = np.abs(res[name]["xi"][ni, pi].astype(np.float64) - ref["xi"])
        ok = same & (dphi <= PATH_ATOL) & (dxi <= PATH_ATOL)
        assert ok.mean() >= PATH_FRAC, (name, ok.mean())
        if name == "fp64":
            # FP64 paths: exit indices agree, scores to the FP32 rounding of the emission
            assert same.mean() >= 0.9999
            assert dphi[same].max() < 2e-6 and dxi[same].max() < 2e-6
    se = res["fp64"]["se_cv"]
    d = np.abs(res["fp32"]["mean_cv"] - res["fp64"]["mean_cv"])
    live = se > 0  # nodes inside the shrinkage layer finish at k = 0
    assert np.all(d[live] <= np.maximum(1e-5 * np.abs(res["fp64"]["mean_cv"][live]), 3 * se[live]))
    ctx.close()
