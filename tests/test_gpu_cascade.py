"""The levels Algorithm 4 schedules, run as Algorithm 5's nodal loop (one
launch for all levels), against the oracle at the same per-node time steps,
path counts and random streams.

Small case: the 24 nodes of the 2D problem, Algorithm 3 on a short cloud,
the schedule from a0 = 0.02, previous iterates v = u + (a_{j+1}/2) w.  Every
segment's sampled paths must match the oracle path by path; segments small
enough for the oracle are compared node by node in full; every level's
statistical error must be the balanced a_j / 2 (eq. F:N_y_h).
"""
import numpy as np
import pytest

from paper_1512_02818_gb300 import workloads as W
from parity import PATH_ATOL, compare_nodes

pytestmark = pytest.mark.gpu


def test_scheduled_cascade_matches_oracle():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import oracle
    from paper_1512_02818_gb300 import build, pdd
    from paper_1512_02818_gb300 import cascade as C
    build.build()
    oracle.build()
    ctx = pdd.Context(0)
    prob = pdd.Problem(ctx, pdd.PDD_PROBLEM_CFG0_2D)
    gn = 65
    w = W.control_grid(0, gn, 1.0) - W.control_grid(0, gn, 0.0)
    prob.set_control_grid(7, w)
    nodes = W.workload_nodes("c0")
    fit = prob.fit_constants(nodes, 2000, 2e-3, 1e-2, 12, grid_id=7, stream_tag_base=300)
    assert fit["status"] == 0
    a0 = 0.02
    a, _ = pdd.pdd_schedule(fit["K"], fit["beta"], fit["alpha"], fit["V_phi"], fit["V_psi"],
                            fit["rho_phi_psi"], 1.0, 1.2, a0, max_levels=3)
    assert a[0] == a0 and len(a) >= 2, a
    grads = {}
    for j in range(len(a) - 1):
        v = W.control_grid(0, gn, a[j + 1] / 2.0)
        prob.set_control_grid(j, v)
        grads[j] = oracle.build_gradient(2, v)
    levels = C.plan_levels(fit, a, h_min=1e-3, h_max=1e-2)
    run = C.run_levels(prob, nodes, levels, n_pilot=1000, n_max=20000, emit=True)
    torch.cuda.synchronize()
    assert run["status"] == 0 and run["pilot_status"] == 0
    rng = np.random.default_rng(21)
    n_full = 0
    for j, idx, n_paths, tag, h, res in run["segments"]:
        lv = levels[j]
        cv = oracle.CV_GRID if lv["controlled"] else oracle.CV_NONE
        grad, g_n = (grads[j], gn) if lv["controlled"] else (None, 0)
        sub = nodes[idx]
        work = idx.size * n_paths * float(res["mean_steps"].cpu().numpy().mean())
        if work <= 3e6:  # the oracle runs the whole segment: per path and per node
            ref = oracle.estimate_nodes(0, sub, n_paths, h, seed=1234, tag=tag, cv=cv, grad=grad,
                                        grid_n=g_n)
            same = res["steps"].cpu().numpy() == ref["steps"]
            ok = same & (np.abs(res["phi"].cpu().numpy() - ref["phi"]) <= PATH_ATOL) & (
                np.abs(res["xi"].cpu().numpy() - ref["xi"]) <= PATH_ATOL)
            assert ok.mean() >= 0.999, (j, ok.mean())
            nd = compare_nodes(res, ref)
            assert nd["mean_phi"]["ok"] and nd["mean_cv"]["ok"], (j, nd)
            n_full += 1
        else:  # sampled paths
            m = 64
            ni = rng.integers(0, idx.size, size=m)
            pi = rng.integers(0, n_paths, size=m)
            ref = oracle.sample_paths(0, sub, ni, pi, h, seed=1234, tag=tag, cv=cv, grad=grad,
                                      grid_n=g_n)
            t = (torch.from_numpy(ni), torch.from_numpy(pi))
            same = res["steps"][t].cpu().numpy() == ref["steps"]
            ok = same & (np.abs(res["phi"][t].cpu().numpy() - ref["phi"]) <= PATH_ATOL) & (
                np.abs(res["xi"][t].cpu().numpy() - ref["xi"]) <= PATH_ATOL)
            assert ok.mean() >= 0.98, (j, ok.mean())
    assert n_full >= 1
    # balanced statistical error: q SE = a_j / 2 up to sampling error (the
    # pilot's variance and the run's own standard error, both from a finite
    # sample; coarse levels run only a few hundred paths per node)
    for lv, ob in zip(levels, run["levels"]):
        capped = lv["n_paths"] >= 20000
        ratio = (2.0 * 2.0 * ob["se"] / lv["a"])[~capped]
        assert np.all(np.isfinite(ratio)), (lv["a"], ratio)
        assert np.median(ratio) <= 1.1 and ratio.max() <= 1.6, (
            lv["a"], lv["controlled"], np.median(ratio), ratio.max(),
            lv["n_paths"][~capped][np.argmax(ratio)])
    prob.close()
    ctx.close()
