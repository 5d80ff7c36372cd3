"""Multilevel coupling and the multilevel driver on the GPU through the C ABI.

* Coupled pairs (2D and 3D) against the oracle's coupling on the same
  streams: per path (fine and coarse exit indices and scores) and per node;
  the fine level equals pdd_estimate_nodes at dt/2; the level difference has
  a small variance.
* pdd_accumulate_coupled in slices gives the records of one call, bit for bit.
* pdd_mlmc: its counts are the allocation rule applied to its own level
  moments; its estimate is the sum of independently computed level means
  (bit for bit) and matches the oracle's levels at the same counts; the
  Talay-Tubaro extrapolation and the variances follow from the levels.
"""
import numpy as np
import pytest

from paper_1512_02818_gb300 import workloads as W
from parity import PATH_ATOL, PATH_FRAC

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind,cv", [(0, "grid"), (0, "none"), (4, "exact"), (1, "grid")])
def test_coupled_matches_oracle(kind, cv):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import oracle
    from paper_1512_02818_gb300 import build, pdd
    build.build()
    oracle.build()
    ctx = pdd.Context(0)
    prob = pdd.Problem(ctx, kind)
    nodes = (W.workload_nodes("paper") if kind == 4 else W.workload_nodes("c1")[::16])
    grad, gid, ocv = None, pdd.PDD_CV_NONE, oracle.CV_NONE
    if cv == "grid":
        v = W.control_grid(kind, 65, 1e-2)
        prob.set_control_grid(0, v)
        grad, gid, ocv = oracle.build_gradient(2, v), 0, oracle.CV_GRID
    elif cv == "exact":
        gid, ocv = pdd.PDD_CV_EXACT, oracle.CV_EXACT
    N, h = 300, 2e-3
    fine, diff = prob.estimate_coupled(nodes, N, h, grid_id=gid, seed=3, stream_tag=11,
                                       emit_paths=True)
    torch.cuda.synchronize()
    assert fine["status"] == 0
    ref = oracle.coupled_paths(kind, nodes, N, h, seed=3, tag=11, cv=ocv, grad=grad,
                               grid_n=65 if cv == "grid" else 0)
    ok = np.ones(ref["phi_f"].shape, dtype=bool)
    for lvl, res in (("f", fine), ("c", diff)):
        st = res["steps"].cpu().numpy()
        same = st == ref["steps_" + lvl]
        ok &= same
        ok &= np.abs(res["phi"].cpu().numpy() - ref["phi_" + lvl]) <= PATH_ATOL
        ok &= np.abs(res["xi"].cpu().numpy() - ref["xi_" + lvl]) <= PATH_ATOL
    assert ok.mean() >= PATH_FRAC, ok.mean()
    # fine level == the plain estimate at dt/2 on the same streams (a different
    # kernel: FP32 contraction choices may differ in the last bits)
    alone = prob.estimate(nodes, N, h / 2, grid_id=gid, seed=3, stream_tag=11)
    for f in ("mean_phi", "mean_cv", "var_phi", "var_cv", "mean_steps"):
        assert np.allclose(fine[f].cpu().numpy(), alone[f].cpu().numpy(), rtol=1e-5, atol=1e-6,
                           equal_nan=True), f
    assert np.array_equal(fine["n_paths"].cpu().numpy(), alone["n_paths"].cpu().numpy())
    # the difference statistics are those of the emitted pairs
    d = fine["phi"].cpu().numpy().astype(np.float64) - diff["phi"].cpu().numpy()
    assert np.allclose(diff["mean_phi"].cpu().numpy(), d.mean(1), atol=1e-6)
    assert np.allclose(diff["var_phi"].cpu().numpy(), d.var(1, ddof=1), rtol=1e-3, atol=1e-7)
    # (nodes inside the shrinkage layer finish at k = 0: both variances are 0)
    assert np.all(diff["var_phi"].cpu().numpy() <= 0.5 * fine["var_phi"].cpu().numpy() + 1e-12)
    assert np.allclose(diff["mean_steps"].cpu().numpy(), ref["steps_c"].mean(1), rtol=1e-3)
    with pytest.raises(pdd.PddError):  # coupling runs FP32 paths only
        pdd.Problem(ctx, kind, precision=pdd.PDD_PATH_FP64).estimate_coupled(nodes[:2], 10, 1e-2)
    prob.close()
    ctx.close()


def _env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import oracle
    from paper_1512_02818_gb300 import build, pdd
    build.build()
    oracle.build()
    return torch, oracle, pdd


def _interior_3d(count):
    nodes = W.workload_nodes("c2")
    d = np.minimum(nodes, 1.0 - nodes).min(axis=1)
    return nodes[np.argsort(-d)[:count]]


@pytest.mark.parametrize("cv", ["grid", "exact"])
def test_coupled_3d_matches_oracle(cv):
    torch, oracle, pdd = _env()
    ctx = pdd.Context(0)
    prob = pdd.Problem(ctx, pdd.PDD_PROBLEM_CUBE_3D)
    nodes = np.concatenate([_interior_3d(24), W.workload_nodes("c2")[::400]])
    grad, gid, ocv, gn = None, pdd.PDD_CV_EXACT, oracle.CV_EXACT, 0
    if cv == "grid":
        v = W.control_grid(2, 17, 1e-2)
        prob.set_control_grid(0, v)
        grad, gid, ocv, gn = oracle.build_gradient(3, v), 0, oracle.CV_GRID_CELLS16, 17
    N, h = 200, 4e-3
    fine, diff = prob.estimate_coupled(nodes, N, h, grid_id=gid, seed=7, stream_tag=5,
                                       emit_paths=True)
    torch.cuda.synchronize()
    assert fine["status"] == 0
    ref = oracle.coupled_paths(2, nodes, N, h, seed=7, tag=5, cv=ocv, grad=grad, grid_n=gn)
    ok = np.ones(ref["phi_f"].shape, dtype=bool)
    for lvl, res in (("f", fine), ("c", diff)):
        ok &= res["steps"].cpu().numpy() == ref["steps_" + lvl]
        ok &= np.abs(res["phi"].cpu().numpy() - ref["phi_" + lvl]) <= PATH_ATOL
        ok &= np.abs(res["xi"].cpu().numpy() - ref["xi_" + lvl]) <= PATH_ATOL
    assert ok.mean() >= PATH_FRAC, ok.mean()
    assert ref["steps_c"].max() > 4  # the coarse paths take several steps
    alone = prob.estimate(nodes, N, h / 2, grid_id=gid, seed=7, stream_tag=5)
    for f in ("mean_phi", "mean_cv", "mean_steps"):
        assert np.allclose(fine[f].cpu().numpy(), alone[f].cpu().numpy(), rtol=1e-5, atol=1e-6), f
    prob.close()
    ctx.close()


@pytest.mark.parametrize("kind", [0, 2])
def test_accumulate_coupled_in_slices_is_one_call(kind):
    torch, oracle, pdd = _env()
    ctx = pdd.Context(0)
    prob = pdd.Problem(ctx, kind)
    nodes = W.workload_nodes("c1")[::8] if kind == 0 else _interior_3d(40)
    n = len(nodes)
    dev = torch.device("cuda", 0)
    rf = torch.zeros((n, pdd.PDD_RECORD_WORDS), dtype=torch.int64, device=dev)
    rd = torch.zeros_like(rf)
    for off, cnt in ((0, 130), (130, 1), (131, 169)):
        assert prob.accumulate_coupled(nodes, cnt, 3e-3, rf, rd, path_offset=off,
                                       grid_id=pdd.PDD_CV_EXACT, seed=2, stream_tag=9) == 0
    fine, diff = prob.estimate_coupled(nodes, 300, 3e-3, grid_id=pdd.PDD_CV_EXACT, seed=2,
                                       stream_tag=9)
    for res, rec in ((fine, rf), (diff, rd)):
        got = ctx.finalize_records(rec)
        for f in pdd.STAT_FIELDS + pdd.COUNT_FIELDS:
            assert torch.equal(got[f], res[f]) or np.array_equal(
                got[f].cpu().numpy(), res[f].cpu().numpy(), equal_nan=True), f
    prob.close()
    ctx.close()


def test_mlmc_driver():
    torch, oracle, pdd = _env()
    ctx = pdd.Context(0)
    prob = pdd.Problem(ctx, pdd.PDD_PROBLEM_CFG0_2D)
    v = W.control_grid(0, 65, 1e-1)
    prob.set_control_grid(0, v)
    nodes = W.workload_nodes("c0")[::3]
    eps, dt0, base = 5e-3, 0.02, 40
    res = prob.mlmc(nodes, dt0, eps, grid_id=0, min_levels=2, max_levels=6, n_pilot=400,
                    stream_tag_base=base)
    assert res["status"] in (pdd.PDD_OK, pdd.PDD_WARN_NOT_CONVERGED)
    L, N = res["n_levels"], res["n_paths"]
    assert L >= 2 and np.all(N >= 400)
    # the counts meet the allocation rule on the driver's own level moments
    alloc = oracle.mlmc_allocation(res["var_mean"], res["cost_mean"], eps)
    assert np.all(N >= alloc)
    assert np.sum(res["var_mean"] / N) <= eps**2 / 2 * (1 + 1e-12)
    if res["status"] == pdd.PDD_OK:
        assert res["bias_estimate"] <= eps / np.sqrt(2)
    # the estimate is the sum of the level means of independent calls, bit for bit
    lv0 = prob.estimate(nodes, int(N[0]), dt0, grid_id=0, seed=1234, stream_tag=base)
    levels = [lv0]
    for l in range(1, L):
        _, d = prob.estimate_coupled(nodes, int(N[l]), dt0 / 2 ** (l - 1), grid_id=0, seed=1234,
                                     stream_tag=base + l)
        levels.append(d)
    est = np.zeros(len(nodes))
    var = np.zeros(len(nodes))
    steps = 0.0
    for l, r in enumerate(levels):
        est = est + r["mean_cv"].cpu().numpy()
        var = var + r["var_cv"].cpu().numpy() / N[l]
    assert np.array_equal(res["estimate"], est)
    assert np.allclose(res["variance"], var, rtol=1e-12, atol=0)
    m_last = levels[-1]["mean_cv"].cpu().numpy()
    assert np.allclose(res["extrapolated"], est + m_last, rtol=0, atol=1e-15)
    v_last = levels[-1]["var_cv"].cpu().numpy() / N[L - 1]
    assert np.allclose(res["extrap_variance"], var + 3 * v_last, rtol=1e-12, atol=0)
    # same arguments, same bits
    again = prob.mlmc(nodes, dt0, eps, grid_id=0, min_levels=2, max_levels=6, n_pilot=400,
                      stream_tag_base=base)
    assert np.array_equal(again["estimate"], res["estimate"])
    assert np.array_equal(again["n_paths"], N)
    # against the oracle's levels at the same counts (FP64 paths)
    m, vv, c = oracle.mlmc_levels(0, nodes, dt0, N, seed=1234, tag_base=base, cv=oracle.CV_GRID,
                                  grad=oracle.build_gradient(2, v), grid_n=65, controlled=True)
    ref = oracle.mlmc_combine(m, vv, N)
    se = np.sqrt(ref["variance"] + res["variance"])
    err = np.abs(res["estimate"] - ref["estimate"])
    assert np.all((err <= 1e-5 * np.abs(ref["estimate"])) | (err <= 3 * se)), err / se
    assert np.allclose(res["cost_mean"], np.maximum(c.mean(axis=1), 1.0), rtol=1e-3)
    assert res["path_steps"] == pytest.approx(float((c.sum(axis=1) * N).sum()), rel=1e-3)
    # the RMSE against the exact solution is of the order of the target
    u = W.exact_u(0, nodes.astype(np.float64))
    assert np.sqrt(np.mean((res["estimate"] - u) ** 2)) < 3 * eps
    prob.close()
    ctx.close()
