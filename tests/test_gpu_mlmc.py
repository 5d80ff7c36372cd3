"""Multilevel coupling on the GPU through the C ABI, against the oracle's
coupling on the same streams: per path (fine and coarse exit indices and
scores) and per node; the fine level equals pdd_estimate_nodes at dt/2 bit
for bit; the level difference has a small variance."""
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
    with pytest.raises(pdd.PddError):
        pdd.Problem(ctx, pdd.PDD_PROBLEM_CUBE_3D).estimate_coupled(
            W.workload_nodes("c2")[:2], 10, 1e-2)
    prob.close()
    ctx.close()
