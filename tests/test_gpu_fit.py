"""Fast fit of nodal constants (Algorithm 3) on the GPU against the oracle's
fit on the same random streams: the clouds agree within the path tolerance
and the fitted constants within what those differences allow."""
import numpy as np
import pytest

from paper_1512_02818_gb300 import workloads as W
from parity import NODE_RTOL, PATH_FRAC, compare_paths

pytestmark = pytest.mark.gpu


def test_fit_constants_match_oracle():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import oracle
    from paper_1512_02818_gb300 import build, pdd
    build.build()
    oracle.build()
    ctx = pdd.Context(0)
    prob = pdd.Problem(ctx, pdd.PDD_PROBLEM_CFG0_2D)
    # synthetic error-propagation function w = sin(3 pi x) sin(2 pi y), zero on the boundary
    wg = W.control_grid(0, 65, 1.0) - W.control_grid(0, 65, 0.0)
    prob.set_control_grid(0, wg)
    nodes = W.workload_nodes("c0")[::4]
    kw = dict(n_paths=400, h_min=2e-3, h_max=1e-2, n_h=6, delta=1.0, q=2.0, seed=31)
    g = prob.fit_constants(nodes, grid_id=0, stream_tag_base=100, **kw)
    o = oracle.fit_constants(0, nodes, kw["n_paths"], kw["h_min"], kw["h_max"], kw["n_h"],
                             delta=1.0, q=2.0, seed=31, tag_base=100, cv=oracle.CV_GRID,
                             grad=oracle.build_gradient(2, wg), grid_n=65)
    assert g["status"] == 0
    assert np.allclose(g["cloud"][:, :, 0], o["cloud"][:, :, 0], rtol=0, atol=0)
    # One h of the cloud path by path: the fit runs h_j on the stream tagged
    # stream_tag_base + j, so the same estimate with per-path output must match
    # the oracle path by path, and its node means must be the fit's cloud
    # entries bit for bit (exact integer sums over the same paths).
    j = 3
    hj = float(g["cloud"][0, j, 0])
    one = prob.estimate(nodes, kw["n_paths"], hj, grid_id=0, seed=31, stream_tag=100 + j,
                        emit_paths=True)
    torch.cuda.synchronize()
    ref = oracle.estimate_nodes(0, nodes, kw["n_paths"], hj, seed=31, tag=100 + j,
                                cv=oracle.CV_GRID, grad=oracle.build_gradient(2, wg), grid_n=65)
    p = compare_paths(one, ref)
    assert p["frac_ok"] >= PATH_FRAC, p
    assert np.array_equal(one["mean_phi"].cpu().numpy(), g["cloud"][:, j, 1])
    assert np.array_equal(one["var_phi"].cpu().numpy(), g["cloud"][:, j, 2])
    # The whole cloud against the oracle's: means within the per-node rule
    # (1e-5 relative or 3 combined standard errors; the paths agree to FP32
    # rounding, so the sample means differ far less than that), the mean exit
    # time tau = k h exactly unless a path's exit step flipped (one flip moves
    # the mean by h / n_paths = 2.5e-5), and the second moments within 1 %
    se = np.sqrt(o["cloud"][:, :, 2] / kw["n_paths"])
    tol = np.maximum(NODE_RTOL * np.abs(o["cloud"][:, :, 1]), 3 * np.sqrt(2) * se)
    assert np.all(np.abs(g["cloud"][:, :, 1] - o["cloud"][:, :, 1]) <= tol)
    assert np.allclose(g["cloud"][:, :, 3], o["cloud"][:, :, 3], rtol=0,
                       atol=2 * 1e-2 / kw["n_paths"])
    for col in (2, 4, 5):
        assert np.allclose(g["cloud"][:, :, col], o["cloud"][:, :, col], rtol=1e-2,
                           atol=1e-6), col
    # fits are linear (or nearly) in the cloud: same constants up to those differences
    assert np.allclose(g["E_phi"], o["E_phi"], atol=5e-3)
    assert np.allclose(g["E_tau"], o["E_tau"], atol=1e-4)
    assert np.allclose(g["V_phi"], o["V_phi"], rtol=3e-2)
    assert np.allclose(g["V_psi"], o["V_psi"], rtol=3e-2)
    assert np.allclose(g["rho_phi_psi"], o["rho_phi_psi"], atol=2e-2)
    assert np.all(np.isfinite(g["K"])) and np.all(g["K"] > 0)
    with pytest.raises(pdd.PddError):
        prob.fit_constants(nodes, n_paths=10, h_min=1e-2, h_max=1e-3, n_h=4)
    prob.close()
    ctx.close()
