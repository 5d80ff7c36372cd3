"""GPU-vs-oracle parity of the path kernels, through the C ABI.

Each case runs the CUDA path (libpdd.so via the ctypes binding) and the FP64
oracle on the same seeded inputs and Philox streams and compares per path
(exit index, phi, xi) and per node (means within 1e-5 relative or 3 combined
standard errors).  Sizes span many warps and a ragged tail (path counts not
multiples of 32) while keeping the oracle to seconds.
"""
import numpy as np
import pytest

from paper_1512_02818_gb300 import workloads as W
from parity import PATH_FRAC, compare_nodes, compare_paths, stats_from_paths

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import oracle
    from paper_1512_02818_gb300 import build, pdd
    build.build()
    oracle.build()
    ctx = pdd.Context(0)
    yield {"torch": torch, "oracle": oracle, "pdd": pdd, "ctx": ctx}
    ctx.close()


def _grid(env, prob, kind, n, eps, slot=0):
    v = W.control_grid(kind, n, eps)
    prob.set_control_grid(slot, v)
    dim = 3 if kind == W.CUBE_3D else 2
    return env["oracle"].build_gradient(dim, v)


CASES = [
    # name, kind, nodes (workload, stride, count), n_paths, dt, cv, grid (n, eps), exit, y_exp
    ("c0_plain", 0, ("c0", 1, 24), 1000, 1e-3, "none", None, "gm", False),
    ("c0_exact_cv", 0, ("c0", 1, 24), 1000, 1e-3, "exact", None, "gm", False),
    ("c1_grid_cv", 0, ("c1", 16, 16), 400, 1e-4, "grid", (129, 1e-2), "gm", False),
    ("c1_grid_cv_eps1", 0, ("c1", 32, 8), 333, 1e-3, "grid", (129, 1e-1), "gm", False),
    ("aniso_grid_cv", 1, ("c4", 997, 32), 300, 1e-3, "grid", (65, 1e-2), "gm", False),
    ("aniso_plain", 1, ("c4", 1999, 16), 300, 1e-3, "none", None, "gm", False),
    ("cube_grid_cv_h2", 2, ("c2", 389, 24), 300, 1e-2, "grid", (65, 1e-1), "gm", False),
    ("cube_grid_cv_h3", 2, ("c2", 769, 12), 200, 1e-3, "grid", (65, 1e-2), "gm", False),
    ("cube_exact_cv", 2, ("c2", 1531, 6), 250, 1e-3, "exact", None, "gm", False),
    ("harmonic_naive", 3, ("c0", 3, 8), 1000, 1e-3, "none", None, "naive", False),
    ("c0_yexp_exact", 0, ("c0", 3, 8), 500, 1e-3, "exact", None, "gm", True),
    ("paper_plain", 4, ("paper", 1, 18), 500, 1e-3, "none", None, "gm", False),
    ("paper_grid_cv", 4, ("paper", 1, 18), 400, 5e-4, "grid", (65, 1e-2), "gm", False),
    ("paper_exact_naive", 4, ("paper", 2, 9), 400, 1e-3, "exact", None, "naive", False),
]


def _run_case(env, case, precision=0, cells16=False):
    name, kind, (wl, stride, count), n_paths, dt, cv, grid, rule, y_exp = case
    pdd, oracle = env["pdd"], env["oracle"]
    nodes = W.workload_nodes(wl)[::stride][:count]
    prob = pdd.Problem(env["ctx"], kind,
                       exit_rule=pdd.PDD_EXIT_NAIVE if rule == "naive" else pdd.PDD_EXIT_GOBET_MENOZZI,
                       y_rule=pdd.PDD_Y_EXP if y_exp else pdd.PDD_Y_EULER, precision=precision)
    grad, gn, grid_id, ocv = None, 0, pdd.PDD_CV_NONE, oracle.CV_NONE
    if cv == "grid":
        gn = grid[0]
        grad = _grid(env, prob, kind, gn, grid[1])
        # FP32 3D paths read the binary16 cell table; they are compared with the
        # oracle's plain trilinear interpolation of the nodal table all the same
        grid_id, ocv = 0, (oracle.CV_GRID_CELLS16 if cells16 else oracle.CV_GRID)
    elif cv == "exact":
        grid_id, ocv = pdd.PDD_CV_EXACT, oracle.CV_EXACT
    g = prob.estimate(nodes, n_paths, dt, grid_id=grid_id, seed=1234, stream_tag=7,
                      emit_paths=True)
    env["torch"].cuda.synchronize()
    ref = oracle.estimate_nodes(kind, nodes, n_paths, dt, seed=1234, tag=7, cv=ocv, grad=grad,
                                grid_n=gn, c0=0.0 if rule == "naive" else oracle.GOBET_MENOZZI_C0,
                                y_exp=y_exp)
    prob.close()
    return g, ref


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_paths_and_nodes_match_oracle(env, case):
    g, ref = _run_case(env, case)
    assert g["status"] == 0
    p = compare_paths(g, ref)
    print(case[0], p)
    assert p["frac_ok"] >= PATH_FRAC, p
    n = compare_nodes(g, ref)
    assert n["mean_phi"]["ok"] and n["mean_cv"]["ok"], n
    # finalisation agrees with numpy statistics of the GPU's own per-path output
    s = stats_from_paths(g["phi"].cpu().numpy(), g["xi"].cpu().numpy(), g["steps"].cpu().numpy())
    for key, rtol in (("mean_phi", 1e-6), ("mean_cv", 1e-6), ("var_phi", 1e-4),
                      ("mean_steps", 1e-12)):
        assert np.allclose(g[key].cpu().numpy(), s[key], rtol=rtol, atol=1e-7), key
    assert np.allclose(g["var_cv"].cpu().numpy(), s["var_cv"], rtol=2e-3, atol=1e-9)
    assert np.all(g["n_paths"].cpu().numpy() == case[3])


CASES_3D_GRID = [c for c in CASES if c[1] == W.CUBE_3D and c[5] == "grid"]


@pytest.mark.parametrize("case", CASES_3D_GRID, ids=[c[0] for c in CASES_3D_GRID])
def test_3d_cell_table_error_budget(env, case):
    """Diagnostic split of the 3D FP32 error: against the oracle's model of
    the binary16 cell table the paths agree more tightly than against the
    plain trilinear table (which the parity test above uses), and the part
    the table's rounding adds stays well inside the per-path tolerance."""
    g, plain = _run_case(env, case)
    _, cells = _run_case(env, case, cells16=True)
    p_plain, p_cells = compare_paths(g, plain), compare_paths(g, cells)
    print(case[0], "trilinear", p_plain, "cells16", p_cells)
    assert p_cells["max_err_xi"] <= p_plain["max_err_xi"] + 1e-6
    assert p_plain["max_err_xi"] <= 0.5e-4
    gap = np.abs(plain["xi"] - cells["xi"])[plain["steps"] == cells["steps"]]
    assert gap.max() <= 3e-5, gap.max()


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_fp64_paths_match_oracle(env, case):
    g, ref = _run_case(env, case, precision=1)
    steps = g["steps"].cpu().numpy()
    assert (steps == ref["steps"]).mean() >= 0.9999
    same = steps == ref["steps"]
    # per-path outputs are emitted as FP32
    assert np.abs(g["phi"].cpu().numpy()[same] - ref["phi"][same]).max() < 2e-6
    if not np.all(same):
        return
    for m in ("mean_phi", "mean_cv"):
        d = np.abs(g[m].cpu().numpy() - ref[m])
        assert np.all(d <= 1e-8 * np.abs(ref[m]) + 1e-12), (m, (d / np.abs(ref[m])).max())
    assert np.allclose(g["var_phi"].cpu().numpy(), ref["var_phi"], rtol=1e-7)


def test_emit_flag_does_not_change_results(env):
    pdd = env["pdd"]
    nodes = W.workload_nodes("c0")
    prob = pdd.Problem(env["ctx"], pdd.PDD_PROBLEM_CFG0_2D)
    a = prob.estimate(nodes, 777, 1e-3, grid_id=pdd.PDD_CV_EXACT, emit_paths=True)
    b = prob.estimate(nodes, 777, 1e-3, grid_id=pdd.PDD_CV_EXACT)
    c = prob.estimate(nodes, 777, 1e-3, grid_id=pdd.PDD_CV_EXACT)
    for f in pdd.STAT_FIELDS + pdd.COUNT_FIELDS:
        x, y, z = (t[f].cpu().numpy() for t in (a, b, c))
        assert np.array_equal(x, y, equal_nan=True) and np.array_equal(y, z, equal_nan=True), f
    prob.close()


def test_host_and_device_buffers_agree(env):
    pdd = env["pdd"]
    nodes = W.workload_nodes("c0")
    prob = pdd.Problem(env["ctx"], pdd.PDD_PROBLEM_CFG0_2D)
    a = prob.estimate(nodes, 500, 1e-3)
    b = prob.estimate(nodes, 500, 1e-3, device_out=False, host_inputs=True)
    for f in pdd.STAT_FIELDS + pdd.COUNT_FIELDS:
        assert np.array_equal(a[f].cpu().numpy(), b[f].numpy(), equal_nan=True), f
    prob.close()


def test_async_flag_orders_on_stream(env):
    torch, pdd = env["torch"], env["pdd"]
    nodes = W.workload_nodes("c0")
    prob = pdd.Problem(env["ctx"], pdd.PDD_PROBLEM_CFG0_2D)
    a = prob.estimate_on_stream(nodes, 300, 1e-3, async_=True)
    env["ctx"].stream.synchronize()
    b = prob.estimate(nodes, 300, 1e-3)
    assert np.array_equal(a["mean_phi"].cpu().numpy(), b["mean_phi"].cpu().numpy())
    with pytest.raises(pdd.PddError):
        prob.estimate(nodes, 300, 1e-3, async_=True, host_inputs=True)
    prob.close()


def test_edge_cases(env):
    torch, pdd, oracle = env["torch"], env["pdd"], env["oracle"]
    prob = pdd.Problem(env["ctx"], pdd.PDD_PROBLEM_CFG0_2D)
    # empty input
    r = prob.estimate(np.zeros((0, 2), np.float32), 100, 1e-3)
    assert r["status"] == 0 and r["mean_phi"].numel() == 0
    # one path: the mean is that path's score, variances are undefined
    one = W.workload_nodes("c0")[:3]
    r = prob.estimate(one, 1, 1e-3, emit_paths=True)
    assert np.allclose(r["mean_phi"].cpu().numpy(), r["phi"].cpu().numpy()[:, 0], atol=1e-6)
    assert np.all(np.isnan(r["var_phi"].cpu().numpy()))
    # ragged single node
    r = prob.estimate(one[:1], 33, 1e-3, emit_paths=True)
    ref = oracle.estimate_nodes(0, one[:1], 33, 1e-3)
    assert compare_paths(r, ref)["frac_ok"] == 1.0
    # node already inside the shrinkage layer: zero steps, phi = g(Pi x0)
    near = np.array([[0.01, 0.6]], dtype=np.float32)
    r = prob.estimate(near, 64, 1e-3, emit_paths=True)
    assert np.all(r["steps"].cpu().numpy() == 0)
    gx = W.exact_u(0, np.array([0.0, np.float32(0.6)], dtype=np.float64))
    assert np.allclose(r["phi"].cpu().numpy(), gx, atol=1e-5)
    assert r["var_phi"].cpu().numpy()[0] == 0.0
    # plain run: xi = 0, rho undefined, vr = 1
    r = prob.estimate(one, 200, 1e-3)
    assert np.all(r["var_xi"].cpu().numpy() == 0.0)
    assert np.all(np.isnan(r["rho"].cpu().numpy()))
    assert np.all(r["vr"].cpu().numpy() == 1.0)
    # invalid arguments are rejected before any launch
    with pytest.raises(pdd.PddError) as e:
        prob.estimate(one, 100, 1e-3, grid_id=5)
    assert e.value.status == pdd.PDD_ERR_INVALID
    for bad in (dict(n_paths=0, dt=1e-3), dict(n_paths=10, dt=0.0), dict(n_paths=10, dt=-1.0)):
        with pytest.raises(pdd.PddError):
            prob.estimate(one, bad["n_paths"], bad["dt"])
    with pytest.raises(pdd.PddError):
        prob.set_control_grid(0, np.zeros((2, 2)))
    with pytest.raises(pdd.PddError):
        prob.set_control_grid(pdd.PDD_MAX_GRIDS, np.zeros((9, 9)))
    prob.close()


def test_truncation_reported(env):
    pdd, oracle = env["pdd"], env["oracle"]
    nodes = np.array([[0.5, 0.5], [0.5, 0.25]], dtype=np.float32)
    prob = pdd.Problem(env["ctx"], pdd.PDD_PROBLEM_CFG0_2D, max_steps=40)
    r = prob.estimate(nodes, 500, 1e-3, emit_paths=True)
    assert r["status"] == pdd.PDD_WARN_TRUNCATED
    ref = oracle.estimate_nodes(0, nodes, 500, 1e-3, max_steps=40)
    assert np.abs(r["n_truncated"].cpu().numpy() - ref["n_truncated"]).max() <= 1
    assert r["steps"].cpu().numpy().max() == 40
    prob.close()


def test_grid_gradient_table_matches_oracle(env):
    """VALUES grids are differentiated on the device; a GRADIENT grid built
    from the oracle's table must give the same paths bit for bit."""
    pdd, oracle = env["pdd"], env["oracle"]
    nodes = W.workload_nodes("c1")[::64]
    prob = pdd.Problem(env["ctx"], pdd.PDD_PROBLEM_CFG0_2D)
    v = W.control_grid(0, 33, 5e-2)
    prob.set_control_grid(0, v)
    prob.set_control_grid(1, oracle.build_gradient(2, v).reshape(33, 33, 2),
                          kind=pdd.PDD_GRID_GRADIENT)
    prob.set_control_grid(2, v.astype(np.float32))
    a = prob.estimate(nodes, 300, 1e-3, grid_id=0, emit_paths=True)
    b = prob.estimate(nodes, 300, 1e-3, grid_id=1, emit_paths=True)
    c = prob.estimate(nodes, 300, 1e-3, grid_id=2, emit_paths=True)
    # device differencing (FP64, FMA-contracted) vs the oracle's table: equal up to
    # the last bit of the FP32 rounding
    assert np.abs(a["xi"].cpu().numpy() - b["xi"].cpu().numpy()).max() < 1e-5
    assert np.array_equal(a["steps"].cpu().numpy(), b["steps"].cpu().numpy())
    # FP32 input values give a table within FP32 rounding of the FP64 one
    assert np.abs(a["xi"].cpu().numpy() - c["xi"].cpu().numpy()).max() < 1e-4
    prob.close()


def test_3d_cell_table_range(env):
    """FP32 3D paths read binary16 difference coefficients: a grid whose
    neighbouring gradient values differ by more than 65504 is refused for
    them and accepted for FP64 paths (which read the FP32 nodal table)."""
    pdd = env["pdd"]
    n = 9
    g = np.linspace(0, 1, n)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    v = 1e5 * X**2  # grad_x = 2e5 x: neighbours differ by 2.5e4 ... fine
    p32 = pdd.Problem(env["ctx"], pdd.PDD_PROBLEM_CUBE_3D)
    p32.set_control_grid(0, v)
    with pytest.raises(pdd.PddError) as e:
        p32.set_control_grid(1, 1e6 * X**2)  # neighbours differ by 2.5e5
    assert e.value.status == pdd.PDD_ERR_INVALID
    p64 = pdd.Problem(env["ctx"], pdd.PDD_PROBLEM_CUBE_3D, precision=pdd.PDD_PATH_FP64)
    p64.set_control_grid(1, 1e6 * X**2)
    p32.close()
    p64.close()
