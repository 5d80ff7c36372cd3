"""Pins of the oracle's path integrator (Algorithm 1) and nodal statistics.

Each check below is fixed by the paper or by mathematics, not by the oracle:

* zero-step exit: a start point already beyond the shrunken boundary finishes
  at k = 0 with phi = g(Pi x0) (Algorithm 1, the "finish" branch).
* one step (max_steps = 1): phi, xi, Y, Z written out by hand from the Euler
  step eq. F:E_M with the Feynman-Kac weights of eq. F:VR_Milstein_sys.
* harmonic data (b = c = f = 0, sigma = I): optional stopping of the discrete
  martingale X_k gives E[X_stop] = x0, E|X_stop - x0|^2 = D h E[k] (Wald), and
  E[x^2 - y^2](X_stop) = x0^2 - y0^2, at every h.
* exit time from the centre of the unit square against the torsion series
  E[tau] = 2 w(1/2,1/2), Delta w = -1 (Fourier series); Gobet-Menozzi has
  O(h) bias, the naive test O(sqrt h) (Sec. 2.3).
* manufactured solutions: E[phi_h] -> u(x0); the exact control variate
  (grad v = grad u) keeps the mean (E[xi] = 0, Sec. 2.3) and leaves a variance
  O(h) (eqs. F:Combining_method, F:VR_cap); Lemma 1's identities hold up to
  O(h).
* arbitrary grid: E[xi] = 0 and E[xi^2] = E[sum_k h Y_k^2 |sigma^T grad v|^2]
  (discrete Ito isometry, eq. F:Variance_VRSystem).
* per-node moments: numpy brute force from the per-path arrays.
"""
import math

import numpy as np
import pytest

from paper_1512_02818_gb300 import workloads as W

C0 = 0.5826


def test_zero_step_exit(oracle_mod):
    h = 0.04  # c0 sqrt(h) = 0.1165 > 0.1
    x0 = np.array([[0.1, 0.6]])
    r = oracle_mod.estimate_nodes(0, x0, 5, h)
    assert np.all(r["steps"] == 0)
    g = W.exact_u(0, np.array([0.0, 0.6]))
    assert np.allclose(r["phi"], g, rtol=1e-15)
    assert np.all(r["xi"] == 0.0)


def test_exit_tie_finishes(oracle_mod):
    """d_k equal to -c0 |sigma^T N| sqrt(h) finishes (first touch, Sec. 2.1)."""
    h = 0.01
    x0 = np.array([[C0 * math.sqrt(h), 0.5]])  # distance to the x = 0 face is exactly the threshold
    r = oracle_mod.estimate_nodes(0, x0, 3, h)
    assert np.all(r["steps"] == 0)
    x1 = np.array([[np.nextafter(C0 * math.sqrt(h), 1.0), 0.5]])
    assert np.all(oracle_mod.estimate_nodes(0, x1, 3, h)["steps"] > 0)


@pytest.mark.parametrize("kind", [0, 1, 2])
@pytest.mark.parametrize("y_exp", [False, True])
def test_one_step_by_hand(oracle_mod, kind, y_exp):
    dim = oracle_mod.problem_dim(kind)
    h = 1e-3
    x0 = np.array([0.5, 0.45, 0.4][:dim])
    seed, tag = 77, 2
    r = oracle_mod.estimate_nodes(kind, x0[None], 6, h, seed=seed, tag=tag, max_steps=1,
                                  cv=oracle_mod.CV_EXACT, y_exp=y_exp)
    o = oracle_mod.coeffs(kind, x0)
    sig = o["sigma"][:dim, :dim]
    for p in range(6):
        n = oracle_mod.normals(seed, tag, 0, p, dim)
        dW = math.sqrt(h) * n
        X1 = x0 + h * o["b"][:dim] + sig @ dW
        Y1 = math.exp(-h * o["c"]) if y_exp else 1.0 - h * o["c"]
        Z1 = -h * o["f"]
        g = W.exact_u(kind, oracle_mod.box_project(dim, X1))
        xi = -(sig.T @ o["grad_u"][:dim]) @ dW
        assert r["steps"][0, p] == 1
        assert r["phi"][0, p] == pytest.approx(g * Y1 + Z1, rel=1e-14)
        assert r["xi"][0, p] == pytest.approx(xi, rel=1e-13, abs=1e-16)
    assert r["n_truncated"][0] == 6


@pytest.mark.parametrize("c0", [C0, 0.0])
def test_harmonic_martingale_and_wald(oracle_mod, c0):
    h = 2e-3
    x0 = np.array([0.3, 0.6])
    N = 6000
    r = oracle_mod.estimate_nodes(3, x0[None], N, h, c0=c0)
    xs = r["x_stop"][0]
    k = r["steps"][0]
    assert k.min() >= 1
    for j in range(2):
        se = xs[:, j].std() / math.sqrt(N)
        assert abs(xs[:, j].mean() - x0[j]) < 4 * se
    disp2 = ((xs - x0) ** 2).sum(1)
    diff = disp2 - 2 * h * k  # zero-mean by Wald's identity
    assert abs(diff.mean()) < 4 * diff.std() / math.sqrt(N)
    gq = xs[:, 0] ** 2 - xs[:, 1] ** 2 - (x0[0] ** 2 - x0[1] ** 2)
    assert abs(gq.mean()) < 4 * gq.std() / math.sqrt(N)


def _torsion_centre():
    s = 0.0
    for m in range(1, 301, 2):
        for n in range(1, 301, 2):
            s += 16 / (math.pi**4 * m * n * (m * m + n * n)) * (-1) ** ((m - 1) // 2 + (n - 1) // 2)
    return 2 * s  # tau solves 1/2 Delta w = -1


def test_exit_time_torsion_series(oracle_mod):
    et = _torsion_centre()
    assert et == pytest.approx(0.14734, abs=2e-5)
    centre = np.array([[0.5, 0.5]])
    h = 1e-3
    N = 20000
    gm = oracle_mod.estimate_nodes(3, centre, N, h, c0=C0)["steps"][0] * h
    se = gm.std() / math.sqrt(N)
    assert abs(gm.mean() - et) < 3 * se + 2 * h
    h2 = 4e-3
    nv = oracle_mod.estimate_nodes(3, centre, 8000, h2, c0=0.0)["steps"][0] * h2
    se2 = nv.std() / math.sqrt(nv.size)
    # naive test: overshoot bias of order sqrt(h) -- clearly positive
    assert nv.mean() - et > 6 * se2


def test_manufactured_mean_and_exact_cv(oracle_mod):
    nodes = W.workload_nodes("c0")[[0, 5, 13]]
    u = W.exact_u(0, nodes.astype(np.float64))
    h = 1e-3
    N = 4000
    r = oracle_mod.estimate_nodes(0, nodes, N, h, cv=oracle_mod.CV_EXACT)
    # plain mean within the CLT band (bias O(h) is far below 3 SE here)
    assert np.all(np.abs(r["mean_phi"] - u) < 3.5 * r["se_phi"] + 5 * h)
    # exact CV: same mean, variance O(h)
    assert np.all(np.abs(r["mean_cv"] - u) < 4 * r["se_cv"] + 5 * h)
    assert np.all(r["var_cv"] < 0.02 * r["var_phi"])
    # Lemma 1: V[xi] = V[phi], Cov[phi, xi] = -V[phi], up to O(h)
    assert np.allclose(r["var_xi"], r["var_phi"], rtol=0.08)
    assert np.allclose(r["cov_phi_xi"], -r["var_phi"], rtol=0.08)
    assert np.all(r["rho"] < -0.98)


def test_exact_cv_variance_scales_with_h(oracle_mod):
    node = np.array([[0.5, 0.25]])
    ratios = []
    for h in (4e-3, 2e-3, 1e-3):
        r = oracle_mod.estimate_nodes(0, node, 3000, h, cv=oracle_mod.CV_EXACT, per_path=False)
        ratios.append(r["var_cv"][0] / h)
    ratios = np.array(ratios)
    # V[phi + xi] / h roughly constant (VR cap proportional to h)
    assert ratios.max() / ratios.min() < 1.6


def test_gobet_menozzi_bias_order(oracle_mod):
    """Exact CV makes the bias measurable: naive bias ~ sqrt(h), GM ~ h."""
    node = np.array([[0.5, 0.25]])
    u = float(W.exact_u(0, node.astype(np.float64))[0])
    hs = np.array([1e-2, 5e-3, 2.5e-3])
    bias = {}
    for name, c0 in (("gm", C0), ("naive", 0.0)):
        b = []
        for h in hs:
            r = oracle_mod.estimate_nodes(0, node, 6000, h, cv=oracle_mod.CV_EXACT, c0=c0,
                                          per_path=False)
            b.append(r["mean_cv"][0] - u)
        bias[name] = np.array(b)
    # naive: bias of one sign with a sqrt(h) law, clearly larger than GM's
    assert np.all(np.abs(bias["naive"]) > 3 * np.abs(bias["gm"]))
    slope = np.polyfit(np.log(hs), np.log(np.abs(bias["naive"])), 1)[0]
    assert 0.2 < slope < 0.8
    assert np.all(bias["naive"] > 0) and np.all(np.diff(bias["naive"]) < 0)


@pytest.mark.parametrize("eps", [1e-1, 1e-2])
def test_grid_cv_martingale_and_isometry(oracle_mod, eps):
    n = 33
    v = W.control_grid(0, n, eps)
    grad = oracle_mod.build_gradient(2, v)
    node = np.array([[0.5, 0.3]])
    N = 5000
    r = oracle_mod.estimate_nodes(0, node, N, 2e-3, cv=oracle_mod.CV_GRID, grad=grad, grid_n=n)
    xi = r["xi"][0]
    iso = r["iso"][0]
    assert abs(xi.mean()) < 4 * xi.std() / math.sqrt(N)
    d = xi**2 - iso
    assert abs(d.mean()) < 4 * d.std() / math.sqrt(N)
    assert r["var_cv"][0] < 0.1 * r["var_phi"][0]


def test_cv_variance_tracks_eps(oracle_mod):
    n = 65
    node = np.array([[0.5, 0.3]])
    vs = []
    for eps in (2e-1, 1e-1, 5e-2, 0.0):
        grad = oracle_mod.build_gradient(2, W.control_grid(0, n, eps))
        r = oracle_mod.estimate_nodes(0, node, 3000, 1e-3, cv=oracle_mod.CV_GRID, grad=grad,
                                      grid_n=n, per_path=False)
        vs.append(r["var_cv"][0])
    # eq. F:Variance_VRSystem: V[phi + xi] = E int Y^2 |sigma^T grad(u - v)|^2 dt + O(h);
    # with v - u = eps * bump the excess over the eps = 0 floor scales as eps^2
    excess = np.array(vs[:3]) - vs[3]
    assert np.all(excess > 0)
    ratios = excess[:-1] / excess[1:]
    assert np.all((ratios > 3.0) & (ratios < 5.3))


def test_node_stats_brute_force(oracle_mod):
    nodes = W.workload_nodes("c0")[:3]
    kappa = 1.7
    r = oracle_mod.estimate_nodes(0, nodes, 500, 2e-3, cv=oracle_mod.CV_EXACT, kappa=kappa)
    for i in range(3):
        phi, xi, k = r["phi"][i], r["xi"][i], r["steps"][i]
        psi = phi + xi
        assert r["mean_phi"][i] == pytest.approx(phi.mean(), rel=1e-13)
        assert r["var_phi"][i] == pytest.approx(phi.var(ddof=1), rel=1e-12)
        assert r["mean_cv"][i] == pytest.approx(psi.mean(), rel=1e-13)
        assert r["var_cv"][i] == pytest.approx(psi.var(ddof=1), rel=1e-11)
        assert r["var_xi"][i] == pytest.approx(xi.var(ddof=1), rel=1e-12)
        cov = np.cov(phi, xi, ddof=1)[0, 1]
        assert r["cov_phi_xi"][i] == pytest.approx(cov, rel=1e-12)
        assert r["rho"][i] == pytest.approx(np.corrcoef(phi, xi)[0, 1], rel=1e-12)
        assert r["se_phi"][i] == pytest.approx(math.sqrt(phi.var(ddof=1) / 500), rel=1e-12)
        assert r["vr"][i] == pytest.approx(psi.var(ddof=1) / phi.var(ddof=1), rel=1e-11)
        assert r["pred_speedup"][i] == pytest.approx(
            phi.var(ddof=1) / (kappa * psi.var(ddof=1)), rel=1e-11)
        assert r["mean_steps"][i] == pytest.approx(k.mean(), rel=1e-15)


def test_truncation_counted(oracle_mod):
    r = oracle_mod.estimate_nodes(0, np.array([[0.5, 0.5]]), 200, 1e-3, max_steps=40)
    k = r["steps"][0]
    assert k.max() == 40
    assert r["n_truncated"][0] == np.count_nonzero(k == 40)
    assert 0 < r["n_truncated"][0] < 200


def test_sample_paths_match_full_run(oracle_mod):
    nodes = W.workload_nodes("c0")[:4]
    r = oracle_mod.estimate_nodes(0, nodes, 50, 1e-3)
    ni = np.array([3, 0, 2, 1, 3])
    pi = np.array([49, 0, 17, 8, 2])
    s = oracle_mod.sample_paths(0, nodes, ni, pi, 1e-3)
    assert np.array_equal(s["phi"], r["phi"][ni, pi])
    assert np.array_equal(s["steps"], r["steps"][ni, pi])
