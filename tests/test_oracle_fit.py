"""Pins of the oracle's fits of nodal constants (Sec. 5 H5, Algorithm 3).

* The normal-identity GLM is ordinary least squares: numpy.polyfit.
* The gamma-identity GLM maximises the gamma likelihood: the deviance
  sum 2[-log(y/mu) + (y - mu)/mu] minimised by scipy.optimize reaches the same
  coefficients.
* Synthetic clouds with known constants are recovered; on a real node the
  fitted E[phi] matches the exact solution.
"""
import math

import numpy as np
import pytest

from paper_1512_02818_gb300 import workloads as W


def test_ols_is_polyfit(oracle_mod):
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 1, 30)
    y = 2.0 - 3.0 * x + rng.normal(0, 0.1, 30)
    a, b = oracle_mod.ols_fit(x, y)
    pb, pa = np.polyfit(x, y, 1)
    assert a == pytest.approx(pa, rel=1e-12) and b == pytest.approx(pb, rel=1e-12)


def test_gamma_identity_is_gamma_mle(oracle_mod):
    from scipy import optimize
    rng = np.random.default_rng(1)
    x = np.linspace(1e-3, 1e-2, 40)
    mu = 1.5 + 40.0 * x
    shape = (1000 - 1) / 2
    y = rng.gamma(shape, mu / shape)
    a, b = oracle_mod.gamma_identity_fit(x, y)

    def dev(p):
        m = p[0] + p[1] * x
        if np.any(m <= 0):
            return 1e300
        return float(np.sum(2 * (-np.log(y / m) + (y - m) / m)))

    res = optimize.minimize(dev, [1.0, 10.0], method="Nelder-Mead",
                            options=dict(xatol=1e-12, fatol=1e-14, maxiter=40000))
    assert a == pytest.approx(res.x[0], rel=1e-5)
    assert b == pytest.approx(res.x[1], rel=1e-3, abs=1e-3)
    # and the known constants are recovered within the sampling error
    se_a = 1.5 * math.sqrt(2 / 999 / 40) * 3
    assert abs(a - 1.5) < 4 * se_a


def test_fit_recovers_solution_and_exit_time(oracle_mod):
    node = W.workload_nodes("c0")[[3]]
    u = float(W.exact_u(0, node.astype(np.float64))[0])
    r = oracle_mod.fit_constants(0, node, 2000, 2e-3, 1e-2, 5, delta=1.0, cv=oracle_mod.CV_EXACT)
    c = r["cloud"][0]
    se = math.sqrt(np.mean(c[:, 2]) / 2000 / 5) * 3  # 3 x SE of the averaged intercept
    assert abs(r["E_phi"][0] - u) < 4 * se
    assert r["V_phi"][0] > 0 and r["E_tau"][0] > 0
    # exact control variate: Cov[phi, psi] = -V[phi] (Lemma 1), rho ~ -1
    assert r["rho_phi_psi"][0] < -0.98
    assert r["K"][0] > 0
    assert np.allclose(c[:, 0], oracle_mod.h_cloud(2e-3, 1e-2, 5))


def test_node_inside_shrinkage_layer_is_not_fitted(oracle_mod):
    """A node within c0 sqrt(h_max) of the boundary has every path leave at
    k = 0 at the coarse end of the cloud (mean exit time 0, phi deterministic): the
    fitted model does not hold and its constants are NaN, while a node away
    from the boundary in the same call is fitted."""
    nodes = np.array([[0.01, 0.5], [0.5, 0.3]], dtype=np.float32)
    r = oracle_mod.fit_constants(0, nodes, 200, 2e-3, 1e-2, 4, delta=1.0)
    c = r["cloud"][0]
    assert c[0, 3] == 0.0  # h = 1e-2: 0.5826 * 0.1 > 0.01, every path stops at once
    assert c[0, 2] < 1e-20  # phi is deterministic there
    for k in ("E_phi", "beta", "V_phi", "K", "E_tau"):
        assert np.isnan(r[k][0]) and np.isfinite(r[k][1]), k
