"""Pins of the oracle's multilevel coupling.

* The fine half is Algorithm 1 at h/2 on the path's own stream: bit for bit
  the standard estimate at h/2.
* The coarse half is an Euler path at h driven by N(0,1) increments
  (n(2k) + n(2k+1)) / sqrt(2): its mean is that of an independent run at h,
  and its increments have unit variance.
* The level difference has a variance far below the score's and shrinking
  with h (strong coupling); with the exact control variate the controlled
  difference keeps the mean of the plain difference (E[xi] = 0 on each level).
"""
import math

import numpy as np
import pytest

from paper_1512_02818_gb300 import workloads as W


def test_fine_half_is_the_standard_path(oracle_mod):
    nodes = W.workload_nodes("c0")[:3]
    h = 2e-3
    c = oracle_mod.coupled_paths(0, nodes, 40, h, seed=5, tag=3, cv=oracle_mod.CV_EXACT)
    f = oracle_mod.estimate_nodes(0, nodes, 40, h / 2, seed=5, tag=3, cv=oracle_mod.CV_EXACT)
    assert np.array_equal(c["phi_f"], f["phi"]) and np.array_equal(c["steps_f"], f["steps"])
    assert np.array_equal(c["xi_f"], f["xi"])


def test_coarse_half_mean_and_strong_coupling(oracle_mod):
    node = W.workload_nodes("c0")[[4]]
    N = 6000
    res = {}
    for h in (8e-3, 2e-3):
        c = oracle_mod.coupled_paths(0, node, N, h, seed=9, tag=1)
        ind = oracle_mod.estimate_nodes(0, node, N, h, seed=9, tag=77, per_path=False)
        pc = c["phi_c"][0]
        se = math.sqrt(pc.var(ddof=1) / N + ind["var_phi"][0] / N)
        assert abs(pc.mean() - ind["mean_phi"][0]) < 4 * se
        d = c["phi_f"][0] - pc
        res[h] = d.var(ddof=1)
        assert res[h] < 0.25 * pc.var(ddof=1)
    assert res[2e-3] < res[8e-3]
    # the coarse normals combine two fine ones: unit variance, zero mean
    nn = np.array([(a + b) / math.sqrt(2) for a, b in
                   zip(oracle_mod.normals(9, 1, 0, 0, 2000, 0)[0::2],
                       oracle_mod.normals(9, 1, 0, 0, 2000, 0)[1::2])])
    assert abs(nn.var() - 1) < 0.15 and abs(nn.mean()) < 0.1


def test_controlled_difference_keeps_the_mean(oracle_mod):
    node = W.workload_nodes("c0")[[7]]
    N = 3000
    c = oracle_mod.coupled_paths(0, node, N, 4e-3, seed=2, tag=8, cv=oracle_mod.CV_EXACT)
    d_plain = c["phi_f"][0] - c["phi_c"][0]
    d_cv = d_plain + c["xi_f"][0] - c["xi_c"][0]
    se = math.sqrt(d_plain.var(ddof=1) / N)
    assert abs(d_cv.mean() - d_plain.mean()) < 4 * se + 1e-12
    assert d_cv.var() < d_plain.var()


# ---- 3D coupling -----------------------------------------------------------
def _interior_3d(count):
    nodes = W.workload_nodes("c2")
    d = np.minimum(nodes, 1.0 - nodes).min(axis=1)
    return nodes[np.argsort(-d)[:count]]


def test_fine_half_is_the_standard_path_3d(oracle_mod):
    nodes = _interior_3d(2)
    h = 4e-3
    c = oracle_mod.coupled_paths(2, nodes, 30, h, seed=5, tag=3, cv=oracle_mod.CV_EXACT)
    f = oracle_mod.estimate_nodes(2, nodes, 30, h / 2, seed=5, tag=3, cv=oracle_mod.CV_EXACT)
    assert np.array_equal(c["phi_f"], f["phi"]) and np.array_equal(c["steps_f"], f["steps"])
    assert np.array_equal(c["xi_f"], f["xi"])
    assert c["steps_f"].min() > 0 and c["steps_c"].min() > 0


def test_coarse_first_step_by_hand_3d(oracle_mod):
    """One coarse step at h from the cube's centre, written out: the
    increment is sqrt(h/2) (n(0..2) + n(3..5)) of the path's normal stream
    (fine steps 0 and 1), Y = 1 - h c, Z = -h f(X0) (b = 0, sigma = I)."""
    x0 = np.array([[0.5, 0.5, 0.5]])
    h = 0.5  # threshold c0 sqrt(h) = 0.41 < 0.5: the centre takes one step
    seen = 0
    for p in range(40):
        n = oracle_mod.normals(11, 2, 0, p, 6)
        x1 = x0[0] + math.sqrt(h / 2) * (n[:3] + n[3:6])
        d, _, _ = oracle_mod.box_distance(3, x1)
        if d < -oracle_mod.GOBET_MENOZZI_C0 * math.sqrt(h):
            continue  # a second step would follow; only one-step paths are checked
        seen += 1
        c = oracle_mod.coupled_paths(2, x0, p + 1, h, seed=11, tag=2)
        co = oracle_mod.coeffs(2, x0[0])
        g = W.exact_u(2, oracle_mod.box_project(3, x1)[None])[0]
        phi = g * (1.0 - h * co["c"]) - h * co["f"]
        assert c["steps_c"][0, p] == 1
        assert c["phi_c"][0, p] == pytest.approx(phi, rel=1e-13, abs=1e-13)
    assert seen >= 10


# ---- sample allocation and extrapolation -----------------------------------
def test_allocation_is_the_constrained_optimum(oracle_mod):
    V = np.array([1.4, 0.12, 0.035, 0.009])
    C = np.array([10.0, 31.0, 62.0, 124.0])
    eps = 2e-3
    N = oracle_mod.mlmc_allocation(V, C, eps)
    assert np.sum(V / N) <= eps**2 / 2 * (1 + 1e-12)
    # continuous optimum: N_l^2 C_l / V_l is the same for every level, and no
    # feasible perturbation that moves work between two levels is cheaper
    x = 2 / eps**2 * np.sqrt(V / C) * np.sum(np.sqrt(V * C))
    assert np.allclose(x**2 * C / V, (x**2 * C / V)[0], rtol=1e-12)
    assert np.sum(V / x) == pytest.approx(eps**2 / 2, rel=1e-12)
    cost = np.sum(x * C)
    rng = np.random.default_rng(0)
    for _ in range(200):
        i, j = rng.choice(4, 2, replace=False)
        y = x.copy()
        y[i] *= 1 + rng.uniform(-0.3, 0.3)
        # re-solve level j so that the variance budget stays exact
        rest = eps**2 / 2 - np.sum(np.delete(V / y, j))
        if rest <= 0:
            continue
        y[j] = V[j] / rest
        assert np.sum(y * C) >= cost * (1 - 1e-12)
    assert np.all(N == np.ceil(x).astype(np.int64))


def test_library_allocation_matches_oracle(oracle_mod):
    from paper_1512_02818_gb300 import build, pdd
    build.build()
    rng = np.random.default_rng(8)
    for L in (1, 2, 5, 16):
        V = rng.uniform(1e-4, 2.0, L)
        C = rng.uniform(1.0, 500.0, L)
        for eps in (1e-1, 3e-3):
            st, N = pdd.pdd_mlmc_allocate(V, C, eps)
            assert st == pdd.PDD_OK
            assert np.array_equal(N, oracle_mod.mlmc_allocation(V, C, eps))
    st, N = pdd.pdd_mlmc_allocate([1.0], [1.0], 1e-6)  # needs 2e12 paths
    assert st == pdd.PDD_WARN_NOT_CONVERGED and N[0] == 2**32 - 1
    with pytest.raises(pdd.PddError):
        pdd.pdd_mlmc_allocate([1.0, -1.0], [1.0, 1.0], 1e-2)
    with pytest.raises(pdd.PddError):
        pdd.pdd_mlmc_allocate([1.0], [0.0], 1e-2)


def test_richardson_removes_a_linear_bias(oracle_mod):
    """With E[phi_h] = u + c h exactly, level 0 at h0 and the correction
    E[phi_(h0/2)] - E[phi_h0]: the plain estimate keeps c h0 / 2, the
    extrapolation returns u."""
    u, c, h0 = np.array([1.3, -0.4]), np.array([0.7, 2.0]), 0.02
    m = np.array([u + c * h0, (u + c * h0 / 2) - (u + c * h0)])
    v = np.array([[0.5, 0.5], [0.01, 0.02]])
    r = oracle_mod.mlmc_combine(m, v, [100, 40])
    assert np.allclose(r["estimate"], u + c * h0 / 2, rtol=0, atol=1e-15)
    assert np.allclose(r["extrapolated"], u, rtol=0, atol=1e-15)
    assert np.allclose(r["variance"], v[0] / 100 + v[1] / 40)
    assert np.allclose(r["extrap_variance"], v[0] / 100 + 4 * v[1] / 40)


def test_levels_telescope_to_the_finest(oracle_mod):
    """sum_l m_l estimates E[phi_(h_L)]: against an independent run at h_L."""
    node = W.workload_nodes("c0")[[8]]
    counts = [4000, 2000, 1000]
    m, v, c = oracle_mod.mlmc_levels(0, node, 0.02, counts, seed=4, tag_base=20)
    est = m.sum(axis=0)[0]
    se = math.sqrt(float((v[:, 0] / np.array(counts)).sum()))
    ind = oracle_mod.estimate_nodes(0, node, 20000, 0.005, seed=4, tag=99, per_path=False)
    se2 = math.sqrt(se**2 + ind["var_phi"][0] / 20000)
    assert abs(est - ind["mean_phi"][0]) < 4 * se2
    # the corrections' variances fall with h (strong coupling) and the costs
    # grow like 1/h
    assert v[2, 0] < v[1, 0] < v[0, 0]
    assert c[2, 0] > 1.8 * c[1, 0] / 1.5
