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
