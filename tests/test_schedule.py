"""Algorithm 4 (scheduling by the sensitivity formula).

* The oracle's minimiser is pinned to a closed form: for one node with
  alpha = 0 the objective is K V (kappa c a^2 + (a_j/a)^p) with
  c = V[psi](1 - rho^2)/(4 V[phi]), p = 2 + 1/delta, whose minimum is at
  a^(p+2) = p a_j^p / (2 kappa c).
* The library's host implementation (pdd_schedule, no GPU involved) agrees
  with the oracle on multi-node constants, and stops where the predicted
  speedup falls below the threshold.
"""
import numpy as np
import pytest


def test_oracle_schedule_closed_form(oracle_mod):
    K, V, Vpsi, rho, kappa, delta, a0 = 2.0, 1.4, 50.0, 0.3, 1.8, 1.0, 0.01
    c = Vpsi * (1 - rho**2) / (4 * V)
    p = 2 + 1 / delta
    a, sp = oracle_mod.schedule([K], [-0.5], [0.0], [V], [Vpsi], [rho], delta, kappa, a0,
                                max_levels=1)
    want = (p * a0**p / (2 * kappa * c)) ** (1 / (p + 2))
    assert a[1] == pytest.approx(want, rel=1e-6)
    f = K * V * (kappa * c * want**2 + (a0 / want) ** p)
    assert sp[0] == pytest.approx(K * V / f, rel=1e-6)


def test_library_schedule_matches_oracle(oracle_mod):
    from paper_1512_02818_gb300 import build, pdd
    build.build()
    rng = np.random.default_rng(4)
    n = 18
    K = rng.uniform(0.5, 3, n)
    beta = rng.uniform(-1, -0.1, n)
    alpha = rng.uniform(-2, 2, n)
    V = rng.uniform(1, 6, n)
    Vpsi = rng.uniform(20, 80, n)
    rho = rng.uniform(-0.4, 0.4, n)
    for delta, kappa, a0 in ((1.0, 1.8, 0.01), (0.5, 1.3, 0.0025)):
        a_o, s_o = oracle_mod.schedule(K, beta, alpha, V, Vpsi, rho, delta, kappa, a0)
        a_l, s_l = pdd.pdd_schedule(K, beta, alpha, V, Vpsi, rho, delta, kappa, a0)
        assert len(a_l) == len(a_o) >= 2
        assert np.allclose(a_l, a_o, rtol=1e-6)
        assert np.allclose(s_l[: len(s_o)], s_o, rtol=1e-6)
        assert np.all(np.diff(a_l) > 0)
        assert np.all(s_l[:-1] >= 1.5) and (len(s_l) == len(a_l) - 1 or s_l[-1] < 1.5)
    with pytest.raises(pdd.PddError):
        pdd.pdd_schedule(K, beta, alpha, V, Vpsi, rho, 0.0, 1.0, 0.01)


def test_balanced_plan_meets_both_halves_of_the_tolerance():
    """eq. F:N_y_h: the time step puts the bias |beta| h^delta at a/2 and N is
    the least path count whose statistical error q sqrt(V/N) is at most a/2."""
    from paper_1512_02818_gb300 import build, pdd
    build.build()
    rng = np.random.default_rng(8)
    n = 40
    beta = rng.uniform(-3, 3, n)
    beta[0] = 0.0
    V = rng.uniform(1e-4, 5, n)
    V[1] = 0.0
    for a, q, delta in ((0.01, 2.0, 1.0), (0.003, 1.0, 0.5)):
        h, N = pdd.pdd_balanced_plan(a, beta, V, q=q, delta=delta, h_min=1e-9, h_max=0.5)
        free = (beta != 0) & (h > 1e-9) & (h < 0.5)
        assert np.allclose(np.abs(beta[free]) * h[free] ** delta, a / 2, rtol=1e-12)
        assert h[0] == 0.5  # beta = 0: no bias, largest step allowed
        pos = V > 0
        assert np.all(q * np.sqrt(V[pos] / N[pos]) <= a / 2 * (1 + 1e-12))
        big = pos & (N > 2)
        assert np.all(q * np.sqrt(V[big] / (N[big] - 1)) > a / 2)
        assert N[1] == 2  # no variance: the floor
    h, N = pdd.pdd_balanced_plan(1e-6, [1.0], [1.0], h_min=1e-4, h_max=1e-3, n_max=1000)
    assert h[0] == 1e-4 and N[0] == 1000  # clamped
    with pytest.raises(pdd.PddError):
        pdd.pdd_balanced_plan(0.0, [1.0], [1.0])


def test_schedule_prediction_sums_to_the_minimised_objective(oracle_mod):
    """Per-level predictions of the library (pdd_schedule_predict) against the
    oracle's Algorithm 4 objective: the controlled level's predicted cost times
    kappa plus the coarser plain level's cost, scaled by a_j^(2+1/delta), is
    the objective the oracle minimises; and the predicted rho^2 is r^2 minus
    the sensitivity formula's discretisation term."""
    from paper_1512_02818_gb300 import build, pdd
    build.build()
    rng = np.random.default_rng(9)
    n = 18
    K = rng.uniform(0.5, 3, n)
    beta = rng.uniform(-1, -0.1, n)
    alpha = rng.uniform(-2, 2, n)
    V = rng.uniform(1, 6, n)
    Vpsi = rng.uniform(20, 80, n)
    rho = rng.uniform(-0.4, 0.4, n)
    delta, kappa = 1.0, 1.4
    p = 2 + 1 / delta
    for a, aj in ((0.2, 0.01), (0.05, 0.02), (0.6, 0.1)):
        rho2, cost = pdd.pdd_schedule_predict(K, beta, alpha, V, Vpsi, rho, delta, a, aj)
        _, plain = pdd.pdd_schedule_predict(K, beta, alpha, V, Vpsi, rho, delta, -1.0, a)
        obj = oracle_mod.schedule_cost(a, aj, K, beta, alpha, V, Vpsi, rho, delta, kappa)
        assert (kappa * cost.sum() + plain.sum()) * aj**p == pytest.approx(obj, rel=1e-12)
        r2 = np.maximum(1 - Vpsi * a * a * (1 - rho**2) / (4 * V), 0)
        assert np.all(rho2 <= r2 + 1e-15) and np.all(rho2 >= 0)
        w = cost * aj**p / (K * V)  # 1 - r^2 + |alpha r / beta| a_j
        kept = w <= 1
        assert np.allclose(1 - rho2[kept], w[kept], rtol=1e-12)
        assert np.all(rho2[~kept] == 0)


def test_cascade_plan_groups_partition_the_nodes():
    """Host planning of the scheduled levels: every level's groups partition
    the nodes, are contiguous in the planned time step and fit the launch's
    segment limit together; the plain level is the coarsest."""
    from paper_1512_02818_gb300 import build
    from paper_1512_02818_gb300 import cascade as C
    build.build()
    rng = np.random.default_rng(12)
    n = 256
    fit = {"K": rng.uniform(0.5, 3, n), "beta": rng.uniform(-1, 1, n),
           "alpha": rng.uniform(-2, 2, n), "V_phi": rng.uniform(1, 2, n),
           "V_psi": rng.uniform(20, 80, n), "rho_phi_psi": rng.uniform(-0.4, 0.4, n)}
    a = [0.001, 0.01, 0.05, 0.2]
    levels = C.plan_levels(fit, a, h_min=1e-5, h_max=1e-2)
    assert sum(len(lv["groups"]) for lv in levels) <= 128
    assert [lv["controlled"] for lv in levels] == [True, True, True, False]
    for lv in levels:
        allidx = np.sort(np.concatenate(lv["groups"]))
        assert np.array_equal(allidx, np.arange(n))
        hs = [lv["h"][g] for g in lv["groups"]]
        for x, y in zip(hs, hs[1:]):
            assert x.max() <= y.min()
        assert np.all((lv["h"] >= 1e-5) & (lv["h"] <= 1e-2))
        assert np.all(lv["pred_path_steps"] > 0)


def test_cascade_regroup_is_the_cheapest_contiguous_cut():
    """After the pilot every node of a level has its N; the main launch cuts
    the nodes, in order of h or of N, into contiguous groups of least
    predicted cost (each group at its smallest h and largest N).  Brute force
    over every cut of tiny levels finds no cheaper grouping, and the groups
    partition the nodes."""
    import itertools

    from paper_1512_02818_gb300 import cascade as C
    rng = np.random.default_rng(5)
    for n, k in ((1, 3), (4, 2), (6, 3), (7, 4), (8, 8)):
        h = rng.uniform(1e-4, 1e-2, n)
        N = np.ceil(rng.lognormal(8.0, 1.0, n))
        e = rng.uniform(0.02, 0.2, n)
        groups, cost = C.regroup(h, N, e, k)
        assert np.array_equal(np.sort(np.concatenate(groups)), np.arange(n))
        assert len(groups) <= k
        assert np.isclose(C.grouped_cost(groups, h, N, e), cost, rtol=1e-12)
        best = np.inf
        for key in (h, N):
            order = np.argsort(key, kind="stable")
            for m in range(1, min(k, n) + 1):
                for cuts in itertools.combinations(range(1, n), m - 1):
                    bounds = (0,) + cuts + (n,)
                    gs = [order[bounds[i]:bounds[i + 1]] for i in range(m)]
                    best = min(best, C.grouped_cost(gs, h, N, e))
        assert cost <= best * (1 + 1e-12)
        assert cost >= best * (1 - 1e-12)
    # one group per node when there are enough segments: no inflation
    h = rng.uniform(1e-4, 1e-2, 5)
    N = rng.uniform(10, 1e4, 5)
    e = rng.uniform(0.02, 0.2, 5)
    groups, cost = C.regroup(h, N, e, 8)
    assert np.isclose(cost, np.sum(N * e / h), rtol=1e-12)


def test_unfit_nodes_are_left_out(oracle_mod):
    """A node with NaN constants (Algorithm 3 could not fit it) does not change
    the schedule: library and oracle give the sequence of the other nodes."""
    from paper_1512_02818_gb300 import build, pdd
    build.build()
    rng = np.random.default_rng(14)
    n = 12
    K = rng.uniform(0.5, 3, n)
    beta = rng.uniform(-1, -0.1, n)
    alpha = rng.uniform(-2, 2, n)
    V = rng.uniform(1, 6, n)
    Vpsi = rng.uniform(20, 80, n)
    rho = rng.uniform(-0.4, 0.4, n)
    args = (1.0, 1.4, 0.01)
    a_ref, s_ref = pdd.pdd_schedule(K, beta, alpha, V, Vpsi, rho, *args)
    o_ref, os_ref = oracle_mod.schedule(K, beta, alpha, V, Vpsi, rho, *args)
    nan = np.array([np.nan])
    ext = [np.concatenate([v, nan]) for v in (K, beta, alpha, V, Vpsi, rho)]
    a_nan, s_nan = pdd.pdd_schedule(*ext, *args)
    o_nan, os_nan = oracle_mod.schedule(*ext, *args)
    assert np.array_equal(a_nan, a_ref) and np.array_equal(s_nan, s_ref)
    assert np.allclose(o_nan, o_ref, rtol=1e-12) and np.allclose(os_nan, os_ref, rtol=1e-12)
    allnan = [np.full(3, np.nan) for _ in range(6)]
    with pytest.raises(pdd.PddError):
        pdd.pdd_schedule(*allnan, *args)
