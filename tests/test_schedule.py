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
