"""FP64 CPU oracle for the Monte Carlo nodal stage of Probabilistic Domain
Decomposition (Bernal & Acebron, Sec. 2 and Algorithm 1).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline load it; the library never does.  The arithmetic lives in
``pdd_oracle.c`` (plain C, FP64, single-threaded); this module compiles it
with gcc on first use and wraps it with ctypes and numpy.

Parity pins (what fixes the oracle other than itself) are in
``tests/test_oracle_*.py``.  Functions with no independent pin: none of the
per-path arithmetic; the paper's Tables 2 and 3 are not reproduced (they need
the subdomain FEM/RBF stage and the missing Fig. 1 geometry) -- parity
unpinned for those, and they are out of scope.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pdd_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libpdd_oracle.so")
_lock = threading.Lock()
_lib = None

# problem kinds (same numbering as the library's public enum, by definition of
# the workloads, not by shared code)
CFG0_2D, ANISO_2D, CUBE_3D, HARMONIC_2D, PAPER_EX_2D = 0, 1, 2, 3, 4
CV_NONE, CV_GRID, CV_EXACT = 0, 1, 2
CV_GRID_CELLS16 = 3  # 3D grid as the FP32 paths read it (cell polynomials, binary16 differences)
GOBET_MENOZZI_C0 = 0.5826  # Algorithm 1, shrinkage constant as printed

STAT_NAMES = [
    "mean_phi", "var_phi", "mean_cv", "var_cv", "cov_phi_xi", "var_xi", "rho",
    "se_phi", "se_cv", "vr", "pred_speedup", "mean_steps", "n_truncated", "mean_iso",
    "mean_xi",
]


def build(force: bool = False) -> str:
    """Compile pdd_oracle.c into libpdd_oracle.so (gcc, -O2, strict IEEE)."""
    if force or not os.path.exists(_LIB_PATH) or (
        os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    ):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared",
             "-fno-fast-math", "-ffp-contract=off", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        u32, u64, i64, dbl, i32 = (ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64,
                                   ctypes.c_double, ctypes.c_int)
        P = ctypes.c_void_p
        lib.or_philox4x32_10.argtypes = [P, P, P]
        lib.or_uniform.argtypes = [u32]
        lib.or_uniform.restype = dbl
        lib.or_normal.argtypes = [u64, u32, u32, u32, u64]
        lib.or_normal.restype = dbl
        lib.or_eval.argtypes = [i32, P, P]
        lib.or_box_distance.argtypes = [i32, P, P, P]
        lib.or_box_distance.restype = dbl
        lib.or_box_project.argtypes = [i32, P, P]
        lib.or_build_gradient.argtypes = [i32, i32, P, P]
        lib.or_build_gradient.restype = i32
        lib.or_grad_interp.argtypes = [i32, i32, P, P, P]
        lib.or_grad_interp_cells16.argtypes = [i32, P, P, P]
        lib.or_round_f16.argtypes = [dbl]
        lib.or_round_f16.restype = dbl
        lib.or_nstat.restype = i32
        lib.or_node_stats.argtypes = [i64, P, P, P, P, P, dbl, P]
        lib.or_estimate_nodes.argtypes = [i32, dbl, i32, i64, i32, i32, P, i64, P, P, P, i64,
                                          dbl, u64, u32, dbl, P, P, P, P, P, P]
        lib.or_estimate_nodes.restype = i32
        lib.or_sample_paths.argtypes = [i32, dbl, i32, i64, i32, i32, P, i64, P, P, P, P, P,
                                        dbl, u64, u32, P, P, P]
        lib.or_sample_paths.restype = i32
        lib.or_coupled_paths.argtypes = [i32, dbl, i32, i64, i32, i32, P, i64, P, P, P, i64, dbl,
                                         u64, u32, P, P, P, P, P, P]
        lib.or_coupled_paths.restype = i32
        assert lib.or_nstat() == len(STAT_NAMES)
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def philox4x32_10(ctr, key) -> np.ndarray:
    """Philox4x32-10 block for one 128-bit counter and 64-bit key."""
    lib = _load()
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def uniform(x: int) -> float:
    return _load().or_uniform(int(x))


def normals(seed: int, tag: int, node: int, path: int, count: int, first: int = 0) -> np.ndarray:
    lib = _load()
    return np.array([lib.or_normal(seed, tag, node, path, first + i) for i in range(count)])


class Coeffs(ctypes.Structure):
    _fields_ = [("b", ctypes.c_double * 3), ("sigma", (ctypes.c_double * 3) * 3),
                ("A", (ctypes.c_double * 3) * 3), ("c", ctypes.c_double),
                ("f", ctypes.c_double), ("u", ctypes.c_double), ("grad_u", ctypes.c_double * 3)]


def coeffs(kind: int, x) -> dict:
    """Coefficients b, sigma, A, c, f, u, grad u of a workload at point x."""
    lib = _load()
    xx = np.zeros(3)
    xx[: len(x)] = x
    o = Coeffs()
    lib.or_eval(kind, _ptr(xx), ctypes.byref(o))
    return {"b": np.array(o.b[:]), "sigma": np.array([r[:] for r in o.sigma]),
            "A": np.array([r[:] for r in o.A]), "c": o.c, "f": o.f, "u": o.u,
            "grad_u": np.array(o.grad_u[:])}


def box_distance(dim: int, x):
    lib = _load()
    xx = np.zeros(3)
    xx[:dim] = x[:dim]
    ax, sd = ctypes.c_int(0), ctypes.c_int(0)
    d = lib.or_box_distance(dim, _ptr(xx), ctypes.byref(ax), ctypes.byref(sd))
    return d, ax.value, sd.value


def box_project(dim: int, x) -> np.ndarray:
    lib = _load()
    xx = np.zeros(3)
    xx[:dim] = x[:dim]
    out = np.zeros(3)
    lib.or_box_project(dim, _ptr(xx), _ptr(out))
    return out[:dim]


def build_gradient(dim: int, v: np.ndarray) -> np.ndarray:
    """Gradient table (n^D, D) of grid values v (x index fastest)."""
    lib = _load()
    n = v.shape[0]
    vv = np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
    grad = np.zeros(vv.size * dim)
    rc = lib.or_build_gradient(dim, n, _ptr(vv), _ptr(grad))
    if rc != 0:
        raise ValueError("bad grid")
    return grad


def grad_interp(dim: int, n: int, grad: np.ndarray, x) -> np.ndarray:
    lib = _load()
    xx = np.zeros(3)
    xx[:dim] = x[:dim]
    out = np.zeros(3)
    lib.or_grad_interp(dim, n, _ptr(grad), _ptr(xx), _ptr(out))
    return out[:dim]


def grad_interp_cells16(n: int, grad: np.ndarray, x) -> np.ndarray:
    """3D control-grid gradient through the cell polynomials with binary16
    difference coefficients (the FP32 paths' representation)."""
    lib = _load()
    xx = np.ascontiguousarray(x, dtype=np.float64)[:3].copy()
    out = np.zeros(3)
    lib.or_grad_interp_cells16(n, _ptr(np.ascontiguousarray(grad, dtype=np.float64)), _ptr(xx),
                               _ptr(out))
    return out


def round_f16(x: float) -> float:
    return _load().or_round_f16(float(x))


def problem_dim(kind: int) -> int:
    return 3 if kind == CUBE_3D else 2


def default_max_steps(h: float) -> int:
    """No cap in the paper; ceil(100 / h) steps, i.e. tau_h <= 100."""
    return int(np.ceil(100.0 / h))


def estimate_nodes(kind: int, nodes: np.ndarray, n_paths: int, h: float, seed: int = 1234,
                   tag: int = 0, cv: int = CV_NONE, grad: np.ndarray | None = None,
                   grid_n: int = 0, c0: float = GOBET_MENOZZI_C0, y_exp: bool = False,
                   max_steps: int | None = None, kappa: float = 1.0, per_path: bool = True):
    """Run Algorithm 1 for every (node, path) and return per-path arrays and
    per-node statistics.  nodes: (n_nodes, D) float array (any float dtype;
    the coordinates are used as given, in FP64)."""
    lib = _load()
    dim = problem_dim(kind)
    nodes = np.asarray(nodes, dtype=np.float64).reshape(-1, dim)
    n = nodes.shape[0]
    xs = np.ascontiguousarray(nodes[:, 0])
    ys = np.ascontiguousarray(nodes[:, 1])
    zs = np.ascontiguousarray(nodes[:, 2]) if dim == 3 else None
    if max_steps is None:
        max_steps = default_max_steps(h)
    tot = n * n_paths
    phi = np.zeros(tot) if per_path else None
    xi = np.zeros(tot) if per_path else None
    steps = np.zeros(tot, dtype=np.int64) if per_path else None
    iso = np.zeros(tot) if per_path else None
    xstop = np.zeros(tot * 3) if per_path else None
    stats = np.zeros(n * len(STAT_NAMES))
    if grad is not None:
        grad = np.ascontiguousarray(grad, dtype=np.float64)
    rc = lib.or_estimate_nodes(kind, c0, int(y_exp), int(max_steps), cv, grid_n, _ptr(grad), n,
                               _ptr(xs), _ptr(ys), _ptr(zs), int(n_paths), float(h), int(seed),
                               int(tag), float(kappa), _ptr(phi), _ptr(xi), _ptr(steps),
                               _ptr(iso), _ptr(xstop), _ptr(stats))
    if rc != 0:
        raise RuntimeError(f"or_estimate_nodes failed: {rc}")
    st = stats.reshape(n, len(STAT_NAMES))
    out = {name: st[:, j].copy() for j, name in enumerate(STAT_NAMES)}
    if per_path:
        out["phi"] = phi.reshape(n, n_paths)
        out["xi"] = xi.reshape(n, n_paths)
        out["steps"] = steps.reshape(n, n_paths)
        out["iso"] = iso.reshape(n, n_paths)
        out["x_stop"] = xstop.reshape(n, n_paths, 3)[:, :, :dim]
    return out


def sample_paths(kind: int, nodes: np.ndarray, node_idx, path_idx, h: float, seed: int = 1234,
                 tag: int = 0, cv: int = CV_NONE, grad: np.ndarray | None = None,
                 grid_n: int = 0, c0: float = GOBET_MENOZZI_C0, y_exp: bool = False,
                 max_steps: int | None = None):
    """Per-path (phi, xi, steps) for explicitly listed (node, path) pairs."""
    lib = _load()
    dim = problem_dim(kind)
    nodes = np.asarray(nodes, dtype=np.float64).reshape(-1, dim)
    node_idx = np.ascontiguousarray(node_idx, dtype=np.uint32)
    path_idx = np.ascontiguousarray(path_idx, dtype=np.uint32)
    sel = nodes[node_idx.astype(np.int64)]
    xs = np.ascontiguousarray(sel[:, 0])
    ys = np.ascontiguousarray(sel[:, 1])
    zs = np.ascontiguousarray(sel[:, 2]) if dim == 3 else None
    if max_steps is None:
        max_steps = default_max_steps(h)
    m = node_idx.size
    phi, xi, steps = np.zeros(m), np.zeros(m), np.zeros(m, dtype=np.int64)
    if grad is not None:
        grad = np.ascontiguousarray(grad, dtype=np.float64)
    lib.or_sample_paths(kind, c0, int(y_exp), int(max_steps), cv, grid_n, _ptr(grad), m,
                        _ptr(xs), _ptr(ys), _ptr(zs), _ptr(node_idx), _ptr(path_idx), float(h),
                        int(seed), int(tag), _ptr(phi), _ptr(xi), _ptr(steps))
    return {"phi": phi, "xi": xi, "steps": steps}


def node_stats(phi, xi, steps, kappa: float = 1.0) -> dict:
    """Per-node statistics of one node's per-path arrays (two-pass FP64)."""
    lib = _load()
    phi = np.ascontiguousarray(phi, dtype=np.float64)
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    steps = np.ascontiguousarray(steps, dtype=np.int64)
    n = phi.size
    tr = np.zeros(n, dtype=np.int32)
    iso = np.zeros(n)
    st = np.zeros(len(STAT_NAMES))
    lib.or_node_stats(n, _ptr(phi), _ptr(xi), _ptr(steps), _ptr(tr), _ptr(iso), float(kappa),
                      _ptr(st))
    return {name: st[j] for j, name in enumerate(STAT_NAMES)}


# ---------------------------------------------------------------------------
# Fast fit of nodal constants (Sec. 5 H5, Algorithm 3), plain numpy.
# ---------------------------------------------------------------------------
def ols_fit(x, y):
    """(intercept, slope) of y = a + b x: the normal-noise, identity-link GLM
    of the first-moment model, i.e. ordinary least squares."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    xm, ym = x.mean(), y.mean()
    sxx = float(((x - xm) ** 2).sum())
    b = float(((x - xm) * (y - ym)).sum()) / sxx if sxx > 0 else 0.0
    return ym - b * xm, b


def gamma_identity_fit(x, y, iters=200):
    """(intercept, slope) of E[y] = a + b x for gamma-distributed y (variance
    proportional to the mean squared), identity link: Fisher scoring, i.e.
    weighted least squares with weights 1/mu^2 recomputed from each fit."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    a, b = ols_fit(x, y)
    floor_mu = max(np.abs(y).min() * 1e-6, 1e-300)
    for _ in range(iters):
        mu = np.maximum(a + b * x, floor_mu)
        w = 1.0 / mu**2
        X = np.stack([np.ones_like(x), x], 1)
        A = X.T @ (w[:, None] * X)
        rhs = X.T @ (w * y)
        na, nb = np.linalg.solve(A, rhs)
        done = abs(na - a) + abs(nb - b) <= 1e-14 * (abs(na) + abs(nb) + 1e-300)
        a, b = float(na), float(nb)
        if done:
            break
    return a, b


def h_cloud(h_min, h_max, n_h):
    """Equispaced time steps h_max = h_1 > ... > h_{n_h} = h_min."""
    return np.array([h_max - (h_max - h_min) * j / (n_h - 1) for j in range(n_h)])


def fit_constants(kind, nodes, n_paths, h_min, h_max, n_h, delta=1.0, q=2.0, seed=1234,
                  tag_base=0, cv=CV_NONE, grad=None, grid_n=0, c0=GOBET_MENOZZI_C0):
    """Algorithm 3: per node, n_paths realisations at every h of the cloud
    (random streams keyed by tag_base + j for step j), then the moment fits.
    Returns a dict of per-node arrays and the cloud (n_nodes, n_h, 6):
    h, E[phi_h], V[phi_h], E[tau_h], Cov[phi_h, psi_h], V[psi_h]."""
    hs = h_cloud(h_min, h_max, n_h)
    dim = problem_dim(kind)
    nodes = np.asarray(nodes, dtype=np.float64).reshape(-1, dim)
    n = nodes.shape[0]
    cloud = np.zeros((n, n_h, 6))
    for j, h in enumerate(hs):
        r = estimate_nodes(kind, nodes, n_paths, h, seed=seed, tag=tag_base + j, cv=cv,
                           grad=grad, grid_n=grid_n, c0=c0, per_path=False)
        cloud[:, j, 0] = h
        cloud[:, j, 1] = r["mean_phi"]
        cloud[:, j, 2] = r["var_phi"]
        cloud[:, j, 3] = r["mean_steps"] * h
        cloud[:, j, 4] = r["cov_phi_xi"]
        cloud[:, j, 5] = r["var_xi"]
    x = hs**delta
    out = {k: np.zeros(n) for k in ("E_phi", "beta", "V_phi", "alpha", "E_tau", "K",
                                     "cov_phi_psi", "V_psi", "rho_phi_psi")}
    for i in range(n):
        out["E_phi"][i], out["beta"][i] = ols_fit(x, cloud[i, :, 1])
        out["E_tau"][i], _ = ols_fit(x, cloud[i, :, 3])
        out["V_phi"][i], out["alpha"][i] = gamma_identity_fit(x, cloud[i, :, 2])
        if cv != CV_NONE:
            out["cov_phi_psi"][i], _ = ols_fit(x, cloud[i, :, 4])
            out["V_psi"][i], _ = gamma_identity_fit(x, cloud[i, :, 5])
        else:
            out["cov_phi_psi"][i] = out["V_psi"][i] = np.nan
        out["rho_phi_psi"][i] = out["cov_phi_psi"][i] / np.sqrt(out["V_phi"][i] * out["V_psi"][i])
        # nodal cost constant of eq. F:Pointwise_cost
        out["K"][i] = 4 * q * q * out["E_tau"][i] * (2 * abs(out["beta"][i])) ** (1 / delta)
        # every path left at k = 0 at some h (mean exit time exactly 0, phi
        # deterministic: the node is inside the shrinkage layer there): the
        # fitted model does not hold
        if np.any(~(cloud[i, :, 3] > 0)):
            for k in out:
                out[k][i] = np.nan
    out["cloud"] = cloud
    return out


# ---------------------------------------------------------------------------
# Algorithm 4 (scheduling) with the sensitivity formula, plain numpy/scipy.
# ---------------------------------------------------------------------------
def schedule_cost(a, aj, K, beta, alpha, V_phi, V_psi, rho, delta, kappa):
    """Predicted cost of the level with tolerance aj when the control variate
    comes from the coarser level with tolerance a (Algorithm 4's objective)."""
    r2 = 1.0 - V_psi * a * a * (1.0 - rho * rho) / (4.0 * V_phi)
    r2 = np.maximum(r2, 0.0)
    r = np.sqrt(r2)
    p = 2.0 + 1.0 / delta
    return float(np.sum(K * V_phi * (kappa * (1.0 - r2 + np.abs(alpha * r / beta) * aj)
                                     + (aj / a) ** p)))


def schedule(K, beta, alpha, V_phi, V_psi, rho, delta, kappa, a0, min_speedup=1.5,
             max_levels=20):
    """Tolerance sequence a0 < a1 < ... and the predicted speedup of each
    step; stops when the predicted speedup drops below min_speedup."""
    from scipy import optimize
    K, beta, alpha, V_phi, V_psi, rho = (np.asarray(v, dtype=np.float64)
                                         for v in (K, beta, alpha, V_phi, V_psi, rho))
    # nodes with constants Algorithm 3 could not fit (NaN) are left out
    use = (np.isfinite(K) & np.isfinite(beta) & np.isfinite(alpha) & np.isfinite(V_phi)
           & np.isfinite(V_psi) & np.isfinite(rho) & (V_phi > 0) & (beta != 0))
    K, beta, alpha, V_phi, V_psi, rho = (v[use] for v in (K, beta, alpha, V_phi, V_psi, rho))
    plain = float(np.sum(K * V_phi))
    c = V_psi * (1 - rho * rho) / (4 * V_phi)
    amax = float(np.max(1 / np.sqrt(c[c > 0])))
    seq, sp = [a0], []
    aj = a0
    while len(seq) - 1 < max_levels and aj < amax:
        f = lambda la: schedule_cost(np.exp(la), aj, K, beta, alpha, V_phi, V_psi, rho, delta,
                                     kappa)
        grid = np.linspace(np.log(aj), np.log(amax), 4001)[1:]
        vals = np.array([f(g) for g in grid])
        k = int(np.argmin(vals))
        lo, hi = grid[max(k - 1, 0)], grid[min(k + 1, len(grid) - 1)]
        res = optimize.minimize_scalar(f, bounds=(lo, hi), method="bounded",
                                       options=dict(xatol=1e-12))
        best = res.x if res.fun <= vals[k] else grid[k]
        S = plain / min(res.fun, vals[k])
        sp.append(S)
        if S < min_speedup:
            break
        aj = float(np.exp(best))
        seq.append(aj)
    return np.array(seq), np.array(sp)


def coupled_paths(kind, nodes, n_paths, h, seed=1234, tag=0, cv=CV_NONE, grad=None, grid_n=0,
                  c0=GOBET_MENOZZI_C0, y_exp=False, max_steps=None):
    """Multilevel coupling: per (node, path) the fine path at h/2 (own normal
    stream) and the coarse path at h driven by the sums of pairs of fine
    increments.  Returns per-path arrays (n_nodes, n_paths)."""
    lib = _load()
    dim = 3 if kind == CUBE_3D else 2
    nodes = np.asarray(nodes, dtype=np.float64).reshape(-1, dim)
    n = nodes.shape[0]
    xs = np.ascontiguousarray(nodes[:, 0])
    ys = np.ascontiguousarray(nodes[:, 1])
    zs = np.ascontiguousarray(nodes[:, 2]) if dim == 3 else None
    if max_steps is None:
        max_steps = default_max_steps(0.5 * h)
    tot = n * n_paths
    out = {k: np.zeros(tot) for k in ("phi_f", "xi_f", "phi_c", "xi_c")}
    out["steps_f"] = np.zeros(tot, dtype=np.int64)
    out["steps_c"] = np.zeros(tot, dtype=np.int64)
    if grad is not None:
        grad = np.ascontiguousarray(grad, dtype=np.float64)
    rc = lib.or_coupled_paths(kind, c0, int(y_exp), int(max_steps), cv, grid_n, _ptr(grad), n,
                              _ptr(xs), _ptr(ys), _ptr(zs), int(n_paths), float(h), int(seed),
                              int(tag),
                              _ptr(out["phi_f"]), _ptr(out["xi_f"]), _ptr(out["steps_f"]),
                              _ptr(out["phi_c"]), _ptr(out["xi_c"]), _ptr(out["steps_c"]))
    if rc != 0:
        raise RuntimeError("or_coupled_paths failed")
    return {k: v.reshape(n, n_paths) for k, v in out.items()}


# ---------------------------------------------------------------------------
# Multilevel Monte Carlo on top of the coupled paths (the variant the paper
# names as future work, Sec. 1 and Sec. 7).
# ---------------------------------------------------------------------------
def mlmc_allocation(var_mean, cost_mean, target_rmse):
    """Sample counts of a multilevel estimator: minimise sum_l N_l C_l subject
    to sum_l V_l / N_l = eps^2 / 2.  Stationarity of the Lagrangian gives
    N_l = mu sqrt(V_l / C_l); the constraint fixes mu = 2 eps^-2
    sum_k sqrt(V_k C_k).  Rounded up, at least one path."""
    V = np.asarray(var_mean, dtype=np.float64)
    C = np.asarray(cost_mean, dtype=np.float64)
    mu = 2.0 / target_rmse**2 * np.sum(np.sqrt(V * C))
    return np.maximum(np.ceil(mu * np.sqrt(V / C)), 1.0).astype(np.int64)


def mlmc_levels(kind, nodes, dt0, counts, seed=1234, tag_base=0, cv=CV_NONE, grad=None,
                grid_n=0, controlled=False):
    """Per-node means, variances (N-1) and costs (exit indices per sample) of
    the multilevel levels with the given counts: level 0 is Algorithm 1 at
    dt0 (stream tag_base), level l >= 1 the coupled difference of a path at
    dt0 / 2^l and one at dt0 / 2^(l-1) (stream tag_base + l).  The score is
    phi, or phi + xi when `controlled`.  Returns arrays (levels, nodes)."""
    nodes = np.asarray(nodes, dtype=np.float64)
    m, v, c = [], [], []
    for l, N in enumerate(counts):
        if l == 0:
            r = estimate_nodes(kind, nodes, int(N), dt0, seed=seed, tag=tag_base, cv=cv, grad=grad,
                               grid_n=grid_n)
            s = r["phi"] + r["xi"] if controlled else r["phi"]
            cost = r["steps"].astype(np.float64)
        else:
            r = coupled_paths(kind, nodes, int(N), dt0 / 2.0 ** (l - 1), seed=seed,
                              tag=tag_base + l, cv=cv, grad=grad, grid_n=grid_n)
            sf = r["phi_f"] + r["xi_f"] if controlled else r["phi_f"]
            sc = r["phi_c"] + r["xi_c"] if controlled else r["phi_c"]
            s = sf - sc
            cost = (r["steps_f"] + r["steps_c"]).astype(np.float64)
        m.append(s.mean(axis=1))
        v.append(s.var(axis=1, ddof=1))
        c.append(cost.mean(axis=1))
    return np.array(m), np.array(v), np.array(c)


def mlmc_combine(m, v, counts, alpha=1.0):
    """The multilevel estimate sum_l m_l with variance sum_l v_l / N_l, and
    the Richardson (Talay-Tubaro) extrapolation on the finest pair: with
    E[phi_h] = u + c h^alpha + ..., the finest correction m_L estimates
    c h_L^alpha (2^alpha - 1), so u ~ estimate + m_L / (2^alpha - 1)."""
    m = np.asarray(m, dtype=np.float64)
    v = np.asarray(v, dtype=np.float64)
    N = np.asarray(counts, dtype=np.float64)[:, None]
    r = 2.0 ** alpha
    est = m.sum(axis=0)
    var = (v / N).sum(axis=0)
    ext = est + m[-1] / (r - 1.0)
    ext_var = var - v[-1] / N[-1] + (r / (r - 1.0)) ** 2 * v[-1] / N[-1]
    return {"estimate": est, "variance": var, "extrapolated": ext, "extrap_variance": ext_var}
