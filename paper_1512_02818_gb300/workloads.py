"""Seeded synthetic inputs for the PDD Monte Carlo nodal stage.

This module holds no step of the method: it only lays out interfacial nodes
and samples the synthetic "previous iterate" v on a control grid.  Both the
CUDA library's tests/benchmark and the FP64 oracle receive these arrays as
inputs.

Workloads (all on the unit box, the boxes split into equal subdomains):

* ``c0`` -- 2D, 2x2 subdomains, 4 interface segments x 6 nodes = 24 nodes,
  10^4 paths, dt = 1e-3, no control variate.
* ``c1`` -- same problem, 4 x 64 = 256 nodes, 10^5 paths, dt = 1e-4, control
  grid 129^2 of v = u + eps sin(3 pi x) sin(2 pi y), eps in {1e-1,1e-2,1e-3}.
* ``c2`` -- 3D cube, 4^3 subdomains, 144 interior faces x 8x8 = 9,216 nodes,
  three levels (10^3, 10^4, 10^5 paths; dt 1e-2, 1e-3, 1e-4; eps 1e-1, 1e-2,
  1e-3 on a 65^3 grid, v = u + eps sin(3 pi x) sin(2 pi y) sin(pi z)).
* ``c4`` -- 2D anisotropic diffusion, 32x32 subdomains, 1,984 segments x 16 =
  31,744 nodes, 10^4 paths, dt = 1e-4, eps = 1e-2 on 513^2.
* ``paper`` -- the paper's example PDE on an assumed domain (its Fig. 1 is
  missing): the unit box cut into 4 vertical strips, 3 interfaces x 6 nodes =
  18 nodes.

Node placement on an interface segment of length L: n equispaced interior
points j L / (n+1), j = 1..n (end points excluded).  Canonical node order
(this order is the node index that keys the random streams): axis normal to
the interface, then interface index, then segment (face) index, then the
in-segment index.
"""
from __future__ import annotations

import math

import numpy as np

CFG0_2D, ANISO_2D, CUBE_3D, HARMONIC_2D, PAPER_EX_2D = 0, 1, 2, 3, 4


def nodes_2d(subdomains: int, per_segment: int) -> np.ndarray:
    """(n, 2) float32 interfacial nodes of [0,1]^2 split into S x S squares."""
    S, n = subdomains, per_segment
    L = 1.0 / S
    pts = []
    for axis in (0, 1):
        for i in range(1, S):
            for s in range(S):
                for j in range(1, n + 1):
                    a = i * L
                    t = s * L + j * L / (n + 1)
                    pts.append((a, t) if axis == 0 else (t, a))
    return np.asarray(pts, dtype=np.float32).reshape(-1, 2)


def nodes_strips(strips: int, per_interface: int) -> np.ndarray:
    """(n, 2) float32 nodes of [0,1]^2 cut into vertical strips: interfaces
    x = i/strips (i = 1..strips-1), per_interface interior points each."""
    pts = [(i / strips, j / (per_interface + 1)) for i in range(1, strips)
           for j in range(1, per_interface + 1)]
    return np.asarray(pts, dtype=np.float32).reshape(-1, 2)


def nodes_3d(subdomains: int, per_face: int) -> np.ndarray:
    """(n, 3) float32 interfacial nodes of [0,1]^3 split into S^3 cubes."""
    S, n = subdomains, per_face
    L = 1.0 / S
    pts = []
    for axis in (0, 1, 2):
        u_ax, w_ax = [a for a in (0, 1, 2) if a != axis]
        for i in range(1, S):
            for s in range(S):
                for t in range(S):
                    for p in range(n):
                        for q in range(n):
                            x = [0.0, 0.0, 0.0]
                            x[axis] = i * L
                            x[u_ax] = (s + (p + 1) / (n + 1)) * L
                            x[w_ax] = (t + (q + 1) / (n + 1)) * L
                            pts.append(tuple(x))
    return np.asarray(pts, dtype=np.float32).reshape(-1, 3)


def exact_u(kind: int, x: np.ndarray) -> np.ndarray:
    """Manufactured exact solution of each workload (for v grids and RMSE)."""
    x = np.asarray(x, dtype=np.float64)
    if kind in (CFG0_2D, ANISO_2D):
        return np.exp(x[..., 0] + x[..., 1]) * np.cos(x[..., 0] - x[..., 1])
    if kind == CUBE_3D:
        return (np.exp(x[..., 0]) * np.sin(x[..., 1]) * np.cos(x[..., 2])
                + x[..., 0] * x[..., 1] * x[..., 2])
    if kind == HARMONIC_2D:
        return x[..., 0] ** 2 - x[..., 1] ** 2
    if kind == PAPER_EX_2D:
        X, Y = x[..., 0], x[..., 1]
        return 2 * np.cos(2 * (Y - 2) * X) + np.sin(3 * (X - 2) * Y) + 3.1
    raise ValueError(kind)


def control_grid(kind: int, n: int, eps: float) -> np.ndarray:
    """Synthetic previous iterate v = u + eps * bump on n^D points of [0,1]^D.

    Returned as float64 array of shape (n, n) or (n, n, n), indexed [y, x] or
    [z, y, x] (x fastest in memory).  The bump vanishes on the boundary.
    """
    g = np.linspace(0.0, 1.0, n)
    if kind == CUBE_3D:
        Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
        pts = np.stack([X, Y, Z], axis=-1)
        bump = np.sin(3 * np.pi * X) * np.sin(2 * np.pi * Y) * np.sin(np.pi * Z)
    else:
        Y, X = np.meshgrid(g, g, indexing="ij")
        pts = np.stack([X, Y], axis=-1)
        bump = np.sin(3 * np.pi * X) * np.sin(2 * np.pi * Y)
    return np.ascontiguousarray(exact_u(kind, pts) + eps * bump)


WORKLOADS = {
    "c0": dict(kind=CFG0_2D, dim=2, subdomains=2, per_segment=6, n_paths=10_000, dt=1e-3,
               seed=1234, eps=None, grid_n=None),
    "c1": dict(kind=CFG0_2D, dim=2, subdomains=2, per_segment=64, n_paths=100_000, dt=1e-4,
               seed=1234, eps=[1e-1, 1e-2, 1e-3], grid_n=129),
    "c2": dict(kind=CUBE_3D, dim=3, subdomains=4, per_segment=8, seed=1234, grid_n=65,
               levels=[dict(n_paths=1_000, dt=1e-2, eps=1e-1),
                       dict(n_paths=10_000, dt=1e-3, eps=1e-2),
                       dict(n_paths=100_000, dt=1e-4, eps=1e-3)]),
    "c4": dict(kind=ANISO_2D, dim=2, subdomains=32, per_segment=16, n_paths=10_000, dt=1e-4,
               seed=1234, eps=[1e-2], grid_n=513),
}


def workload_nodes(name: str) -> np.ndarray:
    if name == "paper":
        return nodes_strips(4, 6)
    w = WORKLOADS[name]
    if w["dim"] == 3:
        return nodes_3d(w["subdomains"], w["per_segment"])
    return nodes_2d(w["subdomains"], w["per_segment"])


def random_interface_nodes(rng: np.random.Generator, count: int) -> np.ndarray:
    """Uniform positions on the 4 interface segments of the 2x2 split."""
    seg = rng.integers(0, 4, size=count)
    t = rng.uniform(0.02, 0.48, size=count) + 0.5 * (seg % 2)
    pts = np.where((seg // 2 == 0)[:, None], np.stack([np.full(count, 0.5), t], 1),
                   np.stack([t, np.full(count, 0.5)], 1))
    return pts.astype(np.float32)


def serving_requests(seed: int, rate_hz: float, window_s: float, max_nodes: int = 4096,
                     n_paths_range=(1e3, 1e6), dts=(1e-2, 1e-3, 1e-4),
                     eps_choices=(None, 1e-1, 1e-2)):
    """Poisson arrivals; log-uniform node counts and path counts; uniform dt
    and eps choices.  Returns a list of dicts sorted by arrival time."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate_hz)
        if t > window_s:
            break
        n_nodes = int(round(math.exp(rng.uniform(0.0, math.log(max_nodes)))))
        n_paths = int(round(math.exp(rng.uniform(math.log(n_paths_range[0]),
                                                 math.log(n_paths_range[1])))))
        out.append(dict(arrival=t, n_nodes=max(1, n_nodes), n_paths=max(2, n_paths),
                        dt=float(dts[rng.integers(0, len(dts))]),
                        eps=eps_choices[rng.integers(0, len(eps_choices))],
                        nodes=random_interface_nodes(rng, max(1, n_nodes)),
                        tag=len(out) + 1))
    return out
