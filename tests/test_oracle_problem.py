"""Pins of the oracle's problem definitions, geometry and control-grid table.

* Coefficients: sympy differentiates each manufactured u and rebuilds
  f = 1/2 sum a_ij u_ij + b.grad u - c u from the generator of Sec. 2.1; the
  oracle's f, u and grad u must agree.  sigma sigma^T = A with sigma lower
  triangular (Cholesky, Sec. 2.1), and A is uniformly elliptic.
* Geometry: hand-placed points with known signed distance, projection and
  face (corners, edges, outside, on the boundary).
* Gradient table: centred and second-order one-sided differences are exact
  for quadratics, and multilinear interpolation reproduces the (affine)
  gradient of a quadratic exactly, up to the FP32 rounding of the table.
"""
import numpy as np
import pytest

sympy = pytest.importorskip("sympy")


def _sym_problem(kind):
    x, y, z = sympy.symbols("x y z", real=True)
    if kind in (0, 1):
        u = sympy.exp(x + y) * sympy.cos(x - y)
        b = [sympy.sin(y) / 2, sympy.cos(x) / 2]
        c = 1 + x**2 + y**2
        if kind == 0:
            A = sympy.eye(2)
        else:
            a = 1 + sympy.sin(2 * sympy.pi * x) / 2
            A = a * sympy.Matrix([[1, sympy.Rational(1, 2)], [sympy.Rational(1, 2), 1]])
        X = [x, y]
    elif kind == 2:
        u = sympy.exp(x) * sympy.sin(y) * sympy.cos(z) + x * y * z
        b = [0, 0, 0]
        c = sympy.Integer(1)
        A = sympy.eye(3)
        X = [x, y, z]
    elif kind == 4:  # the paper's example, eq. F:PDE_ejemplo (sigma = sqrt(2) I)
        u = 2 * sympy.cos(2 * (y - 2) * x) + sympy.sin(3 * (x - 2) * y) + sympy.Rational(31, 10)
        den = sympy.Rational(11, 10) + sympy.sin(x + y)
        b = [sympy.cos(x + y) / den, sympy.cos(x + y) / den]
        c = (x**2 + y**2) / den
        A = 2 * sympy.eye(2)
        X = [x, y]
    else:
        u = x**2 - y**2
        b = [0, 0]
        c = sympy.Integer(0)
        A = sympy.eye(2)
        X = [x, y]
    D = len(X)
    f = sum(sympy.Rational(1, 2) * A[i, j] * sympy.diff(u, X[i], X[j])
            for i in range(D) for j in range(D))
    f += sum(b[i] * sympy.diff(u, X[i]) for i in range(D)) - c * u
    grad = [sympy.diff(u, v) for v in X]
    return X, u, f, grad, A, b, c


@pytest.mark.parametrize("kind", [0, 1, 2, 3, 4])
def test_coefficients_solve_the_pde(oracle_mod, kind):
    X, u, f, grad, A, b, c = _sym_problem(kind)
    D = len(X)
    fu = sympy.lambdify(X, u)
    ff = sympy.lambdify(X, f)
    fg = [sympy.lambdify(X, g) for g in grad]
    fA = sympy.lambdify(X, A)
    fb = [sympy.lambdify(X, bi) for bi in b]
    fc = sympy.lambdify(X, c)
    rng = np.random.default_rng(kind)
    for _ in range(25):
        p = rng.uniform(-0.05, 1.05, size=D)
        o = oracle_mod.coeffs(kind, p)
        assert o["u"] == pytest.approx(fu(*p), rel=1e-13, abs=1e-13)
        assert o["f"] == pytest.approx(ff(*p), rel=1e-12, abs=1e-12)
        assert np.allclose(o["grad_u"][:D], [g(*p) for g in fg], rtol=1e-13, atol=1e-13)
        assert np.allclose(o["A"][:D, :D], np.array(fA(*p), dtype=float), rtol=1e-14)
        assert np.allclose(o["b"][:D], [bi(*p) for bi in fb], rtol=1e-14, atol=1e-15)
        assert o["c"] == pytest.approx(float(fc(*p)), rel=1e-14)
        s = o["sigma"][:D, :D]
        assert np.allclose(np.triu(s, 1), 0.0)
        assert np.allclose(s @ s.T, o["A"][:D, :D], rtol=1e-14, atol=1e-15)
        ev = np.linalg.eigvalsh(o["A"][:D, :D])
        assert ev.min() > 0.2 and ev.max() < 2.3  # aniso: 0.5a .. 1.5a, a in [.5, 1.5]


GEOM_CASES = [
    # (point, distance, axis, side, projection)
    ((0.5, 0.5), -0.5, 0, 0, (0.0, 0.5)),           # centre: tie -> axis 0, lo face
    ((0.1, 0.5), -0.1, 0, 0, (0.0, 0.5)),
    ((0.5, 0.93), -0.07, 1, 1, (0.5, 1.0)),
    ((0.2, 0.2), -0.2, 0, 0, (0.0, 0.2)),           # tie between axes -> axis 0
    ((0.8, 0.2), -0.2, 0, 1, (1.0, 0.2)),           # tie x-hi / y-lo -> axis 0 first
    ((0.0, 0.3), 0.0, 0, 0, (0.0, 0.3)),            # on the boundary
    ((-0.1, 0.5), 0.1, 0, 0, (0.0, 0.5)),           # outside, one coordinate
    ((1.3, -0.4), 0.5, 1, 0, (1.0, 0.0)),           # outside a corner: 0.3-0.4-0.5 triangle
    ((0.5, 0.5, 0.95), -0.05, 2, 1, (0.5, 0.5, 1.0)),
    ((1.2, 0.5, 1.1), np.hypot(0.2, 0.1), 0, 1, (1.0, 0.5, 1.0)),
]


@pytest.mark.parametrize("pt,dist,axis,side,proj", GEOM_CASES)
def test_box_geometry(oracle_mod, pt, dist, axis, side, proj):
    dim = len(pt)
    d, ax, sd = oracle_mod.box_distance(dim, np.array(pt, dtype=float))
    assert d == pytest.approx(dist, abs=1e-15)
    assert (ax, sd) == (axis, side)
    assert np.allclose(oracle_mod.box_project(dim, np.array(pt, dtype=float)), proj, atol=0)


@pytest.mark.parametrize("dim,n", [(2, 9), (2, 129), (3, 7)])
def test_gradient_table_exact_for_quadratics(oracle_mod, dim, n):
    g = np.linspace(0, 1, n)
    if dim == 2:
        Y, X = np.meshgrid(g, g, indexing="ij")
        v = 0.3 + X**2 + 3 * X * Y - 2 * Y**2 - 0.7 * X
        exact = lambda p: np.array([2 * p[0] + 3 * p[1] - 0.7, 3 * p[0] - 4 * p[1]])
        pts = np.stack([X, Y], -1).reshape(-1, 2)
    else:
        Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
        v = X * Y - Z**2 + 2 * X * Z + Y
        exact = lambda p: np.array([p[1] + 2 * p[2], p[0] + 1, -2 * p[2] + 2 * p[0]])
        pts = np.stack([X, Y, Z], -1).reshape(-1, 3)
    grad = oracle_mod.build_gradient(dim, v).reshape(-1, dim)
    ref = np.array([exact(p) for p in pts])
    # FP32 storage: relative rounding 2^-24, plus FP64 differencing noise
    assert np.allclose(grad, ref, rtol=2e-7, atol=1e-9)
    rng = np.random.default_rng(3)
    for _ in range(50):
        p = rng.uniform(0, 1, size=dim)
        gi = oracle_mod.grad_interp(dim, n, grad.reshape(-1), p)
        assert np.allclose(gi, exact(p), rtol=1e-6, atol=1e-6)
    # points on grid lines and at the far corner use the last cell
    corner = np.ones(dim)
    assert np.allclose(oracle_mod.grad_interp(dim, n, grad.reshape(-1), corner), exact(corner),
                       rtol=1e-6, atol=1e-6)


# ---- the 3D cell table of the FP32 paths (binary16 difference coefficients) --
def test_round_f16_matches_numpy(oracle_mod):
    rng = np.random.default_rng(5)
    mags = np.exp(rng.uniform(np.log(1e-9), np.log(7e4), 20000))
    xs = list(mags * rng.choice([-1.0, 1.0], mags.size))
    # exact ties between binary16 neighbours (normal and subnormal), and the overflow edge
    for e in (-20, -14, -3, 0, 7, 14):
        ulp = 2.0 ** max(e - 10, -24)
        for k in (1, 2, 3, 1023):
            xs.append((2.0**e) + (k + 0.5) * ulp)
    xs += [65504.0, 65519.99, 65520.0, 2.0**-24, 2.0**-25, 3 * 2.0**-26, 0.0, -0.0]
    with np.errstate(over="ignore"):
        ref = np.asarray(xs, dtype=np.float64).astype(np.float16).astype(np.float64)
    got = np.array([oracle_mod.round_f16(x) for x in xs])
    assert np.array_equal(got, ref)


def test_cells16_exact_for_dyadic_gradients(oracle_mod):
    """v = x^2 + 3y^2 + 5z^2 + xy + 2yz on 17^3 points: the nodal gradient is exact
    and all its cell differences are dyadic, so the binary16 cell polynomials
    reproduce grad v = (2x + y, 6y + x + 2z, 10z + 2y) exactly."""
    n = 17
    g = np.linspace(0, 1, n)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    v = X**2 + 3 * Y**2 + 5 * Z**2 + X * Y + 2 * Y * Z
    grad = oracle_mod.build_gradient(3, v)
    rng = np.random.default_rng(2)
    for _ in range(200):
        p = rng.uniform(0, 1, 3)
        want = np.array([2 * p[0] + p[1], 6 * p[1] + p[0] + 2 * p[2], 10 * p[2] + 2 * p[1]])
        assert np.allclose(oracle_mod.grad_interp_cells16(n, grad, p), want, rtol=0, atol=1e-13)
        assert np.allclose(oracle_mod.grad_interp(3, n, grad, p), want, rtol=0, atol=1e-13)


def test_cells16_within_the_rounding_bound(oracle_mod):
    """On a general smooth grid the cell polynomials differ from the exact
    trilinear interpolation only by the binary16 rounding of the seven
    difference coefficients: |err| <= sum_j |c_j| 2^-11 |monomial_j| per component."""
    n = 33
    v = __import__("paper_1512_02818_gb300.workloads", fromlist=["x"]).control_grid(2, n, 1e-1)
    grad = oracle_mod.build_gradient(3, v).reshape(n, n, n, 3)
    rng = np.random.default_rng(3)
    for _ in range(300):
        p = rng.uniform(0, 1, 3)
        t = p * (n - 1)
        i = np.minimum(np.floor(t).astype(int), n - 2)
        f = t - i
        c = grad[i[2]:i[2] + 2, i[1]:i[1] + 2, i[0]:i[0] + 2]  # [dz, dy, dx, comp]
        d = [c[0, 0, 1] - c[0, 0, 0], c[0, 1, 0] - c[0, 0, 0], c[1, 0, 0] - c[0, 0, 0],
             c[0, 1, 1] - c[0, 0, 1] - c[0, 1, 0] + c[0, 0, 0],
             c[1, 0, 1] - c[0, 0, 1] - c[1, 0, 0] + c[0, 0, 0],
             c[1, 1, 0] - c[0, 1, 0] - c[1, 0, 0] + c[0, 0, 0],
             c[1, 1, 1] - c[0, 1, 1] - c[1, 0, 1] - c[1, 1, 0] + c[0, 0, 1] + c[0, 1, 0]
             + c[1, 0, 0] - c[0, 0, 0]]
        mono = [f[0], f[1], f[2], f[0] * f[1], f[0] * f[2], f[1] * f[2], f[0] * f[1] * f[2]]
        bound = sum(np.abs(dj) * 2.0**-11 * m for dj, m in zip(d, mono)) + 1e-12
        err = np.abs(oracle_mod.grad_interp_cells16(n, grad.reshape(-1), p)
                     - oracle_mod.grad_interp(3, n, grad.reshape(-1), p))
        assert np.all(err <= bound), (err, bound)
        assert np.any(err > 0) or np.all(bound < 1e-9)
