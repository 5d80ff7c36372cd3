/*
 * pdd_oracle.c -- plain, single-threaded FP64 CPU oracle for the Monte Carlo
 * nodal stage of Probabilistic Domain Decomposition (Bernal & Acebron,
 * "A multigrid-like algorithm for probabilistic domain decomposition").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load this file.  It shares no code, header,
 * table or constant generator with the CUDA library: everything below is
 * written out again from the paper and from the published definition of the
 * Philox4x32-10 generator (Salmon, Moraes, Dror, Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3", SC'11).
 *
 * What it computes, per interfacial node x0 and path index p:
 *   - the Euler-Maruyama discretisation of the diffusion dX = b dt + sigma dW
 *     (Sec. 2.1, eq. F:SDE), stopped by the Gobet-Menozzi shrunken-boundary
 *     test or by the naive test (Algorithm 1);
 *   - the Feynman-Kac weights Y and Z of eq. F:Dynkin / eq. F:VR_Milstein_sys;
 *   - the pathwise control variate xi = -int Y sigma^T grad(v) . dW
 *     (eq. F:xiControlVariate, eq. F:ExactF with mu = 0);
 *   - the scores phi = g(X_tau) Y_tau + Z_tau and phi + xi, and the discrete
 *     Ito-isometry quadrature sum_k h Y_k^2 |sigma_k^T grad v(X_k)|^2
 *     (eq. F:Variance_VRSystem), which the tests compare with E[xi^2];
 *   - per-node two-pass FP64 moments (eqs. F:Statistics_VR .. F:Rho) and the
 *     predicted speedup V[phi] / (kappa V[phi+xi]) (eqs. F:Pointwise_cost,
 *     F:VR_Pointwise_cost).
 *
 * Sign convention: the PDE is  1/2 sum a_ij d_ij u + b.grad u - c u = f  with
 * c >= 0, i.e. the paper's c is replaced by -c.  Hence Y_{k+1} = Y_k (1 - h c_k)
 * (Euler, the paper's choice) or Y_k exp(-h c_k), and Z_{k+1} = Z_k - h Y_k f_k.
 *
 * Readings of the places where Algorithm 1 is garbled (the step condition is
 * printed the wrong way round; the xi update lacks its dW and sign; the Z
 * update adds xi): step while d_k < -c0 |sigma^T N_k| sqrt(h) and finish
 * otherwise; xi_{k+1} = xi_k - Y_k (sigma_k^T grad v(X_k)) . dW_k with the same
 * dW_k as the X step; Z_{k+1} = Z_k - h Y_k f_k, with xi kept separate.
 *
 * Domain: the unit box [0,1]^D (D = 2 or 3).  d(x) is the signed distance
 * (negative inside), Pi the closest boundary point, N the outward normal of
 * the face Pi lands on (corners: lowest axis first, the 0 face before the 1
 * face; outside the box: the face of the most violated coordinate).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11, Sec. 4 and Table 2).                */
/* Round function: with multipliers M0, M1 and round key (k0, k1),          */
/*   (c0,c1,c2,c3) -> (hi(M1*c2)^c1^k0, lo(M1*c2), hi(M0*c0)^c3^k1, lo(M0*c0)) */
/* and the key is bumped by the Weyl constants W0, W1 after every round.    */
/* W0 = frac(golden ratio) * 2^32 and W1 = (sqrt(3) - 1) * 2^32 (truncated). */
/* ------------------------------------------------------------------------ */
#define OR_PHILOX_M0 0xD2511F53u
#define OR_PHILOX_M1 0xCD9E8D57u
#define OR_PHILOX_W0 0x9E3779B9u
#define OR_PHILOX_W1 0xBB67AE85u

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)OR_PHILOX_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)OR_PHILOX_M1 * (uint64_t)c2;
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += OR_PHILOX_W0;
    k1 += OR_PHILOX_W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform in (0,1): the top 23 bits plus one half, scaled by 2^-23.  Every  */
/* value is exactly representable in FP32 and FP64.                          */
double or_uniform(uint32_t x) {
  return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* Normal number i of the stream of path (node, path): Philox block i/4 with  */
/* key (seed_lo, tag) and counter (i/4, path, node, seed_hi); words (w0,w1)   */
/* give the Box-Muller pair for positions 0,1 and (w2,w3) for positions 2,3:  */
/*   r = sqrt(-2 ln u_a), first = r cos(2 pi u_b), second = r sin(2 pi u_b).  */
double or_normal(uint64_t seed, uint32_t tag, uint32_t node, uint32_t path, uint64_t i) {
  uint32_t ctr[4] = {(uint32_t)(i / 4), path, node, (uint32_t)(seed >> 32)};
  uint32_t key[2] = {(uint32_t)seed, tag};
  uint32_t w[4];
  or_philox4x32_10(ctr, key, w);
  int pos = (int)(i % 4);
  int pair = pos / 2;
  double ua = or_uniform(w[2 * pair]);
  double ub = or_uniform(w[2 * pair + 1]);
  double r = sqrt(-2.0 * log(ua));
  const double two_pi = 6.283185307179586476925286766559;
  return (pos % 2 == 0) ? r * cos(two_pi * ub) : r * sin(two_pi * ub);
}

/* ------------------------------------------------------------------------ */
/* Problems (the synthetic workloads).  Each supplies the coefficients of    */
/* 1/2 sum a_ij d_ij u + b.grad u - c u = f, the diffusion matrix sigma with */
/* sigma sigma^T = A (lower Cholesky factor, Sec. 2.1), the Dirichlet data   */
/* g = u and the analytic gradient of u.                                     */
/* ------------------------------------------------------------------------ */
enum { OR_CFG0_2D = 0, OR_ANISO_2D = 1, OR_CUBE_3D = 2, OR_HARMONIC_2D = 3, OR_PAPER_EX_2D = 4 };

int or_problem_dim(int kind) { return kind == OR_CUBE_3D ? 3 : 2; }

typedef struct {
  double b[3];
  double sigma[3][3]; /* lower triangular */
  double A[3][3];
  double c, f, u, grad_u[3];
} or_coeffs;

/* u = e^{x+y} cos(x-y) and its gradient (harmonic in 2D). */
static void or_u_exp_cos(double x, double y, double* u, double g[2]) {
  double e = exp(x + y), t = x - y;
  *u = e * cos(t);
  g[0] = e * (cos(t) - sin(t));
  g[1] = e * (cos(t) + sin(t));
}

void or_eval(int kind, const double* x, or_coeffs* o) {
  memset(o, 0, sizeof(*o));
  if (kind == OR_CFG0_2D || kind == OR_ANISO_2D) {
    double u, gu[2];
    or_u_exp_cos(x[0], x[1], &u, gu);
    o->u = u; o->grad_u[0] = gu[0]; o->grad_u[1] = gu[1];
    o->b[0] = 0.5 * sin(x[1]);
    o->b[1] = 0.5 * cos(x[0]);
    o->c = 1.0 + x[0] * x[0] + x[1] * x[1];
    double a = 1.0;
    if (kind == OR_ANISO_2D) a = 1.0 + 0.5 * sin(2.0 * M_PI * x[0]);
    if (kind == OR_CFG0_2D) {
      o->A[0][0] = o->A[1][1] = 1.0;
      o->sigma[0][0] = o->sigma[1][1] = 1.0;
    } else {
      o->A[0][0] = o->A[1][1] = a;
      o->A[0][1] = o->A[1][0] = 0.5 * a;
      double sa = sqrt(a);
      o->sigma[0][0] = sa;
      o->sigma[1][0] = 0.5 * sa;
      o->sigma[1][1] = 0.5 * sqrt(3.0) * sa;
    }
    /* f = 1/2 sum a_ij u_ij + b.grad u - c u.  Delta u = 0; the only second  */
    /* derivative left for the anisotropic operator is the mixed one,         */
    /* u_xy = 2 e^{x+y} cos(x-y) = 2u, entering as 1/2 * 2 * (a/2) * u_xy.    */
    double second = 0.0;
    if (kind == OR_ANISO_2D) second = 0.5 * (o->A[0][1] + o->A[1][0]) * (2.0 * u);
    o->f = second + o->b[0] * gu[0] + o->b[1] * gu[1] - o->c * u;
  } else if (kind == OR_CUBE_3D) {
    double ex = exp(x[0]);
    double sy = sin(x[1]), cy = cos(x[1]), sz = sin(x[2]), cz = cos(x[2]);
    o->u = ex * sy * cz + x[0] * x[1] * x[2];
    o->grad_u[0] = ex * sy * cz + x[1] * x[2];
    o->grad_u[1] = ex * cy * cz + x[0] * x[2];
    o->grad_u[2] = -ex * sy * sz + x[0] * x[1];
    o->c = 1.0;
    for (int i = 0; i < 3; ++i) { o->A[i][i] = 1.0; o->sigma[i][i] = 1.0; }
    /* Delta u = -e^x sin y cos z (the xyz term is harmonic). */
    double lap = -ex * sy * cz;
    o->f = 0.5 * lap - o->c * o->u;
  } else if (kind == OR_PAPER_EX_2D) {
    /* The paper's example (Sec. 6): Laplacian + b.grad u - c u + f = 0 with
       sigma = sqrt(2) I (A = 2I), b = cos(x+y) [1,1] / (1.1 + sin(x+y)),
       c = (x^2 + y^2) / (1.1 + sin(x+y)) and exact
       u = 2 cos(2 (y-2) x) + sin(3 (x-2) y) + 3.1.  In the form
       1/2 sum a_ij u_ij + b.grad u - c u = f used here, f = -(the paper's f). */
    double x0 = x[0], y0 = x[1];
    double p = 2.0 * x0 * (y0 - 2.0), q = 3.0 * y0 * (x0 - 2.0);
    o->u = 2.0 * cos(p) + sin(q) + 3.1;
    o->grad_u[0] = -4.0 * (y0 - 2.0) * sin(p) + 3.0 * y0 * cos(q);
    o->grad_u[1] = -4.0 * x0 * sin(p) + 3.0 * (x0 - 2.0) * cos(q);
    double lap = -8.0 * ((y0 - 2.0) * (y0 - 2.0) + x0 * x0) * cos(p) -
                 9.0 * (y0 * y0 + (x0 - 2.0) * (x0 - 2.0)) * sin(q);
    double den = 1.1 + sin(x0 + y0);
    o->b[0] = o->b[1] = cos(x0 + y0) / den;
    o->c = (x0 * x0 + y0 * y0) / den;
    o->A[0][0] = o->A[1][1] = 2.0;
    o->sigma[0][0] = o->sigma[1][1] = sqrt(2.0);
    o->f = lap + o->b[0] * o->grad_u[0] + o->b[1] * o->grad_u[1] - o->c * o->u;
  } else { /* OR_HARMONIC_2D: b = c = f = 0, sigma = I, u = x^2 - y^2 */
    o->u = x[0] * x[0] - x[1] * x[1];
    o->grad_u[0] = 2.0 * x[0];
    o->grad_u[1] = -2.0 * x[1];
    o->A[0][0] = o->A[1][1] = 1.0;
    o->sigma[0][0] = o->sigma[1][1] = 1.0;
  }
}

/* ------------------------------------------------------------------------ */
/* Geometry of the unit box (Algorithm 1's distance map, projection, normal) */
/* ------------------------------------------------------------------------ */
/* Signed distance to the boundary of [0,1]^D (negative inside).  axis/side */
/* return the face used for the normal (side 0 = the x_axis = 0 face).      */
double or_box_distance(int dim, const double* x, int* axis, int* side) {
  int inside = 1;
  for (int j = 0; j < dim; ++j)
    if (x[j] < 0.0 || x[j] > 1.0) inside = 0;
  if (inside) {
    double best = INFINITY;
    int ba = 0, bs = 0;
    for (int j = 0; j < dim; ++j) {
      double dlo = x[j], dhi = 1.0 - x[j];
      if (dlo < best) { best = dlo; ba = j; bs = 0; }
      if (dhi < best) { best = dhi; ba = j; bs = 1; }
    }
    if (axis) *axis = ba;
    if (side) *side = bs;
    return -best;
  }
  double s2 = 0.0, worst = -1.0;
  int wa = 0, ws = 0;
  for (int j = 0; j < dim; ++j) {
    double ex = 0.0;
    int sd = 0;
    if (x[j] < 0.0) { ex = -x[j]; sd = 0; }
    else if (x[j] > 1.0) { ex = x[j] - 1.0; sd = 1; }
    s2 += ex * ex;
    if (ex > worst) { worst = ex; wa = j; ws = sd; }
  }
  if (axis) *axis = wa;
  if (side) *side = ws;
  return sqrt(s2);
}

/* Closest point of the boundary: clamp outside; inside, move the coordinate */
/* of the nearest face onto that face.                                       */
void or_box_project(int dim, const double* x, double* out) {
  int inside = 1;
  for (int j = 0; j < dim; ++j)
    if (x[j] < 0.0 || x[j] > 1.0) inside = 0;
  for (int j = 0; j < dim; ++j) out[j] = x[j];
  if (!inside) {
    for (int j = 0; j < dim; ++j) out[j] = x[j] < 0.0 ? 0.0 : (x[j] > 1.0 ? 1.0 : x[j]);
    return;
  }
  int axis = 0, side = 0;
  or_box_distance(dim, x, &axis, &side);
  out[axis] = side ? 1.0 : 0.0;
}

/* ------------------------------------------------------------------------ */
/* Control grid: gradient table of a previous iterate v sampled on n^D      */
/* equispaced points of [0,1]^D (x index fastest).  Centred differences     */
/* inside, second-order one-sided differences on the edges; each component */
/* is rounded to FP32 (the precision the table is stored in) and returned   */
/* in FP64.  Layout: grad[point * D + component].                            */
/* ------------------------------------------------------------------------ */
int or_build_gradient(int dim, int n, const double* v, double* grad) {
  if (n < 3 || (dim != 2 && dim != 3)) return -1;
  double delta = 1.0 / (double)(n - 1);
  long npts = (dim == 2) ? (long)n * n : (long)n * n * n;
  long stride[3] = {1, n, (long)n * n};
  for (long pt = 0; pt < npts; ++pt) {
    long idx[3] = {pt % n, (pt / n) % n, (dim == 3) ? pt / ((long)n * n) : 0};
    for (int a = 0; a < dim; ++a) {
      long i = idx[a], s = stride[a];
      double d;
      if (i == 0)
        d = (-3.0 * v[pt] + 4.0 * v[pt + s] - v[pt + 2 * s]) / (2.0 * delta);
      else if (i == n - 1)
        d = (3.0 * v[pt] - 4.0 * v[pt - s] + v[pt - 2 * s]) / (2.0 * delta);
      else
        d = (v[pt + s] - v[pt - s]) / (2.0 * delta);
      grad[pt * dim + a] = (double)(float)d;
    }
  }
  return 0;
}

/* Multilinear interpolation of the gradient table at x (cell index clamped */
/* to [0, n-2]).                                                             */
void or_grad_interp(int dim, int n, const double* grad, const double* x, double* out) {
  long i[3];
  double w[3];
  for (int a = 0; a < dim; ++a) {
    double t = x[a] * (double)(n - 1);
    long c = (long)floor(t);
    if (c < 0) c = 0;
    if (c > n - 2) c = n - 2;
    i[a] = c;
    w[a] = t - (double)c;
  }
  for (int comp = 0; comp < dim; ++comp) out[comp] = 0.0;
  int corners = 1 << dim;
  for (int cnr = 0; cnr < corners; ++cnr) {
    double wt = 1.0;
    long pt = 0, mul = 1;
    for (int a = 0; a < dim; ++a) {
      int bit = (cnr >> a) & 1;
      wt *= bit ? w[a] : (1.0 - w[a]);
      pt += (i[a] + bit) * mul;
      mul *= n;
    }
    for (int comp = 0; comp < dim; ++comp) out[comp] += wt * grad[pt * dim + comp];
  }
}

/* Nearest IEEE 754 binary16 value of x (ties to even), returned as a double. */
/* binary16 keeps 11 significant bits for |x| >= 2^-14 and the fixed quantum  */
/* 2^-24 below it; results above the largest finite value 65504 overflow to  */
/* infinity.                                                                 */
double or_round_f16(double x) {
  if (x == 0.0 || !isfinite(x)) return x;
  double ax = fabs(x);
  int e;
  frexp(ax, &e);        /* ax = m 2^e, m in [0.5, 1): ulp of a normal = 2^(e - 11) */
  int q = e - 11;
  if (q < -24) q = -24; /* subnormal range */
  double r = ldexp(rint(ldexp(ax, -q)), q); /* rint: ties to even */
  if (r > 65504.0) r = INFINITY;
  return copysign(r, x);
}

/* Gradient of the 3D control grid as the FP32 paths see it: per cell, the   */
/* trilinear polynomial of every component, g = c000 + c100 fx + c010 fy +   */
/* c001 fz + c110 fx fy + c101 fx fz + c011 fy fz + c111 fx fy fz, with the  */
/* coefficients formed from the 8 corner values of the (FP32-rounded) nodal  */
/* table, c000 kept as is and the seven others rounded to binary16.          */
void or_grad_interp_cells16(int n, const double* grad, const double* x, double* out) {
  long i[3];
  double f[3];
  for (int a = 0; a < 3; ++a) {
    double t = x[a] * (double)(n - 1);
    long c = (long)floor(t);
    if (c < 0) c = 0;
    if (c > n - 2) c = n - 2;
    i[a] = c;
    f[a] = t - (double)c;
  }
  for (int comp = 0; comp < 3; ++comp) {
    double v[2][2][2]; /* [dz][dy][dx] */
    for (int dz = 0; dz < 2; ++dz)
      for (int dy = 0; dy < 2; ++dy)
        for (int dx = 0; dx < 2; ++dx) {
          long pt = ((i[2] + dz) * (long)n + (i[1] + dy)) * (long)n + (i[0] + dx);
          v[dz][dy][dx] = grad[pt * 3 + comp];
        }
    double c000 = v[0][0][0];
    double c100 = or_round_f16(v[0][0][1] - c000);
    double c010 = or_round_f16(v[0][1][0] - c000);
    double c001 = or_round_f16(v[1][0][0] - c000);
    double c110 = or_round_f16(v[0][1][1] - v[0][0][1] - v[0][1][0] + c000);
    double c101 = or_round_f16(v[1][0][1] - v[0][0][1] - v[1][0][0] + c000);
    double c011 = or_round_f16(v[1][1][0] - v[0][1][0] - v[1][0][0] + c000);
    double c111 = or_round_f16(v[1][1][1] - v[0][1][1] - v[1][0][1] - v[1][1][0] + v[0][0][1] +
                               v[0][1][0] + v[1][0][0] - c000);
    out[comp] = c000 + c100 * f[0] + c010 * f[1] + c001 * f[2] + c110 * f[0] * f[1] +
                c101 * f[0] * f[2] + c011 * f[1] * f[2] + c111 * f[0] * f[1] * f[2];
  }
}

/* ------------------------------------------------------------------------ */
/* One path of Algorithm 1.                                                  */
/* ------------------------------------------------------------------------ */
/* OR_CV_GRID: multilinear interpolation of the nodal gradient table;        */
/* OR_CV_GRID_CELLS16: the 3D cell polynomials above (binary16 differences). */
enum { OR_CV_NONE = 0, OR_CV_GRID = 1, OR_CV_EXACT = 2, OR_CV_GRID_CELLS16 = 3 };

typedef struct {
  int kind;          /* OR_CFG0_2D ... */
  double c0;         /* 0.5826 (Gobet-Menozzi) or 0 (naive test) */
  int y_exp;         /* 0: Y *= 1 - h c (Euler, as printed); 1: Y *= exp(-h c) */
  int64_t max_steps; /* truncation cap */
  int cv_mode;       /* OR_CV_* */
  int grid_n;        /* points per axis of the control grid */
  const double* grad;/* gradient table (or_build_gradient layout) */
} or_problem;

typedef struct {
  double phi;        /* g(Pi X_tau) Y_tau + Z_tau */
  double xi;         /* control variate */
  double iso;        /* sum_k h Y_k^2 |sigma_k^T grad v(X_k)|^2 */
  double y, z;       /* Y_tau, Z_tau */
  double x_stop[3];  /* X at the stopping index (unprojected) */
  double x_exit[3];  /* Pi(X_stop) */
  int64_t steps;     /* stopping index k */
  int truncated;     /* 1 if stopped by max_steps */
} or_path;

void or_simulate_path(const or_problem* pb, const double* x0, double h, uint64_t seed,
                      uint32_t tag, uint32_t node, uint32_t path, or_path* res) {
  int dim = or_problem_dim(pb->kind);
  double X[3] = {0, 0, 0};
  for (int j = 0; j < dim; ++j) X[j] = x0[j];
  double Y = 1.0, Z = 0.0, xi = 0.0, iso = 0.0;
  double sqh = sqrt(h);
  int64_t k = 0;
  int trunc = 0;
  or_coeffs o;
  for (;;) {
    int axis = 0, side = 0;
    double d = or_box_distance(dim, X, &axis, &side);
    or_eval(pb->kind, X, &o);
    /* |sigma^T N| for the axis-aligned unit normal N = +-e_axis */
    double s = sqrt(o.A[axis][axis]);
    if (d >= -pb->c0 * s * sqh) break; /* finish: on or beyond the shrunken boundary */
    double n[3], dW[3], sdW[3] = {0, 0, 0};
    for (int j = 0; j < dim; ++j) {
      n[j] = or_normal(seed, tag, node, path, (uint64_t)dim * (uint64_t)k + (uint64_t)j);
      dW[j] = sqh * n[j];
    }
    for (int i = 0; i < dim; ++i)
      for (int j = 0; j <= i; ++j) sdW[i] += o.sigma[i][j] * dW[j];
    if (pb->cv_mode != OR_CV_NONE) {
      double gv[3] = {0, 0, 0};
      if (pb->cv_mode == OR_CV_GRID) or_grad_interp(dim, pb->grid_n, pb->grad, X, gv);
      else if (pb->cv_mode == OR_CV_GRID_CELLS16) or_grad_interp_cells16(pb->grid_n, pb->grad, X, gv);
      else for (int j = 0; j < dim; ++j) gv[j] = o.grad_u[j];
      double dot = 0.0, st2 = 0.0;
      for (int i = 0; i < dim; ++i) dot += gv[i] * sdW[i];
      for (int j = 0; j < dim; ++j) { /* (sigma^T grad v)_j */
        double sj = 0.0;
        for (int i = 0; i < dim; ++i) sj += o.sigma[i][j] * gv[i];
        st2 += sj * sj;
      }
      xi -= Y * dot;
      iso += h * Y * Y * st2;
    }
    Z -= h * Y * o.f;
    for (int j = 0; j < dim; ++j) X[j] += h * o.b[j] + sdW[j];
    Y *= pb->y_exp ? exp(-h * o.c) : (1.0 - h * o.c);
    k += 1;
    if (k >= pb->max_steps) { trunc = 1; break; }
  }
  double P[3] = {0, 0, 0};
  or_box_project(dim, X, P);
  or_coeffs oe;
  or_eval(pb->kind, P, &oe);
  res->phi = oe.u * Y + Z;
  res->xi = xi;
  res->iso = iso;
  res->y = Y;
  res->z = Z;
  for (int j = 0; j < 3; ++j) { res->x_stop[j] = X[j]; res->x_exit[j] = P[j]; }
  res->steps = k;
  res->truncated = trunc;
}

/* ------------------------------------------------------------------------ */
/* Multilevel coupling (the multilevel Monte Carlo variant the paper names as */
/* future work): the fine path runs Algorithm 1 at h/2 on the path's own      */
/* normal stream; the coarse path runs it at h with increment                  */
/* dW_c(k) = dW_f(2k) + dW_f(2k+1), i.e. normals (n(2k) + n(2k+1)) / sqrt(2)   */
/* per component.  Each path has its own exit.                                 */
/* ------------------------------------------------------------------------ */
typedef struct {
  double phi_f, xi_f, phi_c, xi_c;
  int64_t steps_f, steps_c;
} or_coupled;

static void or_run_path(const or_problem* pb, const double* x0, double h, uint64_t seed,
                        uint32_t tag, uint32_t node, uint32_t path, int coarse, or_path* res) {
  int dim = or_problem_dim(pb->kind);
  double X[3] = {0, 0, 0};
  for (int j = 0; j < dim; ++j) X[j] = x0[j];
  double Y = 1.0, Z = 0.0, xi = 0.0;
  double sqh = sqrt(h);
  int64_t k = 0;
  int trunc = 0;
  or_coeffs o;
  for (;;) {
    int axis = 0, side = 0;
    double d = or_box_distance(dim, X, &axis, &side);
    or_eval(pb->kind, X, &o);
    double s = sqrt(o.A[axis][axis]);
    if (d >= -pb->c0 * s * sqh) break;
    double n[3], dW[3], sdW[3] = {0, 0, 0};
    for (int j = 0; j < dim; ++j) {
      if (coarse) {
        double a = or_normal(seed, tag, node, path, (uint64_t)dim * (uint64_t)(2 * k) + (uint64_t)j);
        double b = or_normal(seed, tag, node, path, (uint64_t)dim * (uint64_t)(2 * k + 1) + (uint64_t)j);
        n[j] = (a + b) / sqrt(2.0);
      } else {
        n[j] = or_normal(seed, tag, node, path, (uint64_t)dim * (uint64_t)k + (uint64_t)j);
      }
      dW[j] = sqh * n[j];
    }
    for (int i = 0; i < dim; ++i)
      for (int j = 0; j <= i; ++j) sdW[i] += o.sigma[i][j] * dW[j];
    if (pb->cv_mode != OR_CV_NONE) {
      double gv[3] = {0, 0, 0};
      if (pb->cv_mode == OR_CV_GRID) or_grad_interp(dim, pb->grid_n, pb->grad, X, gv);
      else if (pb->cv_mode == OR_CV_GRID_CELLS16) or_grad_interp_cells16(pb->grid_n, pb->grad, X, gv);
      else for (int j = 0; j < dim; ++j) gv[j] = o.grad_u[j];
      double dot = 0.0;
      for (int i = 0; i < dim; ++i) dot += gv[i] * sdW[i];
      xi -= Y * dot;
    }
    Z -= h * Y * o.f;
    for (int j = 0; j < dim; ++j) X[j] += h * o.b[j] + sdW[j];
    Y *= pb->y_exp ? exp(-h * o.c) : (1.0 - h * o.c);
    k += 1;
    if (k >= pb->max_steps) { trunc = 1; break; }
  }
  double P[3] = {0, 0, 0};
  or_box_project(dim, X, P);
  or_coeffs oe;
  or_eval(pb->kind, P, &oe);
  res->phi = oe.u * Y + Z;
  res->xi = xi;
  res->steps = k;
  res->truncated = trunc;
}

/* Coupled pairs for n_nodes x n_paths; h is the COARSE step (fine: h/2).    */
/* Per-path outputs indexed node * n_paths + path; max_steps caps each path. */
int or_coupled_paths(int kind, double c0, int y_exp, int64_t max_steps, int cv_mode, int grid_n,
                     const double* grad, int64_t n_nodes, const double* xs, const double* ys,
                     const double* zs, int64_t n_paths, double h, uint64_t seed, uint32_t tag,
                     double* phi_f, double* xi_f, int64_t* steps_f, double* phi_c, double* xi_c,
                     int64_t* steps_c) {
  or_problem pb = {kind, c0, y_exp, max_steps, cv_mode, grid_n, grad};
  if (or_problem_dim(kind) == 3 && zs == NULL) return -1;
  for (int64_t i = 0; i < n_nodes; ++i) {
    double x0[3] = {xs[i], ys[i], zs ? zs[i] : 0.0};
    for (int64_t p = 0; p < n_paths; ++p) {
      or_path f, c;
      or_run_path(&pb, x0, 0.5 * h, seed, tag, (uint32_t)i, (uint32_t)p, 0, &f);
      or_run_path(&pb, x0, h, seed, tag, (uint32_t)i, (uint32_t)p, 1, &c);
      int64_t q = i * n_paths + p;
      phi_f[q] = f.phi; xi_f[q] = f.xi; steps_f[q] = f.steps;
      phi_c[q] = c.phi; xi_c[q] = c.xi; steps_c[q] = c.steps;
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Per-node statistics from the per-path scores: plain two-pass FP64        */
/* sample moments with the N-1 normalisation.                                */
/* Output columns (stats[node * OR_NSTAT + col]):                            */
/* ------------------------------------------------------------------------ */
enum {
  OR_MEAN_PHI = 0, OR_VAR_PHI, OR_MEAN_CV, OR_VAR_CV, OR_COV_PHI_XI, OR_VAR_XI, OR_RHO,
  OR_SE_PHI, OR_SE_CV, OR_VR, OR_PRED_SPEEDUP, OR_MEAN_STEPS, OR_N_TRUNC, OR_MEAN_ISO,
  OR_MEAN_XI, OR_NSTAT
};

int or_nstat(void) { return OR_NSTAT; }

void or_node_stats(int64_t n, const double* phi, const double* xi, const int64_t* steps,
                   const int* trunc, const double* iso, double kappa, double* st) {
  double nd = (double)n;
  double mphi = 0, mcv = 0, mxi = 0, msteps = 0, miso = 0;
  double ntr = 0;
  for (int64_t p = 0; p < n; ++p) {
    mphi += phi[p];
    mcv += phi[p] + xi[p];
    mxi += xi[p];
    msteps += (double)steps[p];
    miso += iso[p];
    ntr += trunc[p];
  }
  mphi /= nd; mcv /= nd; mxi /= nd; msteps /= nd; miso /= nd;
  double vphi = 0, vcv = 0, vxi = 0, cpx = 0;
  for (int64_t p = 0; p < n; ++p) {
    double a = phi[p] - mphi, b = phi[p] + xi[p] - mcv, c = xi[p] - mxi;
    vphi += a * a;
    vcv += b * b;
    vxi += c * c;
    cpx += a * c;
  }
  vphi /= (nd - 1.0); vcv /= (nd - 1.0); vxi /= (nd - 1.0); cpx /= (nd - 1.0);
  st[OR_MEAN_PHI] = mphi;
  st[OR_VAR_PHI] = vphi;
  st[OR_MEAN_CV] = mcv;
  st[OR_VAR_CV] = vcv;
  st[OR_COV_PHI_XI] = cpx;
  st[OR_VAR_XI] = vxi;
  st[OR_RHO] = cpx / sqrt(vphi * vxi);
  st[OR_SE_PHI] = sqrt(vphi / nd);
  st[OR_SE_CV] = sqrt(vcv / nd);
  st[OR_VR] = vcv / vphi;
  st[OR_PRED_SPEEDUP] = vphi / (kappa * vcv);
  st[OR_MEAN_STEPS] = msteps;
  st[OR_N_TRUNC] = ntr;
  st[OR_MEAN_ISO] = miso;
  st[OR_MEAN_XI] = mxi;
}

/* ------------------------------------------------------------------------ */
/* Whole estimate: n_nodes nodes (SoA coordinates), n_paths paths each.      */
/* Per-path outputs (any may be NULL) are indexed node * n_paths + path.     */
/* stats (may be NULL) receives OR_NSTAT doubles per node.                   */
/* ------------------------------------------------------------------------ */
int or_estimate_nodes(int kind, double c0, int y_exp, int64_t max_steps, int cv_mode, int grid_n,
                      const double* grad, int64_t n_nodes, const double* xs, const double* ys,
                      const double* zs, int64_t n_paths, double h, uint64_t seed, uint32_t tag,
                      double kappa, double* out_phi, double* out_xi, int64_t* out_steps,
                      double* out_iso, double* out_xstop, double* stats) {
  if (n_paths < 1 || h <= 0.0) return -1;
  or_problem pb = {kind, c0, y_exp, max_steps, cv_mode, grid_n, grad};
  int dim = or_problem_dim(kind);
  double* phi = (double*)malloc(sizeof(double) * (size_t)n_paths);
  double* xi = (double*)malloc(sizeof(double) * (size_t)n_paths);
  double* iso = (double*)malloc(sizeof(double) * (size_t)n_paths);
  int64_t* steps = (int64_t*)malloc(sizeof(int64_t) * (size_t)n_paths);
  int* trunc = (int*)malloc(sizeof(int) * (size_t)n_paths);
  if (!phi || !xi || !iso || !steps || !trunc) {
    free(phi); free(xi); free(iso); free(steps); free(trunc);
    return -2;
  }
  for (int64_t i = 0; i < n_nodes; ++i) {
    double x0[3] = {xs[i], ys[i], dim == 3 ? zs[i] : 0.0};
    for (int64_t p = 0; p < n_paths; ++p) {
      or_path r;
      or_simulate_path(&pb, x0, h, seed, tag, (uint32_t)i, (uint32_t)p, &r);
      phi[p] = r.phi; xi[p] = r.xi; iso[p] = r.iso; steps[p] = r.steps; trunc[p] = r.truncated;
      int64_t q = i * n_paths + p;
      if (out_phi) out_phi[q] = r.phi;
      if (out_xi) out_xi[q] = r.xi;
      if (out_steps) out_steps[q] = r.steps;
      if (out_iso) out_iso[q] = r.iso;
      if (out_xstop) for (int j = 0; j < 3; ++j) out_xstop[q * 3 + j] = r.x_stop[j];
    }
    if (stats) or_node_stats(n_paths, phi, xi, steps, trunc, iso, kappa, stats + i * OR_NSTAT);
  }
  free(phi); free(xi); free(iso); free(steps); free(trunc);
  return 0;
}

/* Sampled paths: (node, path) pairs listed explicitly, for checks on a few */
/* outputs of a full-size run.                                               */
int or_sample_paths(int kind, double c0, int y_exp, int64_t max_steps, int cv_mode, int grid_n,
                    const double* grad, int64_t n_samples, const double* xs, const double* ys,
                    const double* zs, const uint32_t* node_idx, const uint32_t* path_idx, double h,
                    uint64_t seed, uint32_t tag, double* out_phi, double* out_xi,
                    int64_t* out_steps) {
  or_problem pb = {kind, c0, y_exp, max_steps, cv_mode, grid_n, grad};
  int dim = or_problem_dim(kind);
  for (int64_t s = 0; s < n_samples; ++s) {
    double x0[3] = {xs[s], ys[s], dim == 3 ? zs[s] : 0.0};
    or_path r;
    or_simulate_path(&pb, x0, h, seed, tag, node_idx[s], path_idx[s], &r);
    out_phi[s] = r.phi;
    out_xi[s] = r.xi;
    out_steps[s] = r.steps;
  }
  return 0;
}
