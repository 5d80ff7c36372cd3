// pdd_device.cuh -- device building blocks of the PDD Monte Carlo nodal stage:
// the counter-based generator, the normal transform, the built-in problems,
// the box geometry, the control-grid interpolation and the exact fixed-point
// per-node accumulators.  Method: Bernal & Acebron, Sec. 2 and Algorithm 1.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pdd_internal.h"

namespace pdd {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  Each of the ten rounds
// multiplies words 0 and 2 by the two round multipliers, swaps the halves and
// xors in the round key; the key is then bumped by the two Weyl increments.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    // one 32x32 -> 64-bit multiply gives both halves of each product
    const unsigned long long p0 = (unsigned long long)c.x * 0xD2511F53u;
    const unsigned long long p1 = (unsigned long long)c.z * 0xCD9E8D57u;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k.x, (uint32_t)p1,
                   (uint32_t)(p0 >> 32) ^ c.w ^ k.y, (uint32_t)p0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

// ---------------------------------------------------------------------------
// Math in the path precision.  FP32 uses the SFU approximations (their error
// is far below the Monte Carlo tolerance); FP64 uses the IEEE library calls.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float m_sin(float x) { return __sinf(x); }
__device__ __forceinline__ float m_cos(float x) { return __cosf(x); }
__device__ __forceinline__ float m_exp(float x) { return __expf(x); }
__device__ __forceinline__ void m_sincos(float x, float* s, float* c) { __sincosf(x, s, c); }
__device__ __forceinline__ float m_sqrt(float x) { return x * rsqrtf(x); }  // x > 0
__device__ __forceinline__ double m_sin(double x) { return sin(x); }
__device__ __forceinline__ double m_cos(double x) { return cos(x); }
__device__ __forceinline__ double m_exp(double x) { return exp(x); }
__device__ __forceinline__ void m_sincos(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ double m_sqrt(double x) { return sqrt(x); }

// Explicitly rounded arithmetic.  A multiply and an add written as separate
// operators may or may not be fused into one FMA, and the compiler decides
// per inlined copy of the code (the path step is inlined into the ordinary
// and the drain iterations of every kernel variant).  The arithmetic whose
// result must not depend on that choice -- the grid interpolation, the
// control-variate increment and the compensated sums -- uses these, which
// are never contracted, so a path computes the same bits in every copy.
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }

// Uniform (0,1) from a 32-bit word: ((w >> 9) + 1/2) 2^-23, exact in FP32.
// Formed without an int-to-float conversion (conversions issue to a narrower
// pipe than integer logic and FP32 adds): 1 + (w >> 9) 2^-23 is the float
// with those mantissa bits and exponent 0, and subtracting 1 - 2^-24 from it
// is exact (Sterbenz), which gives the same value.  Measured on the C1 step:
// plain pass +3.6 %, control-variate passes +2.3 % path-steps/s.
__device__ __forceinline__ float unit_f(uint32_t w) {
  return __fsub_rn(__uint_as_float((w >> 9) | 0x3F800000u), 1.0f - 0x1p-24f);
}

// Box-Muller pair from words (wa, wb): r = sqrt(-2 ln u_a), angle 2 pi u_b.
// The angle is evaluated as theta = 2 pi (u_b - 1/2) in [-pi, pi] (where the
// fast sine/cosine are accurate) and the signs flipped back:
// cos(2 pi u) = -cos(theta), sin(2 pi u) = -sin(theta).
// `scale` multiplies both outputs (the kernels pass sqrt(h) to get dW directly).
__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, float& n0, float& n1,
                                           float scale = 1.0f) {
  const float ua = unit_f(wa), ub = unit_f(wb);
  const float t = -2.0f * __logf(ua);  // > 0 since ua < 1
  const float r = (scale * t) * rsqrtf(t);
  const float th = fmaf(ub, 6.28318530717958647692f, -3.14159265358979323846f);
  float s, c;
  __sincosf(th, &s, &c);
  n0 = -r * c;
  n1 = -r * s;
}
__device__ __forceinline__ void box_muller(uint32_t wa, uint32_t wb, double& n0, double& n1,
                                           double scale = 1.0) {
  const double ua = ((double)(wa >> 9) + 0.5) * 0x1p-23;
  const double ub = ((double)(wb >> 9) + 0.5) * 0x1p-23;
  const double r = scale * sqrt(-2.0 * log(ua));
  const double th = (ub - 0.5) * 6.283185307179586476925286766559;
  double s, c;
  sincos(th, &s, &c);
  n0 = -r * c;
  n1 = -r * s;
}

// ---------------------------------------------------------------------------
// Built-in problems (1/2 sum a_ij d_ij u + b.grad u - c u = f on [0,1]^D,
// g = u).  eval() returns b, c, f at X_k and, when asked, the analytic grad u
// used by the exact control variate.  sa = sqrt(a(x)) scales sigma for the
// anisotropic problem, whose A = a(x) [[1, 1/2], [1/2, 1]] has equal diagonal
// entries, so |sigma^T N| = sqrt(a) for either face normal.
// ---------------------------------------------------------------------------
template <class T>
struct Coef {
  T b0, b1, b2, c, f, g0, g1, g2, sa;
};

// u = e^{x+y} cos(x-y); Delta u = 0.  Without the gradient (GRAD: the exact
// control variate) f is formed with the common factor e^{x+y} taken out, two
// multiplies fewer per step (C1 plain pass +2 %, control variate +0.7 %).
template <class T, bool GRAD>
__device__ __forceinline__ void exp_cos_2d(T x, T y, Coef<T>& o, T& u) {
  const T sy = m_sin(y), cx = m_cos(x);
  const T E = m_exp(add_rn(x, y));
  T sn, cs;
  m_sincos(sub_rn(x, y), &sn, &cs);
  u = mul_rn(E, cs);
  // b = (sin y, cos x) / 2 is returned without the 1/2 (kDriftHalf: the
  // Euler step multiplies it by h/2, which is exact, so X is unchanged)
  o.b0 = sy;
  o.b1 = cx;
  o.b2 = T(0);
  o.c = fma_rn(y, y, fma_rn(x, x, T(1)));  // 1 + x^2 + y^2
  const T d1 = sub_rn(cs, sn), d2 = add_rn(cs, sn);  // grad u = E (d1, d2)
  if (GRAD) {
    const T ux = mul_rn(E, d1), uy = mul_rn(E, d2);
    // b . grad u - c u
    o.f = fma_rn(T(0.5), fma_rn(cx, uy, mul_rn(sy, ux)), mul_rn(-o.c, u));
    o.g0 = ux;
    o.g1 = uy;
  } else {
    // the same with the common factor E taken out: E (b . (d1, d2) - c cs)
    o.f = mul_rn(E, fma_rn(T(0.5), fma_rn(cx, d2, mul_rn(sy, d1)), mul_rn(-o.c, cs)));
    o.g0 = o.g1 = T(0);
  }
  o.g2 = T(0);
}

struct Cfg0 {
  static constexpr bool kDriftHalf = true;  // eval returns 2 b
  static constexpr bool kIsoScaled = false;
  static constexpr int kDim = 2;
  static constexpr bool kAniso = false;
  static constexpr bool kUnitY = false;
  template <class T, bool GRAD>
  __device__ __forceinline__ static void eval(T x, T y, T, Coef<T>& o) {
    T u;
    exp_cos_2d<T, GRAD>(x, y, o, u);
    o.sa = T(1);
  }
  template <class T>
  __device__ __forceinline__ static T g(T x, T y, T) {
    return mul_rn(m_exp(add_rn(x, y)), m_cos(sub_rn(x, y)));
  }
  template <class T>
  __device__ __forceinline__ static T exit_scale(T, T, T) { return T(1); }
};

struct Aniso {
  static constexpr bool kDriftHalf = true;  // eval returns 2 b
  static constexpr bool kIsoScaled = false;
  static constexpr int kDim = 2;
  static constexpr bool kAniso = true;
  static constexpr bool kUnitY = false;
  // a(x) = 1 + sin(2 pi x)/2, with sin(2 pi x) = -sin(2 pi (x - 1/2)).
  template <class T>
  __device__ __forceinline__ static T a_of(T x) {
    return fma_rn(T(-0.5), m_sin(mul_rn(T(6.283185307179586476925286766559), sub_rn(x, T(0.5)))),
                  T(1));
  }
  template <class T, bool GRAD>
  __device__ __forceinline__ static void eval(T x, T y, T, Coef<T>& o) {
    T u;
    exp_cos_2d<T, GRAD>(x, y, o, u);
    const T a = a_of(x);
    // 1/2 sum a_ij u_ij = 1/2 * 2 * (a/2) * u_xy with u_xy = 2u
    o.f = fma_rn(a, u, o.f);
    o.sa = m_sqrt(a);
  }
  template <class T>
  __device__ __forceinline__ static T g(T x, T y, T) {
    return mul_rn(m_exp(add_rn(x, y)), m_cos(sub_rn(x, y)));
  }
  template <class T>
  __device__ __forceinline__ static T exit_scale(T x, T, T) { return m_sqrt(a_of(x)); }
};

struct Cube3 {
  static constexpr bool kDriftHalf = false;
  static constexpr bool kIsoScaled = false;
  static constexpr int kDim = 3;
  static constexpr bool kAniso = false;
  static constexpr bool kUnitY = false;
  template <class T, bool GRAD>
  __device__ __forceinline__ static void eval(T x, T y, T z, Coef<T>& o) {
    const T ex = m_exp(x);
    T sy, cy, sz, cz;
    if (GRAD) {
      m_sincos(y, &sy, &cy);
      m_sincos(z, &sz, &cz);
    } else {
      sy = m_sin(y);
      cz = m_cos(z);
      cy = sz = T(0);
    }
    const T e = mul_rn(mul_rn(ex, sy), cz);
    o.b0 = o.b1 = o.b2 = T(0);
    o.c = T(1);
    // 1/2 Delta u - u with Delta u = -e^x sin y cos z
    o.f = fma_rn(T(-1.5), e, -mul_rn(mul_rn(x, y), z));
    o.g0 = fma_rn(y, z, e);
    o.g1 = fma_rn(x, z, mul_rn(mul_rn(ex, cy), cz));
    o.g2 = fma_rn(x, y, -mul_rn(mul_rn(ex, sy), sz));
    o.sa = T(1);
  }
  template <class T>
  __device__ __forceinline__ static T g(T x, T y, T z) {
    return fma_rn(mul_rn(x, y), z, mul_rn(mul_rn(m_exp(x), m_sin(y)), m_cos(z)));
  }
  template <class T>
  __device__ __forceinline__ static T exit_scale(T, T, T) { return T(1); }
};

// The paper's example PDE (Sec. 6): sigma = sqrt(2) I, b = cos(x+y)/(1.1+sin(x+y)) [1,1],
// c = (x^2+y^2)/(1.1+sin(x+y)), u = 2 cos(2(y-2)x) + sin(3(x-2)y) + 3.1.
struct PaperEx {
  static constexpr bool kDriftHalf = false;
  static constexpr int kDim = 2;
  static constexpr bool kAniso = false;
  static constexpr bool kIsoScaled = true;  // sigma = sa * I with sa = sqrt(2)
  static constexpr bool kUnitY = false;
  template <class T, bool GRAD>
  __device__ __forceinline__ static void eval(T x, T y, T, Coef<T>& o) {
    T sp, cp, sq, cq, ss, cs;
    const T ym2 = sub_rn(y, T(2)), xm2 = sub_rn(x, T(2));
    const T p = mul_rn(mul_rn(T(2), x), ym2), q = mul_rn(mul_rn(T(3), y), xm2);
    m_sincos(p, &sp, &cp);
    m_sincos(q, &sq, &cq);
    m_sincos(add_rn(x, y), &ss, &cs);
    const T inv = T(1) / add_rn(T(1.1), ss);
    const T u = add_rn(fma_rn(T(2), cp, sq), T(3.1));
    const T ux = fma_rn(mul_rn(T(3), y), cq, mul_rn(mul_rn(T(-4), ym2), sp));
    const T uy = fma_rn(mul_rn(T(3), xm2), cq, mul_rn(mul_rn(T(-4), x), sp));
    const T lap = fma_rn(mul_rn(T(-9), fma_rn(xm2, xm2, mul_rn(y, y))), sq,
                         mul_rn(mul_rn(T(-8), fma_rn(x, x, mul_rn(ym2, ym2))), cp));
    o.b0 = o.b1 = mul_rn(cs, inv);
    o.b2 = T(0);
    o.c = mul_rn(fma_rn(y, y, mul_rn(x, x)), inv);
    o.f = fma_rn(-o.c, u, fma_rn(o.b0, add_rn(ux, uy), lap));
    o.g0 = ux;
    o.g1 = uy;
    o.g2 = T(0);
    o.sa = T(1.41421356237309504880);
  }
  template <class T>
  __device__ __forceinline__ static T g(T x, T y, T) {
    return add_rn(fma_rn(T(2), m_cos(mul_rn(mul_rn(T(2), x), sub_rn(y, T(2)))),
                         m_sin(mul_rn(mul_rn(T(3), y), sub_rn(x, T(2))))),
                  T(3.1));
  }
  template <class T>
  __device__ __forceinline__ static T exit_scale(T, T, T) { return T(1.41421356237309504880); }
};

struct Harmonic {
  static constexpr bool kDriftHalf = false;
  static constexpr bool kIsoScaled = false;
  static constexpr int kDim = 2;
  static constexpr bool kAniso = false;
  static constexpr bool kUnitY = true;  // c = f = 0: Y = 1, Z = 0 on every path
  template <class T, bool GRAD>
  __device__ __forceinline__ static void eval(T x, T y, T, Coef<T>& o) {
    o.b0 = o.b1 = o.b2 = T(0);
    o.c = T(0);
    o.f = T(0);
    o.g0 = T(2) * x;
    o.g1 = T(-2) * y;
    o.g2 = T(0);
    o.sa = T(1);
  }
  template <class T>
  __device__ __forceinline__ static T g(T x, T y, T) { return fma_rn(x, x, -mul_rn(y, y)); }
  template <class T>
  __device__ __forceinline__ static T exit_scale(T, T, T) { return T(1); }
};

// ---------------------------------------------------------------------------
// Box geometry.  Inside [0,1]^D the exit test only needs the distance to the
// nearest face, m = min_j min(x_j, 1 - x_j): d = -m, and outside the box m < 0
// makes the finish condition hold as well.  The projection Pi clamps outside
// points and moves the nearest coordinate onto its face inside (corner ties:
// lowest axis first, the 0 face before the 1 face).
// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T face_distance(T x, T y) {
  return fmin(fmin(x, T(1) - x), fmin(y, T(1) - y));
}
template <class T>
__device__ __forceinline__ T face_distance(T x, T y, T z) {
  return fmin(face_distance(x, y), fmin(z, T(1) - z));
}

template <class T>
__device__ __forceinline__ void project_box(T* p, int dim) {
  bool outside = false;
  for (int j = 0; j < dim; ++j) outside |= (p[j] < T(0)) | (p[j] > T(1));
  if (outside) {
    for (int j = 0; j < dim; ++j) p[j] = fmin(fmax(p[j], T(0)), T(1));
    return;
  }
  T best = p[0];
  int sel = 0;
  if (T(1) - p[0] < best) { best = T(1) - p[0]; sel = 1; }
  for (int j = 1; j < dim; ++j) {
    if (p[j] < best) { best = p[j]; sel = 2 * j; }
    if (T(1) - p[j] < best) { best = T(1) - p[j]; sel = 2 * j + 1; }
  }
  p[sel >> 1] = (sel & 1) ? T(1) : T(0);
}

// ---------------------------------------------------------------------------
// Control-grid interpolation: n points per axis on [0,1]^D, cell index
// clamped to [0, n-2], multilinear weights.  2D tables are float2 (gx, gy),
// 3D tables float4 (gx, gy, gz, 0) so every corner is one 8- or 16-byte load.
// ---------------------------------------------------------------------------
// Bounds-checked build (-DPDD_DEBUG_BOUNDS=1): `ok` false sets `bit` in the
// launch's error word and the caller skips the guarded access; the host turns
// a non-zero word into PDD_ERR_BOUNDS.  The release build evaluates nothing.
__device__ __forceinline__ bool bounds_ok(unsigned* err, bool ok, unsigned bit) {
  if (!ok) atomicOr(err, bit);
  return ok;
}
#if PDD_DEBUG_BOUNDS
#define PDD_IN_BOUNDS(a, ok, bit) ::pdd::bounds_ok((a).err, (ok), (bit))
#else
#define PDD_IN_BOUNDS(a, ok, bit) true
#endif

// Bounds-checked build: a cell index outside [0, n-2] sets kErrBoundsGrid in
// the launch's error word (`err`) and the lookup is skipped.  The release
// build checks nothing (the indices are clamped by construction).
__device__ __forceinline__ bool cell_in_table(unsigned* err, int ix, int iy, int iz, int n) {
#if PDD_DEBUG_BOUNDS
  const bool ok = ix >= 0 && ix <= n - 2 && iy >= 0 && iy <= n - 2 && iz >= 0 && iz <= n - 2 &&
                  n >= 2;
  return err ? bounds_ok(err, ok, kErrBoundsGrid) : ok;
#else
  (void)err; (void)ix; (void)iy; (void)iz; (void)n;
  return true;
#endif
}

// Cell index min(max(floor(x s), 0), n - 2) and the offset of x s in it,
// frac = x s - i with one rounding.  For x s >= 0 truncation is the floor,
// and for x s < 0 both give an index that the clamp takes to 0, so the
// truncating conversion gives the same cell and frac.
template <class T>
__device__ __forceinline__ int cell_of(T x, T s, int n, T& frac) {
  int i = (int)mul_rn(x, s);
  i = min(max(i, 0), n - 2);
  frac = fma_rn(x, s, -(T)i);
  return i;
}

template <class T>
__device__ __forceinline__ void grid_grad_2d(const float2* __restrict__ G, int n, T x, T y, T& gx,
                                             T& gy, unsigned* err = nullptr) {
  const T s = (T)(n - 1);
  T fx, fy;
  const int ix = cell_of(x, s, n, fx), iy = cell_of(y, s, n, fy);
  if (!cell_in_table(err, ix, iy, 0, n)) {
    gx = gy = T(0);
    return;
  }
  const float2* p = G + (size_t)iy * n + ix;
  const float2 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + n), d = __ldg(p + n + 1);
  const T lx0 = fma_rn(fx, sub_rn((T)b.x, (T)a.x), (T)a.x);
  const T lx1 = fma_rn(fx, sub_rn((T)d.x, (T)c.x), (T)c.x);
  const T ly0 = fma_rn(fx, sub_rn((T)b.y, (T)a.y), (T)a.y);
  const T ly1 = fma_rn(fx, sub_rn((T)d.y, (T)c.y), (T)c.y);
  gx = fma_rn(fy, sub_rn(lx1, lx0), lx0);
  gy = fma_rn(fy, sub_rn(ly1, ly0), ly0);
}

template <class T>
__device__ __forceinline__ void grid_grad_3d(const float4* __restrict__ G, int n, T x, T y, T z,
                                             T& gx, T& gy, T& gz, unsigned* err = nullptr) {
  const T s = (T)(n - 1);
  T fx, fy, fz;
  const int ix = cell_of(x, s, n, fx), iy = cell_of(y, s, n, fy),
            iz = cell_of(z, s, n, fz);
  if (!cell_in_table(err, ix, iy, iz, n)) {
    gx = gy = gz = T(0);
    return;
  }
  const size_t nn = (size_t)n * n;
  const float4* p = G + (size_t)iz * nn + (size_t)iy * n + ix;
  T acc[3][2][2];  // [component][y corner][z corner] after the x lerp
#pragma unroll
  for (int cz = 0; cz < 2; ++cz) {
#pragma unroll
    for (int cy = 0; cy < 2; ++cy) {
      const float4* q = p + cz * nn + cy * n;
      const float4 a = __ldg(q), b = __ldg(q + 1);
      acc[0][cy][cz] = fma_rn(fx, sub_rn((T)b.x, (T)a.x), (T)a.x);
      acc[1][cy][cz] = fma_rn(fx, sub_rn((T)b.y, (T)a.y), (T)a.y);
      acc[2][cy][cz] = fma_rn(fx, sub_rn((T)b.z, (T)a.z), (T)a.z);
    }
  }
  T out[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T l0 = fma_rn(fy, sub_rn(acc[c][1][0], acc[c][0][0]), acc[c][0][0]);
    const T l1 = fma_rn(fy, sub_rn(acc[c][1][1], acc[c][0][1]), acc[c][0][1]);
    out[c] = fma_rn(fz, sub_rn(l1, l0), l0);
  }
  gx = out[0];
  gy = out[1];
  gz = out[2];
}

// ---------------------------------------------------------------------------
// Cell-coefficient tables (FP32 paths).  For every grid cell the multilinear
// interpolant of each gradient component is stored as polynomial coefficients
// in the cell's local coordinates (fx, fy[, fz]) in [0,1]:
//   2D: g = c0 + c1 fx + c2 fy + c3 fx fy                  (2 x float4 = 32 B)
//   3D: g = c000 + c100 fx + c010 fy + c001 fz + c110 fx fy + c101 fx fz
//           + c011 fy fz + c111 fx fy fz                      (64 B)
// so a lane reads one contiguous 32 B / 64 B record per step instead of 4 / 8
// scattered corner values.  2D coefficients are FP32 (the multilinear
// interpolation of the nodal table up to their FP32 rounding).  A 3D record
// holds c000 of the three components as FP32 (words 0-2) and the seven other
// coefficients of each component (c100 c010 c001 c110 c101 c011 c111, x then
// y then z) as 21 binary16 values, two per word, low half first (words 3-13;
// words 14-15 are zero): two 256-bit loads per step instead of three, which
// relieves the L1 data path that bounds the 3D kernel.  The table follows the
// nodal table in the grid's allocation, at offset cell_table_offset(n, dim).
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ size_t cell_table_offset(int n, int dim) {
  const size_t pts = dim == 2 ? (size_t)n * n : (size_t)n * n * n;
  const size_t bytes = pts * (dim == 2 ? 8 : 16);
  return (bytes + 255) / 256 * 256;
}

// 32-byte load through the non-coherent (read-only) path: one 256-bit vector
// load per record chunk, so a lane's chunk is one full sector.  `p` must be
// 32-byte aligned (records start at multiples of 32 bytes of a 256-byte
// aligned table).  The tables do not change while a kernel runs, so the load
// is a pure function of its address (not volatile): the compiler may schedule
// it as early as the address is known.
__device__ __forceinline__ void ldg_v8(const float4* p, float4& a, float4& b) {
  asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z),
                 "=f"(b.w)
               : "l"(p));
}

template <class T>
__device__ __forceinline__ void grid_cells_2d(const float4* __restrict__ C, int n, T x, T y,
                                              T& gx, T& gy, unsigned* err = nullptr) {
  const T s = (T)(n - 1);
  T fx, fy;
  const int ix = cell_of(x, s, n, fx), iy = cell_of(y, s, n, fy);
  if (!cell_in_table(err, ix, iy, 0, n)) {
    gx = gy = T(0);
    return;
  }
  const float4* p = C + 2 * ((size_t)iy * (n - 1) + ix);
  float4 a, b;
  ldg_v8(p, a, b);
  gx = fma_rn(fy, fma_rn(fx, (T)a.w, (T)a.z), fma_rn(fx, (T)a.y, (T)a.x));
  gy = fma_rn(fy, fma_rn(fx, (T)b.w, (T)b.z), fma_rn(fx, (T)b.y, (T)b.x));
}

template <class T>
__device__ __forceinline__ T cell_poly3(const float4 lo, const float4 hi, T fx, T fy, T fz) {
  // lo = (c000, c100, c010, c001), hi = (c110, c101, c011, c111)
  const T a = fma_rn(fz, (T)lo.w, (T)lo.x);  // c000 + c001 fz
  const T b = fma_rn(fz, (T)hi.z, (T)lo.z);  // c010 + c011 fz
  const T c = fma_rn(fz, (T)hi.y, (T)lo.y);  // c100 + c101 fz
  const T d = fma_rn(fz, (T)hi.w, (T)hi.x);  // c110 + c111 fz
  return fma_rn(fx, fma_rn(fy, d, c), fma_rn(fy, b, a));
}

__device__ __forceinline__ float half_lo(float w) {
  return __half2float(__ushort_as_half((unsigned short)(__float_as_uint(w) & 0xFFFFu)));
}
__device__ __forceinline__ float half_hi(float w) {
  return __half2float(__ushort_as_half((unsigned short)(__float_as_uint(w) >> 16)));
}

template <class T>
__device__ __forceinline__ void grid_cells_3d(const float4* __restrict__ C, int n, T x, T y, T z,
                                              T& gx, T& gy, T& gz, unsigned* err = nullptr) {
  const T s = (T)(n - 1);
  T fx, fy, fz;
  const int ix = cell_of(x, s, n, fx), iy = cell_of(y, s, n, fy),
            iz = cell_of(z, s, n, fz);
  if (!cell_in_table(err, ix, iy, iz, n)) {
    gx = gy = gz = T(0);
    return;
  }
  const size_t m = (size_t)(n - 1);
  const float4* p = C + 4 * (((size_t)iz * m + iy) * m + ix);
  float4 a, b, c, d;  // words 0-3, 4-7, 8-11, 12-15
  ldg_v8(p, a, b);
  ldg_v8(p + 2, c, d);
  // binary16 coefficients h[0..20]: word 3 + k holds h[2k] (low) and h[2k+1]
  const float h[21] = {half_lo(a.w), half_hi(a.w), half_lo(b.x), half_hi(b.x), half_lo(b.y),
                       half_hi(b.y), half_lo(b.z), half_hi(b.z), half_lo(b.w), half_hi(b.w),
                       half_lo(c.x), half_hi(c.x), half_lo(c.y), half_hi(c.y), half_lo(c.z),
                       half_hi(c.z), half_lo(c.w), half_hi(c.w), half_lo(d.x), half_hi(d.x),
                       half_lo(d.y)};
  gx = cell_poly3<T>(make_float4(a.x, h[0], h[1], h[2]), make_float4(h[3], h[4], h[5], h[6]),
                     fx, fy, fz);
  gy = cell_poly3<T>(make_float4(a.y, h[7], h[8], h[9]), make_float4(h[10], h[11], h[12], h[13]),
                     fx, fy, fz);
  gz = cell_poly3<T>(make_float4(a.z, h[14], h[15], h[16]),
                     make_float4(h[17], h[18], h[19], h[20]), fx, fy, fz);
}

// ---------------------------------------------------------------------------
// Compensated (Kahan) summation for the FP32 Z and xi accumulators.
// ---------------------------------------------------------------------------
// The term enters as a product p * q, formed with the compensation's
// subtraction in one rounding: y = p q - comp.
template <class T>
__device__ __forceinline__ void kahan_add(T& sum, T& comp, T p, T q) {
  const T y = fma_rn(p, q, -comp);
  const T t = add_rn(sum, y);
  comp = sub_rn(sub_rn(t, sum), y);
  sum = t;
}

// ---------------------------------------------------------------------------
// Exact per-node accumulators.  Scores are converted to 64-bit fixed point
// with 32 fractional bits (|score| < 2^15), products are formed exactly in
// 128 bits, and 128-bit sums are kept in two 64-bit words with the carry of
// the low word propagated by the adding thread.  Integer addition commutes, so
// the totals do not depend on the order in which paths finish.
// Layout of one node record (16 x u64):
//   [0,1] sum q_phi   [2,3] sum q_phi^2   [4,5] sum q_psi   [6,7] sum q_psi^2
//   [8,9] sum q_phi q_psi   [10,11] sum k   [12,13] sum k^2   [14] n   [15] n_trunc
// (psi = phi + xi, the controlled score).
// ---------------------------------------------------------------------------

constexpr double kFxScale = 4294967296.0;  // 2^32
constexpr double kFxLimit = 32768.0;       // |score| < 2^15

__device__ __forceinline__ void atomic_add_u128(unsigned long long* p, unsigned long long lo,
                                                unsigned long long hi) {
  const unsigned long long old = atomicAdd(p, lo);
  hi += (old + lo < old) ? 1ull : 0ull;
  if (hi != 0ull) atomicAdd(p + 1, hi);
}

__device__ __forceinline__ void atomic_add_s64(unsigned long long* p, long long v) {
  atomic_add_u128(p, (unsigned long long)v, v < 0 ? ~0ull : 0ull);
}

__device__ __forceinline__ void atomic_add_prod(unsigned long long* p, long long a, long long b) {
  atomic_add_u128(p, (unsigned long long)a * (unsigned long long)b,
                  (unsigned long long)__mul64hi(a, b));
}

__device__ __forceinline__ bool to_fixed(double v, long long& q) {
  if (!(fabs(v) < kFxLimit)) {
    q = 0;
    return false;
  }
  q = __double2ll_rn(v * kFxScale);
  return true;
}
// FP32 scores: scaling by 2^32 is exact in FP32, so no FP64 work is needed.
__device__ __forceinline__ bool to_fixed(float v, long long& q) {
  if (!(fabsf(v) < (float)kFxLimit)) {
    q = 0;
    return false;
  }
  q = __float2ll_rn(v * 4294967296.0f);
  return true;
}

// 128-bit two's-complement value (lo, hi) to double.
__device__ __forceinline__ double s128_to_double(unsigned long long lo, unsigned long long hi) {
  return (double)(long long)hi * 18446744073709551616.0 + (double)lo;
}
__device__ __forceinline__ double u128_to_double(unsigned long long lo, unsigned long long hi) {
  return (double)hi * 18446744073709551616.0 + (double)lo;
}

}  // namespace pdd
