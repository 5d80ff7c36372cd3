// pdd_paths.cu -- the path kernels of the PDD Monte Carlo nodal stage
// (Bernal & Acebron, Algorithm 1 with the pathwise control variate of
// eq. F:xiControlVariate) and the per-node finalisation (eqs. F:Statistics_VR
// .. F:Rho, F:Pointwise_cost, F:VR_Pointwise_cost, F:nu).
//
// Execution model.  One path per lane.  The paths of all nodes form one flat
// index space g = node * n_paths + path; warps take batches of 32 indices
// from a global cursor (atomicAdd) and every lane whose path has finished
// takes the next index of its warp's batch at the next iteration boundary, so
// lanes stay busy whatever the spread of exit times (paths of one node range
// over ~12x the mean number of steps).  The grid is persistent (occupancy x
// SM count blocks).  Per-node sums are exact integers, so which lane or warp
// runs a path changes nothing in the results.
//
// One iteration takes as many Euler steps as one Philox block has normals
// for: two steps in 2D (4 normals), four steps in 3D (3 blocks, 12 normals),
// so no random word is wasted and every path's stream is the one fixed by
// its (seed, stream_tag, node, path) key.
#include <cuda_runtime.h>
#include <stdint.h>

#include "pdd_device.cuh"
#include "pdd_internal.h"

namespace pdd {

constexpr int kBlockThreads = 256;
#ifndef PDD_MIN_BLOCKS
#define PDD_MIN_BLOCKS 1
#endif
constexpr unsigned kFull = 0xFFFFFFFFu;
enum { kCvNone = 0, kCvGrid = 1, kCvExact = 2 };

// Per-lane path state.
template <class T>
struct PathState {
  T x[3];
  T Y, Z, Zc, XI, XIc;
  int k;
  uint32_t node, path;
};

// Start path g of the flat index space.
template <class T, int D>
__device__ __forceinline__ void start_path(const PathArgs& a, unsigned long long g,
                                           PathState<T>& s) {
  if (a.total <= 0xFFFFFFFFull) {  // 32-bit division when the index space allows
    const uint32_t gg = (uint32_t)g, np = (uint32_t)a.n_paths;
    s.node = gg / np;
    s.path = gg - s.node * np;
  } else {
    s.node = (uint32_t)(g / a.n_paths);
    s.path = (uint32_t)(g - (unsigned long long)s.node * a.n_paths);
  }
  s.x[0] = (T)__ldg(a.cx + s.node);
  s.x[1] = (T)__ldg(a.cy + s.node);
  s.x[2] = (D == 3) ? (T)__ldg(a.cz + s.node) : T(0);
  s.Y = T(1);
  s.Z = s.Zc = s.XI = s.XIc = T(0);
  s.k = 0;
}

// Finish test of Algorithm 1: d(X_k) >= -c0 |sigma^T N| sqrt(h).
template <class P, class T, int D>
__device__ __forceinline__ bool should_finish(const PathState<T>& s, T thr0) {
  const T m = (D == 3) ? face_distance(s.x[0], s.x[1], s.x[2]) : face_distance(s.x[0], s.x[1]);
  T thr = thr0;
  if (P::kAniso) thr *= P::template exit_scale<T>(s.x[0], s.x[1], s.x[2]);
  return m <= thr;
}

// One Euler-Maruyama step (eq. F:E_M) with the Feynman-Kac weights and the
// control variate, all right-hand sides at X_k.
template <class P, class T, int D, int CV>
__device__ __forceinline__ void euler_step(const PathArgs& a, PathState<T>& s, T h,
                                           const T* dW) {
  Coef<T> o;
  P::template eval<T, CV == kCvExact>(s.x[0], s.x[1], s.x[2], o);
  T sdW[3];
  const T dW0 = dW[0], dW1 = dW[1];
  if (P::kAniso) {  // sigma = sqrt(a) [[1, 0], [1/2, sqrt(3)/2]]
    sdW[0] = o.sa * dW0;
    sdW[1] = o.sa * (T(0.5) * dW0 + T(0.86602540378443864676) * dW1);
  } else {
    sdW[0] = dW0;
    sdW[1] = dW1;
  }
  sdW[2] = (D == 3) ? dW[2] : T(0);
  if (CV != kCvNone) {
    T gv[3] = {T(0), T(0), T(0)};
    if (CV == kCvGrid) {
      if (D == 2)
        grid_grad_2d<T>((const float2*)a.grad, a.grid_n, s.x[0], s.x[1], gv[0], gv[1]);
      else
        grid_grad_3d<T>((const float4*)a.grad, a.grid_n, s.x[0], s.x[1], s.x[2], gv[0], gv[1],
                        gv[2]);
    } else {
      gv[0] = o.g0;
      gv[1] = o.g1;
      gv[2] = o.g2;
    }
    T dot = gv[0] * sdW[0] + gv[1] * sdW[1];
    if (D == 3) dot += gv[2] * sdW[2];
    kahan_add(s.XI, s.XIc, -s.Y * dot);
  }
  if (!P::kUnitY) kahan_add(s.Z, s.Zc, -h * s.Y * o.f);
  s.x[0] += h * o.b0 + sdW[0];
  s.x[1] += h * o.b1 + sdW[1];
  if (D == 3) s.x[2] += h * o.b2 + sdW[2];
  if (!P::kUnitY) s.Y *= a.y_exp ? m_exp(-h * o.c) : (T(1) - h * o.c);
  s.k += 1;
}

// Exit scoring: X_tau = Pi(X_k), phi = g(X_tau) Y + Z, xi, and the exact
// fixed-point accumulation into the node record.
template <class P, class T, int D>
__device__ __forceinline__ void finish_path(const PathArgs& a, const PathState<T>& s, bool trunc) {
  T p[3] = {s.x[0], s.x[1], s.x[2]};
  project_box<T>(p, D);
  const T g = P::template g<T>(p[0], p[1], p[2]);
  const T phi = g * s.Y + (s.Z - s.Zc);
  const T xi = s.XI - s.XIc;
  const T psi = phi + xi;
  long long qa, qb;
  const bool ok = to_fixed(phi, qa) & to_fixed(psi, qb);
  if (!ok) atomicOr(a.err, kErrOverflow);
  unsigned long long* w = a.acc + (size_t)s.node * kAccWords;
  atomic_add_s64(w + 0, qa);
  atomic_add_prod(w + 2, qa, qa);
  atomic_add_s64(w + 4, qb);
  atomic_add_prod(w + 6, qb, qb);
  atomic_add_prod(w + 8, qa, qb);
  const unsigned long long k = (unsigned long long)s.k;
  atomic_add_u128(w + 10, k, 0ull);
  atomic_add_u128(w + 12, k * k, 0ull);
  atomicAdd(w + 14, 1ull);
  if (trunc) {
    atomicAdd(w + 15, 1ull);
    atomicAdd(a.trunc_total, 1ull);
  }
  if (a.emit_phi != nullptr) {
    const size_t i = (size_t)s.node * a.n_paths + s.path;
    a.emit_phi[i] = (float)phi;
    a.emit_xi[i] = (float)xi;
    a.emit_steps[i] = s.k;
  }
}

// Refill idle lanes from the warp's batch; returns false when no lane of the
// warp has a path left to run.  All arguments except the lane state are
// warp-uniform.
template <class T, int D>
__device__ __forceinline__ bool refill(const PathArgs& a, PathState<T>& s, bool& active,
                                       unsigned long long& bnext, unsigned long long& bend,
                                       bool& exhausted) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned lt = (1u << lane) - 1u;
  unsigned idle = __ballot_sync(kFull, !active);
  while (idle != 0u && !exhausted) {
    if (bnext >= bend) {
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(a.cursor, (unsigned long long)kWarpBatch);
      base = __shfl_sync(kFull, base, 0);
      if (base >= a.total) {
        exhausted = true;
        break;
      }
      bnext = base;
      bend = min(base + (unsigned long long)kWarpBatch, a.total);
    }
    const unsigned avail = (unsigned)min(bend - bnext, 32ull);
    const unsigned rank = __popc(idle & lt);
    if (!active && rank < avail) {
      start_path<T, D>(a, bnext + rank, s);
      active = true;
    }
    bnext += min((unsigned)__popc(idle), avail);
    idle = __ballot_sync(kFull, !active);
  }
  return __ballot_sync(kFull, active) != 0u;
}

template <class P, class T, int CV>
__global__ void __launch_bounds__(kBlockThreads, PDD_MIN_BLOCKS) paths_2d(const __grid_constant__ PathArgs a) {
  const T h = (T)a.h, sqh = (T)a.sqrt_h, thr0 = (T)a.thr0;
  const uint2 key = make_uint2(a.key0, a.key1);
  PathState<T> s;
  s.x[0] = s.x[1] = s.x[2] = T(0);
  s.Y = s.Z = s.Zc = s.XI = s.XIc = T(0);
  s.k = 0;
  s.node = s.path = 0;
  bool active = false, exhausted = false;
  unsigned long long bnext = 0, bend = 0;
  while (refill<T, 2>(a, s, active, bnext, bend, exhausted)) {
    bool fin = false, trunc = false;
    uint4 w = make_uint4(0, 0, 0, 0);
    if (active) fin = should_finish<P, T, 2>(s, thr0);
    if (active && !fin) {
      w = philox4x32_10(make_uint4((uint32_t)(s.k >> 1), s.path, s.node, a.seed_hi), key);
      T n[3];
      box_muller(w.x, w.y, n[0], n[1], sqh);
      n[2] = T(0);
      euler_step<P, T, 2, CV>(a, s, h, n);
      if (s.k >= a.max_steps) fin = trunc = true;
    }
    if (active && !fin) fin = should_finish<P, T, 2>(s, thr0);
    if (active && !fin) {
      T n[3];
      box_muller(w.z, w.w, n[0], n[1], sqh);
      n[2] = T(0);
      euler_step<P, T, 2, CV>(a, s, h, n);
      if (s.k >= a.max_steps) fin = trunc = true;
    }
    if (active && fin) {
      finish_path<P, T, 2>(a, s, trunc);
      active = false;
    }
  }
}

// 3D: steps 4j .. 4j+3 use normals 12j .. 12j+11, i.e. Philox blocks 3j,
// 3j+1, 3j+2 (words a0..a3, b0..b3, c0..c3):
//   step 0: a0 a1 a2   step 1: a3 b0 b1   step 2: b2 b3 c0   step 3: c1 c2 c3
// Blocks are drawn only when the path is still running.
template <class P, class T, int CV>
__global__ void __launch_bounds__(kBlockThreads, PDD_MIN_BLOCKS) paths_3d(const __grid_constant__ PathArgs a) {
  const T h = (T)a.h, sqh = (T)a.sqrt_h, thr0 = (T)a.thr0;
  const uint2 key = make_uint2(a.key0, a.key1);
  PathState<T> s;
  s.x[0] = s.x[1] = s.x[2] = T(0);
  s.Y = s.Z = s.Zc = s.XI = s.XIc = T(0);
  s.k = 0;
  s.node = s.path = 0;
  bool active = false, exhausted = false;
  unsigned long long bnext = 0, bend = 0;
  while (refill<T, 3>(a, s, active, bnext, bend, exhausted)) {
    bool fin = false, trunc = false;
    T carry0 = T(0), carry1 = T(0);  // normals left over from the previous block
    uint4 w = make_uint4(0, 0, 0, 0);
    const uint32_t blk0 = 3u * ((uint32_t)s.k >> 2);
    // step 0
    if (active) fin = should_finish<P, T, 3>(s, thr0);
    if (active && !fin) {
      w = philox4x32_10(make_uint4(blk0, s.path, s.node, a.seed_hi), key);
      T n[3], n3;
      box_muller(w.x, w.y, n[0], n[1], sqh);
      box_muller(w.z, w.w, n[2], n3, sqh);
      carry0 = n3;
      euler_step<P, T, 3, CV>(a, s, h, n);
      if (s.k >= a.max_steps) fin = trunc = true;
    }
    // step 1
    if (active && !fin) fin = should_finish<P, T, 3>(s, thr0);
    if (active && !fin) {
      w = philox4x32_10(make_uint4(blk0 + 1u, s.path, s.node, a.seed_hi), key);
      T n[3];
      n[0] = carry0;
      box_muller(w.x, w.y, n[1], n[2], sqh);
      euler_step<P, T, 3, CV>(a, s, h, n);
      if (s.k >= a.max_steps) fin = trunc = true;
    }
    // step 2
    if (active && !fin) fin = should_finish<P, T, 3>(s, thr0);
    if (active && !fin) {
      T n[3];
      box_muller(w.z, w.w, n[0], n[1], sqh);
      w = philox4x32_10(make_uint4(blk0 + 2u, s.path, s.node, a.seed_hi), key);
      box_muller(w.x, w.y, n[2], carry1, sqh);
      euler_step<P, T, 3, CV>(a, s, h, n);
      if (s.k >= a.max_steps) fin = trunc = true;
    }
    // step 3
    if (active && !fin) fin = should_finish<P, T, 3>(s, thr0);
    if (active && !fin) {
      T n[3];
      n[0] = carry1;
      box_muller(w.z, w.w, n[1], n[2], sqh);
      euler_step<P, T, 3, CV>(a, s, h, n);
      if (s.k >= a.max_steps) fin = trunc = true;
    }
    if (active && fin) {
      finish_path<P, T, 3>(a, s, trunc);
      active = false;
    }
  }
}

// ---------------------------------------------------------------------------
// Finalisation: one thread per node turns the exact sums into FP64 moments.
// ---------------------------------------------------------------------------
__global__ void finalize_nodes(const unsigned long long* __restrict__ acc, uint32_t n_nodes,
                               double kappa, const __grid_constant__ StatPtrs out) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  const unsigned long long* w = acc + (size_t)i * kAccWords;
  const double inv1 = 1.0 / kFxScale, inv2 = inv1 * inv1;
  const double n = (double)w[14];
  const double s_phi = s128_to_double(w[0], w[1]) * inv1;
  const double s_phi2 = s128_to_double(w[2], w[3]) * inv2;
  const double s_psi = s128_to_double(w[4], w[5]) * inv1;
  const double s_psi2 = s128_to_double(w[6], w[7]) * inv2;
  const double s_pp = s128_to_double(w[8], w[9]) * inv2;
  const double s_k = u128_to_double(w[10], w[11]);
  const double m_phi = s_phi / n, m_psi = s_psi / n;
  const double v_phi = (s_phi2 - s_phi * m_phi) / (n - 1.0);
  const double v_psi = (s_psi2 - s_psi * m_psi) / (n - 1.0);
  const double c_pp = (s_pp - s_phi * m_psi) / (n - 1.0);  // Cov[phi, phi + xi]
  const double c_px = c_pp - v_phi;                         // Cov[phi, xi]
  const double v_xi = v_psi + v_phi - 2.0 * c_pp;           // V[xi]
  if (out.mean_phi) out.mean_phi[i] = m_phi;
  if (out.var_phi) out.var_phi[i] = v_phi;
  if (out.mean_cv) out.mean_cv[i] = m_psi;
  if (out.var_cv) out.var_cv[i] = v_psi;
  if (out.cov_phi_xi) out.cov_phi_xi[i] = c_px;
  if (out.var_xi) out.var_xi[i] = v_xi;
  if (out.rho) out.rho[i] = c_px / sqrt(v_phi * v_xi);
  if (out.se_phi) out.se_phi[i] = sqrt(v_phi / n);
  if (out.se_cv) out.se_cv[i] = sqrt(v_psi / n);
  if (out.vr) out.vr[i] = v_psi / v_phi;
  if (out.pred_speedup) out.pred_speedup[i] = v_phi / (kappa * v_psi);
  if (out.mean_steps) out.mean_steps[i] = s_k / n;
  if (out.n_paths) out.n_paths[i] = w[14];
  if (out.n_truncated) out.n_truncated[i] = w[15];
}

// ---------------------------------------------------------------------------
// Launch dispatch.
// ---------------------------------------------------------------------------
template <class P, class T, int CV>
static cudaError_t launch_one(const PathArgs& a, int num_sms, cudaStream_t st, int* blocks) {
  void (*kern)(PathArgs);
  if constexpr (P::kDim == 3)
    kern = paths_3d<P, T, CV>;
  else
    kern = paths_2d<P, T, CV>;
  static int per_sm = 0;  // occupancy of this instantiation (same for every device here)
  if (per_sm == 0) {
    int v = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, kBlockThreads, 0);
    if (e != cudaSuccess) return e;
    per_sm = v > 0 ? v : 1;
  }
  const unsigned long long warps_needed = (a.total + 31ull) / 32ull;
  const unsigned long long blocks_needed =
      (warps_needed + (kBlockThreads / 32) - 1) / (kBlockThreads / 32);
  unsigned long long nb = (unsigned long long)per_sm * (unsigned long long)num_sms;
  if (a.max_blocks > 0 && nb > (unsigned long long)a.max_blocks) nb = a.max_blocks;
  if (nb > blocks_needed) nb = blocks_needed;
  if (nb < 1) nb = 1;
  *blocks = (int)nb;
  kern<<<(unsigned)nb, kBlockThreads, 0, st>>>(a);
  return cudaGetLastError();
}

template <class P, class T>
static cudaError_t launch_cv(int cv, const PathArgs& a, int sms, cudaStream_t st, int* blocks) {
  switch (cv) {
    case kCvNone: return launch_one<P, T, kCvNone>(a, sms, st, blocks);
    case kCvGrid: return launch_one<P, T, kCvGrid>(a, sms, st, blocks);
    default: return launch_one<P, T, kCvExact>(a, sms, st, blocks);
  }
}

template <class T>
static cudaError_t launch_kind(int kind, int cv, const PathArgs& a, int sms, cudaStream_t st,
                               int* blocks) {
  switch (kind) {
    case 0: return launch_cv<Cfg0, T>(cv, a, sms, st, blocks);
    case 1: return launch_cv<Aniso, T>(cv, a, sms, st, blocks);
    case 2: return launch_cv<Cube3, T>(cv, a, sms, st, blocks);
    default: return launch_cv<Harmonic, T>(cv, a, sms, st, blocks);
  }
}

cudaError_t launch_paths(int kind, int precision, int cv, const PathArgs& a, int num_sms,
                         cudaStream_t st, int* blocks) {
  return precision == 1 ? launch_kind<double>(kind, cv, a, num_sms, st, blocks)
                        : launch_kind<float>(kind, cv, a, num_sms, st, blocks);
}

cudaError_t launch_finalize(const unsigned long long* acc, uint32_t n_nodes, double kappa,
                            const StatPtrs& out, cudaStream_t st) {
  const unsigned threads = 128;
  const unsigned blocks = (n_nodes + threads - 1) / threads;
  finalize_nodes<<<blocks, threads, 0, st>>>(acc, n_nodes, kappa, out);
  return cudaGetLastError();
}

}  // namespace pdd
