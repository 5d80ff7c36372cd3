// pdd_paths.cu -- the path kernels of the PDD Monte Carlo nodal stage
// (Bernal & Acebron, Algorithm 1 with the pathwise control variate of
// eq. F:xiControlVariate) and the per-node finalisation (eqs. F:Statistics_VR
// .. F:Rho, F:Pointwise_cost, F:VR_Pointwise_cost, F:nu).
//
// Execution model.  One path per lane.  The paths of all nodes form one flat
// path-major index space g = path * n_nodes + node (consecutive indices are
// different nodes, so the paths in flight at any moment spread their record
// atomics over all node records instead of queueing on one record's cache
// line); warps take batches of 32 indices from a global cursor (atomicAdd)
// and every lane whose path has finished takes the next index of its warp's
// batch at the next iteration boundary, so lanes stay busy whatever the
// spread of exit times (paths of one node range over ~12x the mean number of
// steps).  The grid is persistent (occupancy x SM count blocks).  A finished
// path parks in its warp's exit ring in shared memory and is scored and
// recorded later, 32 at a time by the whole warp; launches with at most 512
// node records add into a per-block shared-memory copy of the records, which
// the block adds into the global ones at the end.  Per-node sums are exact
// integers, so which lane, warp or block runs a path changes nothing in the
// results.
//
// One iteration takes as many Euler steps as one Philox block has normals
// for: two steps in 2D (4 normals), four steps in 3D (3 blocks, 12 normals),
// so no random word is wasted and every path's stream is the one fixed by
// its (seed, stream_tag, node, path) key.
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "pdd_device.cuh"
#include "pdd_internal.h"

namespace pdd {

constexpr int kBlockThreads = 128;     // default block size (smaller blocks retire sooner as a launch drains)
constexpr int kMaxBlockThreads = 512;  // largest block size a launch may ask for
// Minimum resident blocks per SM requested from the compiler (register cap).
#ifndef PDD_MIN_BLOCKS_2D
#define PDD_MIN_BLOCKS_2D 1
#endif
#ifndef PDD_MIN_BLOCKS_3D
#define PDD_MIN_BLOCKS_3D 2  // 64 registers: twice the warps of the unconstrained 3D kernel
#endif
constexpr unsigned kFull = 0xFFFFFFFFu;
// Euler steps per iteration of the path kernels (between lane refills and
// exit parking): 4 in 2D (two Philox blocks; 8 for the plain estimator, see
// LongSteps2D) and 8 in 3D (six) halve the
// per-step share of the refill, ring and loop work against 2 and 4, but a
// lane whose path ends early in an iteration idles for the rest of it, which
// costs on short paths.  A launch takes the longer iterations when segments
// with time steps above kLongPathH (paths of under ~100 steps) hold at most
// kShortWorkShare of its expected path-steps (n_nodes x n_paths / h per
// segment).
constexpr double kLongPathH = 2e-3;
// The long 2D iteration: eight steps (four Philox blocks) for the plain
// estimator, whose step is short enough that the refill and ring bookkeeping
// still weigh (+3 % path-steps/s against four), and four with a control
// variate (eight measured no faster).
template <class T, int CV>
struct LongSteps2D {
  static constexpr int value = sizeof(T) == 4 ? (CV == 0 ? 8 : 4) : 2;
};
constexpr double kShortWorkShare = 0.05;
enum { kCvNone = 0, kCvGrid = 1, kCvExact = 2 };

// Per-lane path state.
template <class T>
struct PathState {
  T x[3];
  T Y, Z, Zc, XI, XIc;
  int k;
  uint32_t node, path, seg;
};

// Per-lane copy of the parameters of the segment the lane's path belongs to.
// With a single segment they are the same for every lane and never change.
// FP32 paths read the cell-coefficient table, FP64 paths the nodal table
// (whose multilinear interpolation they evaluate in FP64, as the oracle does).
#ifndef PDD_CELLS_2D
#define PDD_CELLS_2D 1
#endif
#ifndef PDD_CELLS_3D
#define PDD_CELLS_3D 1
#endif
template <class T, int D>
struct UseCells {
  static constexpr bool value =
      sizeof(T) == 4 && ((D == 2 && PDD_CELLS_2D) || (D == 3 && PDD_CELLS_3D));
};

template <class T>
struct LaneSeg {
  T h, sqh, thr0;
  const void* grad;  // the table this lane reads (cells or nodal); null: no grid
  int gn, max_steps;
};

template <class T, int D>
__device__ __forceinline__ void load_seg(const SegArgs& sg, LaneSeg<T>& ls) {
  ls.h = (T)sg.h;
  ls.sqh = (T)sg.sqrt_h;
  ls.thr0 = (T)sg.thr0;
  ls.grad = sg.grad;
  if (UseCells<T, D>::value && sg.grad != nullptr)
    ls.grad = (const char*)sg.grad + cell_table_offset(sg.grid_n, D);
  ls.gn = sg.grid_n;
  ls.max_steps = sg.max_steps;
}

// Start path g of the launch's flat index space.
template <class T, int D, bool MULTI>
__device__ __forceinline__ void start_path(const PathArgs& a, unsigned long long g,
                                           PathState<T>& s, LaneSeg<T>& ls) {
  uint32_t si = 0;
  if (MULTI) {  // last segment whose begin <= g (segments in increasing begin)
    int lo = 0, hi = a.n_segs - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.seg[mid].begin <= g) lo = mid;
      else hi = mid - 1;
    }
    si = (uint32_t)lo;
  }
  const SegArgs& sg = a.seg[si];
  const unsigned long long li = g - sg.begin;
  if (!PDD_IN_BOUNDS(a, si < (uint32_t)a.n_segs && g >= sg.begin && li < sg.total && g < a.total,
                     kErrBoundsIndex)) {
    // leave the lane on node 0, path 0 of segment 0 (in bounds); the call fails
    s.node = s.path = s.seg = 0;
    s.x[0] = s.x[1] = s.x[2] = T(0.5);
    s.Y = T(1);
    s.Z = s.Zc = s.XI = s.XIc = T(0);
    s.k = 0;
    if (MULTI) load_seg<T, D>(a.seg[0], ls);
    return;
  }
  if (sg.total <= 0xFFFFFFFFull) {  // 32-bit division when the index space allows
    const uint32_t gg = (uint32_t)li, nn = (uint32_t)sg.n_nodes;
    const uint32_t p = gg / nn;
    s.node = gg - p * nn;
    s.path = sg.path_off + p;
  } else {
    const unsigned long long p = li / sg.n_nodes;
    s.node = (uint32_t)(li - p * sg.n_nodes);
    s.path = sg.path_off + (uint32_t)p;
  }
  s.seg = si;
  if (!PDD_IN_BOUNDS(a, s.node < sg.n_nodes && s.path - sg.path_off < sg.n_paths,
                     kErrBoundsIndex))
    s.node = 0;
  s.x[0] = (T)__ldg(sg.cx + s.node);
  s.x[1] = (T)__ldg(sg.cy + s.node);
  s.x[2] = (D == 3) ? (T)__ldg(sg.cz + s.node) : T(0);
  s.Y = T(1);
  s.Z = s.Zc = s.XI = s.XIc = T(0);
  s.k = 0;
  if (MULTI) load_seg<T, D>(sg, ls);
}

#ifndef PDD_EXIT_CENTRED
#define PDD_EXIT_CENTRED 1
#endif
// Finish test of Algorithm 1: d(X_k) >= -c0 |sigma^T N| sqrt(h).
template <class P, class T, int D>
__device__ __forceinline__ bool should_finish(const PathState<T>& s, T thr0) {
  T thr = thr0;
  if (P::kAniso || P::kIsoScaled) thr = mul_rn(thr, P::template exit_scale<T>(s.x[0], s.x[1], s.x[2]));
  if (sizeof(T) == 4 && PDD_EXIT_CENTRED) {
    // FP32: the distance to the unit box's faces is 1/2 - max_i |X_i - 1/2|,
    // one instruction fewer than the minimum over the 2D faces
    T e = fmaxf(fabsf(sub_rn(s.x[0], T(0.5))), fabsf(sub_rn(s.x[1], T(0.5))));
    if (D == 3) e = fmaxf(e, fabsf(sub_rn(s.x[2], T(0.5))));
    return e >= sub_rn(T(0.5), thr);
  }
  const T m = (D == 3) ? face_distance(s.x[0], s.x[1], s.x[2]) : face_distance(s.x[0], s.x[1]);
  return m <= thr;
}

// Philox block `blk` of the lane's path.
template <bool MULTI>
__device__ __forceinline__ uint4 path_block(const PathArgs& a, uint32_t seg, uint32_t blk,
                                            uint32_t path, uint32_t node) {
  const SegArgs& sg = a.seg[MULTI ? seg : 0];
  return philox4x32_10(make_uint4(blk, path, node, sg.seed_hi), make_uint2(sg.key0, sg.key1));
}

// One Euler-Maruyama step (eq. F:E_M) with the Feynman-Kac weights and the
// control variate, all right-hand sides at X_k.  dW holds sqrt(h) * normals.
// YRULE: the step honours the launch's Y rule (a.y_exp); without it the step
// uses the default Euler rule Y(1 - h c).  The single-segment build of the
// path kernels has YRULE = false and launches with the exponential rule go to
// the segment-table build: dropping the per-step choice made the
// single-segment build 2.4 % faster with the control variate, 5 % without.
template <class P, class T, int D, int CV, bool MULTI, bool YRULE = MULTI>
__device__ __forceinline__ void euler_step(const PathArgs& a, PathState<T>& s,
                                           const LaneSeg<T>& ls, const T* dW) {
  const T h = ls.h;
  // with several segments a segment without a grid runs the plain estimator
  constexpr bool kCv = CV != kCvNone;
  const bool use_cv = kCv && (CV != kCvGrid || !MULTI || ls.grad != nullptr);
  // The cell-record gather depends only on X_k: it is issued before the
  // coefficients are evaluated, so its latency overlaps their arithmetic.
  T gv[3] = {T(0), T(0), T(0)};
  if (CV == kCvGrid && use_cv) {
    if (D == 2) {
      if (UseCells<T, 2>::value)
        grid_cells_2d<T>((const float4*)ls.grad, ls.gn, s.x[0], s.x[1], gv[0], gv[1],
                         PDD_DEBUG_BOUNDS ? a.err : nullptr);
      else
        grid_grad_2d<T>((const float2*)ls.grad, ls.gn, s.x[0], s.x[1], gv[0], gv[1],
                        PDD_DEBUG_BOUNDS ? a.err : nullptr);
    } else {
      if (UseCells<T, 3>::value)
        grid_cells_3d<T>((const float4*)ls.grad, ls.gn, s.x[0], s.x[1], s.x[2], gv[0], gv[1],
                         gv[2], PDD_DEBUG_BOUNDS ? a.err : nullptr);
      else
        grid_grad_3d<T>((const float4*)ls.grad, ls.gn, s.x[0], s.x[1], s.x[2], gv[0], gv[1],
                        gv[2], PDD_DEBUG_BOUNDS ? a.err : nullptr);
    }
  }
  Coef<T> o;
  P::template eval<T, CV == kCvExact>(s.x[0], s.x[1], s.x[2], o);
  T sdW[3];
  const T dW0 = dW[0], dW1 = dW[1];
  if (P::kAniso) {  // sigma = sqrt(a) [[1, 0], [1/2, sqrt(3)/2]]
    sdW[0] = mul_rn(o.sa, dW0);
    sdW[1] = mul_rn(o.sa, fma_rn(T(0.86602540378443864676), dW1, mul_rn(T(0.5), dW0)));
  } else if (P::kIsoScaled) {  // sigma = sa I
    sdW[0] = mul_rn(o.sa, dW0);
    sdW[1] = mul_rn(o.sa, dW1);
  } else {
    sdW[0] = dW0;
    sdW[1] = dW1;
  }
  sdW[2] = (D == 3) ? dW[2] : T(0);
  if (use_cv) {
    if (CV == kCvExact) {
      gv[0] = o.g0;
      gv[1] = o.g1;
      gv[2] = o.g2;
    }
    T dot = fma_rn(gv[1], sdW[1], mul_rn(gv[0], sdW[0]));
    if (D == 3) dot = fma_rn(gv[2], sdW[2], dot);
    kahan_add(s.XI, s.XIc, -s.Y, dot);
  }
  // h Y_k serves the Z increment and the Euler rule Y_k (1 - h c) = Y_k - (h Y_k) c
  const T hY = P::kUnitY ? T(0) : mul_rn(h, s.Y);
  if (!P::kUnitY) kahan_add(s.Z, s.Zc, -hY, o.f);
  // the drift's step: h b, or (h/2)(2 b) for problems whose eval returns 2 b
  // (the same product: halving h is exact)
  const T hb = P::kDriftHalf ? mul_rn(T(0.5), h) : h;
  s.x[0] = add_rn(s.x[0], fma_rn(hb, o.b0, sdW[0]));
  s.x[1] = add_rn(s.x[1], fma_rn(hb, o.b1, sdW[1]));
  if (D == 3) s.x[2] = add_rn(s.x[2], fma_rn(hb, o.b2, sdW[2]));
  if (!P::kUnitY)
    s.Y = (YRULE && a.y_exp) ? mul_rn(s.Y, m_exp(mul_rn(-h, o.c))) : fma_rn(-hY, o.c, s.Y);
  s.k += 1;
}

// Exact fixed-point accumulation of one path's (phi, psi = phi + xi, k) into a
// node record (global, or the block's shared-memory copy), and of k into the
// launch's step counter `steps` when there is one.
template <class T>
__device__ __forceinline__ void accumulate(const PathArgs& a, unsigned long long* w,
                                           unsigned long long* steps, T phi, T psi, int k_steps,
                                           bool trunc) {
  long long qa, qb;
  const bool ok = to_fixed(phi, qa) & to_fixed(psi, qb);
  if (!ok) atomicOr(a.err, kErrOverflow);
  atomic_add_s64(w + 0, qa);
  atomic_add_prod(w + 2, qa, qa);
  atomic_add_s64(w + 4, qb);
  atomic_add_prod(w + 6, qb, qb);
  atomic_add_prod(w + 8, qa, qb);
  const unsigned long long k = (unsigned long long)k_steps;
  atomic_add_u128(w + 10, k, 0ull);
  atomic_add_u128(w + 12, k * k, 0ull);
  atomicAdd(w + 14, 1ull);
  if (trunc) {
    atomicAdd(w + 15, 1ull);
    atomicAdd(a.trunc_total, 1ull);
  }
  if (steps != nullptr) atomicAdd(steps, k);
}

// Block-level record cache.  When the launch's segments hold at most
// kCacheMaxNodes node records, every block keeps its own copy of them in
// shared memory: exits add into the copy with shared-memory atomics (exits of
// different nodes no longer meet on a few cache lines of L2), and once all
// warps of the block have finished the block adds its non-empty records into
// the global ones (128-bit adds with carry: the same exact sums).  Slot
// seg.cache_base + node holds the record of `node` of segment `seg`; the word
// after the last slot counts the block's exit indices for a.steps_total.
extern __shared__ unsigned long long s_cache[];
// Slot stride in 64-bit words: one word of padding per record, so the same
// word of consecutive slots falls in different shared-memory banks.
constexpr uint32_t kCacheStride = kAccWords + 1;

__device__ __forceinline__ void cache_init(const PathArgs& a) {
  if (a.cache_nodes == 0) return;
  const uint32_t words = a.cache_nodes * kCacheStride + 1;
  for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) s_cache[i] = 0ull;
  __syncthreads();
}

__device__ __forceinline__ void cache_flush(const PathArgs& a) {
  if (a.cache_nodes == 0) return;
  __syncthreads();
  const uint32_t pairs = a.cache_nodes * (kAccWords / 2);
  for (uint32_t i = threadIdx.x; i < pairs; i += blockDim.x) {
    const uint32_t slot = i / (kAccWords / 2), q = i % (kAccWords / 2);
    const unsigned long long* s = s_cache + (size_t)slot * kCacheStride;
    if (s[14] == 0ull) continue;  // no path of this node ended in this block
    int lo = 0, hi = a.n_segs - 1;  // last segment whose cache_base <= slot
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.seg[mid].cache_base <= slot) lo = mid;
      else hi = mid - 1;
    }
    const SegArgs& sg = a.seg[lo];
    if (!PDD_IN_BOUNDS(a, slot >= sg.cache_base && slot - sg.cache_base < sg.n_nodes,
                       kErrBoundsRecord))
      continue;
    unsigned long long* g = sg.acc + (size_t)(slot - sg.cache_base) * kAccWords;
    if (q < 7) {
      if ((s[2 * q] | s[2 * q + 1]) != 0ull) atomic_add_u128(g + 2 * q, s[2 * q], s[2 * q + 1]);
    } else {
      atomicAdd(g + 14, s[14]);
      if (s[15] != 0ull) atomicAdd(g + 15, s[15]);
    }
  }
  if (threadIdx.x == 0 && a.steps_total != nullptr) {
    const unsigned long long st = s_cache[(size_t)a.cache_nodes * kCacheStride];
    if (st != 0ull) atomicAdd(a.steps_total, st);
  }
}

// Add one path into the record of `node` of segment `sg` (cached or global).
template <class T>
__device__ __forceinline__ void record_path(const PathArgs& a, const SegArgs& sg, uint32_t node,
                                            T phi, T psi, int k_steps, bool trunc) {
  if (!PDD_IN_BOUNDS(a, node < sg.n_nodes, kErrBoundsRecord)) return;
  if (a.cache_nodes != 0) {
    if (!PDD_IN_BOUNDS(a, sg.cache_base + node < a.cache_nodes, kErrBoundsRecord)) return;
    accumulate(a, s_cache + (size_t)(sg.cache_base + node) * kCacheStride,
               a.steps_total != nullptr ? s_cache + (size_t)a.cache_nodes * kCacheStride : nullptr,
               phi, psi, k_steps, trunc);
  } else {
    accumulate(a, sg.acc + (size_t)node * kAccWords, a.steps_total, phi, psi, k_steps, trunc);
  }
}

// Exit scoring: X_tau = Pi(X_k), phi = g(X_tau) Y + Z, and xi.
template <class P, class T, int D>
__device__ __forceinline__ void score_path(const PathState<T>& s, T& phi, T& xi) {
  T p[3] = {s.x[0], s.x[1], s.x[2]};
  project_box<T>(p, D);
  const T g = P::template g<T>(p[0], p[1], p[2]);
  phi = fma_rn(g, s.Y, sub_rn(s.Z, s.Zc));
  xi = sub_rn(s.XI, s.XIc);
}

// Exit scoring and the exact fixed-point accumulation into the node record.
template <class P, class T, int D, bool MULTI>
__device__ __forceinline__ void finish_path(const PathArgs& a, const PathState<T>& s, bool trunc) {
  T phi, xi;
  score_path<P, T, D>(s, phi, xi);
  const SegArgs& sg = a.seg[MULTI ? s.seg : 0];
  record_path(a, sg, s.node, phi, phi + xi, s.k, trunc);
  if (sg.emit_phi != nullptr) {
    const size_t i = (size_t)s.node * sg.emit_stride + s.path;
    if (!PDD_IN_BOUNDS(a, i < sg.n_nodes * sg.emit_stride, kErrBoundsEmit)) return;
    sg.emit_phi[i] = (float)phi;
    sg.emit_xi[i] = (float)xi;
    sg.emit_steps[i] = s.k;
  }
}

// Refill idle lanes from the warp's batch; returns false when no lane of the
// warp has a path left to run.  All arguments except the lane state are
// warp-uniform.
template <class T, int D, bool MULTI>
__device__ __forceinline__ bool refill(const PathArgs& a, PathState<T>& s, LaneSeg<T>& ls,
                                       bool& active, unsigned long long& bnext,
                                       unsigned long long& bend, bool& exhausted) {
  const unsigned lane = threadIdx.x & 31u;
  const unsigned lt = (1u << lane) - 1u;
  unsigned idle = __ballot_sync(kFull, !active);
  while (idle != 0u && !exhausted) {
    if (bnext >= bend) {
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(a.cursor, a.warp_batch);
      base = __shfl_sync(kFull, base, 0);
      if (base >= a.total) {
        exhausted = true;
        break;
      }
      bnext = base;
      bend = min(base + a.warp_batch, a.total);
    }
    const unsigned avail = (unsigned)min(bend - bnext, 32ull);
    const unsigned rank = __popc(idle & lt);
    if (!active && rank < avail) {
      start_path<T, D, MULTI>(a, bnext + rank, s, ls);
      active = true;
    }
    bnext += min((unsigned)__popc(idle), avail);
    idle = __ballot_sync(kFull, !active);
  }
  return __ballot_sync(kFull, active) != 0u;
}

// Per-warp exit ring.  A lane whose path has ended parks the path's final
// state (X, Y, Z, xi, k, node, path, segment | truncated) in its warp's ring
// in shared memory and takes a new path at once; whenever 32 exits are
// parked, the whole warp scores and records them, one per lane.  Exit work
// (projection, g, fixed-point conversion, the record's 13 atomic adds) thus
// runs with all lanes busy instead of one lane at a time while the rest of
// the warp waits.  Rings follow the record cache in dynamic shared memory.
constexpr uint32_t kRing = 64;  // entries per warp (>= 2 x 32: a full batch plus one iteration)
template <class T, int D>
struct ExitRing {
  static constexpr size_t kBytes = kRing * ((D + 3) * sizeof(T) + 4 * sizeof(uint32_t));
  T* f;         // (D + 3) x kRing: X_0 .. X_(D-1), Y, Z, xi
  uint32_t* u;  // 4 x kRing: k, node, path, segment | truncated << 31
};

__host__ __device__ __forceinline__ size_t cache_bytes(uint32_t cache_nodes) {
  if (cache_nodes == 0) return 0;
  return (((size_t)cache_nodes * (kAccWords + 1) + 1) * 8 + 15) / 16 * 16;
}

template <class T, int D>
__device__ __forceinline__ ExitRing<T, D> ring_of_warp(const PathArgs& a) {
  char* base = (char*)s_cache + cache_bytes(a.cache_nodes) +
               (size_t)(threadIdx.x >> 5) * ExitRing<T, D>::kBytes;
  ExitRing<T, D> r;
  r.f = (T*)base;
  r.u = (uint32_t*)(base + kRing * (D + 3) * sizeof(T));
  return r;
}

template <class T, int D>
__device__ __forceinline__ void ring_put(const ExitRing<T, D>& r, uint32_t j,
                                         const PathState<T>& s, bool trunc) {
#pragma unroll
  for (int d = 0; d < D; ++d) r.f[d * kRing + j] = s.x[d];
  r.f[D * kRing + j] = s.Y;
  r.f[(D + 1) * kRing + j] = s.Z - s.Zc;
  r.f[(D + 2) * kRing + j] = s.XI - s.XIc;
  r.u[j] = (uint32_t)s.k;
  r.u[kRing + j] = s.node;
  r.u[2 * kRing + j] = s.path;
  r.u[3 * kRing + j] = s.seg | (trunc ? 0x80000000u : 0u);
}

// Score and record `count` (<= 32) parked exits starting at ring slot `first`.
template <class P, class T, int D, bool MULTI>
__device__ __forceinline__ void ring_drain(const PathArgs& a, const ExitRing<T, D>& r,
                                           uint32_t first, uint32_t count) {
  __syncwarp();
  const uint32_t lane = threadIdx.x & 31u;
  if (lane < count) {
    const uint32_t j = (first + lane) & (kRing - 1);
    PathState<T> e;
    e.x[0] = e.x[1] = e.x[2] = T(0);
#pragma unroll
    for (int d = 0; d < D; ++d) e.x[d] = r.f[d * kRing + j];
    e.Y = r.f[D * kRing + j];
    e.Z = r.f[(D + 1) * kRing + j];
    e.XI = r.f[(D + 2) * kRing + j];
    e.Zc = e.XIc = T(0);
    e.k = (int)r.u[j];
    e.node = r.u[kRing + j];
    e.path = r.u[2 * kRing + j];
    const uint32_t st = r.u[3 * kRing + j];
    e.seg = st & 0x7FFFFFFFu;
    finish_path<P, T, D, MULTI>(a, e, (st >> 31) != 0u);
  }
  __syncwarp();
}

// Warp-uniform ring cursor: `head` counts parked exits, `held` those not yet
// drained.
struct RingCursor {
  uint32_t head = 0, held = 0;
};

// Park the exits of this iteration (`done` lanes) and drain a full batch.
template <class P, class T, int D, bool MULTI>
__device__ __forceinline__ void ring_exit(const PathArgs& a, const ExitRing<T, D>& r,
                                          RingCursor& c, const PathState<T>& s, bool done,
                                          bool trunc) {
  const unsigned m = __ballot_sync(kFull, done);
  if (m == 0u) return;
  // never more than kRing parked: fewer than 32 are held before this iteration
  if (!PDD_IN_BOUNDS(a, c.held + __popc(m) <= kRing, kErrBoundsRing)) return;
  if (done) {
    const unsigned lt = (1u << (threadIdx.x & 31u)) - 1u;
    ring_put<T, D>(r, (c.head + __popc(m & lt)) & (kRing - 1), s, trunc);
  }
  c.head += __popc(m);
  c.held += __popc(m);
  if (c.held >= 32u) {
    ring_drain<P, T, D, MULTI>(a, r, c.head - c.held, 32u);
    c.held -= 32u;
  }
}

template <class T, int D>
__device__ __forceinline__ void init_lane(const PathArgs& a, PathState<T>& s, LaneSeg<T>& ls) {
  s.x[0] = s.x[1] = s.x[2] = T(0);
  s.Y = s.Z = s.Zc = s.XI = s.XIc = T(0);
  s.k = 0;
  s.node = s.path = s.seg = 0;
  load_seg<T, D>(a.seg[0], ls);
}

// One ordinary iteration: STEPS / 2 Philox blocks, two steps each; the exit
// test precedes every step.  `fin` / `trunc` report a path that ended.
template <class P, class T, int CV, bool MULTI, int STEPS>
__device__ __forceinline__ void iteration_2d(const PathArgs& a, PathState<T>& s,
                                             const LaneSeg<T>& ls, bool active, bool& fin,
                                             bool& trunc) {
#pragma unroll
  for (int half = 0; half < STEPS / 2; ++half) {
    uint4 w = make_uint4(0, 0, 0, 0);
    if (active && !fin) fin = should_finish<P, T, 2>(s, ls.thr0);
    if (active && !fin) {
      w = path_block<MULTI>(a, s.seg, (uint32_t)(s.k >> 1), s.path, s.node);
      T n[3];
      box_muller(w.x, w.y, n[0], n[1], ls.sqh);
      n[2] = T(0);
      euler_step<P, T, 2, CV, MULTI>(a, s, ls, n);
      if (s.k >= ls.max_steps) fin = trunc = true;
    }
    if (active && !fin) fin = should_finish<P, T, 2>(s, ls.thr0);
    if (active && !fin) {
      T n[3];
      box_muller(w.z, w.w, n[0], n[1], ls.sqh);
      n[2] = T(0);
      euler_step<P, T, 2, CV, MULTI>(a, s, ls, n);
      if (s.k >= ls.max_steps) fin = trunc = true;
    }
  }
}

// Drain iterations.  Once the launch's cursor is exhausted a warp only
// finishes the paths it holds; as lanes retire, the launch's time becomes the
// serial latency of its longest paths, and a lone path spends most of each
// step drawing its random numbers (Philox rounds, Box-Muller), which do not
// depend on the path's state.  When at most half the lanes of a warp still
// run a path, the idle lanes draw them: with A running lanes, every lane L
// computes Philox block m = L / A of running lane L mod A (counted from that
// lane's current block) and its four normals, and the running lanes then take
// 2 * floor(32 / A) steps reading their normals from the helpers with warp
// shuffles.  The values are the ones a lane would draw itself (same key,
// same counter, same arithmetic), so results do not change.
#ifndef PDD_TAIL_COOP
#define PDD_TAIL_COOP 1
#endif

// Position of the q-th (from 0) set bit of m, q < popc(m): the largest p
// with fewer than q + 1 set bits below it, by binary search.
__device__ __forceinline__ int nth_set_bit(unsigned m, int q) {
  int p = 0;
#pragma unroll
  for (int w = 16; w >= 1; w >>= 1)
    if (__popc(m & ((1u << (p + w)) - 1u)) <= q) p += w;
  return p;
}

// Helper side: this lane's Philox block (block blk + m, m = lane / A, of
// running lane lane % A, whose current block counter is `blk`) as four scaled
// normals; lanes with lane / A >= blocks draw none.
template <class T, bool MULTI>
__device__ __forceinline__ void coop_draw(const PathArgs& a, const PathState<T>& s,
                                          const LaneSeg<T>& ls, unsigned runm, int blocks,
                                          uint32_t blk, T (&nv)[4]) {
  const int lane = (int)(threadIdx.x & 31u), A = __popc(runm);
  const int q = lane % A, m = lane / A;
  const int owner = nth_set_bit(runm, q);
  const uint32_t o_seg = __shfl_sync(kFull, s.seg, owner);
  const uint32_t o_path = __shfl_sync(kFull, s.path, owner);
  const uint32_t o_node = __shfl_sync(kFull, s.node, owner);
  const uint32_t o_blk = __shfl_sync(kFull, blk, owner);
  const T o_sqh = __shfl_sync(kFull, ls.sqh, owner);
  nv[0] = nv[1] = nv[2] = nv[3] = T(0);
  if (m < blocks) {
    const uint4 w = path_block<MULTI>(a, o_seg, o_blk + (uint32_t)m, o_path, o_node);
    box_muller(w.x, w.y, nv[0], nv[1], o_sqh);
    box_muller(w.z, w.w, nv[2], nv[3], o_sqh);
  }
}

// 2D: block m of a running lane feeds its steps 2m and 2m + 1 (normals 4m ..
// 4m + 3), so the lane's counter at the iteration start is even.
template <class P, class T, int CV, bool MULTI>
__device__ __forceinline__ void coop_iteration_2d(const PathArgs& a, PathState<T>& s,
                                                  const LaneSeg<T>& ls, bool active,
                                                  unsigned runm, bool& fin, bool& trunc) {
  const unsigned lane = threadIdx.x & 31u;
  const int A = __popc(runm), blocks = 32 / A;
  T nv[4];
  coop_draw<T, MULTI>(a, s, ls, runm, blocks, (uint32_t)s.k >> 1, nv);
  const int r = __popc(runm & ((1u << lane) - 1u));  // rank among running lanes
  bool run = active;
  for (int m = 0; m < blocks; ++m) {
    const int src = (r + A * m) & 31;
#pragma unroll
    for (int h2 = 0; h2 < 2; ++h2) {
      T n[3];
      n[0] = __shfl_sync(kFull, nv[2 * h2], src);
      n[1] = __shfl_sync(kFull, nv[2 * h2 + 1], src);
      n[2] = T(0);
      if (run) run = !should_finish<P, T, 2>(s, ls.thr0);
      if (run) {
        euler_step<P, T, 2, CV, MULTI>(a, s, ls, n);
        if (s.k >= ls.max_steps) {
          trunc = true;
          run = false;
        }
      }
    }
    if (__ballot_sync(kFull, run) == 0u) break;
  }
  fin = active && !run;
}

// The segment-table build keeps per-lane segment parameters in registers; at
// 65 registers a 512-thread block rounds up to 72 per thread and only one
// block fits an SM, so it is capped at 64 (two blocks), which measured faster
// than the uncapped build.
template <class P, class T, int CV, bool MULTI, int STEPS>
__global__ void __launch_bounds__(kMaxBlockThreads, (MULTI && sizeof(T) == 4) ? 2
                                                                               : PDD_MIN_BLOCKS_2D)
    paths_2d(const __grid_constant__ PathArgs a) {
  PathState<T> s;
  LaneSeg<T> ls;
  init_lane<T, 2>(a, s, ls);
  cache_init(a);
  const ExitRing<T, 2> ring = ring_of_warp<T, 2>(a);
  RingCursor rc;
  bool active = false, exhausted = false;
  unsigned long long bnext = 0, bend = 0;
  while (refill<T, 2, MULTI>(a, s, ls, active, bnext, bend, exhausted)) {
    if (PDD_TAIL_COOP && exhausted) break;  // warp-uniform: on to the drain
    bool fin = false, trunc = false;
    // the body of iteration_2d, written out: inlining the function here
    // changes the compiler's schedule of this loop (measured slower)
#pragma unroll
    for (int half = 0; half < STEPS / 2; ++half) {
      uint4 w = make_uint4(0, 0, 0, 0);
      if (active && !fin) fin = should_finish<P, T, 2>(s, ls.thr0);
      if (active && !fin) {
        w = path_block<MULTI>(a, s.seg, (uint32_t)(s.k >> 1), s.path, s.node);
        T n[3];
        box_muller(w.x, w.y, n[0], n[1], ls.sqh);
        n[2] = T(0);
        euler_step<P, T, 2, CV, MULTI>(a, s, ls, n);
        if (s.k >= ls.max_steps) fin = trunc = true;
      }
      if (active && !fin) fin = should_finish<P, T, 2>(s, ls.thr0);
      if (active && !fin) {
        T n[3];
        box_muller(w.z, w.w, n[0], n[1], ls.sqh);
        n[2] = T(0);
        euler_step<P, T, 2, CV, MULTI>(a, s, ls, n);
        if (s.k >= ls.max_steps) fin = trunc = true;
      }
    }
    ring_exit<P, T, 2, MULTI>(a, ring, rc, s, active && fin, trunc);
    if (fin) active = false;
  }
  // drain: the cursor is exhausted and the warp finishes the paths it holds
  while (PDD_TAIL_COOP && exhausted) {
    const unsigned runm = __ballot_sync(kFull, active);
    if (runm == 0u) break;
    bool fin = false, trunc = false;
    coop_iteration_2d<P, T, CV, MULTI>(a, s, ls, active, runm, fin, trunc);
    ring_exit<P, T, 2, MULTI>(a, ring, rc, s, active && fin, trunc);
    if (fin) active = false;
  }
  if (rc.held > 0u) ring_drain<P, T, 2, MULTI>(a, ring, rc.head - rc.held, rc.held);
  cache_flush(a);
}

// 3D: steps 4j .. 4j+3 use normals 12j .. 12j+11, i.e. Philox blocks 3j,
// 3j+1, 3j+2 (words a0..a3, b0..b3, c0..c3):
//   step 0: a0 a1 a2   step 1: a3 b0 b1   step 2: b2 b3 c0   step 3: c1 c2 c3
// Blocks are drawn only when the path is still running.  STEPS / 4 such
// groups of four steps run per iteration (between lane refills).
// One ordinary 3D iteration runs STEPS / 4 such groups; the exit test
// precedes every step.
template <class P, class T, int CV, bool MULTI, int STEPS>
__device__ __forceinline__ void iteration_3d(const PathArgs& a, PathState<T>& s,
                                             const LaneSeg<T>& ls, bool active, bool& fin,
                                             bool& trunc) {
#pragma unroll
  for (int quad = 0; quad < STEPS / 4; ++quad) {
    T carry0 = T(0), carry1 = T(0);  // normals left over from the previous block
    uint4 w = make_uint4(0, 0, 0, 0);
    const uint32_t blk0 = 3u * ((uint32_t)s.k >> 2);
    // step 0
    if (active && !fin) fin = should_finish<P, T, 3>(s, ls.thr0);
    if (active && !fin) {
      w = path_block<MULTI>(a, s.seg, blk0, s.path, s.node);
      T n[3], n3;
      box_muller(w.x, w.y, n[0], n[1], ls.sqh);
      box_muller(w.z, w.w, n[2], n3, ls.sqh);
      carry0 = n3;
      euler_step<P, T, 3, CV, MULTI>(a, s, ls, n);
      if (s.k >= ls.max_steps) fin = trunc = true;
    }
    // step 1
    if (active && !fin) fin = should_finish<P, T, 3>(s, ls.thr0);
    if (active && !fin) {
      w = path_block<MULTI>(a, s.seg, blk0 + 1u, s.path, s.node);
      T n[3];
      n[0] = carry0;
      box_muller(w.x, w.y, n[1], n[2], ls.sqh);
      euler_step<P, T, 3, CV, MULTI>(a, s, ls, n);
      if (s.k >= ls.max_steps) fin = trunc = true;
    }
    // step 2
    if (active && !fin) fin = should_finish<P, T, 3>(s, ls.thr0);
    if (active && !fin) {
      T n[3];
      box_muller(w.z, w.w, n[0], n[1], ls.sqh);
      w = path_block<MULTI>(a, s.seg, blk0 + 2u, s.path, s.node);
      box_muller(w.x, w.y, n[2], carry1, ls.sqh);
      euler_step<P, T, 3, CV, MULTI>(a, s, ls, n);
      if (s.k >= ls.max_steps) fin = trunc = true;
    }
    // step 3
    if (active && !fin) fin = should_finish<P, T, 3>(s, ls.thr0);
    if (active && !fin) {
      T n[3];
      n[0] = carry1;
      box_muller(w.z, w.w, n[1], n[2], ls.sqh);
      euler_step<P, T, 3, CV, MULTI>(a, s, ls, n);
      if (s.k >= ls.max_steps) fin = trunc = true;
    }
  }
}

// The 3D drain iteration: a running lane's block counter at the iteration
// start is 3 k / 4 (k a multiple of four); with A <= 10 running lanes each
// takes 4 * floor(floor(32 / A) / 3) steps, normal i of a group of four steps
// coming from helper block i / 4 of that group, word i mod 4.
template <class P, class T, int CV, bool MULTI>
__device__ __forceinline__ void coop_iteration_3d(const PathArgs& a, PathState<T>& s,
                                                  const LaneSeg<T>& ls, bool active,
                                                  unsigned runm, bool& fin, bool& trunc) {
  const unsigned lane = threadIdx.x & 31u;
  const int A = __popc(runm), quads = (32 / A) / 3;
  T nv[4];
  coop_draw<T, MULTI>(a, s, ls, runm, 3 * quads, 3u * ((uint32_t)s.k >> 2), nv);
  const int r = __popc(runm & ((1u << lane) - 1u));
  bool run = active;
  for (int j = 0; j < quads; ++j) {
#pragma unroll
    for (int st = 0; st < 4; ++st) {
      T n[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int i = 3 * st + c;  // normal index within the group of four steps
        n[c] = __shfl_sync(kFull, nv[i & 3], (r + A * (3 * j + (i >> 2))) & 31);
      }
      if (run) run = !should_finish<P, T, 3>(s, ls.thr0);
      if (run) {
        euler_step<P, T, 3, CV, MULTI>(a, s, ls, n);
        if (s.k >= ls.max_steps) {
          trunc = true;
          run = false;
        }
      }
    }
    if (__ballot_sync(kFull, run) == 0u) break;
  }
  fin = active && !run;
}

template <class P, class T, int CV, bool MULTI, int STEPS>
__global__ void __launch_bounds__(kMaxBlockThreads, PDD_MIN_BLOCKS_3D)
    paths_3d(const __grid_constant__ PathArgs a) {
  PathState<T> s;
  LaneSeg<T> ls;
  init_lane<T, 3>(a, s, ls);
  cache_init(a);
  const ExitRing<T, 3> ring = ring_of_warp<T, 3>(a);
  RingCursor rc;
  bool active = false, exhausted = false;
  unsigned long long bnext = 0, bend = 0;
  // The ordinary iterations run until the cursor is exhausted and at most
  // ten lanes of the warp still run a path (warp-uniform); then drain
  // iterations alternate with the check.
  for (;;) {
  while (refill<T, 3, MULTI>(a, s, ls, active, bnext, bend, exhausted)) {
    if (PDD_TAIL_COOP && exhausted && __popc(__ballot_sync(kFull, active)) <= 10) break;
    bool fin = false, trunc = false;
    // the body of iteration_3d, written out (as in paths_2d)
#pragma unroll
    for (int quad = 0; quad < STEPS / 4; ++quad) {
      T carry0 = T(0), carry1 = T(0);  // normals left over from the previous block
      uint4 w = make_uint4(0, 0, 0, 0);
      const uint32_t blk0 = 3u * ((uint32_t)s.k >> 2);
      // step 0
      if (active && !fin) fin = should_finish<P, T, 3>(s, ls.thr0);
      if (active && !fin) {
        w = path_block<MULTI>(a, s.seg, blk0, s.path, s.node);
        T n[3], n3;
        box_muller(w.x, w.y, n[0], n[1], ls.sqh);
        box_muller(w.z, w.w, n[2], n3, ls.sqh);
        carry0 = n3;
        euler_step<P, T, 3, CV, MULTI>(a, s, ls, n);
        if (s.k >= ls.max_steps) fin = trunc = true;
      }
      // step 1
      if (active && !fin) fin = should_finish<P, T, 3>(s, ls.thr0);
      if (active && !fin) {
        w = path_block<MULTI>(a, s.seg, blk0 + 1u, s.path, s.node);
        T n[3];
        n[0] = carry0;
        box_muller(w.x, w.y, n[1], n[2], ls.sqh);
        euler_step<P, T, 3, CV, MULTI>(a, s, ls, n);
        if (s.k >= ls.max_steps) fin = trunc = true;
      }
      // step 2
      if (active && !fin) fin = should_finish<P, T, 3>(s, ls.thr0);
      if (active && !fin) {
        T n[3];
        box_muller(w.z, w.w, n[0], n[1], ls.sqh);
        w = path_block<MULTI>(a, s.seg, blk0 + 2u, s.path, s.node);
        box_muller(w.x, w.y, n[2], carry1, ls.sqh);
        euler_step<P, T, 3, CV, MULTI>(a, s, ls, n);
        if (s.k >= ls.max_steps) fin = trunc = true;
      }
      // step 3
      if (active && !fin) fin = should_finish<P, T, 3>(s, ls.thr0);
      if (active && !fin) {
        T n[3];
        n[0] = carry1;
        box_muller(w.z, w.w, n[1], n[2], ls.sqh);
        euler_step<P, T, 3, CV, MULTI>(a, s, ls, n);
        if (s.k >= ls.max_steps) fin = trunc = true;
      }
    }
    ring_exit<P, T, 3, MULTI>(a, ring, rc, s, active && fin, trunc);
    if (fin) active = false;
  }
  const unsigned runm = __ballot_sync(kFull, active);
  if (!PDD_TAIL_COOP || runm == 0u) break;
  bool fin = false, trunc = false;
  coop_iteration_3d<P, T, CV, MULTI>(a, s, ls, active, runm, fin, trunc);
  ring_exit<P, T, 3, MULTI>(a, ring, rc, s, active && fin, trunc);
  if (fin) active = false;
  }
  if (rc.held > 0u) ring_drain<P, T, 3, MULTI>(a, ring, rc.head - rc.held, rc.held);
  cache_flush(a);
}

// ---------------------------------------------------------------------------
// Multilevel coupling: per lane a fine path at h_f = h/2 on the path's own
// stream and a coarse path at h driven by the sums of pairs of fine
// increments, dW_c(m) = dW_f(2m) + dW_f(2m+1).  Iteration j draws the
// Philox blocks that feed kFine fine steps (2D: block j, normals 4j .. 4j+3,
// two fine steps; 3D: blocks 3j .. 3j+2, normals 12j .. 12j+11, four fine
// steps) and the kFine / 2 coarse steps those increments make.  Each path
// has its own exit test; when both have finished the lane adds
// (phi_f, phi_f + xi_f) to the fine records (seg[0].acc) and the differences
// (phi_f - phi_c, psi_f - psi_c) with the coarse exit index to the
// difference records (seg[1].acc).  seg[0] holds the fine step and the node /
// path layout (path_off included), seg[1] the coarse step; emit pointers of
// seg[0] / seg[1] receive fine / coarse per-path output.
// ---------------------------------------------------------------------------
template <int D>
struct CoupledShape {
  static constexpr int kBlocks = D == 2 ? 1 : 3;        // Philox blocks per iteration
  static constexpr int kNormals = 4 * kBlocks;
  static constexpr int kFine = kNormals / D;            // fine steps per iteration
  static constexpr int kCoarse = kFine / 2;
};

// Per-warp ring of finished pairs (the coupled counterpart of ExitRing): the
// two scores of each path, both exit indices, node, path and truncation
// flags; drained 32 pairs at a time into the fine and difference records.
template <class T>
struct PairRing {
  static constexpr size_t kBytes = kRing * (4 * sizeof(T) + 5 * sizeof(uint32_t));
  T* f;         // 4 x kRing: phi_f, xi_f, phi_c, xi_c
  uint32_t* u;  // 5 x kRing: k_f, k_c, node, path, truncated (bit 0 fine, bit 1 coarse)
};

template <class T>
__device__ __forceinline__ PairRing<T> pair_ring_of_warp(const PathArgs& a) {
  char* base = (char*)s_cache + cache_bytes(a.cache_nodes) +
               (size_t)(threadIdx.x >> 5) * PairRing<T>::kBytes;
  PairRing<T> r;
  r.f = (T*)base;
  r.u = (uint32_t*)(base + kRing * 4 * sizeof(T));
  return r;
}

template <class T>
__device__ __forceinline__ void pair_drain(const PathArgs& a, const PairRing<T>& r,
                                           uint32_t first, uint32_t count) {
  __syncwarp();
  const uint32_t lane = threadIdx.x & 31u;
  if (lane < count) {
    const uint32_t j = (first + lane) & (kRing - 1);
    const T phif = r.f[j], xif = r.f[kRing + j], phic = r.f[2 * kRing + j],
            xic = r.f[3 * kRing + j];
    const int kf = (int)r.u[j], kc = (int)r.u[kRing + j];
    const uint32_t node = r.u[2 * kRing + j], path = r.u[3 * kRing + j];
    const uint32_t tr = r.u[4 * kRing + j];
    const SegArgs& s0 = a.seg[0];
    const SegArgs& s1 = a.seg[1];
    record_path(a, s0, node, phif, phif + xif, kf, (tr & 1u) != 0u);
    record_path(a, s1, node, phif - phic, (phif + xif) - (phic + xic), kc, (tr & 2u) != 0u);
    if (s0.emit_phi != nullptr &&
        PDD_IN_BOUNDS(a, (size_t)node * s0.emit_stride + path < s0.n_nodes * s0.emit_stride,
                      kErrBoundsEmit)) {
      const size_t i = (size_t)node * s0.emit_stride + path;
      s0.emit_phi[i] = (float)phif;
      s0.emit_xi[i] = (float)xif;
      s0.emit_steps[i] = kf;
      s1.emit_phi[i] = (float)phic;
      s1.emit_xi[i] = (float)xic;
      s1.emit_steps[i] = kc;
    }
  }
  __syncwarp();
}

template <class P, class T, int CV, int D>
__global__ void __launch_bounds__(kMaxBlockThreads, 1) paths_coupled(
    const __grid_constant__ PathArgs a) {
  using S = CoupledShape<D>;
  const PairRing<T> ring = pair_ring_of_warp<T>(a);
  RingCursor rc;
  PathState<T> f, c;
  LaneSeg<T> lf, lc;
  init_lane<T, D>(a, f, lf);
  init_lane<T, D>(a, c, lc);
  load_seg<T, D>(a.seg[1], lc);
  cache_init(a);
  bool active = false, exhausted = false;  // active: the pair still has work
  bool af = false, ac = false;             // fine / coarse path running
  bool tf = false, tc = false;             // truncated
  T phif = T(0), xif = T(0), phic = T(0), xic = T(0);
  uint32_t j = 0;
  unsigned long long bnext = 0, bend = 0;
  while (refill<T, D, false>(a, f, lf, active, bnext, bend, exhausted)) {
    if (active && f.k == 0 && !af && !ac) {  // refill has just started a new pair in f
      c = f;
      af = ac = true;
      tf = tc = false;
      j = 0;
    }
    if (active) {
      T n[S::kNormals];
#pragma unroll
      for (int b = 0; b < S::kBlocks; ++b) {
        const uint4 w = path_block<false>(a, 0, S::kBlocks * j + b, f.path, f.node);
        box_muller(w.x, w.y, n[4 * b], n[4 * b + 1], lf.sqh);
        box_muller(w.z, w.w, n[4 * b + 2], n[4 * b + 3], lf.sqh);
      }
      if (af) {
#pragma unroll
        for (int q = 0; q < S::kFine; ++q) {
          if (af) {
            if (should_finish<P, T, D>(f, lf.thr0)) {
              af = false;
            } else {
              T d[3] = {n[D * q], n[D * q + 1], D == 3 ? n[D * q + 2] : T(0)};
              euler_step<P, T, D, CV, false, true>(a, f, lf, d);
              if (f.k >= lf.max_steps) {
                af = false;
                tf = true;
              }
            }
          }
        }
        if (!af) score_path<P, T, D>(f, phif, xif);
      }
      if (ac) {
#pragma unroll
        for (int q = 0; q < S::kCoarse; ++q) {
          if (ac) {
            if (should_finish<P, T, D>(c, lc.thr0)) {
              ac = false;
            } else {
              const int o = 2 * D * q;  // fine steps 2q and 2q+1 of this iteration
              T d[3] = {n[o] + n[o + D], n[o + 1] + n[o + D + 1],
                        D == 3 ? n[o + 2] + n[o + D + 2] : T(0)};
              euler_step<P, T, D, CV, false, true>(a, c, lc, d);
              if (c.k >= lc.max_steps) {
                ac = false;
                tc = true;
              }
            }
          }
        }
        if (!ac) score_path<P, T, D>(c, phic, xic);
      }
      j += 1;
    }
    // park finished pairs; drain 32 at a time with the whole warp
    const bool done = active && !af && !ac;
    const unsigned m = __ballot_sync(kFull, done);
    // never more than kRing parked: fewer than 32 are held before this iteration
    // (bounds-checked build: an over-full ring drops the pairs, never stalls)
    if (m != 0u && !PDD_IN_BOUNDS(a, rc.held + __popc(m) <= kRing, kErrBoundsRing)) {
      if (done) active = false;
    } else if (m != 0u) {
      if (done) {
        const unsigned lt = (1u << (threadIdx.x & 31u)) - 1u;
        const uint32_t q = (rc.head + __popc(m & lt)) & (kRing - 1);
        ring.f[q] = phif;
        ring.f[kRing + q] = xif;
        ring.f[2 * kRing + q] = phic;
        ring.f[3 * kRing + q] = xic;
        ring.u[q] = (uint32_t)f.k;
        ring.u[kRing + q] = (uint32_t)c.k;
        ring.u[2 * kRing + q] = f.node;
        ring.u[3 * kRing + q] = f.path;
        ring.u[4 * kRing + q] = (tf ? 1u : 0u) | (tc ? 2u : 0u);
        active = false;
      }
      rc.head += __popc(m);
      rc.held += __popc(m);
      if (rc.held >= 32u) {
        pair_drain<T>(a, ring, rc.head - rc.held, 32u);
        rc.held -= 32u;
      }
    }
  }
  if (rc.held > 0u) pair_drain<T>(a, ring, rc.head - rc.held, rc.held);
  cache_flush(a);
}

template <class P, class T, int CV, int D>
static cudaError_t launch_coupled_one(const PathArgs& a, int num_sms, cudaStream_t st,
                                      int* blocks) {
  static std::atomic<int> per_sm[kMaxBlockThreads / 32 + 1];
  static std::atomic<int> attr{0};
  return launch_persistent(paths_coupled<P, T, CV, D>, a, num_sms, st, blocks,
                           PairRing<T>::kBytes, &attr, per_sm);
}

template <class P, class T, int D>
static cudaError_t launch_coupled_cv(int cv, const PathArgs& a, int sms, cudaStream_t st,
                                     int* blocks) {
  switch (cv) {
    case kCvNone: return launch_coupled_one<P, T, kCvNone, D>(a, sms, st, blocks);
    case kCvGrid: return launch_coupled_one<P, T, kCvGrid, D>(a, sms, st, blocks);
    default: return launch_coupled_one<P, T, kCvExact, D>(a, sms, st, blocks);
  }
}

cudaError_t launch_coupled(int kind, int cv, const PathArgs& a, int num_sms, cudaStream_t st,
                           int* blocks) {
  switch (kind) {
    case 0: return launch_coupled_cv<Cfg0, float, 2>(cv, a, num_sms, st, blocks);
    case 1: return launch_coupled_cv<Aniso, float, 2>(cv, a, num_sms, st, blocks);
    case 2: return launch_coupled_cv<Cube3, float, 3>(cv, a, num_sms, st, blocks);
    case 3: return launch_coupled_cv<Harmonic, float, 2>(cv, a, num_sms, st, blocks);
    case 4: return launch_coupled_cv<PaperEx, float, 2>(cv, a, num_sms, st, blocks);
    default: return cudaErrorInvalidValue;
  }
}

// ---------------------------------------------------------------------------
// Finalisation: one thread per node turns the exact sums into FP64 moments.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void finalize_one(const unsigned long long* __restrict__ w,
                                             uint32_t i, double kappa, const StatPtrs& out) {
  const double inv1 = 1.0 / kFxScale, inv2 = inv1 * inv1;
  const double n = (double)w[14];
  const double s_phi = s128_to_double(w[0], w[1]) * inv1;
  const double s_phi2 = s128_to_double(w[2], w[3]) * inv2;
  const double s_psi = s128_to_double(w[4], w[5]) * inv1;
  const double s_psi2 = s128_to_double(w[6], w[7]) * inv2;
  const double s_pp = s128_to_double(w[8], w[9]) * inv2;
  const double s_k = u128_to_double(w[10], w[11]);
  const double m_phi = s_phi / n, m_psi = s_psi / n;
  // the exact sums' conversion to FP64 can leave a zero variance a rounding
  // below zero; clamp it (n = 1 stays NaN: 0 / 0)
  double v_phi = (s_phi2 - s_phi * m_phi) / (n - 1.0);
  double v_psi = (s_psi2 - s_psi * m_psi) / (n - 1.0);
  v_phi = v_phi < 0.0 ? 0.0 : v_phi;
  v_psi = v_psi < 0.0 ? 0.0 : v_psi;
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

__global__ void finalize_nodes(const unsigned long long* __restrict__ acc, uint32_t n_nodes,
                               double kappa, const __grid_constant__ StatPtrs out) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_nodes) return;
  finalize_one(acc + (size_t)i * kAccWords, i, kappa, out);
}

// All levels of a launch in one kernel: thread t finalises record t of the
// contiguous record array, whose level is the last one with base <= t.
struct FinalizeLevels {
  uint32_t n_levels;
  uint32_t total;
  uint32_t base[kMaxSegments + 1];  // first record of each level; base[n_levels] = total
  double kappa[kMaxSegments];
  StatPtrs out[kMaxSegments];
};
static_assert(sizeof(FinalizeLevels) < 32000, "kernel parameter size");

__global__ void finalize_levels(const unsigned long long* __restrict__ acc,
                                const __grid_constant__ FinalizeLevels f) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= f.total) return;
  int lo = 0, hi = (int)f.n_levels - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (f.base[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  finalize_one(acc + (size_t)t * kAccWords, t - f.base[lo], f.kappa[lo], f.out[lo]);
}

// ---------------------------------------------------------------------------
// Launch dispatch.
// ---------------------------------------------------------------------------
// Shared-memory record slots of a launch (the segments' nodes in segment
// order) when they fit kCacheMaxNodes; returns the dynamic shared memory the
// cache needs (0: no cache).
static size_t plan_cache(PathArgs& b) {
  unsigned long long tot = 0;
  for (int i = 0; i < b.n_segs; ++i) tot += b.seg[i].n_nodes;
  b.cache_nodes = 0;
  if (tot == 0 || tot > kCacheMaxNodes) return 0;
  uint32_t base = 0;
  for (int i = 0; i < b.n_segs; ++i) {
    b.seg[i].cache_base = base;
    base += (uint32_t)b.seg[i].n_nodes;
  }
  b.cache_nodes = base;
  return cache_bytes(base);
}
constexpr int kCacheBlockThreads = 512;  // default block size of cached launches

// Persistent launch of `kern` over the flat index space of `a`: occupancy x
// SM count blocks (at most one warp per 32 paths), with the record cache
// when the launch's nodes fit it and `ring_per_warp` bytes of exit ring per
// warp.  `attr_set` / `occ_cache` are the kernel's own (static) state: the
// dynamic shared memory limit set so far and the occupancy per block size
// without the cache.
static bool long_iterations(const PathArgs& a) {
  double all = 0.0, shorter = 0.0;
  for (int i = 0; i < a.n_segs; ++i) {
    const double w = (double)a.seg[i].total / a.seg[i].h;
    all += w;
    if (!(a.seg[i].h <= kLongPathH)) shorter += w;
  }
  return shorter <= kShortWorkShare * all;
}

// Paths per lane a warp claims from the launch's cursor at once.  Automatic:
// 4 when the launch's paths are short (the segments with time steps of at
// most kLongPathH hold at most kShortWorkShare of its expected path-steps)
// and it has at least kAutoClaim x 32 paths for every warp that can be
// resident (64 per SM), else 1.  A claim of c paths per lane means one
// cursor atomic per 32 c paths: with ~10-step paths the cursor is hit at a
// rate where that matters (measured +4.5 % path-steps/s with c = 4 on
// 10-step paths; no change on 100-step paths), while with long paths the
// paths a warp still holds unstarted lengthen the end of the launch.
constexpr int kAutoClaim = 4;
static int resolve_claim(const PathArgs& a, int num_sms) {
  if (a.claim > 0) return a.claim;
  double all = 0.0, longer = 0.0;
  for (int i = 0; i < a.n_segs; ++i) {
    const double w = (double)a.seg[i].total / a.seg[i].h;
    all += w;
    if (a.seg[i].h <= kLongPathH) longer += w;
  }
  const unsigned long long enough =
      (unsigned long long)kAutoClaim * kWarpBatch * 64ull * (unsigned long long)num_sms;
  return (longer <= kShortWorkShare * all && a.total >= enough) ? kAutoClaim : 1;
}

template <class K>
static cudaError_t launch_persistent(K kern, const PathArgs& a, int num_sms, cudaStream_t st,
                                     int* blocks, size_t ring_per_warp,
                                     std::atomic<int>* attr_set, std::atomic<int>* occ_cache) {
  PathArgs b = a;
  b.warp_batch = kWarpBatch * (unsigned long long)resolve_claim(a, num_sms);
  const size_t cache = plan_cache(b);
  const int threads =
      a.block_threads > 0 ? a.block_threads : (cache > 0 ? kCacheBlockThreads : kBlockThreads);
  if (threads % 32 != 0 || threads > kMaxBlockThreads) return cudaErrorInvalidValue;
  const size_t smem = cache + (size_t)(threads / 32) * ring_per_warp;
  if (smem > 48u * 1024u && (int)smem > attr_set->load(std::memory_order_relaxed)) {
    const int lim = (int)(cache_bytes(kCacheMaxNodes) + (kMaxBlockThreads / 32) * ring_per_warp);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
    if (e != cudaSuccess) return e;
    attr_set->store(lim, std::memory_order_relaxed);
  }
  int occ = 0;
  const int known = occ_cache[threads / 32].load(std::memory_order_relaxed);
  if (cache == 0 && known != 0) {
    occ = known;
  } else {
    int v = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, threads, smem);
    if (e != cudaSuccess) return e;
    occ = v > 0 ? v : 1;
    if (cache == 0) occ_cache[threads / 32].store(occ, std::memory_order_relaxed);
  }
  const unsigned long long warps_needed = (a.total + b.warp_batch - 1ull) / b.warp_batch;
  const unsigned long long blocks_needed =
      (warps_needed + (threads / 32) - 1) / (threads / 32);
  unsigned long long nb = (unsigned long long)occ * (unsigned long long)num_sms;
  if (a.max_blocks > 0 && nb > (unsigned long long)a.max_blocks) nb = a.max_blocks;
  if (nb > blocks_needed) nb = blocks_needed;
  if (nb < 1) nb = 1;
  *blocks = (int)nb;
  kern<<<(unsigned)nb, (unsigned)threads, smem, st>>>(b);
  return cudaGetLastError();
}


template <class P, class T, int CV, bool MULTI>
static cudaError_t launch_one(const PathArgs& a, int num_sms, cudaStream_t st, int* blocks) {
  // FP64 paths: the step dominates, they always take the short iteration
  const bool longer = sizeof(T) == 4 && (a.iter_mode == PDD_ITER_LONG ||
                                         (a.iter_mode == PDD_ITER_AUTO && long_iterations(a)));
  if constexpr (P::kDim == 3) {
    if (longer) {
      static std::atomic<int> per_sm[kMaxBlockThreads / 32 + 1];
      static std::atomic<int> attr{0};
      return launch_persistent(paths_3d<P, T, CV, MULTI, sizeof(T) == 4 ? 8 : 4>, a, num_sms,
                               st, blocks, ExitRing<T, 3>::kBytes, &attr, per_sm);
    }
    static std::atomic<int> per_sm[kMaxBlockThreads / 32 + 1];
    static std::atomic<int> attr{0};
    return launch_persistent(paths_3d<P, T, CV, MULTI, 4>, a, num_sms, st, blocks,
                             ExitRing<T, 3>::kBytes, &attr, per_sm);
  } else if (longer) {
    static std::atomic<int> per_sm[kMaxBlockThreads / 32 + 1];
    static std::atomic<int> attr{0};
    return launch_persistent(paths_2d<P, T, CV, MULTI, LongSteps2D<T, CV>::value>, a, num_sms, st,
                             blocks, ExitRing<T, 2>::kBytes, &attr, per_sm);
  } else {
    static std::atomic<int> per_sm[kMaxBlockThreads / 32 + 1];
    static std::atomic<int> attr{0};
    return launch_persistent(paths_2d<P, T, CV, MULTI, 2>, a, num_sms, st, blocks,
                             ExitRing<T, 2>::kBytes, &attr, per_sm);
  }
}

template <class P, class T, int CV, bool MULTI>
static cudaError_t occupancy_one(int threads, int* occ) {
  void (*kern)(PathArgs);
  if constexpr (P::kDim == 3)
    kern = paths_3d<P, T, CV, MULTI, sizeof(T) == 4 ? 8 : 4>;
  else
    kern = paths_2d<P, T, CV, MULTI, LongSteps2D<T, CV>::value>;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      occ, kern, threads, (size_t)(threads / 32) * ExitRing<T, P::kDim>::kBytes);
}

template <class P, class T, bool MULTI>
static cudaError_t occupancy_cv(int cv, int threads, int* occ) {
  switch (cv) {
    case kCvNone: return occupancy_one<P, T, kCvNone, MULTI>(threads, occ);
    case kCvGrid: return occupancy_one<P, T, kCvGrid, MULTI>(threads, occ);
    default: return occupancy_one<P, T, kCvExact, MULTI>(threads, occ);
  }
}

template <class T, bool MULTI>
static cudaError_t occupancy_kind(int kind, int cv, int threads, int* occ) {
  switch (kind) {
    case 0: return occupancy_cv<Cfg0, T, MULTI>(cv, threads, occ);
    case 1: return occupancy_cv<Aniso, T, MULTI>(cv, threads, occ);
    case 2: return occupancy_cv<Cube3, T, true>(cv, threads, occ);  // see launch_kind
    case 4: return occupancy_cv<PaperEx, T, MULTI>(cv, threads, occ);
    default: return occupancy_cv<Harmonic, T, MULTI>(cv, threads, occ);
  }
}

cudaError_t occupancy_paths(int kind, int precision, int cv, bool multi, int threads, int* occ) {
  if (threads % 32 != 0 || threads < 32 || threads > kMaxBlockThreads) return cudaErrorInvalidValue;
  if (precision == 1)
    return multi ? occupancy_kind<double, true>(kind, cv, threads, occ)
                 : occupancy_kind<double, false>(kind, cv, threads, occ);
  return multi ? occupancy_kind<float, true>(kind, cv, threads, occ)
               : occupancy_kind<float, false>(kind, cv, threads, occ);
}

template <class P, class T, bool MULTI>
static cudaError_t launch_cv(int cv, const PathArgs& a, int sms, cudaStream_t st, int* blocks) {
  switch (cv) {
    case kCvNone: return launch_one<P, T, kCvNone, MULTI>(a, sms, st, blocks);
    case kCvGrid: return launch_one<P, T, kCvGrid, MULTI>(a, sms, st, blocks);
    default: return launch_one<P, T, kCvExact, MULTI>(a, sms, st, blocks);
  }
}

template <class T, bool MULTI>
static cudaError_t launch_kind(int kind, int cv, const PathArgs& a, int sms, cudaStream_t st,
                               int* blocks) {
  switch (kind) {
    case 0: return launch_cv<Cfg0, T, MULTI>(cv, a, sms, st, blocks);
    case 1: return launch_cv<Aniso, T, MULTI>(cv, a, sms, st, blocks);
    // 3D launches always run the segment-table build of the kernel: on GB300
    // it measured 1.43x faster than the single-segment build on one segment
    // (1.26e11 vs 8.8e10 path-steps/s; ncu showed the single-segment build
    // stalled on the texture/MIO queues), so the latter is not instantiated
    case 2: return launch_cv<Cube3, T, true>(cv, a, sms, st, blocks);
    case 4: return launch_cv<PaperEx, T, MULTI>(cv, a, sms, st, blocks);
    default: return launch_cv<Harmonic, T, MULTI>(cv, a, sms, st, blocks);
  }
}

cudaError_t launch_paths(int kind, int precision, int cv, const PathArgs& a, int num_sms,
                         cudaStream_t st, int* blocks) {
  if (a.n_segs < 1 || a.n_segs > kMaxSegments) return cudaErrorInvalidValue;
  // the single-segment build follows the Euler Y rule only (see euler_step)
  const bool multi = a.n_segs > 1 || a.y_exp != 0;
  if (precision == 1)
    return multi ? launch_kind<double, true>(kind, cv, a, num_sms, st, blocks)
                 : launch_kind<double, false>(kind, cv, a, num_sms, st, blocks);
  return multi ? launch_kind<float, true>(kind, cv, a, num_sms, st, blocks)
               : launch_kind<float, false>(kind, cv, a, num_sms, st, blocks);
}

cudaError_t launch_finalize_levels(const unsigned long long* acc, int n_levels,
                                   const uint32_t* node_base, const uint32_t* n_nodes,
                                   const double* kappa, const StatPtrs* out, cudaStream_t st) {
  if (n_levels < 1 || n_levels > kMaxSegments) return cudaErrorInvalidValue;
  FinalizeLevels f{};
  uint32_t total = 0;
  int k = 0;
  for (int l = 0; l < n_levels; ++l) {
    if (n_nodes[l] == 0) continue;
    if (node_base[l] != total) return cudaErrorInvalidValue;  // records must be contiguous
    f.base[k] = total;
    f.kappa[k] = kappa[l];
    f.out[k] = out[l];
    total += n_nodes[l];
    ++k;
  }
  if (k == 0) return cudaSuccess;
  f.n_levels = (uint32_t)k;
  f.base[k] = total;
  f.total = total;
  const unsigned threads = 128;
  finalize_levels<<<(total + threads - 1) / threads, threads, 0, st>>>(acc, f);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const unsigned long long* acc, uint32_t n_nodes, double kappa,
                            const StatPtrs& out, cudaStream_t st) {
  const unsigned threads = 128;
  const unsigned blocks = (n_nodes + threads - 1) / threads;
  finalize_nodes<<<blocks, threads, 0, st>>>(acc, n_nodes, kappa, out);
  return cudaGetLastError();
}

}  // namespace pdd
