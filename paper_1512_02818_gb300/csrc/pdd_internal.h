// pdd_internal.h -- structures shared by the host runtime and the kernels of
// libpdd.so (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/pdd.h"

namespace pdd {

constexpr unsigned kErrOverflow = 1u;       // a score left the fixed-point range
// Bits of the bounds-checked build (compiled with -DPDD_DEBUG_BOUNDS=1): an
// index that would leave its buffer sets its bit and the access is skipped.
// The release build computes no check and never sets them.
constexpr unsigned kErrBoundsGrid = 2u;     // control-grid cell outside the table
constexpr unsigned kErrBoundsIndex = 4u;    // flat path index, segment, node or path out of range
constexpr unsigned kErrBoundsRecord = 8u;   // node record or shared-memory record slot
constexpr unsigned kErrBoundsRing = 16u;    // exit ring over-full
constexpr unsigned kErrBoundsEmit = 32u;    // per-path output index
constexpr unsigned kErrBoundsAll = 62u;
#ifndef PDD_DEBUG_BOUNDS
#define PDD_DEBUG_BOUNDS 0
#endif
constexpr int kAccWords = 16;               // 64-bit words per node record
static_assert(kAccWords == PDD_RECORD_WORDS, "node record size");
constexpr unsigned long long kWarpBatch = 32;  // path indices of a warp claim per path per lane

constexpr int kMaxSegments = 128;          // segments (levels / requests) per launch
// Launches whose segments hold at most this many node records in total keep a
// per-block copy of the records in shared memory (68 KB with padding).
constexpr uint32_t kCacheMaxNodes = 512;

// One segment of a launch: n_nodes x n_paths paths with their own nodes,
// time step, control grid, random-stream key and output records.
// The segment covers paths path_off .. path_off + n_paths - 1 of each of its
// n_nodes nodes (a slice of a request when a request is spread over launches).
struct SegArgs {
  const float* cx;
  const float* cy;
  const float* cz;
  unsigned long long begin;    // first index of the segment in the launch's flat path space
  unsigned long long total;    // n_nodes * n_paths
  unsigned long long n_paths;  // paths per node in this segment
  unsigned long long n_nodes;  // nodes of this segment
  unsigned long long* acc;     // node records of the segment's nodes (16 words each)
  const void* grad;            // float2 (2D) / float4 (3D) gradient table; null: no grid
  float* emit_phi;             // optional per-path outputs: [node * emit_stride + path]
  float* emit_xi;
  int* emit_steps;
  unsigned long long emit_stride;
  double h;
  double sqrt_h;
  double thr0;                 // c0 sqrt(h)
  uint32_t path_off;           // first path index of the segment
  uint32_t cache_base;         // first shared-memory record slot of the segment's nodes
  uint32_t key0, key1, seed_hi;
  int grid_n;
  int max_steps;
};

// Arguments of one path-kernel launch (passed by value as a grid constant).
struct PathArgs {
  unsigned long long total;    // sum of the segments' totals
  unsigned long long* cursor;  // flat path cursor, zeroed before the launch
  unsigned* err;               // error bits (kErr*)
  unsigned long long* trunc_total;
  unsigned long long* steps_total;  // optional: sum of the exit indices of all paths run
  int y_exp;
  int max_blocks;              // 0 = occupancy x SM count
  int block_threads;           // 0 = default (256)
  int iter_mode;               // Euler steps per iteration: PDD_ITER_AUTO / _SHORT / _LONG
  int claim;                   // paths per lane a warp claims from the cursor at once (0: auto)
  unsigned long long warp_batch;  // kWarpBatch x the resolved claim; set by the launcher
  int n_segs;                  // 1 .. kMaxSegments; segments in increasing `begin`
  uint32_t cache_nodes;        // record slots cached in shared memory per block (0: none);
                               // set by the launchers
  SegArgs seg[kMaxSegments];
};

// Per-node output pointers (device; any may be null).
struct StatPtrs {
  double* mean_phi;
  double* var_phi;
  double* mean_cv;
  double* var_cv;
  double* cov_phi_xi;
  double* var_xi;
  double* rho;
  double* se_phi;
  double* se_cv;
  double* vr;
  double* pred_speedup;
  double* mean_steps;
  unsigned long long* n_paths;
  unsigned long long* n_truncated;
};

// Makes `dev` current for the lifetime of the guard.  cudaSetDevice is called
// even when `dev` is already the current device: it (re)binds the device's
// primary context to the calling thread, which other libraries in the process
// may have changed.  A stale error left by an unchecked earlier call is
// cleared so that it cannot be reported against this call.
struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = cudaSetDevice(dev) == cudaSuccess;
    (void)cudaGetLastError();
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

// What the allocation-free entry point needs to know about a problem.
struct ProblemView {
  int device;
  cudaStream_t stream;
  int num_sms;
  int kind, precision, exit_rule, y_rule, dim;
  int64_t max_steps;
  const void* grid_table[8];
  int grid_n[8];
  std::mutex* mu;
  int64_t* launches;
};

static_assert(PDD_MAX_GRIDS == 8, "ProblemView holds 8 grid slots");
// Status of a launch's error word: PDD_ERR_BOUNDS (bounds-checked build) or
// PDD_ERR_OVERFLOW with a message naming `who`, PDD_OK when no bit is set.
int error_word_status(unsigned err, const char* who);
bool problem_view(pdd_problem* p, ProblemView* v);
bool ctx_view(pdd_ctx* c, int* device, int* num_sms, int* block_threads, int* max_blocks);
int ctx_iter_mode(pdd_ctx* c);  // the context's PDD_ITER_* choice
int ctx_claim(pdd_ctx* c);      // the context's paths-per-lane claim (0: automatic)
pdd_ctx* problem_ctx(pdd_problem* p);

cudaError_t launch_paths(int kind, int precision, int cv, const PathArgs& a, int num_sms,
                         cudaStream_t st, int* blocks);
// Resident blocks per SM of the path kernel of (kind, precision, cv, multi) at
// `threads` threads per block.
cudaError_t occupancy_paths(int kind, int precision, int cv, bool multi, int threads, int* occ);
// Coupled fine (seg[0]) / coarse (seg[1]) pairs, FP32 paths (2D and 3D problems).
cudaError_t launch_coupled(int kind, int cv, const PathArgs& a, int num_sms, cudaStream_t st,
                           int* blocks);
cudaError_t launch_finalize(const unsigned long long* acc, uint32_t n_nodes, double kappa,
                            const StatPtrs& out, cudaStream_t st);
// One launch for the records of up to kMaxSegments levels stored back to
// back from `acc` (level l at record node_base[l]; empty levels skipped).
cudaError_t launch_finalize_levels(const unsigned long long* acc, int n_levels,
                                   const uint32_t* node_base, const uint32_t* n_nodes,
                                   const double* kappa, const StatPtrs* out, cudaStream_t st);
// Gradient table of grid values v (FP64, n^D, x fastest) into float2/float4.
cudaError_t launch_grid_gradient(const double* v, int n, int dim, void* table, cudaStream_t st);
// Pack D interleaved gradient components (FP64) into float2/float4.
cudaError_t launch_grid_pack(const double* g, int n, int dim, void* table, cudaStream_t st);
// Per-cell multilinear coefficients from a nodal table (2D: 32-byte FP32
// records; 3D: 64-byte records with binary16 differences, *overflow set when
// one leaves the binary16 range).
cudaError_t launch_grid_cells(const void* nodal, int n, int dim, void* cells, unsigned* overflow,
                              cudaStream_t st);
// FP32 -> FP64 copy on the device.
cudaError_t launch_f32_to_f64(const float* src, double* dst, size_t count, cudaStream_t st);

}  // namespace pdd
