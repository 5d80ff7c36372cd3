/*
 * pdd_debug.h -- test hooks of libpdd.so.  They expose the device random
 * number stages on their own so that tests can compare them with the oracle
 * and with cuRAND's Philox4_32_10 generator; they are not part of the
 * estimation path.  All pointers are device pointers; calls are synchronous;
 * return a pdd_status (see pdd.h).
 */
#ifndef PDD_DEBUG_H
#define PDD_DEBUG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Philox4x32-10 blocks: ctr[4*i..4*i+3], key[2*i..2*i+1] -> out[4*i..4*i+3]
   (Salmon et al., SC'11), computed by the library's device generator.       */
int pdd_debug_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n);

/* The same blocks from cuRAND's device API (curand_init(seed, subsequence,
   offset) + curand4), as an independent implementation: seed = key0 |
   key1 << 32, subsequence = ctr2 | ctr3 << 32, offset = 4 (ctr0 | ctr1 << 32). */
int pdd_debug_philox_curand(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n);

/* Normals first .. first+count-1 of the stream of (seed, tag, node, path), in
   the path precision (precision 0: FP32 into out_f32; 1: FP64 into out_f64). */
int pdd_debug_normals(uint64_t seed, uint32_t tag, uint32_t node, uint32_t path, uint64_t first,
                      int64_t count, int precision, float* out_f32, double* out_f64);

/* Issue-rate probe (no counterpart in the paper): thread-operations per second
   of one instruction class, run by 4 x SM-count blocks of 512 threads on the
   current device, each thread `iters` x 32 operations in 8 independent
   chains.  kind 0: FP32 fused multiply-add, 1: 32-bit integer multiply-add,
   2: SFU base-2 exponential, 3: 3-input logic operation.  It measures the
   per-class issue limits that the path kernels' roofline assumes (one warp
   instruction per scheduler per cycle).  Allocates and frees a sink of 4 B
   per thread; synchronous.  iters in [1, 2^24].                            */
int pdd_debug_issue_rate(int kind, int iters, double* ops_per_s, double* ms);

/* Self-test of the bounds checks (no counterpart in the paper).  A one-thread
   kernel feeds the checks of the bounds-checked build (libpdd_bounds.so,
   compiled with -DPDD_DEBUG_BOUNDS=1) one failing case of each kind -- a
   grid cell index of -1, and false conditions for the path-index, record,
   exit-ring and per-path-output checks -- without performing any of the
   guarded accesses, and returns the resulting error word in *bits (host
   pointer): 62 (all five bounds bits) in the bounds-checked build, 0 in the
   release build, whose checks compile to nothing.  Synchronous; allocates
   and frees one device word.                                                */
int pdd_debug_bounds_selftest(uint32_t* bits);

#ifdef __cplusplus
}
#endif
#endif /* PDD_DEBUG_H */
