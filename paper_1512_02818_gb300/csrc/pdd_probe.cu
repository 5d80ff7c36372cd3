// pdd_probe.cu -- issue-rate microbenchmark of the instruction classes the
// path step is made of, to check the instruction-issue roofline the path
// kernels are measured against (one warp instruction per scheduler per
// cycle) on the GPU at hand instead of taking pipe rates from a data sheet.
//
// Every thread runs `iters` rounds of 8 independent dependency chains of one
// instruction class (kind 0: FP32 fused multiply-add; 1: 32-bit integer
// multiply-add; 2: SFU base-2 exponential; 3: 3-input logic op); the loop is
// unrolled so that loop control is a few percent of the instructions.  The
// only memory traffic is one store per thread at the end, which keeps the
// chains alive.
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pdd.h"
#include "../../include/pdd_debug.h"

namespace pdd {
void set_error(const char* fmt, ...);
}

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 4;

__device__ __forceinline__ float ex2_neg(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(-x));  // 2^-x in (1/4, 1] for x in [0, 2)
  return y;
}

__device__ __forceinline__ uint32_t mad_lo(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));  // opaque: not folded
  return d;
}

__device__ __forceinline__ uint32_t lop3_xor3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, 0x96;" : "=r"(d) : "r"(a), "r"(b), "r"(c));  // a ^ b ^ c
  return d;
}

template <int KIND>
__global__ void __launch_bounds__(512) issue_probe(int iters, float* __restrict__ sink) {
  const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
  float f[kChains];
  uint32_t u[kChains];
#pragma unroll
  for (int j = 0; j < kChains; ++j) {
    f[j] = 1e-3f * (float)((t + j) & 255);
    u[j] = t * 2654435761u + (uint32_t)j;
  }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < kUnroll; ++r) {
#pragma unroll
      for (int j = 0; j < kChains; ++j) {
        if (KIND == 0) f[j] = fmaf(f[j], 0.999999f, 1e-7f);
        if (KIND == 1) u[j] = mad_lo(u[j], 1664525u + 2u * (uint32_t)r, 1013904223u);
        if (KIND == 2) f[j] = ex2_neg(f[j]);
        if (KIND == 3) u[j] = lop3_xor3(u[j], 0x9E3779B9u + (uint32_t)r, 0x7F4A7C15u * (uint32_t)(j + 1));
      }
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int j = 0; j < kChains; ++j) s += f[j] + (float)(u[j] & 1023u);
  sink[t] = s;
}

template <int KIND>
cudaError_t run_probe(int blocks, int threads, int iters, float* sink) {
  issue_probe<KIND><<<blocks, threads>>>(iters, sink);
  return cudaGetLastError();
}

}  // namespace

extern "C" int pdd_debug_issue_rate(int kind, int iters, double* ops_per_s, double* ms) {
  if (kind < 0 || kind > 3 || iters < 1 || iters > (1 << 24) || !ops_per_s || !ms) {
    pdd::set_error("pdd_debug_issue_rate: kind in [0, 3], iters in [1, 2^24], non-NULL outputs");
    return PDD_ERR_INVALID;
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    pdd::set_error("pdd_debug_issue_rate: no device");
    return PDD_ERR_CUDA;
  }
  const int threads = 512, blocks = 4 * sms;  // 2048 resident threads per SM
  float* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&sink, sizeof(float) * (size_t)threads * blocks);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  auto launch = [&](int it) -> cudaError_t {
    switch (kind) {
      case 0: return run_probe<0>(blocks, threads, it, sink);
      case 1: return run_probe<1>(blocks, threads, it, sink);
      case 2: return run_probe<2>(blocks, threads, it, sink);
      default: return run_probe<3>(blocks, threads, it, sink);
    }
  };
  if (e == cudaSuccess) e = launch(iters < 16 ? iters : 16);  // warm-up
  if (e == cudaSuccess) e = cudaEventRecord(e0);
  if (e == cudaSuccess) e = launch(iters);
  if (e == cudaSuccess) e = cudaEventRecord(e1);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float t = 0.0f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess) {
    pdd::set_error("pdd_debug_issue_rate: %s", cudaGetErrorString(e));
    return PDD_ERR_CUDA;
  }
  *ms = t;
  *ops_per_s = (double)threads * blocks * (double)iters * kUnroll * kChains / (t * 1e-3);
  return PDD_OK;
}
