// pdd_debug.cu -- test hooks: the device Philox4x32-10 and normal stream on
// their own, and cuRAND's Philox4_32_10 as an independent reference.
#include <cuda_runtime.h>
#include <curand_kernel.h>
#include <stdint.h>

#include "../../include/pdd.h"
#include "../../include/pdd_debug.h"
#include "pdd_device.cuh"

namespace pdd {
void set_error(const char* fmt, ...);
}

namespace {

__global__ void philox_kernel(const uint32_t* ctr, const uint32_t* key, uint32_t* out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
  const uint4 r = pdd::philox4x32_10(c, make_uint2(key[2 * i], key[2 * i + 1]));
  out[4 * i] = r.x;
  out[4 * i + 1] = r.y;
  out[4 * i + 2] = r.z;
  out[4 * i + 3] = r.w;
}

__global__ void curand_philox_kernel(const uint32_t* ctr, const uint32_t* key, uint32_t* out,
                                     int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned long long seed = (unsigned long long)key[2 * i] |
                                  ((unsigned long long)key[2 * i + 1] << 32);
  const unsigned long long subseq = (unsigned long long)ctr[4 * i + 2] |
                                    ((unsigned long long)ctr[4 * i + 3] << 32);
  const unsigned long long blk = (unsigned long long)ctr[4 * i] |
                                 ((unsigned long long)ctr[4 * i + 1] << 32);
  curandStatePhilox4_32_10_t st;
  curand_init(seed, subseq, 4ull * blk, &st);
  const uint4 r = curand4(&st);
  out[4 * i] = r.x;
  out[4 * i + 1] = r.y;
  out[4 * i + 2] = r.z;
  out[4 * i + 3] = r.w;
}

template <class T>
__global__ void normals_kernel(uint64_t seed, uint32_t tag, uint32_t node, uint32_t path,
                               uint64_t first, int64_t count, T* out) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= count) return;
  const uint64_t i = first + (uint64_t)j;
  const uint4 w = pdd::philox4x32_10(
      make_uint4((uint32_t)(i / 4), path, node, (uint32_t)(seed >> 32)),
      make_uint2((uint32_t)seed, tag));
  T a, b;
  if ((i % 4) < 2)
    pdd::box_muller(w.x, w.y, a, b);
  else
    pdd::box_muller(w.z, w.w, a, b);
  out[j] = (i % 2 == 0) ? a : b;
}

int finish(cudaError_t e) {
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    pdd::set_error("CUDA error: %s", cudaGetErrorString(e));
    return PDD_ERR_CUDA;
  }
  return PDD_OK;
}

}  // namespace

extern "C" int pdd_debug_philox(const uint32_t* ctr, const uint32_t* key, uint32_t* out,
                                int64_t n) {
  if (n < 0 || (n > 0 && (!ctr || !key || !out))) {
    pdd::set_error("pdd_debug_philox: bad arguments");
    return PDD_ERR_INVALID;
  }
  if (n == 0) return PDD_OK;
  philox_kernel<<<(unsigned)((n + 255) / 256), 256>>>(ctr, key, out, n);
  return finish(cudaGetLastError());
}

extern "C" int pdd_debug_philox_curand(const uint32_t* ctr, const uint32_t* key, uint32_t* out,
                                       int64_t n) {
  if (n < 0 || (n > 0 && (!ctr || !key || !out))) {
    pdd::set_error("pdd_debug_philox_curand: bad arguments");
    return PDD_ERR_INVALID;
  }
  if (n == 0) return PDD_OK;
  curand_philox_kernel<<<(unsigned)((n + 255) / 256), 256>>>(ctr, key, out, n);
  return finish(cudaGetLastError());
}

extern "C" int pdd_debug_normals(uint64_t seed, uint32_t tag, uint32_t node, uint32_t path,
                                 uint64_t first, int64_t count, int precision, float* out_f32,
                                 double* out_f64) {
  if (count < 0 || (precision == 0 && count > 0 && !out_f32) ||
      (precision == 1 && count > 0 && !out_f64) || (precision != 0 && precision != 1)) {
    pdd::set_error("pdd_debug_normals: bad arguments");
    return PDD_ERR_INVALID;
  }
  if (count == 0) return PDD_OK;
  const unsigned blocks = (unsigned)((count + 255) / 256);
  if (precision == 0)
    normals_kernel<float><<<blocks, 256>>>(seed, tag, node, path, first, count, out_f32);
  else
    normals_kernel<double><<<blocks, 256>>>(seed, tag, node, path, first, count, out_f64);
  return finish(cudaGetLastError());
}

// ---------------------------------------------------------------------------
// Self-test of the bounds checks: every check fails once, nothing is accessed.
// ---------------------------------------------------------------------------
namespace {
struct ErrOnly {
  unsigned* err;
};
__global__ void bounds_selftest_kernel(unsigned* err) {
  const ErrOnly a{err};
  (void)a;
  (void)pdd::cell_in_table(err, -1, 0, 0, 9);
  (void)PDD_IN_BOUNDS(a, false, pdd::kErrBoundsIndex);
  (void)PDD_IN_BOUNDS(a, false, pdd::kErrBoundsRecord);
  (void)PDD_IN_BOUNDS(a, false, pdd::kErrBoundsRing);
  (void)PDD_IN_BOUNDS(a, false, pdd::kErrBoundsEmit);
}
}  // namespace

extern "C" int pdd_debug_bounds_selftest(uint32_t* bits) {
  if (!bits) {
    pdd::set_error("pdd_debug_bounds_selftest: bits is NULL");
    return PDD_ERR_INVALID;
  }
  unsigned* d = nullptr;
  cudaError_t e = cudaMalloc(&d, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(d, 0, sizeof(unsigned));
  if (e == cudaSuccess) {
    bounds_selftest_kernel<<<1, 1>>>(d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpy(bits, d, sizeof(unsigned), cudaMemcpyDeviceToHost);
  if (d) cudaFree(d);
  if (e != cudaSuccess) {
    pdd::set_error("pdd_debug_bounds_selftest: %s", cudaGetErrorString(e));
    return PDD_ERR_CUDA;
  }
  return PDD_OK;
}
