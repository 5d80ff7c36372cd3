// pdd_grid.cu -- control-grid preparation: the gradient lookup table of a
// previous iterate v (the "D-dimensional array holding pointwise values" of
// Sec. 3.1, entering the control variate F = -sigma^T grad v, eq. F:ExactF).
// Centred differences inside, second-order one-sided differences on the
// edges, in FP64; stored in FP32 as float2 (2D) or float4 (3D, w = 0).
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "pdd_internal.h"

namespace pdd {

__device__ __forceinline__ double diff_axis(const double* v, long long pt, long long i, long long n,
                                            long long stride, double inv2d) {
  if (i == 0) return (-3.0 * v[pt] + 4.0 * v[pt + stride] - v[pt + 2 * stride]) * inv2d;
  if (i == n - 1) return (3.0 * v[pt] - 4.0 * v[pt - stride] + v[pt - 2 * stride]) * inv2d;
  return (v[pt + stride] - v[pt - stride]) * inv2d;
}

__global__ void grid_gradient_kernel(const double* __restrict__ v, int n, int dim,
                                     void* __restrict__ table) {
  const long long nn = (long long)n;
  const long long npts = (dim == 2) ? nn * nn : nn * nn * nn;
  const long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= npts) return;
  // 1 / (2 delta) with delta = 1 / (n - 1)
  const double inv2d = 0.5 * (double)(n - 1);
  const long long ix = pt % nn, iy = (pt / nn) % nn, iz = (dim == 3) ? pt / (nn * nn) : 0;
  const double gx = diff_axis(v, pt, ix, nn, 1, inv2d);
  const double gy = diff_axis(v, pt, iy, nn, nn, inv2d);
  if (dim == 2) {
    ((float2*)table)[pt] = make_float2((float)gx, (float)gy);
  } else {
    const double gz = diff_axis(v, pt, iz, nn, nn * nn, inv2d);
    ((float4*)table)[pt] = make_float4((float)gx, (float)gy, (float)gz, 0.0f);
  }
}

__global__ void grid_pack_kernel(const double* __restrict__ g, int n, int dim,
                                 void* __restrict__ table) {
  const long long nn = (long long)n;
  const long long npts = (dim == 2) ? nn * nn : nn * nn * nn;
  const long long pt = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (pt >= npts) return;
  if (dim == 2)
    ((float2*)table)[pt] = make_float2((float)g[2 * pt], (float)g[2 * pt + 1]);
  else
    ((float4*)table)[pt] =
        make_float4((float)g[3 * pt], (float)g[3 * pt + 1], (float)g[3 * pt + 2], 0.0f);
}

__global__ void f32_to_f64_kernel(const float* __restrict__ src, double* __restrict__ dst,
                                  size_t count) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) dst[i] = (double)src[i];
}

// Multilinear polynomial coefficients of every cell, from the FP32 nodal table
// (promoted to FP64).  2D: FP32 coefficients; 3D: c000 in FP32 and the seven
// difference coefficients rounded to binary16 (a 64-byte record; `overflow`
// is set when one of them leaves the binary16 range).  Record layouts: see
// pdd_device.cuh.
__global__ void grid_cells_kernel(const void* __restrict__ nodal, int n, int dim,
                                  float4* __restrict__ cells, unsigned* __restrict__ overflow) {
  const long long m = n - 1;
  const long long ncell = dim == 2 ? m * m : m * m * m;
  const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncell) return;
  const long long nn = n;
  if (dim == 2) {
    const long long ix = c % m, iy = c / m;
    const float2* G = (const float2*)nodal;
    const float2 g00 = G[iy * nn + ix], g10 = G[iy * nn + ix + 1];
    const float2 g01 = G[(iy + 1) * nn + ix], g11 = G[(iy + 1) * nn + ix + 1];
    const double a[2][4] = {{g00.x, g10.x, g01.x, g11.x}, {g00.y, g10.y, g01.y, g11.y}};
    for (int comp = 0; comp < 2; ++comp) {
      const double v00 = a[comp][0], v10 = a[comp][1], v01 = a[comp][2], v11 = a[comp][3];
      cells[2 * c + comp] = make_float4((float)v00, (float)(v10 - v00), (float)(v01 - v00),
                                        (float)(v11 - v10 - v01 + v00));
    }
    return;
  }
  const long long ix = c % m, iy = (c / m) % m, iz = c / (m * m);
  const float4* G = (const float4*)nodal;
  float4 g[2][2][2];  // [dz][dy][dx]
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx)
        g[dz][dy][dx] = G[((iz + dz) * nn + (iy + dy)) * nn + ix + dx];
  uint32_t w[16] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
  unsigned short h[22] = {0};
  bool bad = false;
  for (int comp = 0; comp < 3; ++comp) {
    auto v = [&](int dx, int dy, int dz) -> double {
      const float4 q = g[dz][dy][dx];
      return comp == 0 ? q.x : (comp == 1 ? q.y : q.z);
    };
    const double c000 = v(0, 0, 0);
    const double d[7] = {
        v(1, 0, 0) - c000,                                  // c100
        v(0, 1, 0) - c000,                                  // c010
        v(0, 0, 1) - c000,                                  // c001
        v(1, 1, 0) - v(1, 0, 0) - v(0, 1, 0) + c000,        // c110
        v(1, 0, 1) - v(1, 0, 0) - v(0, 0, 1) + c000,        // c101
        v(0, 1, 1) - v(0, 1, 0) - v(0, 0, 1) + c000,        // c011
        v(1, 1, 1) - v(1, 1, 0) - v(1, 0, 1) - v(0, 1, 1) + v(1, 0, 0) + v(0, 1, 0) +
            v(0, 0, 1) - c000};                             // c111
    w[comp] = __float_as_uint((float)c000);
    for (int j = 0; j < 7; ++j) {
      const __half q = __double2half(d[j]);
      bad |= __hisinf(q) != 0;
      h[7 * comp + j] = __half_as_ushort(q);
    }
  }
  for (int k = 0; k < 11; ++k) w[3 + k] = (uint32_t)h[2 * k] | ((uint32_t)h[2 * k + 1] << 16);
  uint4* out = (uint4*)cells + 4 * c;
  for (int k = 0; k < 4; ++k) out[k] = make_uint4(w[4 * k], w[4 * k + 1], w[4 * k + 2], w[4 * k + 3]);
  if (bad && overflow != nullptr) atomicOr(overflow, 1u);
}

static unsigned blocks_for(long long count, unsigned threads) {
  return (unsigned)((count + threads - 1) / threads);
}

cudaError_t launch_grid_gradient(const double* v, int n, int dim, void* table, cudaStream_t st) {
  const long long npts = (dim == 2) ? (long long)n * n : (long long)n * n * n;
  grid_gradient_kernel<<<blocks_for(npts, 256), 256, 0, st>>>(v, n, dim, table);
  return cudaGetLastError();
}

cudaError_t launch_grid_pack(const double* g, int n, int dim, void* table, cudaStream_t st) {
  const long long npts = (dim == 2) ? (long long)n * n : (long long)n * n * n;
  grid_pack_kernel<<<blocks_for(npts, 256), 256, 0, st>>>(g, n, dim, table);
  return cudaGetLastError();
}

cudaError_t launch_f32_to_f64(const float* src, double* dst, size_t count, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  f32_to_f64_kernel<<<blocks_for((long long)count, 256), 256, 0, st>>>(src, dst, count);
  return cudaGetLastError();
}

}  // namespace pdd

namespace pdd {
cudaError_t launch_grid_cells(const void* nodal, int n, int dim, void* cells, unsigned* overflow,
                              cudaStream_t st) {
  const long long m = n - 1;
  const long long ncell = dim == 2 ? m * m : m * m * m;
  grid_cells_kernel<<<blocks_for(ncell, 256), 256, 0, st>>>(nodal, n, dim, (float4*)cells,
                                                            overflow);
  return cudaGetLastError();
}
}  // namespace pdd
