// simt.cuh -- FP32 CUDA-core tiles in the thread-per-user layout.
//
// A CTA of 128 threads owns 128 users (thread t <-> user u0 + t).  User rows
// are staged transposed in shared memory, Us[k * 128 + t]; a tile of TX items
// is staged transposed, Xs[k * TX + j].  Each thread accumulates the FMA chain
// over k = 0 .. d-1 for its user and all TX items of the tile.
#pragma once

#include "common.cuh"

namespace rkr {

__device__ __forceinline__ void load_users_T(const float *__restrict__ U, int64_t n, int d,
                                             int64_t u0, float *__restrict__ Us) {
  for (int e = threadIdx.x; e < 128 * d; e += blockDim.x) {
    int t = e / d, k = e - t * d;
    int64_t u = u0 + t;
    Us[k * 128 + t] = u < n ? U[u * d + k] : 0.0f;
  }
}

template <int TX>
__device__ __forceinline__ void load_items_T(const float *__restrict__ X, int64_t nx, int d,
                                             int64_t x0, float *__restrict__ Xs) {
  for (int e = threadIdx.x; e < TX * d; e += blockDim.x) {
    int j = e / d, k = e - j * d;
    int64_t x = x0 + j;
    Xs[k * TX + j] = x < nx ? X[x * d + k] : 0.0f;
  }
}

template <int TX>
__device__ __forceinline__ void tile_dots(const float *__restrict__ Us,
                                          const float *__restrict__ Xs, int d, int t,
                                          float (&acc)[TX]) {
#pragma unroll
  for (int j = 0; j < TX; ++j) acc[j] = 0.0f;
  for (int k = 0; k < d; ++k) {
    float uk = Us[k * 128 + t];
    const float4 *xr = reinterpret_cast<const float4 *>(Xs + k * TX);
#pragma unroll
    for (int q = 0; q < TX / 4; ++q) {
      float4 x = xr[q];
      acc[4 * q + 0] = fmaf(uk, x.x, acc[4 * q + 0]);
      acc[4 * q + 1] = fmaf(uk, x.y, acc[4 * q + 1]);
      acc[4 * q + 2] = fmaf(uk, x.z, acc[4 * q + 2]);
      acc[4 * q + 3] = fmaf(uk, x.w, acc[4 * q + 3]);
    }
  }
}

}  // namespace rkr
