// sort.cuh -- in-place bitonic sort of a power-of-two number of records.
//
// The network is the textbook one: for stage k = 2, 4, ..., N and step
// j = k/2, ..., 1, record i (bit j clear) is compared with i + j and the pair is
// put in ascending order when bit k of i is clear, descending otherwise.  Steps
// with j below the tile (2,048 records) touch only records of one tile, so they
// run in shared memory, all of a stage's small steps in one launch; only the
// steps with j >= the tile go through global memory, one launch each.  A sort of
// 2^17 records takes 21 launches instead of 153.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace rkr {

constexpr int kSortTile = 2048;

// (64-bit key, int32 value) records, ordered by key then value.
struct Sort64 {
  uint64_t *key;
  int32_t *val;
  struct R {
    uint64_t k;
    int32_t v;
  };
  __device__ __forceinline__ R load(int64_t i) const { return R{key[i], val[i]}; }
  __device__ __forceinline__ void store(int64_t i, const R &r) const {
    key[i] = r.k;
    val[i] = r.v;
  }
  __device__ __forceinline__ static bool gt(const R &a, const R &b) {
    return a.k > b.k || (a.k == b.k && a.v > b.v);
  }
};

// (128-bit key as hi, lo, int32 value) records, ordered lexicographically.
struct Sort128 {
  uint64_t *hi, *lo;
  int32_t *val;
  struct R {
    uint64_t h, l;
    int32_t v;
  };
  __device__ __forceinline__ R load(int64_t i) const { return R{hi[i], lo[i], val[i]}; }
  __device__ __forceinline__ void store(int64_t i, const R &r) const {
    hi[i] = r.h;
    lo[i] = r.l;
    val[i] = r.v;
  }
  __device__ __forceinline__ static bool gt(const R &a, const R &b) {
    return a.h > b.h || (a.h == b.h && (a.l > b.l || (a.l == b.l && a.v > b.v)));
  }
};

// One global step (j >= the tile): thread i handles the pair (i, i ^ j) if i < i ^ j.
template <class S>
__global__ void k_sort_global(S s, int64_t N, int64_t j, int64_t k) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int64_t ixj = i ^ j;
  if (ixj <= i) return;
  const bool asc = (i & k) == 0;
  const typename S::R a = s.load(i), b = s.load(ixj);
  if (S::gt(a, b) == asc) {
    s.store(i, b);
    s.store(ixj, a);
  }
}

// One tile of n = min(N, kSortTile) records per block.  stage == 0: every stage
// k = 2..n with all its steps; stage > n: the steps j = n/2..1 of that stage.
template <class S>
__global__ void __launch_bounds__(1024) k_sort_tile(S s, int64_t N, int64_t stage) {
  __shared__ typename S::R buf[kSortTile];
  const int n = (int)(N < kSortTile ? N : kSortTile);
  const int64_t base = (int64_t)blockIdx.x * n;
  for (int t = threadIdx.x; t < n; t += blockDim.x) buf[t] = s.load(base + t);
  __syncthreads();
  auto step = [&](int64_t k, int j) {
    for (int p = threadIdx.x; p < n / 2; p += blockDim.x) {
      const int i = 2 * j * (p / j) + (p % j);   // bit j of i is clear
      const bool asc = ((base + i) & k) == 0;
      const typename S::R a = buf[i], b = buf[i + j];
      if (S::gt(a, b) == asc) {
        buf[i] = b;
        buf[i + j] = a;
      }
    }
    __syncthreads();
  };
  if (stage == 0) {
    for (int64_t k = 2; k <= n; k <<= 1)
      for (int j = (int)(k >> 1); j > 0; j >>= 1) step(k, j);
  } else {
    for (int j = n >> 1; j > 0; j >>= 1) step(stage, j);
  }
  for (int t = threadIdx.x; t < n; t += blockDim.x) s.store(base + t, buf[t]);
}

// Sorts N records (N a power of two, N >= 1) on stream st.
template <class S>
rkr_status bitonic_sort(const S &s, int64_t N, const char *name, cudaStream_t st) {
  if (N < 2) return RKR_OK;
  const int64_t n = N < kSortTile ? N : kSortTile;
  const unsigned tiles = (unsigned)(N / n);
  const int threads = (int)(n / 2 < 1024 ? n / 2 : 1024);
  const unsigned gblocks = (unsigned)((N + 255) / 256);
  const int slot = prof_begin(name, st);
  k_sort_tile<S><<<tiles, threads, 0, st>>>(s, N, 0);
  note_launch();
  for (int64_t k = 2 * n; k <= N; k <<= 1) {
    for (int64_t j = k >> 1; j >= n; j >>= 1) {
      k_sort_global<S><<<gblocks, 256, 0, st>>>(s, N, j, k);
      note_launch();
    }
    k_sort_tile<S><<<tiles, threads, 0, st>>>(s, N, k);
    note_launch();
  }
  prof_end(slot, st, 0.0);
  RKR_CUDA(cudaGetLastError());
  return RKR_OK;
}

}  // namespace rkr
