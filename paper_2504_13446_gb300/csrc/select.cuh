// select.cuh -- block-wide selection and sorting helpers (one CTA per query).
#pragma once

#include "common.cuh"

namespace rkr {

// k-th smallest (1-based k) of the keys fn(i, key) yields for i in [0, cnt)
// (fn returns false for elements that do not take part).  MSB-first radix
// select on 8-bit digits over an nbits-wide key.  Every thread of the block must
// call it with the same arguments; the k-th smallest must exist.
// A thread evaluates four keys before it adds any to the histogram, so that
// their loads are in flight together: one CTA may have to walk a million keys.
template <class F>
__device__ uint64_t block_kth(int64_t cnt, uint64_t k, int nbits, F fn, uint32_t *hist,
                              uint64_t *bc) {
  uint64_t prefix = 0, mask = 0;
  const int64_t T = blockDim.x;
  for (int shift = nbits - 8; shift >= 0; shift -= 8) {
    for (int i = threadIdx.x; i < 256; i += blockDim.x) hist[i] = 0;
    __syncthreads();
    int64_t i = threadIdx.x;
    for (; i + 3 * T < cnt; i += 4 * T) {
      uint64_t key[4];
      bool in[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) in[j] = fn(i + j * T, key[j]);
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (in[j] && (key[j] & mask) == prefix) atomicAdd(&hist[(key[j] >> shift) & 255u], 1u);
    }
    for (; i < cnt; i += T) {
      uint64_t key;
      if (fn(i, key) && (key & mask) == prefix) atomicAdd(&hist[(key >> shift) & 255u], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      uint64_t acc = 0;
      int sel = 255;
      for (int dg = 0; dg < 256; ++dg) {
        if (acc + hist[dg] >= k) { sel = dg; break; }
        acc += hist[dg];
      }
      bc[0] = prefix | ((uint64_t)sel << shift);
      bc[1] = k - acc;
    }
    __syncthreads();
    prefix = bc[0];
    k = bc[1];
    mask |= (uint64_t)255 << shift;
    __syncthreads();
  }
  return prefix;
}

// Number of i in [0, cnt) with pred(i).
template <class F>
__device__ int64_t block_count(int64_t cnt, F pred, unsigned long long *acc) {
  if (threadIdx.x == 0) *acc = 0;
  __syncthreads();
  unsigned long long mine = 0;
  for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) mine += pred(i) ? 1 : 0;
  for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
  if ((threadIdx.x & 31) == 0 && mine) atomicAdd(acc, mine);
  __syncthreads();
  int64_t r = (int64_t)*acc;
  __syncthreads();
  return r;
}

// Entries sorted in shared memory: ascending by (k1, k2).
struct SortEnt {
  uint64_t k1;
  uint32_t k2;
  int32_t idx;
};

__device__ __forceinline__ bool ent_less(const SortEnt &a, const SortEnt &b) {
  return a.k1 < b.k1 || (a.k1 == b.k1 && a.k2 < b.k2);
}

// Bitonic sort of e[0 .. count) in shared memory; e must have room for the next
// power of two, the tail is padded with maximal keys.
__device__ void block_sort(SortEnt *e, int count) {
  int np2 = 1;
  while (np2 < count) np2 <<= 1;
  for (int i = count + threadIdx.x; i < np2; i += blockDim.x) {
    e[i].k1 = ~0ull;
    e[i].k2 = 0xffffffffu;
    e[i].idx = -1;
  }
  __syncthreads();
  for (int k = 2; k <= np2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < np2; i += blockDim.x) {
        int ixj = i ^ j;
        if (ixj > i) {
          bool asc = (i & k) == 0;
          SortEnt a = e[i], b = e[ixj];
          if (ent_less(b, a) == asc) { e[i] = b; e[ixj] = a; }
        }
      }
      __syncthreads();
    }
  }
}

}  // namespace rkr
