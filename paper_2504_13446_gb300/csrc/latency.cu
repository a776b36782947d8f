// latency.cu -- c-approximate queries one at a time (latency mode).
//
// The paper answers each query on its own: u.q for every user and the table
// lookup of Section 4.3 step 1 (its dominant cost, O(nd) per query), then the
// k-th smallest bounds, the Case A/B filter and the interpolation.  Per query
// this runs four launches with no host synchronization between them:
//
//   k_latency_scan     one pass over U (FP32, coalesced): u.q of every user by
//                      warp-level FP32 products with a rigorous error bound; the
//                      bin j of Section 4.3 step 1 from that interval (canonical
//                      FP64 u.q only when the interval straddles a threshold);
//                      r_low, r_up numerators from the table; a histogram of
//                      the upper-bound numerators
//   k_latency_cut      from the histogram, T >= R_up_k (the k-th smallest upper
//                      bound numerator), the bound of the users that can matter
//   k_latency_compact  the users with r_low <= T
//   k_select_approx    steps 1-3 on those users (query.cu)
//
// Every user that step 2 or 3 can return has r_low <= R_up_k (Case A takes the
// k smallest r_up, all <= R_up_k, and r_low <= r_up; Case B prunes r_low >
// R_up_k), and R_low_k <= R_up_k <= T, so the k smallest lower and upper
// bounds lie among the compacted users: the answer equals the batched one bit
// for bit.  The scan is bound by HBM: it reads U once (4d bytes per user) and
// a few bytes of per-user data and table cells.
#include <math.h>
#include <string.h>

#include <new>

#include "index.cuh"

namespace rkr {
namespace lat {

constexpr int kLatThreads = 256;
constexpr int kLatRows = 8;      // rows per warp and sub-batch
constexpr int kLatSub = 4;       // sub-batches: 32 rows per warp iteration, one per lane
constexpr int kLatBins = 2048;

// Bound factor of the warp product: every rounding (d FMAs in the lanes' chains,
// 31 additions of the warp reduction) errs by at most 2^-24 times a partial sum,
// and every partial sum is at most sum_k |u_k q_k| <= ||u|| ||q||; the canonical
// FP64 sum differs from the exact value by at most d 2^-53 ||u|| ||q||.
__host__ __device__ inline float latency_cfac(int d) {
  const double c = ((double)(d + 36) * 0x1p-24 + (double)d * 0x1p-53 + 0x1p-40) * (1.0 + 0x1p-20);
  return (float)c * (1.0f + 0x1p-20f);
}

// This lane's part of the dot products of kLatRows consecutive rows with q: every
// load of the batch is issued before the first product, so a warp keeps
// kLatRows rows in flight (row r0 + rr; rows at or past n contribute 0).
template <int VEC>
__device__ __forceinline__ void lane_dots(const float *__restrict__ U, int64_t r0, int64_t n,
                                          int d, const float *qs, int lane,
                                          float (&part)[kLatRows]) {
  if (VEC == 4) {
    const int dv = d >> 2;
    float4 a[kLatRows][2];
#pragma unroll
    for (int rr = 0; rr < kLatRows; ++rr) {
      const float4 *r4 = reinterpret_cast<const float4 *>(U + (r0 + rr) * d);
      const bool ok = r0 + rr < n;
#pragma unroll
      for (int p = 0; p < 2; ++p) {  // d <= 256: at most two float4 per lane
        const int c = lane + 32 * p;
        a[rr][p] = ok && c < dv ? __ldcs(r4 + c) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    const float4 *q4 = reinterpret_cast<const float4 *>(qs);
    const float4 b0 = q4[lane], b1 = q4[lane + 32];   // zero beyond d (qs is padded)
#pragma unroll
    for (int rr = 0; rr < kLatRows; ++rr) {
      float acc = 0.0f;
      acc = __fmaf_rn(a[rr][0].x, b0.x, acc);
      acc = __fmaf_rn(a[rr][0].y, b0.y, acc);
      acc = __fmaf_rn(a[rr][0].z, b0.z, acc);
      acc = __fmaf_rn(a[rr][0].w, b0.w, acc);
      acc = __fmaf_rn(a[rr][1].x, b1.x, acc);
      acc = __fmaf_rn(a[rr][1].y, b1.y, acc);
      acc = __fmaf_rn(a[rr][1].z, b1.z, acc);
      acc = __fmaf_rn(a[rr][1].w, b1.w, acc);
      part[rr] = acc;
    }
  } else {
#pragma unroll
    for (int rr = 0; rr < kLatRows; ++rr) {
      const float *row = U + (r0 + rr) * d;
      const bool ok = r0 + rr < n;
      float acc = 0.0f;
#pragma unroll
      for (int p = 0; p < 8; ++p) {  // d <= 256
        const int c = lane + 32 * p;
        if (ok && c < d) acc = __fmaf_rn(__ldcs(row + c), qs[c], acc);
      }
      part[rr] = acc;
    }
  }
}

template <int VEC>
__global__ void __launch_bounds__(kLatThreads)
    k_latency_scan(const float *__restrict__ U, int64_t n, int d, const float *__restrict__ q,
                   const float *__restrict__ qn_p, const float *__restrict__ unrm,
                   const BinFP *__restrict__ bf, const double *__restrict__ fmin,
                   const double *__restrict__ delta, const uint32_t *__restrict__ N, int tau,
                   uint32_t top, int shift, uint32_t *__restrict__ nlo,
                   uint32_t *__restrict__ nup, int32_t *__restrict__ jout,
                   uint32_t *__restrict__ ghist, unsigned long long *__restrict__ nfp64) {
  __shared__ __align__(16) float qs[kMaxD];
  __shared__ uint32_t hist[kLatBins];
  for (int i = threadIdx.x; i < kMaxD; i += blockDim.x) qs[i] = i < d ? q[i] : 0.0f;
  for (int i = threadIdx.x; i < kLatBins; i += blockDim.x) hist[i] = 0;
  __syncthreads();
  const float qn = *qn_p;
  const float cf = latency_cfac(d);
  const int lane = threadIdx.x & 31;
  const int64_t gw = (int64_t)blockIdx.x * (kLatThreads / 32) + (threadIdx.x >> 5);
  const int64_t nw = (int64_t)gridDim.x * (kLatThreads / 32);
  constexpr int kPerIter = kLatRows * kLatSub;  // 32 rows: lane r finishes row r0 + r
  uint32_t fp64 = 0;
  for (int64_t r0 = gw * kPerIter; r0 < n; r0 += nw * kPerIter) {
    float mine = 0.0f;
    // this lane's user: its bound and bin data are loaded while the rows stream in
    const int64_t u = r0 + lane;
    const bool live = u < n;
    const float un = live ? unrm[u] : 0.0f;
    const BinFP bu = live ? bf[u] : BinFP{0.f, 0.f, 0.f, 0.f};
    const double fm = live ? fmin[u] : 0.0;
#pragma unroll 1
    for (int sb = 0; sb < kLatSub; ++sb) {
      float part[kLatRows];
      lane_dots<VEC>(U, r0 + sb * kLatRows, n, d, qs, lane, part);
#pragma unroll
      for (int rr = 0; rr < kLatRows; ++rr) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
          part[rr] = __fadd_rn(part[rr], __shfl_xor_sync(0xffffffffu, part[rr], o));
        if (lane == sb * kLatRows + rr) mine = part[rr];
      }
    }
    if (!live) continue;
    const float b = __fadd_ru(__fmul_ru(__fmul_ru(cf, un), qn), 1e-30f);
    int jlo, jhi;
    bin_interval(bu, fm, tau, __fsub_rd(mine, b), __fadd_ru(mine, b), jlo, jhi);
    int j = jlo;
    if (jlo != jhi) {
      ++fp64;
      j = exact_j(canon_dot_slow(U + u * d, qs, d), fm, delta[u], tau);
    }
    const uint32_t lo = j < tau ? N[u * tau + j] : 0u;
    const uint32_t up = j >= 1 ? N[u * tau + j - 1] : top;
    nlo[u] = lo;
    nup[u] = up;
    jout[u] = j;
    // lanes with the same bin add once (upper bounds crowd into few bins)
    const unsigned bin = min(up >> shift, (uint32_t)(kLatBins - 1));
    const unsigned peers = __match_any_sync(__activemask(), bin);
    if (lane == __ffs(peers) - 1) atomicAdd(&hist[bin], (uint32_t)__popc(peers));
  }
  __syncthreads();
  // this CTA's histogram, stored whole (no atomics across CTAs)
  uint32_t *mine_h = ghist + (size_t)blockIdx.x * kLatBins;
  for (int i = threadIdx.x; i < kLatBins; i += blockDim.x) mine_h[i] = hist[i];
  fp64 = __reduce_add_sync(0xffffffffu, fp64);
  if (lane == 0 && fp64) atomicAdd(nfp64, (unsigned long long)fp64);
}

// ------------------------------------------------------------------
// Bulk-staged form (d a multiple of 4): the rows of U are contiguous, so a chunk
// of kBulkRows users is one cp.async.bulk copy.  Warp kBulkWarps (one lane)
// streams chunks into a ring of kBulkStages shared-memory stages; warps
// 0..kBulkWarps-1 each take kBulkRows / kBulkWarps rows of a stage, free the
// stage as soon as their products are formed, then finish their users.  One CTA
// per SM; every wait is bounded (a timeout sets *err and ends the CTA after the
// copies it issued have landed).
constexpr int kBulkWarps = 8;
constexpr int kBulkRows = 64;
constexpr int kBulkStages = 3;
constexpr int kBulkRowsPerWarp = kBulkRows / kBulkWarps;   // 8
constexpr uint32_t kBulkWait = 1u << 22;

__device__ __forceinline__ uint32_t bulk_smem(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ bool bulk_wait(uint64_t *bar, uint32_t parity) {
  const uint32_t addr = bulk_smem(bar);
  for (uint32_t i = 0; i < kBulkWait; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

size_t bulk_smem_bytes(int d) {
  return 128 + (size_t)kBulkStages * kBulkRows * d * 4 + 16 * kBulkStages +
         sizeof(float) * kMaxD + sizeof(uint32_t) * kLatBins;
}

__global__ void __launch_bounds__((kBulkWarps + 1) * 32, 1)
    k_latency_scan_bulk(const float *__restrict__ U, int64_t n, int d,
                        const float *__restrict__ q, const float *__restrict__ qn_p,
                        const float *__restrict__ unrm, const BinFP *__restrict__ bf,
                        const double *__restrict__ fmin, const double *__restrict__ delta,
                        const uint32_t *__restrict__ N, int tau, uint32_t top, int shift,
                        uint32_t *__restrict__ nlo, uint32_t *__restrict__ nup,
                        int32_t *__restrict__ jout, uint32_t *__restrict__ ghist,
                        unsigned long long *__restrict__ nfp64, int *__restrict__ err) {
  extern __shared__ __align__(128) unsigned char bsm[];
  unsigned char *base = (unsigned char *)(((uintptr_t)bsm + 127) & ~(uintptr_t)127);
  const size_t stage_bytes = (size_t)kBulkRows * d * 4;
  unsigned char *stages = base;
  uint64_t *full = (uint64_t *)(stages + kBulkStages * stage_bytes);
  uint64_t *empty = full + kBulkStages;
  float *qs = (float *)(empty + kBulkStages);
  uint32_t *hist = (uint32_t *)(qs + kMaxD);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = threadIdx.x; i < kMaxD; i += blockDim.x) qs[i] = i < d ? q[i] : 0.0f;
  for (int i = threadIdx.x; i < kLatBins; i += blockDim.x) hist[i] = 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kBulkStages; ++s) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bulk_smem(&full[s])), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bulk_smem(&empty[s])),
                   "r"(kBulkWarps));
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int64_t nch = (n + kBulkRows - 1) / kBulkRows;
  bool failed = false;
  uint32_t fp64 = 0;
  if (warp == kBulkWarps) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      uint32_t it = 0;
      for (int64_t ch = blockIdx.x; ch < nch; ch += gridDim.x, ++it) {
        const int s = it % kBulkStages;
        if (!bulk_wait(&empty[s], ((it / kBulkStages) & 1) ^ 1)) { failed = true; break; }
        const int64_t rows = min((int64_t)kBulkRows, n - ch * kBulkRows);
        const uint32_t bytes = (uint32_t)(rows * d * 4);
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                         bulk_smem(&full[s])),
                     "r"(bytes)
                     : "memory");
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
            "[%3];" ::"r"(bulk_smem(stages + s * stage_bytes)),
            "l"(reinterpret_cast<uint64_t>(U + ch * kBulkRows * d)), "r"(bytes),
            "r"(bulk_smem(&full[s]))
            : "memory");
      }
      if (failed) {
        atomicExch(err, 1);
        // the copies already issued land before the CTA can exit
        for (uint32_t j = (it > kBulkStages ? it - kBulkStages : 0); j < it; ++j)
          bulk_wait(&full[j % kBulkStages], (j / kBulkStages) & 1);
      }
    }
  } else {
    // ------------------------------------------------------------ consumers
    const float qn = *qn_p;
    const float cf = latency_cfac(d);
    const float4 *q4 = reinterpret_cast<const float4 *>(qs);
    const float4 b0 = q4[lane], b1 = q4[lane + 32];
    const int dv = d >> 2;
    uint32_t it = 0;
    for (int64_t ch = blockIdx.x; ch < nch; ch += gridDim.x, ++it) {
      const int s = it % kBulkStages;
      if (!bulk_wait(&full[s], (it / kBulkStages) & 1)) { failed = true; break; }
      const float *st = (const float *)(stages + s * stage_bytes);
      const int64_t u0 = ch * kBulkRows + warp * kBulkRowsPerWarp;
      float mine = 0.0f;
#pragma unroll
      for (int rr = 0; rr < kBulkRowsPerWarp; ++rr) {
        const float4 *r4 =
            reinterpret_cast<const float4 *>(st + (size_t)(warp * kBulkRowsPerWarp + rr) * d);
        float acc = 0.0f;
        if (u0 + rr < n) {
          if (lane < dv) {
            const float4 a = r4[lane];
            acc = __fmaf_rn(a.x, b0.x, acc);
            acc = __fmaf_rn(a.y, b0.y, acc);
            acc = __fmaf_rn(a.z, b0.z, acc);
            acc = __fmaf_rn(a.w, b0.w, acc);
          }
          if (lane + 32 < dv) {
            const float4 a = r4[lane + 32];
            acc = __fmaf_rn(a.x, b1.x, acc);
            acc = __fmaf_rn(a.y, b1.y, acc);
            acc = __fmaf_rn(a.z, b1.z, acc);
            acc = __fmaf_rn(a.w, b1.w, acc);
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
          acc = __fadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
        if (lane == rr) mine = acc;
      }
      // this warp is done with the stage
      __syncwarp();
      if (lane == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bulk_smem(&empty[s]))
                     : "memory");
      const int64_t u = u0 + lane;
      if (lane < kBulkRowsPerWarp && u < n) {
        const float b = __fadd_ru(__fmul_ru(__fmul_ru(cf, unrm[u]), qn), 1e-30f);
        int jlo, jhi;
        const double fm = fmin[u];
        bin_interval(bf[u], fm, tau, __fsub_rd(mine, b), __fadd_ru(mine, b), jlo, jhi);
        int j = jlo;
        if (jlo != jhi) {
          ++fp64;
          j = exact_j(canon_dot_slow(U + u * d, qs, d), fm, delta[u], tau);
        }
        const uint32_t lo = j < tau ? N[u * tau + j] : 0u;
        const uint32_t up = j >= 1 ? N[u * tau + j - 1] : top;
        nlo[u] = lo;
        nup[u] = up;
        jout[u] = j;
        atomicAdd(&hist[min(up >> shift, (uint32_t)(kLatBins - 1))], 1u);
      }
    }
    if (failed && lane == 0) atomicExch(err, 2);
  }
  __syncthreads();
  uint32_t *mine_h = ghist + (size_t)blockIdx.x * kLatBins;
  for (int i = threadIdx.x; i < kLatBins; i += blockDim.x) mine_h[i] = hist[i];
  fp64 = __reduce_add_sync(0xffffffffu, fp64);
  if (lane == 0 && fp64) atomicAdd(nfp64, (unsigned long long)fp64);
}

// Sum of the scan CTAs' histograms: thread b adds bin b over the `parts` rows.
__global__ void __launch_bounds__(128)
    k_latency_hsum(const uint32_t *__restrict__ parts_h, int parts, uint32_t *__restrict__ ghist) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= kLatBins) return;
  uint32_t acc = 0;
#pragma unroll 8
  for (int g = 0; g < parts; ++g) acc += parts_h[(size_t)g * kLatBins + b];
  ghist[b] = acc;
}

// T = upper end of the histogram bin holding the k-th smallest upper-bound
// numerator (so T >= R_up_k); the candidate count of query q is zeroed.
__global__ void __launch_bounds__(1024)
    k_latency_cut(uint32_t *__restrict__ ghist, const int32_t *__restrict__ kq, int q, int shift,
                  uint32_t *__restrict__ T, uint32_t *__restrict__ qcount) {
  __shared__ uint32_t h[kLatBins];
  __shared__ uint32_t part[1024];
  const int t = threadIdx.x;
  for (int i = t; i < kLatBins; i += blockDim.x) h[i] = ghist[i];
  __syncthreads();
  // each thread sums two bins; inclusive scan of the pair sums
  const uint32_t mine = h[2 * t] + h[2 * t + 1];
  part[t] = mine;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const uint32_t v = t >= o ? part[t - o] : 0u;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  const uint32_t k = (uint32_t)kq[q];
  const uint32_t before = part[t] - mine;
  if (before < k && part[t] >= k) {
    const int bin = before + h[2 * t] >= k ? 2 * t : 2 * t + 1;
    const uint64_t hi = ((uint64_t)(bin + 1) << shift) - 1;
    *T = bin == kLatBins - 1 || hi > 0xffffffffull ? 0xffffffffu : (uint32_t)hi;
    qcount[q] = 0;
  }
}

__global__ void k_latency_compact(int64_t n, const uint32_t *__restrict__ nlo,
                                  const uint32_t *__restrict__ nup, const int32_t *__restrict__ j,
                                  const uint32_t *__restrict__ T, int q,
                                  uint32_t *__restrict__ qcount, int32_t *__restrict__ cu,
                                  uint32_t *__restrict__ clo, uint32_t *__restrict__ cup,
                                  int32_t *__restrict__ cj, double *__restrict__ cth) {
  const uint32_t t = *T;
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < n;
       u += (int64_t)gridDim.x * blockDim.x) {
    const bool take = nlo[u] <= t;
    const unsigned act = __ballot_sync(__activemask(), take);
    if (!take) continue;
    const int lane = threadIdx.x & 31, leader = __ffs(act) - 1;
    uint32_t base = 0;
    if (lane == leader) base = atomicAdd(&qcount[q], (uint32_t)__popc(act));
    base = __shfl_sync(act, base, leader);
    const uint32_t pos = base + __popc(act & ((1u << lane) - 1u));
    cu[pos] = (int32_t)u;
    clo[pos] = nlo[u];
    cup[pos] = nup[u];
    cj[pos] = j[u];
    cth[pos] = __longlong_as_double(0x7ff8000000000000ll);  // u.q formed on demand
  }
}

// Step-3 estimate of each compacted candidate (canonical u.q) and its outputs at
// `base`, with global user ids (local id + user_offset).
__global__ void k_candidate_out(const uint32_t *__restrict__ qcount, int q,
                                const int32_t *__restrict__ cu, const uint32_t *__restrict__ clo,
                                const uint32_t *__restrict__ cup, const int32_t *__restrict__ cj,
                                const float *__restrict__ U, const float *__restrict__ qrow, int d,
                                const double *__restrict__ fmin, const double *__restrict__ delta,
                                int tau, uint32_t s, int64_t user_offset, int64_t base,
                                int32_t *__restrict__ ou, uint32_t *__restrict__ olo,
                                uint32_t *__restrict__ oup, double *__restrict__ oest) {
  const int64_t cnt = qcount[q];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < cnt;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = cu[i];
    const double th = canon_dot(U + u * d, qrow, d);
    ou[base + i] = (int32_t)(u + user_offset);
    olo[base + i] = clo[i];
    oup[base + i] = cup[i];
    oest[base + i] = interp_est(th, cj[i], clo[i], cup[i], fmin[u], delta[u], tau, s);
  }
}

// Scratch of the per-query bounds pass.
struct ScanBufs {
  uint32_t *nlo, *nup, *parts, *ghist, *T, *qcount;
  int32_t *jall;
  unsigned long long *nfp64;   // [0] canonical evaluations, [1] select error, [2] scan error
  int grid, shift;
  uint32_t top;
  bool vec4, bulk;
  size_t bulk_smem;
};

rkr_status alloc_scan(const rkr_index *idx, int nq, int ctas_per_sm, DevBuf (&b)[8], ScanBufs &sb,
                      cudaStream_t st) {
  const int64_t n = idx->n;
  sb.top = (uint32_t)(idx->m * idx->s);
  sb.shift = 0;
  while ((sb.top >> sb.shift) >= (uint32_t)kLatBins) ++sb.shift;
  sb.vec4 = (idx->d % 4) == 0 && ((uintptr_t)idx->U % 16) == 0;
  int occ = 0;
  if (sb.vec4)
    RKR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_latency_scan<4>, kLatThreads, 0));
  else
    RKR_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_latency_scan<1>, kLatThreads, 0));
  occ = std::max(occ, 1);
  if (ctas_per_sm > 0) occ = std::min(occ, ctas_per_sm);
  const int64_t warps_needed = (n + 31) / 32;
  sb.grid = (int)std::max<int64_t>(
      1, std::min<int64_t>((int64_t)sm_count() * occ,
                           (warps_needed + kLatThreads / 32 - 1) / (kLatThreads / 32)));
  // bulk-staged scan: rows of a multiple of 16 bytes and a U base aligned to 16
  sb.bulk = tuning().latency_bulk && sb.vec4;
  if (sb.bulk) {
    sb.bulk_smem = bulk_smem_bytes(idx->d);
    RKR_CUDA(cudaFuncSetAttribute(k_latency_scan_bulk,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sb.bulk_smem));
    sb.grid = (int)std::max<int64_t>(
        1, std::min<int64_t>(sm_count(), (n + kBulkRows - 1) / kBulkRows));
  }
  RKR_TRY(tmp_alloc(b[0], &sb.nlo, n, st));
  RKR_TRY(tmp_alloc(b[1], &sb.nup, n, st));
  RKR_TRY(tmp_alloc(b[2], &sb.jall, n, st));
  RKR_TRY(tmp_alloc(b[3], &sb.parts, (size_t)sb.grid * kLatBins, st));
  RKR_TRY(tmp_alloc(b[4], &sb.ghist, kLatBins, st));
  RKR_TRY(tmp_alloc(b[5], &sb.T, 1, st));
  RKR_TRY(tmp_alloc(b[6], &sb.qcount, nq, st));
  RKR_TRY(tmp_alloc(b[7], &sb.nfp64, 3, st));
  RKR_CUDA(cudaMemsetAsync(sb.qcount, 0, sizeof(uint32_t) * nq, st));
  RKR_CUDA(cudaMemsetAsync(sb.nfp64, 0, 3 * sizeof(unsigned long long), st));
  return RKR_OK;
}

// Bounds of every user for query q, their histogram and the cut T.
rkr_status scan_pass(const rkr_index *idx, const QueryCommon &qc, int q, const ScanBufs &sb,
                     cudaStream_t st) {
  const float *qrow = qc.Qd + (int64_t)q * idx->d;
  {
    ProfScope prof("k_latency_scan", st,
                   (double)idx->n * (4.0 * idx->d + 4 + sizeof(BinFP) + 8 + 8 + 12));
    if (sb.bulk)
      k_latency_scan_bulk<<<sb.grid, (kBulkWarps + 1) * 32, sb.bulk_smem, st>>>(
          idx->U, idx->n, idx->d, qrow, qc.qnrm + q, idx->unrm, qc.bf, idx->fmin, idx->delta,
          idx->N, idx->tau, sb.top, sb.shift, sb.nlo, sb.nup, sb.jall, sb.parts, sb.nfp64,
          (int *)(sb.nfp64 + 2));
    else if (sb.vec4)
      k_latency_scan<4><<<sb.grid, kLatThreads, 0, st>>>(
          idx->U, idx->n, idx->d, qrow, qc.qnrm + q, idx->unrm, qc.bf, idx->fmin, idx->delta,
          idx->N, idx->tau, sb.top, sb.shift, sb.nlo, sb.nup, sb.jall, sb.parts, sb.nfp64);
    else
      k_latency_scan<1><<<sb.grid, kLatThreads, 0, st>>>(
          idx->U, idx->n, idx->d, qrow, qc.qnrm + q, idx->unrm, qc.bf, idx->fmin, idx->delta,
          idx->N, idx->tau, sb.top, sb.shift, sb.nlo, sb.nup, sb.jall, sb.parts, sb.nfp64);
    note_launch();
  }
  {
    const int prof_slot = prof_begin("k_latency_hsum", st);
    k_latency_hsum<<<kLatBins / 128, 128, 0, st>>>(sb.parts, sb.grid, sb.ghist);
    prof_end(prof_slot, st, 0.0);
    note_launch();
  }
  {
    const int prof_slot = prof_begin("k_latency_cut", st);
    k_latency_cut<<<1, 1024, 0, st>>>(sb.ghist, qc.kq_d, q, sb.shift, sb.T, sb.qcount);
    prof_end(prof_slot, st, 0.0);
    note_launch();
  }
  RKR_CUDA(cudaGetLastError());
  return RKR_OK;
}

}  // namespace lat

using namespace lat;

// Per query, the users of this index whose lower bound is at most an upper
// estimate T of this index's R_up_k, with their bounds and step-3 estimates.
rkr_status run_query_approx_candidates(const rkr_index *idx, const QueryCommon &qc, int nq,
                                       int64_t user_offset, int64_t capacity, int64_t *offs_host,
                                       int32_t *users_d, uint32_t *nlo_d, uint32_t *nup_d,
                                       double *est_d, cudaStream_t st) {
  const int64_t n = idx->n;
  const int d = idx->d;
  DevBuf bs[8], b7, b8, b9, b10, b11;
  ScanBufs sb;
  RKR_TRY(alloc_scan(idx, nq, tuning().latency_ctas_per_sm, bs, sb, st));
  uint32_t *clo, *cup;
  int32_t *cu, *cj;
  double *cth;
  RKR_TRY(tmp_alloc(b7, &cu, n, st));
  RKR_TRY(tmp_alloc(b8, &clo, n, st));
  RKR_TRY(tmp_alloc(b9, &cup, n, st));
  RKR_TRY(tmp_alloc(b10, &cj, n, st));
  RKR_TRY(tmp_alloc(b11, &cth, n, st));
  const int cgrid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 8);
  offs_host[0] = 0;
  for (int q = 0; q < nq; ++q) {
    const float *qrow = qc.Qd + (int64_t)q * d;
    RKR_TRY(scan_pass(idx, qc, q, sb, st));
    k_latency_compact<<<cgrid, 256, 0, st>>>(n, sb.nlo, sb.nup, sb.jall, sb.T, q, sb.qcount, cu,
                                             clo, cup, cj, cth);
    note_launch();
    RKR_CUDA(cudaGetLastError());
    uint32_t cnt = 0;
    RKR_CUDA(cudaMemcpyAsync(&cnt, sb.qcount + q, sizeof(cnt), cudaMemcpyDeviceToHost, st));
    RKR_CUDA(cudaStreamSynchronize(st));
    offs_host[q + 1] = offs_host[q] + cnt;
    if (offs_host[q + 1] <= capacity && cnt > 0) {
      k_candidate_out<<<(unsigned)std::min<int64_t>((cnt + 255) / 256, 4 * sm_count()), 256, 0,
                        st>>>(sb.qcount, q, cu, clo, cup, cj, idx->U, qrow, d, idx->fmin,
                              idx->delta, idx->tau, (uint32_t)idx->s, user_offset, offs_host[q],
                              users_d, nlo_d, nup_d, est_d);
      note_launch();
      RKR_CUDA(cudaGetLastError());
    }
  }
  RKR_CUDA(cudaStreamSynchronize(st));
  {
    unsigned long long h[3] = {0, 0, 0};
    RKR_CUDA(cudaMemcpy(h, sb.nfp64, sizeof(h), cudaMemcpyDeviceToHost));
    if ((int)h[2]) return fail(RKR_ETIMEOUT, "latency scan wait timed out (%d)", (int)h[2]);
  }
  if (offs_host[nq] > capacity)
    return fail(RKR_ENOMEM, "candidate capacity %lld is below the %lld candidates found",
                (long long)capacity, (long long)offs_host[nq]);
  return RKR_OK;
}

rkr_status run_query_approx_single(const rkr_index *idx, const QueryCommon &qc, int nq, double c,
                                   int32_t *users_d, uint32_t *nlo_d, uint32_t *nup_d,
                                   double *est_d, int32_t *case_d, int32_t *nc_d,
                                   rkr_query_stats *stats, cudaStream_t st) {
  const int64_t n = idx->n;
  DevBuf bs[8], b7, b8, b9, b10, b11;
  ScanBufs sb;
  RKR_TRY(alloc_scan(idx, nq, tuning().latency_ctas_per_sm, bs, sb, st));
  uint32_t *clo, *cup;
  int32_t *cu, *cj;
  double *cth;
  RKR_TRY(tmp_alloc(b7, &cu, n, st));
  RKR_TRY(tmp_alloc(b8, &clo, n, st));
  RKR_TRY(tmp_alloc(b9, &cup, n, st));
  RKR_TRY(tmp_alloc(b10, &cj, n, st));
  RKR_TRY(tmp_alloc(b11, &cth, n, st));
  int *err = (int *)(sb.nfp64 + 1);
  const int cgrid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 8);
  Timer t1(st);
  for (int q = 0; q < nq; ++q) {
    RKR_TRY(scan_pass(idx, qc, q, sb, st));
    {
      const int prof_slot = prof_begin("k_latency_compact", st);
      k_latency_compact<<<cgrid, 256, 0, st>>>(n, sb.nlo, sb.nup, sb.jall, sb.T, q, sb.qcount, cu,
                                               clo, cup, cj, cth);
      prof_end(prof_slot, st, 0.0);
      note_launch();
    }
    RKR_TRY(launch_select_approx(q, 1, qc.out_off_d, sb.qcount, cu, clo, cup, cth, cj, qc.Qd,
                                 qc.kq_d, c, qc.out_off_d, users_d, nlo_d, nup_d, est_d, case_d,
                                 nc_d, err, st, idx));
  }
  RKR_CUDA(cudaGetLastError());
  const double ms = t1.stop();
  unsigned long long h[3] = {0, 0, 0};
  RKR_CUDA(cudaMemcpyAsync(h, sb.nfp64, sizeof(h), cudaMemcpyDeviceToHost, st));
  RKR_CUDA(cudaStreamSynchronize(st));
  if ((int)h[2]) return fail(RKR_ETIMEOUT, "latency scan wait timed out (%d)", (int)h[2]);
  if ((int)h[1]) return fail(RKR_EINTERNAL, "fewer than k candidates for a query");
  if (stats) {
    stats->pairs = n * (int64_t)nq;
    stats->candidates = 0;
    stats->fp64_dots = (int64_t)h[0];
    stats->ms_theta = ms;
  }
  return RKR_OK;
}

}  // namespace rkr

// ------------------------------------------------------------------ session
// A serving form of the one-at-a-time path: persistent device buffers for one
// query and a CUDA graph of its launches (query norm, scan, histogram sum, cut,
// compaction, steps 2-3), captured once at creation and replayed per query.
struct rkr_session {
  rkr_index *idx = nullptr;
  int max_k = 0, d = 0;
  double c = 2.0;
  cudaStream_t st = nullptr;
  float *q_dev = nullptr, *qn_dev = nullptr;
  int32_t *k_dev = nullptr;
  int64_t *off_dev = nullptr;
  int32_t *users = nullptr, *ocase = nullptr, *onc = nullptr;
  uint32_t *onlo = nullptr, *onup = nullptr;
  double *oest = nullptr;
  rkr::DevBuf scan_bufs[8], cand_bufs[5], out_bufs[10];
  rkr::lat::ScanBufs sb;
  uint32_t *clo = nullptr, *cup = nullptr;
  int32_t *cu = nullptr, *cj = nullptr;
  double *cth = nullptr;
  // pinned host staging: query, k, then the outputs and the two error words
  float *q_h = nullptr;
  int32_t *k_h = nullptr;
  unsigned char *out_h = nullptr;
  size_t out_bytes = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace rkr {
namespace {

rkr_status session_enqueue(rkr_session *s) {
  QueryCommon qc;
  qc.Qd = s->q_dev;
  qc.qnrm = s->qn_dev;
  qc.kq_d = s->k_dev;
  qc.out_off_d = s->off_dev;
  qc.bf = s->idx->binfp;
  qc.xbf = s->idx->xbin;
  RKR_TRY(row_norms(s->q_dev, 1, s->d, nullptr, s->qn_dev, s->st));
  RKR_TRY(scan_pass(s->idx, qc, 0, s->sb, s->st));
  const int64_t n = s->idx->n;
  const int cgrid = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 8);
  k_latency_compact<<<cgrid, 256, 0, s->st>>>(n, s->sb.nlo, s->sb.nup, s->sb.jall, s->sb.T, 0,
                                              s->sb.qcount, s->cu, s->clo, s->cup, s->cj,
                                              s->cth);
  note_launch();
  RKR_TRY(launch_select_approx(0, 1, s->off_dev, s->sb.qcount, s->cu, s->clo, s->cup, s->cth,
                               s->cj, s->q_dev, s->k_dev, s->c, s->off_dev, s->users, s->onlo,
                               s->onup, s->oest, s->ocase, s->onc, (int *)(s->sb.nfp64 + 1),
                               s->st, s->idx));
  return RKR_OK;
}

void session_release(rkr_session *s) {
  if (!s) return;
  if (s->exec) cudaGraphExecDestroy(s->exec);
  if (s->graph) cudaGraphDestroy(s->graph);
  if (s->q_h) cudaFreeHost(s->q_h);
  if (s->k_h) cudaFreeHost(s->k_h);
  if (s->out_h) cudaFreeHost(s->out_h);
  // device blocks go back to the pool on the session's stream, before it goes
  for (DevBuf *group : {s->scan_bufs, s->cand_bufs, s->out_bufs}) {
    const int count = group == s->scan_bufs ? 8 : (group == s->cand_bufs ? 5 : 10);
    for (int i = 0; i < count; ++i)
      if (group[i].p) {
        cudaFreeAsync(group[i].p, group[i].st);
        group[i].p = nullptr;
      }
  }
  if (s->st) {
    cudaStreamSynchronize(s->st);
    cudaStreamDestroy(s->st);
  }
  delete s;
}

}  // namespace
}  // namespace rkr

using namespace rkr;

extern "C" rkr_status rkr_session_create(rkr_index *idx, int32_t max_k, double c, void *stream,
                                         rkr_session **out) {
  set_error("%s", "");
  if (!idx || !out) return fail(RKR_EINVAL, "null argument");
  *out = nullptr;
  if (max_k < 1 || max_k > kMaxK || max_k > idx->n)
    return fail(RKR_EINVAL, "max_k must be in [1, min(n, %d)]", kMaxK);
  if (!(c >= 1.0) || !isfinite(c)) return fail(RKR_EINVAL, "c must be a finite value >= 1");
  RKR_TRY(check_device());
  rkr_session *s = new (std::nothrow) rkr_session();
  if (!s) return fail(RKR_ENOMEM, "host allocation failed");
  struct Guard {
    rkr_session *s;
    ~Guard() { session_release(s); }
  } guard{s};
  s->idx = idx;
  s->max_k = max_k;
  s->c = c;
  s->d = idx->d;
  RKR_CUDA(cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking));
  (void)stream;  // the session keeps its own stream: the graph is captured on it
  cudaStream_t st = s->st;
  const int64_t n = idx->n;
  RKR_TRY(alloc_scan(idx, 1, tuning().latency_ctas_per_sm, s->scan_bufs, s->sb, st));
  RKR_TRY(tmp_alloc(s->cand_bufs[0], &s->cu, n, st));
  RKR_TRY(tmp_alloc(s->cand_bufs[1], &s->clo, n, st));
  RKR_TRY(tmp_alloc(s->cand_bufs[2], &s->cup, n, st));
  RKR_TRY(tmp_alloc(s->cand_bufs[3], &s->cj, n, st));
  RKR_TRY(tmp_alloc(s->cand_bufs[4], &s->cth, n, st));
  RKR_TRY(tmp_alloc(s->out_bufs[0], &s->q_dev, kMaxD, st));
  RKR_TRY(tmp_alloc(s->out_bufs[1], &s->qn_dev, 1, st));
  RKR_TRY(tmp_alloc(s->out_bufs[2], &s->k_dev, 1, st));
  RKR_TRY(tmp_alloc(s->out_bufs[3], &s->off_dev, 2, st));
  RKR_TRY(tmp_alloc(s->out_bufs[4], &s->users, max_k, st));
  RKR_TRY(tmp_alloc(s->out_bufs[5], &s->onlo, max_k, st));
  RKR_TRY(tmp_alloc(s->out_bufs[6], &s->onup, max_k, st));
  RKR_TRY(tmp_alloc(s->out_bufs[7], &s->oest, max_k, st));
  RKR_TRY(tmp_alloc(s->out_bufs[8], &s->ocase, 1, st));
  RKR_TRY(tmp_alloc(s->out_bufs[9], &s->onc, 1, st));
  RKR_CUDA(cudaMemsetAsync(s->off_dev, 0, 2 * sizeof(int64_t), st));
  RKR_CUDA(cudaMemsetAsync(s->q_dev, 0, kMaxD * sizeof(float), st));
  const int32_t one = 1;
  RKR_CUDA(cudaMemcpyAsync(s->k_dev, &one, sizeof(one), cudaMemcpyHostToDevice, st));
  s->out_bytes = (size_t)max_k * (4 + 4 + 4 + 8) + 4 + 4 + 8 + 8;
  RKR_CUDA(cudaMallocHost(&s->q_h, sizeof(float) * kMaxD));
  RKR_CUDA(cudaMallocHost(&s->k_h, sizeof(int32_t)));
  RKR_CUDA(cudaMallocHost(&s->out_h, s->out_bytes));
  // one uncaptured run (sets function attributes, warms the pool), then the capture
  RKR_TRY(session_enqueue(s));
  RKR_CUDA(cudaStreamSynchronize(st));
  RKR_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  const rkr_status es = session_enqueue(s);
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(st, &g);
  s->graph = g;
  RKR_TRY(es);
  if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
  RKR_CUDA(cudaGraphInstantiate(&s->exec, s->graph, 0));
  *out = s;
  guard.s = nullptr;
  return RKR_OK;
}

extern "C" rkr_status rkr_session_query(rkr_session *s, const float *q, int32_t k,
                                        int32_t *out_users, uint32_t *out_nlow,
                                        uint32_t *out_nup, double *out_est, int32_t *out_case,
                                        int32_t *out_nc) {
  set_error("%s", "");
  if (!s || !q || !out_users) return fail(RKR_EINVAL, "null argument");
  if (k < 1 || k > s->max_k) return fail(RKR_EINVAL, "k must be in [1, %d]", s->max_k);
  const int d = s->d;
  cudaStream_t st = s->st;
  cudaPointerAttributes pa;
  const bool qdev = cudaPointerGetAttributes(&pa, q) == cudaSuccess &&
                    (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged);
  cudaGetLastError();
  if (qdev) RKR_CUDA(cudaMemcpy(s->q_h, q, sizeof(float) * d, cudaMemcpyDeviceToHost));
  else memcpy(s->q_h, q, sizeof(float) * d);
  double ss = 0.0;
  for (int i = 0; i < d; ++i) {
    if (!isfinite(s->q_h[i])) return fail(RKR_EINVAL, "q must be finite");
    ss += (double)s->q_h[i] * (double)s->q_h[i];
  }
  if (sqrt(ss) * (1.0 + 0x1p-20) > (double)s->idx->pmax) {
    // outside the item norms: the bin bounds of this query need a wider range,
    // which the captured launches do not cover
    return rkr_query_approx_single(s->idx, q, 1, &k, s->c, out_users, out_nlow, out_nup,
                                   out_est, out_case, out_nc, nullptr, st);
  }
  *s->k_h = k;
  RKR_CUDA(cudaMemcpyAsync(s->q_dev, s->q_h, sizeof(float) * d, cudaMemcpyHostToDevice, st));
  RKR_CUDA(cudaMemcpyAsync(s->k_dev, s->k_h, sizeof(int32_t), cudaMemcpyHostToDevice, st));
  RKR_CUDA(cudaGraphLaunch(s->exec, st));
  unsigned char *o = s->out_h;
  const size_t K = (size_t)k;
  RKR_CUDA(cudaMemcpyAsync(o, s->users, 4 * K, cudaMemcpyDeviceToHost, st));
  RKR_CUDA(cudaMemcpyAsync(o + 4 * K, s->onlo, 4 * K, cudaMemcpyDeviceToHost, st));
  RKR_CUDA(cudaMemcpyAsync(o + 8 * K, s->onup, 4 * K, cudaMemcpyDeviceToHost, st));
  RKR_CUDA(cudaMemcpyAsync(o + 12 * K, s->oest, 8 * K, cudaMemcpyDeviceToHost, st));
  RKR_CUDA(cudaMemcpyAsync(o + 20 * K, s->ocase, 4, cudaMemcpyDeviceToHost, st));
  RKR_CUDA(cudaMemcpyAsync(o + 20 * K + 4, s->onc, 4, cudaMemcpyDeviceToHost, st));
  RKR_CUDA(cudaMemcpyAsync(o + 20 * K + 8, s->sb.nfp64 + 1, 16, cudaMemcpyDeviceToHost, st));
  RKR_CUDA(cudaStreamSynchronize(st));
  unsigned long long ew[2];
  memcpy(ew, o + 20 * K + 8, 16);
  if ((int)ew[1]) return fail(RKR_ETIMEOUT, "latency scan wait timed out (%d)", (int)ew[1]);
  if ((int)ew[0]) return fail(RKR_EINTERNAL, "fewer than k candidates for the query");
  struct Out {
    void *dst;
    size_t off, bytes;
  } outs[] = {{out_users, 0, 4 * K},       {out_nlow, 4 * K, 4 * K}, {out_nup, 8 * K, 4 * K},
              {out_est, 12 * K, 8 * K},    {out_case, 20 * K, 4},    {out_nc, 20 * K + 4, 4}};
  for (const Out &x : outs) {
    if (!x.dst) continue;
    cudaPointerAttributes a;
    const bool dev = cudaPointerGetAttributes(&a, x.dst) == cudaSuccess &&
                     (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    if (dev) RKR_CUDA(cudaMemcpy(x.dst, o + x.off, x.bytes, cudaMemcpyHostToDevice));
    else memcpy(x.dst, o + x.off, x.bytes);
  }
  return RKR_OK;
}

extern "C" void rkr_session_free(rkr_session *s) { session_release(s); }
