// tc_pair.cuh -- the CTA-pair form of the screen kernel, for single-GPU builds.
//
// The two CTAs of a cluster share each B chunk: each loads one half with a TMA
// load multicast to both.  The tensor maps cover buffers of this GPU only.
// This header is compiled only into the single-GPU library (RKR_CLUSTER_MULTICAST
// defined, the default build); the replica build used when one process runs per
// GPU of a multi-GPU job leaves it out and runs every screen on k_screen.
#pragma once

#ifndef RKR_CLUSTER_MULTICAST
#error "tc_pair.cuh belongs to the single-GPU build (RKR_CLUSTER_MULTICAST)"
#endif

#include "tc_screen.cuh"

namespace rkr {
namespace tc {

// Multicast form of tma_load_2d: the box lands at the same shared-memory offset
// in every CTA of the cluster named in `mask`, and completes bytes on the
// mbarrier at the same offset in each of them.
__device__ __forceinline__ void tma_load_2d_mc(void *dst, const CUtensorMap *map, int x, int y,
                                               uint64_t *bar, uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      ".multicast::cluster [%0], [%1, {%2, %3}], [%4], %5;" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar)), "h"(mask)
      : "memory");
}

// Arrives once on the mbarrier at this offset in every CTA of `mask` when the
// MMAs issued so far by this thread complete.
__device__ __forceinline__ void umma_commit_mc(uint64_t *bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(smem_u32(bar)), "h"(mask)
      : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Every thread of every CTA in the cluster.
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}

// Pair form for row-owned units (ROW schedule): the two CTAs of a cluster take
// row blocks 2p and 2p + 1 of the same pair p and walk the same column tiles in
// step.  Each loads its own A chunk and one half of the B chunk, multicast to
// both, so a stage still holds a full A and B chunk while each SM reads two
// thirds of the bytes from L2.  A stage is free for the next multicast only
// when the MMAs of both CTAs have used it: their commits arrive on the empty
// barrier of both (count 2).  The MMA sequence is that of k_screen, so both
// kernels give the same bits.  A CTA whose row block lies past the end (odd
// count) loads zero rows, still feeds its half of B, and skips the epilogue.
//
// After a timeout: each role stops, the CTA records the failure, and at exit
// both CTAs first pass a cluster barrier (after which neither issues a load),
// then the producer of a failed CTA waits again for the stages still in flight
// (loads the peer issued just before it stopped included), and a second
// cluster barrier keeps either CTA from leaving while the other still waits.
template <int BN, int STAGES, class Epi>
__global__ void __launch_bounds__(kThreads, 1)
    k_screen_pair(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
                  const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl,
                  Operands op, Schedule sch, Epi epi, int *err) {
  using L = Layout<BN>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *stages = base;
  uint64_t *full = (uint64_t *)(stages + (size_t)STAGES * L::kStage);
  uint64_t *empty = full + STAGES;
  uint64_t *acc_full = empty + STAGES;
  uint64_t *acc_empty = acc_full + 2;
  uint64_t *drain = acc_empty + 2;
  uint32_t *tmem_slot = (uint32_t *)(drain + 1);
  // tmem_slot[1] records a failure of any role (the dynamic region is already at
  // the shared-memory limit, so no static shared variable is added)
  volatile uint32_t *s_failed = tmem_slot + 1;
  char *escratch = (char *)(tmem_slot + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rank = (int)cluster_rank();               // 0 or 1
  const int pair0 = blockIdx.x >> 1, npair_ctas = gridDim.x >> 1;
  const int npairs = (sch.nunits + 1) >> 1;
  const int nseg = op.split ? 3 : 1;
  const int nk = op.kchunks * nseg;
  constexpr uint32_t kTmemCols = 2 * BN;
  constexpr uint32_t kHalfB = (BN / 2) * KCH * 2;     // bytes of one B half

  if (threadIdx.x == 0) {
    *s_failed = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 2);   // the MMA commits of both CTAs
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], kEpiWarps);
    }
    mbar_init(drain, 1);
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc(tmem_slot, kTmemCols);
  tc_fence_before();
  __syncthreads();
  cluster_sync();   // the peer's barriers exist before anything is multicast to them
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  bool failed = false;
  uint32_t issued = 0;  // producer: loads issued

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA
    if (lane == 0) {
      prefetch_map(&mAh); prefetch_map(&mBh);
      if (op.split) { prefetch_map(&mAl); prefetch_map(&mBl); }
      uint32_t it = 0;
      for (int p = pair0; p < npairs && !failed; p += npair_ctas) {
        const int rb = 2 * p + rank;    // may be one past the last row block
        for (int ct = 0; ct < sch.nct && !failed; ++ct)
          for (int kc = 0; kc < nk; ++kc, ++it) {
            const int s = it % STAGES;
            const uint32_t ph = (it / STAGES) & 1;
            if (!mbar_wait(&empty[s], ph ^ 1)) { failed = true; break; }
            unsigned char *sa = stages + (size_t)s * L::kStage;
            unsigned char *sb = sa + L::kA;
            const int g = kc / op.kchunks, c = kc - g * op.kchunks;
            mbar_expect_tx(&full[s], L::kStage);
            // split order: hi.lo, lo.hi, then hi.hi (small terms first)
            const bool alo = op.split && g == 1, blo = op.split && g == 0;
            const int kx = c * KCH;
            tma_load_2d(sa, alo ? &mAl : &mAh, kx, rb * BM, &full[s]);
            tma_load_2d_mc(sb + (size_t)rank * kHalfB, blo ? &mBl : &mBh, kx,
                           ct * BN + rank * (BN / 2), &full[s], (uint16_t)0x3);
          }
      }
      issued = it;
      if (failed) {
        atomicExch(err, 1);
        *s_failed = 1;
        for (uint32_t j = (it > STAGES ? it - STAGES : 0); j < it; ++j)
          mbar_wait(&full[j % STAGES], (j / STAGES) & 1);
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA
    if (lane == 0) {
      const uint32_t idesc = idesc_bf16(BM, BN);
      uint32_t it = 0, t = 0;
      for (int p = pair0; p < npairs && !failed; p += npair_ctas)
        for (int ct = 0; ct < sch.nct && !failed; ++ct, ++t) {
          const int b = t & 1;
          const uint32_t aph = (t >> 1) & 1;
          if (!mbar_wait(&acc_empty[b], aph ^ 1)) { failed = true; break; }
          tc_fence_after();
          const uint32_t dt = tmem + (uint32_t)(b * BN);
          for (int kc = 0; kc < nk; ++kc, ++it) {
            const int s = it % STAGES;
            const uint32_t ph = (it / STAGES) & 1;
            if (!mbar_wait(&full[s], ph)) { failed = true; break; }
            tc_fence_after();
            const uint32_t sa = smem_u32(stages + (size_t)s * L::kStage);
            const uint32_t sb = sa + L::kA;
            const int c = kc % op.kchunks;
            const int steps = min(4, op.ksteps - c * 4);
            for (int k = 0; k < steps; ++k)
              umma_bf16(dt, sw128_desc(sa + k * 32), sw128_desc(sb + k * 32), idesc,
                        (kc > 0 || k > 0) ? 1u : 0u);
            umma_commit_mc(&empty[s], (uint16_t)0x3);
          }
          if (failed) break;
          umma_commit(&acc_full[b]);
        }
      if (failed) {
        atomicExch(err, 2);
        *s_failed = 1;
      }
      umma_commit(drain);
      mbar_wait(drain, 0);
    }
  } else {
    // ----------------------------------------------------------- epilogue
    const int e = warp - 2;
    const int et = threadIdx.x - 64;
    const int quarter = warp & 3;
    const int half = e >> 2;
    const int r = quarter * 32 + lane;
    uint32_t t = 0;
    typename Epi::Thread ts;
    for (int p = pair0; p < npairs && !failed; p += npair_ctas) {
      const int rb = 2 * p + rank;
      const bool real = rb < sch.nunits;   // ROW schedule: unit index = row block
      Unit u;
      u.rb0 = rb; u.rb1 = rb + 1; u.ct0 = 0; u.ct1 = sch.nct;
      if (real) epi.unit_begin(escratch, u, et, ts);
      epi_sync();
      for (int ct = 0; ct < sch.nct && !failed; ++ct, ++t) {
        const int b = t & 1;
        const uint32_t aph = (t >> 1) & 1;
        const bool ok = mbar_wait(&acc_full[b], aph, op.epi_wait);
        if (epi_vote_any(!ok)) { failed = true; break; }
        tc_fence_after();
        if (real) {
          epi.tile_begin(escratch, rb, ct, r, half, ts);
          const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * BN);
#pragma unroll 1
          for (int cc = 0; cc < BN / 64; ++cc) {
            const int col = half * (BN / 2) + cc * 32;
            float v[32];
            tmem_ld32(trow + col, v);
            epi.chunk(escratch, rb, ct, r, col, trow + (uint32_t)col, v, ts);
          }
          epi.tile_end(escratch, rb, ct, r, half, ts);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[b]);
      }
      epi_sync();
      if (!failed && real) epi.unit_end(escratch, u, et, ts);
      epi_sync();
    }
    if (failed && lane == 0) {
      atomicExch(err, 3);
      *s_failed = 1;
    }
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();   // from here on neither CTA issues a load
  if (warp == 0 && lane == 0 && *s_failed) {
    for (uint32_t j = (issued > STAGES ? issued - STAGES : 0); j < issued; ++j)
      mbar_wait(&full[j % STAGES], (j / STAGES) & 1);
  }
  __syncthreads();
  cluster_sync();   // neither CTA leaves while the other may still be waiting on it
  tc_fence_after();
  if (warp == 1) {
    __syncwarp();
    tmem_dealloc(tmem, kTmemCols);
  }
}

}  // namespace tc
}  // namespace rkr
