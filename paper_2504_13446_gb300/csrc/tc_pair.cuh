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
            if (!mbar_wait(&empty[s], ph ^ 1, kWaitLimit, true)) { failed = true; break; }
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
          if (!mbar_wait(&acc_empty[b], aph ^ 1, kWaitLimit, true)) { failed = true; break; }
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
          epi_tile_columns<BN>(epi, escratch, rb, ct, r, half, trow, ts);
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

// ------------------------------------------------------------- 2-SM MMA form
// Shared-memory address of the same offset in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t map_to_rank(uint32_t saddr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
  return r;
}

// TMA load into this CTA's shared memory whose bytes complete on an mbarrier of
// either CTA of the pair (`bar` is a cluster address).
__device__ __forceinline__ void tma_load_2d_peerbar(void *dst, const CUtensorMap *map, int x,
                                                    int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.cta_group::2"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
      : "memory");
}

// One MMA over the CTA pair: D (M = 256 rows, 128 in each CTA's TMEM) += A.B^T,
// A's rows 0..127 in this CTA's shared memory and 128..255 in the peer's at the
// same offset, B's rows (columns of D) split the same way.
__device__ __forceinline__ void umma_bf16_pair(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                               uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// Arrives once on the mbarrier at this offset in every CTA of `mask` when the
// pair MMAs issued so far by this thread complete.
__device__ __forceinline__ void umma_commit_pair(uint64_t *bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64"
      " [%0], %1;" ::"r"(smem_u32(bar)), "h"(mask)
      : "memory");
}

// TMEM allocation for pair MMAs: one warp of each CTA of the pair takes part.
__device__ __forceinline__ void tmem_alloc_pair(uint32_t *dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

// Arrive on an mbarrier given by its cluster address (this CTA's or the peer's).
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar)
               : "memory");
}

template <int BN>
struct Layout2 {
  static constexpr uint32_t kA = BM * KCH * 2;            // 16 KB: this CTA's 128 rows
  static constexpr uint32_t kB = (BN / 2) * KCH * 2;      // this CTA's half of the B chunk
  static constexpr uint32_t kStage = kA + kB;
};

// Stages of the 2-SM form that fit beside the epilogue's scratch (at most 8).
template <int BN, class Epi>
constexpr int stages2() {
  constexpr size_t avail = 232448 - 1024 - 16 - 8 * 21 - Epi::kSmem;
  constexpr int s = (int)(avail / Layout2<BN>::kStage);
  return s > 8 ? 8 : s;
}

template <int BN, int STAGES, class Epi>
constexpr size_t screen2_smem_bytes() {
  return 1024 + (size_t)STAGES * Layout2<BN>::kStage + 8 * (2 * STAGES + 5) + 16 + Epi::kSmem;
}

// 2-SM form for row-owned units (ROW schedule).  The CTAs of a cluster take row
// blocks 2p and 2p + 1 and walk the same column tiles in step, as in
// k_screen_pair, but the pair's MMAs are single instructions over both SMs
// (tcgen05 cta_group::2, M = 256): each CTA stages only its own A chunk and one
// half of the B chunk, so a stage takes two thirds of the shared memory of the
// multicast form and more stages fit.  The leader CTA (rank 0) issues every
// MMA; each CTA's TMEM holds the accumulators of its own 128 rows, and its
// epilogue is that of the other forms.
//
// Barriers: full[s] of the leader counts the bytes of both CTAs' loads (the
// leader arrives with the expected total); empty[s] and acc_full[b] of both
// CTAs are signalled by the leader's commits, multicast to the pair;
// acc_empty[b] of the leader counts the epilogue warps of both CTAs; drain of
// both CTAs signals that the leader's MMAs have completed (they read the peer's
// shared memory and write its TMEM).  After a timeout each role stops, the
// leader's MMAs are drained, both CTAs pass a cluster barrier, the leader's
// producer waits again for the stages still in flight, and a second cluster
// barrier keeps either CTA from leaving while the other still waits.
template <int BN, int STAGES, class Epi>
__global__ void __launch_bounds__(kThreads, 1)
    k_screen_2sm(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
                 const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl,
                 Operands op, Schedule sch, Epi epi, int *err) {
  using L = Layout2<BN>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *stages = base;
  uint64_t *full = (uint64_t *)(stages + (size_t)STAGES * L::kStage);
  uint64_t *empty = full + STAGES;
  uint64_t *acc_full = empty + STAGES;
  uint64_t *acc_empty = acc_full + 2;
  uint64_t *drain = acc_empty + 2;
  uint32_t *tmem_slot = (uint32_t *)(drain + 1);
  volatile uint32_t *s_failed = tmem_slot + 1;
  char *escratch = (char *)(tmem_slot + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rank = (int)cluster_rank();               // 0 (leader) or 1
  const int pair0 = blockIdx.x >> 1, npair_ctas = gridDim.x >> 1;
  const int npairs = (sch.nunits + 1) >> 1;
  const int nseg = op.split ? 3 : 1;
  const int nk = op.kchunks * nseg;
  constexpr uint32_t kTmemCols = 2 * BN;

  if (threadIdx.x == 0) {
    *s_failed = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 2 * kEpiWarps);
    }
    mbar_init(drain, 1);
    fence_barrier_init();
  }
  if (warp == 1) tmem_alloc_pair(tmem_slot, kTmemCols);
  tc_fence_before();
  __syncthreads();
  cluster_sync();   // the peer's barriers exist before anything signals them
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  bool failed = false;
  uint32_t issued = 0;  // producer: loads issued

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA
    if (lane == 0) {
      prefetch_map(&mAh); prefetch_map(&mBh);
      if (op.split) { prefetch_map(&mAl); prefetch_map(&mBl); }
      const uint32_t full0 = map_to_rank(smem_u32(full), 0);
      uint32_t it = 0;
      for (int p = pair0; p < npairs && !failed; p += npair_ctas) {
        const int rb = 2 * p + rank;    // may be one past the last row block
        for (int ct = 0; ct < sch.nct && !failed; ++ct)
          for (int kc = 0; kc < nk; ++kc, ++it) {
            const int s = it % STAGES;
            const uint32_t ph = (it / STAGES) & 1;
            if (!mbar_wait(&empty[s], ph ^ 1, kWaitLimit, true)) { failed = true; break; }
            unsigned char *sa = stages + (size_t)s * L::kStage;
            unsigned char *sb = sa + L::kA;
            const int g = kc / op.kchunks, c = kc - g * op.kchunks;
            if (rank == 0) mbar_expect_tx(&full[s], 2 * L::kStage);
            // split order: hi.lo, lo.hi, then hi.hi (small terms first)
            const bool alo = op.split && g == 1, blo = op.split && g == 0;
            const int kx = c * KCH;
            const uint32_t fb = full0 + (uint32_t)(s * sizeof(uint64_t));
            tma_load_2d_peerbar(sa, alo ? &mAl : &mAh, kx, rb * BM, fb);
            tma_load_2d_peerbar(sb, blo ? &mBl : &mBh, kx, ct * BN + rank * (BN / 2), fb);
          }
      }
      issued = it;
      if (failed) {
        atomicExch(err, 1);
        *s_failed = 1;
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA
    if (lane == 0 && rank == 0) {
      const uint32_t idesc = idesc_bf16(2 * BM, BN);
      uint32_t it = 0, t = 0;
      for (int p = pair0; p < npairs && !failed; p += npair_ctas)
        for (int ct = 0; ct < sch.nct && !failed; ++ct, ++t) {
          const int b = t & 1;
          const uint32_t aph = (t >> 1) & 1;
          if (!mbar_wait(&acc_empty[b], aph ^ 1, kWaitLimit, true)) { failed = true; break; }
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
              umma_bf16_pair(dt, sw128_desc(sa + k * 32), sw128_desc(sb + k * 32), idesc,
                             (kc > 0 || k > 0) ? 1u : 0u);
            umma_commit_pair(&empty[s], (uint16_t)0x3);
          }
          if (failed) break;
          umma_commit_pair(&acc_full[b], (uint16_t)0x3);
        }
      if (failed) {
        atomicExch(err, 2);
        *s_failed = 1;
      }
      // the drain barriers of both CTAs complete once every MMA above has
      umma_commit_pair(drain, (uint16_t)0x3);
    }
  } else {
    // ----------------------------------------------------------- epilogue
    const int e = warp - 2;
    const int et = threadIdx.x - 64;
    const int quarter = warp & 3;
    const int half = e >> 2;
    const int r = quarter * 32 + lane;
    const uint32_t ae0 = map_to_rank(smem_u32(acc_empty), 0);
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
          epi_tile_columns<BN>(epi, escratch, rb, ct, r, half, trow, ts);
          epi.tile_end(escratch, rb, ct, r, half, ts);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive_cluster(ae0 + (uint32_t)(b * sizeof(uint64_t)));
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
  // every MMA of the pair has completed before either CTA goes on (waited for
  // only once this CTA's roles are done: the peer's MMA warp has no loop)
  if (warp == 1 && lane == 0 && !mbar_wait(drain, 0)) {
    atomicExch(err, 4);
    *s_failed = 1;
  }
  cluster_sync();   // from here on neither CTA issues a load
  if (warp == 0 && lane == 0 && rank == 0 && (*s_failed || *(volatile int *)err)) {
    for (uint32_t j = (issued > STAGES ? issued - STAGES : 0); j < issued; ++j)
      mbar_wait(&full[j % STAGES], (j / STAGES) & 1);
  }
  __syncthreads();
  cluster_sync();   // neither CTA leaves while the other may still be waiting on it
  tc_fence_after();
  if (warp == 1) {
    __syncwarp();
    tmem_dealloc_pair(tmem, kTmemCols);
  }
}

}  // namespace tc
}  // namespace rkr
