// tc_screen.cuh -- persistent tcgen05 screen kernel with a pluggable epilogue.
//
// Work is a list of units; a unit is a rectangle of tiles [rb0, rb1) x [ct0, ct1)
// (row blocks of 128 users, column tiles of BN items or queries), walked
// row-major.  Row-owned units (one row block, all columns) keep per-user
// epilogue state in the CTA; column-owned units (one column tile, a range of
// row blocks) keep per-column state.
//
// Epi must provide (all called by the 256 epilogue threads, const members):
//   struct Thread;                                    per-thread state
//   static constexpr size_t kSmem;                    bytes of epilogue scratch
//   void unit_begin(char *S, const Unit &u, int et, Thread &)   et = 0..255
//   void tile_begin(char *S, int rb, int ct, int r, int h, Thread &)
//   void chunk(char *S, int rb, int ct, int r, int col, uint32_t tm, const float (&v)[32], Thread &)
//   void tile_end(char *S, int rb, int ct, int r, int h, Thread &)
//   void unit_end(char *S, const Unit &u, int et, Thread &)
// r is the accumulator row (0..127), h the column half, col the first of the
// 32 columns of the chunk within the tile.  Named barrier 1 (256 threads) is
// available to unit_begin/unit_end and tile_begin/tile_end as tc::epi_sync().
#pragma once

#include "tc.cuh"

namespace rkr {
namespace tc {

struct Unit {
  int rb0, rb1, ct0, ct1;
};

// How units are formed: ROW = one row block each; COL = one column tile and
// one of `parts` slices of the row blocks.
struct Schedule {
  int mode;       // 0 ROW, 1 COL
  int nrb, nct;   // row blocks, column tiles
  int parts;      // COL: row-block slices per column tile
  int nunits;
};

__device__ __forceinline__ Unit unit_of(const Schedule &s, int i) {
  Unit u;
  if (s.mode == 0) {
    u.rb0 = i; u.rb1 = i + 1; u.ct0 = 0; u.ct1 = s.nct;
  } else {
    int ct = i / s.parts, part = i - ct * s.parts;
    u.ct0 = ct; u.ct1 = ct + 1;
    u.rb0 = (int)((int64_t)s.nrb * part / s.parts);
    u.rb1 = (int)((int64_t)s.nrb * (part + 1) / s.parts);
  }
  return u;
}

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

// Barrier of the 256 epilogue threads that also ORs a predicate over them, so
// that every epilogue warp takes the same decision after a bounded wait (a
// warp that gave up and one that did not would otherwise disagree on the
// number of barriers still to come).
__device__ __forceinline__ bool epi_vote_any(bool p) {
  uint32_t r;
  asm volatile(
      "{\n .reg .pred a, b;\n setp.ne.u32 a, %1, 0;\n"
      " barrier.red.or.pred b, 1, 256, a;\n selp.u32 %0, 1, 0, b;\n}\n"
      : "=r"(r)
      : "r"((uint32_t)p)
      : "memory");
  return r != 0;
}

// This thread's half row of an accumulator tile (TMEM row address trow): 64
// columns per TMEM load (one wait), handed to the epilogue as chunks of 32.
template <int BN, class Epi>
__device__ __forceinline__ void epi_tile_columns(const Epi &epi, char *S, int rb, int ct, int r,
                                                 int half, uint32_t trow,
                                                 typename Epi::Thread &ts) {
#pragma unroll 1
  for (int cc = 0; cc < BN / 64; cc += 2) {
    const int col = half * (BN / 2) + cc * 32;
    float v[64];
    tmem_ld64(trow + col, v);
    epi.chunk(S, rb, ct, r, col, trow + (uint32_t)col,
              *reinterpret_cast<const float(*)[32]>(v), ts);
    epi.chunk(S, rb, ct, r, col + 32, trow + (uint32_t)(col + 32),
              *reinterpret_cast<const float(*)[32]>(v + 32), ts);
  }
}

template <int BN>
struct Layout {
  static_assert(BN == 128 || BN == 256, "column tiles of 128 or 256");
  static constexpr uint32_t kA = BM * KCH * 2;      // 16 KB
  static constexpr uint32_t kB = BN * KCH * 2;
  static constexpr uint32_t kStage = kA + kB;
};

template <int BN, int STAGES, class Epi>
__global__ void __launch_bounds__(kThreads, 1)
    k_screen(const __grid_constant__ CUtensorMap mAh, const __grid_constant__ CUtensorMap mAl,
             const __grid_constant__ CUtensorMap mBh, const __grid_constant__ CUtensorMap mBl,
             Operands op, Schedule sch, Epi epi, int *err) {
  using L = Layout<BN>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte alignment for the swizzled tiles
  unsigned char *base = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *stages = base;
  uint64_t *full = (uint64_t *)(stages + (size_t)STAGES * L::kStage);
  uint64_t *empty = full + STAGES;
  uint64_t *acc_full = empty + STAGES;
  uint64_t *acc_empty = acc_full + 2;
  uint64_t *drain = acc_empty + 2;
  uint32_t *tmem_slot = (uint32_t *)(drain + 1);
  char *escratch = (char *)(tmem_slot + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nseg = op.split ? 3 : 1;
  const int nk = op.kchunks * nseg;
  constexpr uint32_t kTmemCols = 2 * BN;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
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
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  bool failed = false;

  if (warp == 0) {
    // ---------------------------------------------------------------- TMA
    if (lane == 0) {
      prefetch_map(&mAh); prefetch_map(&mBh);
      if (op.split) { prefetch_map(&mAl); prefetch_map(&mBl); }
      uint32_t it = 0;
      for (int ui = blockIdx.x; ui < sch.nunits && !failed; ui += gridDim.x) {
        Unit u = unit_of(sch, ui);
        for (int rb = u.rb0; rb < u.rb1 && !failed; ++rb)
          for (int ct = u.ct0; ct < u.ct1 && !failed; ++ct)
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
              const int kx = c * (op.fp8 ? 2 * KCH : KCH);  // elements of 128 bytes
              tma_load_2d(sa, alo ? &mAl : &mAh, kx, rb * BM, &full[s]);
              tma_load_2d(sb, blo ? &mBl : &mBh, kx, ct * BN, &full[s]);
            }
      }
      if (failed) {
        atomicExch(err, 1);
        // let every load already issued land before the CTA can exit
        for (uint32_t j = (it > STAGES ? it - STAGES : 0); j < it; ++j)
          mbar_wait(&full[j % STAGES], (j / STAGES) & 1);
      }
    }
  } else if (warp == 1) {
    // ---------------------------------------------------------------- MMA
    if (lane == 0) {
      const uint32_t idesc = op.fp8 ? idesc_e4m3(BM, BN) : idesc_bf16(BM, BN);
      uint32_t it = 0, t = 0;
      for (int ui = blockIdx.x; ui < sch.nunits && !failed; ui += gridDim.x) {
        Unit u = unit_of(sch, ui);
        for (int rb = u.rb0; rb < u.rb1 && !failed; ++rb)
          for (int ct = u.ct0; ct < u.ct1 && !failed; ++ct, ++t) {
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
              for (int k = 0; k < steps; ++k) {
                if (op.fp8)
                  umma_e4m3(dt, sw128_desc(sa + k * 32), sw128_desc(sb + k * 32), idesc,
                            (kc > 0 || k > 0) ? 1u : 0u);
                else
                  umma_bf16(dt, sw128_desc(sa + k * 32), sw128_desc(sb + k * 32), idesc,
                            (kc > 0 || k > 0) ? 1u : 0u);
              }
              umma_commit(&empty[s]);
            }
            if (failed) break;
            umma_commit(&acc_full[b]);
          }
      }
      if (failed) atomicExch(err, 2);
      // all MMAs issued by this thread complete before the CTA releases TMEM
      umma_commit(drain);
      mbar_wait(drain, 0);
    }
  } else {
    // ----------------------------------------------------------- epilogue
    const int e = warp - 2;                 // 0..7
    const int et = threadIdx.x - 64;        // 0..255
    const int quarter = warp & 3;
    const int half = e >> 2;
    const int r = quarter * 32 + lane;      // accumulator row (user within the block)
    uint32_t t = 0;
    typename Epi::Thread ts;
    for (int ui = blockIdx.x; ui < sch.nunits && !failed; ui += gridDim.x) {
      Unit u = unit_of(sch, ui);
      epi.unit_begin(escratch, u, et, ts);
      epi_sync();
      for (int rb = u.rb0; rb < u.rb1 && !failed; ++rb)
        for (int ct = u.ct0; ct < u.ct1 && !failed; ++ct, ++t) {
          const int b = t & 1;
          const uint32_t aph = (t >> 1) & 1;
          const bool ok = mbar_wait(&acc_full[b], aph, op.epi_wait);
          if (epi_vote_any(!ok)) { failed = true; break; }
          tc_fence_after();
          epi.tile_begin(escratch, rb, ct, r, half, ts);
          const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * BN);
          epi_tile_columns<BN>(epi, escratch, rb, ct, r, half, trow, ts);
          epi.tile_end(escratch, rb, ct, r, half, ts);
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&acc_empty[b]);
        }
      epi_sync();
      if (!failed) epi.unit_end(escratch, u, et, ts);
      epi_sync();
    }
    if (failed && lane == 0) atomicExch(err, 3);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    __syncwarp();
    tmem_dealloc(tmem, kTmemCols);
  }
}

// Stages of the single-CTA and multicast forms that fit beside the epilogue's
// scratch (at most 4).
template <int BN, class Epi>
constexpr int stages1() {
  constexpr size_t avail = 232448 - 1024 - 16 - 8 * 13 - Epi::kSmem;
  constexpr int s = (int)(avail / Layout<BN>::kStage);
  return s > 4 ? 4 : s;
}

template <int BN, int STAGES, class Epi>
constexpr size_t screen_smem_bytes() {
  return 1024 + (size_t)STAGES * Layout<BN>::kStage + 8 * (2 * STAGES + 5) + 16 + Epi::kSmem;
}

}  // namespace tc
}  // namespace rkr
