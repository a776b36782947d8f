// tc.cuh -- tcgen05 / TMEM / TMA building blocks for sm_103a and the screen
// mainloop shared by every tensor-core pass.
//
// Screen tile: D[128 x BN] = A[128 x K] . B[BN x K]^T in BF16 with FP32
// accumulation in TMEM.  A rows are users, B rows items or queries; both are
// K-major (rows of K contiguous bf16), staged by TMA with the 128-byte swizzle
// in 64-element K chunks.  A "split" product sums three segments along K,
// hi.lo + lo.hi + hi.hi (in that order), with hi = bf16(x) and lo = bf16(x - hi).
//
// Warp roles (one CTA per SM, persistent):
//   warp 0      TMA producer (one lane)
//   warp 1      TMEM allocation and MMA issue (one lane)
//   warps 2..9  epilogue: warp w reads TMEM lanes 32*(w%4) .. +31 and half
//               (w-2)/4 of the columns, so each accumulator row (user) is
//               handled by two threads
// All waits are bounded; a timeout sets an error word, drains what is in
// flight and returns.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace rkr {
namespace tc {

constexpr int BM = 128;
constexpr int KCH = 64;               // bf16 elements per K chunk (128 bytes)
constexpr int kEpiWarps = 8;
constexpr int kThreads = 32 * (2 + kEpiWarps);
constexpr uint32_t kWaitLimit = 1u << 22;   // try_wait rounds before giving up

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Wait until the phase of the given parity has completed; false after `limit`
// unsuccessful try_wait rounds (limit 0 gives up at once).  With `backoff`,
// rounds after the first 32 also sleep briefly, so that a warp waiting long
// (a producer waiting for a slow consumer) leaves its scheduler's issue slots
// to the warps doing work.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          uint32_t limit = kWaitLimit, bool backoff = false) {
  const uint32_t addr = smem_u32(bar);
  for (uint32_t i = 0; i < limit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    if (ok) return true;
    if (backoff && i >= 32) __nanosleep(128);
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void prefetch_map(const CUtensorMap *map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);       // start address
  d |= (uint64_t)1 << 16;                         // leading byte offset (unused here)
  d |= (uint64_t)(1024 >> 4) << 32;               // stride byte offset
  d |= (uint64_t)1 << 46;                         // descriptor version
  d |= (uint64_t)2 << 61;                         // 128-byte swizzle
  return d;
}

// Instruction descriptor: E4M3 x E4M3 -> FP32 (kind::f8f6f4), both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_e4m3(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_e4m3(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// Instruction descriptor: BF16 x BF16 -> FP32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                          uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(dst)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// 64 consecutive FP32 columns of this thread's TMEM lane (one load, one wait).
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float (&v)[64]) {
  uint32_t r[64];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {"
      "%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31, "
      "%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, "
      "%48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63"
      "}, [%64];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
        "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
        "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]),
        "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
        "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
}

// One accumulator column of the warp's 32 lanes (warp-convergent).
__device__ __forceinline__ float tmem_ld1(uint32_t taddr) {
  uint32_t r;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r) : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  return __uint_as_float(r);
}

// Four accumulator columns of the warp's 32 lanes, loaded together (warp-convergent).
__device__ __forceinline__ void tmem_ld1x4(uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                           float (&x)[4]) {
  uint32_t r0, r1, r2, r3;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r0) : "r"(a0));
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r1) : "r"(a1));
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r2) : "r"(a2));
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x1.b32 {%0}, [%1];" : "=r"(r3) : "r"(a3));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  x[0] = __uint_as_float(r0);
  x[1] = __uint_as_float(r1);
  x[2] = __uint_as_float(r2);
  x[3] = __uint_as_float(r3);
}

// Operands of one screen: row maps (A) and column maps (B) for the hi and lo
// parts; ncol_rows = rows of B.  ksteps = K / 16 per segment (K padded to 16).
struct Operands {
  int64_t nrows;       // rows of A (users)
  int64_t ncols;       // rows of B (items or queries)
  int kchunks;         // 128-byte K chunks per segment
  int ksteps;          // MMA steps per segment (32 bytes of K each)
  int split;           // 0: one segment hi.hi; 1: three segments hi.lo, lo.hi, hi.hi
  int fp8 = 0;         // 1: E4M3 operands (kind::f8f6f4, 128 elements per chunk)
  uint32_t epi_wait = kWaitLimit;  // try_wait rounds of the epilogue's accumulator wait
};

// Per-row bound terms (FP32 upper bounds), see screen_bound_tc.
struct RowBound {
  float a0;  // ||x - xhi - xlo||   (single mode: ||x - xhi||)
  float a1;  // ||xhi + xlo||       (single mode: ||xhi||)
  float a2;  // ||x||
  float a3;  // ||xlo||             (single mode: 0)
  float a4;  // ||xhi||
};

// Accumulation factors.  Model: adding a product t to the FP32 accumulator D
// in the tensor core errs by at most 2^-23 (|D| + |t|) (twice the unit
// roundoff, so truncating adders are covered).  The split product accumulates
// its 2 Kp small terms (hi.lo, lo.hi) first and the Kp terms hi.hi last, so
//   |err| <= 2^-22 (3 Kp L + (Kp + 1) H),  L = sum |lo terms|, H = sum |hi.hi terms|
// (again a factor 2 of margin); single products: 2^-22 (Kp + 1) H.
struct Gacc {
  float h;  // factor of H <= ||u_hi|| ||x_hi||
  float l;  // factor of L <= ||u_hi|| ||x_lo|| + ||u_lo|| ||x_hi||
};

// Bound on |s_hat - s(u,x)| for a user row ru and the maxima rt of the
// item-side terms over a column tile.  The representation error is
// ||u - u~|| ||x|| + ||u~|| ||x - x~|| (+ ||u_lo|| ||x_lo|| for the dropped
// lo.lo term), by Cauchy-Schwarz; gcan = d 2^-52 covers the canonical sum's
// own rounding; a tiny absolute term covers flushed subnormals.
__device__ __forceinline__ float screen_bound_tc(const RowBound &ru, const RowBound &rt,
                                                 const Gacc &g, float gcan) {
  float b = __fmul_ru(ru.a0, rt.a2);
  b = __fadd_ru(b, __fmul_ru(ru.a1, rt.a0));
  b = __fadd_ru(b, __fmul_ru(ru.a3, rt.a3));
  b = __fadd_ru(b, __fmul_ru(g.h, __fmul_ru(ru.a4, rt.a4)));
  b = __fadd_ru(b, __fmul_ru(g.l, __fadd_ru(__fmul_ru(ru.a4, rt.a3), __fmul_ru(ru.a3, rt.a4))));
  b = __fadd_ru(b, __fmul_ru(gcan, __fmul_ru(ru.a2, rt.a2)));
  b = __fadd_ru(b, __fmul_ru(0x1p-110f, __fadd_ru(ru.a2, rt.a2)));
  return __fadd_ru(b, 1e-36f);
}

}  // namespace tc
}  // namespace rkr
