// common.cuh -- shared definitions of the GB300 reverse k-ranks library.
//
// Score arithmetic.  The canonical score s(u,x) is the left-to-right FP64 sum
// of the exact products (double)u[k]*(double)x[k] (the library's reading of
// Def. 1, which fixes no precision).  Bulk work computes cheaper screened
// scores s_hat together with a rigorous bound b such that
// |s_hat - s(u,x)| <= b; a decision is taken from the screen when the bound
// settles it and from canonical FP64 otherwise.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rkr.h"

namespace rkr {

// Device memory of the library comes from one stream-ordered pool per device
// that keeps what is freed (its release threshold is unlimited), so index
// builds and query batches reuse the same blocks instead of mapping and
// unmapping tens of GB each time.  rkr_release_cached_memory trims it.
cudaMemPool_t lib_pool();

// Count of device allocations the library has requested (rkr_device_allocations).
void note_alloc();

template <class T>
inline cudaError_t pool_malloc_async(T **p, size_t bytes, cudaStream_t st) {
  note_alloc();
  return cudaMallocFromPoolAsync((void **)p, bytes, lib_pool(), st);
}


constexpr int kMaxD = 256;          // largest supported dimension
constexpr int kMaxLevels = 32;      // rank levels 2^L used by the candidate filter
constexpr int kMaxK = 4096;         // largest k per query

// ------------------------------------------------------------ error state

void set_error(const char *fmt, ...);
rkr_status fail(rkr_status st, const char *fmt, ...);
rkr_status cuda_fail(cudaError_t e, const char *what);

// Count of kernels this library has launched (reported by rkr_kernel_launches).
void note_launch();

// RKR_EUNSUPPORTED unless the current device is sm_103 (GB300).
rkr_status check_device();

// The process-wide tuning (rkr_tuning_set / rkr_autotune), read at launch time.
rkr_tuning tuning();

// Per-kernel device-time accounting, on while rkr_profile_start is in effect:
// CUDA events recorded on the launching stream around a launch.  `work` is the
// launch's algorithmic work (flops of a screen; 0 when not stated).
int prof_begin(const char *name, cudaStream_t st);
void prof_end(int slot, cudaStream_t st, double work);
struct ProfScope {
  int slot;
  cudaStream_t st;
  double work;
  ProfScope(const char *name, cudaStream_t s, double w = 0.0)
      : slot(prof_begin(name, s)), st(s), work(w) {}
  ~ProfScope() { prof_end(slot, st, work); }
};

#define RKR_CUDA(expr)                                            \
  do {                                                            \
    cudaError_t _e = (expr);                                      \
    if (_e != cudaSuccess) return ::rkr::cuda_fail(_e, #expr);    \
  } while (0)

#define RKR_TRY(expr)                                             \
  do {                                                            \
    rkr_status _s = (expr);                                       \
    if (_s != RKR_OK) return _s;                                  \
  } while (0)

// ------------------------------------------------------- canonical scores

// s(a, b): left-to-right FP64 sum of exact float products.
__device__ __forceinline__ double canon_dot(const float *__restrict__ a,
                                            const float *__restrict__ b, int d) {
  double acc = 0.0;
  for (int k = 0; k < d; ++k) acc = __dadd_rn(acc, __dmul_rn((double)a[k], (double)b[k]));
  return acc;
}

// Out-of-line copy for rarely taken paths inside unrolled loops.
static __device__ __noinline__ double canon_dot_slow(const float *__restrict__ a,
                                                     const float *__restrict__ b, int d) {
  return canon_dot(a, b, d);
}

// Interval [lo, hi] that holds the canonical score s(a, b).  A compensated FP32
// dot product (Ogita, Rump and Oishi's Dot2: each product split exactly by an
// FMA, each addition by an error-free two-sum, the low parts summed apart)
// satisfies |(p + s) - a.b| <= gamma_d^2 sum|a_k b_k| (gamma_d = d u / (1 - d u),
// u = 2^-24); the final p + s is formed in FP64 (error <= 2^-53 |p + s|) and the
// canonical sum differs from a.b by at most gamma'_d sum|a_k b_k| with the FP64
// unit 2^-53.  Intrinsics keep the compiler from fusing or reordering the steps.
// A tiny absolute term covers products in the subnormal range.
__device__ __forceinline__ void dot2_interval(const float *__restrict__ a,
                                              const float *__restrict__ b, int d, double &lo,
                                              double &hi) {
  float p = 0.0f, s = 0.0f, asum = 0.0f;
  for (int k = 0; k < d; ++k) {
    const float x = a[k], y = b[k];
    const float h = __fmul_rn(x, y);
    const float r = __fmaf_rn(x, y, -h);
    const float t = __fadd_rn(p, h);
    const float z = __fsub_rn(t, p);
    const float e = __fadd_rn(__fsub_rn(p, __fsub_rn(t, z)), __fsub_rn(h, z));
    p = t;
    s = __fadd_rn(s, __fadd_rn(e, r));
    asum = __fadd_ru(asum, fabsf(h));
  }
  const double res = (double)p + (double)s;
  const double g = (double)d * 0x1p-24;
  const double gam = g / (1.0 - g);
  const double gc = (double)d * 0x1p-53 / (1.0 - (double)d * 0x1p-53);
  const double E = ((gam * gam + gc) * (double)asum * (1.0 + 0x1p-20) + fabs(res) * 0x1p-52 +
                    (double)d * 0x1p-140) * (1.0 + 0x1p-20);
  lo = res - E;
  hi = res + E;
}

// Threshold t_{j+1} (0-based i = j): f_min + i * delta, delta = (f_max - f_min) / (tau - 1),
// each operation rounded to double in that order (Section 4.2, step 2).
__device__ __forceinline__ double thr_at(double fmin, double delta, int i) {
  return __dadd_rn(fmin, __dmul_rn((double)i, delta));
}

// j(theta) = #{i in [0, tau) : t_i <= theta}: the 1-based index of the largest
// threshold not above theta (0 when theta < t_1), Section 4.3 step 1.
__device__ __forceinline__ int exact_j(double theta, double fmin, double delta, int tau) {
  int g;
  if (delta > 0.0) {
    double x = (theta - fmin) / delta;
    g = x < 0.0 ? 0 : (x >= (double)tau ? tau : (int)floor(x) + 1);
  } else {
    g = theta >= fmin ? tau : 0;
  }
  while (g < tau && thr_at(fmin, delta, g) <= theta) ++g;
  while (g > 0 && thr_at(fmin, delta, g - 1) > theta) --g;
  return g;
}

// Step-3 estimate (Section 4.3): linear in u.q between (t_j, r_up) and (t_{j+1}, r_low).
__device__ __forceinline__ double interp_est(double theta, int j, uint32_t nlo, uint32_t nup,
                                             double fm, double dl, int tau, uint32_t s) {
  double r_up = __dadd_rn(1.0, __ddiv_rn((double)nup, (double)s));
  double r_low = __dadd_rn(1.0, __ddiv_rn((double)nlo, (double)s));
  if (j >= 1 && j <= tau - 1) {
    double tj = thr_at(fm, dl, j - 1);
    double tj1 = thr_at(fm, dl, j);
    double frac = __ddiv_rn(__dsub_rn(theta, tj), __dsub_rn(tj1, tj));
    return __dsub_rn(r_up, __dmul_rn(__dsub_rn(r_up, r_low), frac));
  }
  return r_up;
}

// c(s) = #{i in [0, tau) : t_i < s}: the number of thresholds a score exceeds
// (Alg. 1 counts p in column j when s(u,p) > t_j).
__device__ __forceinline__ int exact_c(double s, double fmin, double delta, int tau) {
  int g;
  if (delta > 0.0) {
    double x = (s - fmin) / delta;
    g = x < 0.0 ? 0 : (x >= (double)tau ? tau : (int)floor(x) + 1);
  } else {
    g = s > fmin ? tau : 0;
  }
  while (g < tau && thr_at(fmin, delta, g) < s) ++g;
  while (g > 0 && thr_at(fmin, delta, g - 1) >= s) --g;
  return g;
}

// Per-user data for fast FP32 bin estimates.  For a value x the ideal bin
// coordinate is v = (x - f_min) / delta; t_i <= x iff i <= v.  v is computed
// in FP32 as (x - fmin32) * invd32 with an error of at most err bins (see
// make_binfp), so every integer outside [v - err, v + err] is decided.
struct BinFP {
  float fmin32;
  float invd32;   // 1/delta, or -1 when delta == 0 (degenerate grid)
  float err;      // error bound of v in bins; > 1e6 means "never decide by FP32"
  float pad;
};

// Upper bound of the bin coordinate of x (non-decreasing in x where it is not NaN).
__device__ __forceinline__ float bin_vhi(const BinFP &b, float x) {
  return __fadd_ru(__fmul_ru(__fsub_ru(x, b.fmin32), b.invd32), b.err);
}

// FP32 bin coordinate lower/upper bounds for x in [xlo, xhi].
__device__ __forceinline__ void bin_coord(const BinFP &b, float xlo, float xhi, float &vlo,
                                          float &vhi) {
  vlo = __fsub_rd(__fmul_rd(__fsub_rd(xlo, b.fmin32), b.invd32), b.err);
  vhi = bin_vhi(b, xhi);
}

// Lower end: ceil(v) clamped into [0, tau] (a lower bound of both c and j).
__device__ __forceinline__ int bin_lo(float v, int tau) {
  if (!(v > 0.0f)) return 0;            // also catches NaN
  if (v >= (float)tau) return tau;
  return (int)ceilf(v);
}

// Upper end: floor(v) + 1 clamped into [0, tau] (an upper bound of both c and j).
__device__ __forceinline__ int bin_hi(float v, int tau) {
  if (!(v >= 0.0f)) return v == v ? 0 : tau;
  if (v >= (float)tau) return tau;
  return (int)floorf(v) + 1;
}

// Rigorous interval [jlo, jhi] containing j(x) = #{t_i <= x} and c(x) = #{t_i < x}
// for every x in [xlo, xhi].  jlo == jhi means both are decided and equal.
// fmin is the FP64 grid origin, used only when delta == 0.
__device__ __forceinline__ void bin_interval(const BinFP &b, double fmin, int tau, float xlo,
                                             float xhi, int &jlo, int &jhi) {
  if (b.invd32 < 0.0f) {  // delta == 0: all thresholds equal f_min
    jlo = ((double)xlo > fmin) ? tau : 0;
    jhi = ((double)xhi >= fmin) ? tau : 0;
    return;
  }
  if (b.err > 1e6f) { jlo = 0; jhi = tau; return; }
  float vlo, vhi;
  bin_coord(b, xlo, xhi, vlo, vhi);
  jlo = bin_lo(vlo, tau);
  jhi = bin_hi(vhi, tau);
}

// FP32 screen bound: |fma-chain(u,x) - s(u,x)| <= cfac * |u| * |x| with
// cfac = ((d + 4) 2^-24 + d 2^-53 + 2^-40)(1 + 2^-20); nu, nx are FP32 upper
// bounds of the Euclidean norms.  The FMA chain rounds once per step, each
// partial sum is at most sum_k |u_k x_k| <= |u||x| (Cauchy-Schwarz); the extra
// terms cover the canonical sum's own rounding and the rounding of s_hat -+ b.
__host__ __device__ __forceinline__ float screen_cfac(int d) {
  double c = ((double)(d + 4) * 0x1p-24 + (double)d * 0x1p-53 + 0x1p-40) * (1.0 + 0x1p-20);
  return (float)c * (1.0f + 0x1p-20f);
}

__device__ __forceinline__ float screen_bound(float cfac, float nu, float nx) {
  return __fadd_ru(__fmul_ru(__fmul_ru(cfac, nu), nx), 1e-30f);
}

// Per-query user subsets as bitmaps: word q * words + u / 32, bit u % 32.  A null
// bitmap means every user belongs to every query.
__device__ __forceinline__ bool in_subset(const uint32_t *__restrict__ member, int64_t words,
                                          int64_t q, int64_t u) {
  return !member || ((member[q * words + (u >> 5)] >> (u & 31)) & 1u);
}

// Level boundaries: level L holds counts N <= B_L = scale * (2^L - 1).
__host__ __device__ __forceinline__ uint64_t level_bound(int L, uint32_t scale) {
  return (uint64_t)scale * (((uint64_t)1 << L) - 1);
}

// Float with the given bit pattern (host and device).
__host__ __device__ __forceinline__ float u32_float(uint32_t b) {
  union {
    uint32_t u;
    float f;
  } x;
  x.u = b;
  return x.f;
}

// ------------------------------------------------------- host helpers

// A stream-ordered temporary from the library pool, freed when it goes out of scope.
struct DevBuf {
  void *p = nullptr;
  cudaStream_t st = nullptr;
  ~DevBuf() {
    if (p) cudaFreeAsync(p, st);
  }
};

template <class T>
inline rkr_status tmp_alloc(DevBuf &b, T **out, size_t count, cudaStream_t st) {
  if (count == 0) count = 1;
  cudaError_t e = pool_malloc_async(&b.p, count * sizeof(T), st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return fail(RKR_ENOMEM, "device allocation of %zu bytes failed", count * sizeof(T));
  }
  b.st = st;
  *out = (T *)b.p;
  return RKR_OK;
}

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaStream_t st;
  explicit Timer(cudaStream_t s) : st(s) {
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, st);
  }
  double stop() {
    cudaEventRecord(b, st);
    cudaEventSynchronize(b);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, a, b);
    return ms;
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

// Order-preserving key of a non-negative double.
__device__ __forceinline__ uint64_t dkey(double x) { return (uint64_t)__double_as_longlong(x); }

}  // namespace rkr
