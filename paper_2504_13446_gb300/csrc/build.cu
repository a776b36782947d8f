// build.cu -- pre-processing on the GPU (Alg. 1) and the exact count table.
//
// Steps, each a kernel on the caller's stream:
//   norms of P (FP64, canonical) and sort by (descending norm, index)   Alg. 1, norm/sort
//   buckets and sampled rows                                           Alg. 1, partition/sample
//   f_min / f_max per user (exact scan or Cauchy-Schwarz bound)        Section 4.2, step 2
//   rank-table numerators N from the sampled rows                      Alg. 1 step 3, Eq. 1
//   level tables JU / JL that map a bin to the rank level it implies   (candidate filter)
//   exact count table XLO / XHI bounding #{p : s(u,p) > t_j}           (exact path)
//   deep count grid DLO / DHI below the tail lists (exact_table = 2)   (exact path)
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "index.cuh"
#include "sort.cuh"
#include "simt.cuh"

namespace rkr {

// ----------------------------------------------------------------- norms

__global__ void k_row_norms(const float *__restrict__ X, int64_t rows, int d,
                            double *__restrict__ nrm64, float *__restrict__ nrm32) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= rows) return;
  const float *x = X + i * d;
  double ss = canon_dot(x, x, d);
  double nv = sqrt(ss);
  if (nrm64) nrm64[i] = nv;
  // upper bound of the exact norm: the canonical sum is within d 2^-53 (relative)
  if (nrm32) nrm32[i] = __double2float_ru(nv * (1.0 + 0x1p-40) + 1e-300);
}

rkr_status row_norms(const float *X, int64_t rows, int d, double *nrm64, float *nrm32,
                     cudaStream_t st) {
  if (rows <= 0) return RKR_OK;
  int bs = 128;
  {
    const int prof_slot = prof_begin("k_row_norms", st);
    k_row_norms<<<(unsigned)((rows + bs - 1) / bs), bs, 0, st>>>(X, rows, d, nrm64, nrm32);
    prof_end(prof_slot, st, 0.0);
    note_launch();
  }
  RKR_CUDA(cudaGetLastError());
  return RKR_OK;
}

__global__ void k_max_float(const float *__restrict__ x, int64_t count, unsigned *out) {
  float m = 0.0f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, x[i]);
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));  // m >= 0
}

rkr_status max_float(const float *x, int64_t count, float *out_host, cudaStream_t st) {
  unsigned *dv;
  RKR_CUDA(pool_malloc_async(&dv, sizeof(unsigned), st));
  RKR_CUDA(cudaMemsetAsync(dv, 0, sizeof(unsigned), st));
  k_max_float<<<256, 256, 0, st>>>(x, count, dv); note_launch();
  unsigned h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, dv, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(dv, st);
  if (e != cudaSuccess) return cuda_fail(e, "max_float");
  memcpy(out_host, &h, sizeof(float));
  return RKR_OK;
}

__global__ void k_all_finite(const float *__restrict__ x, int64_t count, int *bad) {
  int b = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    b |= !isfinite(x[i]);
  if (__any_sync(0xffffffffu, b) && (threadIdx.x & 31) == 0) atomicOr(bad, 1);
}

rkr_status all_finite(const float *x, int64_t count, int *ok_host, cudaStream_t st) {
  int *dv;
  RKR_CUDA(pool_malloc_async(&dv, sizeof(int), st));
  RKR_CUDA(cudaMemsetAsync(dv, 0, sizeof(int), st));
  k_all_finite<<<512, 256, 0, st>>>(x, count, dv); note_launch();
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, dv, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(dv, st);
  if (e != cudaSuccess) return cuda_fail(e, "all_finite");
  *ok_host = h == 0;
  return RKR_OK;
}

// ------------------------------------------------------------------ sort

// Sorts of (key, val) records use the tiled bitonic sort of sort.cuh, ascending
// by (key, val).  Padding entries carry key = UINT64_MAX, val = INT32_MAX.

// FNV-1a over the 32-bit patterns of a row.
__device__ __forceinline__ uint64_t row_hash(const float *x, int d) {
  uint64_t h = 1469598103934665603ull;
  for (int k = 0; k < d; ++k) {
    h ^= (uint64_t)__float_as_uint(x[k]);
    h *= 1099511628211ull;
  }
  return h == ~0ull ? h - 1 : h;  // ~0 marks padding
}

__global__ void k_row_hashes(const float *__restrict__ X, int64_t rows, int d, int64_t Np2,
                             uint64_t *__restrict__ keys, int32_t *__restrict__ vals) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= Np2) return;
  keys[i] = i < rows ? row_hash(X + i * d, d) : ~0ull;
  vals[i] = (int32_t)i;
}

rkr_status row_hashes(const float *X, int64_t rows, int d, int64_t Np2, uint64_t *keys,
                      int32_t *vals, cudaStream_t st) {
  k_row_hashes<<<(unsigned)((Np2 + 255) / 256), 256, 0, st>>>(X, rows, d, Np2, keys, vals);
  note_launch();
  RKR_CUDA(cudaGetLastError());
  return RKR_OK;
}

// Sorted-item position of an item row bitwise equal to each query row, or -1.
__global__ void k_query_self(int nq, const float *__restrict__ Q, int d,
                             const uint64_t *__restrict__ phk, const int32_t *__restrict__ phv,
                             int64_t phn, const float *__restrict__ Ps,
                             int32_t *__restrict__ qself) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const float *x = Q + (int64_t)q * d;
  const uint64_t h = row_hash(x, d);
  int64_t a = 0, b = phn;
  while (a < b) {
    int64_t md = (a + b) >> 1;
    if (phk[md] < h) a = md + 1; else b = md;
  }
  int32_t found = -1;
  for (; a < phn && phk[a] == h && found < 0; ++a) {
    const float *y = Ps + (int64_t)phv[a] * d;
    bool eq = true;
    for (int k = 0; k < d && eq; ++k) eq = __float_as_uint(x[k]) == __float_as_uint(y[k]);
    if (eq) found = phv[a];
  }
  qself[q] = found;
}

rkr_status query_self(const rkr_index *idx, const float *Q, int nq, int32_t *qself,
                      cudaStream_t st) {
  if (nq <= 0) return RKR_OK;
  k_query_self<<<(nq + 127) / 128, 128, 0, st>>>(nq, Q, idx->d, idx->phk, idx->phv, idx->phn,
                                                 idx->Ps, qself);
  note_launch();
  RKR_CUDA(cudaGetLastError());
  return RKR_OK;
}

rkr_status sort_pairs(uint64_t *key, int32_t *val, int64_t N_pow2, cudaStream_t st) {
  return bitonic_sort(Sort64{key, val}, N_pow2, "k_sort<64>", st);
}

// Keys for the descending-norm sort: ~bits(norm) (norms are >= +0).
__global__ void k_norm_keys(const double *__restrict__ nrm, int64_t m, int64_t N,
                            uint64_t *key, int32_t *val) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  if (i < m) {
    key[i] = ~(uint64_t)__double_as_longlong(nrm[i]);
    val[i] = (int32_t)i;
  } else {
    key[i] = ~0ull;
    val[i] = 0x7fffffff;
  }
}

// Ps[i] = P[perm[i]], pnrm_s[i] = pnrm32[perm[i]].
__global__ void k_gather_sorted(const float *__restrict__ P, const int32_t *__restrict__ perm,
                                const float *__restrict__ pn32, int64_t m, int d,
                                float *__restrict__ Ps, float *__restrict__ pnrm_s) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  int64_t src = perm[i];
  for (int k = 0; k < d; ++k) Ps[i * d + k] = P[src * d + k];
  pnrm_s[i] = pn32[src];
}

// ------------------------------------------------------------- f-bounds

// Exact f_max / f_min (canonical max/min of s(u,p) over P), one thread per user.
// The FP32 screen decides most items; an item is evaluated canonically only if
// its screened upper bound exceeds the running maximum (lower bound below the
// running minimum), so the result is the canonical extreme.
__global__ void __launch_bounds__(128) k_fbounds(const float *__restrict__ U, int64_t n,
                                                 const float *__restrict__ Ps,
                                                 const float *__restrict__ pnrm_s, int64_t m,
                                                 int d, const float *__restrict__ unrm,
                                                 double *__restrict__ fmin,
                                                 double *__restrict__ fmax) {
  extern __shared__ float smem[];
  float *Us = smem;                      // [d][128]
  float *Xs = smem + (size_t)d * 128;    // [d][32]
  const int t = threadIdx.x;
  const int64_t u0 = (int64_t)blockIdx.x * 128;
  const int64_t u = u0 + t;
  load_users_T(U, n, d, u0, Us);
  const float cfac = screen_cfac(d);
  const float nu = u < n ? unrm[u] : 0.0f;
  double mx = -INFINITY, mn = INFINITY;
  float mx_f = -INFINITY, mn_f = INFINITY;  // FP32 bounds: mx_f <= mx, mn_f >= mn
  for (int64_t x0 = 0; x0 < m; x0 += 32) {
    __syncthreads();
    load_items_T<32>(Ps, m, d, x0, Xs);
    __syncthreads();
    float acc[32];
    tile_dots<32>(Us, Xs, d, t, acc);
    if (u >= n) continue;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      int64_t p = x0 + j;
      if (p >= m) continue;
      float b = screen_bound(cfac, nu, pnrm_s[p]);
      float hi = __fadd_ru(acc[j], b), lo = __fsub_rd(acc[j], b);
      bool need_max = hi > mx_f, need_min = lo < mn_f;
      if (need_max || need_min) {
        double sc = canon_dot_slow(U + u * d, Ps + p * d, d);
        if (sc > mx) { mx = sc; mx_f = __double2float_rd(sc); }
        if (sc < mn) { mn = sc; mn_f = __double2float_ru(sc); }
      }
    }
  }
  if (u < n) { fmax[u] = mx; fmin[u] = mn; }
}

// Cauchy-Schwarz variant: f_max = ||u|| * max ||p||, f_min = -f_max.
__global__ void k_fbounds_cs(const float *__restrict__ U, int64_t n, int d, double pmax64,
                             double *fmin, double *fmax) {
  int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= n) return;
  const float *x = U + u * d;
  double nu = sqrt(canon_dot(x, x, d));
  double f = __dmul_rn(nu, pmax64);
  fmax[u] = f;
  fmin[u] = -f;
}

// delta = (f_max - f_min) / (tau - 1) and the FP32 bin parameters.
// err bounds |v32 - v| in bins for |x| <= ||u|| * R (see BinFP).
__global__ void k_binfp(int64_t n, const double *__restrict__ fmin,
                        const double *__restrict__ fmax, int tau, const float *__restrict__ unrm,
                        float R, double *__restrict__ delta_out, BinFP *__restrict__ out) {
  int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= n) return;
  double fm = fmin[u];
  double dl = __ddiv_rn(__dsub_rn(fmax[u], fm), (double)(tau - 1));
  if (delta_out) delta_out[u] = dl;
  BinFP b;
  b.fmin32 = (float)fm;
  b.pad = 0.0f;
  if (!(dl > 0.0)) {
    b.invd32 = -1.0f;
    b.err = 0.0f;
  } else {
    double xmax = (double)unrm[u] * (double)R * 1.001 + 1e-30;
    double e = (ldexp(xmax + fabs(fm), -20) + ldexp(fabs(fm), -40)) / dl + ldexp((double)tau, -40) +
               0x1p-30;
    double inv = 1.0 / dl;
    if (!(e < 1e6) || !(inv < 3e38)) {
      b.invd32 = 1.0f;
      b.err = 2e6f;
    } else {
      b.invd32 = (float)inv;
      b.err = __double2float_ru(e * (1.0 + 0x1p-10));
    }
  }
  out[u] = b;
}

rkr_status make_binfp(const rkr_index *idx, float R, BinFP *out, cudaStream_t st) {
  int bs = 256;
  k_binfp<<<(unsigned)((idx->n + bs - 1) / bs), bs, 0, st>>>(idx->n, idx->fmin, idx->fmax,
                                                              idx->tau, idx->unrm, R, nullptr,
                                                              out); note_launch();
  RKR_CUDA(cudaGetLastError());
  return RKR_OK;
}

rkr_status make_binfp_grid(const rkr_index *idx, const double *g0, const double *gmax, int G,
                           float R, double *delta_out, BinFP *out, cudaStream_t st) {
  int bs = 256;
  k_binfp<<<(unsigned)((idx->n + bs - 1) / bs), bs, 0, st>>>(idx->n, g0, gmax, G, idx->unrm, R,
                                                              delta_out, out);
  note_launch();
  RKR_CUDA(cudaGetLastError());
  return RKR_OK;
}

// ------------------------------------------------------------ rank table

// Sampled rows and their weights, bucket after bucket.
__global__ void k_gather_samples(const float *__restrict__ Ps, const float *__restrict__ pnrm_s,
                                 const int32_t *__restrict__ perm, int d,
                                 const int64_t *__restrict__ samp_sorted_pos,
                                 const uint32_t *__restrict__ samp_w, int nsamp,
                                 float *__restrict__ S, float *__restrict__ snrm,
                                 int32_t *__restrict__ items) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nsamp) return;
  int64_t p = samp_sorted_pos[i];
  for (int k = 0; k < d; ++k) S[(int64_t)i * d + k] = Ps[p * d + k];
  snrm[i] = pnrm_s[p];
  items[i] = perm[p];
}

// Warp-per-user rank-table fill (Alg. 1 step 3, Eq. 1).  For each sampled row
// the number of thresholds it exceeds, c = #{j : s(u,p) > t_j}, is decided by
// the FP32 screen when its bin interval is a single value and by canonical
// FP64 otherwise; W[c] += w.  Then N[j] = sum_{c > j} W[c].  Undecided samples
// are queued per warp and evaluated after the screen one per lane, so the
// canonical FP64 dot products run in full warps.
constexpr int kTableWarps = 8;
constexpr int kTableTile = 64;
constexpr int kTableQueue = 128;  // undecided samples queued per warp

__global__ void __launch_bounds__(kTableWarps * 32)
    k_rank_table(const float *__restrict__ U, int64_t n, int d, const float *__restrict__ unrm,
                 const float *__restrict__ S, const float *__restrict__ snrm,
                 const uint32_t *__restrict__ sw, int nsamp, const double *__restrict__ fmin,
                 const double *__restrict__ delta, const BinFP *__restrict__ binfp, int tau,
                 uint32_t *__restrict__ N) {
  extern __shared__ float smem[];
  float *Xs = smem;                                   // [d][kTableTile + 1]
  float *Uw = Xs + (size_t)d * (kTableTile + 1);      // [warps][d]
  uint32_t *W = (uint32_t *)(Uw + (size_t)kTableWarps * d);  // [warps][tau+1]
  int32_t *Qs = (int32_t *)(W + (size_t)kTableWarps * (tau + 1));  // [warps][kTableQueue]
  __shared__ int qn[kTableWarps];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t u = (int64_t)blockIdx.x * kTableWarps + warp;
  const bool active = u < n;
  uint32_t *Wu = W + (size_t)warp * (tau + 1);
  int32_t *Qw = Qs + warp * kTableQueue;
  for (int c = lane; c <= tau; c += 32) Wu[c] = 0;
  if (lane == 0) qn[warp] = 0;
  for (int k = lane; k < d; k += 32) Uw[warp * d + k] = active ? U[u * d + k] : 0.0f;
  const float cfac = screen_cfac(d);
  const float nu = active ? unrm[u] : 0.0f;
  BinFP bf;
  double fm = 0.0, dl = 0.0;
  if (active) { bf = binfp[u]; fm = fmin[u]; dl = delta[u]; }
  for (int x0 = 0; x0 < nsamp; x0 += kTableTile) {
    __syncthreads();
    for (int e = threadIdx.x; e < kTableTile * d; e += blockDim.x) {
      int j = e / d, k = e - j * d;
      int p = x0 + j;
      Xs[k * (kTableTile + 1) + j] = p < nsamp ? S[(int64_t)p * d + k] : 0.0f;
    }
    __syncthreads();
    if (!active) continue;
    float acc0 = 0.0f, acc1 = 0.0f;
    const float *uw = Uw + warp * d;
    for (int k = 0; k < d; ++k) {
      float uk = uw[k];
      acc0 = fmaf(uk, Xs[k * (kTableTile + 1) + lane], acc0);
      acc1 = fmaf(uk, Xs[k * (kTableTile + 1) + lane + 32], acc1);
    }
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      int p = x0 + lane + 32 * h;
      if (p >= nsamp) continue;
      float sh = h ? acc1 : acc0;
      float b = screen_bound(cfac, nu, snrm[p]);
      int jlo, jhi;
      bin_interval(bf, fm, tau, __fsub_rd(sh, b), __fadd_ru(sh, b), jlo, jhi);
      if (jlo == jhi) {
        atomicAdd(&Wu[jlo], sw[p]);
      } else {
        const int slot = atomicAdd(&qn[warp], 1);
        if (slot < kTableQueue) {
          Qw[slot] = p;
        } else {  // queue full: evaluate here
          double sc = canon_dot_slow(U + u * d, S + (int64_t)p * d, d);
          atomicAdd(&Wu[exact_c(sc, fm, dl, tau)], sw[p]);
        }
      }
    }
  }
  __syncwarp();
  if (!active) return;
  const int nqd = min(qn[warp], kTableQueue);
  for (int i = lane; i < nqd; i += 32) {
    const int p = Qw[i];
    double sc = canon_dot(U + u * d, S + (int64_t)p * d, d);
    atomicAdd(&Wu[exact_c(sc, fm, dl, tau)], sw[p]);
  }
  __syncwarp();
  // suffix sums: N[j] = sum_{c = j+1 .. tau} W[c]; lanes own contiguous chunks
  const int chunk = (tau + 1 + 31) / 32;
  int c0 = lane * chunk, c1 = min(tau + 1, c0 + chunk);
  uint32_t part = 0;
  for (int c = c0; c < c1; ++c) part += Wu[c];
  uint32_t incl = part;  // inclusive suffix over lanes >= lane
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t v = __shfl_down_sync(0xffffffffu, incl, o);
    if (lane + o < 32) incl += v;
  }
  uint32_t run = incl - part;  // sum over c >= c1
  for (int c = c1 - 1; c >= c0; --c) {
    // N[c - 1] = sum over c' >= c
    run += Wu[c];
    if (c >= 1) N[u * tau + (c - 1)] = run;
  }
}

// ---------------------------------------------------------- level tables

// For each user and level L (bound B_L = scale (2^L - 1)):
//   JU[L] = min{j in [0,tau] : UB(j) <= B_L},  UB(0) = top, UB(j) = hi[j-1]
//   JL[L] = min{j in [0,tau] : LB(j) <= B_L},  LB(j) = lo[j] (j < tau), LB(tau) = 0
// Both are non-increasing in L; levels >= nlev hold -1.
__global__ void k_levels(int64_t n, int tau, const uint32_t *__restrict__ hi,
                         const uint32_t *__restrict__ lo, uint32_t top, uint32_t scale, int nlev,
                         int16_t *__restrict__ JU, int16_t *__restrict__ JL) {
  int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= n) return;
  const uint32_t *h = hi + u * tau;
  const uint32_t *l = lo + u * tau;
  for (int L = 0; L < kMaxLevels; ++L) {
    int16_t ju = -1, jl = -1;
    if (L < nlev) {
      uint64_t B = level_bound(L, scale);
      // UB is non-increasing in j: binary search the first j with UB(j) <= B
      int a = 0, b = tau + 1;
      while (a < b) {
        int mid = (a + b) >> 1;
        uint64_t v = mid == 0 ? top : h[mid - 1];
        if (v <= B) b = mid; else a = mid + 1;
      }
      ju = (int16_t)a;
      a = 0; b = tau;
      while (a < b) {
        int mid = (a + b) >> 1;
        if ((uint64_t)l[mid] <= B) b = mid; else a = mid + 1;
      }
      jl = (int16_t)a;  // LB(tau) = 0 <= B always
    }
    JU[u * kMaxLevels + L] = ju;
    JL[u * kMaxLevels + L] = jl;
  }
}

// ------------------------------------------------------ exact count table

// floor column per user: the last column whose estimated count is at least
// floor_rank (0 if none).  Counts are exact-bounded only for columns >= floor.
__global__ void k_floor_cols(int64_t n, int tau, const uint32_t *__restrict__ N, uint32_t s,
                             uint64_t floor_rank, int32_t *__restrict__ fl) {
  int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= n) return;
  const uint32_t *r = N + u * tau;
  uint64_t need = floor_rank * (uint64_t)s;
  int a = 0, b = tau;  // first column with N < need
  while (a < b) {
    int mid = (a + b) >> 1;
    if ((uint64_t)r[mid] < need) b = mid; else a = mid + 1;
  }
  fl[u] = a > 0 ? a - 1 : 0;
}

// Per user: the deep grid's base (the sampled table's threshold of column
// col[u]), its top point x_0 rounded up and its base rounded down to float.
__global__ void k_ygrid(int64_t n, const double *__restrict__ fmin,
                        const double *__restrict__ delta, const int32_t *__restrict__ col,
                        const int32_t *__restrict__ xfloor, const double *__restrict__ xg0,
                        double *__restrict__ yg0, float *__restrict__ ytop,
                        float *__restrict__ ybot) {
  int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= n) return;
  // the base never lies above x_0
  const int c = col[u] < xfloor[u] ? col[u] : xfloor[u];
  const double g = thr_at(fmin[u], delta[u], c);
  yg0[u] = g;
  ytop[u] = __double2float_ru(xg0[u]);
  ybot[u] = __double2float_rd(g);
}

// Capacity of each user's tail list: 1.5 times the sampled table's estimate of
// the count above the floor threshold, plus 256, at most kListCapMax (0 when
// lists are disabled).  Lists that overflow are detected and not used.
__global__ void k_list_caps(int64_t n, int tau, const uint32_t *__restrict__ N, uint32_t s,
                            const int32_t *__restrict__ fl, int enabled, uint32_t *__restrict__ cap) {
  int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= n) return;
  if (!enabled) { cap[u] = 0; return; }
  uint64_t est = (uint64_t)N[u * tau + fl[u]] / s;
  uint64_t c = est + est / 2 + 256;
  cap[u] = (uint32_t)(c < (uint64_t)kListCapMax ? c : kListCapMax);
}

// ------------------------------------------------------------- sampling

// SplitMix64 (Steele, Lea and Flood, 2014), used only when the caller supplies
// no sample positions.
static uint64_t splitmix64(uint64_t &x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// ----------------------------------------------------------------- build

template <class T>
static rkr_status dalloc(T **p, size_t count) {
  // index arrays: from the library pool, usable on every stream once this returns
  if (count == 0) count = 1;
  cudaError_t e = pool_malloc_async(p, count * sizeof(T), (cudaStream_t)0);
  if (e == cudaSuccess) e = cudaStreamSynchronize((cudaStream_t)0);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(RKR_ENOMEM, "device allocation of %zu bytes failed", count * sizeof(T));
  }
  return RKR_OK;
}

static int levels_for(uint64_t top_count) {
  int L = 0;
  while ((((uint64_t)1 << L) - 1) < top_count) ++L;
  return L + 1;
}

rkr_status build_index(rkr_index *idx, const float *U_dev, const float *P_dev,
                       const rkr_build_params *prm, const int32_t *sample_pos_host,
                       cudaStream_t st) {
  const int64_t n = idx->n, m = idx->m;
  const int d = idx->d, tau = idx->tau, omega = idx->omega, s = idx->s;
  const int bs = 256;
  cudaEvent_t ev[7];
  for (auto &e : ev) RKR_CUDA(cudaEventCreate(&e));
  struct EvGuard {
    cudaEvent_t *e;
    ~EvGuard() {
      for (int i = 0; i < 7; ++i) cudaEventDestroy(e[i]);
    }
  } evg{ev};
  RKR_CUDA(cudaEventRecord(ev[0], st));

  // users: own copy + norm bounds
  RKR_TRY(dalloc(&idx->U, (size_t)n * d));
  RKR_CUDA(cudaMemcpyAsync(idx->U, U_dev, sizeof(float) * n * d, cudaMemcpyDeviceToDevice, st));
  RKR_TRY(dalloc(&idx->unrm, n));
  RKR_TRY(row_norms(idx->U, n, d, nullptr, idx->unrm, st));

  // items: FP64 norms, sort by (descending norm, index)
  float *pn32 = nullptr;
  RKR_TRY(dalloc(&idx->pnorm, m));
  RKR_TRY(dalloc(&pn32, m));
  RKR_TRY(row_norms(P_dev, m, d, idx->pnorm, pn32, st));
  int64_t Np2 = 1;
  while (Np2 < m) Np2 <<= 1;
  uint64_t *keys = nullptr;
  int32_t *vals = nullptr;
  RKR_TRY(dalloc(&keys, Np2));
  RKR_TRY(dalloc(&vals, Np2));
  k_norm_keys<<<(unsigned)((Np2 + bs - 1) / bs), bs, 0, st>>>(idx->pnorm, m, Np2, keys, vals); note_launch();
  RKR_TRY(sort_pairs(keys, vals, Np2, st));
  RKR_TRY(dalloc(&idx->perm, m));
  RKR_CUDA(cudaMemcpyAsync(idx->perm, vals, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice, st));
  RKR_TRY(dalloc(&idx->Ps, (size_t)m * d));
  RKR_TRY(dalloc(&idx->pnrm_s, m));
  {
    const int prof_slot = prof_begin("k_gather_sorted", st);
    k_gather_sorted<<<(unsigned)((m + 127) / 128), 128, 0, st>>>(P_dev, idx->perm, pn32, m, d,
                                                                 idx->Ps, idx->pnrm_s);
    prof_end(prof_slot, st, 0.0);
    note_launch();
  }
  RKR_CUDA(cudaGetLastError());
  RKR_TRY(max_float(idx->pnrm_s, m, &idx->pmax, st));
  RKR_TRY(tc_stage(idx->U, n, d, idx->Ut, st));
  RKR_TRY(tc_stage(idx->Ps, m, d, idx->Pt, st));
  RKR_TRY(tc_make_cat(idx->Ut, 1, st));
  RKR_TRY(tc_make_cat(idx->Pt, 2, st));
  // hash table of the sorted item rows (a query equal to an item ties with it exactly)
  idx->phn = Np2;
  RKR_TRY(dalloc(&idx->phk, Np2));
  RKR_TRY(dalloc(&idx->phv, Np2));
  RKR_TRY(row_hashes(idx->Ps, m, d, Np2, idx->phk, idx->phv, st));
  RKR_TRY(sort_pairs(idx->phk, idx->phv, Np2, st));
  cudaFreeAsync(keys, st);
  cudaFreeAsync(vals, st);
  cudaFreeAsync(pn32, st);

  RKR_CUDA(cudaEventRecord(ev[1], st));
  // buckets and samples (positions inside buckets of the sorted order)
  std::vector<int64_t> size(omega), off(omega + 1, 0);
  for (int l = 0; l < omega; ++l) size[l] = m / omega + (l < m % omega ? 1 : 0);
  for (int l = 0; l < omega; ++l) off[l + 1] = off[l] + size[l];
  std::vector<int64_t> spos;
  std::vector<uint32_t> sw;
  std::vector<int32_t> scratch;
  uint64_t rng = prm->seed;
  for (int l = 0; l < omega; ++l) {
    bool take_all = size[l] <= s;
    if (sample_pos_host) {
      const int32_t *row = sample_pos_host + (size_t)l * s;
      std::vector<int32_t> got;
      for (int i = 0; i < s; ++i)
        if (row[i] >= 0) got.push_back(row[i]);
      if (take_all) {
        if ((int64_t)got.size() != size[l])
          return fail(RKR_EINVAL, "bucket %d has %lld items: all must be listed", l,
                      (long long)size[l]);
        std::vector<int32_t> chk = got;
        std::sort(chk.begin(), chk.end());
        for (int64_t i = 0; i < size[l]; ++i)
          if (chk[i] != i) return fail(RKR_EINVAL, "bucket %d must list positions 0..%lld", l,
                                       (long long)size[l] - 1);
      } else {
        if ((int)got.size() != s)
          return fail(RKR_EINVAL, "bucket %d needs %d sample positions", l, s);
        std::vector<int32_t> chk = got;
        std::sort(chk.begin(), chk.end());
        for (int i = 0; i < s; ++i)
          if (chk[i] >= size[l] || (i > 0 && chk[i] == chk[i - 1]))
            return fail(RKR_EINVAL, "bucket %d: positions must be distinct and < %lld", l,
                        (long long)size[l]);
      }
      for (int32_t v : got) {
        spos.push_back(off[l] + v);
        sw.push_back(take_all ? (uint32_t)s : (uint32_t)size[l]);
      }
    } else if (take_all) {
      for (int64_t v = 0; v < size[l]; ++v) {
        spos.push_back(off[l] + v);
        sw.push_back((uint32_t)s);
      }
    } else {  // partial Fisher-Yates
      scratch.resize(size[l]);
      for (int64_t v = 0; v < size[l]; ++v) scratch[v] = (int32_t)v;
      for (int i = 0; i < s; ++i) {
        uint64_t r = splitmix64(rng) % (uint64_t)(size[l] - i);
        std::swap(scratch[i], scratch[i + r]);
        spos.push_back(off[l] + scratch[i]);
        sw.push_back((uint32_t)size[l]);
      }
    }
  }
  idx->nsamp = (int)spos.size();
  int64_t *spos_d = nullptr;
  RKR_TRY(dalloc(&spos_d, spos.size()));
  RKR_TRY(dalloc(&idx->sw, sw.size()));
  RKR_CUDA(cudaMemcpyAsync(spos_d, spos.data(), sizeof(int64_t) * spos.size(),
                           cudaMemcpyHostToDevice, st));
  RKR_CUDA(cudaMemcpyAsync(idx->sw, sw.data(), sizeof(uint32_t) * sw.size(),
                           cudaMemcpyHostToDevice, st));
  RKR_TRY(dalloc(&idx->S, (size_t)idx->nsamp * d));
  RKR_TRY(dalloc(&idx->snrm, idx->nsamp));
  RKR_TRY(dalloc(&idx->samp_items, idx->nsamp));
  k_gather_samples<<<(idx->nsamp + 127) / 128, 128, 0, st>>>(idx->Ps, idx->pnrm_s, idx->perm, d,
                                                             spos_d, idx->sw, idx->nsamp, idx->S,
                                                             idx->snrm, idx->samp_items); note_launch();
  RKR_CUDA(cudaGetLastError());
  // host vectors above are read by the async copies: keep them alive until done
  RKR_CUDA(cudaStreamSynchronize(st));
  cudaFreeAsync(spos_d, st);

  RKR_CUDA(cudaEventRecord(ev[2], st));
  // f_min / f_max and bins
  RKR_TRY(dalloc(&idx->fmin, n));
  RKR_TRY(dalloc(&idx->fmax, n));
  RKR_TRY(dalloc(&idx->delta, n));
  RKR_TRY(dalloc(&idx->binfp, n));
  bool fb_done = false;
  if (idx->fbounds == 0) {
    rkr_status fs = tc_fbounds(idx, idx->Ut, idx->Pt, idx->fmin, idx->fmax, st);
    if (fs == RKR_OK) fb_done = true;
    else if (fs != RKR_EINTERNAL) return fs;
    set_error("");
  }
  if (idx->fbounds == 0 && !fb_done) {
    // candidate overflow on the tensor-core path: exact scan on the CUDA cores
    size_t sm = sizeof(float) * ((size_t)d * 128 + (size_t)d * 32);
    RKR_CUDA(cudaFuncSetAttribute(k_fbounds, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
    {
      const int prof_slot = prof_begin("k_fbounds", st);
      k_fbounds<<<(unsigned)((n + 127) / 128), 128, sm, st>>>(idx->U, n, idx->Ps, idx->pnrm_s, m, d,
                                                              idx->unrm, idx->fmin, idx->fmax);
      prof_end(prof_slot, st, 0.0);
      note_launch();
    }
  } else if (idx->fbounds == 1) {
    double pmax64 = 0.0;
    // max FP64 norm: the first item of the sorted order
    int32_t first = 0;
    RKR_CUDA(cudaMemcpyAsync(&first, idx->perm, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    RKR_CUDA(cudaStreamSynchronize(st));
    RKR_CUDA(cudaMemcpyAsync(&pmax64, idx->pnorm + first, sizeof(double), cudaMemcpyDeviceToHost,
                             st));
    RKR_CUDA(cudaStreamSynchronize(st));
    k_fbounds_cs<<<(unsigned)((n + bs - 1) / bs), bs, 0, st>>>(idx->U, n, d, pmax64, idx->fmin,
                                                               idx->fmax); note_launch();
  }
  RKR_CUDA(cudaGetLastError());
  k_binfp<<<(unsigned)((n + bs - 1) / bs), bs, 0, st>>>(n, idx->fmin, idx->fmax, tau, idx->unrm,
                                                        idx->pmax, idx->delta, idx->binfp); note_launch();
  RKR_CUDA(cudaGetLastError());

  RKR_CUDA(cudaEventRecord(ev[3], st));
  // sampled rank table
  RKR_TRY(dalloc(&idx->N, (size_t)n * tau));
  bool table_done = false;
  RKR_TRY(tc_rank_table(idx, idx->Ut, st, &table_done));
  if (!table_done) {
    size_t sm = sizeof(float) * ((size_t)d * (kTableTile + 1) + (size_t)kTableWarps * d) +
                sizeof(uint32_t) * (size_t)kTableWarps * (tau + 1) +
                sizeof(int32_t) * kTableWarps * kTableQueue;
    if (sm > 227 * 1024) return fail(RKR_EINVAL, "tau too large for the table kernel");
    RKR_CUDA(cudaFuncSetAttribute(k_rank_table, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sm));
    {
      const int prof_slot = prof_begin("k_rank_table", st);
      k_rank_table<<<(unsigned)((n + kTableWarps - 1) / kTableWarps), kTableWarps * 32, sm, st>>>(
          idx->U, n, d, idx->unrm, idx->S, idx->snrm, idx->sw, idx->nsamp, idx->fmin, idx->delta,
          idx->binfp, tau, idx->N);
      prof_end(prof_slot, st, 0.0);
      note_launch();
    }
    RKR_CUDA(cudaGetLastError());
  }
  RKR_CUDA(cudaEventRecord(ev[4], st));
  idx->nlev_a = levels_for((uint64_t)m);
  RKR_TRY(dalloc(&idx->JU, (size_t)n * kMaxLevels));
  RKR_TRY(dalloc(&idx->JL, (size_t)n * kMaxLevels));
  k_levels<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(n, tau, idx->N, idx->N,
                                                        (uint32_t)(m * s), (uint32_t)s,
                                                        idx->nlev_a, idx->JU, idx->JL); note_launch();
  RKR_CUDA(cudaGetLastError());

  RKR_CUDA(cudaEventRecord(ev[5], st));
  // exact count table
  if (idx->has_exact) {
    idx->xg = kXGrid;
    RKR_TRY(dalloc(&idx->xfloor, n));
    RKR_TRY(dalloc(&idx->xg0, n));
    RKR_TRY(dalloc(&idx->xdx, n));
    RKR_TRY(dalloc(&idx->xbin, n));
    RKR_TRY(dalloc(&idx->XLO, (size_t)n * kXGrid));
    RKR_TRY(dalloc(&idx->XHI, (size_t)n * kXGrid));
    RKR_TRY(dalloc(&idx->xlcnt, n));
    RKR_TRY(dalloc(&idx->xcoff, (size_t)n * (kListG + 2)));
    RKR_TRY(dalloc(&idx->ldx, n));
    RKR_TRY(dalloc(&idx->lbin, n));
    RKR_TRY(dalloc(&idx->xbmax, n));
    RKR_TRY(dalloc(&idx->ptile3, (size_t)((m + 255) / 256)));
    RKR_TRY(dalloc(&idx->xlcap, n));
    RKR_TRY(dalloc(&idx->xloff, n + 1));
    k_floor_cols<<<(unsigned)((n + bs - 1) / bs), bs, 0, st>>>(n, tau, idx->N, (uint32_t)s,
                                                               (uint64_t)idx->floor_rank,
                                                               idx->xfloor); note_launch();
    idx->lists = 1;
    k_list_caps<<<(unsigned)((n + bs - 1) / bs), bs, 0, st>>>(n, tau, idx->N, (uint32_t)s,
                                                              idx->xfloor, idx->lists,
                                                              idx->xlcap); note_launch();
    {
      std::vector<uint32_t> cap(n);
      std::vector<int64_t> off(n + 1, 0);
      RKR_CUDA(cudaMemcpyAsync(cap.data(), idx->xlcap, sizeof(uint32_t) * n,
                               cudaMemcpyDeviceToHost, st));
      RKR_CUDA(cudaStreamSynchronize(st));
      for (int64_t u = 0; u < n; ++u) off[u + 1] = off[u] + cap[u];
      RKR_TRY(dalloc(&idx->xlist, (size_t)std::max<int64_t>(off[n], 1)));
      RKR_CUDA(cudaMemcpyAsync(idx->xloff, off.data(), sizeof(int64_t) * (n + 1),
                               cudaMemcpyHostToDevice, st));
      RKR_CUDA(cudaStreamSynchronize(st));
    }
    RKR_TRY(tc_exact_table(idx, idx->Ut, idx->Pt, st, nullptr));
    if (idx->has_exact == 2) {
      // deep count grid from the sampled table's threshold of estimated count
      // m / 8 up to x_0
      idx->dg = kDGrid;
      RKR_TRY(dalloc(&idx->yg0, n));
      RKR_TRY(dalloc(&idx->ydx, n));
      RKR_TRY(dalloc(&idx->ybin, n));
      RKR_TRY(dalloc(&idx->DLO, (size_t)n * kDGrid));
      RKR_TRY(dalloc(&idx->DHI, (size_t)n * kDGrid));
      DevBuf bcol, btop, bbot;
      int32_t *col;
      float *ytop, *ybot;
      RKR_TRY(tmp_alloc(bcol, &col, n, st));
      RKR_TRY(tmp_alloc(btop, &ytop, n, st));
      RKR_TRY(tmp_alloc(bbot, &ybot, n, st));
      k_floor_cols<<<(unsigned)((n + bs - 1) / bs), bs, 0, st>>>(
          n, tau, idx->N, (uint32_t)s, (uint64_t)(m / 8 > 1 ? m / 8 : 1), col);
      note_launch();
      k_ygrid<<<(unsigned)((n + bs - 1) / bs), bs, 0, st>>>(n, idx->fmin, idx->delta, col,
                                                            idx->xfloor, idx->xg0, idx->yg0,
                                                            ytop, ybot);
      note_launch();
      RKR_TRY(make_binfp_grid(idx, idx->yg0, idx->xg0, kDGrid, idx->pmax, idx->ydx, idx->ybin,
                              st));
      RKR_TRY(tc_deep_table(idx, idx->Ut, idx->Pt, ytop, ybot, st));
    }
    idx->nlev_x = levels_for((uint64_t)m);
    RKR_TRY(dalloc(&idx->XJU, (size_t)n * kMaxLevels));
    RKR_TRY(dalloc(&idx->XJL, (size_t)n * kMaxLevels));
    k_levels<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(n, kXGrid, idx->XHI, idx->XLO,
                                                          (uint32_t)m, 1u, idx->nlev_x, idx->XJU,
                                                          idx->XJL); note_launch();
    RKR_CUDA(cudaGetLastError());
  }
  RKR_CUDA(cudaEventRecord(ev[6], st));
  RKR_CUDA(cudaStreamSynchronize(st));
  for (int i = 0; i < 6; ++i) {
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
    idx->build_ms[i] = ms;
  }
  float tot = 0.0f;
  cudaEventElapsedTime(&tot, ev[0], ev[6]);
  idx->build_ms[6] = tot;
  return RKR_OK;
}

void index_release(rkr_index *idx) {
  void *ptrs[] = {idx->U,      idx->Ps,   idx->perm, idx->pnorm, idx->unrm,
                  idx->pnrm_s, idx->fmin, idx->fmax, idx->delta, idx->binfp, idx->N,
                  idx->JU,     idx->JL,   idx->S,    idx->snrm, idx->sw,    idx->samp_items,
                  idx->xg0,    idx->xdx,  idx->xbin, idx->XLO,  idx->XHI,   idx->XJU,   idx->XJL,
                  idx->xfloor, idx->xloff, idx->xlcap, idx->xlist, idx->xlcnt,
                  idx->xbmax, idx->ptile3, idx->xcoff, idx->ldx, idx->lbin, idx->phk, idx->phv,
                  idx->yg0,   idx->ydx,  idx->ybin, idx->DLO,  idx->DHI};
  // nothing may still use the arrays when they go back to the pool
  cudaDeviceSynchronize();
  for (void *p : ptrs)
    if (p) cudaFreeAsync(p, (cudaStream_t)0);
  cudaStreamSynchronize((cudaStream_t)0);
  tc_free(idx->Ut);
  tc_free(idx->Pt);
}

}  // namespace rkr
