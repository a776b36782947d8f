// screen_epi.cu -- epilogues of the tensor-core screens and their drivers.
//
//   f-bounds   U.P^T, two passes: per-user max(s_hat - b) / min(s_hat + b), then
//              every item that may reach the extreme is evaluated canonically
//   exact table U.P^T (split product): per user, exact counts #{p : s(u,p) > x_j}
//              on a grid x_0 < .. < x_{G-1} spanning the upper tail of u's scores
//   theta      U.Q^T: bin interval of u.q on a grid -> per-query level histograms
//              (pass 1) or candidate lists (pass 2)
//   recount    U'.P^T over users with candidates (split product): each score is
//              located in the user's sorted block of candidate thresholds
// Undecided cases (bound straddling a boundary) are queued as (row, item) pairs
// and resolved by canonical FP64 afterwards.
#include <math.h>

#include <algorithm>
#include <vector>

#include "index.cuh"
#include "tcops.cuh"

namespace rkr {

namespace {

__device__ __forceinline__ uint64_t dkey_signed(double x) {
  uint64_t b = (uint64_t)__double_as_longlong(x);
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}

__device__ __forceinline__ double dkey_inverse(uint64_t k) {
  uint64_t b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double((long long)b);
}

// The bound terms of a column tile, loaded one tile ahead: take(ct) returns
// tile ct's terms (prefetched when ct is the tile expected next) and starts the
// load of tile ct + 1, whose latency then overlaps the current tile's work.
// 32-bit mask of a predicate over the columns j = 0..31 of a chunk, built as four
// independent OR chains (one chain of 32 dependent ORs serializes the epilogue
// warps, of which only two share a scheduler).
template <class F>
__device__ __forceinline__ uint32_t bitmask32(F &&pred) {
  uint32_t m0 = 0, m1 = 0, m2 = 0, m3 = 0;
#pragma unroll
  for (int j = 0; j < 32; j += 4) {
    m0 |= (pred(j) ? 1u : 0u) << j;
    m1 |= (pred(j + 1) ? 1u : 0u) << (j + 1);
    m2 |= (pred(j + 2) ? 1u : 0u) << (j + 2);
    m3 |= (pred(j + 3) ? 1u : 0u) << (j + 3);
  }
  return (m0 | m1) | (m2 | m3);
}

struct TilePrefetch {
  tc::RowBound next;
  int nct;   // the column tile `next` holds
  __device__ __forceinline__ void start(const tc::RowBound *tileb, int ct) {
    nct = ct;
    next = tileb[ct];
  }
  __device__ __forceinline__ tc::RowBound take(const tc::RowBound *tileb, int ct, int64_t ncols,
                                               int bn) {
    const tc::RowBound cur = ct == nct ? next : tileb[ct];
    if ((int64_t)(ct + 1) * bn < ncols) {
      nct = ct + 1;
      next = tileb[ct + 1];
    }
    return cur;
  }
};

// Queue of (row, column) pairs with a capacity; overflow raises a flag.
struct PairQueue {
  int2 *items;
  unsigned long long *count;
  unsigned long long cap;
  int *overflow;
  __device__ __forceinline__ void push(int a, int b) const {
    unsigned long long i = atomicAdd(count, 1ull);
    if (i < cap) items[i] = make_int2(a, b);
    else atomicExch(overflow, 1);
  }
  // push from every lane active at this point with one atomic per group
  __device__ __forceinline__ void push_agg(int a, int b) const {
    const unsigned act = __activemask();
    const int lane = threadIdx.x & 31, leader = __ffs(act) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(count, (unsigned long long)__popc(act));
    base = __shfl_sync(act, base, leader);
    const unsigned long long i = base + __popc(act & ((1u << lane) - 1u));
    if (i < cap) items[i] = make_int2(a, b);
    else atomicExch(overflow, 1);
  }
};

}  // namespace

// ============================================================== f-bounds

// f_min / f_max in one single-product pass.  Each thread keeps, over the
// columns it has seen, the largest lower end (mxlo) and the smallest upper end
// (mnhi) of the screened scores; an item is queued when its upper end reaches
// mxlo or its lower end reaches mnhi after the chunk is folded in.  The item
// holding the exact maximum is always queued: when it is seen, mxlo is at most
// the maximum, which is at most its upper end (and likewise for the minimum).
// A short seeding launch over the first (largest-norm) columns starts every
// thread at near-final extremes, so few items are queued.
struct EpiFb {
  static const char *name() { return "k_screen<EpiFb>"; }
  struct Thread {
    float b, mxlo, mnhi;
    int64_t row;
    tc::RowBound ru;     // the row's bound terms
    TilePrefetch tp;     // the bound terms of the next column tile
  };
  static constexpr size_t kSmem = 0;
  int64_t nrows, ncols;
  int bn;
  const tc::RowBound *rowb, *tileb;
  tc::Gacc gacc;
  float gcan;
  PairQueue q;
  const float2 *seed;   // per row: (largest lower end, smallest upper end) to start from, or null
  float2 *seed_out;     // seeding launch: per (row, column half) extremes, no queue
  __device__ __forceinline__ void unit_begin(char *, const tc::Unit &u, int et,
                                             Thread &ts) const {
    ts.mxlo = -INFINITY;
    ts.mnhi = INFINITY;
    ts.row = -1;
    ts.tp.start(tileb, u.ct0);
    if (seed) {
      const int w = (et >> 5) + 2, lane = et & 31;
      const int64_t row = (int64_t)u.rb0 * tc::BM + (w & 3) * 32 + lane;
      if (row < nrows) {
        const float2 a = seed[2 * row], b = seed[2 * row + 1];
        ts.mxlo = fmaxf(a.x, b.x);
        ts.mnhi = fminf(a.y, b.y);
      }
    }
  }
  __device__ __forceinline__ void tile_begin(char *, int rb, int ct, int r, int,
                                             Thread &ts) const {
    const int64_t row = (int64_t)rb * tc::BM + r;
    if (row != ts.row && row < nrows) ts.ru = rowb[row];   // once per row
    ts.row = row;
    const tc::RowBound tb = ts.tp.take(tileb, ct, ncols, bn);
    ts.b = ts.row < nrows ? tc::screen_bound_tc(ts.ru, tb, gacc, gcan) : 0.0f;
  }
  __device__ __forceinline__ void chunk(char *, int, int ct, int, int col, uint32_t,
                                        const float (&v)[32], Thread &ts) const {
    const int64_t c0 = (int64_t)ct * bn + col;
    const int64_t left = ncols - c0;
    uint32_t keep = left >= 32 ? 0xffffffffu : left <= 0 ? 0u : (1u << left) - 1u;
    if (ts.row >= nrows) keep = 0;  // the warp stays together for the reservation below
    float mx, mn;   // extremes of the chunk's kept scores
    if (keep == 0xffffffffu) {
      float a[16], c[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        a[j] = fmaxf(v[2 * j], v[2 * j + 1]);
        c[j] = fminf(v[2 * j], v[2 * j + 1]);
      }
#pragma unroll
      for (int w = 8; w > 0; w >>= 1)
#pragma unroll
        for (int j = 0; j < w; ++j) {
          a[j] = fmaxf(a[j], a[j + w]);
          c[j] = fminf(c[j], c[j + w]);
        }
      mx = a[0];
      mn = c[0];
    } else {
      mx = -INFINITY;
      mn = INFINITY;
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const bool in = (keep >> j) & 1u;
        mx = fmaxf(mx, in ? v[j] : -INFINITY);
        mn = fminf(mn, in ? v[j] : INFINITY);
      }
    }
    ts.mxlo = fmaxf(ts.mxlo, __fsub_rd(mx, ts.b));
    ts.mnhi = fminf(ts.mnhi, __fadd_ru(mn, ts.b));
    if (seed_out) return;
    // v + b >= mxlo  <=  v >= mxlo - b rounded down (and likewise for the minimum);
    // a chunk whose own extremes pass neither test has nothing to queue
    const float tmax = __fsub_rd(ts.mxlo, ts.b), tmin = __fadd_ru(ts.mnhi, ts.b);
    const bool hit = mx >= tmax || mn <= tmin;
    if (!__any_sync(0xffffffffu, hit)) return;
    uint32_t mask = 0;
    if (hit) {
#pragma unroll
      mask = bitmask32([&](int j) { return v[j] >= tmax || v[j] <= tmin; });
      mask &= keep;
    }
    // one queue reservation per warp and chunk
    const int lane = threadIdx.x & 31;
    const int cnt = __popc(mask);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0) return;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(q.count, (unsigned long long)total);
    base = __shfl_sync(0xffffffffu, base, 0) + (unsigned long long)(incl - cnt);
    while (mask) {
      const int j = __ffs(mask) - 1;
      mask &= mask - 1;
      if (base < q.cap) q.items[base] = make_int2((int)ts.row, (int)(c0 + j));
      else atomicExch(q.overflow, 1);
      ++base;
    }
  }
  __device__ __forceinline__ void tile_end(char *, int, int, int, int, Thread &) const {}
  __device__ __forceinline__ void unit_end(char *, const tc::Unit &u, int et, Thread &ts) const {
    if (!seed_out) return;
    const int w = (et >> 5) + 2, lane = et & 31;
    const int64_t row = (int64_t)u.rb0 * tc::BM + (w & 3) * 32 + lane;
    if (row < nrows) seed_out[2 * row + ((et >> 5) >> 2)] = make_float2(ts.mxlo, ts.mnhi);
  }
};

__global__ void k_fb_init(int64_t n, unsigned long long *kmax, unsigned long long *kmin) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  kmax[i] = 0ull;
  kmin[i] = ~0ull;
}

// Queued items, first pass: per user the largest lower end and the smallest
// upper end of the compensated intervals holding the canonical scores.
__global__ void k_fb_bracket(const int2 *__restrict__ items, const unsigned long long *count,
                             unsigned long long cap, const float *__restrict__ U,
                             const float *__restrict__ Ps, int d,
                             unsigned long long *__restrict__ kmaxlo,
                             unsigned long long *__restrict__ kminhi,
                             double2 *__restrict__ ival) {
  unsigned long long c = *count;
  if (c > cap) c = cap;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < c;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const int2 it = items[i];
    double lo, hi;
    dot2_interval(U + (int64_t)it.x * d, Ps + (int64_t)it.y * d, d, lo, hi);
    ival[i] = make_double2(lo, hi);
    atomicMax(&kmaxlo[it.x], (unsigned long long)dkey_signed(lo));
    atomicMin(&kminhi[it.x], (unsigned long long)dkey_signed(hi));
  }
}

// Second pass: only items whose interval reaches the bracket can hold an
// extreme; those get the canonical score.
__global__ void k_fb_resolve(const int2 *__restrict__ items, const unsigned long long *count,
                             unsigned long long cap, const float *__restrict__ U,
                             const float *__restrict__ Ps, int d,
                             const unsigned long long *__restrict__ kmaxlo,
                             const unsigned long long *__restrict__ kminhi,
                             const double2 *__restrict__ ival, unsigned long long *kmax,
                             unsigned long long *kmin) {
  unsigned long long c = *count;
  if (c > cap) c = cap;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < c;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const int2 it = items[i];
    const float *uu = U + (int64_t)it.x * d, *pp = Ps + (int64_t)it.y * d;
    const double lo = ival[i].x, hi = ival[i].y;
    const bool maxc = dkey_signed(hi) >= kmaxlo[it.x], minc = dkey_signed(lo) <= kminhi[it.x];
    if (!maxc && !minc) continue;
    const uint64_t k = dkey_signed(canon_dot(uu, pp, d));
    if (maxc) atomicMax(&kmax[it.x], (unsigned long long)k);
    if (minc) atomicMin(&kmin[it.x], (unsigned long long)k);
  }
}

__global__ void k_fb_finish(int64_t n, const unsigned long long *kmax,
                            const unsigned long long *kmin, double *fmin, double *fmax,
                            int *bad) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (kmax[i] == 0ull || kmin[i] == ~0ull) {
    atomicExch(bad, 1);
    return;
  }
  fmax[i] = dkey_inverse(kmax[i]);
  fmin[i] = dkey_inverse(kmin[i]);
}

// Exact canonical f_min / f_max per user from one tensor-core pass.
// Returns RKR_EINTERNAL (after which the caller uses the CUDA-core scan) when
// the candidate queue overflows.
rkr_status tc_fbounds(const rkr_index *idx, const TcSide &Ut, const TcSide &Pt, double *fmin,
                      double *fmax, cudaStream_t st) {
  constexpr int BN = 256;
  const int64_t n = idx->n, m = idx->m;
  tc::RowBound *tb = nullptr;
  RKR_TRY(tc_tile_bounds(Pt, BN, 0, &tb, st));
  unsigned long long *kmax, *kmin, *kmaxlo, *kminhi, *qcount;
  int2 *qitems;
  int *flags;  // [0] screen error, [1] overflow, [2] missing extreme
  const unsigned long long cap = std::max<int64_t>(64 * n, 1 << 16);
  RKR_CUDA(pool_malloc_async(&kmaxlo, sizeof(unsigned long long) * n, st));
  RKR_CUDA(pool_malloc_async(&kminhi, sizeof(unsigned long long) * n, st));
  RKR_CUDA(pool_malloc_async(&kmax, sizeof(unsigned long long) * n, st));
  RKR_CUDA(pool_malloc_async(&kmin, sizeof(unsigned long long) * n, st));
  RKR_CUDA(pool_malloc_async(&qcount, sizeof(unsigned long long), st));
  RKR_CUDA(pool_malloc_async(&qitems, sizeof(int2) * cap, st));
  double2 *ival;
  RKR_CUDA(pool_malloc_async(&ival, sizeof(double2) * cap, st));
  RKR_CUDA(pool_malloc_async(&flags, sizeof(int) * 4, st));
  RKR_CUDA(cudaMemsetAsync(qcount, 0, sizeof(unsigned long long), st));
  RKR_CUDA(cudaMemsetAsync(flags, 0, sizeof(int) * 4, st));
  const tc::Schedule sch = row_schedule(n, m, BN);
  EpiFb a;
  a.nrows = n; a.ncols = m; a.bn = BN; a.rowb = Ut.rb1; a.tileb = tb;
  a.gacc = tc_gacc(Ut.kp, 0); a.gcan = tc_gcan(idx->d);
  a.q = PairQueue{qitems, qcount, cap, flags + 1};
  // seeding launch over the first columns (the largest norms), then the full pass
  float2 *seed;
  RKR_CUDA(pool_malloc_async(&seed, sizeof(float2) * 2 * n, st));
  TcSide head = Pt;
  head.owned = false;
  head.rows = std::min<int64_t>(m, 4 * BN);
  EpiFb a0 = a;
  a0.seed = nullptr;
  a0.seed_out = seed;
  a0.ncols = head.rows;
  rkr_status s = launch_screen<BN, 4>(Ut, head, 0, row_schedule(n, head.rows, BN), a0, flags, st);
  a.seed = seed;
  a.seed_out = nullptr;
  if (s == RKR_OK) s = launch_screen<BN, 4>(Ut, Pt, 0, sch, a, flags, st);
  cudaFreeAsync(seed, st);
  if (s == RKR_OK) {
    k_fb_init<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, kmaxlo, kminhi);
    note_launch();
    k_fb_init<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, kmax, kmin);
    note_launch();
    {
      ProfScope prof("k_fb_bracket", st);
      k_fb_bracket<<<8 * sm_count(), 256, 0, st>>>(qitems, qcount, cap, idx->U, idx->Ps, idx->d,
                                                   kmaxlo, kminhi, ival);
    }
    note_launch();
    {
      ProfScope prof("k_fb_resolve", st);
      k_fb_resolve<<<8 * sm_count(), 256, 0, st>>>(qitems, qcount, cap, idx->U, idx->Ps, idx->d,
                                                   kmaxlo, kminhi, ival, kmax, kmin);
    }
    note_launch();
    k_fb_finish<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, kmax, kmin, fmin, fmax,
                                                             flags + 2);
    note_launch();
  }
  int hf[4] = {0, 0, 0, 0};
  cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  for (void *p : {(void *)tb, (void *)kmax, (void *)kmin, (void *)kmaxlo, (void *)kminhi,
                  (void *)qcount, (void *)qitems, (void *)ival, (void *)flags})
    cudaFreeAsync(p, st);
  if (e != cudaSuccess) return cuda_fail(e, "tc_fbounds");
  RKR_TRY(s);
  if (hf[0]) return fail(RKR_ETIMEOUT, "f-bounds screen wait timed out (%d)", hf[0]);
  if (hf[1] || hf[2]) return fail(RKR_EINTERNAL, "f-bounds candidate queue overflow");
  return RKR_OK;
}

// =========================================================== exact table

constexpr int kXG = kXGrid;  // columns of the exact grid

// Exact grid of each user: x_i = g0 + i * dx, i = 0..G-1, dx = (f_max - g0) / (G - 1),
// where g0 is the paper threshold t_{floor+1} whose estimated count is still at
// least the floor rank.  The grid spans the upper tail of u's scores.
__global__ void k_xgrid(int64_t n, const double *__restrict__ fmin,
                        const double *__restrict__ delta, const int32_t *__restrict__ fl,
                        double *__restrict__ g0, float *__restrict__ g0f) {
  int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= n) return;
  double g = thr_at(fmin[u], delta[u], fl[u]);
  g0[u] = g;
  g0f[u] = __double2float_rd(g);
}

// Interval counts on the exact grid: an item whose count c(s) = #{j : x_j < s}
// is known to lie in [clo, chi] adds to Hlo[clo] and Hhi[chi]; then
// XLO[j] = #{clo > j} <= #{p : s(u,p) > x_j} <= #{chi > j} = XHI[j].
// Histograms are 16-bit pairs packed in 32-bit words; a row whose tail holds
// more than 65535 items gets the trivial bounds 0 and m instead.
struct EpiXT {
  static const char *name() { return "k_screen<EpiXT>"; }
  struct Thread {
    float skip, b, g0;
    int64_t row;
    int64_t off;
    uint32_t cap;
    tc::RowBound ru;     // the row's bound terms
    TilePrefetch tp;     // the bound terms of the next column tile
  };
  // list cursors of the block's 128 rows, then a 32 x 32 staging tile per warp
  // stored [column][lane] (a lane's lookups hit its own bank)
  static constexpr size_t kStageOff = sizeof(uint32_t) * 128;
  static constexpr size_t kSmem = kStageOff + sizeof(float) * 8 * 32 * 32;
  int64_t nrows, ncols;
  int bn;
  const tc::RowBound *rowb, *tileb;
  tc::Gacc gacc;
  float gcan;
  const float *g0f;
  // tail lists: every above-floor item is appended to its user's list; the
  // count table is derived from the lists when they are grouped
  uint2 *list;
  const int64_t *loff;
  const uint32_t *lcapv;
  uint32_t *lcnt;      // n: entries (> capacity marks an overflow)
  __device__ uint32_t *lslot(char *S) const { return (uint32_t *)S; }
  __device__ void unit_begin(char *S, const tc::Unit &u, int et, Thread &ts) const {
    if (et < 128) lslot(S)[et] = 0;
    ts.row = -1;
    ts.tp.start(tileb, u.ct0);
  }
  __device__ void tile_begin(char *, int rb, int ct, int r, int, Thread &ts) const {
    const int64_t row = (int64_t)rb * tc::BM + r;
    if (row != ts.row && row < nrows) {   // the row's data, once per row
      ts.ru = rowb[row];
      ts.g0 = g0f[row];
      ts.off = loff[row];
      ts.cap = lcapv[row];
    }
    ts.row = row;
    const tc::RowBound tb = ts.tp.take(tileb, ct, ncols, bn);
    if (ts.row < nrows) {
      ts.b = tc::screen_bound_tc(ts.ru, tb, gacc, gcan);
      ts.skip = __fsub_rd(ts.g0, ts.b);  // s_hat <= skip implies s <= x_0
    } else {
      ts.skip = INFINITY;
    }
  }
  // Scores above the floor are a few per cent and scattered over lanes: each
  // lane parks its 32 scores in a shared tile, reserves its slots with one
  // atomic and walks only its own above-floor ones.
  __device__ void chunk(char *S, int, int ct, int r, int col, uint32_t, const float (&v)[32],
                        Thread &ts) const {
    const int64_t c0 = (int64_t)ct * bn + col;
    const int lane = threadIdx.x & 31, warp = (threadIdx.x >> 5) - 2;
    float *tile = (float *)(S + kStageOff) + warp * 32 * 32 + lane;
#pragma unroll
    for (int j = 0; j < 32; ++j) tile[j * 32] = v[j];
    uint32_t mask = bitmask32([&](int j) { return v[j] > ts.skip; });
    const int64_t left = ncols - c0;
    if (left < 32) mask &= left <= 0 ? 0u : (1u << left) - 1u;
    if (!mask) return;
    uint32_t pos = atomicAdd(&lslot(S)[r], (uint32_t)__popc(mask));
    while (mask) {
      const int j = __ffs(mask) - 1;
      mask &= mask - 1;
      if (pos < ts.cap)
        list[ts.off + pos] = make_uint2((uint32_t)(c0 + j), __float_as_uint(tile[j * 32]));
      ++pos;
    }
  }
  __device__ void tile_end(char *, int, int, int, int, Thread &) const {}
  __device__ void unit_end(char *S, const tc::Unit &u, int et, Thread &) const {
    tc::epi_sync();
    if (et >= 128) return;
    const int64_t g = (int64_t)u.rb0 * tc::BM + et;
    if (g < nrows) lcnt[g] = lslot(S)[et];
  }
};


// Group each user's tail list by the exact-grid column of the screened score,
// col(v) = #{j : x_j <= v} in 0..G (counting sort), and record the column
// offsets and the largest screen bound of the entries.  One CTA of 512 threads
// per user, two resident per SM so that one user's list loads overlap another's
// counting; overflowed lists are left as they are and marked unusable.  A thread
// keeps kGroupPer entries in registers (64 registers a thread), so that a list
// is in flight at once and can be written back in place.  Lists longer than
// 512 * kGroupPer entries are set aside and grouped by a second launch whose
// threads also keep up to kGroupExt entries in shared memory (a larger shared
// footprint for every CTA of the first launch would leave less room for L1).
constexpr int kGroupThreads = 512;
constexpr int kGroupPer = 16;                            // list entries per thread, registers
constexpr int kGroupExt = 16;                            // and in shared memory
static_assert(kGroupThreads * (kGroupPer + kGroupExt) == kListCapMax, "list capacity");

// j(theta) = #{i < tau : t_i <= theta} when it is known to lie in [jlo, jhi]:
// the thresholds inside the bracket are compared in FP64 (no division).
__device__ __forceinline__ int exact_j_near(double theta, double fmin, double delta, int jlo,
                                           int jhi) {
  int g = jlo;
  while (g < jhi && thr_at(fmin, delta, g) <= theta) ++g;
  return g;
}

struct ListGroupArgs {
  int64_t n;
  uint2 *list;
  const int64_t *loff;
  const uint32_t *lcap, *lcnt;
  const BinFP *lbin;
  const double *ldx;
  int G;
  const BinFP *xbin;
  const double *xg0;
  uint32_t *XLO, *XHI;
  uint32_t mcount;
  const tc::RowBound *rowb, *tileb;
  int bn_shift;
  tc::Gacc gacc;
  float gcan;
  uint16_t *coff;
  float *bmax;
};

template <bool EXT>
constexpr size_t list_group_smem(int G) {
  return sizeof(uint2) * (EXT ? kGroupThreads * kGroupExt : 0) +
         sizeof(uint32_t) * (G + 2 + 2 * (kXG + 1)) + sizeof(uint32_t) * (kGroupThreads / 32) +
         sizeof(float) * (kGroupThreads / 32) +
         sizeof(uint16_t) * kGroupThreads * (kGroupPer + (EXT ? kGroupExt : 0));
}

// One user's list: (1) the exact count table XLO/XHI on the kXG-column grid
// from the user's list (every item above x_0 is in it; each entry's interval
// uses the screen bound of its item tile), (2) the list grouped by the
// kListG-column list grid with column offsets, (3) the largest entry bound.  An
// overflowed list gives the trivial table XLO = 0, XHI = m.  All entries are
// loaded up front, so the grouping can be written back in place after one barrier.
template <bool EXT>
__device__ __forceinline__ void list_group_user(const ListGroupArgs &a, int64_t u,
                                                unsigned char *lsm) {
  constexpr int T = kGroupThreads;
  const int G = a.G;
  uint2 *ext = (uint2 *)lsm;                                  // T * kGroupExt (EXT)
  uint32_t *cnt = (uint32_t *)(ext + (EXT ? T * kGroupExt : 0));   // G + 2
  uint32_t *hlo = cnt + G + 2;                                // kXG + 1
  uint32_t *hhi = hlo + kXG + 1;                              // kXG + 1
  uint32_t *wsum = hhi + kXG + 1;                             // T / 32
  float *red = (float *)(wsum + T / 32);                      // T / 32
  uint16_t *cols = (uint16_t *)(red + T / 32);                // T * (kGroupPer [+ kGroupExt])
  const uint32_t L = a.lcnt[u];
  uint16_t *co = a.coff + u * (G + 2);
  if (L > a.lcap[u]) {  // overflow: the list is incomplete
    if (threadIdx.x == 0) a.bmax[u] = INFINITY;
    for (int c = threadIdx.x; c < kXG; c += T) {
      a.XLO[u * kXG + c] = 0u;
      a.XHI[u * kXG + c] = a.mcount;
    }
    return;
  }
  for (int c = threadIdx.x; c < G + 2; c += T) cnt[c] = 0;
  for (int c = threadIdx.x; c <= kXG; c += T) {
    hlo[c] = 0;
    hhi[c] = 0;
  }
  __syncthreads();
  uint2 *row = a.list + a.loff[u];
  const BinFP lb = a.lbin[u], xb = a.xbin[u];
  const double g0 = a.xg0[u], dx = a.ldx[u];
  const tc::RowBound ru = a.rowb[u];
  float bm = 0.0f;
  uint2 ent[kGroupPer];
#pragma unroll
  for (int k = 0; k < kGroupPer; ++k) {
    const uint32_t i = threadIdx.x + (uint32_t)k * T;
    if (i < L) ent[k] = row[i];
  }
  if (EXT)
    for (uint32_t i = T * kGroupPer + threadIdx.x; i < L; i += T) ext[i - T * kGroupPer] = row[i];
  // Column c = #{x_j <= v} of the list grid x_j = g0 + j dx.  The FP32 column
  // coordinate (v - f)(1/dx), f = fl(g0), taken with directed roundings, is
  // within e(v) = (|v - f| 2^-21 + |g0| 2^-23) / dx of (v - g0) / dx: the
  // roundings of f, of 1/dx, of the difference and of the product add up to less
  // than |g0| 2^-24 / dx + |v - f| 2^-21.6 / dx.  Only a coordinate interval that
  // straddles a column edge is settled in FP64.
  // (1/dx <= invd32 (1 + 2^-22), since invd32 is 1/dx rounded to nearest twice, and
  // |g0| <= |f| (1 + 2^-23); both factors are formed in FP32 rounding up)
  const bool tight = lb.invd32 > 0.0f && lb.err <= 1e6f;
  const float inv_up = __fmul_ru(lb.invd32, 1.0f + 0x1p-22f);
  const float e1 = __fmul_ru(inv_up, 0x1p-21f * (1.0f + 0x1p-20f));
  const float e0 = __fadd_ru(
      __fmul_ru(__fmul_ru(fabsf(lb.fmin32), (1.0f + 0x1p-23f) * 0x1p-23f), inv_up), 0x1p-30f);
  auto list_col = [&](float v) {
    int jlo, jhi;
    if (tight) {
      const float alo = __fsub_rd(v, lb.fmin32), ahi = __fsub_ru(v, lb.fmin32);
      const float e = __fmaf_ru(fmaxf(fabsf(alo), fabsf(ahi)), e1, e0);
      jlo = bin_lo(__fsub_rd(__fmul_rd(alo, lb.invd32), e), G);
      jhi = bin_hi(__fadd_ru(__fmul_ru(ahi, lb.invd32), e), G);
    } else {
      bin_interval(lb, g0, G, v, v, jlo, jhi);
    }
    return jlo == jhi ? jlo : exact_j_near((double)v, g0, dx, jlo, jhi);
  };
  auto count_entry = [&](uint32_t i, const uint2 e) {
    const float v = __uint_as_float(e.y);
    const float b = tc::screen_bound_tc(ru, a.tileb[e.x >> a.bn_shift], a.gacc, a.gcan);
    bm = fmaxf(bm, b);
    int clo, chi;
    bin_interval(xb, g0, kXG, __fsub_rd(v, b), __fadd_ru(v, b), clo, chi);
    if (chi > 0) {
      atomicAdd(&hlo[clo], 1u);
      atomicAdd(&hhi[chi], 1u);
    }
    const int col = list_col(v);
    cols[i] = (uint16_t)col;
    atomicAdd(&cnt[col], 1u);
  };
#pragma unroll
  for (int k = 0; k < kGroupPer; ++k) {
    const uint32_t i = threadIdx.x + (uint32_t)k * T;
    if (i >= L) break;
    count_entry(i, ent[k]);
  }
  // (each thread reads back only the shared entries it stored itself)
  if (EXT)
    for (uint32_t i = T * kGroupPer + threadIdx.x; i < L; i += T)
      count_entry(i, ext[i - T * kGroupPer]);
  for (int o = 16; o > 0; o >>= 1) bm = fmaxf(bm, __shfl_xor_sync(0xffffffffu, bm, o));
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) red[wid] = bm;
  __syncthreads();
  if (wid == 0) {
    // count table: XLO[c-1] = sum_{c' >= c} hlo[c'], c = 1..kXG (4 columns per lane)
    constexpr int kPer = kXG / 32;
    uint32_t sl = 0, sh = 0;
    for (int t = 0; t < kPer; ++t) {
      sl += hlo[1 + lane * kPer + t];
      sh += hhi[1 + lane * kPer + t];
    }
    uint32_t al = sl, ah = sh;  // inclusive suffix over lanes >= lane
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t xl = __shfl_down_sync(0xffffffffu, al, o);
      const uint32_t xh = __shfl_down_sync(0xffffffffu, ah, o);
      if (lane + o < 32) { al += xl; ah += xh; }
    }
    uint32_t rl = al - sl, rh = ah - sh;  // sums over columns above this lane's block
    for (int t = kPer - 1; t >= 0; --t) {
      const int c = 1 + lane * kPer + t;
      rl += hlo[c];
      rh += hhi[c];
      a.XLO[u * kXG + (c - 1)] = rl;
      a.XHI[u * kXG + (c - 1)] = rh;
    }
    if (lane == 0) {
      float m2 = 0.0f;
      for (int w = 0; w < T / 32; ++w) m2 = fmaxf(m2, red[w]);
      a.bmax[u] = m2;
    }
  }
  // list grid: exclusive prefix over the G + 1 columns, a contiguous run per thread
  const int per = (G + 1 + T - 1) / T;
  const int c0 = threadIdx.x * per, c1 = min(G + 1, c0 + per);
  uint32_t part = 0;
  for (int c = c0; c < c1; ++c) part += cnt[c];
  uint32_t incl = part;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t x = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += x;
  }
  if (lane == 31) wsum[wid] = incl;
  __syncthreads();
  uint32_t base = 0;
  for (int w = 0; w < wid; ++w) base += wsum[w];
  uint32_t run = base + incl - part;
  for (int c = c0; c < c1; ++c) {
    const uint32_t t = cnt[c];
    cnt[c] = run;
    co[c] = (uint16_t)run;
    run += t;
  }
  if (threadIdx.x == T - 1) co[G + 1] = (uint16_t)run;
  __syncthreads();
#pragma unroll
  for (int k = 0; k < kGroupPer; ++k) {
    const uint32_t i = threadIdx.x + (uint32_t)k * T;
    if (i >= L) break;
    const uint32_t pos = atomicAdd(&cnt[cols[i]], 1u);
    row[pos] = ent[k];
  }
  if (EXT)
    for (uint32_t i = T * kGroupPer + threadIdx.x; i < L; i += T) {
      const uint32_t pos = atomicAdd(&cnt[cols[i]], 1u);
      row[pos] = ext[i - T * kGroupPer];
    }
}

// Every user whose list fits the registers (and overflowed lists); the longer
// ones are appended to longu for k_list_group_long.
__global__ void __launch_bounds__(kGroupThreads, 2) k_list_group(ListGroupArgs a,
                                                                int32_t *longu,
                                                                unsigned int *nlong) {
  extern __shared__ __align__(16) unsigned char lsm[];
  const int64_t u = blockIdx.x;
  const uint32_t L = a.lcnt[u];
  if (L > (uint32_t)(kGroupThreads * kGroupPer) && L <= a.lcap[u]) {
    if (threadIdx.x == 0) longu[atomicAdd(nlong, 1u)] = (int32_t)u;
    return;
  }
  list_group_user<false>(a, u, lsm);
}

// The longer lists, persistent CTAs over the users k_list_group set aside.
__global__ void __launch_bounds__(kGroupThreads, 2) k_list_group_long(ListGroupArgs a,
                                                                     const int32_t *longu,
                                                                     const unsigned int *nlong) {
  extern __shared__ __align__(16) unsigned char lsm[];
  const unsigned int cnt = *nlong;
  for (unsigned int i = blockIdx.x; i < cnt; i += gridDim.x) {
    list_group_user<true>(a, longu[i], lsm);
    __syncthreads();   // the shared tables are reused by the next user
  }
}

rkr_status tc_sort_lists(rkr_index *idx, const tc::RowBound *tb, int bn, cudaStream_t st) {
  // keep the item tile bounds for query-time lookups
  const int ntiles = (int)((idx->m + bn - 1) / bn);
  RKR_CUDA(cudaMemcpyAsync(idx->ptile3, tb, sizeof(tc::RowBound) * ntiles,
                           cudaMemcpyDeviceToDevice, st));
  idx->ptile_bn = bn;
  int bn_shift = 0;
  while ((1 << bn_shift) < bn) ++bn_shift;
  if ((1 << bn_shift) != bn) return fail(RKR_EINTERNAL, "item tile width %d is not a power of two", bn);
  const int G = kListG;
  RKR_TRY(make_binfp_grid(idx, idx->xg0, idx->fmax, G, idx->pmax, idx->ldx, idx->lbin, st));
  ListGroupArgs a;
  a.n = idx->n; a.list = idx->xlist; a.loff = idx->xloff; a.lcap = idx->xlcap;
  a.lcnt = idx->xlcnt; a.lbin = idx->lbin; a.ldx = idx->ldx; a.G = G; a.xbin = idx->xbin;
  a.xg0 = idx->xg0; a.XLO = idx->XLO; a.XHI = idx->XHI; a.mcount = (uint32_t)idx->m;
  a.rowb = idx->Ut.rb3; a.tileb = idx->ptile3; a.bn_shift = bn_shift;
  a.gacc = tc_gacc(idx->Ut.kp, 1); a.gcan = tc_gcan(idx->d); a.coff = idx->xcoff;
  a.bmax = idx->xbmax;
  DevBuf bl, bc;
  int32_t *longu;
  unsigned int *nlong;
  RKR_TRY(tmp_alloc(bl, &longu, idx->n, st));
  RKR_TRY(tmp_alloc(bc, &nlong, 1, st));
  RKR_CUDA(cudaMemsetAsync(nlong, 0, sizeof(unsigned int), st));
  const size_t sm1 = list_group_smem<false>(G), sm2 = list_group_smem<true>(G);
  RKR_CUDA(cudaFuncSetAttribute(k_list_group, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sm1));
  RKR_CUDA(cudaFuncSetAttribute(k_list_group_long, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sm2));
  {
    const int prof_slot = prof_begin("k_list_group", st);
    k_list_group<<<(unsigned)idx->n, kGroupThreads, sm1, st>>>(a, longu, nlong);
    note_launch();
    k_list_group_long<<<(unsigned)(2 * sm_count()), kGroupThreads, sm2, st>>>(a, longu, nlong);
    note_launch();
    prof_end(prof_slot, st, 0.0);
  }
  RKR_CUDA(cudaGetLastError());
  return RKR_OK;
}

rkr_status tc_exact_table(rkr_index *idx, const TcSide &Ut, const TcSide &Pt, cudaStream_t st,
                          int64_t *) {
  constexpr int BN = 256;
  const int64_t n = idx->n, m = idx->m;
  tc::RowBound *tb = nullptr;
  RKR_TRY(tc_tile_bounds(Pt, BN, 1, &tb, st));
  float *g0f;
  int *flags;
  RKR_CUDA(pool_malloc_async(&g0f, sizeof(float) * n, st));
  RKR_CUDA(pool_malloc_async(&flags, sizeof(int) * 2, st));
  RKR_CUDA(cudaMemsetAsync(flags, 0, sizeof(int) * 2, st));
  k_xgrid<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, idx->fmin, idx->delta, idx->xfloor,
                                                       idx->xg0, g0f);
  note_launch();

  RKR_TRY(make_binfp_grid(idx, idx->xg0, idx->fmax, kXG, idx->pmax, idx->xdx, idx->xbin, st));
  EpiXT e;
  e.nrows = n; e.ncols = m; e.bn = BN; e.rowb = Ut.rb3; e.tileb = tb;
  e.gacc = tc_gacc(Ut.kp, 1); e.gcan = tc_gcan(idx->d);
  e.g0f = g0f;
  e.list = idx->xlist; e.loff = idx->xloff; e.lcapv = idx->xlcap; e.lcnt = idx->xlcnt;
  static_assert(tc::screen_smem_bytes<BN, 4, EpiXT>() <= 232448, "exact-table smem");
  rkr_status s = launch_screen<BN, 4>(Ut, Pt, 1, row_schedule(n, m, BN), e, flags, st);
  if (s == RKR_OK) s = tc_sort_lists(idx, tb, BN, st);
  int hf[2] = {0, 0};
  cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, st);
  cudaError_t err = cudaStreamSynchronize(st);
  for (void *p : {(void *)tb, (void *)g0f, (void *)flags}) cudaFreeAsync(p, st);
  if (err != cudaSuccess) return cuda_fail(err, "tc_exact_table");
  RKR_TRY(s);
  if (hf[0]) return fail(RKR_ETIMEOUT, "exact-table screen wait timed out (%d)", hf[0]);
  return RKR_OK;
}

// ============================================================ deep grid

// Count intervals on the deep grid y_c = yg0 + c * ydx, c = 0 .. G - 1 (G =
// kDGrid), every item of P: the interval [v - b, v + b] of a screened score
// gives bounds [jl, jh] of c(s) = #{c : y_c < s} (bin_interval); the item adds
// to Hlo[jl] and Hhi[jh], and DLO[c] = #{jl > c} <= #{p : s(u,p) > y_c} <=
// #{jh > c} = DHI[c], as for the exact grid of the tail lists.  Items whose
// upper end lies below y_0 add to no count; items certainly above the whole
// grid go to bin G of both histograms.  Scores reaching the grid are about an
// eighth of all: each lane marks them in a bit mask, parks the chunk in a
// shared tile and walks only its own marked ones (branch-free bin arithmetic),
// so a warp spends it on the largest per-lane count of the chunk instead of on
// all 32 columns.  The histograms are 32-bit counters per row in shared memory,
// stored [bin][row] so that a warp's 32 rows never share a bank.
struct EpiDeep {
  static const char *name() { return "k_screen<EpiDeep>"; }
  static constexpr int kBins = kDGrid + 1;
  struct Thread {
    float b, top_lo;     // bound; lower ends above top_lo are above the whole grid
    float bot_hi;        // upper ends below bot_hi are below the whole grid
    int64_t row;
    BinFP bf;
    double g0;
    tc::RowBound ru;
    TilePrefetch tp;
  };
  static constexpr size_t kHist = sizeof(uint32_t) * 128 * kBins;   // one of Hlo, Hhi
  static constexpr size_t kStageOff = 2 * kHist;
  static constexpr size_t kSmem = kStageOff + sizeof(float) * 8 * 32 * 32;
  int64_t nrows, ncols;
  int bn;
  const tc::RowBound *rowb, *tileb;
  tc::Gacc gacc;
  float gcan;
  const BinFP *ybin;
  const double *yg0;
  const float *ytop;       // per row: the grid's top point rounded up to float
  const float *ybot;       // per row: the grid's first point rounded down to float
  uint32_t *DLO, *DHI;     // n x kDGrid
  __device__ static uint32_t *hlo(char *S, int r) { return (uint32_t *)S + r; }
  __device__ static uint32_t *hhi(char *S, int r) { return (uint32_t *)(S + kHist) + r; }
  __device__ void unit_begin(char *S, const tc::Unit &u, int et, Thread &ts) const {
    for (int i = et; i < 2 * 128 * kBins; i += 256) ((uint32_t *)S)[i] = 0u;
    ts.row = -1;
    ts.tp.start(tileb, u.ct0);
  }
  __device__ void tile_begin(char *, int rb, int ct, int r, int, Thread &ts) const {
    const int64_t row = (int64_t)rb * tc::BM + r;
    if (row != ts.row && row < nrows) {   // the row's data, once per row
      ts.ru = rowb[row];
      ts.bf = ybin[row];
      ts.g0 = yg0[row];
      ts.top_lo = ytop[row];
      ts.bot_hi = ybot[row];
    }
    ts.row = row;
    const tc::RowBound tb = ts.tp.take(tileb, ct, ncols, bn);
    ts.b = ts.row < nrows ? tc::screen_bound_tc(ts.ru, tb, gacc, gcan) : 0.0f;
  }
  __device__ void chunk(char *S, int, int ct, int r, int col, uint32_t, const float (&v)[32],
                        Thread &ts) const {
    if (ts.row >= nrows) return;
    const int64_t c0 = (int64_t)ct * bn + col;
    const int lane = threadIdx.x & 31, warp = (threadIdx.x >> 5) - 2;
    float *tile = (float *)(S + kStageOff) + warp * 32 * 32 + lane;
    // scores whose upper end reaches the grid's first point (the others count nowhere)
#pragma unroll
    for (int j = 0; j < 32; ++j) tile[j * 32] = v[j];
    uint32_t mask = bitmask32([&](int j) { return __fadd_ru(v[j], ts.b) >= ts.bot_hi; });
    const int64_t left = ncols - c0;
    if (left < 32) mask &= left <= 0 ? 0u : (1u << left) - 1u;
    const BinFP &bf = ts.bf;
    const bool fast = bf.invd32 > 0.0f && bf.err <= 1e6f;   // the row's grid has a step
    while (mask) {
      const int j = __ffs(mask) - 1;
      mask &= mask - 1;
      const float x = tile[j * 32];
      const float lo = __fsub_rd(x, ts.b), hi = __fadd_ru(x, ts.b);
      int jl, jh;
      if (fast) {
        // bin_interval without branches: the clamps of bin_lo / bin_hi by fminf /
        // fmaxf (which also send a NaN lower end to 0), a NaN upper end to G
        float vlo, vhi;
        bin_coord(bf, lo, hi, vlo, vhi);
        jl = (int)ceilf(fminf(fmaxf(vlo, 0.0f), (float)kDGrid));
        const float ch = fminf(floorf(fmaxf(vhi, -1.0f)) + 1.0f, (float)kDGrid);
        jh = vhi == vhi ? (int)ch : kDGrid;
      } else {
        bin_interval(bf, ts.g0, kDGrid, lo, hi, jl, jh);
      }
      // certainly above the whole grid: c = G exactly; jh = 0 adds to bin 0, which no
      // count reads
      const bool top = lo > ts.top_lo;
      jl = top ? kDGrid : jl;
      jh = top ? kDGrid : jh;
      atomicAdd(&hlo(S, r)[jl * 128], 1u);
      atomicAdd(&hhi(S, r)[jh * 128], 1u);
    }
  }
  __device__ void tile_end(char *, int, int, int, int, Thread &) const {}
  __device__ void unit_end(char *S, const tc::Unit &u, int et, Thread &ts) const {
    const int w = (et >> 5) + 2, lane = et & 31;
    const int r = (w & 3) * 32 + lane, half = et >> 7;
    const int64_t row = (int64_t)u.rb0 * tc::BM + r;
    tc::epi_sync();
    if (row >= nrows || half != 0) return;
    // DLO[c] = sum over bins above c
    uint32_t rl = 0, rh = 0;
    for (int c = kDGrid; c >= 1; --c) {
      rl += hlo(S, r)[c * 128];
      rh += hhi(S, r)[c * 128];
      DLO[row * kDGrid + (c - 1)] = rl;
      DHI[row * kDGrid + (c - 1)] = rh;
    }
  }
};

rkr_status tc_deep_table(rkr_index *idx, const TcSide &Ut, const TcSide &Pt, const float *ytop,
                         const float *ybot, cudaStream_t st) {
  // 128-column tiles: four 32 KB stages fit beside the histograms and the tile
  constexpr int BN = 128;
  const int64_t n = idx->n, m = idx->m;
  int *flags;
  tc::RowBound *tb = nullptr;
  RKR_CUDA(pool_malloc_async(&flags, sizeof(int) * 2, st));
  RKR_CUDA(cudaMemsetAsync(flags, 0, sizeof(int) * 2, st));
  RKR_TRY(tc_tile_bounds(Pt, BN, 0, &tb, st));
  EpiDeep e;
  e.nrows = n; e.ncols = m; e.bn = BN; e.rowb = Ut.rb1; e.tileb = tb;
  e.gacc = tc_gacc(Ut.kp, 0); e.gcan = tc_gcan(idx->d);
  e.ybin = idx->ybin; e.yg0 = idx->yg0; e.ytop = ytop; e.ybot = ybot;
  e.DLO = idx->DLO; e.DHI = idx->DHI;
  rkr_status s = launch_screen<BN, tc::stages1<BN, EpiDeep>()>(Ut, Pt, 0, row_schedule(n, m, BN),
                                                              e, flags, st);
  int hf[2] = {0, 0};
  cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, st);
  cudaError_t err = cudaStreamSynchronize(st);
  for (void *p : {(void *)tb, (void *)flags}) cudaFreeAsync(p, st);
  if (err != cudaSuccess) return cuda_fail(err, "tc_deep_table");
  RKR_TRY(s);
  if (hf[0]) return fail(RKR_ETIMEOUT, "deep-grid screen wait timed out (%d)", hf[0]);
  return RKR_OK;
}

// ================================================================= theta

constexpr int kThetaBN = 128;

// Pass 1 accumulates, per query, histograms of the rank level of the upper
// bound (from the low end of the bin interval) and of the lower bound (from
// its high end).  Pass 3 refines the cutoff inside the boundary level L*: each
// pair whose upper bound falls in level L* adds its exact upper-bound value to
// a 1024-bucket histogram of that level's range.  Pass 2 writes (user, query)
// when the lower bound may reach the query's cutoff: level test first, then
// the exact lower-bound value against the refined cap.
constexpr int kFine = 1024;

__device__ __forceinline__ void level_range(int L, uint32_t scale, uint64_t &base,
                                            uint64_t &width) {
  uint64_t hi = level_bound(L, scale);
  base = L == 0 ? 0 : level_bound(L - 1, scale) + 1;
  width = (hi - base + kFine) / kFine;  // ceil((hi - base + 1) / kFine)
}

template <int PASS>
struct EpiTheta {
  static const char *name() {
    return PASS == 1 ? "k_screen<EpiTheta1>" : PASS == 2 ? "k_screen<EpiTheta2>" : "k_screen<EpiTheta3>";
  }
  static constexpr int kJS = 34;  // int16 row stride of the level tables (conflict-free)
  struct Thread {
    float b;
    BinFP bf;
    double fm;
    int64_t u;
    int rb1;                 // end of the unit's row blocks (prefetch stays inside)
    uint4 pju[2], pjl[2];    // prefetched level-table words for the next row block
    BinFP pbf;
    double pfm;
    tc::RowBound prb, rb;
    float xsb, pxs;          // skip pairs with screened score <= xsb
    bool have_pf;
  };
  static constexpr size_t kSmem = sizeof(int16_t) * 2 * 128 * kJS +
                                  sizeof(int) * (2 * kThetaBN * 32 + 3 * kThetaBN) +
                                  sizeof(tc::RowBound) * kThetaBN;
  int64_t nrows, ncols;
  int tau;
  int qa;  // global index of query column 0
  const tc::RowBound *rowb, *tileb;
  const tc::RowBound *colb;     // per-column (query) bound terms, local column index
  tc::Gacc gacc;
  float gcan;
  const BinFP *binfp;
  const double *fmin;
  const int16_t *JU, *JL;
  const uint32_t *thi, *tlo;    // tables behind the upper and lower bounds
  uint32_t top, scale;          // upper bound below the grid; level scale
  uint32_t *hist_up, *hist_lo;  // PASS 1: [nq][32], indexed by global query
  const int32_t *lstar;         // PASS 2, 3: indexed by global query
  const uint32_t *cap;          // PASS 2
  uint32_t *fine;               // PASS 3: [nq][kFine]
  const int64_t *qoff;
  uint32_t *qcursor;
  int32_t *cand_u, *cand_q;
  int *ovf;                     // PASS 2: set when a query's segment would overflow
  const float *xs;              // per user: pairs scoring <= xs[u] - b are skipped (or null)
  const uint32_t *member;       // per-query user subsets (bitmaps), or null
  int64_t mwords;
  const int32_t *qmap;          // global query of each column (null: qa + column)
  int lskip;                    // passes 2, 3: columns whose L* exceeds this are left out

  __device__ int16_t *jtab(char *S) const { return (int16_t *)S; }
  __device__ int *hist(char *S) const { return (int *)(S + sizeof(int16_t) * 2 * 128 * kJS); }
  __device__ int *lst(char *S) const { return hist(S) + 2 * kThetaBN * 32; }
  __device__ uint32_t *caps(char *S) const { return (uint32_t *)(lst(S) + kThetaBN); }
  __device__ int *qglob(char *S) const { return (int *)(caps(S) + kThetaBN); }
  __device__ tc::RowBound *qbnd(char *S) const { return (tc::RowBound *)(qglob(S) + kThetaBN); }

  // Thread et fetches words [16 et, 16 et + 16) of the 2 x 128 x 32 int16 tables
  // (JU block then JL block) of row block rb: two uint4 of each table.
  __device__ void fetch(int rb, int et, Thread &ts) const {
    const int64_t base = (int64_t)rb * tc::BM * kMaxLevels;  // int16 index of row 0
    const int64_t lim = nrows * kMaxLevels;
    for (int h = 0; h < 2; ++h) {
      int64_t e = base + (int64_t)(et * 2 + h) * 8;  // 8 int16 per uint4
      ts.pju[h] = e < lim ? *(const uint4 *)(JU + e) : make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu);
      ts.pjl[h] = e < lim ? *(const uint4 *)(JL + e) : make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu);
    }
  }
  __device__ void fetch_row(int rb, int r, Thread &ts) const {
    int64_t u = (int64_t)rb * tc::BM + r;
    if (u < nrows) {
      ts.pbf = binfp[u];
      ts.pfm = fmin[u];
      ts.prb = rowb[u];
      ts.pxs = xs ? xs[u] : -INFINITY;
    }
  }
  __device__ void unit_begin(char *S, const tc::Unit &u, int et, Thread &ts) const {
    ts.rb1 = u.rb1;
    ts.have_pf = false;
    int *QG = qglob(S);
    tc::RowBound *QB = qbnd(S);
    for (int i = et; i < kThetaBN; i += 256) {
      int64_t q = (int64_t)u.ct0 * kThetaBN + i;
      QG[i] = q < ncols ? (qmap ? qmap[q] : qa + (int)q) : 0;
      QB[i] = q < ncols ? colb[q] : tc::RowBound{0, 0, 0, 0, 0};
    }
    if (PASS == 1) {
      int *H = hist(S);
      for (int i = et; i < 2 * kThetaBN * 32; i += 256) H[i] = 0;
    } else {
      int *L = lst(S);
      uint32_t *C = caps(S);
      for (int i = et; i < kThetaBN; i += 256) {
        int64_t q = (int64_t)u.ct0 * kThetaBN + i;
        const int g = q < ncols ? (qmap ? qmap[q] : qa + (int)q) : 0;
        L[i] = q < ncols ? lstar[g] : 0;
        if (PASS == 2) C[i] = q < ncols ? cap[g] : 0u;
      }
    }
  }
  __device__ void tile_begin(char *S, int rb, int ct, int r, int h, Thread &ts) const {
    const int w = (threadIdx.x >> 5), et = threadIdx.x - 64;
    (void)w;
    if (!ts.have_pf) {
      fetch(rb, et, ts);
      fetch_row(rb, r, ts);
    }
    tc::epi_sync();  // readers of the previous tile are done with the level tables
    // scatter the 32 words this thread holds into padded rows
    int16_t *J = jtab(S);
    for (int t2 = 0; t2 < 2; ++t2) {
      const uint4 *src = t2 ? ts.pjl : ts.pju;
      for (int hh = 0; hh < 2; ++hh) {
        int e = (et * 2 + hh) * 8;       // first int16 of this uint4 inside the 128 x 32 block
        int row = e >> 5, colL = e & 31;
        const uint32_t wv[4] = {src[hh].x, src[hh].y, src[hh].z, src[hh].w};
        uint32_t *dst = (uint32_t *)(J + t2 * 128 * kJS + row * kJS + colL);
        for (int q2 = 0; q2 < 4; ++q2) dst[q2] = wv[q2];
      }
    }
    ts.u = (int64_t)rb * tc::BM + r;
    if (ts.u < nrows) {
      ts.b = tc::screen_bound_tc(ts.prb, tileb[ct], gacc, gcan);
      ts.rb = ts.prb;
      ts.bf = ts.pbf;
      ts.fm = ts.pfm;
      ts.xsb = __fsub_rd(ts.pxs, ts.b);
    }
    tc::epi_sync();
    // prefetch the next row block of this unit while this tile is processed
    ts.have_pf = rb + 1 < ts.rb1;
    if (ts.have_pf) {
      fetch(rb + 1, et, ts);
      fetch_row(rb + 1, r, ts);
    }
  }
  // The chunk's 32 columns are first tested with one compare each; the warp then
  // walks the union of its lanes' surviving columns four at a time, reloading
  // those accumulator columns together so that the four bin and level
  // computations are independent.
  __device__ void chunk(char *S, int, int ct, int r, int col, uint32_t tm, const float (&v)[32],
                        Thread &ts) const {
    const int64_t c0 = (int64_t)ct * kThetaBN + col;
    // v <= xsb: lower bound above the skip level (NaN kept)
    uint32_t pm = bitmask32([&](int j) { return !(v[j] <= ts.xsb); });
    const int64_t left = ncols - c0;
    if (left < 32) pm &= left <= 0 ? 0u : (1u << left) - 1u;
    if (ts.u >= nrows) pm = 0;
    uint32_t any = __reduce_or_sync(0xffffffffu, pm);
    while (any) {
      int jj[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        jj[i] = any ? __ffs(any) - 1 : -1;
        any &= any - 1u;
      }
      float x[4];
      tc::tmem_ld1x4(tm + (uint32_t)jj[0], tm + (uint32_t)(jj[1] < 0 ? jj[0] : jj[1]),
                     tm + (uint32_t)(jj[2] < 0 ? jj[0] : jj[2]),
                     tm + (uint32_t)(jj[3] < 0 ? jj[0] : jj[3]), x);
      bool on[4];
      int cl[4], jlo[4], jhi[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        on[i] = jj[i] >= 0 && ((pm >> (jj[i] & 31)) & 1u);
        cl[i] = col + (jj[i] < 0 ? jj[0] : jj[i]);
        on[i] = on[i] && in_subset(member, mwords, qglob(S)[cl[i]], ts.u);
        // the pair's own bound (the tile's maximum only decides the skip), so that a
        // pair's bin interval does not depend on which queries share its tile
        const float b = tc::screen_bound_tc(ts.rb, qbnd(S)[cl[i]], gacc, gcan);
        bin_interval(ts.bf, ts.fm, tau, __fsub_rd(x[i], b), __fadd_ru(x[i], b), jlo[i], jhi[i]);
      }
      const int16_t *ju = jtab(S) + r * kJS, *jl = jtab(S) + 128 * kJS + r * kJS;
      if (PASS == 1) {
        int lu[4], ll[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) { lu[i] = 0; ll[i] = 0; }
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            if (ju[lu[i] + step - 1] > jlo[i]) lu[i] += step;
            if (jl[ll[i] + step - 1] > jhi[i]) ll[i] += step;
          }
        }
        int *H = hist(S);
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (on[i]) {
            atomicAdd(&H[cl[i] * 32 + lu[i]], 1);
            atomicAdd(&H[kThetaBN * 32 + cl[i] * 32 + ll[i]], 1);
          }
      } else if (PASS == 3) {
        // level of the upper bound is L* exactly: above every smaller level's start
        uint32_t val[4];
        int Lq[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          Lq[i] = lst(S)[cl[i]];
          on[i] = on[i] && Lq[i] <= lskip && jlo[i] >= ju[Lq[i]] &&
                  (Lq[i] == 0 || jlo[i] < ju[Lq[i] - 1]);
          val[i] = on[i] ? (jlo[i] >= 1 ? thi[ts.u * tau + jlo[i] - 1] : top) : 0u;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (on[i]) refine(qglob(S)[cl[i]], val[i], Lq[i]);
      } else {
        uint32_t lb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int Lq = lst(S)[cl[i]];
          on[i] = on[i] && Lq <= lskip && jhi[i] >= jl[Lq];
          lb[i] = on[i] ? (jhi[i] < tau ? tlo[ts.u * tau + jhi[i]] : 0u) : 0u;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (on[i] && lb[i] <= caps(S)[cl[i]]) emit(qglob(S)[cl[i]], ts.u);
      }
    }
  }
  __device__ void refine(int q, uint64_t v, int Lq) const {
    uint64_t base, width;
    level_range(Lq, scale, base, width);
    uint64_t bkt = v >= base ? (v - base) / width : 0;
    if (bkt >= kFine) bkt = kFine - 1;
    atomicAdd(&fine[(int64_t)q * kFine + bkt], 1u);
  }
  __device__ void emit(int q, int64_t u) const {
    uint32_t pos = atomicAdd(&qcursor[q], 1u);
    int64_t at = qoff[q] + pos;
    if (at >= qoff[q + 1]) {  // more than the pass-1 count: never written out of the segment
      atomicExch(ovf, 1);
      return;
    }
    cand_u[at] = (int32_t)u;
    cand_q[at] = q;
  }
  __device__ void tile_end(char *, int, int, int, int, Thread &) const {}
  __device__ void unit_end(char *S, const tc::Unit &u, int et, Thread &) const {
    if (PASS != 1) return;
    const int *H = hist(S);
    const int *QG = qglob(S);
    for (int i = et; i < kThetaBN * 32; i += 256) {
      int64_t q = (int64_t)u.ct0 * kThetaBN + (i >> 5);
      if (q >= ncols) continue;
      const int64_t g = QG[i >> 5];
      int a = H[i], b = H[kThetaBN * 32 + i];
      if (a) atomicAdd(&hist_up[g * 32 + (i & 31)], (uint32_t)a);
      if (b) atomicAdd(&hist_lo[g * 32 + (i & 31)], (uint32_t)b);
    }
  }
};

template <int PASS>
static rkr_status theta_launch(const rkr_index *idx, const TcSide &Ut, const TcSide &Qt,
                               const ThetaArgs &a, int split, int *err, cudaStream_t st) {
  const int64_t n = idx->n, nq = Qt.rows;
  tc::RowBound *tb = nullptr;
  RKR_TRY(tc_tile_bounds(Qt, kThetaBN, split, &tb, st));
  int nct = (int)((nq + kThetaBN - 1) / kThetaBN);
  int parts = std::max(1, (2 * sm_count() + nct - 1) / nct);
  tc::Schedule sch = col_schedule(n, nq, kThetaBN, parts);
  EpiTheta<PASS> e;
  e.nrows = n; e.ncols = nq; e.tau = a.tau; e.qa = a.qa;
  e.rowb = split ? Ut.rb3 : Ut.rb1; e.tileb = tb;
  e.colb = split ? Qt.rb3 : Qt.rb1;
  e.gacc = tc_gacc(Ut.kp, split); e.gcan = tc_gcan(idx->d);
  e.binfp = a.binfp; e.fmin = a.fmin; e.JU = a.JU; e.JL = a.JL;
  e.thi = a.thi; e.tlo = a.tlo; e.top = a.top; e.scale = a.scale;
  e.hist_up = a.hist; e.hist_lo = a.hist ? a.hist + (size_t)a.nq_all * 32 : nullptr;
  e.xs = a.xs; e.qmap = a.qmap; e.lskip = a.lskip; e.ovf = a.ovf;
  e.member = a.member; e.mwords = a.mwords;
  e.lstar = a.lstar; e.cap = a.cap; e.fine = a.fine;
  e.qoff = a.qoff; e.qcursor = a.qcursor; e.cand_u = a.cand_u; e.cand_q = a.cand_q;
  static_assert(tc::screen_smem_bytes<kThetaBN, 4, EpiTheta<1>>() <= 232448, "theta smem");
  rkr_status s = launch_screen<kThetaBN, 4>(Ut, Qt, split, sch, e, err, st);
  cudaFreeAsync(tb, st);
  return s;
}

rkr_status tc_theta_pass(int pass, const rkr_index *idx, const TcSide &Ut, const TcSide &Qt,
                         const ThetaArgs &a, int split, int *err, cudaStream_t st) {
  if (pass == 1) return theta_launch<1>(idx, Ut, Qt, a, split, err, st);
  if (pass == 2) return theta_launch<2>(idx, Ut, Qt, a, split, err, st);
  return theta_launch<3>(idx, Ut, Qt, a, split, err, st);
}

// ============================================================ rank table

// Alg. 1 step 3 / Eq. 1 on the tensor cores: for every (user, sampled row) the
// number of thresholds the score exceeds, c = #{j : s(u,p) > t_j}, decided by
// the split screen with the pair's own bound when its bin interval is a single
// value; W[u][c] += weight of the sample with a global reduction.  Undecided
// pairs are queued for the canonical FP64 evaluation.
struct EpiTable {
  static const char *name() { return "k_screen<EpiTable>"; }
  struct Thread {
    int64_t u;
    tc::RowBound ru;
    BinFP bf;
    double fm;
  };
  static constexpr size_t kSmem = 0;
  int64_t nrows, ncols;
  int tau;
  const tc::RowBound *rowb, *colb;
  tc::Gacc gacc;
  float gcan;
  const BinFP *binfp;
  const double *fmin;
  const uint32_t *w;        // weight of each sampled row
  uint32_t *W;              // n x (tau + 1)
  PairQueue q;
  __device__ __forceinline__ void unit_begin(char *, const tc::Unit &, int, Thread &ts) const {
    ts.u = -1;
  }
  __device__ __forceinline__ void tile_begin(char *, int rb, int, int r, int, Thread &ts) const {
    const int64_t u = (int64_t)rb * tc::BM + r;
    if (u != ts.u && u < nrows) {   // the row's data, once per row
      ts.ru = rowb[u];
      ts.bf = binfp[u];
      ts.fm = fmin[u];
    }
    ts.u = u;
  }
  __device__ __forceinline__ void chunk(char *, int, int ct, int, int col, uint32_t,
                                        const float (&v)[32], Thread &ts) const {
    if (ts.u >= nrows) return;
    const int64_t c0 = (int64_t)ct * kTableBN + col;
    uint32_t *Wu = W + ts.u * (tau + 1);
    // fully unrolled with predicates so that v stays in registers
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int64_t p = c0 + j;
      if (p >= ncols) continue;
      const float b = tc::screen_bound_tc(ts.ru, colb[p], gacc, gcan);
      int jlo, jhi;
      bin_interval(ts.bf, ts.fm, tau, __fsub_rd(v[j], b), __fadd_ru(v[j], b), jlo, jhi);
      if (jlo == jhi) atomicAdd(&Wu[jlo], w[p]);
      else q.push_agg((int)ts.u, (int)p);
    }
  }
  __device__ __forceinline__ void tile_end(char *, int, int, int, int, Thread &) const {}
  __device__ __forceinline__ void unit_end(char *, const tc::Unit &, int, Thread &) const {}
  static constexpr int kTableBN = 256;
};

// The rank table with every sampled row of the same weight w (equal buckets):
// the decided pairs of a row block are counted per (user, count c) in shared
// memory, 16-bit counters packed two to a word, and each unit writes its users'
// rows W[u][c] = w * count once, instead of one global reduction per pair.
// Undecided pairs are queued exactly as in EpiTable.  Needs tau + 1 <= 512 bins
// and fewer than 2^16 sampled rows.
struct EpiTableSm {
  static const char *name() { return "k_screen<EpiTable>"; }
  static constexpr bool kResident = true;
  static constexpr int kBinWords = 256;   // 512 16-bit counters per user
  struct Thread {
    int64_t u;
    tc::RowBound ru;
    BinFP bf;
    double fm;
  };
  static constexpr size_t kSmem = sizeof(uint32_t) * tc::BM * kBinWords;
  int64_t nrows, ncols;
  int tau;
  const tc::RowBound *rowb, *colb;
  tc::Gacc gacc;
  float gcan;
  const BinFP *binfp;
  const double *fmin;
  uint32_t wconst;          // the common weight of the sampled rows
  uint32_t *W;              // n x (tau + 1)
  PairQueue q;
  __device__ void unit_begin(char *S, const tc::Unit &, int et, Thread &ts) const {
    uint32_t *H = (uint32_t *)S;
    for (int i = et; i < tc::BM * kBinWords; i += 256) H[i] = 0u;
    ts.u = -1;
  }
  __device__ __forceinline__ void tile_begin(char *, int rb, int, int r, int, Thread &ts) const {
    const int64_t u = (int64_t)rb * tc::BM + r;
    if (u != ts.u && u < nrows) {   // the row's data, once per row
      ts.ru = rowb[u];
      ts.bf = binfp[u];
      ts.fm = fmin[u];
    }
    ts.u = u;
  }
  __device__ __forceinline__ void chunk(char *S, int, int ct, int r, int col, uint32_t,
                                        const float (&v)[32], Thread &ts) const {
    if (ts.u >= nrows) return;
    const int64_t c0 = (int64_t)ct * EpiTable::kTableBN + col;
    uint32_t *H = (uint32_t *)S + r * kBinWords;
    // fully unrolled with predicates so that v stays in registers
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int64_t p = c0 + j;
      if (p >= ncols) continue;
      const float b = tc::screen_bound_tc(ts.ru, colb[p], gacc, gcan);
      int jlo, jhi;
      bin_interval(ts.bf, ts.fm, tau, __fsub_rd(v[j], b), __fadd_ru(v[j], b), jlo, jhi);
      if (jlo == jhi) atomicAdd(&H[jlo >> 1], 1u << ((jlo & 1) * 16));
      else q.push_agg((int)ts.u, (int)p);
    }
  }
  __device__ __forceinline__ void tile_end(char *, int, int, int, int, Thread &) const {}
  __device__ void unit_end(char *S, const tc::Unit &u, int et, Thread &) const {
    const uint32_t *H = (const uint32_t *)S;
    const int bins = tau + 1;
    const int64_t row0 = (int64_t)u.rb0 * tc::BM;
    for (int i = et; i < tc::BM * bins; i += 256) {
      const int r = i / bins, c = i - r * bins;
      if (row0 + r >= nrows) continue;
      const uint32_t cnt = (H[r * kBinWords + (c >> 1)] >> ((c & 1) * 16)) & 0xffffu;
      W[(row0 + r) * bins + c] = cnt * wconst;
    }
  }
};

// Queued pairs: canonical score, its threshold count, weighted add.
__global__ void k_table_resolve(const int2 *__restrict__ items,
                                const unsigned long long *__restrict__ count,
                                unsigned long long cap, const float *__restrict__ U,
                                const float *__restrict__ S, int d,
                                const double *__restrict__ fmin, const double *__restrict__ delta,
                                int tau, const uint32_t *__restrict__ w, uint32_t *__restrict__ W) {
  // c(s) = #{t_j < s} is non-decreasing in s: equal at both ends of an interval
  // holding s(u,p) means it is decided
  unsigned long long c = *count;
  if (c > cap) c = cap;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < c;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const int2 it = items[i];
    const int64_t u = it.x;
    const float *uu = U + u * d, *pp = S + (int64_t)it.y * d;
    // the compensated interval decides almost every pair; canonical FP64 otherwise
    double lo, hi;
    dot2_interval(uu, pp, d, lo, hi);
    int c;
    const int clo = exact_c(lo, fmin[u], delta[u], tau), chi = exact_c(hi, fmin[u], delta[u], tau);
    if (clo == chi) {
      c = clo;
    } else {
      c = exact_c(canon_dot(uu, pp, d), fmin[u], delta[u], tau);
    }
    atomicAdd(&W[u * (tau + 1) + c], w[it.y]);
  }
}

// N[u][j] = sum_{c > j} W[u][c], j < tau: one warp per user.
__global__ void k_table_suffix(int64_t n, int tau, const uint32_t *__restrict__ W,
                               uint32_t *__restrict__ N) {
  const int64_t u = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (u >= n) return;
  const uint32_t *Wu = W + u * (tau + 1);
  const int chunk = (tau + 1 + 31) / 32;
  const int c0 = lane * chunk, c1 = min(tau + 1, c0 + chunk);
  uint32_t part = 0;
  for (int c = c0; c < c1; ++c) part += Wu[c];
  uint32_t incl = part;  // inclusive suffix over lanes >= lane
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t x = __shfl_down_sync(0xffffffffu, incl, o);
    if (lane + o < 32) incl += x;
  }
  uint32_t run = incl - part;
  for (int c = c1 - 1; c >= c0; --c) {
    run += Wu[c];
    if (c >= 1) N[u * tau + (c - 1)] = run;
  }
}

rkr_status tc_rank_table(const rkr_index *idx, const TcSide &Ut, cudaStream_t st, bool *done) {
  *done = false;
  const int64_t n = idx->n;
  const int tau = idx->tau, nsamp = idx->nsamp;
  TcSide St;
  struct Guard {
    TcSide *s;
    ~Guard() { tc_free(*s); }
  } g{&St};
  RKR_TRY(tc_stage(idx->S, nsamp, idx->d, St, st));
  uint32_t *W = nullptr;
  int2 *qitems = nullptr;
  unsigned long long *qcount = nullptr;
  int *flags = nullptr;
  const unsigned long long cap =
      (unsigned long long)std::max<int64_t>(n * (int64_t)nsamp / 32, 1 << 16);
  auto cleanup = [&]() {
    for (void *p : {(void *)W, (void *)qitems, (void *)qcount, (void *)flags})
      if (p) cudaFreeAsync(p, st);
  };
  if (pool_malloc_async((void **)&W, sizeof(uint32_t) * (size_t)n * (tau + 1), st) != cudaSuccess ||
      pool_malloc_async((void **)&qitems, sizeof(int2) * cap, st) != cudaSuccess ||
      pool_malloc_async((void **)&qcount, sizeof(unsigned long long), st) != cudaSuccess ||
      pool_malloc_async((void **)&flags, sizeof(int) * 2, st) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return RKR_OK;  // not enough memory for the scratch: the CUDA-core kernel runs instead
  }
  RKR_CUDA(cudaMemsetAsync(W, 0, sizeof(uint32_t) * (size_t)n * (tau + 1), st));
  RKR_CUDA(cudaMemsetAsync(qcount, 0, sizeof(unsigned long long), st));
  RKR_CUDA(cudaMemsetAsync(flags, 0, sizeof(int) * 2, st));
  EpiTable e;
  e.nrows = n; e.ncols = nsamp; e.tau = tau;
  e.rowb = Ut.rb3; e.colb = St.rb3;
  e.gacc = tc_gacc(Ut.kp, 1); e.gcan = tc_gcan(idx->d);
  e.binfp = idx->binfp; e.fmin = idx->fmin; e.w = idx->sw; e.W = W;
  e.q = PairQueue{qitems, qcount, cap, flags + 1};
  constexpr int BN = EpiTable::kTableBN;
  // every sampled row of one weight (equal buckets): counts in shared memory
  std::vector<uint32_t> wh(nsamp);
  RKR_CUDA(cudaMemcpyAsync(wh.data(), idx->sw, sizeof(uint32_t) * nsamp, cudaMemcpyDeviceToHost,
                           st));
  RKR_CUDA(cudaStreamSynchronize(st));
  bool uniform = nsamp > 0 && nsamp < 65536 && tau + 1 <= 2 * EpiTableSm::kBinWords;
  for (int i = 1; i < nsamp && uniform; ++i) uniform = wh[i] == wh[0];
  rkr_status s;
  if (uniform) {
    EpiTableSm es;
    es.nrows = n; es.ncols = nsamp; es.tau = tau;
    es.rowb = Ut.rb3; es.colb = St.rb3;
    es.gacc = e.gacc; es.gcan = e.gcan;
    es.binfp = idx->binfp; es.fmin = idx->fmin; es.wconst = wh[0]; es.W = W;
    es.q = e.q;
    static_assert(tc::screen_smem_bytes<BN, 2, EpiTableSm>() <= 232448, "table smem");
    s = launch_screen<BN, 2>(Ut, St, 1, row_schedule(n, nsamp, BN), es, flags, st);
  } else {
    s = launch_screen<BN, 4>(Ut, St, 1, row_schedule(n, nsamp, BN), e, flags, st);
  }
  if (s == RKR_OK) {
    {
      ProfScope prof("k_table_resolve", st);
      k_table_resolve<<<8 * sm_count(), 256, 0, st>>>(qitems, qcount, cap, idx->U, idx->S, idx->d,
                                                      idx->fmin, idx->delta, tau, idx->sw, W);
    }
    note_launch();
    {
      ProfScope prof("k_table_suffix", st);
      k_table_suffix<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(n, tau, W, idx->N);
    }
    note_launch();
  }
  int hf[2] = {0, 0};
  cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, st);
  cudaError_t err = cudaStreamSynchronize(st);
  cleanup();
  if (err != cudaSuccess) return cuda_fail(err, "tc_rank_table");
  RKR_TRY(s);
  if (hf[0]) return fail(RKR_ETIMEOUT, "rank-table screen wait timed out (%d)", hf[0]);
  *done = hf[1] == 0;  // a queue overflow leaves the table to the CUDA-core kernel
  return RKR_OK;
}

// ================================================================== skim

// One screening pass that only records: every pair whose screened score passes
// the skip test (its lower rank bound may lie at or below the skip level) is
// appended as (user, query, screened score) to the list region of the CTA that
// screened it.  Levels, cutoffs, refinement and emission then run on the list
// with plain CUDA-core kernels, one thread per entry, instead of inside the
// warp-synchronous epilogue.
constexpr int kSkimBN = 256;

struct EpiSkim {
  static const char *name() { return "k_screen<EpiSkim>"; }
  struct Thread {
    float b, xsb, pxs;
    int64_t u, fu;      // current row; row whose terms prb, pxs hold
    tc::RowBound prb;
  };
  // a 32 x 32 staging tile per epilogue warp, stored [column][lane]: a lane reads
  // back its own emitted scores from shared memory, not from TMEM
  static constexpr size_t kSmem = sizeof(float) * 8 * 32 * 32;
  int64_t nrows, ncols;
  const tc::RowBound *rowb, *tileb;
  tc::Gacc gacc;
  float gcan;
  const float *xs;
  SkimList L;

  __device__ void unit_begin(char *, const tc::Unit &, int, Thread &ts) const { ts.fu = -1; }
  // row-owned units: a row's bound terms are loaded once for all its column tiles
  __device__ void tile_begin(char *, int rb, int ct, int r, int, Thread &ts) const {
    ts.u = (int64_t)rb * tc::BM + r;
    if (ts.u != ts.fu && ts.u < nrows) {
      ts.prb = rowb[ts.u];
      ts.pxs = xs[ts.u];
      ts.fu = ts.u;
    }
    if (ts.u < nrows) {
      ts.b = tc::screen_bound_tc(ts.prb, tileb[ct], gacc, gcan);
      ts.xsb = __fsub_rd(ts.pxs, ts.b);
    }
  }
  __device__ void chunk(char *S, int, int ct, int, int col, uint32_t, const float (&v)[32],
                        Thread &ts) const {
    const int64_t c0 = (int64_t)ct * kSkimBN + col;
    // v <= xsb: lower bound above the skip level (NaN kept)
    uint32_t pm = bitmask32([&](int j) { return !(v[j] <= ts.xsb); });
    const int64_t left = ncols - c0;
    if (left < 32) pm &= left <= 0 ? 0u : (1u << left) - 1u;
    if (ts.u >= nrows) pm = 0;
    // warp-aggregated reservation of this warp's entries in the CTA's region
    const int lane = threadIdx.x & 31;
    const int n = __popc(pm);
    int incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0) return;
    uint32_t base = 0;
    if (lane == 0) base = atomicAdd(&L.cnt[blockIdx.x], (uint32_t)total);
    base = __shfl_sync(0xffffffffu, base, 0);
    int64_t pos = (int64_t)base + incl - n;
    const int64_t rbase = (int64_t)blockIdx.x * L.rcap;
    // each lane walks its own emitted columns, in column order
    float *tile = (float *)S + ((threadIdx.x >> 5) - 2) * 32 * 32 + lane;
#pragma unroll
    for (int j = 0; j < 32; ++j) tile[j * 32] = v[j];
    uint32_t mine = pm;
    while (mine) {
      const int j = __ffs(mine) - 1;
      mine &= mine - 1u;
      if (pos < L.rcap) {  // entries past the region are dropped; cnt records them
        L.u[rbase + pos] = (int32_t)ts.u;
        L.q[rbase + pos] = (int32_t)(c0 + j);
        L.x[rbase + pos] = tile[j * 32];
      }
      ++pos;
    }
  }
  __device__ void tile_end(char *, int, int, int, int, Thread &) const {}
  __device__ void unit_end(char *, const tc::Unit &, int, Thread &) const {}
};

int skim_regions(int64_t n, int64_t) {
  const int nrb = (int)((n + tc::BM - 1) / tc::BM);
  return std::max(1, std::min(nrb, sm_count()));
}

rkr_status tc_skim(const rkr_index *idx, const TcSide &Ut, const TcSide &Qt, const float *xs,
                   const SkimList &list, int *err, cudaStream_t st) {
  const int64_t n = idx->n, nq = Qt.rows;
  tc::RowBound *tb = nullptr;
  RKR_TRY(tc_tile_bounds(Qt, kSkimBN, 1, &tb, st));
  // row-owned units: U is read once, the query tiles stay in L2 (a launch of
  // CTA pairs uses at most as many regions as this)
  const tc::Schedule sch = row_schedule(n, nq, kSkimBN);
  if (std::min(sch.nunits, sm_count()) != list.regions) {
    cudaFreeAsync(tb, st);
    return fail(RKR_EINTERNAL, "skim list regions do not match the launch");
  }
  EpiSkim e;
  e.nrows = n;
  e.ncols = nq;
  e.rowb = Ut.rb3;
  e.tileb = tb;
  e.gacc = tc_gacc(Ut.kp, 1);
  e.gcan = tc_gcan(idx->d);
  e.xs = xs;
  e.L = list;
  static_assert(tc::screen_smem_bytes<kSkimBN, 4, EpiSkim>() <= 232448, "skim smem");
  rkr_status s = launch_screen<kSkimBN, 4>(Ut, Qt, 1, sch, e, err, st);
  cudaFreeAsync(tb, st);
  return s;
}

// =============================================================== recount

struct EpiRC {
  static const char *name() { return "k_screen<EpiRC>"; }
  // One threshold per row (segments of one candidate): an item is certainly above
  // u.q when its lower end exceeds u.q, possibly above when its upper end does.
  struct Thread {
    float b, tdn, tup;           // bound; u.q rounded down / up to float
    int64_t sg;
    int64_t self;                // item tying exactly with u.q (never above), or -1
    uint32_t *h, *hh;
    uint32_t clo, chi;           // items certainly / possibly above u.q
    tc::RowBound ru;             // the row's bound terms
    TilePrefetch tp;             // the bound terms of the next column tile
  };
  static constexpr size_t kSmem = 0;
  int64_t nseg, ncols;
  int bn;
  const tc::RowBound *rowb, *tileb;
  tc::Gacc gacc;
  float gcan;
  const int64_t *seg_start;
  const int32_t *seg_len;
  const double *ths;
  const int32_t *seg_self;
  uint32_t *hist;
  // Bounds mode (hist_hi not null): the possibly-above count goes to hist_hi and
  // nothing is queued; exact mode queues the items between the two ends.
  uint32_t *hist_hi;
  PairQueue q;
  __device__ __forceinline__ void unit_begin(char *, const tc::Unit &u, int et,
                                             Thread &ts) const {
    const int w = (et >> 5) + 2, lane = et & 31;
    const int r = (w & 3) * 32 + lane;
    ts.sg = (int64_t)u.rb0 * tc::BM + r;
    ts.clo = 0;
    ts.chi = 0;
    ts.tp.start(tileb, u.ct0);
    if (ts.sg < nseg) {
      ts.ru = rowb[ts.sg];
      const int64_t st0 = seg_start[ts.sg];
      const double t = ths[st0];
      ts.h = hist + 2 * st0;
      ts.hh = hist_hi ? hist_hi + 2 * st0 : nullptr;
      ts.tdn = __double2float_rd(t);
      ts.tup = __double2float_ru(t);
      ts.self = seg_self[ts.sg];
    } else {
      ts.self = -1;
      ts.tdn = INFINITY;
      ts.tup = INFINITY;
    }
  }
  __device__ __forceinline__ void tile_begin(char *, int, int ct, int, int, Thread &ts) const {
    const tc::RowBound tb = ts.tp.take(tileb, ct, ncols, bn);
    ts.b = ts.sg < nseg ? tc::screen_bound_tc(ts.ru, tb, gacc, gcan) : 0.0f;
  }
  __device__ __forceinline__ void chunk(char *, int, int ct, int, int col, uint32_t,
                                        const float (&v)[32], Thread &ts) const {
    const int64_t c0 = (int64_t)ct * bn + col;
    uint32_t mlo = bitmask32([&](int j) { return __fsub_rd(v[j], ts.b) > ts.tup; });
    uint32_t mhi = bitmask32([&](int j) { return __fadd_ru(v[j], ts.b) > ts.tdn; });
    const int64_t left = ncols - c0;
    if (left < 32) {
      const uint32_t keep = left <= 0 ? 0u : (1u << left) - 1u;
      mlo &= keep;
      mhi &= keep;
    }
    if (ts.self >= c0 && ts.self < c0 + 32) mhi &= ~(1u << (int)(ts.self - c0));
    ts.clo += __popc(mlo);
    ts.chi += __popc(mhi);
    if (!hist_hi) {
      uint32_t und = mhi & ~mlo;
      while (und) {
        const int j = __ffs(und) - 1;
        und &= und - 1u;
        q.push((int)ts.sg, (int)(c0 + j));
      }
    }
  }
  __device__ __forceinline__ void tile_end(char *, int, int, int, int, Thread &) const {}
  __device__ __forceinline__ void unit_end(char *, const tc::Unit &, int, Thread &ts) const {
    if (ts.sg >= nseg) return;
    if (ts.clo) atomicAdd(&ts.h[1], ts.clo);      // position 1: above the one threshold
    if (ts.hh && ts.chi) atomicAdd(&ts.hh[1], ts.chi);
  }
};


// Several thresholds per row (segments of one user's candidates, at most
// kRecountSeg, sorted ascending): the user's scores are compared with all of
// them.  Per item, pos_lo = #{i : t_i certainly below the score} and pos_hi =
// #{i : t_i possibly below it} (binary searches over the row's thresholds in
// shared memory); the position histograms of the row give the counts after a
// suffix sum.  Bounds mode histograms pos_lo and pos_hi; exact mode histograms
// the items with pos_lo = pos_hi and queues the others.  Items scoring
// certainly above every threshold are only counted, items certainly below all
// of them skipped.  The item equal to a threshold's query (its canonical score
// is that threshold) has a known position and is counted there.
struct EpiRCm {
  static const char *name() { return "k_screen<EpiRCm>"; }
  static constexpr int kL = kRecountSeg;
  struct Thread {
    float b, t0, tl;     // bound; lowest threshold rounded down, highest rounded up
    int64_t sg, st0;
    int L;
    uint32_t top;        // this thread's items certainly above every threshold
    int scur, send;      // cursor over the segment's self columns
    int64_t snext;       // next self column, or INT64_MAX
    tc::RowBound ru;     // the row's bound terms
    TilePrefetch tp;     // the bound terms of the next column tile
  };
  // Per row the thresholds (rounded down; +inf beyond L, so that a search over
  // all kL slots needs no bound) and the pos_lo and pos_hi histograms.  Every
  // table is stored index-major (element i of row r at i * 128 + r), so the 32
  // lanes of a warp, which hold 32 rows, always hit 32 different banks whatever
  // index each lane looks up.
  static_assert(kL == 32, "the branch-free search takes five steps");
  static constexpr size_t kThrOff = 0;
  static constexpr size_t kHloOff = kThrOff + sizeof(float) * 128 * kL;
  static constexpr size_t kHhiOff = kHloOff + sizeof(uint32_t) * 128 * (kL + 1);
  static constexpr size_t kSmem = kHhiOff + sizeof(uint32_t) * 128 * (kL + 1);
  int64_t nseg, ncols;
  int bn;
  const tc::RowBound *rowb, *tileb;
  tc::Gacc gacc;
  float gcan;
  const int64_t *seg_start;
  const int32_t *seg_len;
  const double *ths;
  const int32_t *self_col;   // per segment slot i: a self column (ascending), or -1
  const int32_t *self_pos;   // its exact position among the thresholds
  uint32_t *hist, *hist_hi;  // hist_hi null: exact mode
  PairQueue q;
  // row r's tables; element i at [i * 128]
  __device__ static float *thr(char *S, int r) { return (float *)(S + kThrOff) + r; }
  __device__ static uint32_t *hlo(char *S, int r) { return (uint32_t *)(S + kHloOff) + r; }
  __device__ static uint32_t *hhi(char *S, int r) { return (uint32_t *)(S + kHhiOff) + r; }
  // #{i < 32 : t[i] < x} over ascending t (stride 128): five branch-free steps
  __device__ static int count_below(const float *t, float x) {
    int p = 0;
#pragma unroll
    for (int step = 16; step >= 1; step >>= 1)
      p += t[(p + step - 1) * 128] < x ? step : 0;
    return p + (t[p * 128] < x ? 1 : 0);
  }
  __device__ void next_self(Thread &ts) const {
    ++ts.scur;
    const int c = ts.scur < ts.send ? self_col[ts.scur] : -1;
    ts.snext = c >= 0 ? (int64_t)c : INT64_MAX;
  }
  __device__ __forceinline__ void unit_begin(char *S, const tc::Unit &u, int et,
                                             Thread &ts) const {
    const int w = (et >> 5) + 2, lane = et & 31;
    const int r = (w & 3) * 32 + lane, half = et >> 7;
    ts.sg = (int64_t)u.rb0 * tc::BM + r;
    ts.top = 0;
    ts.L = 0;
    ts.snext = INT64_MAX;
    ts.tp.start(tileb, u.ct0);
    if (ts.sg >= nseg) return;
    ts.ru = rowb[ts.sg];
    ts.st0 = seg_start[ts.sg];
    ts.L = seg_len[ts.sg];
    const double *t = ths + ts.st0;
    ts.t0 = __double2float_rd(t[0]);
    ts.tl = __double2float_ru(t[ts.L - 1]);
    if (half == 0) {
      float *tr = thr(S, r);
      for (int i = 0; i < kL; ++i) tr[i * 128] = i < ts.L ? __double2float_rd(t[i]) : INFINITY;
      for (int i = 0; i <= ts.L; ++i) {
        hlo(S, r)[i * 128] = 0;
        hhi(S, r)[i * 128] = 0;
      }
    }
    ts.scur = (int)ts.st0 - 1;
    ts.send = (int)(ts.st0 + ts.L);
    next_self(ts);
  }
  __device__ __forceinline__ void tile_begin(char *, int, int ct, int, int, Thread &ts) const {
    const tc::RowBound tb = ts.tp.take(tileb, ct, ncols, bn);
    ts.b = ts.sg < nseg ? tc::screen_bound_tc(ts.ru, tb, gacc, gcan) : 0.0f;
  }
  __device__ __forceinline__ void chunk(char *S, int, int ct, int r, int col, uint32_t,
                                        const float (&v)[32], Thread &ts) const {
    if (ts.L == 0) return;
    const int64_t c0 = (int64_t)ct * bn + col;
    // self columns before this chunk belong to the other half of the row
    while (ts.snext < c0) next_self(ts);
    uint32_t smask = 0;
    while (ts.snext < c0 + 32) {
      smask |= 1u << (int)(ts.snext - c0);
      const int pos = self_pos[ts.scur];
      atomicAdd(&hlo(S, r)[pos * 128], 1u);
      if (hist_hi) atomicAdd(&hhi(S, r)[pos * 128], 1u);
      next_self(ts);
    }
    uint32_t any = bitmask32([&](int j) { return __fadd_ru(v[j], ts.b) > ts.t0; });
    uint32_t topm = bitmask32([&](int j) { return __fsub_rd(v[j], ts.b) > ts.tl; });
    const int64_t left = ncols - c0;
    uint32_t keep = ~smask;
    if (left < 32) keep &= left <= 0 ? 0u : (1u << left) - 1u;
    topm &= keep;
    any &= keep;
    ts.top += __popc(topm);
    const uint32_t mid = any & ~topm;
    if (!mid) return;
    const float *tr = thr(S, r);
    // every column in a static slot (no staging, no data-dependent loop); the
    // searches of different columns are independent, so their loads overlap
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      if (!((mid >> j) & 1u)) continue;
      const float lo = __fsub_rd(v[j], ts.b), hi = __fadd_ru(v[j], ts.b);
      // with d_i = t_i rounded down: lo > d_i gives lo >= next(d_i) > t_i
      // (certainly above); hi > t_i gives hi > d_i (so d_i < hi: possibly above)
      const int plo = count_below(tr, lo);
      const int phi = count_below(tr, hi);
      if (hist_hi) {
        atomicAdd(&hlo(S, r)[plo * 128], 1u);
        atomicAdd(&hhi(S, r)[phi * 128], 1u);
      } else if (plo == phi) {
        atomicAdd(&hlo(S, r)[plo * 128], 1u);
      } else {
        q.push((int)ts.sg, (int)(c0 + j));
      }
    }
  }
  __device__ __forceinline__ void tile_end(char *, int, int, int, int, Thread &) const {}
  __device__ __forceinline__ void unit_end(char *S, const tc::Unit &, int et, Thread &ts) const {
    const int w = (et >> 5) + 2, lane = et & 31;
    const int r = (w & 3) * 32 + lane, half = et >> 7;
    if (ts.L > 0 && ts.top) {
      atomicAdd(&hlo(S, r)[ts.L * 128], ts.top);
      if (hist_hi) atomicAdd(&hhi(S, r)[ts.L * 128], ts.top);
    }
    tc::epi_sync();
    if (ts.L == 0 || half != 0) return;
    // position 0 (above no threshold) is never read
    uint32_t *h = hist + 2 * ts.st0, *hh = hist_hi ? hist_hi + 2 * ts.st0 : nullptr;
    for (int i = 1; i <= ts.L; ++i) {
      const uint32_t a = hlo(S, r)[i * 128];
      if (a) atomicAdd(&h[i], a);
      if (hh) {
        const uint32_t b2 = hhi(S, r)[i * 128];
        if (b2) atomicAdd(&hh[i], b2);
      }
    }
  }
};

// Exact position of each queued score among its segment's thresholds.  A
// CUDA-core FP32 dot product with its bound settles most items; the rest are
// evaluated canonically.
__global__ void k_rc_refine(const int2 *__restrict__ items, const unsigned long long *count,
                            unsigned long long cap, const int64_t *__restrict__ seg_start,
                            const int32_t *__restrict__ seg_len,
                            const int32_t *__restrict__ seg_user, const double *__restrict__ ths,
                            const float *__restrict__ U, const float *__restrict__ unrm,
                            const float *__restrict__ Ps, const float *__restrict__ pnrm_s, int d,
                            uint32_t *__restrict__ hist, unsigned long long *nfp64) {
  unsigned long long c = *count;
  if (c > cap) c = cap;
  const float cfac = screen_cfac(d);
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < c;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    int2 it = items[i];
    int64_t st0 = seg_start[it.x];
    int L = seg_len[it.x];
    const int64_t u = seg_user[it.x];
    const float *uu = U + u * d, *pp = Ps + (int64_t)it.y * d;
    float acc = 0.0f;
    for (int k = 0; k < d; ++k) acc = fmaf(uu[k], pp[k], acc);
    float b = screen_bound(cfac, unrm[u], pnrm_s[it.y]);
    double lo = (double)__fsub_rd(acc, b), hi = (double)__fadd_ru(acc, b);
    const double *t = ths + st0;
    int a0 = 0, a1 = L;
    while (a0 < a1) { int md = (a0 + a1) >> 1; if (t[md] < lo) a0 = md + 1; else a1 = md; }
    int pa = a0;
    a1 = L;
    while (a0 < a1) { int md = (a0 + a1) >> 1; if (t[md] < hi) a0 = md + 1; else a1 = md; }
    int pos = pa;
    if (a0 != pa) {
      atomicAdd(nfp64, 1ull);
      double s = canon_dot(uu, pp, d);
      while (pos < a0 && t[pos] < s) ++pos;
    }
    atomicAdd(&hist[2 * st0 + pos], 1u);
  }
}

// Gather rows of a side: out row i = side row idx[i].
__global__ void k_gather_side(const __nv_bfloat16 *__restrict__ hi,
                              const __nv_bfloat16 *__restrict__ lo,
                              const tc::RowBound *__restrict__ rb1,
                              const tc::RowBound *__restrict__ rb3, int kp,
                              const int32_t *__restrict__ rows, int64_t count,
                              __nv_bfloat16 *__restrict__ ohi, __nv_bfloat16 *__restrict__ olo,
                              tc::RowBound *__restrict__ orb1, tc::RowBound *__restrict__ orb3) {
  int64_t i = blockIdx.x * (int64_t)blockDim.y + threadIdx.y;
  if (i >= count) return;
  int64_t src = rows[i];
  for (int k = threadIdx.x; k < kp; k += blockDim.x) {
    ohi[i * kp + k] = hi[src * kp + k];
    olo[i * kp + k] = lo[src * kp + k];
  }
  if (threadIdx.x == 0) {
    orb1[i] = rb1[src];
    orb3[i] = rb3[src];
  }
}

template <int BN, int STAGES, class Epi>
static rkr_status tc_recount_bn(const rkr_index *idx, const TcSide &Ut, const TcSide &Pt,
                                int64_t nseg, int64_t ncand, const int64_t *seg_start,
                                const int32_t *seg_len, const int32_t *seg_user,
                                const int32_t *seg_self, const double *ths, uint32_t *hist,
                                uint32_t *hist_hi, cudaStream_t st, int64_t *refined, int split,
                                const int32_t *self_col, const int32_t *self_pos);

rkr_status tc_recount(const rkr_index *idx, const TcSide &Ut, const TcSide &Pt, int64_t nseg,
                      int64_t ncand, const int64_t *seg_start, const int32_t *seg_len,
                      const int32_t *seg_user, const int32_t *seg_self, const double *ths,
                      uint32_t *hist, uint32_t *hist_hi, cudaStream_t st, int64_t *refined,
                      int split, const int32_t *self_col, const int32_t *self_pos) {
  // the exact mode places every item, so it always runs the split product
  if (!hist_hi) split = 1;
  if (self_col) {   // segments of several thresholds
    if (tuning().rc_bn == 128)
      return tc_recount_bn<128, tc::stages1<128, EpiRCm>(), EpiRCm>(
          idx, Ut, Pt, nseg, ncand, seg_start, seg_len, seg_user, seg_self, ths, hist, hist_hi,
          st, refined, split, self_col, self_pos);
    return tc_recount_bn<256, tc::stages1<256, EpiRCm>(), EpiRCm>(
        idx, Ut, Pt, nseg, ncand, seg_start, seg_len, seg_user, seg_self, ths, hist, hist_hi, st,
        refined, split, self_col, self_pos);
  }
  if (tuning().rc_bn == 128)
    return tc_recount_bn<128, 6, EpiRC>(idx, Ut, Pt, nseg, ncand, seg_start, seg_len, seg_user,
                                        seg_self, ths, hist, hist_hi, st, refined, split,
                                        nullptr, nullptr);
  return tc_recount_bn<256, 4, EpiRC>(idx, Ut, Pt, nseg, ncand, seg_start, seg_len, seg_user,
                                      seg_self, ths, hist, hist_hi, st, refined, split, nullptr,
                                      nullptr);
}

template <class Epi>
static void set_recount_fields(Epi &e, const int32_t *, const int32_t *, const int32_t *seg_self) {
  e.seg_self = seg_self;
}
template <>
void set_recount_fields<EpiRCm>(EpiRCm &e, const int32_t *self_col, const int32_t *self_pos,
                                const int32_t *) {
  e.self_col = self_col;
  e.self_pos = self_pos;
}

template <int BN, int STAGES, class Epi>
static rkr_status tc_recount_bn(const rkr_index *idx, const TcSide &Ut, const TcSide &Pt,
                                int64_t nseg, int64_t ncand, const int64_t *seg_start,
                                const int32_t *seg_len, const int32_t *seg_user,
                                const int32_t *seg_self, const double *ths, uint32_t *hist,
                                uint32_t *hist_hi, cudaStream_t st, int64_t *refined, int split,
                                const int32_t *self_col, const int32_t *self_pos) {
  const int64_t m = Pt.rows;   // all of P, or a prefix of the norm-sorted items
  if (nseg <= 0) return RKR_OK;
  TcSide A;
  A.rows = nseg;
  A.d = Ut.d;
  A.kp = Ut.kp;
  A.owned = false;
  size_t cnt = (size_t)nseg * A.kp;
  RKR_CUDA(pool_malloc_async((void **)&A.hi, cnt * 2, st));
  RKR_CUDA(pool_malloc_async((void **)&A.lo, cnt * 2, st));
  RKR_CUDA(pool_malloc_async((void **)&A.rb1, sizeof(tc::RowBound) * nseg, st));
  RKR_CUDA(pool_malloc_async((void **)&A.rb3, sizeof(tc::RowBound) * nseg, st));
  dim3 blk(32, 8);
  {
    const int prof_slot = prof_begin("k_gather_side", st);
    k_gather_side<<<(unsigned)((nseg + 7) / 8), blk, 0, st>>>(Ut.hi, Ut.lo, Ut.rb1, Ut.rb3, A.kp,
                                                               seg_user, nseg, A.hi, A.lo, A.rb1,
                                                               A.rb3);
    prof_end(prof_slot, st, 0.0);
  }
  note_launch();
  tc::RowBound *tb = nullptr;
  RKR_TRY(tc_tile_bounds(Pt, BN, split, &tb, st));
  unsigned long long *qcount;
  int2 *qitems;
  int *flags;
  const unsigned long long cap =
      hist_hi ? 1ull
              : (unsigned long long)std::min<int64_t>(std::max<int64_t>(128 * ncand, 1 << 24),
                                                      (int64_t)1 << 30);
  unsigned long long *nfp64;
  RKR_CUDA(pool_malloc_async(&nfp64, sizeof(unsigned long long), st));
  RKR_CUDA(cudaMemsetAsync(nfp64, 0, sizeof(unsigned long long), st));
  RKR_CUDA(pool_malloc_async(&qcount, sizeof(unsigned long long), st));
  RKR_CUDA(pool_malloc_async(&qitems, sizeof(int2) * cap, st));
  RKR_CUDA(pool_malloc_async(&flags, sizeof(int) * 2, st));
  RKR_CUDA(cudaMemsetAsync(qcount, 0, sizeof(unsigned long long), st));
  RKR_CUDA(cudaMemsetAsync(flags, 0, sizeof(int) * 2, st));
  Epi e;
  e.nseg = nseg; e.ncols = m; e.bn = BN; e.rowb = split ? A.rb3 : A.rb1; e.tileb = tb;
  e.gacc = tc_gacc(A.kp, split); e.gcan = tc_gcan(idx->d);
  e.seg_start = seg_start; e.seg_len = seg_len; e.ths = ths; e.hist = hist;
  e.hist_hi = hist_hi;
  set_recount_fields(e, self_col, self_pos, seg_self);
  e.q = PairQueue{qitems, qcount, cap, flags + 1};
  rkr_status s =
      launch_screen<BN, STAGES>(A, Pt, split, row_schedule(nseg, m, BN), e, flags, st);
  if (s == RKR_OK && !hist_hi) {
    {
      const int prof_slot = prof_begin("k_rc_refine", st);
      k_rc_refine<<<8 * sm_count(), 256, 0, st>>>(qitems, qcount, cap, seg_start, seg_len,
                                                  seg_user, ths, idx->U, idx->unrm, idx->Ps,
                                                  idx->pnrm_s, idx->d, hist, nfp64);
      prof_end(prof_slot, st, 0.0);
    }
    note_launch();
  }
  int hf[2] = {0, 0};
  unsigned long long hq = 0, h64 = 0;
  cudaMemcpyAsync(hf, flags, sizeof(hf), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(&hq, qcount, sizeof(hq), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(&h64, nfp64, sizeof(h64), cudaMemcpyDeviceToHost, st);
  cudaError_t err = cudaStreamSynchronize(st);
  for (void *p : {(void *)A.hi, (void *)A.lo, (void *)A.rb1, (void *)A.rb3, (void *)tb,
                  (void *)qcount, (void *)qitems, (void *)flags, (void *)nfp64})
    cudaFreeAsync(p, st);
  if (err != cudaSuccess) return cuda_fail(err, "tc_recount");
  RKR_TRY(s);
  if (hf[0]) return fail(RKR_ETIMEOUT, "recount screen wait timed out (%d)", hf[0]);
  if (hf[1]) return fail(RKR_EINTERNAL, "recount refinement queue overflow (%llu items)", hq);
  if (refined) { refined[0] = (int64_t)hq; refined[1] = (int64_t)h64; }
  return RKR_OK;
}

}  // namespace rkr
