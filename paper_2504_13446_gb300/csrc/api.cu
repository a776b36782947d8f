// api.cu -- the extern "C" entry points of librkr.so (see include/rkr.h).
//
// Argument checking, host/device staging of arrays, and dispatch to the build
// (build.cu) and query (query.cu) code.  No entry point throws or aborts.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "index.cuh"
#include "tcops.cuh"

namespace rkr {

static thread_local char g_err[512] = "";
static std::atomic<uint64_t> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

static std::atomic<uint64_t> g_allocs{0};
void note_alloc() { g_allocs.fetch_add(1, std::memory_order_relaxed); }

static std::atomic<uint64_t> g_index_serial{0};
uint64_t next_index_serial() { return g_index_serial.fetch_add(1, std::memory_order_relaxed) + 1; }

// Epilogue wait limit of the screens (rkr_set_wait_limit); negative = default.
static std::atomic<int64_t> g_epi_wait{-1};
uint32_t epi_wait_limit() {
  const int64_t v = g_epi_wait.load(std::memory_order_relaxed);
  return v < 0 ? tc::kWaitLimit : (uint32_t)v;
}

// One pool per device, created on first use with that device current; freed
// blocks stay in it for later allocations.  Falls back to the device's default
// pool if a pool cannot be created.
cudaMemPool_t lib_pool() {
  constexpr int kMaxDev = 64;
  static std::mutex mu;
  static cudaMemPool_t pools[kMaxDev] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
    cudaGetLastError();
    cudaMemPool_t d = nullptr;
    cudaDeviceGetDefaultMemPool(&d, dev < 0 ? 0 : dev);
    return d;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (!pools[dev]) {
    cudaMemPoolProps pr = {};
    pr.allocType = cudaMemAllocationTypePinned;
    pr.location.type = cudaMemLocationTypeDevice;
    pr.location.id = dev;
    cudaMemPool_t p = nullptr;
    if (cudaMemPoolCreate(&p, &pr) == cudaSuccess) {
      uint64_t keep = UINT64_MAX;
      cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
    } else {
      cudaGetLastError();
      cudaDeviceGetDefaultMemPool(&p, dev);
    }
    pools[dev] = p;
  }
  return pools[dev];
}

struct ProfRec {
  const char *name;
  cudaEvent_t a, b;
  double work;
};
static std::mutex g_prof_mu;
static bool g_prof_on = false;
static std::vector<ProfRec> g_prof;

int prof_begin(const char *name, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_prof_on) return -1;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) cudaGetLastError();
  if (cs != cudaStreamCaptureStatusNone) return -1;  // no timing events inside a graph
  ProfRec r{name, nullptr, nullptr, 0.0};
  if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  cudaEventRecord(r.a, st);
  g_prof.push_back(r);
  return (int)g_prof.size() - 1;
}

void prof_end(int slot, cudaStream_t st, double work) {
  if (slot < 0) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (slot >= (int)g_prof.size()) return;
  cudaEventRecord(g_prof[slot].b, st);
  g_prof[slot].work = work;
}

static void prof_clear() {
  for (auto &r : g_prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g_prof.clear();
}

void set_error(const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

rkr_status fail(rkr_status st, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

rkr_status cuda_fail(cudaError_t e, const char *what) {
  set_error("CUDA error %d (%s) in %s", (int)e, cudaGetErrorString(e), what);
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? RKR_ENOMEM : RKR_ECUDA;
}



// 1 if p is memory of the current device (or managed), 0 for host memory.
static int is_device(const void *p) {
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

rkr_status check_device() {
  int dev = 0;
  RKR_CUDA(cudaGetDevice(&dev));
  cudaDeviceProp pr;
  RKR_CUDA(cudaGetDeviceProperties(&pr, dev));
  if (!(pr.major == 10 && pr.minor == 3))
    return fail(RKR_EUNSUPPORTED, "device sm_%d%d: this library is built for sm_103a (GB300)",
                pr.major, pr.minor);
  return RKR_OK;
}

// A device view of a caller array: the array itself if it is device memory,
// else a stream-ordered device copy (owned here) of `bytes` bytes.
struct InView {
  const void *dev = nullptr;
  void *own = nullptr;
  cudaStream_t st = nullptr;
  rkr_status init(const void *p, size_t bytes, cudaStream_t s) {
    st = s;
    if (is_device(p)) {
      dev = p;
      return RKR_OK;
    }
    cudaError_t e = pool_malloc_async(&own, bytes ? bytes : 1, s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      own = nullptr;
      return fail(RKR_ENOMEM, "device allocation of %zu bytes failed", bytes);
    }
    RKR_CUDA(cudaMemcpyAsync(own, p, bytes, cudaMemcpyHostToDevice, s));
    dev = own;
    return RKR_OK;
  }
  ~InView() {
    if (own) cudaFreeAsync(own, st);
  }
};

// An output array: written in place if device memory, else through a device
// buffer copied back by finish().
struct OutView {
  void *user = nullptr;
  void *dev = nullptr;
  void *own = nullptr;
  size_t bytes = 0;
  cudaStream_t st = nullptr;
  rkr_status init(void *p, size_t b, cudaStream_t s) {
    user = p;
    bytes = b;
    st = s;
    if (!p) return RKR_OK;
    if (is_device(p)) {
      dev = p;
      return RKR_OK;
    }
    cudaError_t e = pool_malloc_async(&own, b ? b : 1, s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      own = nullptr;
      return fail(RKR_ENOMEM, "device allocation of %zu bytes failed", b);
    }
    dev = own;
    return RKR_OK;
  }
  rkr_status finish() {
    if (own && bytes) RKR_CUDA(cudaMemcpyAsync(user, own, bytes, cudaMemcpyDeviceToHost, st));
    return RKR_OK;
  }
  ~OutView() {
    if (own) cudaFreeAsync(own, st);
  }
};

}  // namespace rkr

using namespace rkr;

__global__ void k_check_pairs(const int32_t *__restrict__ u, const int32_t *__restrict__ q,
                              int64_t npairs, int64_t n, int nq, int *__restrict__ bad) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < npairs && (u[i] < 0 || u[i] >= n || q[i] < 0 || q[i] >= nq)) atomicExch(bad, 1);
}

static rkr_status check_pairs(const int32_t *u, const int32_t *q, int64_t npairs, int64_t n,
                              int nq, int *bad_host, cudaStream_t st) {
  int *bad = nullptr;
  RKR_CUDA(pool_malloc_async(&bad, sizeof(int), st));
  RKR_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
  k_check_pairs<<<(unsigned)((npairs + 255) / 256), 256, 0, st>>>(u, q, npairs, n, nq, bad);
  note_launch();
  RKR_CUDA(cudaMemcpyAsync(bad_host, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  cudaFreeAsync(bad, st);
  RKR_CUDA(cudaStreamSynchronize(st));
  return RKR_OK;
}

__global__ void k_gather_rows(const float *__restrict__ X, int F, const int32_t *__restrict__ rows,
                              int64_t count, float *__restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= count * F) return;
  out[i] = X[(int64_t)rows[i / F] * F + i % F];
}

static rkr_status gather_rows(const float *X, int F, const int32_t *rows, int64_t count,
                              float *out, cudaStream_t st) {
  k_gather_rows<<<(unsigned)((count * F + 255) / 256), 256, 0, st>>>(X, F, rows, count, out);
  note_launch();
  RKR_CUDA(cudaGetLastError());
  return RKR_OK;
}

extern "C" {

const char *rkr_last_error(void) { return g_err; }

const char *rkr_version(void) {
#ifdef RKR_CLUSTER_MULTICAST
  return "rkr 0.2 (sm_103a, single-GPU build: CTA pairs with cluster multicast)";
#else
  return "rkr 0.2 (sm_103a, replica build: no cluster multicast)";
#endif
}

uint64_t rkr_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

uint64_t rkr_device_allocations(void) { return g_allocs.load(std::memory_order_relaxed); }

rkr_status rkr_set_wait_limit(int64_t rounds) {
  if (rounds > (int64_t)UINT32_MAX) return fail(RKR_EINVAL, "wait limit %lld too large",
                                                (long long)rounds);
  g_epi_wait.store(rounds < 0 ? -1 : rounds, std::memory_order_relaxed);
  return RKR_OK;
}

rkr_status rkr_index_timings(const rkr_index *idx, double *out, int32_t count) {
  if (!idx || !out || count < 0) return fail(RKR_EINVAL, "null argument");
  for (int i = 0; i < count; ++i) out[i] = i < (int)(sizeof(idx->build_ms) / sizeof(double)) ? idx->build_ms[i] : 0.0;
  return RKR_OK;
}

rkr_status rkr_build(const float *U, int64_t n, const float *P, int64_t m, int32_t d,
                     const rkr_build_params *params, void *stream, rkr_index **out) {
  g_err[0] = 0;
  if (!U || !P || !params || !out) return fail(RKR_EINVAL, "null argument");
  *out = nullptr;
  if (n < 1 || m < 1 || d < 1) return fail(RKR_EINVAL, "need n, m, d >= 1");
  if (d > kMaxD) return fail(RKR_EINVAL, "d = %d exceeds the supported maximum %d", d, kMaxD);
  if (n > ((int64_t)1 << 31) - 1 || m > ((int64_t)1 << 30))
    return fail(RKR_EINVAL, "n must be < 2^31 and m <= 2^30");
  const rkr_build_params &p = *params;
  if (p.tau < 2 || p.tau > 8192) return fail(RKR_EINVAL, "tau must be in [2, 8192]");
  if (p.omega < 1 || p.omega > m) return fail(RKR_EINVAL, "omega must be in [1, m]");
  if (p.s < 1) return fail(RKR_EINVAL, "s must be >= 1");
  if ((uint64_t)m * (uint64_t)p.s >= ((uint64_t)1 << 32))
    return fail(RKR_EINVAL, "m * s must be < 2^32");
  if ((int64_t)p.omega * p.s > ((int64_t)1 << 26)) return fail(RKR_EINVAL, "omega * s too large");
  if (p.fbounds != 0 && p.fbounds != 1) return fail(RKR_EINVAL, "fbounds must be 0 or 1");
  if (p.exact_table < 0 || p.exact_table > 2) return fail(RKR_EINVAL, "exact_table must be 0, 1 or 2");
  if (p.floor_rank < 0) return fail(RKR_EINVAL, "floor_rank must be >= 0");
  RKR_TRY(check_device());
  cudaStream_t st = (cudaStream_t)stream;

  // sample positions: host copy for validation
  std::vector<int32_t> spos;
  if (p.sample_pos) {
    spos.resize((size_t)p.omega * p.s);
    if (is_device(p.sample_pos)) {
      RKR_CUDA(cudaMemcpyAsync(spos.data(), p.sample_pos, sizeof(int32_t) * spos.size(),
                               cudaMemcpyDeviceToHost, st));
      RKR_CUDA(cudaStreamSynchronize(st));
    } else {
      memcpy(spos.data(), p.sample_pos, sizeof(int32_t) * spos.size());
    }
  }
  InView vu, vp;
  RKR_TRY(vu.init(U, sizeof(float) * n * d, st));
  RKR_TRY(vp.init(P, sizeof(float) * m * d, st));
  int ok_u = 0, ok_p = 0;
  RKR_TRY(all_finite((const float *)vu.dev, n * d, &ok_u, st));
  RKR_TRY(all_finite((const float *)vp.dev, m * d, &ok_p, st));
  if (!ok_u || !ok_p) return fail(RKR_EINVAL, "U and P must be finite");

  rkr_index *idx = new (std::nothrow) rkr_index();
  if (!idx) return fail(RKR_ENOMEM, "host allocation failed");
  idx->n = n;
  idx->m = m;
  idx->d = d;
  idx->tau = p.tau;
  idx->omega = p.omega;
  idx->s = p.s;
  idx->fbounds = p.fbounds;
  idx->has_exact = p.exact_table;
  idx->floor_rank = p.floor_rank ? p.floor_rank : (int)(m / 16 > 2048 ? m / 16 : 2048);
  idx->seed = p.seed;
  idx->sampled_pos = p.sample_pos ? 1 : 0;
  rkr_status stt = build_index(idx, (const float *)vu.dev, (const float *)vp.dev, &p,
                               p.sample_pos ? spos.data() : nullptr, st);
  if (stt != RKR_OK) {
    cudaStreamSynchronize(st);
    index_release(idx);
    delete idx;
    return stt;
  }
  *out = idx;
  return RKR_OK;
}

// Subset bitmaps: block q sets the bits of query q's users; out-of-range ids flag bad.
__global__ void k_subset_bitmap(const int64_t *__restrict__ soff,
                                const int32_t *__restrict__ users, int64_t n, int64_t words,
                                uint32_t *__restrict__ member, int *__restrict__ bad) {
  const int64_t q = blockIdx.x;
  for (int64_t e = soff[q] + threadIdx.x; e < soff[q + 1]; e += blockDim.x) {
    const int64_t u = users[e];
    if (u < 0 || u >= n) {
      atomicExch(bad, 1);
      continue;
    }
    atomicOr(&member[q * words + (u >> 5)], 1u << (u & 31));
  }
}

// Per query: the number of member users and whether a bit at or beyond n is set.
__global__ void k_bitmap_count(const uint32_t *__restrict__ member, int64_t words, int64_t n,
                               unsigned long long *__restrict__ cnt, int *__restrict__ bad) {
  const int64_t q = blockIdx.x;
  const uint32_t *row = member + q * words;
  const uint32_t tail = (n & 31) ? ((1u << (n & 31)) - 1u) : 0xffffffffu;
  unsigned long long c = 0;
  for (int64_t w = threadIdx.x; w < words; w += blockDim.x) {
    uint32_t v = row[w];
    if (w == words - 1) {
      if (v & ~tail) atomicExch(bad, 1);
      v &= tail;
    }
    c += (unsigned long long)__popc(v);
  }
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(&cnt[q], c);
}

static rkr_status query_prologue(rkr_index *idx, const float *Q, int32_t nq, const int32_t *k,
                                 cudaStream_t st, std::vector<int32_t> &kh,
                                 std::vector<int64_t> &off) {
  if (!idx || !Q || !k) return fail(RKR_EINVAL, "null argument");
  if (nq < 1) return fail(RKR_EINVAL, "nq must be >= 1");
  kh.resize(nq);
  if (is_device(k)) {
    RKR_CUDA(cudaMemcpyAsync(kh.data(), k, sizeof(int32_t) * nq, cudaMemcpyDeviceToHost, st));
    RKR_CUDA(cudaStreamSynchronize(st));
  } else {
    memcpy(kh.data(), k, sizeof(int32_t) * nq);
  }
  off.assign(nq + 1, 0);
  for (int q = 0; q < nq; ++q) {
    if (kh[q] < 1 || kh[q] > idx->n || kh[q] > kMaxK)
      return fail(RKR_EINVAL, "k[%d] = %d must be in [1, min(n, %d)]", q, kh[q], kMaxK);
    off[q + 1] = off[q] + kh[q];
  }
  return RKR_OK;
}

struct QueryStage {
  InView vq, vk, vsu;
  uint32_t *member = nullptr;
  int64_t *soff = nullptr;
  float *qnrm = nullptr;
  int64_t *off_d = nullptr;
  BinFP *bf_own = nullptr, *xbf_own = nullptr;
  TcSide Qt;
  cudaStream_t st = nullptr;
  ~QueryStage() {
    if (qnrm) cudaFreeAsync(qnrm, st);
    if (off_d) cudaFreeAsync(off_d, st);
    if (bf_own) cudaFreeAsync(bf_own, st);
    if (xbf_own) cudaFreeAsync(xbf_own, st);
    if (member) cudaFreeAsync(member, st);
    if (soff) cudaFreeAsync(soff, st);
    cudaStreamSynchronize(st);
    tc_free(Qt);
  }
};

// Validate the CSR subsets (host or device arrays) against k and build the bitmaps.
static rkr_status stage_subsets(rkr_index *idx, int32_t nq, const std::vector<int32_t> &kh,
                                const int64_t *subset_offs, const int32_t *subset_users,
                                cudaStream_t st, QueryStage &qs, QueryCommon &qc) {
  if (!subset_offs || !subset_users) return fail(RKR_EINVAL, "null subset argument");
  std::vector<int64_t> so(nq + 1);
  if (is_device(subset_offs)) {
    RKR_CUDA(cudaMemcpyAsync(so.data(), subset_offs, sizeof(int64_t) * (nq + 1),
                             cudaMemcpyDeviceToHost, st));
    RKR_CUDA(cudaStreamSynchronize(st));
  } else {
    memcpy(so.data(), subset_offs, sizeof(int64_t) * (nq + 1));
  }
  if (so[0] != 0) return fail(RKR_EINVAL, "subset_offs[0] must be 0");
  for (int q = 0; q < nq; ++q) {
    if (so[q + 1] < so[q]) return fail(RKR_EINVAL, "subset_offs must be non-decreasing");
    if (kh[q] > so[q + 1] - so[q])
      return fail(RKR_EINVAL, "k[%d] = %d exceeds the subset size %lld", q, kh[q],
                  (long long)(so[q + 1] - so[q]));
  }
  const int64_t total = so[nq];
  RKR_TRY(qs.vsu.init(subset_users, sizeof(int32_t) * (size_t)std::max<int64_t>(total, 1), st));
  const int64_t words = (idx->n + 31) / 32;
  RKR_CUDA(pool_malloc_async(&qs.member, sizeof(uint32_t) * (size_t)words * nq, st));
  RKR_CUDA(cudaMemsetAsync(qs.member, 0, sizeof(uint32_t) * (size_t)words * nq, st));
  RKR_CUDA(pool_malloc_async(&qs.soff, sizeof(int64_t) * (nq + 2), st));
  int *bad = (int *)(qs.soff + nq + 1);
  RKR_CUDA(cudaMemcpyAsync(qs.soff, so.data(), sizeof(int64_t) * (nq + 1),
                           cudaMemcpyHostToDevice, st));
  RKR_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), st));
  k_subset_bitmap<<<nq, 256, 0, st>>>(qs.soff, (const int32_t *)qs.vsu.dev, idx->n, words,
                                      qs.member, bad);
  note_launch();
  RKR_CUDA(cudaGetLastError());
  int hb = 0;
  RKR_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, st));
  RKR_CUDA(cudaStreamSynchronize(st));
  if (hb) return fail(RKR_EINVAL, "subset user ids must lie in [0, n)");
  qc.member = qs.member;
  qc.mwords = words;
  return RKR_OK;
}

// Per-query subsets given directly as bitmaps (nq x words uint32, bit u of query q
// at word q * words + u / 32); host or device memory.
static rkr_status stage_bitmaps(rkr_index *idx, int32_t nq, const std::vector<int32_t> &kh,
                                const uint32_t *member, int64_t words, cudaStream_t st,
                                QueryStage &qs, QueryCommon &qc) {
  if (!member) return fail(RKR_EINVAL, "null subset bitmap");
  if (words != (idx->n + 31) / 32)
    return fail(RKR_EINVAL, "bitmap rows must have (n + 31) / 32 = %lld words",
                (long long)((idx->n + 31) / 32));
  RKR_TRY(qs.vsu.init(member, sizeof(uint32_t) * (size_t)words * nq, st));
  RKR_CUDA(pool_malloc_async(&qs.soff, sizeof(int64_t) * (nq + 1), st));
  unsigned long long *cnt = (unsigned long long *)qs.soff;
  int *bad = (int *)(qs.soff + nq);
  RKR_CUDA(cudaMemsetAsync(qs.soff, 0, sizeof(int64_t) * (nq + 1), st));
  k_bitmap_count<<<nq, 256, 0, st>>>((const uint32_t *)qs.vsu.dev, words, idx->n, cnt, bad);
  note_launch();
  RKR_CUDA(cudaGetLastError());
  std::vector<unsigned long long> hc(nq + 1);
  RKR_CUDA(cudaMemcpyAsync(hc.data(), qs.soff, sizeof(int64_t) * (nq + 1),
                           cudaMemcpyDeviceToHost, st));
  RKR_CUDA(cudaStreamSynchronize(st));
  if ((int)hc[nq]) return fail(RKR_EINVAL, "subset bitmaps set bits at or beyond n");
  for (int q = 0; q < nq; ++q)
    if ((unsigned long long)kh[q] > hc[q])
      return fail(RKR_EINVAL, "k[%d] = %d exceeds the subset size %llu", q, kh[q], hc[q]);
  qc.member = (const uint32_t *)qs.vsu.dev;
  qc.mwords = words;
  return RKR_OK;
}

static rkr_status stage_queries(rkr_index *idx, const float *Q, int nq, const int32_t *k,
                                const std::vector<int64_t> &off, cudaStream_t st,
                                QueryStage &qs, QueryCommon &qc) {
  qs.st = st;
  const int d = idx->d;
  RKR_TRY(qs.vq.init(Q, sizeof(float) * (size_t)nq * d, st));
  RKR_TRY(qs.vk.init(k, sizeof(int32_t) * nq, st));
  int ok = 0;
  RKR_TRY(all_finite((const float *)qs.vq.dev, (int64_t)nq * d, &ok, st));
  if (!ok) return fail(RKR_EINVAL, "Q must be finite");
  RKR_CUDA(pool_malloc_async(&qs.qnrm, sizeof(float) * nq, st));
  RKR_CUDA(pool_malloc_async(&qs.off_d, sizeof(int64_t) * (nq + 1), st));
  RKR_CUDA(cudaMemcpyAsync(qs.off_d, off.data(), sizeof(int64_t) * (nq + 1),
                           cudaMemcpyHostToDevice, st));
  RKR_TRY(row_norms((const float *)qs.vq.dev, nq, d, nullptr, qs.qnrm, st));
  float qmax = 0.0f;
  RKR_TRY(max_float(qs.qnrm, nq, &qmax, st));
  qc.Qd = (float *)qs.vq.dev;
  qc.qnrm = qs.qnrm;
  qc.kq_d = (int32_t *)qs.vk.dev;
  qc.out_off_d = qs.off_d;
  qc.bf = idx->binfp;
  qc.xbf = idx->xbin;
  if (qmax > idx->pmax) {  // |u.q| may exceed the range the stored bin bounds assume
    RKR_CUDA(pool_malloc_async(&qs.bf_own, sizeof(BinFP) * idx->n, st));
    RKR_TRY(make_binfp(idx, qmax, qs.bf_own, st));
    qc.bf = qs.bf_own;
    if (idx->xbin) {
      RKR_CUDA(pool_malloc_async(&qs.xbf_own, sizeof(BinFP) * idx->n, st));
      RKR_TRY(make_binfp_grid(idx, idx->xg0, idx->fmax, idx->xg, qmax, nullptr, qs.xbf_own, st));
      qc.xbf = qs.xbf_own;
    }
  }
  RKR_TRY(tc_stage(qc.Qd, nq, d, qs.Qt, st));
  RKR_TRY(tc_make_cat(qs.Qt, 2, st));
  qc.Qt = qs.Qt;
  return RKR_OK;
}

static rkr_status query_exact_impl(rkr_index *idx, const float *Q, int32_t nq, const int32_t *k,
                                   const int64_t *subset_offs, const int32_t *subset_users,
                                   bool subsets, int32_t *out_users, int32_t *out_ranks,
                                   rkr_query_stats *stats, void *stream,
                                   const uint32_t *member = nullptr, int64_t words = -1) {
  g_err[0] = 0;
  if (!out_users || !out_ranks) return fail(RKR_EINVAL, "null output");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int32_t> kh;
  std::vector<int64_t> off;
  RKR_TRY(query_prologue(idx, Q, nq, k, st, kh, off));
  if (!idx->has_exact) return fail(RKR_EINVAL, "index was built without exact_table");
  QueryStage qs;
  QueryCommon qc;
  if (subsets) RKR_TRY(stage_subsets(idx, nq, kh, subset_offs, subset_users, st, qs, qc));
  if (words >= 0) RKR_TRY(stage_bitmaps(idx, nq, kh, member, words, st, qs, qc));
  RKR_TRY(stage_queries(idx, Q, nq, k, off, st, qs, qc));
  OutView ou, orr;
  size_t tot = (size_t)off[nq];
  RKR_TRY(ou.init(out_users, sizeof(int32_t) * tot, st));
  RKR_TRY(orr.init(out_ranks, sizeof(int32_t) * tot, st));
  RKR_TRY(run_query_exact(idx, qc, nq, (int32_t *)ou.dev, (int32_t *)orr.dev, stats, st));
  RKR_TRY(ou.finish());
  RKR_TRY(orr.finish());
  RKR_CUDA(cudaStreamSynchronize(st));
  return RKR_OK;
}

static rkr_status query_approx_impl(rkr_index *idx, const float *Q, int32_t nq,
                                    const int32_t *k, const int64_t *subset_offs,
                                    const int32_t *subset_users, bool subsets, double c,
                                    int32_t *out_users, uint32_t *out_nlow, uint32_t *out_nup,
                                    double *out_est, int32_t *out_case, int32_t *out_nc,
                                    rkr_query_stats *stats, void *stream, bool single = false,
                                    const uint32_t *member = nullptr, int64_t words = -1) {
  g_err[0] = 0;
  if (!out_users) return fail(RKR_EINVAL, "null output");
  if (!(c >= 1.0) || !isfinite(c)) return fail(RKR_EINVAL, "c must be a finite value >= 1");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int32_t> kh;
  std::vector<int64_t> off;
  RKR_TRY(query_prologue(idx, Q, nq, k, st, kh, off));
  QueryStage qs;
  QueryCommon qc;
  if (subsets) RKR_TRY(stage_subsets(idx, nq, kh, subset_offs, subset_users, st, qs, qc));
  if (words >= 0) RKR_TRY(stage_bitmaps(idx, nq, kh, member, words, st, qs, qc));
  RKR_TRY(stage_queries(idx, Q, nq, k, off, st, qs, qc));
  size_t tot = (size_t)off[nq];
  OutView ou, olo, oup, oes, oca, onc;
  RKR_TRY(ou.init(out_users, sizeof(int32_t) * tot, st));
  RKR_TRY(olo.init(out_nlow, sizeof(uint32_t) * tot, st));
  RKR_TRY(oup.init(out_nup, sizeof(uint32_t) * tot, st));
  RKR_TRY(oes.init(out_est, sizeof(double) * tot, st));
  RKR_TRY(oca.init(out_case, sizeof(int32_t) * nq, st));
  RKR_TRY(onc.init(out_nc, sizeof(int32_t) * nq, st));
  if (single)
    RKR_TRY(run_query_approx_single(idx, qc, nq, c, (int32_t *)ou.dev, (uint32_t *)olo.dev,
                                    (uint32_t *)oup.dev, (double *)oes.dev, (int32_t *)oca.dev,
                                    (int32_t *)onc.dev, stats, st));
  else
    RKR_TRY(run_query_approx(idx, qc, nq, c, (int32_t *)ou.dev, (uint32_t *)olo.dev,
                             (uint32_t *)oup.dev, (double *)oes.dev, (int32_t *)oca.dev,
                             (int32_t *)onc.dev, stats, st));
  RKR_TRY(ou.finish());
  RKR_TRY(olo.finish());
  RKR_TRY(oup.finish());
  RKR_TRY(oes.finish());
  RKR_TRY(oca.finish());
  RKR_TRY(onc.finish());
  RKR_CUDA(cudaStreamSynchronize(st));
  return RKR_OK;
}

rkr_status rkr_query_exact(rkr_index *idx, const float *Q, int32_t nq, const int32_t *k,
                           int32_t *out_users, int32_t *out_ranks, rkr_query_stats *stats,
                           void *stream) {
  return query_exact_impl(idx, Q, nq, k, nullptr, nullptr, false, out_users, out_ranks, stats,
                          stream);
}

rkr_status rkr_query_exact_subsets(rkr_index *idx, const float *Q, int32_t nq, const int32_t *k,
                                   const int64_t *subset_offs, const int32_t *subset_users,
                                   int32_t *out_users, int32_t *out_ranks,
                                   rkr_query_stats *stats, void *stream) {
  return query_exact_impl(idx, Q, nq, k, subset_offs, subset_users, true, out_users, out_ranks,
                          stats, stream);
}

rkr_status rkr_query_approx(rkr_index *idx, const float *Q, int32_t nq, const int32_t *k,
                            double c, int32_t *out_users, uint32_t *out_nlow, uint32_t *out_nup,
                            double *out_est, int32_t *out_case, int32_t *out_nc,
                            rkr_query_stats *stats, void *stream) {
  return query_approx_impl(idx, Q, nq, k, nullptr, nullptr, false, c, out_users, out_nlow,
                           out_nup, out_est, out_case, out_nc, stats, stream);
}

rkr_status rkr_query_exact_bitmap(rkr_index *idx, const float *Q, int32_t nq, const int32_t *k,
                                  const uint32_t *member, int64_t words, int32_t *out_users,
                                  int32_t *out_ranks, rkr_query_stats *stats, void *stream) {
  return query_exact_impl(idx, Q, nq, k, nullptr, nullptr, false, out_users, out_ranks, stats,
                          stream, member, words < 0 ? 0 : words);
}

rkr_status rkr_query_approx_bitmap(rkr_index *idx, const float *Q, int32_t nq, const int32_t *k,
                                   const uint32_t *member, int64_t words, double c,
                                   int32_t *out_users, uint32_t *out_nlow, uint32_t *out_nup,
                                   double *out_est, int32_t *out_case, int32_t *out_nc,
                                   rkr_query_stats *stats, void *stream) {
  return query_approx_impl(idx, Q, nq, k, nullptr, nullptr, false, c, out_users, out_nlow,
                           out_nup, out_est, out_case, out_nc, stats, stream, false, member,
                           words < 0 ? 0 : words);
}

rkr_status rkr_query_approx_single(rkr_index *idx, const float *Q, int32_t nq, const int32_t *k,
                                   double c, int32_t *out_users, uint32_t *out_nlow,
                                   uint32_t *out_nup, double *out_est, int32_t *out_case,
                                   int32_t *out_nc, rkr_query_stats *stats, void *stream) {
  return query_approx_impl(idx, Q, nq, k, nullptr, nullptr, false, c, out_users, out_nlow,
                           out_nup, out_est, out_case, out_nc, stats, stream, true);
}

rkr_status rkr_query_approx_candidates(rkr_index *idx, const float *Q, int32_t nq,
                                       const int32_t *k, int64_t user_offset, int64_t capacity,
                                       int64_t *out_offs, int32_t *out_users, uint32_t *out_nlow,
                                       uint32_t *out_nup, double *out_est, void *stream) {
  g_err[0] = 0;
  if (!out_offs || !out_users || !out_nlow || !out_nup || !out_est)
    return fail(RKR_EINVAL, "null output");
  if (capacity < 0) return fail(RKR_EINVAL, "capacity must be >= 0");
  if (user_offset < 0 || idx == nullptr || user_offset + idx->n > ((int64_t)1 << 31))
    return fail(RKR_EINVAL, "user ids with this offset must fit in int32");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int32_t> kh;
  std::vector<int64_t> off;
  RKR_TRY(query_prologue(idx, Q, nq, k, st, kh, off));
  QueryStage qs;
  QueryCommon qc;
  RKR_TRY(stage_queries(idx, Q, nq, k, off, st, qs, qc));
  const size_t cap = (size_t)capacity;
  OutView ou, olo, oup, oes;
  RKR_TRY(ou.init(out_users, sizeof(int32_t) * cap, st));
  RKR_TRY(olo.init(out_nlow, sizeof(uint32_t) * cap, st));
  RKR_TRY(oup.init(out_nup, sizeof(uint32_t) * cap, st));
  RKR_TRY(oes.init(out_est, sizeof(double) * cap, st));
  std::vector<int64_t> offs(nq + 1, 0);
  const rkr_status rs = run_query_approx_candidates(
      idx, qc, nq, user_offset, capacity, offs.data(), (int32_t *)ou.dev, (uint32_t *)olo.dev,
      (uint32_t *)oup.dev, (double *)oes.dev, st);
  // the offsets are written even when the capacity was too small (they give the size)
  if (is_device(out_offs))
    RKR_CUDA(cudaMemcpyAsync(out_offs, offs.data(), sizeof(int64_t) * (nq + 1),
                             cudaMemcpyHostToDevice, st));
  else
    memcpy(out_offs, offs.data(), sizeof(int64_t) * (nq + 1));
  if (rs != RKR_OK) {
    RKR_CUDA(cudaStreamSynchronize(st));
    return rs;
  }
  const size_t tot = (size_t)offs[nq];
  ou.bytes = sizeof(int32_t) * tot;
  olo.bytes = sizeof(uint32_t) * tot;
  oup.bytes = sizeof(uint32_t) * tot;
  oes.bytes = sizeof(double) * tot;
  RKR_TRY(ou.finish());
  RKR_TRY(olo.finish());
  RKR_TRY(oup.finish());
  RKR_TRY(oes.finish());
  RKR_CUDA(cudaStreamSynchronize(st));
  return RKR_OK;
}

rkr_status rkr_query_approx_subsets(rkr_index *idx, const float *Q, int32_t nq,
                                    const int32_t *k, const int64_t *subset_offs,
                                    const int32_t *subset_users, double c, int32_t *out_users,
                                    uint32_t *out_nlow, uint32_t *out_nup, double *out_est,
                                    int32_t *out_case, int32_t *out_nc, rkr_query_stats *stats,
                                    void *stream) {
  return query_approx_impl(idx, Q, nq, k, subset_offs, subset_users, true, c, out_users,
                           out_nlow, out_nup, out_est, out_case, out_nc, stats, stream);
}

rkr_status rkr_rank_pairs(rkr_index *idx, const float *Q, int32_t nq, int64_t npairs,
                          const int32_t *pair_user, const int32_t *pair_query, int32_t *out_rank,
                          void *stream) {
  g_err[0] = 0;
  if (!idx || !Q || !pair_user || !pair_query || !out_rank)
    return fail(RKR_EINVAL, "null argument");
  if (nq < 1 || npairs < 0) return fail(RKR_EINVAL, "bad sizes");
  if (!idx->has_exact) return fail(RKR_EINVAL, "index was built without exact_table");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int32_t> kh(nq, 1);
  std::vector<int64_t> off(nq + 1, 0);
  for (int q = 0; q < nq; ++q) off[q + 1] = q + 1;
  QueryStage qs;
  QueryCommon qc;
  RKR_TRY(stage_queries(idx, Q, nq, kh.data(), off, st, qs, qc));
  if (npairs == 0) return RKR_OK;
  InView vu, vq;
  RKR_TRY(vu.init(pair_user, sizeof(int32_t) * npairs, st));
  RKR_TRY(vq.init(pair_query, sizeof(int32_t) * npairs, st));
  int bad = 0;
  RKR_TRY(check_pairs((const int32_t *)vu.dev, (const int32_t *)vq.dev, npairs, idx->n, nq,
                      &bad, st));
  if (bad) return fail(RKR_EINVAL, "pair user or query index out of range");
  OutView orr;
  RKR_TRY(orr.init(out_rank, sizeof(int32_t) * npairs, st));
  RKR_TRY(run_rank_pairs(idx, qc, nq, npairs, (const int32_t *)vu.dev, (const int32_t *)vq.dev,
                         (int32_t *)orr.dev, st));
  RKR_TRY(orr.finish());
  RKR_CUDA(cudaStreamSynchronize(st));
  return RKR_OK;
}

rkr_status rkr_pair_features(rkr_index *idx, const float *R, const float *Q, int32_t nq,
                             int64_t npairs, const int32_t *pair_user, const int32_t *pair_query,
                             float *out_X, float *out_t, void *stream) {
  g_err[0] = 0;
  if (!idx || !R || !Q || !pair_user || !pair_query || !out_X || !out_t)
    return fail(RKR_EINVAL, "null argument");
  if (nq < 1 || npairs < 0) return fail(RKR_EINVAL, "bad sizes");
  cudaStream_t st = (cudaStream_t)stream;
  if (npairs == 0) return RKR_OK;
  InView vr, vqq, vu, vq;
  RKR_TRY(vr.init(R, sizeof(float) * 64 * idx->d, st));
  RKR_TRY(vqq.init(Q, sizeof(float) * (size_t)nq * idx->d, st));
  RKR_TRY(vu.init(pair_user, sizeof(int32_t) * npairs, st));
  RKR_TRY(vq.init(pair_query, sizeof(int32_t) * npairs, st));
  int bad = 0;
  RKR_TRY(check_pairs((const int32_t *)vu.dev, (const int32_t *)vq.dev, npairs, idx->n, nq,
                      &bad, st));
  if (bad) return fail(RKR_EINVAL, "pair user or query index out of range");
  float *Xu = nullptr;
  RKR_CUDA(pool_malloc_async(&Xu, sizeof(float) * 65 * (size_t)idx->n, st));
  struct Free {
    float *p;
    cudaStream_t s;
    ~Free() { cudaFreeAsync(p, s); }
  } fr{Xu, st};
  RKR_TRY(user_features(idx, (const float *)vr.dev, Xu, st));
  OutView ox, ot;
  RKR_TRY(ox.init(out_X, sizeof(float) * 65 * (size_t)npairs, st));
  RKR_TRY(ot.init(out_t, sizeof(float) * npairs, st));
  RKR_TRY(gather_rows(Xu, 65, (const int32_t *)vu.dev, npairs, (float *)ox.dev, st));
  RKR_TRY(pair_scores(idx, (const float *)vqq.dev, npairs, (const int32_t *)vu.dev,
                      (const int32_t *)vq.dev, (float *)ot.dev, st));
  RKR_TRY(ox.finish());
  RKR_TRY(ot.finish());
  RKR_CUDA(cudaStreamSynchronize(st));
  return RKR_OK;
}

rkr_status rkr_query_exact_learned(rkr_index *idx, rkr_pruner *pr, const float *R, const float *Q,
                                   int32_t nq, const int32_t *k, const int32_t *keep,
                                   int32_t certify, int32_t *out_users, int32_t *out_ranks,
                                   rkr_query_stats *stats, void *stream) {
  g_err[0] = 0;
  if (!pr || !R || !keep || !out_users || !out_ranks) return fail(RKR_EINVAL, "null argument");
  if (pruner_features(pr) != 65) return fail(RKR_EINVAL, "the pruner must take 65 features");
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<int32_t> kh;
  std::vector<int64_t> off;
  RKR_TRY(query_prologue(idx, Q, nq, k, st, kh, off));
  if (!idx->has_exact) return fail(RKR_EINVAL, "index was built without exact_table");
  std::vector<int32_t> keeph(nq);
  if (is_device(keep)) {
    RKR_CUDA(cudaMemcpyAsync(keeph.data(), keep, sizeof(int32_t) * nq, cudaMemcpyDeviceToHost, st));
    RKR_CUDA(cudaStreamSynchronize(st));
  } else {
    memcpy(keeph.data(), keep, sizeof(int32_t) * nq);
  }
  for (int q = 0; q < nq; ++q)
    if (keeph[q] < kh[q])
      return fail(RKR_EINVAL, "keep[%d] = %d must be at least k[%d] = %d", q, keeph[q], q, kh[q]);
  QueryStage qs;
  QueryCommon qc;
  RKR_TRY(stage_queries(idx, Q, nq, k, off, st, qs, qc));
  InView vr;
  RKR_TRY(vr.init(R, sizeof(float) * 64 * idx->d, st));
  std::vector<float> Rh(64 * (size_t)idx->d);
  RKR_CUDA(cudaMemcpyAsync(Rh.data(), vr.dev, sizeof(float) * Rh.size(), cudaMemcpyDeviceToHost,
                           st));
  RKR_CUDA(cudaStreamSynchronize(st));
  // with tables for this index and projection the features are not needed
  const bool use_table = pruner_table_matches(pr, idx, Rh);
  float *Xu = nullptr;
  int32_t *keep_d = nullptr;
  struct Free {
    void *p;
    cudaStream_t s;
    ~Free() {
      if (p) cudaFreeAsync(p, s);
    }
  };
  if (!use_table) RKR_CUDA(pool_malloc_async(&Xu, sizeof(float) * 65 * (size_t)idx->n, st));
  Free fr{Xu, st};
  RKR_CUDA(pool_malloc_async(&keep_d, sizeof(int32_t) * nq, st));
  Free fk{keep_d, st};
  RKR_CUDA(cudaMemcpyAsync(keep_d, keeph.data(), sizeof(int32_t) * nq, cudaMemcpyHostToDevice, st));
  if (!use_table) RKR_TRY(user_features(idx, (const float *)vr.dev, Xu, st));
  OutView ou, orr;
  size_t tot = (size_t)off[nq];
  RKR_TRY(ou.init(out_users, sizeof(int32_t) * tot, st));
  RKR_TRY(orr.init(out_ranks, sizeof(int32_t) * tot, st));
  if (certify != 0 && certify != 1) return fail(RKR_EINVAL, "certify must be 0 or 1");
  RKR_TRY(run_query_exact_learned(idx, qc, nq, pr, Xu, keep_d, certify, use_table,
                                  (int32_t *)ou.dev, (int32_t *)orr.dev, stats, st));
  RKR_TRY(ou.finish());
  RKR_TRY(orr.finish());
  RKR_CUDA(cudaStreamSynchronize(st));
  return RKR_OK;
}

rkr_status rkr_pruner_invert(rkr_pruner *pr, rkr_index *idx, const float *R, int32_t G,
                             void *stream) {
  g_err[0] = 0;
  if (!pr || !idx) return fail(RKR_EINVAL, "null argument");
  if (G != 0 && (G < 2 || G > 1024)) return fail(RKR_EINVAL, "G must be 0 or in [2, 1024]");
  cudaStream_t st = (cudaStream_t)stream;
  if (G == 0) {
    RKR_CUDA(cudaStreamSynchronize(st));
    pruner_drop_table(pr);
    return RKR_OK;
  }
  if (!R) return fail(RKR_EINVAL, "null argument");
  if (pruner_features(pr) != 65) return fail(RKR_EINVAL, "the pruner must take 65 features");
  RKR_TRY(check_device());
  InView vr;
  RKR_TRY(vr.init(R, sizeof(float) * 64 * idx->d, st));
  std::vector<float> Rh(64 * (size_t)idx->d);
  RKR_CUDA(cudaMemcpyAsync(Rh.data(), vr.dev, sizeof(float) * Rh.size(), cudaMemcpyDeviceToHost,
                           st));
  float *Xu = nullptr;
  RKR_CUDA(pool_malloc_async(&Xu, sizeof(float) * 65 * (size_t)idx->n, st));
  rkr_status s = user_features(idx, (const float *)vr.dev, Xu, st);
  if (s == RKR_OK) s = pruner_build_table(pr, idx, Xu, Rh, G, st);
  cudaFreeAsync(Xu, st);
  RKR_CUDA(cudaStreamSynchronize(st));
  return s;
}

rkr_status rkr_screen_scores(const float *U, int64_t n, const float *X, int64_t mx, int32_t d,
                             int32_t split, float *out_s, float *out_b, void *stream) {
  g_err[0] = 0;
  if (!U || !X || !out_s || !out_b) return fail(RKR_EINVAL, "null argument");
  if (n < 1 || mx < 1 || d < 1 || d > kMaxD) return fail(RKR_EINVAL, "bad sizes");
  if (mx > ((int64_t)1 << 31) / n) return fail(RKR_EINVAL, "n * mx too large");
  RKR_TRY(check_device());
  cudaStream_t st = (cudaStream_t)stream;
  InView vu, vx;
  RKR_TRY(vu.init(U, sizeof(float) * n * d, st));
  RKR_TRY(vx.init(X, sizeof(float) * mx * d, st));
  OutView os, ob;
  RKR_TRY(os.init(out_s, sizeof(float) * n * mx, st));
  RKR_TRY(ob.init(out_b, sizeof(float) * n * mx, st));
  if (split < 0 || split > 2) return fail(RKR_EINVAL, "split must be 0, 1 or 2");
  TcSide A, B;
  struct Guard {
    TcSide *a, *b;
    ~Guard() { tc_free(*a); tc_free(*b); }
  } g{&A, &B};
  int *err;
  RKR_CUDA(pool_malloc_async(&err, sizeof(int), st));
  RKR_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  rkr_status r;
  if (split == 2) {
    r = tc_scores_e4m3((const float *)vu.dev, n, (const float *)vx.dev, mx, d, (float *)os.dev,
                       (float *)ob.dev, err, st);
  } else {
    RKR_TRY(tc_stage((const float *)vu.dev, n, d, A, st));
    RKR_TRY(tc_stage((const float *)vx.dev, mx, d, B, st));
    if (split == 1) {
      RKR_TRY(tc_make_cat(A, 1, st));
      RKR_TRY(tc_make_cat(B, 2, st));
    }
    r = tc_scores(A, B, split, (float *)os.dev, (float *)ob.dev, err, st);
  }
  int herr = 0;
  cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(err, st);
  RKR_CUDA(cudaStreamSynchronize(st));
  RKR_TRY(r);
  if (herr) return fail(RKR_ETIMEOUT, "screen kernel wait timed out (code %d)", herr);
  RKR_TRY(os.finish());
  RKR_TRY(ob.finish());
  RKR_CUDA(cudaStreamSynchronize(st));
  return RKR_OK;
}

rkr_status rkr_index_info(const rkr_index *idx, int64_t *out8) {
  if (!idx || !out8) return fail(RKR_EINVAL, "null argument");
  int64_t *out7 = out8;
  out8[7] = idx->xg;
  out7[0] = idx->n;
  out7[1] = idx->m;
  out7[2] = idx->d;
  out7[3] = idx->tau;
  out7[4] = idx->omega;
  out7[5] = idx->s;
  out7[6] = idx->nsamp;
  return RKR_OK;
}

rkr_status rkr_index_export(const rkr_index *idx, int32_t what, void *dst, int64_t bytes) {
  g_err[0] = 0;
  if (!idx || !dst) return fail(RKR_EINVAL, "null argument");
  const void *src = nullptr;
  int64_t size = 0;
  switch (what) {
    case RKR_EXPORT_PERM: src = idx->perm; size = 4 * idx->m; break;
    case RKR_EXPORT_FMIN: src = idx->fmin; size = 8 * idx->n; break;
    case RKR_EXPORT_FMAX: src = idx->fmax; size = 8 * idx->n; break;
    case RKR_EXPORT_TABLE: src = idx->N; size = 4 * idx->n * idx->tau; break;
    case RKR_EXPORT_SAMPLES: src = idx->samp_items; size = 4 * (int64_t)idx->nsamp; break;
    case RKR_EXPORT_XLO: src = idx->XLO; size = 4 * idx->n * (int64_t)idx->xg; break;
    case RKR_EXPORT_XHI: src = idx->XHI; size = 4 * idx->n * (int64_t)idx->xg; break;
    case RKR_EXPORT_XGRID: {
      if (!idx->xg0) return fail(RKR_EINVAL, "index has no exact table");
      if (bytes != 16 * idx->n) return fail(RKR_EINVAL, "export %d needs %lld bytes", what,
                                            (long long)(16 * idx->n));
      std::vector<double> a(idx->n), b(idx->n), o(2 * idx->n);
      RKR_CUDA(cudaMemcpy(a.data(), idx->xg0, 8 * idx->n, cudaMemcpyDeviceToHost));
      RKR_CUDA(cudaMemcpy(b.data(), idx->xdx, 8 * idx->n, cudaMemcpyDeviceToHost));
      for (int64_t i = 0; i < idx->n; ++i) { o[2 * i] = a[i]; o[2 * i + 1] = b[i]; }
      RKR_CUDA(cudaMemcpy(dst, o.data(), 16 * idx->n, cudaMemcpyDefault));
      return RKR_OK;
    }
    case RKR_EXPORT_PNORM: src = idx->pnorm; size = 8 * idx->m; break;
    case RKR_EXPORT_DLO: src = idx->DLO; size = 4 * idx->n * (int64_t)idx->dg; break;
    case RKR_EXPORT_DHI: src = idx->DHI; size = 4 * idx->n * (int64_t)idx->dg; break;
    case RKR_EXPORT_DGRID: {
      if (!idx->yg0) return fail(RKR_EINVAL, "index has no deep grid");
      if (bytes != 16 * idx->n) return fail(RKR_EINVAL, "export %d needs %lld bytes", what,
                                            (long long)(16 * idx->n));
      std::vector<double> a(idx->n), b(idx->n), o(2 * idx->n);
      RKR_CUDA(cudaMemcpy(a.data(), idx->yg0, 8 * idx->n, cudaMemcpyDeviceToHost));
      RKR_CUDA(cudaMemcpy(b.data(), idx->ydx, 8 * idx->n, cudaMemcpyDeviceToHost));
      for (int64_t i = 0; i < idx->n; ++i) { o[2 * i] = a[i]; o[2 * i + 1] = b[i]; }
      RKR_CUDA(cudaMemcpy(dst, o.data(), 16 * idx->n, cudaMemcpyDefault));
      return RKR_OK;
    }
    default: return fail(RKR_EINVAL, "unknown export %d", what);
  }
  if (!src) return fail(RKR_EINVAL, "export %d is not part of this index", what);
  if (bytes != size) return fail(RKR_EINVAL, "export %d needs %lld bytes", what, (long long)size);
  RKR_CUDA(cudaMemcpy(dst, src, (size_t)size, cudaMemcpyDefault));
  return RKR_OK;
}

rkr_status rkr_release_cached_memory(void) {
  g_err[0] = 0;
  RKR_CUDA(cudaDeviceSynchronize());
  RKR_CUDA(cudaMemPoolTrimTo(lib_pool(), 0));
  return RKR_OK;
}

void rkr_index_free(rkr_index *idx) {
  if (!idx) return;
  cudaDeviceSynchronize();
  index_release(idx);
  delete idx;
}

rkr_status rkr_profile_start(void) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  prof_clear();
  g_prof_on = true;
  return RKR_OK;
}

rkr_status rkr_profile_stop(char *report, int64_t len) {
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = false;
  struct Agg {
    std::string name;
    int64_t launches = 0;
    double ms = 0.0, work = 0.0;
  };
  std::vector<Agg> agg;
  rkr_status st = RKR_OK;
  for (auto &r : g_prof) {
    float ms = 0.0f;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.a, r.b);
    if (e != cudaSuccess) {
      st = cuda_fail(e, "rkr_profile_stop");
      continue;
    }
    Agg *a = nullptr;
    for (auto &x : agg)
      if (x.name == r.name) a = &x;
    if (!a) {
      agg.push_back(Agg{r.name});
      a = &agg.back();
    }
    a->launches += 1;
    a->ms += ms;
    a->work += r.work;
  }
  prof_clear();
  if (report && len > 0) {
    std::string out;
    char line[256];
    for (auto &a : agg) {
      snprintf(line, sizeof(line), "%s %lld %.6f %.6e\n", a.name.c_str(), (long long)a.launches,
               a.ms, a.work);
      out += line;
    }
    if ((int64_t)out.size() + 1 > len) return fail(RKR_EINVAL, "report needs %zu bytes",
                                                   out.size() + 1);
    memcpy(report, out.c_str(), out.size() + 1);
  }
  return st;
}

}  // extern "C"
