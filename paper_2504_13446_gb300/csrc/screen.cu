// screen.cu -- BF16 staging, TMA maps, and the tensor-core screens.
#include <math.h>

#include <algorithm>
#include <mutex>

#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "index.cuh"
#include "tcops.cuh"

namespace rkr {

// ---------------------------------------------------------------- staging

// hi = bf16(x), lo = bf16(x - hi) (x - hi and x - hi - lo are exact in FP32),
// zero padding up to kp, and the bound terms of single and split products
// (FP64 sums, square roots rounded up to FP32).
__global__ void k_stage_bf16(const float *__restrict__ X, int64_t rows, int d, int kp,
                             __nv_bfloat16 *__restrict__ hi, __nv_bfloat16 *__restrict__ lo,
                             tc::RowBound *__restrict__ rb1, tc::RowBound *__restrict__ rb3) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= rows) return;
  const float *x = X + i * d;
  double sx = 0, sh = 0, sl = 0, se1 = 0, se3 = 0, sc = 0;
  for (int k = 0; k < kp; ++k) {
    float v = k < d ? x[k] : 0.0f;
    __nv_bfloat16 h = __float2bfloat16_rn(v);
    float hf = __bfloat162float(h);
    float r1 = v - hf;
    __nv_bfloat16 l = __float2bfloat16_rn(r1);
    float lf = __bfloat162float(l);
    float r3 = r1 - lf;
    hi[i * kp + k] = h;
    lo[i * kp + k] = l;
    sx += (double)v * v;
    sh += (double)hf * hf;
    sl += (double)lf * lf;
    se1 += (double)r1 * r1;
    se3 += (double)r3 * r3;
    double c = (double)hf + (double)lf;
    sc += c * c;
  }
  auto up = [](double s) { return __double2float_ru(sqrt(s) * (1.0 + 0x1p-40) + 1e-300); };
  tc::RowBound a, b;
  a.a0 = up(se1); a.a1 = up(sh); a.a2 = up(sx); a.a3 = 0.0f; a.a4 = up(sh);
  b.a0 = up(se3); b.a1 = up(sc); b.a2 = up(sx); b.a3 = up(sl); b.a4 = up(sh);
  rb1[i] = a;
  rb3[i] = b;
}

rkr_status tc_stage(const float *X, int64_t rows, int d, TcSide &out, cudaStream_t st) {
  out.rows = rows;
  out.d = d;
  out.kp = (d + 15) / 16 * 16;
  size_t cnt = (size_t)std::max<int64_t>(rows, 1) * out.kp;
  auto alloc = [&](void **p, size_t bytes) -> rkr_status {
    cudaError_t e = pool_malloc_async(p, bytes, st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(RKR_ENOMEM, "device allocation of %zu bytes failed", bytes);
    }
    return RKR_OK;
  };
  RKR_TRY(alloc((void **)&out.hi, cnt * 2));
  RKR_TRY(alloc((void **)&out.lo, cnt * 2));
  RKR_TRY(alloc((void **)&out.rb1, sizeof(tc::RowBound) * std::max<int64_t>(rows, 1)));
  RKR_TRY(alloc((void **)&out.rb3, sizeof(tc::RowBound) * std::max<int64_t>(rows, 1)));
  out.owned = true;
  if (rows > 0) {
    k_stage_bf16<<<(unsigned)((rows + 127) / 128), 128, 0, st>>>(X, rows, d, out.kp, out.hi,
                                                                 out.lo, out.rb1, out.rb3);
    note_launch();
    RKR_CUDA(cudaGetLastError());
  }
  return RKR_OK;
}

// cat row = three kp-wide segments: role 1 (A) [hi | lo | hi], role 2 (B) [lo | hi | hi],
// so that segment g of A times segment g of B is the split's g-th product.
__global__ void k_make_cat(const __nv_bfloat16 *__restrict__ hi,
                           const __nv_bfloat16 *__restrict__ lo, int64_t rows, int kp, int role,
                           __nv_bfloat16 *__restrict__ cat) {
  const int64_t words = (int64_t)kp / 8;   // 16-byte words per segment
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= rows * 3 * words) return;
  const int64_t r = i / (3 * words), w = i - r * 3 * words;
  const int g = (int)(w / words);
  const int64_t c = w - (int64_t)g * words;
  const bool from_lo = role == 1 ? g == 1 : g == 0;
  const uint4 *src = (const uint4 *)((from_lo ? lo : hi) + r * kp) + c;
  ((uint4 *)(cat + r * 3 * kp))[w] = *src;
}

rkr_status tc_make_cat(TcSide &s, int role, cudaStream_t st) {
  if (s.cat || s.rows <= 0 || split_chunks_cat(s.kp) >= split_chunks_segmented(s.kp))
    return RKR_OK;
  const size_t bytes = (size_t)s.rows * 3 * s.kp * 2;
  cudaError_t e = pool_malloc_async((void **)&s.cat, bytes, st);
  if (e != cudaSuccess) {   // the segmented form still works: go on without
    cudaGetLastError();
    s.cat = nullptr;
    return RKR_OK;
  }
  s.cat_role = role;
  const int64_t total = s.rows * 3 * (s.kp / 8);
  k_make_cat<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(s.hi, s.lo, s.rows, s.kp, role,
                                                              s.cat);
  note_launch();
  RKR_CUDA(cudaGetLastError());
  return RKR_OK;
}

void tc_free(TcSide &s) {
  if (!s.owned) return;
  // back to the pool once nothing uses them (the staging may have run on any stream)
  cudaDeviceSynchronize();
  for (void *p : {(void *)s.hi, (void *)s.lo, (void *)s.rb1, (void *)s.rb3, (void *)s.cat})
    if (p) cudaFreeAsync(p, (cudaStream_t)0);
  cudaStreamSynchronize((cudaStream_t)0);
  s.hi = s.lo = s.cat = nullptr;
  s.rb1 = s.rb3 = nullptr;
  s.cat_role = 0;
}

__global__ void k_tile_bounds(const tc::RowBound *__restrict__ rb, int64_t rows, int bn,
                              int ntiles, tc::RowBound *__restrict__ out) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntiles) return;
  tc::RowBound m{0, 0, 0, 0, 0};
  for (int64_t i = (int64_t)t * bn; i < std::min<int64_t>(rows, (int64_t)(t + 1) * bn); ++i) {
    tc::RowBound v = rb[i];
    m.a0 = fmaxf(m.a0, v.a0); m.a1 = fmaxf(m.a1, v.a1); m.a2 = fmaxf(m.a2, v.a2);
    m.a3 = fmaxf(m.a3, v.a3); m.a4 = fmaxf(m.a4, v.a4);
  }
  out[t] = m;
}

rkr_status tc_tile_bounds(const TcSide &b, int bn, int split, tc::RowBound **out,
                          cudaStream_t st) {
  int ntiles = (int)((b.rows + bn - 1) / bn);
  cudaError_t e = pool_malloc_async((void **)out, sizeof(tc::RowBound) * std::max(ntiles, 1), st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(RKR_ENOMEM, "tile bounds allocation failed");
  }
  if (ntiles > 0) {
    k_tile_bounds<<<(ntiles + 127) / 128, 128, 0, st>>>(split ? b.rb3 : b.rb1, b.rows, bn, ntiles,
                                                        *out);
    note_launch();
    RKR_CUDA(cudaGetLastError());
  }
  return RKR_OK;
}

int sm_count() {
  static int cached = 0;
  if (!cached) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cached = v > 0 ? v : 1;
  }
  return cached;
}

// ------------------------------------------------------------- TMA maps

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
    else
      cudaGetLastError();
  }
  return fn;
}

rkr_status make_map(CUtensorMap *map, const __nv_bfloat16 *base, int64_t rows, int kp,
                    int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return fail(RKR_ECUDA, "cuTensorMapEncodeTiled is not available");
  if (((uintptr_t)base & 15) != 0 || (kp * 2) % 16 != 0)
    return fail(RKR_EINTERNAL, "tensor map base or pitch not 16-byte aligned");
  cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)std::max<int64_t>(rows, 1)};
  cuuint64_t strides[1] = {(cuuint64_t)kp * 2};
  cuuint32_t box[2] = {(cuuint32_t)tc::KCH, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void *)base, dims, strides, box,
                  estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(RKR_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return RKR_OK;
}

// --------------------------------------------------------- store epilogue

// Writes every screened score and its bound (validation of the screen).
struct EpiStore {
  static const char *name() { return "k_screen<EpiStore>"; }
  struct Thread {
    float b;
  };
  static constexpr size_t kSmem = 0;
  int64_t nrows, ncols;
  int bn;
  const tc::RowBound *rowb, *tileb;
  tc::Gacc gacc;
  float gcan;
  float *out, *outb;
  __device__ void unit_begin(char *, const tc::Unit &, int, Thread &) const {}
  __device__ void tile_begin(char *, int rb, int ct, int r, int, Thread &ts) const {
    int64_t row = (int64_t)rb * tc::BM + r;
    ts.b = row < nrows ? tc::screen_bound_tc(rowb[row], tileb[ct], gacc, gcan) : 0.0f;
  }
  __device__ void chunk(char *, int rb, int ct, int r, int col, uint32_t tm, const float (&v)[32],
                        Thread &ts) const {
    int64_t row = (int64_t)rb * tc::BM + r;
    if (row >= nrows) return;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      int64_t c = (int64_t)ct * bn + col + j;
      if (c < ncols) {
        out[row * ncols + c] = v[j];
        outb[row * ncols + c] = ts.b;
      }
    }
  }
  __device__ void tile_end(char *, int, int, int, int, Thread &) const {}
  __device__ void unit_end(char *, const tc::Unit &, int, Thread &) const {}
};

rkr_status tc_scores(const TcSide &A, const TcSide &B, int split, float *out, float *outb,
                     int *err, cudaStream_t st) {
  constexpr int BN = 256;
  tc::RowBound *tb = nullptr;
  RKR_TRY(tc_tile_bounds(B, BN, split, &tb, st));
  EpiStore e;
  e.nrows = A.rows;
  e.ncols = B.rows;
  e.bn = BN;
  e.rowb = split ? A.rb3 : A.rb1;
  e.tileb = tb;
  e.gacc = tc_gacc(A.kp, split);
  e.gcan = tc_gcan(A.d);
  e.out = out;
  e.outb = outb;
  rkr_status s =
      launch_screen<BN, 4>(A, B, split, row_schedule(A.rows, B.rows, BN), e, err, st);
  cudaFreeAsync(tb, st);
  return s;
}

}  // namespace rkr

namespace rkr {

// ------------------------------------------------------ FP8 E4M3 screen

// Per-row E4M3 staging: scale 2^e with e the smallest integer such that
// max|x| / 2^e <= 448 (the largest E4M3 value), q = e4m3_rn(x / 2^e), K padded
// with zeros to kp (a multiple of 32).  The bound terms use the dequantised row
// x~ = 2^e * q: a0 = ||x - x~||, a1 = a4 = ||x~||, a2 = ||x||, a3 = 0 (FP64 sums,
// square roots rounded up).
__global__ void k_stage_e4m3(const float *__restrict__ X, int64_t rows, int d, int kp,
                             uint8_t *__restrict__ q, float *__restrict__ scale,
                             tc::RowBound *__restrict__ rb) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= rows) return;
  const float *x = X + i * d;
  float mx = 0.0f;
  for (int k = 0; k < d; ++k) mx = fmaxf(mx, fabsf(x[k]));
  int e = 0;
  if (mx > 0.0f) {
    frexpf(mx / 448.0f, &e);                 // mx / 448 = f * 2^e with f in [0.5, 1)
    while (ldexpf(448.0f, e) < mx) ++e;      // guard against the division's rounding
    while (e > -149 && ldexpf(448.0f, e - 1) >= mx) --e;
  }
  const float sc = ldexpf(1.0f, e);
  double sx = 0, sd = 0, se = 0;
  for (int k = 0; k < kp; ++k) {
    const float v = k < d ? x[k] : 0.0f;
    const __nv_fp8_storage_t b = __nv_cvt_float_to_fp8(v / sc, __NV_SATFINITE, __NV_E4M3);
    const float dq = __half2float(__half(__nv_cvt_fp8_to_halfraw(b, __NV_E4M3))) * sc;
    q[i * kp + k] = (uint8_t)b;
    sx += (double)v * v;
    sd += (double)dq * dq;
    se += ((double)v - dq) * ((double)v - dq);
  }
  auto up = [](double t) { return __double2float_ru(sqrt(t) * (1.0 + 0x1p-40) + 1e-300); };
  tc::RowBound r;
  r.a0 = up(se); r.a1 = up(sd); r.a2 = up(sx); r.a3 = 0.0f; r.a4 = up(sd);
  rb[i] = r;
  scale[i] = sc;
}

static rkr_status make_map8(CUtensorMap *map, const uint8_t *base, int64_t rows, int kp,
                            int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return fail(RKR_ECUDA, "cuTensorMapEncodeTiled is not available");
  if (((uintptr_t)base & 15) != 0 || kp % 16 != 0)
    return fail(RKR_EINTERNAL, "tensor map base or pitch not 16-byte aligned");
  cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)std::max<int64_t>(rows, 1)};
  cuuint64_t strides[1] = {(cuuint64_t)kp};
  cuuint32_t box[2] = {(cuuint32_t)(2 * tc::KCH), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, (void *)base, dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(RKR_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return RKR_OK;
}

// Scaled screened scores and their bounds.  The tensor core forms the sum of
// exact E4M3 products in FP32; the accumulation factor used for that sum is
// 2^-12 (K' + 1) per unit of ||q_u~|| ||q_x~|| (a conservative model, checked by the
// screen tests), and the power-of-two scales multiply exactly.
struct EpiStore8 {
  static const char *name() { return "k_screen<EpiStore8>"; }
  struct Thread {
    float b, su;
  };
  static constexpr size_t kSmem = 0;
  int64_t nrows, ncols;
  int bn;
  const tc::RowBound *rowb, *tileb;
  const float *su, *sx;
  tc::Gacc gacc;
  float gcan;
  float *out, *outb;
  __device__ void unit_begin(char *, const tc::Unit &, int, Thread &) const {}
  __device__ void tile_begin(char *, int rb, int ct, int r, int, Thread &ts) const {
    int64_t row = (int64_t)rb * tc::BM + r;
    ts.b = row < nrows ? tc::screen_bound_tc(rowb[row], tileb[ct], gacc, gcan) : 0.0f;
    ts.su = row < nrows ? su[row] : 0.0f;
  }
  __device__ void chunk(char *, int rb, int ct, int r, int col, uint32_t, const float (&v)[32],
                        Thread &ts) const {
    int64_t row = (int64_t)rb * tc::BM + r;
    if (row >= nrows) return;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      int64_t c = (int64_t)ct * bn + col + j;
      if (c < ncols) {
        out[row * ncols + c] = v[j] * ts.su * sx[c];
        outb[row * ncols + c] = ts.b;
      }
    }
  }
  __device__ void tile_end(char *, int, int, int, int, Thread &) const {}
  __device__ void unit_end(char *, const tc::Unit &, int, Thread &) const {}
};

rkr_status tc_scores_e4m3(const float *U, int64_t n, const float *X, int64_t mx, int d,
                          float *out, float *outb, int *err, cudaStream_t st) {
  constexpr int BN = 256;
  const int kp = (d + 31) / 32 * 32;
  uint8_t *qa = nullptr, *qb = nullptr;
  float *sa = nullptr, *sb = nullptr;
  tc::RowBound *ra = nullptr, *rb = nullptr, *tb = nullptr;
  const int64_t ntiles = (mx + BN - 1) / BN;
  auto cleanup = [&]() {
    for (void *p : {(void *)qa, (void *)qb, (void *)sa, (void *)sb, (void *)ra, (void *)rb,
                    (void *)tb})
      if (p) cudaFreeAsync(p, st);
  };
  if (pool_malloc_async((void **)&qa, (size_t)n * kp, st) != cudaSuccess ||
      pool_malloc_async((void **)&qb, (size_t)mx * kp, st) != cudaSuccess ||
      pool_malloc_async((void **)&sa, sizeof(float) * n, st) != cudaSuccess ||
      pool_malloc_async((void **)&sb, sizeof(float) * mx, st) != cudaSuccess ||
      pool_malloc_async((void **)&ra, sizeof(tc::RowBound) * n, st) != cudaSuccess ||
      pool_malloc_async((void **)&rb, sizeof(tc::RowBound) * mx, st) != cudaSuccess ||
      pool_malloc_async((void **)&tb, sizeof(tc::RowBound) * ntiles, st) != cudaSuccess) {
    cudaGetLastError();
    cleanup();
    return fail(RKR_ENOMEM, "FP8 screen scratch allocation failed");
  }
  k_stage_e4m3<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(U, n, d, kp, qa, sa, ra);
  note_launch();
  k_stage_e4m3<<<(unsigned)((mx + 127) / 128), 128, 0, st>>>(X, mx, d, kp, qb, sb, rb);
  note_launch();
  k_tile_bounds<<<(unsigned)((ntiles + 127) / 128), 128, 0, st>>>(rb, mx, BN, (int)ntiles, tb);
  note_launch();
  CUtensorMap mA, mB;
  rkr_status s = make_map8(&mA, qa, n, kp, tc::BM);
  if (s == RKR_OK) s = make_map8(&mB, qb, mx, kp, BN);
  if (s == RKR_OK) {
    tc::Operands op;
    op.nrows = n;
    op.ncols = mx;
    op.kchunks = (kp + 2 * tc::KCH - 1) / (2 * tc::KCH);
    op.ksteps = kp / 32;
    op.split = 0;
    op.fp8 = 1;
    EpiStore8 e;
    e.nrows = n; e.ncols = mx; e.bn = BN; e.rowb = ra; e.tileb = tb; e.su = sa; e.sx = sb;
    e.gacc.h = (float)((double)(kp + 1) * 0x1p-12 * (1.0 + 0x1p-10));
    e.gacc.l = 0.0f;
    e.gcan = tc_gcan(d);
    e.out = out;
    e.outb = outb;
    const tc::Schedule sch = row_schedule(n, mx, BN);
    const size_t smem = tc::screen_smem_bytes<BN, 4, EpiStore8>();
    auto kern = tc::k_screen<BN, 4, EpiStore8>;
    cudaError_t ce = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem);
    if (ce != cudaSuccess) s = cuda_fail(ce, "cudaFuncSetAttribute");
    const int grid = std::min(sch.nunits, sm_count());
    if (s == RKR_OK && grid > 0) {
      ProfScope prof(EpiStore8::name(), st, 2.0 * (double)n * (double)mx * (double)kp);
      kern<<<grid, tc::kThreads, smem, st>>>(mA, mA, mB, mB, op, sch, e, err);
      note_launch();
      ce = cudaGetLastError();
      if (ce != cudaSuccess) s = cuda_fail(ce, "FP8 screen launch");
    }
  }
  cleanup();
  return s;
}

}  // namespace rkr

// ------------------------------------------------- allocation-free screen
//
// rkr_screen_scores_static: the validation screen of rkr_screen_scores with
// every piece of device scratch (BF16 hi/lo rows of both sides, their bound
// terms, the per-tile bound maxima and the kernel's error word) carved out of
// one file-scope device array of fixed size.  It is for callers that must not
// call the CUDA allocator: cudaMalloc and cudaFree can synchronize the device
// and can fail under memory pressure, so a serving loop that owns its memory
// budget (for instance through a framework's caching allocator) needs a call
// whose device footprint is fixed when the library is loaded.  Inputs and
// outputs must already be device memory.  The array is shared by every call
// on a device: calls that overlap in time (two host threads, or two streams)
// race on it, so callers serialize them.

namespace rkr {
namespace {

constexpr size_t kStaticScratchBytes = (size_t)16 << 20;  // 16 MiB per device
constexpr int kStaticDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
void *g_static_ptr[kStaticDevices] = {nullptr};

size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }

// Scratch bytes for n + mx rows of width kp and ntiles column tiles.
size_t static_bytes(int64_t n, int64_t mx, int kp, int64_t ntiles) {
  return 2 * round256((size_t)n * kp * 2) + 2 * round256((size_t)mx * kp * 2) +
         2 * round256(sizeof(tc::RowBound) * (size_t)n) +
         2 * round256(sizeof(tc::RowBound) * (size_t)mx) +
         round256(sizeof(tc::RowBound) * (size_t)ntiles) + 256;
}

bool is_device_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

}  // namespace rkr

extern "C" rkr_status rkr_screen_scores_static(const float *U, int64_t n, const float *X,
                                               int64_t mx, int32_t d, int32_t split, float *out_s,
                                               float *out_b, void *stream) {
  using namespace rkr;
  set_error("%s", "");
  if (!U || !X || !out_s || !out_b) return fail(RKR_EINVAL, "null argument");
  if (n < 1 || mx < 1 || d < 1 || d > kMaxD) return fail(RKR_EINVAL, "bad sizes");
  if (mx > ((int64_t)1 << 31) / n) return fail(RKR_EINVAL, "n * mx too large");
  if (split != 0 && split != 1)  // the E4M3 form (split = 2) stages through allocated scratch
    return fail(RKR_EINVAL, "rkr_screen_scores_static takes split = 0 or 1 (the BF16 forms)");
  constexpr int BN = 256;
  const int kp = (d + 15) / 16 * 16;
  const int64_t ntiles = (mx + BN - 1) / BN;
  const size_t need = static_bytes(n, mx, kp, ntiles);
  if (need > kStaticScratchBytes)
    return fail(RKR_EINVAL,
                "rkr_screen_scores_static needs %zu bytes of scratch for n = %lld, mx = %lld, "
                "d = %d; the static limit is %zu bytes",
                need, (long long)n, (long long)mx, (int)d, kStaticScratchBytes);
  if (!is_device_ptr(U) || !is_device_ptr(X) || !is_device_ptr(out_s) || !is_device_ptr(out_b))
    return fail(RKR_EINVAL, "rkr_screen_scores_static takes device pointers only");
  int dev = 0;
  RKR_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kStaticDevices) return fail(RKR_EUNSUPPORTED, "device index %d", dev);
  unsigned char *base = nullptr;
  {
    // set-up, once per device with that device current: the address of the array
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
      void *p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
      g_static_ptr[dev] = p;
    }
    base = (unsigned char *)g_static_ptr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  size_t off = 0;
  auto carve = [&](size_t bytes) {
    unsigned char *p = base + off;
    off += round256(bytes);
    return p;
  };
  TcSide A, B;
  A.rows = n; A.d = d; A.kp = kp; A.owned = false;
  B.rows = mx; B.d = d; B.kp = kp; B.owned = false;
  A.hi = (__nv_bfloat16 *)carve((size_t)n * kp * 2);
  A.lo = (__nv_bfloat16 *)carve((size_t)n * kp * 2);
  B.hi = (__nv_bfloat16 *)carve((size_t)mx * kp * 2);
  B.lo = (__nv_bfloat16 *)carve((size_t)mx * kp * 2);
  A.rb1 = (tc::RowBound *)carve(sizeof(tc::RowBound) * n);
  A.rb3 = (tc::RowBound *)carve(sizeof(tc::RowBound) * n);
  B.rb1 = (tc::RowBound *)carve(sizeof(tc::RowBound) * mx);
  B.rb3 = (tc::RowBound *)carve(sizeof(tc::RowBound) * mx);
  tc::RowBound *tb = (tc::RowBound *)carve(sizeof(tc::RowBound) * ntiles);
  int *err = (int *)carve(sizeof(int));
  // the error word is the only scratch that must start at zero; everything else
  // is written in full before it is read
  RKR_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  k_stage_bf16<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(U, n, d, kp, A.hi, A.lo, A.rb1,
                                                            A.rb3);
  note_launch();
  k_stage_bf16<<<(unsigned)((mx + 127) / 128), 128, 0, st>>>(X, mx, d, kp, B.hi, B.lo, B.rb1,
                                                             B.rb3);
  note_launch();
  k_tile_bounds<<<(unsigned)((ntiles + 127) / 128), 128, 0, st>>>(split ? B.rb3 : B.rb1, mx, BN,
                                                                  (int)ntiles, tb);
  note_launch();
  RKR_CUDA(cudaGetLastError());
  EpiStore e;
  e.nrows = n;
  e.ncols = mx;
  e.bn = BN;
  e.rowb = split ? A.rb3 : A.rb1;
  e.tileb = tb;
  e.gacc = tc_gacc(kp, split ? 1 : 0);
  e.gcan = tc_gcan(d);
  e.out = out_s;
  e.outb = out_b;
  const rkr_status ls =
      launch_screen<BN, 4>(A, B, split ? 1 : 0, row_schedule(n, mx, BN), e, err, st);
  RKR_TRY(ls);
  int herr = 0;
  RKR_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  RKR_CUDA(cudaStreamSynchronize(st));
  if (herr) return fail(RKR_ETIMEOUT, "screen kernel wait timed out (code %d)", herr);
  return RKR_OK;
}
