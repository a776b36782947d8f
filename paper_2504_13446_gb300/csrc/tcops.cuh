// tcops.cuh -- BF16 operands of the tensor-core screens and their launch helper.
#pragma once

#include <cuda.h>

#include "tc_screen.cuh"
#ifdef RKR_CLUSTER_MULTICAST
#include "tc_pair.cuh"
#endif

namespace rkr {

// One side of a screen: rows of bf16 hi and lo parts (row pitch kp, zero padded
// beyond d), per-row bound terms for single and split products, and TMA maps.
struct TcSide {
  int64_t rows = 0;
  int d = 0, kp = 0;
  __nv_bfloat16 *hi = nullptr, *lo = nullptr;
  tc::RowBound *rb1 = nullptr;   // single product terms
  tc::RowBound *rb3 = nullptr;   // split product terms
  // Split operand with the three products' K ranges side by side (row pitch
  // 3 kp): [hi | lo | hi] for A (cat_role 1), [lo | hi | hi] for B (cat_role 2).
  // One pass over K = 3 kp issues the split's MMAs in the same order on the same
  // slices, so the scores are bit-identical, in fewer pipeline stages when kp is
  // not a multiple of 64 (d = 200: 10 stages per tile instead of 12).
  __nv_bfloat16 *cat = nullptr;
  int cat_role = 0;
  bool owned = true;
};

// Stage float rows into a TcSide (allocates).  rows may be 0.
rkr_status tc_stage(const float *X, int64_t rows, int d, TcSide &out, cudaStream_t st);
// K chunks of one split-product tile: three segments of kp, or one of 3 kp.
inline int split_chunks_segmented(int kp) { return 3 * ((kp + 63) / 64); }
inline int split_chunks_cat(int kp) { return (3 * kp + 63) / 64; }
// Build the side's concatenated split operand for the given role (1 = A, 2 = B)
// from hi and lo (allocates); nothing is built when it would save no stage.
rkr_status tc_make_cat(TcSide &s, int role, cudaStream_t st);
void tc_free(TcSide &s);

// Per column-tile maxima of the bound terms of a side used as B with tiles of bn rows.
rkr_status tc_tile_bounds(const TcSide &b, int bn, int split, tc::RowBound **out,
                          cudaStream_t st);

// Number of SMs of the current device.
int sm_count();

// Encode a 2-D bf16 tensor map over rows x kp with boxes of 64 x box_rows.
rkr_status make_map(CUtensorMap *map, const __nv_bfloat16 *base, int64_t rows, int kp,
                    int box_rows);

// Rounds of the screens' epilogue accumulator wait before it gives up (a test
// hook set by rkr_set_wait_limit; tc::kWaitLimit unless changed).
uint32_t epi_wait_limit();

#ifdef RKR_CLUSTER_MULTICAST
// Launch a CTA-pair kernel (clusters of two, one per pair of row blocks, at most
// as many clusters as fit at once).  False when no cluster fits (nothing launched).
template <class K, class Epi>
bool launch_cluster_pairs(K kern, size_t smem, const tc::Schedule &sch, cudaStream_t st,
                          const CUtensorMap &mAh, const CUtensorMap &mAl, const CUtensorMap &mBh,
                          const CUtensorMap &mBl, const tc::Operands &op, const Epi &epi,
                          int *err_dev) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.blockDim = dim3(tc::kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cfg.gridDim = dim3(2 * (unsigned)((sm_count() + 1) / 2));
  int nclusters = 0;
  if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess) {
    (void)cudaGetLastError();
    nclusters = 0;
  }
  const int npairs = (sch.nunits + 1) / 2;
  if (nclusters < 1) return false;
  cfg.gridDim = dim3(2 * (unsigned)std::min(npairs, nclusters));
  if (cudaLaunchKernelEx(&cfg, kern, mAh, mAl, mBh, mBl, op, sch, epi, err_dev) != cudaSuccess)
    return false;
  note_launch();
  return true;
}
#endif

// Launch the screen kernel over A (users) x B (items or queries).  In the
// single-GPU build row-owned schedules run on CTA pairs, either sharing B by
// cluster multicast or as 2-SM MMAs (the tuning's screen_form), and on the
// single-CTA kernel otherwise.  Every form bounds its scores by the same bound.
template <int BN, int STAGES, class Epi>
rkr_status launch_screen(const TcSide &A, const TcSide &B, int split, const tc::Schedule &sch,
                         const Epi &epi, int *err_dev, cudaStream_t st) {
  // a split product over concatenated operands runs as one pass over K = 3 kp
  const bool cat = split == 1 && tuning().split_cat && A.cat && B.cat && A.cat_role == 1 &&
                   B.cat_role == 2;
  const __nv_bfloat16 *ah = cat ? A.cat : A.hi, *al = cat ? A.cat : A.lo;
  const __nv_bfloat16 *bh = cat ? B.cat : B.hi, *bl = cat ? B.cat : B.lo;
  const int kw = cat ? 3 * A.kp : A.kp;
  CUtensorMap mAh, mAl, mBh, mBl;
  RKR_TRY(make_map(&mAh, ah, A.rows, kw, tc::BM));
  RKR_TRY(make_map(&mAl, al, A.rows, kw, tc::BM));
  RKR_TRY(make_map(&mBh, bh, B.rows, kw, BN));
  RKR_TRY(make_map(&mBl, bl, B.rows, kw, BN));
  tc::Operands op;
  op.nrows = A.rows;
  op.ncols = B.rows;
  op.kchunks = (kw + tc::KCH - 1) / tc::KCH;
  op.ksteps = kw / 16;
  op.split = cat ? 0 : split;
  op.epi_wait = epi_wait_limit();
  const size_t smem = tc::screen_smem_bytes<BN, STAGES, Epi>();
  int grid = std::min(sch.nunits, sm_count());
  if (grid < 1) return RKR_OK;
  // the method's work: one inner product of length d per (row, column) pair,
  // whatever number of products (split) and padding of K the screen issues
  ProfScope prof(Epi::name(), st, 2.0 * (double)A.rows * (double)B.rows * (double)A.d);
#ifdef RKR_CLUSTER_MULTICAST
  const int form = tuning().screen_form;
  if (sch.mode == 0 && sch.nunits >= 2 && form == 2) {
    // row-owned units: 2-SM MMAs over CTA pairs, each CTA staging half of B
    constexpr int S2 = tc::stages2<BN, Epi>();
    const size_t smem2 = tc::screen2_smem_bytes<BN, S2, Epi>();
    auto pk = tc::k_screen_2sm<BN, S2, Epi>;
    RKR_CUDA(cudaFuncSetAttribute(pk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2));
    CUtensorMap mBh2, mBl2;
    RKR_TRY(make_map(&mBh2, bh, B.rows, kw, BN / 2));
    RKR_TRY(make_map(&mBl2, bl, B.rows, kw, BN / 2));
    if (launch_cluster_pairs(pk, smem2, sch, st, mAh, mAl, mBh2, mBl2, op, epi, err_dev))
      return RKR_OK;
    RKR_CUDA(cudaGetLastError());
  }
  if (sch.mode == 0 && sch.nunits >= 2 && form == 1) {
    // row-owned units: CTA pairs share each B chunk by multicast
    auto pk = tc::k_screen_pair<BN, STAGES, Epi>;
    RKR_CUDA(cudaFuncSetAttribute(pk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    CUtensorMap mBh2, mBl2;
    RKR_TRY(make_map(&mBh2, bh, B.rows, kw, BN / 2));
    RKR_TRY(make_map(&mBl2, bl, B.rows, kw, BN / 2));
    if (launch_cluster_pairs(pk, smem, sch, st, mAh, mAl, mBh2, mBl2, op, epi, err_dev))
      return RKR_OK;
    RKR_CUDA(cudaGetLastError());
  }
#endif
  auto kern = tc::k_screen<BN, STAGES, Epi>;
  RKR_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  kern<<<grid, tc::kThreads, smem, st>>>(mAh, mAl, mBh, mBl, op, sch, epi, err_dev);
  note_launch();
  RKR_CUDA(cudaGetLastError());
  return RKR_OK;
}

inline tc::Schedule row_schedule(int64_t rows, int64_t cols, int bn) {
  tc::Schedule s;
  s.mode = 0;
  s.nrb = (int)((rows + tc::BM - 1) / tc::BM);
  s.nct = (int)((cols + bn - 1) / bn);
  s.parts = 1;
  s.nunits = s.nrb;
  return s;
}

inline tc::Schedule col_schedule(int64_t rows, int64_t cols, int bn, int parts) {
  tc::Schedule s;
  s.mode = 1;
  s.nrb = (int)((rows + tc::BM - 1) / tc::BM);
  s.nct = (int)((cols + bn - 1) / bn);
  s.parts = std::max(1, std::min(parts, s.nrb));
  s.nunits = s.nct * s.parts;
  return s;
}

// Accumulation and canonical-rounding factors of the bound for K' products.
inline tc::Gacc tc_gacc(int kp, int split) {
  tc::Gacc g;
  g.h = (float)((double)(kp + 1) * 0x1p-22 * (1.0 + 0x1p-10));
  g.l = split ? (float)(3.0 * (double)kp * 0x1p-22 * (1.0 + 0x1p-10)) : 0.0f;
  return g;
}
inline float tc_gcan(int d) { return (float)((double)d * 0x1p-52 * 2.0); }

// FP8 E4M3 screen with per-row power-of-two scales (single product): scores and
// bounds of every pair, from FP32 rows on the device.
rkr_status tc_scores_e4m3(const float *U, int64_t n, const float *X, int64_t mx, int d,
                          float *out, float *outb, int *err, cudaStream_t st);

// Raw screened scores and bounds of every pair (validation of the screen).
rkr_status tc_scores(const TcSide &A, const TcSide &B, int split, float *out, float *outb,
                     int *err, cudaStream_t st);

}  // namespace rkr
