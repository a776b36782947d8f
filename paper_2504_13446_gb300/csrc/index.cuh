// index.cuh -- the device-resident index behind rkr_index.
#pragma once

#include <vector>

#include "common.cuh"
#include "tcops.cuh"

namespace rkr {
uint64_t next_index_serial();   // a number no other index of this process has had
}

struct rkr_index {
  uint64_t serial = rkr::next_index_serial();
  // sizes
  int64_t n = 0, m = 0;
  int d = 0;
  int tau = 0, omega = 0, s = 0;
  int fbounds = 0;
  int has_exact = 0;
  int floor_rank = 0;
  int nsamp = 0;
  int nlev_a = 0;  // levels used with the sampled table (scale s)
  int nlev_x = 0;  // levels used with the exact table (scale 1)
  uint64_t seed = 0;     // sampling seed of the build (recorded; the samples are stored)
  int sampled_pos = 0;   // 1: sample positions were given by the caller

  // items and users (device)
  float *U = nullptr;        // n x d, caller order
  float *Ps = nullptr;       // m x d, sorted by (descending norm, index)
  int32_t *perm = nullptr;   // m: original index of sorted position
  double *pnorm = nullptr;   // m: FP64 norm, original order
  float *unrm = nullptr;     // n: FP32 upper bound of ||u||
  float *pnrm_s = nullptr;   // m: FP32 upper bound of ||p||, sorted order
  float pmax = 0.0f;         // max over P of the FP32 norm bounds (host copy)

  // sampled rank table (Alg. 1)
  double *fmin = nullptr, *fmax = nullptr, *delta = nullptr;  // n
  rkr::BinFP *binfp = nullptr;                                 // n, built with R = pmax
  uint32_t *N = nullptr;       // n x tau numerators, T-hat = 1 + N / s
  int16_t *JU = nullptr;       // n x 32 level starts of the upper bound (sampled table)
  int16_t *JL = nullptr;       // n x 32 level starts of the lower bound
  float *S = nullptr;          // nsamp x d sampled rows, bucket after bucket
  float *snrm = nullptr;       // nsamp FP32 norm bounds
  uint32_t *sw = nullptr;      // nsamp weights (|P_l| or s)
  int32_t *samp_items = nullptr;  // nsamp original item index

  // exact count table on the exact grid x_j = xg0 + j * xdx, j = 0 .. xg - 1
  int xg = 0;
  double *xg0 = nullptr, *xdx = nullptr;    // n
  rkr::BinFP *xbin = nullptr;               // n, built with R = pmax
  uint32_t *XLO = nullptr, *XHI = nullptr;  // n x xg: bounds of #{p : s(u,p) > x_j}
  int16_t *XJU = nullptr, *XJL = nullptr;   // n x 32
  int32_t *xfloor = nullptr;                // n: paper column of x_0

  // deep count grid below the tail lists (exact_table = 2): y_c = yg0 + c * ydx,
  // c = 0 .. dg - 1, from the sampled table's threshold whose estimated count
  // reaches m / 8 up to x_0; DLO / DHI bound #{p : s(u,p) > y_c}
  int dg = 0;
  double *yg0 = nullptr, *ydx = nullptr;    // n
  rkr::BinFP *ybin = nullptr;               // n
  uint32_t *DLO = nullptr, *DHI = nullptr;  // n x dg

  // tail lists: per user, every item whose screened score may exceed x_0 (the
  // exact grid's floor), grouped by exact-grid column; user u's entries are
  // xlist[xloff[u] .. xloff[u] + xlcnt[u]) within a capacity xlcap[u]
  int lists = 0;
  int64_t *xloff = nullptr;                 // n + 1
  uint32_t *xlcap = nullptr;                // n
  uint2 *xlist = nullptr;                   // (item, float bits of screened score)
  uint32_t *xlcnt = nullptr;                // n: entries, > xlcap[u] marks an overflow
  uint16_t *xcoff = nullptr;                // n x (kListG + 2): start of each list column
  double *ldx = nullptr;                    // n: step of the list grid x_0 + j ldx, j < kListG
  rkr::BinFP *lbin = nullptr;               // n: bin parameters of the list grid
  float *xbmax = nullptr;                   // n: largest screen bound of a user's entries
  uint64_t *phk = nullptr;                  // hashes of the sorted item rows, ascending (phn)
  int32_t *phv = nullptr;                   // sorted-item position of each hash
  int64_t phn = 0;
  rkr::tc::RowBound *ptile3 = nullptr;      // item tile bounds of the split screen
  int ptile_bn = 0;

  // bf16 operands of the tensor-core screens
  rkr::TcSide Ut, Pt;

  // device time of the build stages (ms): items (norms, sort, gather), samples,
  // f-bounds, rank table, level tables, exact table, total
  double build_ms[8] = {0, 0, 0, 0, 0, 0, 0, 0};
};

namespace rkr {

// Free everything the index owns.
void index_release(rkr_index *idx);

// Build steps (build.cu).  All run on `st`.
rkr_status build_index(rkr_index *idx, const float *U_dev, const float *P_dev,
                       const rkr_build_params *prm, const int32_t *sample_pos_host,
                       cudaStream_t st);

// Per-batch bin parameters for values bounded by ||u|| * R (paper grid).
rkr_status make_binfp(const rkr_index *idx, float R, BinFP *out, cudaStream_t st);

// Bin parameters of a grid g0 + j * (gmax - g0) / (G - 1), j < G; writes the
// step to delta_out when it is not null.
rkr_status make_binfp_grid(const rkr_index *idx, const double *g0, const double *gmax, int G,
                           float R, double *delta_out, BinFP *out, cudaStream_t st);

// Tensor-core screens (screen_epi.cu).
rkr_status tc_fbounds(const rkr_index *idx, const TcSide &Ut, const TcSide &Pt, double *fmin,
                      double *fmax, cudaStream_t st);
// Deep count grid (DLO / DHI on y_c, grid in yg0 / ydx / ybin): one
// single-product screen of U x P whose epilogue histograms each score's grid
// interval per user; ytop[u] / ybot[u] = the grid's top point rounded up and
// its first point rounded down to float.
rkr_status tc_deep_table(rkr_index *idx, const TcSide &Ut, const TcSide &Pt, const float *ytop,
                         const float *ybot, cudaStream_t st);
rkr_status tc_exact_table(rkr_index *idx, const TcSide &Ut, const TcSide &Pt, cudaStream_t st,
                          int64_t *refined);
// Arguments of one screening pass over a query batch (see screen_epi.cu).
struct ThetaArgs {
  int qa;                       // global index of the first query of the batch slice
  const BinFP *binfp;
  const double *fmin;           // grid origin per user
  int tau;                      // grid columns
  const int16_t *JU, *JL;       // level tables
  const uint32_t *thi, *tlo;    // tables behind the upper and lower bounds (n x tau)
  uint32_t top, scale;          // upper bound below the grid; level scale
  uint32_t *hist;               // pass 1: [nq][32] upper-bound levels then [nq][32] lower
  const int32_t *lstar;         // passes 2, 3
  const uint32_t *cap;          // pass 2
  uint32_t *fine;               // pass 3: [nq][1024]
  const int64_t *qoff;          // pass 2
  uint32_t *qcursor;
  int32_t *cand_u, *cand_q;
  int nq_all;                   // queries of the whole batch (pass 1 histogram pitch)
  const float *xs;              // per-user skip scores (null: every pair is screened)
  const int32_t *qmap;          // global query of each column (null: qa + column)
  int lskip;                    // passes 2, 3: leave out queries with L* above this
  int *ovf;                     // pass 2: overflow flag of the candidate segments
  const uint32_t *member;       // per-query user subsets, or null
  int64_t mwords;
};
rkr_status tc_theta_pass(int pass, const rkr_index *idx, const TcSide &Ut, const TcSide &Qt,
                         const ThetaArgs &a, int split, int *err, cudaStream_t st);
// Rank table (Alg. 1 step 3, Eq. 1) on the tensor cores; *done stays false when the
// scratch could not be allocated or its queue overflowed (the caller then runs the
// CUDA-core kernel).
rkr_status tc_rank_table(const rkr_index *idx, const TcSide &Ut, cudaStream_t st, bool *done);
// Entries (user, query, screened score) recorded by the skim screen: region r
// (one per CTA of the launch) holds cnt[r] entries from r * rcap on; a count
// above rcap means the region overflowed and dropped the excess.
struct SkimList {
  int32_t *u, *q;
  float *x;
  uint32_t *cnt;
  int64_t rcap;
  int regions;
};
// CTAs (= list regions) of the skim launch for n users and nq queries.
int skim_regions(int64_t n, int64_t nq);
rkr_status tc_skim(const rkr_index *idx, const TcSide &Ut, const TcSide &Qt, const float *xs,
                   const SkimList &list, int *err, cudaStream_t st);
// refined[0] = queued undecided items, refined[1] = of those, canonical FP64 evaluations.
// With hist_hi (bounds mode) nothing is queued: undecided items give count intervals.
// split = 0 screens with the single BF16 product (bounds mode only: wider count
// intervals for a third of the tensor work); the exact mode always splits.
// Segments of one threshold pass seg_self (the item equal to the query, or -1);
// segments of several thresholds (up to kRecountSeg) pass self_col / self_pos
// instead: per candidate slot of the segment, the columns of items equal to a
// threshold's query in ascending order (-1 after the last) and the number of the
// segment's thresholds below each such item's score.
rkr_status tc_recount(const rkr_index *idx, const TcSide &Ut, const TcSide &Pt, int64_t nseg,
                      int64_t ncand, const int64_t *seg_start, const int32_t *seg_len,
                      const int32_t *seg_user, const int32_t *seg_self, const double *ths,
                      uint32_t *hist, uint32_t *hist_hi, cudaStream_t st, int64_t *refined,
                      int split = 1, const int32_t *self_col = nullptr,
                      const int32_t *self_pos = nullptr);
constexpr int kXGrid = 128;
constexpr int kDGrid = RKR_DEEP_GRID;   // points of the deep count grid (exact_table = 2)
constexpr int kRecountSeg = 32;     // thresholds per recount segment (one per screen row)
constexpr int kListCapMax = 16384;  // entries per user list (< 2^16: 16-bit column offsets)
constexpr int kListG = 1024;        // columns of the list grid (finer than the count grid)
rkr_status tc_sort_lists(rkr_index *idx, const tc::RowBound *tb, int bn, cudaStream_t st);

// Hash of each row's float bit patterns; rows past `rows` (up to Np2) get ~0.
rkr_status row_hashes(const float *X, int64_t rows, int d, int64_t Np2, uint64_t *keys,
                      int32_t *vals, cudaStream_t st);
rkr_status sort_pairs(uint64_t *key, int32_t *val, int64_t N_pow2, cudaStream_t st);
// qself[q] = sorted position of an item bitwise equal to query q (its score ties
// with u.q exactly for every user), or -1.
rkr_status query_self(const rkr_index *idx, const float *Q, int nq, int32_t *qself,
                      cudaStream_t st);

// Row norms: FP64 canonical norms (optional) and FP32 upper bounds.
rkr_status row_norms(const float *X, int64_t rows, int d, double *nrm64, float *nrm32,
                     cudaStream_t st);

// Largest element of a float array (device -> host), used for norm bounds.
rkr_status max_float(const float *x, int64_t count, float *out_host, cudaStream_t st);

// Check that every element is finite; *ok_host = 1 if so.
rkr_status all_finite(const float *x, int64_t count, int *ok_host, cudaStream_t st);

// Device views of one query batch.
struct QueryCommon {
  float *Qd;          // nq x d
  float *qnrm;        // nq FP32 norm bounds
  int32_t *kq_d;      // nq
  int64_t *out_off_d; // nq + 1 output offsets
  BinFP *bf;          // n bin parameters of the sampled table's grid, valid for this batch
  BinFP *xbf;         // n bin parameters of the exact grid, valid for this batch
  TcSide Qt;          // bf16 operands of the batch
  const uint32_t *member = nullptr;  // per-query user subsets (bitmaps), or null
  int64_t mwords = 0;                // 32-bit words per query in member
};

rkr_status run_query_approx(const rkr_index *idx, const QueryCommon &qc, int nq, double c,
                            int32_t *users_d, uint32_t *nlo_d, uint32_t *nup_d, double *est_d,
                            int32_t *case_d, int32_t *nc_d, rkr_query_stats *stats,
                            cudaStream_t st);
// Steps 2-3 of Section 4.3 for queries qa .. qa + nblocks - 1 over per-query
// candidate lists (one CTA per query; see k_select_approx in query.cu).
rkr_status launch_select_approx(int qa, int nblocks, const int64_t *qoff, const uint32_t *qcount,
                                const int32_t *uid, const uint32_t *nlo, const uint32_t *nup,
                                double *th, const int32_t *cj, const float *Qd,
                                const int32_t *kq, double c, const int64_t *out_off,
                                int32_t *users_d, uint32_t *nlo_d, uint32_t *nup_d, double *est_d,
                                int32_t *case_d, int32_t *nc_d, int *err, cudaStream_t st,
                                const rkr_index *idx);

// The same query steps one query at a time (latency.cu): per query, u.q of every
// user by an FP32 matrix-vector product with a rigorous bound fused with the
// bounds lookup, then steps 2-3 on the users that can still matter.
rkr_status run_query_approx_single(const rkr_index *idx, const QueryCommon &qc, int nq, double c,
                                   int32_t *users_d, uint32_t *nlo_d, uint32_t *nup_d,
                                   double *est_d, int32_t *case_d, int32_t *nc_d,
                                   rkr_query_stats *stats, cudaStream_t st);

// Per query, the users whose lower-bound numerator is at most an upper estimate of
// this index's R_up_k, with bounds and step-3 estimates (latency.cu); ids are
// local + user_offset; offs_host gets nq + 1 offsets (also when RKR_ENOMEM says
// the capacity was too small).
rkr_status run_query_approx_candidates(const rkr_index *idx, const QueryCommon &qc, int nq,
                                       int64_t user_offset, int64_t capacity, int64_t *offs_host,
                                       int32_t *users_d, uint32_t *nlo_d, uint32_t *nup_d,
                                       double *est_d, cudaStream_t st);

// Learned pruner (pruner.cu): predictions of B pairs from a per-user feature table.
rkr_status pruner_forward_gather(rkr_pruner *pr, const float *Xu, const int32_t *uid,
                                 const float *t, int64_t B, float *y, cudaStream_t st);
int pruner_features(const rkr_pruner *pr);
int pruner_hidden(const rkr_pruner *pr);

// Per-user prediction tables of the pruner (rkr_pruner_invert): tab[u][g] =
// y(x_u, t_g) on a grid of G values of t over [f_min, f_max] / ||u||, built from
// the per-user features Xu of the projection R (64 x d, host copy Rh).
rkr_status pruner_build_table(rkr_pruner *pr, const rkr_index *idx, const float *Xu,
                              const std::vector<float> &Rh, int G, cudaStream_t st);
void pruner_drop_table(rkr_pruner *pr);
// True when the pruner holds tables built for this index and projection.
bool pruner_table_matches(const rkr_pruner *pr, const rkr_index *idx,
                          const std::vector<float> &Rh);
// Predictions of B pairs (users uid, scores t) from the tables: linear
// interpolation in t between the two grid points around it.
rkr_status pruner_table_predict(const rkr_pruner *pr, const int32_t *uid, const float *t,
                                int64_t B, float *y, cudaStream_t st);

// Exact ranks of arbitrary (user, query) pairs of a staged batch (device arrays).
rkr_status run_rank_pairs(const rkr_index *idx, const QueryCommon &qc, int nq, int64_t npairs,
                          const int32_t *cu, const int32_t *cq, int32_t *out_rank,
                          cudaStream_t st);

// Per-user features of the pruner: 64 projections R u / ||u|| and log ||u||
// (F = 65), and per-pair scores t = u.q / ||u||.
rkr_status user_features(const rkr_index *idx, const float *R, float *Xu, cudaStream_t st);
rkr_status pair_scores(const rkr_index *idx, const float *Qd, int64_t npairs, const int32_t *cu,
                       const int32_t *cq, float *t, cudaStream_t st);

// Exact query whose candidates still to be recounted over P are cut to
// keep_d[q] per query (device array) by the pruner's predicted log ranks (an
// approximate form of Def. 2; returned ranks stay exact).
// With use_table the predictions come from the pruner's per-user tables.
rkr_status run_query_exact_learned(const rkr_index *idx, const QueryCommon &qc, int nq,
                                   rkr_pruner *pr, const float *Xu, const int32_t *keep_d,
                                   int certify, bool use_table, int32_t *users_d,
                                   int32_t *ranks_d, rkr_query_stats *stats, cudaStream_t st);

rkr_status run_query_exact(const rkr_index *idx, const QueryCommon &qc, int nq,
                           int32_t *users_d, int32_t *ranks_d, rkr_query_stats *stats,
                           cudaStream_t st);

}  // namespace rkr
