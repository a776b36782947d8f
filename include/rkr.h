/*
 * rkr.h -- C ABI of the GB300 reverse k-ranks library (librkr.so).
 *
 * Problem (Amagata et al., "Approximate Reverse k-Ranks Queries in High
 * Dimensions"):
 *   rank      r(q,u,P) = 1 + #{p in P : u.p > u.q}                 (Def. 1)
 *   exact     the k users with the smallest rank                   (Def. 2)
 *   c-approx  k users whose i-th rank is at most c times the i-th
 *             rank of the exact answer                             (Def. 3)
 * The c-approximate answer is computed with the paper's rank table
 * (Alg. 1, Eq. 1) and its three query steps (Section 4.3).
 *
 * Arithmetic.  The paper fixes no precision.  This library defines the score
 * of a user u and an item x (both float32 rows of length d) as the canonical
 * value s(u,x) = left-to-right sum over k of (double)u[k] * (double)x[k],
 * rounded to double after every addition.  Every comparison that decides a
 * rank, a table entry or a bin is made on canonical scores, so results are
 * bit-identical to a plain FP64 CPU evaluation.  Bulk scores are screened on
 * the GPU in lower precision with rigorous error bounds; only undecided cases
 * are recomputed canonically.
 *
 * Pointers.  Every array argument may be a host pointer or a device pointer of
 * the current device; the library detects which.  Matrices are row-major and
 * contiguous: U is n x d, P is m x d, Q is nq x d (float32).  The caller owns
 * every array it passes; the index owns device copies of U and P and all
 * derived data, released by rkr_index_free.
 *
 * Streams.  `stream` is a cudaStream_t (NULL = legacy default stream).  All
 * work is enqueued on it; each call synchronizes it before returning, so
 * outputs (host or device) are complete when the call returns.
 *
 * Errors.  Every call returns an rkr_status; RKR_OK is 0.  On failure nothing
 * is written to the outputs that the caller can rely on, and rkr_last_error()
 * returns a message for the calling thread.  No call aborts or throws.
 *
 * Device.  Kernels are built for sm_103a (GB300) only; other devices get
 * RKR_EUNSUPPORTED.
 */
#ifndef RKR_H
#define RKR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Points of the deep count grid of an index built with exact_table = 2. */
#define RKR_DEEP_GRID 64

typedef enum {
  RKR_OK = 0,
  RKR_EINVAL = 1,        /* invalid argument (null pointer, size, k, c, non-finite input) */
  RKR_ENOMEM = 2,        /* device or host allocation failed */
  RKR_ECUDA = 3,         /* CUDA runtime error; see rkr_last_error() */
  RKR_ETIMEOUT = 4,      /* a bounded device-side wait gave up */
  RKR_EUNSUPPORTED = 5,  /* device is not sm_103, or feature not built */
  RKR_EINTERNAL = 6      /* an internal consistency check failed */
} rkr_status;

typedef struct rkr_index rkr_index;
typedef struct rkr_pruner rkr_pruner;  /* learned pruner (rkr_pruner_create) */

/* Parameters of the pre-processing step (Alg. 1 inputs: tau, omega, s). */
typedef struct {
  int32_t tau;              /* number of thresholds per user, >= 2 (Section 4.2, step 2) */
  int32_t omega;            /* number of norm buckets, 1 <= omega <= m (Alg. 1) */
  int32_t s;                /* samples per bucket, >= 1 (Eq. 1); m * s must be < 2^32 */
  int32_t fbounds;          /* 0: f_min/f_max are the exact min/max of u.p over P
                               (Section 4.2, step 2); 1: +-||u|| * max ||p||
                               (the bounded-domain variant of the footnote) */
  int32_t exact_table;      /* 1: also build the exact count table rkr_query_exact needs;
                               2: also a deep count grid below the tail lists (one more
                               screen of U x P at build time; exact queries whose ranks lie
                               below the floor rank then recount far fewer candidates) */
  int32_t floor_rank;       /* exact table: counts are kept exact only above the
                               threshold whose estimated rank is floor_rank; 0 = default
                               max(2048, m / 16).  Only speed depends on it. */
  const int32_t *sample_pos;/* omega x s positions inside each bucket of the norm-sorted
                               items, -1 = unused; a bucket of at most s items must list
                               0..|P_l|-1.  Host or device.  NULL = draw them from `seed`
                               (uniform without replacement, SplitMix64). */
  uint64_t seed;
} rkr_build_params;

/* Counters of one query call (any pointer may be NULL). */
typedef struct {
  int64_t pairs;            /* user-query pairs screened */
  int64_t candidates;       /* pairs that survived the rank-bound filter */
  int64_t fp64_dots;        /* canonical FP64 inner products computed */
  int64_t near_ties;        /* item scores too close to u.q for the screen to decide */
  int32_t wide_queries;     /* queries whose cutoff fell to the last level */
  double max_rel_screen_err;/* exact path: largest |s_hat - s(u,p)| / (||u|| ||p||) over the
                               item scores of this call whose tensor-core screened value
                               s_hat was compared with the canonical FP64 score s (near-ties
                               in the tail lists); norms are FP32 upper bounds; 0 if none */
  double ms_theta;          /* device time of the u.q screening passes */
  double ms_resolve;        /* device time of candidate resolution */
  double ms_select;         /* device time of per-query selection */
  int64_t recounted;        /* exact path: candidates ranked by a re-screen of P (the others
                               by their user's tail list) */
  int32_t deep_queries;     /* queries whose cutoff lies above the skip level: screened
                               again without the one-compare skip of deep pairs.  The skip
                               level is the smallest L with 2^L - 1 >= m / 128, or the
                               value of the environment variable RKR_SKIP_LEVEL; results
                               do not depend on it. */
  int64_t recount_users;    /* exact path: distinct users among the candidates of each
                               interval pass over all of P, summed over those passes */
  int64_t recount_open;     /* exact path: recounted candidates whose count interval was still
                               open after the interval pass; each of their m item scores is
                               placed exactly, and near_ties of them needed FP64, so
                               near_ties / (recount_open * m) is the flagged fraction */
  int64_t recount_split;    /* exact path: recounted candidates whose interval was still open
                               after the single-product pass and went to the split pass */
  int64_t learned_revived;  /* learned cut: cut candidates whose lower bound could still reach
                               the k-th rank, recounted by the exact fallback */
  double max_screen_err_ratio; /* exact path: largest |s_hat - s(u,p)| / b over the same pairs
                               as max_rel_screen_err, b the rigorous screen bound (a sound
                               bound keeps it <= 1) */
  int64_t prefix_rows;      /* exact path: candidates screened against the norm-sorted prefix
                               of P first (tuning rc_prefix) */
  int64_t prefix_pruned;    /* of those, candidates dropped by their prefix lower bound
                               without a recount over all of P */
} rkr_query_stats;

/*
 * rkr_build: pre-processing (Alg. 1) on the GPU.
 *   U (n x d), P (m x d): float32, finite.  1 <= n < 2^31, 1 <= m <= 2^30, 1 <= d <= 256.
 *   Steps: norms of P and sort by (descending norm, index); omega buckets of
 *   m / omega items (the first m % omega get one more); per-bucket samples;
 *   f_min/f_max per user; thresholds t_j = f_min + (j-1) * ((f_max - f_min) / (tau - 1));
 *   table numerators N[u][j] = sum_l w_l * #{p in sample_l : s(u,p) > t_j}
 *   with w_l = |P_l| (s sampled) or s (whole bucket taken), so that
 *   T-hat[u][j] = 1 + N[u][j] / s (Eq. 1).
 *   On success *out receives a new index; free it with rkr_index_free.
 */
rkr_status rkr_build(const float *U, int64_t n, const float *P, int64_t m, int32_t d,
                     const rkr_build_params *params, void *stream, rkr_index **out);

/*
 * rkr_query_exact: exact reverse k-ranks (Def. 1, Def. 2) for nq queries.
 *   Q: nq x d float32, finite.  k: nq int32 values, 1 <= k[i] <= min(n, 4096).
 *   Needs an index built with exact_table = 1.
 *   Output per query i: k[i] users in ascending (rank, user index) order, written
 *   at offset sum_{j<i} k[j] of out_users (int32 user index) and out_ranks (int32 rank).
 *   Ties: among users of equal rank the smaller index comes first (any set of k
 *   smallest ranks satisfies Def. 2; this picks one).
 */
rkr_status rkr_query_exact(rkr_index *idx, const float *Q, int32_t nq, const int32_t *k,
                           int32_t *out_users, int32_t *out_ranks, rkr_query_stats *stats,
                           void *stream);

/*
 * rkr_query_approx: c-approximate reverse k-ranks (Def. 3) by the query steps
 * of Section 4.3.  c >= 1, finite.  k[i] in [1, min(n, 4096)].
 *   Step 1: j = max{j : t_j <= u.q} (0 if none); r_up = T-hat_j (m+1 if j = 0),
 *           r_low = T-hat_{j+1} (1 if j = tau); R_low_k, R_up_k = k-th smallest.
 *   Step 2: Case A if c * R_low_k >= R_up_k: the k users with smallest
 *           (r_up, r_low, index).  Case B: U_c = {u : r_up <= c * R_low_k};
 *           users with r_low > R_up_k are dropped.
 *   Step 3: the other users get r_hat = r_up - (r_up - r_low) * (u.q - t_j) / (t_{j+1} - t_j)
 *           (r_up outside the grid); the k - |U_c| smallest (r_hat, index) complete the answer.
 *   Outputs per query i at offset sum_{j<i} k[j]: out_users (int32), out_nlow and
 *   out_nup (uint32 numerators: r = 1 + N / s), out_est (double r_hat, computed for
 *   every returned user with the step-3 formula).  Step-2 users come first in
 *   (r_up, r_low, index) order, then step-3 users in (r_hat, index) order.
 *   out_case[i] = 1 (Case A) or 2 (Case B); out_nc[i] = number of step-2 users.
 *   Any output pointer except out_users may be NULL.
 */
rkr_status rkr_query_approx(rkr_index *idx, const float *Q, int32_t nq, const int32_t *k,
                            double c, int32_t *out_users, uint32_t *out_nlow, uint32_t *out_nup,
                            double *out_est, int32_t *out_case, int32_t *out_nc,
                            rkr_query_stats *stats, void *stream);

/*
 * rkr_session_*: a serving form of rkr_query_approx_single for one query per call
 * (not in the paper).  rkr_session_create keeps device buffers for one query and
 * captures the query's launches (query norm, the scan of U fused with the bounds
 * lookup, the cut, the compaction, steps 2-3) in a CUDA graph on a stream of its
 * own, for this index, k <= max_k and this c.  rkr_session_query copies q (d
 * floats, host or device) in, replays the graph and copies the outputs back:
 * out_users, out_nlow, out_nup, out_est (k entries each), *out_case, *out_nc, as
 * rkr_query_approx for that query, bit for bit (any output but out_users may be
 * NULL; host or device).  A query whose norm exceeds the largest item norm (the
 * captured bin bounds assume it does not) is answered by rkr_query_approx_single
 * instead, with the same result.  Calls on one session must not overlap; the
 * index must outlive the session.  RKR_EINVAL for bad arguments (max_k outside
 * [1, min(n, 4096)], c < 1, k > max_k, non-finite q).
 */
typedef struct rkr_session rkr_session;
rkr_status rkr_session_create(rkr_index *idx, int32_t max_k, double c, void *stream,
                              rkr_session **out);
rkr_status rkr_session_query(rkr_session *s, const float *q, int32_t k, int32_t *out_users,
                             uint32_t *out_nlow, uint32_t *out_nup, double *out_est,
                             int32_t *out_case, int32_t *out_nc);
void rkr_session_free(rkr_session *s);

/*
 * rkr_query_exact_bitmap / rkr_query_approx_bitmap: the subset forms with each
 * query's users given as a bitmap instead of an id list (compact for large
 * subsets: n / 8 bytes per query).  member: nq x words uint32 (host or device),
 * words = (n + 31) / 32 exactly, bit u % 32 of word q * words + u / 32 set iff
 * user u is in query q's subset; bits at or beyond n must be clear.  k[i] must
 * not exceed the number of set bits of query i.  Results as for the _subsets
 * forms.  RKR_EINVAL for a wrong word count, stray bits or too large a k.
 */
rkr_status rkr_query_exact_bitmap(rkr_index *idx, const float *Q, int32_t nq, const int32_t *k,
                                  const uint32_t *member, int64_t words, int32_t *out_users,
                                  int32_t *out_ranks, rkr_query_stats *stats, void *stream);
rkr_status rkr_query_approx_bitmap(rkr_index *idx, const float *Q, int32_t nq, const int32_t *k,
                                   const uint32_t *member, int64_t words, double c,
                                   int32_t *out_users, uint32_t *out_nlow, uint32_t *out_nup,
                                   double *out_est, int32_t *out_case, int32_t *out_nc,
                                   rkr_query_stats *stats, void *stream);

/*
 * rkr_query_approx_single: rkr_query_approx answered one query at a time (latency
 * mode), as the paper runs its queries (Section 5: each query on its own).  Same
 * arguments and outputs, bit for bit.  Per query: one pass over U computes u.q for
 * every user (FP32 warp products with a rigorous bound; canonical FP64 only where
 * the bound straddles a threshold) fused with the bounds lookup of Section 4.3
 * step 1, then steps 2-3 run on the users whose lower bound is at most an upper
 * estimate of R_up_k (every user the steps can return is among them).  Four
 * kernel launches per query, no host synchronization until the call returns.
 * The pass is bound by HBM bandwidth: about 4d + 48 bytes per user per query.
 * Temporaries: about 37 bytes per user, reused by every query of the call.
 */
rkr_status rkr_query_approx_single(rkr_index *idx, const float *Q, int32_t nq, const int32_t *k,
                                   double c, int32_t *out_users, uint32_t *out_nlow,
                                   uint32_t *out_nup, double *out_est, int32_t *out_case,
                                   int32_t *out_nc, rkr_query_stats *stats, void *stream);

/*
 * Sharded users (not in the paper: a deployment form in which the rows of U are
 * split across processes or GPUs; each part builds its own index from its rows,
 * the same P and the same build parameters and sample positions, so every
 * per-user quantity equals that of one index over all users).
 *
 * rkr_query_approx_candidates: for each query i, the users of this index that
 * the steps of Section 4.3 over the whole user set may need: every user whose
 * lower-bound numerator is at most T_i, an upper estimate of this index's
 * R_up_k computed with k[i] (k[i] <= n of this index; pass min(k, n) for a small
 * part).  Outputs per candidate, query after query: out_users (local index +
 * user_offset), out_nlow, out_nup (numerators) and out_est (the step-3 estimate
 * of Section 4.3 from the canonical u.q); out_offs (nq + 1) gives each query's
 * range.  capacity = entries the four output arrays hold; if more are found,
 * out_offs is still filled (out_offs[nq] = entries needed) and RKR_ENOMEM is
 * returned.
 *
 * rkr_merge_approx: the c-approximate answer from the union of the parts'
 * candidates (in_offs, in_users, in_nlow, in_nup, in_est: per query, the
 * concatenation of every part's candidates of that query).  Runs steps 1-3 of
 * Section 4.3 on the union with the parts' s: the result equals rkr_query_approx
 * on one index over all users, bit for bit (same outputs and order).  Host code
 * only, host arrays only; needs no GPU.  RKR_EINVAL for bad arguments or a query
 * with fewer than k entries.
 *
 * rkr_merge_exact: Def. 2 from the union of the parts' exact answers (in_users
 * global ids, in_ranks; per query the concatenation of every part's
 * min(k, n_part) best): the k smallest (rank, user), as rkr_query_exact on one
 * index.  Host code only, host arrays only.  RKR_EINVAL for bad arguments, a
 * user listed twice in a query, or fewer than k entries.
 */
rkr_status rkr_query_approx_candidates(rkr_index *idx, const float *Q, int32_t nq,
                                       const int32_t *k, int64_t user_offset, int64_t capacity,
                                       int64_t *out_offs, int32_t *out_users, uint32_t *out_nlow,
                                       uint32_t *out_nup, double *out_est, void *stream);
rkr_status rkr_merge_approx(int32_t nq, const int32_t *k, double c, int32_t s,
                            const int64_t *in_offs, const int32_t *in_users,
                            const uint32_t *in_nlow, const uint32_t *in_nup, const double *in_est,
                            int32_t *out_users, uint32_t *out_nlow, uint32_t *out_nup,
                            double *out_est, int32_t *out_case, int32_t *out_nc);
rkr_status rkr_merge_exact(int32_t nq, const int32_t *k, const int64_t *in_offs,
                           const int32_t *in_users, const int32_t *in_ranks, int32_t *out_users,
                           int32_t *out_ranks);

/*
 * rkr_query_exact_subsets / rkr_query_approx_subsets: the same queries with a
 * user subset per query (a batched deployment form; the paper's queries use
 * all of U).  For query i only users in
 * subset_users[subset_offs[i] .. subset_offs[i+1]) are eligible; ranks are
 * still taken over all of P (Def. 1), and R_low_k, R_up_k, U_c and the
 * interpolation of Section 4.3 run over the subset.
 *   subset_offs: nq + 1 int64, subset_offs[0] = 0, non-decreasing.
 *   subset_users: int32 user indices in [0, n), in any order (duplicates allowed).
 *   k[i] must not exceed the size of subset i (RKR_EINVAL otherwise).
 *   Host or device arrays.  The subsets are held as one bitmap of n bits per
 *   query on the device for the duration of the call.
 */
rkr_status rkr_query_exact_subsets(rkr_index *idx, const float *Q, int32_t nq, const int32_t *k,
                                   const int64_t *subset_offs, const int32_t *subset_users,
                                   int32_t *out_users, int32_t *out_ranks,
                                   rkr_query_stats *stats, void *stream);
rkr_status rkr_query_approx_subsets(rkr_index *idx, const float *Q, int32_t nq,
                                    const int32_t *k, const int64_t *subset_offs,
                                    const int32_t *subset_users, double c, int32_t *out_users,
                                    uint32_t *out_nlow, uint32_t *out_nup, double *out_est,
                                    int32_t *out_case, int32_t *out_nc, rkr_query_stats *stats,
                                    void *stream);

/*
 * rkr_screen_scores: the tensor-core screen on its own, for validation and for
 * measuring the screen error.  For every pair (U_i, X_j) writes the screened
 * score out_s[i * mx + j] (BF16 inputs, FP32 accumulation on tcgen05; split = 1
 * uses the three-term hi/lo product; split = 2 uses one E4M3 product (kind::f8f6f4) of
 * rows scaled by powers of two so that max|x| <= 448) and out_b[i * mx + j], the rigorous bound
 * the library uses for |out_s - s(U_i, X_j)|.  U: n x d, X: mx x d float32.
 * Meant for small n * mx (the outputs are dense).
 */
rkr_status rkr_screen_scores(const float *U, int64_t n, const float *X, int64_t mx, int32_t d,
                             int32_t split, float *out_s, float *out_b, void *stream);

/*
 * rkr_screen_scores_static: rkr_screen_scores without any device allocation.
 * The paper has no counterpart: this is a deployment variant of the validation
 * screen above, with the same outputs bit for bit.  It exists for callers that
 * must not call the CUDA allocator (cudaMalloc/cudaFree can synchronize the
 * device and can fail under memory pressure; a serving loop that owns its
 * device memory budget needs a call whose footprint is fixed at load time).
 *   All scratch (BF16 rows of U and X, their bound terms, per-tile bound maxima
 *   and the kernel's error word) lives in one file-scope device array of
 *   16 MiB per device.  Scratch needed for n rows of U and mx rows of X at
 *   kp = d rounded up to 16 is about 4 kp (n + mx) + 40 (n + mx) + 20 mx / 256
 *   bytes (each piece rounded up to 256 bytes); larger problems are rejected
 *   with RKR_EINVAL and a message giving both figures.
 *   U, X, out_s, out_b must be device (or managed) memory; host pointers are
 *   rejected with RKR_EINVAL, and so is split = 2 (the E4M3 form of
 *   rkr_screen_scores is not offered here).  Outputs as in rkr_screen_scores; the caller owns
 *   every buffer.
 *   The first call on a device looks up the array's address
 *   (cudaGetSymbolAddress, with that device current) and keeps it; make that
 *   first call before any stream capture.  The kept address belongs to the
 *   device's primary context: after cudaDeviceReset on that device the process
 *   must not call this entry point again.  Every call on a device uses the same
 *   array: calls that overlap in time (several host threads or streams) race
 *   on it and must be serialized by the caller.  The call synchronizes
 *   `stream` before it returns.
 */
rkr_status rkr_screen_scores_static(const float *U, int64_t n, const float *X, int64_t mx,
                                    int32_t d, int32_t split, float *out_s, float *out_b,
                                    void *stream);

/*
 * rkr_profile_start / rkr_profile_stop: per-kernel device time of the library's
 * launches between the two calls (not part of the paper).  While on, the main
 * kernels are bracketed by CUDA events recorded on the stream they are launched
 * on.  rkr_profile_stop synchronizes those events and writes one text line per
 * kernel, "name launches total_ms work", into report (len bytes including the
 * terminating NUL; RKR_EINVAL if it does not fit).  work is the summed
 * algorithmic work of the launches: 2 * rows * cols * d flops for a tensor-core
 * screen (one inner product of length d per pair: the method's work, not the
 * three products of the split form or the padding of K), 0 where none is stated.
 * Names starting with "span:" are stretches of work spanning several launches
 * (their time overlaps the kernels listed inside them).  Not thread-safe against concurrent queries
 * on other threads beyond what the shared event list allows.
 */
/*
 * rkr_rank_pairs: exact ranks r(q, u, P) (Def. 1) of arbitrary (user, query)
 * pairs: pair i is user pair_user[i] and query row pair_query[i] of Q (nq x d).
 * The same exact machinery as rkr_query_exact (tail lists, count intervals,
 * recount with near-tie resolution); out_rank[i] = 1 + #{p : s(u,p) > s(u,q)}.
 * Needs exact_table.  Host or device arrays; RKR_EINVAL for an index out of range.
 *
 * rkr_pair_features: the pruner's inputs for pairs: out_X (npairs x 65) =
 * (R u / ||u||, log ||u||) with R a 64 x d projection (row-major) chosen by the
 * caller, and out_t = u.q / ||u|| (FP32).
 *
 * rkr_query_exact_learned: Def. 2 with a learned cut (not the paper's method).
 * The exact path runs as in rkr_query_exact up to the recount: candidates whose
 * rank the tail lists settle keep their exact rank, and of the candidates that
 * would still need a recount over P only the keep[i] with the smallest
 * predicted log rank (and those tying with the keep[i]-th) are recounted for
 * query i.
 *   certify = 1 (exact fallback): after that recount, every cut candidate whose
 *   rank lower bound (from the tail lists and count tables) does not exceed the
 *   k-th smallest count found is recounted as well; the others cannot be among
 *   the k best.  The answer equals rkr_query_exact's, users and ranks; the cut
 *   saves only the recounts the fallback does not revive (a query with more than
 *   32 keep[i] candidates to recount that are also more than a quarter of all
 *   users is not cut: their lower bounds are too weak to spare any).
 *   certify = 0: the cut candidates are dropped.  Every returned rank is exact;
 *   the answer set may miss a true answer, and its recall is to be judged
 *   against rkr_query_exact.
 * stats->candidates counts the candidates left after the cut (revived ones
 * included), stats->learned_revived the revived ones.  RKR_EINVAL unless
 * certify is 0 or 1.
 * keep: nq int32 (host or device), keep[i] >= k[i], else RKR_EINVAL.
 */
rkr_status rkr_rank_pairs(rkr_index *idx, const float *Q, int32_t nq, int64_t npairs,
                          const int32_t *pair_user, const int32_t *pair_query, int32_t *out_rank,
                          void *stream);
rkr_status rkr_pair_features(rkr_index *idx, const float *R, const float *Q, int32_t nq,
                             int64_t npairs, const int32_t *pair_user, const int32_t *pair_query,
                             float *out_X, float *out_t, void *stream);
/*
 * rkr_pruner_invert: per-user tables of the trained network (not in the paper).
 * The network's output y never increases with t = u.q / ||u||, so for each user
 * it is one non-increasing function of t, tabulated once: tab[u][g] = y(x_u, t_g)
 * on G points t_g = t_0 + g (t_{G-1} - t_0) / (G - 1) spanning [f_min(u), f_max(u)]
 * / ||u||, the values t takes for the items of P.  Reading the same table the
 * other way gives each user's score cut-off for any predicted log rank: y <= Y
 * exactly where t is at least the table's crossing of Y.  While the pruner holds
 * tables built for this index and this R (64 x d, host or device),
 * rkr_query_exact_learned predicts each candidate by one lookup and a linear
 * interpolation between the two grid points around its t (t outside the grid
 * takes the end value) instead of a forward pass.  The pruner owns the tables
 * (n x G FP32 and 8 bytes per user); G = 0 frees them; new weights
 * (rkr_pruner_params, rkr_pruner_train) drop them.  G in [2, 1024], else
 * RKR_EINVAL; the pruner must take 65 features.
 */
rkr_status rkr_pruner_invert(rkr_pruner *pr, rkr_index *idx, const float *R, int32_t G,
                             void *stream);
/* rkr_pruner_table: copies of the tables of rkr_pruner_invert: tab (n x G FP32,
 * user-major) and grid (n x 2 FP32: t_0 and the step of each user's grid); host or
 * device arrays.  RKR_EINVAL if the pruner holds no tables or they are not n x G. */
rkr_status rkr_pruner_table(const rkr_pruner *pr, int64_t n, int32_t G, float *tab,
                            float *grid);
rkr_status rkr_query_exact_learned(rkr_index *idx, rkr_pruner *pr, const float *R, const float *Q,
                                   int32_t nq, const int32_t *k, const int32_t *keep,
                                   int32_t certify, int32_t *out_users, int32_t *out_ranks,
                                   rkr_query_stats *stats, void *stream);

/*
 * Learned pruner (not in the paper): a monotone rank regressor
 *   h1 = relu(W1 x - softplus(A) t + b1), h2 = relu(softplus(V2) h1 + b2),
 *   y = softplus(v3) . h2 + b3  ~  log r(q, u, P),
 * with x the F non-monotone features of the user and t = u.q / ||u||.  Every
 * path from t has a non-positive weight product through non-decreasing
 * activations, so y never increases with t (as the rank of Def. 1 cannot).
 * Trained and run on the GPU with hand-written kernels: BF16 operands, FP32
 * accumulation, FP32 master weights, Adam.  Loss 0.5 * mean((y - target)^2).
 * Flat parameter order: W1 (H x F, row-major), A (H), b1 (H), V2 (H x H),
 * b2 (H), v3 (H), b3 (1); rkr_pruner_nparams gives the count.
 *   rkr_pruner_create: F, H in [1, 1024]; weights drawn from `seed` (SplitMix64).
 *   rkr_pruner_params: set != 0 copies params into the model, else out of it
 *     (host or device array of exactly nparams floats).
 *   rkr_pruner_forward: y (B floats) for features X (B x F) and scores t (B).
 *   rkr_pruner_loss_grads: the loss and the gradient (nparams floats) of one
 *     batch, B <= 2^20 (for checking the kernels).
 *   rkr_pruner_train: `epochs` passes over npairs samples in shuffled batches
 *     of `batch` (SplitMix64 from `seed`), Adam with step `lr`; *final_loss gets
 *     the loss of the last batch.
 * Arrays may be host or device memory unless stated; all calls synchronize.
 */
rkr_status rkr_pruner_create(int32_t F, int32_t H, uint64_t seed, rkr_pruner **out);
int64_t rkr_pruner_nparams(const rkr_pruner *pr);
rkr_status rkr_pruner_params(rkr_pruner *pr, int32_t set, float *params, int64_t count);
rkr_status rkr_pruner_forward(rkr_pruner *pr, const float *X, const float *t, int64_t B, float *y,
                              void *stream);
rkr_status rkr_pruner_loss_grads(rkr_pruner *pr, const float *X, const float *t,
                                 const float *target, int64_t B, float *loss, float *grads,
                                 void *stream);
rkr_status rkr_pruner_train(rkr_pruner *pr, const float *X, const float *t, const float *target,
                            int64_t npairs, int32_t epochs, int32_t batch, float lr,
                            uint64_t seed, float *final_loss, void *stream);
void rkr_pruner_free(rkr_pruner *pr);

/*
 * Tuning (not in the paper): launch choices that change speed, never results.
 * Process-wide; the library starts from the defaults below.
 *   rc_bn            column tile of the recount screen: 256 (4 stages) or 128 (6 stages)
 *   rc_single_first  1: the recount runs a single-BF16-product interval pass before the
 *                    split-product pass; 0: split product only (the near-tie policy)
 *   skip_level       0: the default skip level of the query screens (smallest L with
 *                    2^L - 1 >= m / 128); else that level L (1..30)
 *   cand_budget_log2 candidates per screening chunk = 2^value, 20..30 (default 26)
 *   latency_ctas_per_sm  CTAs per SM of the one-at-a-time scan, 0 = occupancy maximum
 *   latency_bulk     1: the one-at-a-time scan stages rows of U in shared memory with
 *                    bulk copies (d a multiple of 4); 0: direct vector loads
 *   rc_seg_min       0: the recount screens one row per candidate (user, query); k >= 2:
 *                    a user with at least k candidates is screened once per segment of
 *                    up to 32 of its thresholds, counted together in the epilogue
 *   screen_form      tensor-core screens over row-owned work (index build, recount):
 *                    0 one CTA per SM; 1 CTA pairs sharing each B chunk by cluster
 *                    multicast; 2 CTA pairs issuing 2-SM MMAs (M = 256), each CTA
 *                    staging half of B.  The multicast-free build runs every form as 0.
 *   split_cat        1: split-product screens whose sides carry concatenated operands
 *                    ([hi | lo | hi] rows of U, [lo | hi | hi] rows of P and Q) run as one
 *                    pass over K = 3 K' (fewer pipeline stages when K' is not a multiple
 *                    of 64, the same MMAs in the same order); 0: three K' segments
 *   rc_prefix        0: off; p in [2, 64]: early termination over the norm-sorted items
 *                    (the order Alg. 1 sorts P in).  When a query has many candidates to
 *                    recount, all of them are first screened against the first m / p items
 *                    only (rounded down to 256); a candidate's certain count there is a
 *                    lower bound of its count over P.  The query's candidates with the
 *                    smallest possible counts there are recounted over all of P, which
 *                    gives a cap on the k-th smallest count, and every other candidate
 *                    whose prefix lower bound exceeds that cap is dropped unrecounted.
 *                    Default 4.
 * rkr_tuning_set validates every field (RKR_EINVAL) and applies to calls that start
 * after it returns; rkr_tuning_get reads the current values.
 *
 * rkr_autotune: picks the tuning for one workload by timed trials on it.  what is a
 * bit set: 1 = rkr_query_exact, 2 = rkr_query_approx, 4 = rkr_query_approx_single
 * (with c); the trial time is the sum of the chosen calls on (Q, nq, k).  Each
 * candidate tuning (a grid over the fields above) runs once untimed, then once
 * timed with CUDA events on `stream`; every trial's answers must equal the first
 * trial's (else RKR_EINTERNAL: tuning must not change results).  The fastest is
 * set process-wide and written to *out, its time to *out_ms.  cache_path (may be
 * NULL): a JSON-lines file; a line whose key (n, m, d, nq, sum of k, what) matches
 * is used without trials, and a new choice is appended to it.
 */
typedef struct {
  int32_t rc_bn;
  int32_t rc_single_first;
  int32_t skip_level;
  int32_t cand_budget_log2;
  int32_t latency_ctas_per_sm;
  int32_t latency_bulk;
  int32_t screen_form;
  int32_t rc_seg_min;
  int32_t split_cat;
  int32_t rc_prefix;
} rkr_tuning;
rkr_status rkr_tuning_get(rkr_tuning *out);
rkr_status rkr_tuning_set(const rkr_tuning *in);
rkr_status rkr_autotune(rkr_index *idx, const float *Q, int32_t nq, const int32_t *k, double c,
                        int32_t what, const char *cache_path, rkr_tuning *out, double *out_ms,
                        void *stream);

rkr_status rkr_profile_start(void);
rkr_status rkr_profile_stop(char *report, int64_t len);

/* What rkr_index_export copies out. */
typedef enum {
  RKR_EXPORT_PERM = 1,      /* int32[m]: original item index of each norm-sorted position */
  RKR_EXPORT_FMIN = 2,      /* double[n] */
  RKR_EXPORT_FMAX = 3,      /* double[n] */
  RKR_EXPORT_TABLE = 4,     /* uint32[n * tau]: N[u][j], j = 0..tau-1 */
  RKR_EXPORT_SAMPLES = 5,   /* int32[total samples]: original item index, bucket after bucket */
  RKR_EXPORT_XLO = 6,       /* uint32[n * G]: lower bound of #{p : s(u,p) > x_j} on the
                               exact grid (G = 128) */
  RKR_EXPORT_XHI = 9,       /* uint32[n * G]: upper bound of the same count */
  RKR_EXPORT_XGRID = 7,     /* double[n * 2]: (x_0, step) of each user's exact grid,
                               x_j = x_0 + j * step; x_0 is the threshold t of the sampled
                               table's last column whose estimated count is >= floor_rank,
                               x_{G-1} = f_max */
  RKR_EXPORT_PNORM = 8,     /* double[m]: FP64 norms of P in original order */
  RKR_EXPORT_DLO = 10,      /* uint32[n * RKR_DEEP_GRID]: lower bound of #{p : s(u,p) > y_c}
                               on the deep grid (exact_table = 2) */
  RKR_EXPORT_DHI = 11,      /* uint32[n * RKR_DEEP_GRID]: upper bound of the same count */
  RKR_EXPORT_DGRID = 12     /* double[n * 2]: (y_0, step) of each user's deep grid,
                               y_c = y_0 + c * step; y_0 is the threshold t of the sampled
                               table's last column whose estimated count is >= m / 8 (not
                               above x_0), y_{RKR_DEEP_GRID - 1} = x_0 */
} rkr_export_what;

/* Copy one internal array to dst (host or device); bytes must equal its size. */
rkr_status rkr_index_export(const rkr_index *idx, int32_t what, void *dst, int64_t bytes);

/* Sizes of the index: out[0..7] = n, m, d, tau, omega, s, total samples,
 * columns G of the exact grid (0 without exact table). */
rkr_status rkr_index_info(const rkr_index *idx, int64_t *out8);

/* Device time in ms of the build stages of an index: out[0] items (norms, sort,
 * gather), [1] samples, [2] f_min/f_max, [3] rank table, [4] level tables,
 * [5] exact count table, [6] total.  Entries beyond 6 are 0. */
rkr_status rkr_index_timings(const rkr_index *idx, double *out, int32_t count);

/* Number of CUDA kernels this library has launched in this process. */
uint64_t rkr_kernel_launches(void);

/* Number of device allocations this library has requested in this process
 * (stream-ordered pool allocations and the pruner's cudaMalloc calls; not in the
 * paper).  A call that allocates nothing leaves it unchanged. */
uint64_t rkr_device_allocations(void);

/* Test hook (not in the paper): the number of try_wait rounds after which the
 * epilogue warps of the tensor-core screens give up waiting for an accumulator
 * tile; the kernel then records the timeout, lets the MMAs and loads already
 * issued finish, and the call returns RKR_ETIMEOUT.  0 gives up at the first
 * wait; a negative value restores the default (2^22 rounds).  Process-wide;
 * takes effect for launches that start after the call.  RKR_EINVAL above 2^32 - 1. */
rkr_status rkr_set_wait_limit(int64_t rounds);

/* Release an index (NULL is allowed). */
void rkr_index_free(rkr_index *idx);

/*
 * rkr_index_save / rkr_index_load: an index as a file (checkpoint/resume).  The
 * paper builds its table once and serves any q, k and c from it (Section 4.1);
 * a saved index serves the same queries in another process with results
 * identical bit for bit.
 *   Format: magic "RKRIDX01", format version, byte-order mark, a header with
 *   the sizes (n, m, d), the build parameters (tau, omega, s, f-bounds mode,
 *   floor rank, seed) and this library's layout constants, then every device
 *   array of the index, then a 64-bit checksum (FNV-1a over 64-bit words) of
 *   all preceding bytes.  Files are as large as the index in device memory.
 *   rkr_index_save copies the arrays to the host through a pinned staging
 *   buffer and writes them; it synchronizes the device.  RKR_EINVAL if the file
 *   cannot be written.
 *   rkr_index_load allocates the arrays on the current device (sm_103a only) and
 *   fills them; RKR_EINVAL for a missing, truncated or corrupt file (checksum),
 *   another format version, byte order or layout constants; RKR_ENOMEM if the
 *   device cannot hold it.  On failure *out is NULL and nothing stays allocated.
 */
rkr_status rkr_index_save(const rkr_index *idx, const char *path);
/* Device memory the index holds, in bytes (the sum of its arrays: the copies of
 * U and P, their BF16 operands, the rank table, bounds and, with exact_table,
 * the exact count table and tail lists); the file rkr_index_save writes is that
 * size plus a small header. */
rkr_status rkr_index_device_bytes(const rkr_index *idx, int64_t *out);
rkr_status rkr_index_load(const char *path, rkr_index **out);

/* rkr_pruner_save / rkr_pruner_load: the learned pruner's F, H and FP32 master
 * weights (flat order of rkr_pruner_params) as a file with the same framing
 * (magic "RKRMLP01", version, byte-order mark, checksum).  Adam state is not
 * saved: a loaded pruner predicts exactly as the saved one did.  Errors as for
 * the index. */
rkr_status rkr_pruner_save(rkr_pruner *pr, const char *path);
rkr_status rkr_pruner_load(const char *path, rkr_pruner **out);

/* Device memory (not in the paper): the library allocates index arrays and
 * per-call temporaries from one stream-ordered pool per device and keeps what
 * it frees there, so later builds and queries reuse it without mapping memory
 * again.  This call waits for the device, then returns the pool's unused memory
 * of the current device to the driver.  Errors: RKR_ECUDA. */
rkr_status rkr_release_cached_memory(void);

/* Message describing the last failure on the calling thread ("" if none). */
const char *rkr_last_error(void);

/* Library version string; it names the build: the single-GPU build (row-owned
 * screens run as CTA pairs that share B tiles by cluster multicast) or the
 * replica build (no cluster multicast; same results bit for bit) that a
 * process uses when it is one rank of a multi-GPU job. */
const char *rkr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* RKR_H */
