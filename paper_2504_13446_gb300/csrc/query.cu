// query.cu -- query processing for both paths.
//
// Both paths share one plan.  For every user u the index holds a table of
// rank bounds on the threshold grid t_1..t_tau of u (the sampled table N of
// Alg. 1 for the c-approximate path; the exact count bounds XLO/XHI for the
// exact path) and two level tables JU/JL that turn a bin j into the rank level
// 2^L the table implies.  A query batch is processed as
//   pass 1  u.q screened for every (u, q) -> bin interval [jlo, jhi] ->
//           per-query histograms of the upper-bound level and the lower-bound level
//   cutoff  L*(q) = smallest level holding k upper bounds: R_up_k (approximate
//           path) or the k-th smallest rank (exact path) is at most 2^L* on the scale
//   pass 2  u.q screened again; users whose lower bound may reach 2^L* are
//           written to the candidate list of q (all others provably cannot matter)
//   resolve canonical FP64 u.q for each candidate; exact bin and table values
//           (approximate) or an exact recount of the rank over P (exact)
//   select  one CTA per query: Section 4.3 steps 1-3 (approximate) or the k
//           smallest (rank, index) (exact) over the candidates.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>

#include <vector>

#include "index.cuh"
#include "sort.cuh"
#include "select.cuh"
#include "simt.cuh"
#include "tcops.cuh"

namespace rkr {


// Cutoff level of each query: L* = the smallest level holding k upper bounds;
// below = pairs whose upper bound lies in a lower level; ncand = pairs whose
// lower bound lies in a level <= L* (an upper bound of the candidate count).
// Only levels <= lcap are complete in the histograms; a query that does not
// reach k there gets L* = kDeep and is screened again without skipping.
constexpr int kDeep = kMaxLevels;

__global__ void k_cutoff(int nq, const uint32_t *__restrict__ hist_up,
                         const uint32_t *__restrict__ hist_lo, const int32_t *__restrict__ kq,
                         int nlev, int lcap, int32_t *__restrict__ lstar,
                         uint64_t *__restrict__ below, int64_t *__restrict__ ncand) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  uint64_t cum = 0, prev = 0;
  int L = lcap >= nlev - 1 ? nlev - 1 : kDeep;
  const int lend = lcap < 31 ? lcap : 31;
  for (int l = 0; l <= lend; ++l) {
    prev = cum;
    cum += hist_up[(int64_t)q * 32 + l];
    if (cum >= (uint64_t)kq[q]) { L = l; break; }
  }
  if (L == kDeep) {
    lstar[q] = kDeep;
    below[q] = 0;
    ncand[q] = 0;
    return;
  }
  if (L > nlev - 1) L = nlev - 1;
  uint64_t c = 0;
  for (int l = 0; l <= L; ++l) c += hist_lo[(int64_t)q * 32 + l];
  lstar[q] = L;
  below[q] = prev;
  ncand[q] = (int64_t)c;
}

// Skip score of each user for skip level LS: the largest float x such that every
// screened upper end x_hi <= x gives a bin upper bound j_hi < JL[LS], so the
// pair's lower bound lies above level LS.  -inf when no such x is found.
__global__ void k_skip_scores(int64_t n, const BinFP *__restrict__ bf,
                              const int16_t *__restrict__ JL, int LS, float *__restrict__ xs) {
  int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= n) return;
  const int J = JL[u * kMaxLevels + LS];
  const BinFP b = bf[u];
  float x = -INFINITY;
  if (J >= 1 && b.invd32 > 0.0f && !(b.err > 1e6f)) {
    // bin_vhi(x) < J - 1 gives floor(v) + 1 <= J - 1
    const float target = (float)(J - 1);
    double x0 = (double)b.fmin32 + ((double)target - (double)b.err - 1.0) / (double)b.invd32;
    float c = __double2float_rd(x0);
    for (int it = 0; it < 64 && !(bin_vhi(b, c) < target); ++it) c = nextafterf(c, -INFINITY);
    if (bin_vhi(b, c) < target) x = c;
  }
  xs[u] = x;
}

// Rows of the deep queries, gathered for their own screening launches.
__global__ void k_gather_qrows(int nd, const int32_t *__restrict__ rows, int kp,
                               const __nv_bfloat16 *__restrict__ hi,
                               const __nv_bfloat16 *__restrict__ lo,
                               const tc::RowBound *__restrict__ rb1,
                               const tc::RowBound *__restrict__ rb3,
                               __nv_bfloat16 *__restrict__ ohi, __nv_bfloat16 *__restrict__ olo,
                               tc::RowBound *__restrict__ orb1, tc::RowBound *__restrict__ orb3,
                               uint32_t *__restrict__ hist, int nq) {
  const int i = blockIdx.x;
  if (i >= nd) return;
  const int64_t r = rows[i];
  for (int k = threadIdx.x; k < kp; k += blockDim.x) {
    ohi[(int64_t)i * kp + k] = hi[r * kp + k];
    olo[(int64_t)i * kp + k] = lo[r * kp + k];
  }
  if (threadIdx.x < 32) {  // the histograms of the skipping pass are incomplete
    hist[r * 32 + threadIdx.x] = 0;
    hist[((int64_t)nq + r) * 32 + threadIdx.x] = 0;
  }
  if (threadIdx.x == 0) {
    orb1[i] = rb1[r];
    orb3[i] = rb3[r];
  }
}

// Refined cap: the upper edge of the fine bucket of level L* where the running
// count of upper bounds reaches k; the k-th smallest upper bound is <= cap.
__global__ void k_cutoff_fine(int nq, const uint32_t *__restrict__ fine,
                              const uint64_t *__restrict__ below, const int32_t *__restrict__ lstar,
                              const int32_t *__restrict__ kq, uint32_t scale,
                              uint32_t *__restrict__ cap) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const int L = lstar[q];
  uint64_t hi = level_bound(L, scale);
  uint64_t base = L == 0 ? 0 : level_bound(L - 1, scale) + 1;
  uint64_t width = (hi - base + 1024) / 1024;
  uint64_t cum = below[q], c = hi;
  for (int b = 0; b < 1024; ++b) {
    cum += fine[(int64_t)q * 1024 + b];
    if (cum >= (uint64_t)kq[q]) { c = base + (uint64_t)(b + 1) * width - 1; break; }
  }
  if (c > hi) c = hi;
  cap[q] = (uint32_t)(c > 0xffffffffull ? 0xffffffffull : c);
}

// --------------------------------------------------------- approximate path

__global__ void k_resolve_approx(int64_t count, const int32_t *__restrict__ cu,
                                 const int32_t *__restrict__ cq, const float *__restrict__ cx,
                                 const tc::RowBound *__restrict__ urb,
                                 const tc::RowBound *__restrict__ qrb, tc::Gacc gacc, float gcan,
                                 const float *__restrict__ U, const float *__restrict__ Q, int d,
                                 const double *__restrict__ fmin,
                                 const double *__restrict__ delta, const BinFP *__restrict__ bf,
                                 const uint32_t *__restrict__ N,
                                 int tau, uint32_t top, double *__restrict__ th,
                                 int32_t *__restrict__ cj, uint32_t *__restrict__ nlo,
                                 uint32_t *__restrict__ nup,
                                 unsigned long long *__restrict__ nfp64) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= count) return;
  int64_t u = cu[i];
  if (u < 0) return;  // unused slot at the end of a query's segment
  int q = cq[i];
  const float *uu = U + u * d, *qq = Q + (int64_t)q * d;
  // j from the screened score and its bound when both ends fall in one bin (no
  // row is read); else from the compensated interval of u.q; else from the
  // canonical u.q.  u.q itself is formed later, only for the users whose step-3
  // estimate is needed (NaN marks it as not yet formed).
  int jlo = 0, jhi = tau;
  const float x = cx[i];
  if (x == x) {   // NaN: the candidate has no screened score
    const float b = tc::screen_bound_tc(urb[u], qrb[q], gacc, gcan);
    bin_interval(bf[u], fmin[u], tau, __fsub_rd(x, b), __fadd_ru(x, b), jlo, jhi);
  }
  if (jlo != jhi) {
    double tlo, thi;
    dot2_interval(uu, qq, d, tlo, thi);
    bin_interval(bf[u], fmin[u], tau, __double2float_rd(tlo), __double2float_ru(thi), jlo, jhi);
  }
  int j;
  if (jlo == jhi) {
    j = jlo;
    th[i] = __longlong_as_double(0x7ff8000000000000ll);
  } else {
    const double theta = canon_dot(uu, qq, d);
    j = exact_j(theta, fmin[u], delta[u], tau);
    th[i] = theta;
    atomicAdd(nfp64, 1ull);
  }
  cj[i] = j;
  nlo[i] = j < tau ? N[u * tau + j] : 0u;
  nup[i] = j >= 1 ? N[u * tau + j - 1] : top;
}

struct ApproxCand {
  const int32_t *uid;
  const uint32_t *nlo, *nup;
  double *th;          // canonical u.q, NaN until formed
  const int32_t *j;
  const float *U, *Q;  // rows, for forming u.q on demand
  int d;
  unsigned long long *nfp64;   // canonical products formed (may be null)
};

constexpr int kSelThreads = 256;

// One CTA per query: steps 1-3 of Section 4.3 over the query's candidates.
__global__ void __launch_bounds__(kSelThreads)
    k_select_approx(int qa, const int64_t *__restrict__ qoff, const uint32_t *__restrict__ qcount,
                    ApproxCand C,
                    const int32_t *__restrict__ kq, double c, uint32_t s, int tau,
                    const double *__restrict__ fmin, const double *__restrict__ delta,
                    const int64_t *__restrict__ out_off, int32_t *__restrict__ out_users,
                    uint32_t *__restrict__ out_nlo, uint32_t *__restrict__ out_nup,
                    double *__restrict__ out_est, int32_t *__restrict__ out_case,
                    int32_t *__restrict__ out_nc, int *__restrict__ err) {
  extern __shared__ unsigned char sbuf[];
  SortEnt *ent = (SortEnt *)sbuf;                   // kMaxK entries
  __shared__ uint32_t hist[256];
  __shared__ uint64_t bc[2];
  __shared__ unsigned long long cnt_acc;
  __shared__ int gcount;
  const int q = qa + blockIdx.x;
  const int64_t base = qoff[q] - qoff[qa];
  const int64_t cnt = qcount[q];
  const int k = kq[q];
  if (cnt < k) {  // cannot happen when the screening passes are consistent
    if (threadIdx.x == 0) atomicExch(err, 1);
    return;
  }
  const int32_t *uid = C.uid + base;
  const uint32_t *nlo = C.nlo + base, *nup = C.nup + base;
  double *th = C.th + base;
  const int32_t *cj = C.j + base;
  const float *qrow = C.Q + (int64_t)q * C.d;
  auto est_of = [&](int64_t i) {
    int32_t u = uid[i];
    double t = th[i];
    if (t != t) {  // not formed yet: the canonical u.q, kept for later calls
      t = canon_dot(C.U + (int64_t)u * C.d, qrow, C.d);
      th[i] = t;
      if (C.nfp64) atomicAdd(C.nfp64, 1ull);
    }
    return interp_est(t, cj[i], nlo[i], nup[i], fmin[u], delta[u], tau, s);
  };
  // Step 1: k-th smallest lower and upper bound numerators.
  uint64_t Rlo = block_kth(cnt, (uint64_t)k, 32,
                           [&](int64_t i, uint64_t &key) { key = nlo[i]; return true; }, hist, bc);
  uint64_t Rup = block_kth(cnt, (uint64_t)k, 32,
                           [&](int64_t i, uint64_t &key) { key = nup[i]; return true; }, hist, bc);
  const double lhs = c * (double)((uint64_t)s + Rlo);
  const bool caseA = lhs >= (double)((uint64_t)s + Rup);
  const int64_t obase = out_off[q];
  int nc;
  if (caseA) {
    // k smallest (r_up, r_low, index): all with nup < Rup, then ties by (nlo, index)
    int64_t below = block_count(cnt, [&](int64_t i) { return (uint64_t)nup[i] < Rup; }, &cnt_acc);
    uint64_t kth2 = ~0ull;
    if (below < k)
      kth2 = block_kth(cnt, (uint64_t)(k - below), 64,
                       [&](int64_t i, uint64_t &key) {
                         key = ((uint64_t)nlo[i] << 32) | (uint32_t)uid[i];
                         return (uint64_t)nup[i] == Rup;
                       },
                       hist, bc);
    if (threadIdx.x == 0) gcount = 0;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) {
      uint64_t a = nup[i];
      bool take = a < Rup ||
                  (a == Rup && (((uint64_t)nlo[i] << 32) | (uint32_t)uid[i]) <= kth2);
      if (take) {
        int pos = atomicAdd(&gcount, 1);
        if (pos < kMaxK) {
          ent[pos].k1 = ((uint64_t)nup[i] << 32) | nlo[i];
          ent[pos].k2 = (uint32_t)uid[i];
          ent[pos].idx = (int32_t)i;
        }
      }
    }
    __syncthreads();
    int got = min(gcount, kMaxK);
    block_sort(ent, got);
    for (int r = threadIdx.x; r < got && r < k; r += blockDim.x) {
      int64_t i = ent[r].idx;
      out_users[obase + r] = uid[i];
      if (out_nlo) out_nlo[obase + r] = nlo[i];
      if (out_nup) out_nup[obase + r] = nup[i];
      if (out_est) out_est[obase + r] = est_of(i);
    }
    nc = k;
  } else {
    // U_c = {r_up <= c R_low_k}: fewer than k users, (r_up, r_low, index) order
    auto in_c = [&](int64_t i) { return (double)((uint64_t)s + nup[i]) <= lhs; };
    if (threadIdx.x == 0) gcount = 0;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) {
      if (in_c(i)) {
        int pos = atomicAdd(&gcount, 1);
        if (pos < kMaxK) {
          ent[pos].k1 = ((uint64_t)nup[i] << 32) | nlo[i];
          ent[pos].k2 = (uint32_t)uid[i];
          ent[pos].idx = (int32_t)i;
        }
      }
    }
    __syncthreads();
    nc = min(gcount, kMaxK);
    block_sort(ent, nc);
    for (int r = threadIdx.x; r < nc; r += blockDim.x) {
      int64_t i = ent[r].idx;
      out_users[obase + r] = uid[i];
      if (out_nlo) out_nlo[obase + r] = nlo[i];
      if (out_nup) out_nup[obase + r] = nup[i];
      if (out_est) out_est[obase + r] = est_of(i);
    }
    __syncthreads();
    // Step 3: survivors r_low <= R_up_k outside U_c, smallest (r_hat, index)
    auto in_t = [&](int64_t i) { return (uint64_t)nlo[i] <= Rup && !in_c(i); };
    const int need = k - nc;
    uint64_t ke = block_kth(cnt, (uint64_t)need, 64,
                            [&](int64_t i, uint64_t &key) {
                              if (!in_t(i)) return false;
                              key = dkey(est_of(i));
                              return true;
                            },
                            hist, bc);
    int64_t below = block_count(cnt, [&](int64_t i) { return in_t(i) && dkey(est_of(i)) < ke; },
                                &cnt_acc);
    uint64_t ku = ~0ull;
    if (below < need)
      ku = block_kth(cnt, (uint64_t)(need - below), 32,
                     [&](int64_t i, uint64_t &key) {
                       if (!in_t(i) || dkey(est_of(i)) != ke) return false;
                       key = (uint32_t)uid[i];
                       return true;
                     },
                     hist, bc);
    if (threadIdx.x == 0) gcount = 0;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) {
      if (!in_t(i)) continue;
      double e = est_of(i);
      uint64_t ek = dkey(e);
      if (ek < ke || (ek == ke && (uint64_t)(uint32_t)uid[i] <= ku)) {
        int pos = atomicAdd(&gcount, 1);
        if (pos < kMaxK) {
          ent[pos].k1 = ek;
          ent[pos].k2 = (uint32_t)uid[i];
          ent[pos].idx = (int32_t)i;
        }
      }
    }
    __syncthreads();
    int got = min(gcount, kMaxK);
    block_sort(ent, got);
    for (int r = threadIdx.x; r < got && nc + r < k; r += blockDim.x) {
      int64_t i = ent[r].idx;
      out_users[obase + nc + r] = uid[i];
      if (out_nlo) out_nlo[obase + nc + r] = nlo[i];
      if (out_nup) out_nup[obase + nc + r] = nup[i];
      if (out_est) out_est[obase + nc + r] = __longlong_as_double((long long)ent[r].k1);
    }
  }
  if (threadIdx.x == 0) {
    if (out_case) out_case[q] = caseA ? 1 : 2;
    if (out_nc) out_nc[q] = nc;
  }
}

// -------------------------------------------------------------- exact path

// Canonical u.q of each candidate and its sort key (user, order-preserving u.q).
__global__ void k_cand_theta(int64_t count, const int32_t *__restrict__ cu,
                             const int32_t *__restrict__ cq, const float *__restrict__ U,
                             const float *__restrict__ Q, int d, double *__restrict__ th,
                             uint64_t *__restrict__ key_hi, uint64_t *__restrict__ key_lo,
                             int32_t *__restrict__ val, int64_t Np2) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= Np2) return;
  if (i >= count || cu[i] < 0) {  // padding or an unused slot: sorted to the end
    key_hi[i] = ~0ull;
    key_lo[i] = ~0ull;
    val[i] = 0x7fffffff;
    return;
  }
  int64_t u = cu[i];
  double theta = canon_dot(U + u * d, Q + (int64_t)cq[i] * d, d);
  th[i] = theta;
  uint64_t bits = (uint64_t)__double_as_longlong(theta);
  key_hi[i] = (uint64_t)u;
  key_lo[i] = (bits >> 63) ? ~bits : (bits | 0x8000000000000000ull);
  val[i] = (int32_t)i;
}

// Segments of equal user in the sorted order: start index and length.  A user
// with fewer than seg_min thresholds (or every user, seg_min = 0) gets one
// segment per threshold; a longer run is cut into near-equal segments of at
// most kRecountSeg.  Segments
// of one threshold take slots from the front of [0, count), longer ones from
// the back, so that each kind is one range for its recount screen; seg_len of
// the slots between stays 0.
// nseg[0] = front slots, nseg[1] = distinct users, nseg[2] = back slots.
__global__ void k_segments(int64_t count, const uint64_t *__restrict__ key_hi, int seg_min,
                           unsigned long long *__restrict__ nseg, int64_t *__restrict__ seg_start,
                           int32_t *__restrict__ seg_len) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool first = i < count && key_hi[i] != ~0ull && (i == 0 || key_hi[i] != key_hi[i - 1]);
  int64_t e = i + 1;
  if (first)
    while (e < count && key_hi[e] == key_hi[i]) ++e;
  const int64_t run = first ? e - i : 0;
  const bool single = first && (seg_min == 0 || run < seg_min);
  // one atomic per warp for the distinct users and for the one-threshold slots
  // (a million candidates of one query would otherwise queue on one address)
  const int lane = threadIdx.x & 31;
  const unsigned nfirst = __popc(__ballot_sync(0xffffffffu, first));
  unsigned long long mine = single ? (unsigned long long)run : 0ull, incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  const unsigned long long tot = __shfl_sync(0xffffffffu, incl, 31);
  unsigned long long base = 0;
  if (lane == 31) {
    if (tot) base = atomicAdd(&nseg[0], tot);
    if (nfirst) atomicAdd(&nseg[1], (unsigned long long)nfirst);   // distinct users
  }
  base = __shfl_sync(0xffffffffu, base, 31);
  if (single) {   // one row per threshold
    const int64_t slot0 = (int64_t)(base + incl - mine);
    for (int64_t a = i; a < e; ++a) {
      seg_start[slot0 + (a - i)] = a;
      seg_len[slot0 + (a - i)] = 1;
    }
    return;
  }
  if (!first) return;
  // pieces of nearly equal length, at most kRecountSeg each
  const int64_t np = (run + kRecountSeg - 1) / kRecountSeg;
  for (int64_t p = 0; p < np; ++p) {
    const int64_t a = i + run * p / np, b = i + run * (p + 1) / np;
    const int64_t slot = count - 1 - (int64_t)atomicAdd(&nseg[2], 1ull);
    seg_start[slot] = a;
    seg_len[slot] = (int32_t)(b - a);
  }
}

// Per segment: its user, its thresholds in sorted order, and a zeroed histogram
// of L + 1 slots at hist[2 st0] (segments are disjoint since L >= 1).  A
// one-threshold segment records the item tying exactly with its u.q (the query
// itself when it is an item of P) in seg_self; a longer one lists such items
// of all its thresholds in self_col (ascending, each once, -1 after the last),
// each with its exact position in self_pos: its canonical score is its query's
// threshold, so it exceeds exactly the thresholds below that one.
__global__ void k_seg_prep(int64_t nseg, const int64_t *__restrict__ seg_start,
                           const int32_t *__restrict__ seg_len, const uint64_t *__restrict__ key_hi,
                           const int32_t *__restrict__ order, const double *__restrict__ th,
                           const int32_t *__restrict__ cq, const int32_t *__restrict__ qself,
                           int32_t *__restrict__ seg_user, int32_t *__restrict__ seg_self,
                           double *__restrict__ ths, uint32_t *__restrict__ hist,
                           int32_t *__restrict__ self_col, int32_t *__restrict__ self_pos) {
  int64_t sg = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (sg >= nseg) return;
  const int L = seg_len[sg];
  if (L == 0) return;   // a slot between the two ranges
  int64_t st0 = seg_start[sg];
  seg_user[sg] = (int32_t)key_hi[st0];
  seg_self[sg] = L == 1 ? qself[cq[order[st0]]] : -1;
  for (int i = 0; i < L; ++i) ths[st0 + i] = th[order[st0 + i]];
  for (int i = 0; i <= L; ++i) hist[2 * st0 + i] = 0;
  if (L == 1) return;
  int32_t *sc = self_col + st0, *sp = self_pos + st0;
  int ns = 0;
  for (int i = 0; i < L; ++i) {
    const int32_t c = qself[cq[order[st0 + i]]];
    if (c < 0) continue;
    int pos = i;
    while (pos > 0 && ths[st0 + pos - 1] == ths[st0 + i]) --pos;
    int at = ns;
    while (at > 0 && sc[at - 1] > c) --at;
    if (at > 0 && sc[at - 1] == c) continue;   // the same item for an equal query
    for (int j = ns; j > at; --j) {
      sc[j] = sc[j - 1];
      sp[j] = sp[j - 1];
    }
    sc[at] = c;
    sp[at] = pos;
    ++ns;
  }
  for (int j = ns; j < L; ++j) sc[j] = -1;
}

// hist[pos] counts items whose score exceeds exactly the first pos thresholds;
// after the suffix sum h[i] = #{p : s(u,p) > theta_{i-1}}.
__global__ void k_seg_suffix(int64_t nseg, const int64_t *__restrict__ seg_start,
                             const int32_t *__restrict__ seg_len, uint32_t *__restrict__ hist) {
  int64_t sg = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (sg >= nseg || seg_len[sg] == 0) return;
  uint32_t *h = hist + 2 * seg_start[sg];
  uint32_t run = 0;
  for (int i = seg_len[sg]; i >= 1; --i) {
    run += h[i];
    h[i] = run;
  }
}

// count of candidate order[st0 + i] = hist[2 st0 + i + 1] (see k_seg_suffix).
__global__ void k_scatter_counts(int64_t nseg, const int64_t *__restrict__ seg_start,
                                 const int32_t *__restrict__ seg_len,
                                 const int32_t *__restrict__ order,
                                 const uint32_t *__restrict__ hist, uint32_t *__restrict__ ccount) {
  int64_t sg = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (sg >= nseg) return;
  int L = seg_len[sg];
  if (L == 0) return;
  int64_t st0 = seg_start[sg];
  const uint32_t *h = hist + 2 * st0;
  for (int i = 0; i < L; ++i) ccount[order[st0 + i]] = h[i + 1];
}

// The deep count grid of an index (dg = 0: none).
struct DeepGrid {
  int dg;
  const double *yg0, *ydx;
  const uint32_t *DLO, *DHI;
};
inline DeepGrid deep_grid(const rkr_index *idx) {
  return DeepGrid{idx->dg, idx->yg0, idx->ydx, idx->DLO, idx->DHI};
}

// Exact ranks from the tail lists.  A candidate (u, q) with u.q >= x_0(u)
// has rank 1 + #{p in list(u) : s(u,p) > u.q}, since every item scoring above
// x_0 is in the list.  Entries are grouped by exact-grid column: whole
// columns are counted from the column offsets, and the entries of the one or
// two columns within the screen bound of u.q are settled one by one, by their
// own bound, an FP32 dot product with its bound, or canonically.  Candidates below x_0 (or with an overflowed list) are
// passed on, unchanged, in cu_fb for the recount screen; others get -1 there.
// 64 registers a thread (eight 128-thread blocks per SM): the kernel waits on
// scattered reads of each candidate's user data and list, so warps in flight matter.
__global__ void __launch_bounds__(128, 8) k_list_rank(int64_t count, const int32_t *__restrict__ cu,
                            const int32_t *__restrict__ cq, const float *__restrict__ cx,
                            const tc::RowBound *__restrict__ qrb, const float *__restrict__ U,
                            const float *__restrict__ unrm, const float *__restrict__ Q,
                            const float *__restrict__ Ps, const float *__restrict__ pnrm_s, int d,
                            const uint2 *__restrict__ xlist,
                            const int64_t *__restrict__ xloff, const uint32_t *__restrict__ xlcap,
                            const uint16_t *__restrict__ xcoff,
                            const uint32_t *__restrict__ xlcnt,
                            const float *__restrict__ xbmax, const tc::RowBound *__restrict__ rb3,
                            const tc::RowBound *__restrict__ ptile, int pbn, tc::Gacc gacc,
                            float gcan, const double *__restrict__ xg0,
                            const double *__restrict__ xdx, int GX, const double *__restrict__ ldx,
                            int G, const uint32_t *__restrict__ XLO,
                            const uint32_t *__restrict__ XHI, uint32_t mtop,
                            uint32_t *__restrict__ ccount, uint32_t *__restrict__ clb,
                            int32_t *__restrict__ cu_fb, const int32_t *__restrict__ qself,
                            DeepGrid deep, unsigned long long *__restrict__ stat) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= count) return;
  const int64_t u = cu[i];
  if (u < 0) {  // an unused slot or a pruned candidate: never selected
    cu_fb[i] = -1;
    ccount[i] = 0xffffffffu;
    clb[i] = 0xffffffffu;
    return;
  }
  const float *uu = U + u * d;
  const float *qq = Q + (int64_t)cq[i] * d;
  // u.q as an interval [tlo, thi], tightened only where a comparison needs it:
  // first the candidate's screened score and its bound (no row is read), then
  // the compensated product, then the canonical value
  double tlo = -INFINITY, thi = INFINITY;
  int state = 1;   // 0: screened interval, 1: compensated, 2: canonical
  const float sx = cx ? cx[i] : __int_as_float(0x7fffffff);
  if (sx == sx) {
    const float b = tc::screen_bound_tc(rb3[u], qrb[cq[i]], gacc, gcan);
    tlo = (double)__fsub_rd(sx, b);
    thi = (double)__fadd_ru(sx, b);
    state = 0;
  } else {
    dot2_interval(uu, qq, d, tlo, thi);
  }
  double theta = 0.0;
  auto tighten = [&]() {
    if (state == 0) {
      dot2_interval(uu, qq, d, tlo, thi);
      state = 1;
    } else {
      theta = canon_dot(uu, qq, d);
      tlo = thi = theta;
      state = 2;
      atomicAdd(&stat[4], 1ull);
    }
  };
  const uint32_t L = xlcnt[u];
  const double x0 = xg0[u];
  while (state < 2 && L <= xlcap[u] && tlo < x0 && thi >= x0) tighten();
  if (L > xlcap[u] || thi < x0) {
    // bounds from the exact count table at the bins of both ends of u.q
    int jl = exact_j(tlo, x0, xdx[u], GX), jh = exact_j(thi, x0, xdx[u], GX);
    const int G2 = deep.dg;
    const bool below = G2 > 0 && thi < x0;
    int kl = 0, kh = 0;
    if (below) {
      kl = exact_j(tlo, deep.yg0[u], deep.ydx[u], G2);
      kh = exact_j(thi, deep.yg0[u], deep.ydx[u], G2);
    }
    if (state == 0 && (jl != jh || kl != kh)) {   // as tight as the compensated product gives
      tighten();
      jl = exact_j(tlo, x0, xdx[u], GX);
      jh = exact_j(thi, x0, xdx[u], GX);
      if (below) {
        kl = exact_j(tlo, deep.yg0[u], deep.ydx[u], G2);
        kh = exact_j(thi, deep.yg0[u], deep.ydx[u], G2);
      }
    }
    uint32_t ub = jl >= 1 ? XHI[u * GX + jl - 1] : mtop;
    uint32_t lb = jh < GX ? XLO[u * GX + jh] : 0u;
    if (below) {
      // below x_0: the deep grid's counts at y_{kl - 1} <= tlo and y_{kh} > thi
      if (kl >= 1) ub = min(ub, deep.DHI[u * G2 + kl - 1]);
      if (kh < G2) lb = max(lb, deep.DLO[u * G2 + kh]);
    }
    ccount[i] = ub;
    clb[i] = lb;
    cu_fb[i] = (int32_t)u;
    atomicAdd(&stat[0], 1ull);
    return;
  }
  cu_fb[i] = -1;
  // entries are grouped by column c = #{x_j <= v}: x_{c-1} <= v < x_c
  const uint2 *row = xlist + xloff[u];
  const uint16_t *co = xcoff + u * (G + 2);
  const double B = (double)xbmax[u];
  const double g0 = xg0[u], dx = ldx[u];
  // columns c >= chi have v >= x_{c-1} > u.q + B: every entry is above u.q
  const int chi = exact_j(__dadd_ru(thi, B), g0, dx, G) + 1;
  // columns c < clo have v < x_c <= u.q - B: no entry is above u.q
  const int clo = exact_j(__dsub_rd(tlo, B), g0, dx, G);
  uint32_t above = L - (uint32_t)co[chi];
  const tc::RowBound ru = rb3[u];
  const int32_t self = qself[cq[i]];
  for (int e = co[clo]; e < (int)co[chi]; ++e) {
    const uint32_t p = row[e].x;
    if ((int32_t)p == self) continue;  // the query's own item: s(u,p) = u.q, not above
    const float v = __uint_as_float(row[e].y);
    const float b = tc::screen_bound_tc(ru, ptile[p / pbn], gacc, gcan);
    if ((double)__fsub_rd(v, b) > thi) { ++above; continue; }
    if ((double)__fadd_ru(v, b) <= tlo) continue;
    if (state == 0) {   // the screened interval of u.q cannot place it: compensate, look again
      tighten();
      --e;
      continue;
    }
    const float *pp = Ps + (int64_t)p * d;
    double slo, shi;
    dot2_interval(uu, pp, d, slo, shi);
    if (slo > thi) { ++above; continue; }
    if (shi <= tlo) continue;
    atomicAdd(&stat[1], 1ull);
    if (state < 2) tighten();   // the canonical u.q
    const double sc = canon_dot(uu, pp, d);
    if (sc > theta) ++above;
    // screen error of this pair against its canonical score: relative to the
    // bound (at most 1 for a sound bound) and to the norm bounds ||u|| ||p||
    const double er = fabs((double)v - sc);
    const float ratio = (float)(er / (double)b);
    const float rel = (float)(er / ((double)unrm[u] * (double)pnrm_s[p]));
    atomicMax(&stat[2], (unsigned long long)__float_as_uint(ratio));
    atomicMax(&stat[3], (unsigned long long)__float_as_uint(rel));
  }
  ccount[i] = above;
  clb[i] = above;
}

// Threads of the per-query filters: a query may have a million candidates.
constexpr int kFilterThreads = 512;

// Per query: cap = k-th smallest of (exact count, or upper bound for candidates
// still to be recounted).  A candidate whose lower bound exceeds the cap cannot
// be among the k smallest ranks: it is dropped from the recount and given the
// largest key.
__global__ void __launch_bounds__(kFilterThreads)
    k_recount_filter(int qa, const int64_t *__restrict__ qoff, const uint32_t *__restrict__ qcount,
                     const int32_t *__restrict__ kq, uint32_t *__restrict__ ccount,
                     const uint32_t *__restrict__ clb, int32_t *__restrict__ cu_fb) {
  __shared__ uint32_t hist[256];
  __shared__ uint64_t bc[2];
  const int q = qa + blockIdx.x;
  const int64_t base = qoff[q] - qoff[qa];
  const int64_t cnt = qcount[q];
  const int k = kq[q];
  if (cnt < k) return;
  uint32_t *cc = ccount + base;
  const uint32_t *lb = clb + base;
  int32_t *fb = cu_fb + base;
  const uint64_t cap = block_kth(cnt, (uint64_t)k, 32,
                                 [&](int64_t i, uint64_t &key) { key = cc[i]; return true; },
                                 hist, bc);
  for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x)
    if (fb[i] >= 0 && (uint64_t)lb[i] > cap) {
      fb[i] = -1;
      cc[i] = 0xffffffffu;
    }
}

__global__ void k_count_valid(int64_t n, const int32_t *__restrict__ v,
                              unsigned long long *__restrict__ out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  unsigned long long c = (i < n && v[i] >= 0) ? 1ull : 0ull;
  c = __reduce_add_sync(0xffffffffu, (unsigned)c);
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

// Early termination over the norm-sorted items (tuning rc_prefix).  A query
// takes part when at least prefix_min_rows(k) of its candidates still need a
// recount; those candidates are copied to cu_pre for the prefix pass.
__host__ __device__ inline int64_t prefix_pick_rows(int k) { return k * 8 > 256 ? k * 8 : 256; }
__host__ __device__ inline int64_t prefix_min_rows(int k) { return 8 * prefix_pick_rows(k); }

__global__ void __launch_bounds__(256)
    k_prefix_split(int qa, const int64_t *__restrict__ qoff, const uint32_t *__restrict__ qcount,
                   const int32_t *__restrict__ kq, const int32_t *__restrict__ cu_fb,
                   int32_t *__restrict__ cu_pre, unsigned long long *__restrict__ npre) {
  __shared__ unsigned long long acc;
  const int q = qa + blockIdx.x;
  const int64_t base = qoff[q] - qoff[qa];
  const int64_t cnt = qcount[q];
  const int32_t *fb = cu_fb + base;
  const int64_t nr = block_count(cnt, [&](int64_t i) { return fb[i] >= 0; }, &acc);
  if (nr < prefix_min_rows(kq[q])) return;
  for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) cu_pre[base + i] = fb[i];
  if (threadIdx.x == 0) atomicAdd(npre, (unsigned long long)nr);
}

// Per query of the prefix pass: every prefix row's lower bound takes its certain
// count over the prefix (a subset of P); the prefix_pick_rows(k) rows with the
// smallest possible prefix counts (ties included) stay in cu_fb for a recount
// over all of P, the others are parked in cu_park until the cap is known.
__global__ void __launch_bounds__(kFilterThreads)
    k_prefix_pick(int qa, const int64_t *__restrict__ qoff, const uint32_t *__restrict__ qcount,
                  const int32_t *__restrict__ kq, const int32_t *__restrict__ cu_pre,
                  const uint32_t *__restrict__ hi1, const uint32_t *__restrict__ lo1,
                  uint32_t *__restrict__ clb, int32_t *__restrict__ cu_fb,
                  int32_t *__restrict__ cu_park) {
  __shared__ uint32_t hist[256];
  __shared__ uint64_t bc[2];
  __shared__ unsigned long long acc;
  const int q = qa + blockIdx.x;
  const int64_t base = qoff[q] - qoff[qa];
  const int64_t cnt = qcount[q];
  const int32_t *pre = cu_pre + base;
  const int64_t np = block_count(cnt, [&](int64_t i) { return pre[i] >= 0; }, &acc);
  const uint64_t k2 = (uint64_t)prefix_pick_rows(kq[q]);
  if (np <= (int64_t)k2) return;
  const uint32_t *h = hi1 + base, *l = lo1 + base;
  const uint64_t T = block_kth(cnt, k2, 32,
                               [&](int64_t i, uint64_t &key) {
                                 key = h[i];
                                 return pre[i] >= 0;
                               },
                               hist, bc);
  for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) {
    if (pre[i] < 0) continue;
    clb[base + i] = max(clb[base + i], l[i]);
    if ((uint64_t)h[i] > T) {
      cu_park[base + i] = cu_fb[base + i];
      cu_fb[base + i] = -1;
    }
  }
}

// Parked rows that the cap did not drop go back to the recount.
__global__ void k_prefix_unpark(int64_t n, const int32_t *__restrict__ cu_park,
                                int32_t *__restrict__ cu_fb) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n && cu_park[i] >= 0) cu_fb[i] = cu_park[i];
}

// One CTA per query: the k smallest (rank, index) among its candidates.
__global__ void __launch_bounds__(kSelThreads)
    k_select_exact(int qa, const int64_t *__restrict__ qoff, const uint32_t *__restrict__ qcount,
                   const int32_t *__restrict__ cuid,
                   const uint32_t *__restrict__ ccount, const int32_t *__restrict__ kq,
                   const int64_t *__restrict__ out_off, int32_t *__restrict__ out_users,
                   int32_t *__restrict__ out_ranks, int *__restrict__ err) {
  extern __shared__ unsigned char sbuf[];
  SortEnt *ent = (SortEnt *)sbuf;
  __shared__ uint32_t hist[256];
  __shared__ uint64_t bc[2];
  __shared__ int gcount;
  const int q = qa + blockIdx.x;
  const int64_t base = qoff[q] - qoff[qa];
  const int64_t cnt = qcount[q];
  const int k = kq[q];
  if (cnt < k) {
    if (threadIdx.x == 0) atomicExch(err, 1);
    return;
  }
  const int32_t *uid = cuid + base;
  const uint32_t *cc = ccount + base;
  uint64_t kth = block_kth(cnt, (uint64_t)k, 64,
                           [&](int64_t i, uint64_t &key) {
                             key = ((uint64_t)cc[i] << 32) | (uint32_t)uid[i];
                             return true;
                           },
                           hist, bc);
  if (threadIdx.x == 0) gcount = 0;
  __syncthreads();
  for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x) {
    uint64_t key = ((uint64_t)cc[i] << 32) | (uint32_t)uid[i];
    if (key <= kth) {
      int pos = atomicAdd(&gcount, 1);
      if (pos < kMaxK) {
        ent[pos].k1 = key;
        ent[pos].k2 = 0;
        ent[pos].idx = (int32_t)i;
      }
    }
  }
  __syncthreads();
  int got = min(gcount, kMaxK);
  block_sort(ent, got);
  const int64_t obase = out_off[q];
  for (int r = threadIdx.x; r < got && r < k; r += blockDim.x) {
    out_users[obase + r] = (int32_t)(ent[r].k1 & 0xffffffffu);
    out_ranks[obase + r] = (int32_t)(ent[r].k1 >> 32) + 1;
  }
}

// ------------------------------------------------------------------- host

// ------------------------------------------------------------ skim list

// Entry e of region blockIdx.y (thread index within the region's count).
__device__ __forceinline__ bool list_entry(const SkimList &L, int64_t &e) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const uint32_t c = L.cnt[blockIdx.y];
  if (i >= (int64_t)(c < L.rcap ? c : L.rcap)) return false;
  e = (int64_t)blockIdx.y * L.rcap + i;
  return true;
}

// Pass 1 on the list: bin interval of each entry's u.q from its screened score
// and the pair's own bound, the levels of its upper and lower rank bounds
// (histograms per query), and both kept for the later passes.
__global__ void k_list_levels(SkimList L, const tc::RowBound *__restrict__ urb,
                              const tc::RowBound *__restrict__ qrb, tc::Gacc gacc, float gcan,
                              const BinFP *__restrict__ bf, const double *__restrict__ fmin,
                              int tau, const int16_t *__restrict__ JU,
                              const int16_t *__restrict__ JL, uint32_t *__restrict__ hist_up,
                              uint32_t *__restrict__ hist_lo, uint32_t *__restrict__ jj,
                              uint32_t *__restrict__ lv, const uint32_t *__restrict__ member,
                              int64_t mwords) {
  int64_t e;
  if (!list_entry(L, e)) return;
  const int64_t u = L.u[e];
  const int q = L.q[e];
  if (!in_subset(member, mwords, q, u)) {  // outside the query's subset: never counted
    jj[e] = 0;
    lv[e] = 0xffffu;
    return;
  }
  const float x = L.x[e];
  const float b = tc::screen_bound_tc(urb[u], qrb[q], gacc, gcan);
  int jlo, jhi;
  bin_interval(bf[u], fmin[u], tau, __fsub_rd(x, b), __fadd_ru(x, b), jlo, jhi);
  const int16_t *ju = JU + u * kMaxLevels, *jl = JL + u * kMaxLevels;
  int lu = 0, ll = 0;
#pragma unroll
  for (int step = 16; step > 0; step >>= 1) {
    if (ju[lu + step - 1] > jlo) lu += step;
    if (jl[ll + step - 1] > jhi) ll += step;
  }
  atomicAdd(&hist_up[(int64_t)q * 32 + lu], 1u);
  atomicAdd(&hist_lo[(int64_t)q * 32 + ll], 1u);
  jj[e] = (uint32_t)jlo | ((uint32_t)jhi << 16);
  lv[e] = (uint32_t)lu | ((uint32_t)ll << 8);
}

// Pass 3 on the list: entries whose upper bound lies exactly at their query's
// level L* add that bound to the query's fine histogram of the level.
__global__ void k_list_fine(SkimList L, const uint32_t *__restrict__ jj,
                            const uint32_t *__restrict__ lv, const int32_t *__restrict__ lstar,
                            int lskip, const uint32_t *__restrict__ thi, int tau, uint32_t top,
                            uint32_t scale, uint32_t *__restrict__ fine) {
  int64_t e;
  if (!list_entry(L, e)) return;
  const int q = L.q[e];
  const int Lq = lstar[q];
  if (Lq > lskip || (int)(lv[e] & 0xff) != Lq) return;
  const int64_t u = L.u[e];
  const int jlo = (int)(jj[e] & 0xffff);
  const uint64_t v = jlo >= 1 ? thi[u * tau + jlo - 1] : top;
  const uint64_t hi = level_bound(Lq, scale);
  const uint64_t base = Lq == 0 ? 0 : level_bound(Lq - 1, scale) + 1;
  const uint64_t width = (hi - base + 1024) / 1024;
  uint64_t bkt = v >= base ? (v - base) / width : 0;
  if (bkt >= 1024) bkt = 1023;
  atomicAdd(&fine[(int64_t)q * 1024 + bkt], 1u);
}

// Pass 2 on the list: entries of queries [qa, qb) whose lower bound may reach
// the query's refined cap, appended to the query's candidate segment with their
// screened score (its bound settles most later decisions about u.q).
__global__ void k_list_emit(SkimList L, const uint32_t *__restrict__ jj,
                            const uint32_t *__restrict__ lv, int qa, int qb,
                            const int32_t *__restrict__ lstar, int lskip,
                            const uint32_t *__restrict__ cap, const uint32_t *__restrict__ tlo,
                            int tau, const int64_t *__restrict__ qoff,
                            uint32_t *__restrict__ qcursor, int32_t *__restrict__ cand_u,
                            int32_t *__restrict__ cand_q, float *__restrict__ cand_x,
                            int *__restrict__ ovf) {
  int64_t e;
  if (!list_entry(L, e)) return;
  const int q = L.q[e];
  if (q < qa || q >= qb) return;
  const int Lq = lstar[q];
  if (Lq > lskip || (int)((lv[e] >> 8) & 0xff) > Lq) return;
  const int64_t u = L.u[e];
  const int jhi = (int)(jj[e] >> 16);
  const uint32_t lb = jhi < tau ? tlo[u * tau + jhi] : 0u;
  if (lb > cap[q]) return;
  const uint32_t pos = atomicAdd(&qcursor[q], 1u);
  const int64_t at = qoff[q] + pos;
  if (at >= qoff[q + 1]) {
    atomicExch(ovf, 1);
    return;
  }
  cand_u[at] = (int32_t)u;
  cand_q[at] = q;
  cand_x[at] = L.x[e];
}

// Shared front half: passes 1 and 3 and the cutoffs; per-query candidate counts.
// Pairs whose lower bound lies above the skip level are left out by a single
// compare of the screened score; queries whose cutoff lies above it ("deep")
// are gathered and screened again in full by launches of their own.
struct Plan {
  std::vector<int64_t> ncand;
  std::vector<int32_t> lstar;
  int lskip = 1 << 30;          // skip level (no skipping: every level)
  DevBuf bxs;
  float *xs = nullptr;          // per-user skip scores
  std::vector<int32_t> deep;    // deep queries, ascending
  DevBuf bdeep, bdhi, bdlo, bdr1, bdr3;
  int32_t *deep_d = nullptr;
  TcSide dside;                 // their bf16 rows (views of the buffers above)
  bool listed = false;          // passes 1-3 of the other queries run on the skim list
  SkimList list{};
  uint32_t maxcnt = 0;          // largest region count (launch width of list kernels)
  DevBuf blu, blq, blx, blc, bjj, blv;
  uint32_t *jj = nullptr, *lv = nullptr;
};

static rkr_status check_flag(int *flag_d, const char *what, cudaStream_t st);

// Capacity of the skim list: entries of every region together.
static int64_t skim_capacity(int64_t n, int64_t nq) {
  int64_t want = n * nq / 16;
  return std::max<int64_t>((int64_t)1 << 20, std::min<int64_t>(want, (int64_t)1 << 29));
}

static dim3 list_grid(const Plan &plan) {
  return dim3((unsigned)std::max<uint32_t>(1, (plan.maxcnt + 255) / 256),
              (unsigned)plan.list.regions);
}

// Skim screen of all queries into plan.list; plan.listed stays false when the
// list cannot be allocated or a region overflowed (the passes then screen again).
static rkr_status skim_queries(const rkr_index *idx, const QueryCommon &qc, int nq, Plan &plan,
                               int *flag, cudaStream_t st) {
  const int regions = skim_regions(idx->n, nq);
  const int64_t cap = skim_capacity(idx->n, nq);
  SkimList &L = plan.list;
  L.regions = regions;
  L.rcap = cap / regions;
  const size_t ent = (size_t)L.rcap * regions;
  auto try_alloc = [&](DevBuf &b, auto **p, size_t count) -> bool {
    cudaError_t e = pool_malloc_async((void **)p, count * sizeof(**p), st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    b.p = (void *)*p;
    b.st = st;
    return true;
  };
  if (!try_alloc(plan.blu, &L.u, ent) || !try_alloc(plan.blq, &L.q, ent) ||
      !try_alloc(plan.blx, &L.x, ent) || !try_alloc(plan.blc, &L.cnt, regions) ||
      !try_alloc(plan.bjj, &plan.jj, ent) || !try_alloc(plan.blv, &plan.lv, ent))
    return RKR_OK;
  RKR_CUDA(cudaMemsetAsync(L.cnt, 0, sizeof(uint32_t) * regions, st));
  RKR_TRY(tc_skim(idx, idx->Ut, qc.Qt, plan.xs, L, flag, st));
  std::vector<uint32_t> cnt(regions);
  RKR_CUDA(cudaMemcpyAsync(cnt.data(), L.cnt, sizeof(uint32_t) * regions, cudaMemcpyDeviceToHost,
                           st));
  RKR_CUDA(cudaStreamSynchronize(st));
  RKR_TRY(check_flag(flag, "skim screen", st));
  uint32_t mx = 0;
  for (uint32_t c : cnt) {
    if ((int64_t)c > L.rcap) return RKR_OK;  // overflow: not listed
    mx = std::max(mx, c);
  }
  plan.maxcnt = mx;
  plan.listed = true;
  return RKR_OK;
}

// Skip level: the smallest level whose ranks reach m / 128.
static int skip_level(const rkr_index *idx) {
  const char *env = getenv("RKR_SKIP_LEVEL");
  if (env && *env) return atoi(env);
  const int tl = tuning().skip_level;
  if (tl > 0) return tl;
  int64_t r = idx->m / 128;
  int L = 0;
  while (L < 31 && (((int64_t)1 << L) - 1) < r) ++L;
  return L;
}

// Grid, bin parameters, level tables and bound tables of one path.
struct Grid {
  const BinFP *bf;
  const double *fmin;
  int tau;
  const int16_t *JU, *JL;
  int nlev;
  const uint32_t *thi, *tlo;
  uint32_t top, scale;
};

constexpr int kThetaSplit = 1;  // u.q screened with the split (three-term) product

static rkr_status check_flag(int *flag_d, const char *what, cudaStream_t st) {
  int h = 0;
  RKR_CUDA(cudaMemcpyAsync(&h, flag_d, sizeof(int), cudaMemcpyDeviceToHost, st));
  RKR_CUDA(cudaStreamSynchronize(st));
  if (h) return fail(RKR_ETIMEOUT, "%s: screen kernel wait timed out (%d)", what, h);
  return RKR_OK;
}

static ThetaArgs theta_args(const Grid &g, int qa, const QueryCommon &qc) {
  ThetaArgs a{};
  a.qa = qa;
  a.lskip = 1 << 30;
  a.member = qc.member;
  a.mwords = qc.mwords;
  a.binfp = g.bf;
  a.fmin = g.fmin;
  a.tau = g.tau;
  a.JU = g.JU;
  a.JL = g.JL;
  a.thi = g.thi;
  a.tlo = g.tlo;
  a.top = g.top;
  a.scale = g.scale;
  return a;
}

// Passes 1 and 3: per-query cutoff level, refined cap, and candidate-count bounds.
static rkr_status screen_plan(const rkr_index *idx, const QueryCommon &qc, int nq,
                              const Grid &g, cudaStream_t st, int32_t *lstar_d, uint32_t *cap_d,
                              int64_t *ncand_d, Plan &plan) {
  DevBuf bh, bf, bb, bfi;
  uint32_t *hist, *fine;
  uint64_t *below;
  int *flag;
  RKR_TRY(tmp_alloc(bh, &hist, (size_t)nq * 64, st));
  RKR_TRY(tmp_alloc(bfi, &fine, (size_t)nq * 1024, st));
  RKR_TRY(tmp_alloc(bb, &below, nq, st));
  RKR_TRY(tmp_alloc(bf, &flag, 1, st));
  RKR_CUDA(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * (size_t)nq * 64, st));
  RKR_CUDA(cudaMemsetAsync(fine, 0, sizeof(uint32_t) * (size_t)nq * 1024, st));
  RKR_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), st));
  const int LS = skip_level(idx);
  const bool skip = LS >= 0 && LS < g.nlev - 1;
  if (skip) {
    RKR_TRY(tmp_alloc(plan.bxs, &plan.xs, idx->n, st));
    k_skip_scores<<<(unsigned)((idx->n + 255) / 256), 256, 0, st>>>(idx->n, g.bf, g.JL, LS,
                                                                     plan.xs);
    note_launch();
    RKR_CUDA(cudaGetLastError());
    plan.lskip = LS;
  }
  ThetaArgs a = theta_args(g, 0, qc);
  a.nq_all = nq;
  a.hist = hist;
  a.xs = plan.xs;
  a.lskip = plan.lskip;
  if (skip) RKR_TRY(skim_queries(idx, qc, nq, plan, flag, st));
  if (plan.listed) {
    if (plan.maxcnt > 0) {
      {
        const int prof_slot = prof_begin("k_list_levels", st);
        k_list_levels<<<list_grid(plan), 256, 0, st>>>(
            plan.list, idx->Ut.rb3, qc.Qt.rb3, tc_gacc(idx->Ut.kp, 1), tc_gcan(idx->d), g.bf,
            g.fmin, g.tau, g.JU, g.JL, hist, hist + (size_t)nq * 32, plan.jj, plan.lv, qc.member,
          qc.mwords);
        prof_end(prof_slot, st, 0.0);
      }
      note_launch();
      RKR_CUDA(cudaGetLastError());
    }
  } else {
    RKR_TRY(tc_theta_pass(1, idx, idx->Ut, qc.Qt, a, kThetaSplit, flag, st));
  }
  k_cutoff<<<(nq + 127) / 128, 128, 0, st>>>(nq, hist, hist + (size_t)nq * 32, qc.kq_d, g.nlev,
                                             skip ? LS : 31, lstar_d, below, ncand_d);
  note_launch();
  RKR_CUDA(cudaGetLastError());
  ThetaArgs ad = a;  // deep queries: own rows, every pair screened
  ad.xs = nullptr;
  ad.lskip = 1 << 30;
  if (skip) {
    std::vector<int32_t> ls(nq);
    RKR_CUDA(cudaMemcpyAsync(ls.data(), lstar_d, sizeof(int32_t) * nq, cudaMemcpyDeviceToHost,
                             st));
    RKR_CUDA(cudaStreamSynchronize(st));
    for (int q = 0; q < nq; ++q)
      if (ls[q] == kDeep) plan.deep.push_back(q);
  }
  const int nd = (int)plan.deep.size();
  if (nd > 0) {
    const int kp = qc.Qt.kp;
    TcSide &D = plan.dside;
    RKR_TRY(tmp_alloc(plan.bdeep, &plan.deep_d, nd, st));
    RKR_TRY(tmp_alloc(plan.bdhi, &D.hi, (size_t)nd * kp, st));
    RKR_TRY(tmp_alloc(plan.bdlo, &D.lo, (size_t)nd * kp, st));
    RKR_TRY(tmp_alloc(plan.bdr1, &D.rb1, nd, st));
    RKR_TRY(tmp_alloc(plan.bdr3, &D.rb3, nd, st));
    D.rows = nd;
    D.d = qc.Qt.d;
    D.kp = kp;
    D.owned = false;
    RKR_CUDA(cudaMemcpyAsync(plan.deep_d, plan.deep.data(), sizeof(int32_t) * nd,
                             cudaMemcpyHostToDevice, st));
    {
      const int prof_slot = prof_begin("k_gather_qrows", st);
      k_gather_qrows<<<nd, 128, 0, st>>>(nd, plan.deep_d, kp, qc.Qt.hi, qc.Qt.lo, qc.Qt.rb1,
                                         qc.Qt.rb3, D.hi, D.lo, D.rb1, D.rb3, hist, nq);
      prof_end(prof_slot, st, 0.0);
    }
    note_launch();
    RKR_CUDA(cudaGetLastError());
    ad.qmap = plan.deep_d;
    RKR_TRY(tc_theta_pass(1, idx, idx->Ut, D, ad, kThetaSplit, flag, st));
    k_cutoff<<<(nq + 127) / 128, 128, 0, st>>>(nq, hist, hist + (size_t)nq * 32, qc.kq_d,
                                               g.nlev, 31, lstar_d, below, ncand_d);
    note_launch();
    RKR_CUDA(cudaGetLastError());
  }
  a.hist = nullptr;
  a.lstar = lstar_d;
  a.fine = fine;
  if (plan.listed) {
    if (plan.maxcnt > 0) {
      {
        const int prof_slot = prof_begin("k_list_fine", st);
        k_list_fine<<<list_grid(plan), 256, 0, st>>>(plan.list, plan.jj, plan.lv, lstar_d,
                                                     plan.lskip, g.thi, g.tau, g.top, g.scale,
                                                     fine);
        prof_end(prof_slot, st, 0.0);
      }
      note_launch();
      RKR_CUDA(cudaGetLastError());
    }
  } else {
    RKR_TRY(tc_theta_pass(3, idx, idx->Ut, qc.Qt, a, kThetaSplit, flag, st));
  }
  if (nd > 0) {
    ad.hist = nullptr;
    ad.lstar = lstar_d;
    ad.fine = fine;
    RKR_TRY(tc_theta_pass(3, idx, idx->Ut, plan.dside, ad, kThetaSplit, flag, st));
  }
  k_cutoff_fine<<<(nq + 127) / 128, 128, 0, st>>>(nq, fine, below, lstar_d, qc.kq_d, g.scale,
                                                  cap_d);
  note_launch();
  RKR_CUDA(cudaGetLastError());
  RKR_TRY(check_flag(flag, "theta passes 1 and 3", st));
  plan.ncand.resize(nq);
  plan.lstar.resize(nq);
  RKR_CUDA(cudaMemcpyAsync(plan.ncand.data(), ncand_d, sizeof(int64_t) * nq,
                           cudaMemcpyDeviceToHost, st));
  RKR_CUDA(cudaMemcpyAsync(plan.lstar.data(), lstar_d, sizeof(int32_t) * nq,
                           cudaMemcpyDeviceToHost, st));
  RKR_CUDA(cudaStreamSynchronize(st));
  return RKR_OK;
}

// Pass 2: candidates of queries [qa, qb) appended to per-query segments.
static rkr_status emit_candidates(const rkr_index *idx, const QueryCommon &qc, int qa, int qb,
                                  const Grid &g, const Plan &plan, const int32_t *lstar_d,
                                  const uint32_t *cap_d, const int64_t *qoff_d, uint32_t *cursor_d,
                                  int32_t *cand_u, int32_t *cand_q, float *cand_x,
                                  cudaStream_t st) {
  TcSide sub = qc.Qt;
  sub.owned = false;
  sub.rows = qb - qa;
  sub.hi = qc.Qt.hi + (size_t)qa * qc.Qt.kp;
  sub.lo = qc.Qt.lo + (size_t)qa * qc.Qt.kp;
  sub.rb1 = qc.Qt.rb1 + qa;
  sub.rb3 = qc.Qt.rb3 + qa;
  DevBuf bf;
  int *flag;
  RKR_TRY(tmp_alloc(bf, &flag, 2, st));
  RKR_CUDA(cudaMemsetAsync(flag, 0, 2 * sizeof(int), st));
  ThetaArgs a = theta_args(g, qa, qc);
  a.nq_all = qc.Qt.rows;
  a.ovf = flag + 1;
  a.lstar = lstar_d;
  a.cap = cap_d;
  a.qoff = qoff_d;
  a.qcursor = cursor_d;
  a.cand_u = cand_u;
  a.cand_q = cand_q;
  a.xs = plan.xs;
  a.lskip = plan.lskip;
  if (plan.listed) {
    if (plan.maxcnt > 0) {
      {
        const int prof_slot = prof_begin("k_list_emit", st);
        k_list_emit<<<list_grid(plan), 256, 0, st>>>(plan.list, plan.jj, plan.lv, qa, qb, lstar_d,
                                                     plan.lskip, cap_d, g.tlo, g.tau, qoff_d,
                                                     cursor_d, cand_u, cand_q, cand_x, flag + 1);
        prof_end(prof_slot, st, 0.0);
      }
      note_launch();
      RKR_CUDA(cudaGetLastError());
    }
  } else {
    RKR_TRY(tc_theta_pass(2, idx, idx->Ut, sub, a, kThetaSplit, flag, st));
  }
  // deep queries of [qa, qb): a contiguous slice of the gathered rows
  const int da = (int)(std::lower_bound(plan.deep.begin(), plan.deep.end(), qa) - plan.deep.begin());
  const int db = (int)(std::lower_bound(plan.deep.begin(), plan.deep.end(), qb) - plan.deep.begin());
  if (db > da) {
    TcSide ds = plan.dside;
    ds.owned = false;
    ds.rows = db - da;
    ds.hi = plan.dside.hi + (size_t)da * ds.kp;
    ds.lo = plan.dside.lo + (size_t)da * ds.kp;
    ds.rb1 = plan.dside.rb1 + da;
    ds.rb3 = plan.dside.rb3 + da;
    ThetaArgs ad = a;
    ad.qmap = plan.deep_d + da;
    ad.xs = nullptr;
    ad.lskip = 1 << 30;
    RKR_TRY(tc_theta_pass(2, idx, idx->Ut, ds, ad, kThetaSplit, flag, st));
  }
  RKR_TRY(check_flag(flag, "theta pass 2", st));
  int ovf = 0;
  RKR_CUDA(cudaMemcpy(&ovf, flag + 1, sizeof(int), cudaMemcpyDeviceToHost));
  if (ovf) return fail(RKR_EINTERNAL, "candidate segment overflow in theta pass 2");
  return RKR_OK;
}

// Group queries into chunks whose candidate total stays within budget.
static std::vector<std::pair<int, int>> chunk_queries(const std::vector<int64_t> &ncand,
                                                      int64_t budget) {
  std::vector<std::pair<int, int>> out;
  int nq = (int)ncand.size();
  int a = 0;
  while (a < nq) {
    int64_t tot = 0;
    int b = a;
    while (b < nq && (b == a || tot + ncand[b] <= budget)) tot += ncand[b++];
    out.push_back({a, b});
    a = b;
  }
  return out;
}

static int64_t candidate_budget() { return (int64_t)1 << tuning().cand_budget_log2; }



// Exact ranks of `cnt` candidates (cu, cq): canonical u.q, sort by (user, u.q),
// one grouped pass over P per user.  ccount[i] = #{p : s(u_i, p) > u_i.q_i}.
__global__ void k_compact(int64_t n, const int32_t *__restrict__ cu, const int32_t *__restrict__ cq,
                          unsigned long long *__restrict__ cursor, int32_t *__restrict__ ou,
                          int32_t *__restrict__ oq, int32_t *__restrict__ oi) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n || cu[i] < 0) return;
  unsigned long long p = atomicAdd(cursor, 1ull);
  ou[p] = cu[i];
  oq[p] = cq[i];
  oi[p] = (int32_t)i;
}

__global__ void k_scatter_back(int64_t n, const int32_t *__restrict__ oi,
                               const uint32_t *__restrict__ c2, uint32_t *__restrict__ ccount) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  ccount[oi[i]] = c2[i];
}

// Exact ranks of the candidates whose cu entry is valid (the others keep their
// ccount): compact them, canonical u.q, sort by (user, u.q), one grouped
// tensor-core pass over P per user.  ccount[i] = #{p : s(u_i, p) > u_i.q_i}.
// With clb_all (bounds mode) items the screen cannot place are not resolved:
// ccount gets an upper and clb a lower bound of the count instead.
// With ncols > 0 only the first ncols items of the norm-sorted P are screened.
static rkr_status recount_candidates(const rkr_index *idx, const float *Qd, int64_t total,
                                     const int32_t *cu_all, const int32_t *cq_all,
                                     const int32_t *qself, uint32_t *ccount_all,
                                     uint32_t *clb_all, unsigned long long *ties_d,
                                     cudaStream_t st, int64_t *nusers = nullptr,
                                     int split = 1, int64_t ncols = 0,
                                     int64_t *ncanon = nullptr) {
  TcSide Pv = idx->Pt;   // a view: the same rows, possibly fewer of them
  if (ncols > 0 && ncols < Pv.rows) Pv.rows = ncols;
  const int bs = 256;
  DevBuf bcu, bcq, bci, bcc, bcur;
  int32_t *cu, *cq, *ci;
  uint32_t *ccount;
  unsigned long long *cur;
  RKR_TRY(tmp_alloc(bcur, &cur, 1, st));
  RKR_CUDA(cudaMemsetAsync(cur, 0, sizeof(unsigned long long), st));
  RKR_TRY(tmp_alloc(bcu, &cu, total, st));
  RKR_TRY(tmp_alloc(bcq, &cq, total, st));
  RKR_TRY(tmp_alloc(bci, &ci, total, st));
  {
    const int prof_slot = prof_begin("k_compact", st);
    k_compact<<<(unsigned)((total + bs - 1) / bs), bs, 0, st>>>(total, cu_all, cq_all, cur, cu, cq,
                                                                 ci);
    prof_end(prof_slot, st, 0.0);
  }
  note_launch();
  unsigned long long hc = 0;
  RKR_CUDA(cudaMemcpyAsync(&hc, cur, sizeof(hc), cudaMemcpyDeviceToHost, st));
  RKR_CUDA(cudaStreamSynchronize(st));
  const int64_t cnt = (int64_t)hc;
  if (cnt == 0) return RKR_OK;
  if (ncanon) *ncanon += cnt;   // k_cand_theta forms each row's canonical u.q
  RKR_TRY(tmp_alloc(bcc, &ccount, cnt, st));
  int64_t Np2 = 1;
  while (Np2 < cnt) Np2 <<= 1;
  DevBuf b1, b2, b3, b4, b5, b6, b7, b8, b9;
  double *th, *ths;
  uint64_t *khi, *klo;
  int32_t *val, *slen;
  int64_t *sstart;
  uint32_t *hist;
  unsigned long long *nseg_d;
  RKR_TRY(tmp_alloc(b1, &th, cnt, st));
  RKR_TRY(tmp_alloc(b2, &khi, Np2, st));
  RKR_TRY(tmp_alloc(b3, &klo, Np2, st));
  RKR_TRY(tmp_alloc(b4, &val, Np2, st));
  RKR_TRY(tmp_alloc(b5, &sstart, cnt, st));
  RKR_TRY(tmp_alloc(b6, &slen, cnt, st));
  RKR_TRY(tmp_alloc(b7, &hist, 2 * cnt, st));
  RKR_TRY(tmp_alloc(b8, &ths, cnt, st));
  RKR_TRY(tmp_alloc(b9, &nseg_d, 3, st));
  {
    const int prof_slot = prof_begin("k_cand_theta", st);
    k_cand_theta<<<(unsigned)((Np2 + bs - 1) / bs), bs, 0, st>>>(cnt, cu, cq, idx->U, Qd, idx->d,
                                                                  th, khi, klo, val, Np2);
    prof_end(prof_slot, st, 0.0);
  }
  note_launch();
  RKR_CUDA(cudaGetLastError());
  RKR_TRY(bitonic_sort(Sort128{khi, klo, val}, Np2, "k_sort<128>", st));
  RKR_CUDA(cudaMemsetAsync(nseg_d, 0, 3 * sizeof(unsigned long long), st));
  RKR_CUDA(cudaMemsetAsync(slen, 0, sizeof(int32_t) * cnt, st));
  k_segments<<<(unsigned)((cnt + bs - 1) / bs), bs, 0, st>>>(cnt, khi, tuning().rc_seg_min,
                                                              nseg_d, sstart, slen);
  note_launch();
  RKR_CUDA(cudaGetLastError());
  unsigned long long segu[3] = {0, 0, 0};
  RKR_CUDA(cudaMemcpyAsync(segu, nseg_d, sizeof(segu), cudaMemcpyDeviceToHost, st));
  RKR_CUDA(cudaStreamSynchronize(st));
  const int64_t n1 = (int64_t)segu[0], n2 = (int64_t)segu[2], off2 = cnt - n2;
  if (nusers) *nusers += (int64_t)segu[1];
  // per segment slot (front range: one threshold; back range: several)
  DevBuf b10, b11, b12, b13;
  int32_t *suser, *sself, *scol, *spos;
  RKR_TRY(tmp_alloc(b10, &suser, cnt, st));
  RKR_TRY(tmp_alloc(b11, &sself, cnt, st));
  RKR_TRY(tmp_alloc(b12, &scol, cnt, st));
  RKR_TRY(tmp_alloc(b13, &spos, cnt, st));
  k_seg_prep<<<(unsigned)((cnt + bs - 1) / bs), bs, 0, st>>>(
      cnt, sstart, slen, khi, val, th, cq, qself, suser, sself, ths, hist, scol, spos);
  note_launch();
  RKR_CUDA(cudaGetLastError());
  int64_t refined[2] = {0, 0};
  DevBuf bhh;
  uint32_t *hist_hi = nullptr;
  if (clb_all) {
    RKR_TRY(tmp_alloc(bhh, &hist_hi, 2 * cnt, st));
    RKR_CUDA(cudaMemsetAsync(hist_hi, 0, sizeof(uint32_t) * 2 * cnt, st));
  }
  {
    ProfScope prof(ncols > 0   ? "span:recount(prefix)"
                   : clb_all ? (split ? "span:recount(bounds,split)" : "span:recount(bounds,single)")
                             : "span:recount(exact)",
                   st, 0.0);
    if (n1 > 0)
      RKR_TRY(tc_recount(idx, idx->Ut, Pv, n1, cnt, sstart, slen, suser, sself, ths, hist,
                         hist_hi, st, refined, split));
    if (n2 > 0) {
      int64_t ref2[2] = {0, 0};
      RKR_TRY(tc_recount(idx, idx->Ut, Pv, n2, cnt, sstart + off2, slen + off2,
                         suser + off2, sself + off2, ths, hist, hist_hi, st, ref2, split, scol,
                         spos));
      refined[0] += ref2[0];
      refined[1] += ref2[1];
    }
  }
  const int64_t nseg = cnt;   // the kernels below walk every slot and skip the empty ones
  {
    const int prof_slot = prof_begin("k_seg_suffix", st);
    k_seg_suffix<<<(unsigned)((nseg + bs - 1) / bs), bs, 0, st>>>((int64_t)nseg, sstart, slen,
                                                                   hist);
    prof_end(prof_slot, st, 0.0);
  }
  note_launch();
  RKR_CUDA(cudaGetLastError());
  if (ties_d) {  // accumulate over chunks: [0] undecided items, [1] canonical evaluations
    unsigned long long r[2] = {0, 0};
    RKR_CUDA(cudaMemcpyAsync(r, ties_d, sizeof(r), cudaMemcpyDeviceToHost, st));
    RKR_CUDA(cudaStreamSynchronize(st));
    r[0] += (unsigned long long)refined[0];
    r[1] += (unsigned long long)refined[1];
    RKR_CUDA(cudaMemcpyAsync(ties_d, r, sizeof(r), cudaMemcpyHostToDevice, st));
    RKR_CUDA(cudaStreamSynchronize(st));
  }
  {
    const int prof_slot = prof_begin("k_scatter_counts", st);
    k_scatter_counts<<<(unsigned)((nseg + bs - 1) / bs), bs, 0, st>>>((int64_t)nseg, sstart, slen,
                                                                     val, hist, ccount);
    prof_end(prof_slot, st, 0.0);
  }
  note_launch();
  if (clb_all) {  // lower ends into clb, upper ends (below) into ccount
    k_scatter_back<<<(unsigned)((cnt + bs - 1) / bs), bs, 0, st>>>(cnt, ci, ccount, clb_all);
    note_launch();
    k_seg_suffix<<<(unsigned)((nseg + bs - 1) / bs), bs, 0, st>>>((int64_t)nseg, sstart, slen,
                                                                   hist_hi);
    note_launch();
    k_scatter_counts<<<(unsigned)((nseg + bs - 1) / bs), bs, 0, st>>>((int64_t)nseg, sstart,
                                                                     slen, val, hist_hi, ccount);
    note_launch();
  }
  k_scatter_back<<<(unsigned)((cnt + bs - 1) / bs), bs, 0, st>>>(cnt, ci, ccount, ccount_all);
  note_launch();
  RKR_CUDA(cudaGetLastError());
  return RKR_OK;
}

// Candidates whose count interval has closed (lower == upper) need no recount.
__global__ void k_drop_decided(int64_t n, const uint32_t *__restrict__ ccount,
                               const uint32_t *__restrict__ clb, int32_t *__restrict__ cu_fb) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n && cu_fb[i] >= 0 && ccount[i] == clb[i]) cu_fb[i] = -1;
}

static rkr_status count_valid(const int32_t *v, int64_t n, unsigned long long *out,
                              cudaStream_t st) {
  DevBuf b;
  unsigned long long *d;
  RKR_TRY(tmp_alloc(b, &d, 1, st));
  RKR_CUDA(cudaMemsetAsync(d, 0, sizeof(unsigned long long), st));
  k_count_valid<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, v, d);
  note_launch();
  RKR_CUDA(cudaMemcpyAsync(out, d, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
  RKR_CUDA(cudaStreamSynchronize(st));
  return RKR_OK;
}

// Early termination over the norm-sorted items (tuning rc_prefix; Alg. 1 sorts P
// by descending norm).  For the queries with many candidates still to recount,
// every such candidate is first screened against the first m1 items only: its
// certain count there is a lower bound of its count over P, and its possible
// count there ranks how promising it is.  The query's most promising candidates
// are recounted over all of P, the cap (k-th smallest count upper bound) is taken
// again, and every other candidate whose prefix lower bound exceeds the cap is
// dropped unrecounted: it cannot be among the k smallest ranks.  The rest go back
// to the recount.  On return *h2 is the number of candidates still to recount.
static rkr_status prefix_prune(const rkr_index *idx, const QueryCommon &qc, int qa, int qb,
                               int64_t cnt, const int64_t *qoff_rel, const uint32_t *cursor,
                               const int32_t *cq, const int32_t *qself, uint32_t *ccount,
                               uint32_t *clb, int32_t *cu_fb, int64_t *recount_users,
                               unsigned long long *h2, int64_t *rows, int64_t *pruned,
                               int64_t *ncanon, cudaStream_t st) {
  const int64_t m1 = idx->m / tuning().rc_prefix / 256 * 256;
  if (m1 < 256 || m1 >= idx->m) return RKR_OK;
  DevBuf b1, b2, b3, b4, b5;
  int32_t *cu_pre, *cu_park;
  uint32_t *hi1, *lo1;
  unsigned long long *npre_d, npre = 0;
  RKR_TRY(tmp_alloc(b1, &cu_pre, cnt, st));
  RKR_TRY(tmp_alloc(b2, &cu_park, cnt, st));
  RKR_TRY(tmp_alloc(b3, &hi1, cnt, st));
  RKR_TRY(tmp_alloc(b4, &lo1, cnt, st));
  RKR_TRY(tmp_alloc(b5, &npre_d, 1, st));
  RKR_CUDA(cudaMemsetAsync(cu_pre, 0xff, sizeof(int32_t) * cnt, st));
  RKR_CUDA(cudaMemsetAsync(cu_park, 0xff, sizeof(int32_t) * cnt, st));
  RKR_CUDA(cudaMemsetAsync(hi1, 0xff, sizeof(uint32_t) * cnt, st));
  RKR_CUDA(cudaMemsetAsync(lo1, 0, sizeof(uint32_t) * cnt, st));
  RKR_CUDA(cudaMemsetAsync(npre_d, 0, sizeof(unsigned long long), st));
  k_prefix_split<<<qb - qa, 256, 0, st>>>(qa, qoff_rel, cursor, qc.kq_d, cu_fb, cu_pre, npre_d);
  note_launch();
  RKR_CUDA(cudaGetLastError());
  RKR_CUDA(cudaMemcpyAsync(&npre, npre_d, sizeof(npre), cudaMemcpyDeviceToHost, st));
  RKR_CUDA(cudaStreamSynchronize(st));
  if (npre == 0) return RKR_OK;
  *rows += (int64_t)npre;
  // certain (lo1) and possible (hi1) counts over the prefix, single product
  RKR_TRY(recount_candidates(idx, qc.Qd, cnt, cu_pre, cq, qself, hi1, lo1, nullptr, st, nullptr,
                             0, m1, ncanon));
  k_prefix_pick<<<qb - qa, kFilterThreads, 0, st>>>(qa, qoff_rel, cursor, qc.kq_d, cu_pre, hi1, lo1, clb,
                                          cu_fb, cu_park);
  note_launch();
  RKR_CUDA(cudaGetLastError());
  unsigned long long parked = 0, kept = 0, h = 0;
  RKR_TRY(count_valid(cu_park, cnt, &parked, st));
  RKR_TRY(count_valid(cu_fb, cnt, &h, st));
  if (h > 0)  // the promising rows and the other queries' rows, over all of P
    RKR_TRY(recount_candidates(idx, qc.Qd, cnt, cu_fb, cq, qself, ccount, clb, nullptr, st,
                               recount_users, tuning().rc_single_first ? 0 : 1, 0, ncanon));
  {
    const int prof_slot = prof_begin("k_recount_filter", st);
    k_recount_filter<<<qb - qa, kFilterThreads, 0, st>>>(qa, qoff_rel, cursor, qc.kq_d, ccount, clb, cu_fb);
    k_recount_filter<<<qb - qa, kFilterThreads, 0, st>>>(qa, qoff_rel, cursor, qc.kq_d, ccount, clb,
                                              cu_park);
    prof_end(prof_slot, st, 0.0);
  }
  note_launch();
  note_launch();
  k_drop_decided<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(cnt, ccount, clb, cu_fb);
  note_launch();
  RKR_CUDA(cudaGetLastError());
  RKR_TRY(count_valid(cu_park, cnt, &kept, st));
  *pruned += (int64_t)(parked - kept);
  k_prefix_unpark<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(cnt, cu_park, cu_fb);
  note_launch();
  RKR_CUDA(cudaGetLastError());
  RKR_TRY(count_valid(cu_fb, cnt, h2, st));
  return RKR_OK;
}

rkr_status run_query_approx(const rkr_index *idx, const QueryCommon &qc, int nq, double c,
                            int32_t *users_d, uint32_t *nlo_d, uint32_t *nup_d, double *est_d,
                            int32_t *case_d, int32_t *nc_d, rkr_query_stats *stats,
                            cudaStream_t st) {
  DevBuf bl, bn, bcap;
  int32_t *lstar_d;
  int64_t *ncand_d;
  uint32_t *cap_d;
  RKR_TRY(tmp_alloc(bl, &lstar_d, nq, st));
  RKR_TRY(tmp_alloc(bn, &ncand_d, nq, st));
  RKR_TRY(tmp_alloc(bcap, &cap_d, nq, st));
  DevBuf bse, bnf;
  int *sel_err;
  unsigned long long *nfp64_d;
  RKR_TRY(tmp_alloc(bse, &sel_err, 1, st));
  RKR_CUDA(cudaMemsetAsync(sel_err, 0, sizeof(int), st));
  RKR_TRY(tmp_alloc(bnf, &nfp64_d, 1, st));
  RKR_CUDA(cudaMemsetAsync(nfp64_d, 0, sizeof(unsigned long long), st));
  Plan plan;
  Timer t1(st);
  const Grid grid{qc.bf,  idx->fmin, idx->tau, idx->JU, idx->JL, idx->nlev_a,
                  idx->N, idx->N,    (uint32_t)(idx->m * idx->s), (uint32_t)idx->s};
  RKR_TRY(screen_plan(idx, qc, nq, grid, st, lstar_d, cap_d, ncand_d, plan));
  double ms_theta = t1.stop(), ms_res = 0.0, ms_sel = 0.0;
  int64_t total = 0;
  int wide = 0;
  for (int q = 0; q < nq; ++q) wide += plan.lstar[q] >= idx->nlev_a - 1;
  std::vector<int64_t> qoff(nq + 1, 0);
  for (int q = 0; q < nq; ++q) qoff[q + 1] = qoff[q] + plan.ncand[q];
  DevBuf bo;
  int64_t *qoff_d;
  RKR_TRY(tmp_alloc(bo, &qoff_d, nq + 1, st));
  RKR_CUDA(cudaMemcpyAsync(qoff_d, qoff.data(), sizeof(int64_t) * (nq + 1),
                           cudaMemcpyHostToDevice, st));
  for (auto ch : chunk_queries(plan.ncand, candidate_budget())) {
    int qa = ch.first, qb = ch.second;
    int64_t cnt = qoff[qb] - qoff[qa];
    DevBuf b1, b2, b3, b4, b5, b6, b7, b8, b9;
    int32_t *cu, *cq, *cj;
    uint32_t *cursor, *nlo, *nup;
    double *th;
    float *cx;
    int64_t *qoff_rel;
    RKR_TRY(tmp_alloc(b9, &cx, cnt, st));
    RKR_CUDA(cudaMemsetAsync(cx, 0xff, sizeof(float) * std::max<int64_t>(cnt, 1), st));  // NaN
    RKR_TRY(tmp_alloc(b1, &cu, cnt, st));
    RKR_TRY(tmp_alloc(b2, &cq, cnt, st));
    RKR_TRY(tmp_alloc(b3, &cursor, nq, st));
    RKR_TRY(tmp_alloc(b4, &th, cnt, st));
    RKR_TRY(tmp_alloc(b5, &cj, cnt, st));
    RKR_TRY(tmp_alloc(b6, &nlo, cnt, st));
    RKR_TRY(tmp_alloc(b7, &nup, cnt, st));
    RKR_TRY(tmp_alloc(b8, &qoff_rel, nq + 1, st));
    // offsets relative to the chunk start, so candidate arrays hold only this chunk
    std::vector<int64_t> rel(nq + 1, 0);
    for (int q = 0; q <= nq; ++q) rel[q] = qoff[q] - qoff[qa];
    RKR_CUDA(cudaMemcpyAsync(qoff_rel, rel.data(), sizeof(int64_t) * (nq + 1),
                             cudaMemcpyHostToDevice, st));
    RKR_CUDA(cudaMemsetAsync(cursor, 0, sizeof(uint32_t) * nq, st));
    RKR_CUDA(cudaMemsetAsync(cu, 0xff, sizeof(int32_t) * std::max<int64_t>(cnt, 1), st));
    Timer t2(st);
    RKR_TRY(emit_candidates(idx, qc, qa, qb, grid, plan, lstar_d, cap_d, qoff_rel, cursor, cu, cq,
                            cx, st));
    ms_theta += t2.stop();
    {
      std::vector<uint32_t> hc(nq);
      RKR_CUDA(cudaMemcpyAsync(hc.data(), cursor, sizeof(uint32_t) * nq, cudaMemcpyDeviceToHost,
                               st));
      RKR_CUDA(cudaStreamSynchronize(st));
      for (int q = qa; q < qb; ++q) total += hc[q];
    }
    Timer t3(st);
    if (cnt > 0) {
      {
        const int prof_slot = prof_begin("k_resolve_approx", st);
        k_resolve_approx<<<(unsigned)((cnt + 127) / 128), 128, 0, st>>>(
            cnt, cu, cq, cx, idx->Ut.rb3, qc.Qt.rb3, tc_gacc(idx->Ut.kp, 1), tc_gcan(idx->d),
            idx->U, qc.Qd, idx->d, idx->fmin, idx->delta, qc.bf, idx->N, idx->tau,
            (uint32_t)(idx->m * idx->s), th, cj, nlo, nup, nfp64_d);
        prof_end(prof_slot, st, 0.0);
        note_launch();
      }
      RKR_CUDA(cudaGetLastError());
    }
    ms_res += t3.stop();
    Timer t4(st);
    ApproxCand C{cu, nlo, nup, th, cj, idx->U, qc.Qd, idx->d, nfp64_d};
    size_t sm = sizeof(SortEnt) * kMaxK;
    RKR_CUDA(cudaFuncSetAttribute(k_select_approx, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sm));
    {
      const int prof_slot = prof_begin("k_select_approx", st);
      k_select_approx<<<qb - qa, kSelThreads, sm, st>>>(qa, qoff_rel, cursor, C, qc.kq_d, c,
                                                        (uint32_t)idx->s, idx->tau, idx->fmin,
                                                        idx->delta, qc.out_off_d, users_d, nlo_d,
                                                        nup_d, est_d, case_d, nc_d, sel_err);
      prof_end(prof_slot, st, 0.0);
    }
    note_launch();
    RKR_CUDA(cudaGetLastError());
    ms_sel += t4.stop();
  }
  RKR_CUDA(cudaStreamSynchronize(st));
  {
    int h = 0;
    RKR_CUDA(cudaMemcpy(&h, sel_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) return fail(RKR_EINTERNAL, "fewer than k candidates for a query");
  }
  if (stats) {
    stats->pairs = idx->n * (int64_t)nq;
    stats->candidates = total;
    unsigned long long nf = 0;
    RKR_CUDA(cudaMemcpyAsync(&nf, nfp64_d, sizeof(nf), cudaMemcpyDeviceToHost, st));
    RKR_CUDA(cudaStreamSynchronize(st));
    stats->fp64_dots = (int64_t)nf;
    stats->near_ties = 0;
    stats->wide_queries = wide;
    stats->deep_queries = (int32_t)plan.deep.size();
    stats->ms_theta = ms_theta;
    stats->ms_resolve = ms_res;
    stats->ms_select = ms_sel;
  }
  return RKR_OK;
}

rkr_status launch_select_approx(int qa, int nblocks, const int64_t *qoff, const uint32_t *qcount,
                                const int32_t *uid, const uint32_t *nlo, const uint32_t *nup,
                                double *th, const int32_t *cj, const float *Qd,
                                const int32_t *kq, double c, const int64_t *out_off,
                                int32_t *users_d, uint32_t *nlo_d, uint32_t *nup_d, double *est_d,
                                int32_t *case_d, int32_t *nc_d, int *err, cudaStream_t st,
                                const rkr_index *idx) {
  ApproxCand C{uid, nlo, nup, th, cj, idx->U, Qd, idx->d, nullptr};
  size_t sm = sizeof(SortEnt) * kMaxK;
  RKR_CUDA(cudaFuncSetAttribute(k_select_approx, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sm));
  const int prof_slot = prof_begin("k_select_approx", st);
  k_select_approx<<<nblocks, kSelThreads, sm, st>>>(qa, qoff, qcount, C, kq, c, (uint32_t)idx->s,
                                                   idx->tau, idx->fmin, idx->delta, out_off,
                                                   users_d, nlo_d, nup_d, est_d, case_d, nc_d,
                                                   err);
  prof_end(prof_slot, st, 0.0);
  note_launch();
  RKR_CUDA(cudaGetLastError());
  return RKR_OK;
}

struct LearnedPrune {
  rkr_pruner *pr;
  const float *Xu;   // per-user features
  const int32_t *keep;  // candidates kept per query (device, nq)
  int certify;          // 1: exact fallback for cut candidates that could still matter
  bool table;           // predictions from the pruner's per-user tables
};

constexpr int64_t kLearnedUncut = 32;

// Per query (one block), among the candidates still to be recounted (fb >= 0):
// those whose predicted log rank y is above the keep[q]-th smallest prediction
// are cut (fb = cu = -1, count = the largest key, so selection never takes them).
// Candidates whose exact count is known already are not touched.
__global__ void __launch_bounds__(kFilterThreads)
    k_learned_cut(int qa, const int64_t *__restrict__ qoff, const uint32_t *__restrict__ qcount,
                  const int32_t *__restrict__ keep_q, const float *__restrict__ y,
                  int32_t *__restrict__ fb_all, int32_t *__restrict__ cu_all,
                  uint32_t *__restrict__ ccount, int32_t *__restrict__ cutu_all,
                  int64_t n_users, unsigned long long *__restrict__ ncut) {
  __shared__ uint32_t hist[256];
  __shared__ uint64_t bc[2];
  __shared__ unsigned long long acc;
  const int q = qa + blockIdx.x;
  const int64_t base = qoff[q] - qoff[qa];
  const int64_t cnt = qcount[q];
  const int64_t keep = keep_q[q];
  int32_t *fb = fb_all + base, *cu = cu_all + base, *cutu = cutu_all + base;
  uint32_t *cc = ccount + base;
  const float *yy = y + base;
  auto key_of = [&](int64_t i) {
    const uint32_t b = __float_as_uint(yy[i]);
    return (uint64_t)((b & 0x80000000u) ? ~b : (b | 0x80000000u));
  };
  const int64_t open = block_count(cnt, [&](int64_t i) { return fb[i] >= 0; }, &acc);
  // a query whose candidates to recount are a large part of all users and far more
  // than it keeps is left uncut: such candidates have weak rank lower bounds (u.q
  // lies below the tail lists) and the exact fallback would revive them anyway
  if (open <= keep || (n_users > 0 && open > kLearnedUncut * keep && open > n_users / 4)) return;
  const uint64_t kth = block_kth(cnt, (uint64_t)keep, 32,
                                 [&](int64_t i, uint64_t &key) {
                                   if (fb[i] < 0) return false;
                                   key = key_of(i);
                                   return true;
                                 },
                                 hist, bc);
  __syncthreads();
  const int64_t cut = block_count(cnt, [&](int64_t i) { return fb[i] >= 0 && key_of(i) > kth; },
                                  &acc);
  for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x)
    if (fb[i] >= 0 && key_of(i) > kth) {
      cutu[i] = cu[i];   // kept for the exact fallback
      fb[i] = -1;
      cu[i] = -1;
      cc[i] = 0xffffffffu;
    }
  if (threadIdx.x == 0) atomicAdd(ncut, (unsigned long long)cut);
}

// Exact fallback of the learned cut (one block per query).  cap = the k-th
// smallest count among the candidates not cut, an upper bound of the k-th
// smallest count of all candidates.  A cut candidate whose lower bound clb is at
// most cap could still be among the k best: it is revived (its user restored and
// sent to the recount).  The others have count >= clb > cap and cannot be.
__global__ void __launch_bounds__(256)
    k_learned_revive(int qa, const int64_t *__restrict__ qoff,
                     const uint32_t *__restrict__ qcount, const int32_t *__restrict__ kq,
                     const uint32_t *__restrict__ ccount, const uint32_t *__restrict__ clb,
                     int32_t *__restrict__ fb_all, int32_t *__restrict__ cu_all,
                     int32_t *__restrict__ cutu_all, unsigned long long *__restrict__ nrev) {
  __shared__ uint32_t hist[256];
  __shared__ uint64_t bc[2];
  __shared__ unsigned long long acc;
  const int q = qa + blockIdx.x;
  const int64_t base = qoff[q] - qoff[qa];
  const int64_t cnt = qcount[q];
  const int k = kq[q];
  if (cnt < k) return;
  int32_t *fb = fb_all + base, *cu = cu_all + base, *cutu = cutu_all + base;
  const uint32_t *cc = ccount + base, *lb = clb + base;
  const uint64_t cap = block_kth(cnt, (uint64_t)k, 32,
                                 [&](int64_t i, uint64_t &key) { key = cc[i]; return true; },
                                 hist, bc);
  const int64_t rev = block_count(cnt, [&](int64_t i) {
    return cutu[i] >= 0 && (uint64_t)lb[i] <= cap;
  }, &acc);
  for (int64_t i = threadIdx.x; i < cnt; i += blockDim.x)
    if (cutu[i] >= 0 && (uint64_t)lb[i] <= cap) {
      cu[i] = cutu[i];
      fb[i] = cutu[i];
      cutu[i] = -1;
    }
  if (threadIdx.x == 0 && rev) atomicAdd(nrev, (unsigned long long)rev);
}

// Predictions scattered back to candidate slots: y[oi[j]] = yc[j].
__global__ void k_scatter_y(int64_t n, const int32_t *__restrict__ oi,
                            const float *__restrict__ yc, float *__restrict__ y) {
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j < n) y[oi[j]] = yc[j];
}

// t = u.q / ||u|| of each pair (FP32; 0 for an invalid user index).
__global__ void k_pair_scores(int64_t npairs, const int32_t *__restrict__ cu,
                              const int32_t *__restrict__ cq, const float *__restrict__ U,
                              const float *__restrict__ Q, int d, float *__restrict__ t) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= npairs) return;
  const int64_t u = cu[i];
  if (u < 0) { t[i] = 0.0f; return; }
  const float *uu = U + u * d, *qq = Q + (int64_t)cq[i] * d;
  float s = 0.0f, nn = 0.0f;
  for (int k = 0; k < d; ++k) {
    s = fmaf(uu[k], qq[k], s);
    nn = fmaf(uu[k], uu[k], nn);
  }
  t[i] = nn > 0.0f ? s / sqrtf(nn) : 0.0f;
}

// t of compacted candidate pairs: x / ||u|| from the screened score x = cx[fi] of
// the pair (the network needs no exact t), else the FP32 product of the rows.
__global__ void k_pair_t(int64_t npairs, const int32_t *__restrict__ fu,
                         const int32_t *__restrict__ fq, const int32_t *__restrict__ fi,
                         const float *__restrict__ cx, const float *__restrict__ unrm,
                         const float *__restrict__ U, const float *__restrict__ Q, int d,
                         float *__restrict__ t) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= npairs) return;
  const int64_t u = fu[i];
  const float x = cx[fi[i]];
  const float nu = unrm[u];
  if (x == x && nu > 0.0f) {
    t[i] = x / nu;
    return;
  }
  const float *uu = U + u * d, *qq = Q + (int64_t)fq[i] * d;
  float s = 0.0f, nn = 0.0f;
  for (int k = 0; k < d; ++k) {
    s = fmaf(uu[k], qq[k], s);
    nn = fmaf(uu[k], uu[k], nn);
  }
  t[i] = nn > 0.0f ? s / sqrtf(nn) : 0.0f;
}

// Per user: R u / ||u|| (64 values) and log ||u||.
__global__ void k_user_features(int64_t n, int d, const float *__restrict__ U,
                                const float *__restrict__ R, float *__restrict__ Xu) {
  const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= n) return;
  const float *uu = U + u * d;
  float nn = 0.0f;
  for (int k = 0; k < d; ++k) nn = fmaf(uu[k], uu[k], nn);
  const float nrm = sqrtf(nn), inv = nrm > 0.0f ? 1.0f / nrm : 0.0f;
  for (int j = 0; j < 64; ++j) {
    float a = 0.0f;
    for (int k = 0; k < d; ++k) a = fmaf(R[j * d + k], uu[k], a);
    Xu[u * 65 + j] = a * inv;
  }
  Xu[u * 65 + 64] = logf(fmaxf(nrm, 1e-30f));
}

rkr_status user_features(const rkr_index *idx, const float *R, float *Xu, cudaStream_t st) {
  k_user_features<<<(unsigned)((idx->n + 127) / 128), 128, 0, st>>>(idx->n, idx->d, idx->U, R,
                                                                     Xu);
  note_launch();
  RKR_CUDA(cudaGetLastError());
  return RKR_OK;
}

rkr_status pair_scores(const rkr_index *idx, const float *Qd, int64_t npairs, const int32_t *cu,
                       const int32_t *cq, float *t, cudaStream_t st) {
  if (npairs <= 0) return RKR_OK;
  k_pair_scores<<<(unsigned)((npairs + 127) / 128), 128, 0, st>>>(npairs, cu, cq, idx->U, Qd,
                                                                   idx->d, t);
  note_launch();
  RKR_CUDA(cudaGetLastError());
  return RKR_OK;
}

static rkr_status query_exact_core(const rkr_index *idx, const QueryCommon &qc, int nq,
                                   const LearnedPrune *lp, int32_t *users_d, int32_t *ranks_d,
                                   rkr_query_stats *stats, cudaStream_t st);

rkr_status run_query_exact(const rkr_index *idx, const QueryCommon &qc, int nq,
                           int32_t *users_d, int32_t *ranks_d, rkr_query_stats *stats,
                           cudaStream_t st) {
  return query_exact_core(idx, qc, nq, nullptr, users_d, ranks_d, stats, st);
}

rkr_status run_query_exact_learned(const rkr_index *idx, const QueryCommon &qc, int nq,
                                   rkr_pruner *pr, const float *Xu, const int32_t *keep_d,
                                   int certify, bool use_table, int32_t *users_d,
                                   int32_t *ranks_d, rkr_query_stats *stats, cudaStream_t st) {
  const LearnedPrune lp{pr, Xu, keep_d, certify, use_table};
  return query_exact_core(idx, qc, nq, &lp, users_d, ranks_d, stats, st);
}

// The learned cut of one chunk: predictions for the candidates still to be
// recounted (nfb of them, compacted), then k_learned_cut per query.
static rkr_status learned_cut(const rkr_index *idx, const QueryCommon &qc, const LearnedPrune *lp,
                              int qa, int qb, int64_t cnt, int64_t nfb, const int64_t *qoff_rel,
                              const uint32_t *cursor, int32_t *cu, const int32_t *cq,
                              const float *cx, int32_t *cu_fb, uint32_t *ccount, int32_t *cutu,
                              int64_t *cut_total, cudaStream_t st) {
  DevBuf b1, b2, b3, b4, b5, b6, b7, b8;
  int32_t *fu, *fq, *fi;
  unsigned long long *cur, *ncut;
  float *tq, *yc, *y;
  RKR_TRY(tmp_alloc(b1, &fu, nfb, st));
  RKR_TRY(tmp_alloc(b2, &fq, nfb, st));
  RKR_TRY(tmp_alloc(b3, &fi, nfb, st));
  RKR_TRY(tmp_alloc(b4, &cur, 1, st));
  RKR_TRY(tmp_alloc(b5, &ncut, 1, st));
  RKR_TRY(tmp_alloc(b6, &tq, nfb, st));
  RKR_TRY(tmp_alloc(b7, &yc, nfb, st));
  RKR_TRY(tmp_alloc(b8, &y, cnt, st));
  RKR_CUDA(cudaMemsetAsync(cur, 0, sizeof(unsigned long long), st));
  RKR_CUDA(cudaMemsetAsync(ncut, 0, sizeof(unsigned long long), st));
  k_compact<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(cnt, cu_fb, cq, cur, fu, fq, fi);
  note_launch();
  RKR_CUDA(cudaGetLastError());
  // the network's input t = u.q / ||u||: from the candidate's screened score where
  // it has one (no row is read), else from the rows
  k_pair_t<<<(unsigned)((nfb + 127) / 128), 128, 0, st>>>(nfb, fu, fq, fi, cx, idx->unrm, idx->U,
                                                          qc.Qd, idx->d, tq);
  note_launch();
  RKR_CUDA(cudaGetLastError());
  if (lp->table) {   // one lookup per pair in the user's table
    ProfScope prof("pruner_table", st);
    RKR_TRY(pruner_table_predict(lp->pr, fu, tq, nfb, yc, st));
  } else {
    ProfScope prof("pruner_forward", st);
    RKR_TRY(pruner_forward_gather(lp->pr, lp->Xu, fu, tq, nfb, yc, st));
  }
  k_scatter_y<<<(unsigned)((nfb + 255) / 256), 256, 0, st>>>(nfb, fi, yc, y);
  note_launch();
  // the uncut rule exists for the fallback's sake (n_users = 0 switches it off)
  k_learned_cut<<<qb - qa, kFilterThreads, 0, st>>>(qa, qoff_rel, cursor, lp->keep, y, cu_fb, cu, ccount,
                                         cutu, lp->certify ? idx->n : 0, ncut);
  note_launch();
  RKR_CUDA(cudaGetLastError());
  unsigned long long h = 0;
  RKR_CUDA(cudaMemcpyAsync(&h, ncut, sizeof(h), cudaMemcpyDeviceToHost, st));
  RKR_CUDA(cudaStreamSynchronize(st));
  *cut_total += (int64_t)h;
  return RKR_OK;
}

static rkr_status query_exact_core(const rkr_index *idx, const QueryCommon &qc, int nq,
                                   const LearnedPrune *lp, int32_t *users_d, int32_t *ranks_d,
                                   rkr_query_stats *stats, cudaStream_t st) {
  DevBuf bl, bn, bt, bcap;
  int32_t *lstar_d;
  int64_t *ncand_d;
  uint32_t *cap_d;
  unsigned long long *ties_d;
  RKR_TRY(tmp_alloc(bl, &lstar_d, nq, st));
  RKR_TRY(tmp_alloc(bn, &ncand_d, nq, st));
  RKR_TRY(tmp_alloc(bcap, &cap_d, nq, st));
  DevBuf bse;
  int *sel_err;
  RKR_TRY(tmp_alloc(bse, &sel_err, 1, st));
  RKR_CUDA(cudaMemsetAsync(sel_err, 0, sizeof(int), st));
  RKR_TRY(tmp_alloc(bt, &ties_d, 2, st));
  RKR_CUDA(cudaMemsetAsync(ties_d, 0, 2 * sizeof(unsigned long long), st));
  DevBuf bls;
  unsigned long long *lstat;
  RKR_TRY(tmp_alloc(bls, &lstat, 5, st));
  DevBuf bqs;
  int32_t *qself;
  RKR_TRY(tmp_alloc(bqs, &qself, nq, st));
  RKR_TRY(query_self(idx, qc.Qd, nq, qself, st));
  int64_t fallback = 0, list_fp64 = 0, cut_total = 0;
  double err_ratio = 0.0, err_rel = 0.0;
  int64_t recount_users = 0, recount_open = 0, recount_split = 0, revived = 0;
  int64_t prefix_rows = 0, prefix_pruned = 0, canon_rows = 0, canon_theta = 0;
  unsigned long long lstat_host_fb = 0;
  Plan plan;
  Timer t1(st);
  const Grid grid{qc.xbf,   idx->xg0, idx->xg,       idx->XJU, idx->XJL, idx->nlev_x,
                  idx->XHI, idx->XLO, (uint32_t)idx->m, 1u};
  RKR_TRY(screen_plan(idx, qc, nq, grid, st, lstar_d, cap_d, ncand_d, plan));
  double ms_theta = t1.stop(), ms_res = 0.0, ms_sel = 0.0;
  int64_t total = 0;
  int wide = 0;
  for (int q = 0; q < nq; ++q) wide += plan.lstar[q] >= idx->nlev_x - 1;
  std::vector<int64_t> qoff(nq + 1, 0);
  for (int q = 0; q < nq; ++q) qoff[q + 1] = qoff[q] + plan.ncand[q];
  for (auto ch : chunk_queries(plan.ncand, candidate_budget())) {
    int qa = ch.first, qb = ch.second;
    int64_t cnt = qoff[qb] - qoff[qa];
    DevBuf b1, b2, b3, b4, b8, b9;
    int32_t *cu, *cq;
    uint32_t *cursor, *ccount;
    float *cx;
    int64_t *qoff_rel;
    RKR_TRY(tmp_alloc(b9, &cx, cnt, st));
    RKR_CUDA(cudaMemsetAsync(cx, 0xff, sizeof(float) * std::max<int64_t>(cnt, 1), st));  // NaN
    RKR_TRY(tmp_alloc(b1, &cu, cnt, st));
    RKR_TRY(tmp_alloc(b2, &cq, cnt, st));
    RKR_TRY(tmp_alloc(b3, &cursor, nq, st));
    RKR_TRY(tmp_alloc(b4, &ccount, cnt, st));
    RKR_TRY(tmp_alloc(b8, &qoff_rel, nq + 1, st));
    std::vector<int64_t> rel(nq + 1, 0);
    for (int q = 0; q <= nq; ++q) rel[q] = qoff[q] - qoff[qa];
    RKR_CUDA(cudaMemcpyAsync(qoff_rel, rel.data(), sizeof(int64_t) * (nq + 1),
                             cudaMemcpyHostToDevice, st));
    RKR_CUDA(cudaMemsetAsync(cursor, 0, sizeof(uint32_t) * nq, st));
    RKR_CUDA(cudaMemsetAsync(cu, 0xff, sizeof(int32_t) * std::max<int64_t>(cnt, 1), st));
    Timer t2(st);
    RKR_TRY(emit_candidates(idx, qc, qa, qb, grid, plan, lstar_d, cap_d, qoff_rel, cursor, cu, cq,
                            cx, st));
    ms_theta += t2.stop();
    {
      std::vector<uint32_t> hc(nq);
      RKR_CUDA(cudaMemcpyAsync(hc.data(), cursor, sizeof(uint32_t) * nq, cudaMemcpyDeviceToHost,
                               st));
      RKR_CUDA(cudaStreamSynchronize(st));
      for (int q = qa; q < qb; ++q) total += hc[q];
    }
    Timer t3(st);
    if (cnt > 0) {
      DevBuf bfb, blb;
      int32_t *cu_fb;
      uint32_t *clb;
      RKR_TRY(tmp_alloc(bfb, &cu_fb, cnt, st));
      RKR_TRY(tmp_alloc(blb, &clb, cnt, st));
      RKR_CUDA(cudaMemsetAsync(lstat, 0, 5 * sizeof(unsigned long long), st));
      {
        const int prof_slot = prof_begin("k_list_rank", st);
        k_list_rank<<<(unsigned)((cnt + 127) / 128), 128, 0, st>>>(
            cnt, cu, cq, cx, qc.Qt.rb3, idx->U, idx->unrm, qc.Qd, idx->Ps, idx->pnrm_s, idx->d,
            idx->xlist, idx->xloff, idx->xlcap, idx->xcoff, idx->xlcnt, idx->xbmax, idx->Ut.rb3, idx->ptile3,
            idx->ptile_bn, tc_gacc(idx->Ut.kp, 1), tc_gcan(idx->d), idx->xg0, idx->xdx, idx->xg,
            idx->ldx, kListG,
            idx->XLO, idx->XHI, (uint32_t)idx->m, ccount, clb, cu_fb, qself, deep_grid(idx),
            lstat);
        prof_end(prof_slot, st, 0.0);
      }
      note_launch();
      RKR_CUDA(cudaGetLastError());
      {
        const int prof_slot = prof_begin("k_recount_filter", st);
        k_recount_filter<<<qb - qa, kFilterThreads, 0, st>>>(qa, qoff_rel, cursor, qc.kq_d, ccount, clb, cu_fb);
        prof_end(prof_slot, st, 0.0);
      }
      note_launch();
      RKR_CUDA(cudaGetLastError());
      {  // candidates that still need the recount
        DevBuf bn2;
        unsigned long long *nfb;
        RKR_TRY(tmp_alloc(bn2, &nfb, 1, st));
        RKR_CUDA(cudaMemsetAsync(nfb, 0, sizeof(unsigned long long), st));
        k_count_valid<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(cnt, cu_fb, nfb);
        note_launch();
        RKR_CUDA(cudaMemcpyAsync(&lstat_host_fb, nfb, sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, st));
        RKR_CUDA(cudaStreamSynchronize(st));
      }
      unsigned long long ls[5] = {0, 0, 0, 0, 0};
      RKR_CUDA(cudaMemcpyAsync(ls, lstat, sizeof(ls), cudaMemcpyDeviceToHost, st));
      canon_theta += (int64_t)ls[4];
      RKR_CUDA(cudaStreamSynchronize(st));
      err_ratio = std::max(err_ratio, (double)u32_float((uint32_t)ls[2]));
      err_rel = std::max(err_rel, (double)u32_float((uint32_t)ls[3]));
      DevBuf bcut;
      int32_t *cutu = nullptr;
      if (lp) {
        RKR_TRY(tmp_alloc(bcut, &cutu, cnt, st));
        RKR_CUDA(cudaMemsetAsync(cutu, 0xff, sizeof(int32_t) * cnt, st));
      }
      if (lp && lstat_host_fb > 0) {  // learned cut of the candidates still to be recounted
        RKR_TRY(learned_cut(idx, qc, lp, qa, qb, cnt, (int64_t)lstat_host_fb, qoff_rel, cursor,
                            cu, cq, cx, cu_fb, ccount, cutu, &cut_total, st));
        lstat_host_fb = 0;
        DevBuf bn4;
        unsigned long long *nfb4;
        RKR_TRY(tmp_alloc(bn4, &nfb4, 1, st));
        RKR_CUDA(cudaMemsetAsync(nfb4, 0, sizeof(unsigned long long), st));
        k_count_valid<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(cnt, cu_fb, nfb4);
        note_launch();
        RKR_CUDA(cudaMemcpyAsync(&lstat_host_fb, nfb4, sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, st));
        RKR_CUDA(cudaStreamSynchronize(st));
      }
      fallback += (int64_t)lstat_host_fb;
      list_fp64 += (int64_t)ls[1];
      auto recount_open_candidates = [&](unsigned long long h2) -> rkr_status {
        // count intervals for every remaining candidate, then the cap again; only
        // candidates that can still make the k smallest and whose interval is
        // open go on.  The first pass screens with the single BF16 product (a
        // third of the tensor work, wider intervals), the second with the split
        // product on the candidates still open; the exact pass then resolves the
        // undecided items of those that remain.
        for (int pass = tuning().rc_single_first ? 0 : 1; pass < 2 && h2 > 0; ++pass) {
          const bool first = pass == 0 || !tuning().rc_single_first;
          RKR_TRY(recount_candidates(idx, qc.Qd, cnt, cu_fb, cq, qself, ccount, clb, nullptr,
                                     st, first ? &recount_users : nullptr, pass == 0 ? 0 : 1, 0,
                                     &canon_rows));
          if (pass == 1) recount_split += (int64_t)h2;
          {
            const int prof_slot = prof_begin("k_recount_filter", st);
            k_recount_filter<<<qb - qa, kFilterThreads, 0, st>>>(qa, qoff_rel, cursor, qc.kq_d, ccount,
                                                     clb, cu_fb);
            prof_end(prof_slot, st, 0.0);
          }
          note_launch();
          k_drop_decided<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(cnt, ccount, clb, cu_fb);
          note_launch();
          RKR_CUDA(cudaGetLastError());
          DevBuf bn3;
          unsigned long long *nfb2;
          RKR_TRY(tmp_alloc(bn3, &nfb2, 1, st));
          RKR_CUDA(cudaMemsetAsync(nfb2, 0, sizeof(unsigned long long), st));
          k_count_valid<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(cnt, cu_fb, nfb2);
          note_launch();
          RKR_CUDA(cudaMemcpyAsync(&h2, nfb2, sizeof(h2), cudaMemcpyDeviceToHost, st));
          RKR_CUDA(cudaStreamSynchronize(st));
        }
        recount_open += (int64_t)h2;
        if (h2 > 0)
          RKR_TRY(recount_candidates(idx, qc.Qd, cnt, cu_fb, cq, qself, ccount, nullptr, ties_d,
                                     st, nullptr, 1, 0, &canon_rows));
        return RKR_OK;
      };
      if (!lp && tuning().rc_prefix > 0 && lstat_host_fb >= (unsigned long long)prefix_min_rows(1))
        RKR_TRY(prefix_prune(idx, qc, qa, qb, cnt, qoff_rel, cursor, cq, qself, ccount, clb, cu_fb,
                             &recount_users, &lstat_host_fb, &prefix_rows, &prefix_pruned,
                             &canon_rows, st));
      if (lstat_host_fb > 0) RKR_TRY(recount_open_candidates(lstat_host_fb));
      if (lp && lp->certify && cut_total > 0) {
        // exact fallback: cut candidates that could still be among the k best
        DevBuf brv;
        unsigned long long *nrev, hrev = 0;
        RKR_TRY(tmp_alloc(brv, &nrev, 1, st));
        RKR_CUDA(cudaMemsetAsync(nrev, 0, sizeof(unsigned long long), st));
        k_learned_revive<<<qb - qa, 256, 0, st>>>(qa, qoff_rel, cursor, qc.kq_d, ccount, clb,
                                                  cu_fb, cu, cutu, nrev);
        note_launch();
        RKR_CUDA(cudaGetLastError());
        RKR_CUDA(cudaMemcpyAsync(&hrev, nrev, sizeof(hrev), cudaMemcpyDeviceToHost, st));
        RKR_CUDA(cudaStreamSynchronize(st));
        revived += (int64_t)hrev;
        fallback += (int64_t)hrev;
        if (hrev > 0) RKR_TRY(recount_open_candidates(hrev));
      }
    }
    ms_res += t3.stop();
    Timer t4(st);
    size_t sm = sizeof(SortEnt) * kMaxK;
    RKR_CUDA(cudaFuncSetAttribute(k_select_exact, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)sm));
    {
      const int prof_slot = prof_begin("k_select_exact", st);
      k_select_exact<<<qb - qa, kSelThreads, sm, st>>>(qa, qoff_rel, cursor, cu, ccount, qc.kq_d,
                                                       qc.out_off_d, users_d, ranks_d, sel_err);
      prof_end(prof_slot, st, 0.0);
    }
    note_launch();
    RKR_CUDA(cudaGetLastError());
    ms_sel += t4.stop();
  }
  unsigned long long tiesv[2] = {0, 0};
  RKR_CUDA(cudaMemcpyAsync(tiesv, ties_d, sizeof(tiesv), cudaMemcpyDeviceToHost, st));
  RKR_CUDA(cudaStreamSynchronize(st));
  {
    int h = 0;
    RKR_CUDA(cudaMemcpy(&h, sel_err, sizeof(int), cudaMemcpyDeviceToHost));
    if (h) return fail(RKR_EINTERNAL, "fewer than k candidates for a query");
  }
  if (stats) {
    stats->pairs = idx->n * (int64_t)nq;
    stats->candidates = total;
    // canonical u.q of list-ranked candidates that needed it, of every recounted
    // row, the near-tie items of the recount and the list entries next to u.q
    stats->fp64_dots = canon_theta + canon_rows + (int64_t)tiesv[1] + list_fp64;
    stats->near_ties = (int64_t)tiesv[0];
    stats->recounted = fallback;
    stats->recount_users = recount_users;
    stats->recount_open = recount_open;
    stats->recount_split = recount_split;
    stats->max_rel_screen_err = err_rel;
    stats->max_screen_err_ratio = err_ratio;
    if (lp) stats->candidates = total - cut_total + revived;  // left by the learned cut
    stats->learned_revived = revived;
    stats->prefix_rows = prefix_rows;
    stats->prefix_pruned = prefix_pruned;
    stats->wide_queries = wide;
    stats->deep_queries = (int32_t)plan.deep.size();
    stats->ms_theta = ms_theta;
    stats->ms_resolve = ms_res;
    stats->ms_select = ms_sel;
  }
  return RKR_OK;
}

__global__ void k_count_to_rank(int64_t n, const uint32_t *__restrict__ c,
                                int32_t *__restrict__ r) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) r[i] = (int32_t)(c[i] + 1u);
}

rkr_status run_rank_pairs(const rkr_index *idx, const QueryCommon &qc, int nq, int64_t npairs,
                          const int32_t *cu, const int32_t *cq, int32_t *out_rank,
                          cudaStream_t st) {
  if (npairs <= 0) return RKR_OK;
  DevBuf bq, bc, bl, bf, bs, bt;
  int32_t *qself, *cu_fb;
  uint32_t *ccount, *clb;
  unsigned long long *lstat, *ties;
  RKR_TRY(tmp_alloc(bq, &qself, nq, st));
  RKR_TRY(tmp_alloc(bc, &ccount, npairs, st));
  RKR_TRY(tmp_alloc(bl, &clb, npairs, st));
  RKR_TRY(tmp_alloc(bf, &cu_fb, npairs, st));
  RKR_TRY(tmp_alloc(bs, &lstat, 5, st));
  RKR_TRY(tmp_alloc(bt, &ties, 2, st));
  RKR_CUDA(cudaMemsetAsync(lstat, 0, 5 * sizeof(unsigned long long), st));
  RKR_CUDA(cudaMemsetAsync(ties, 0, 2 * sizeof(unsigned long long), st));
  RKR_TRY(query_self(idx, qc.Qd, nq, qself, st));
  k_list_rank<<<(unsigned)((npairs + 127) / 128), 128, 0, st>>>(
      npairs, cu, cq, nullptr, nullptr, idx->U, idx->unrm, qc.Qd, idx->Ps, idx->pnrm_s, idx->d,
      idx->xlist,
      idx->xloff, idx->xlcap, idx->xcoff, idx->xlcnt, idx->xbmax, idx->Ut.rb3, idx->ptile3,
      idx->ptile_bn, tc_gacc(idx->Ut.kp, 1), tc_gcan(idx->d), idx->xg0, idx->xdx, idx->xg,
      idx->ldx, kListG, idx->XLO, idx->XHI, (uint32_t)idx->m, ccount, clb, cu_fb, qself,
      deep_grid(idx), lstat);
  note_launch();
  RKR_CUDA(cudaGetLastError());
  unsigned long long ls[2] = {0, 0};
  RKR_CUDA(cudaMemcpyAsync(ls, lstat, sizeof(ls), cudaMemcpyDeviceToHost, st));
  RKR_CUDA(cudaStreamSynchronize(st));
  if (ls[0] > 0)  // pairs below their user's tail list: exact recount
    RKR_TRY(recount_candidates(idx, qc.Qd, npairs, cu_fb, cq, qself, ccount, nullptr, ties, st));
  k_count_to_rank<<<(unsigned)((npairs + 255) / 256), 256, 0, st>>>(npairs, ccount, out_rank);
  note_launch();
  RKR_CUDA(cudaGetLastError());
  return RKR_OK;
}

}  // namespace rkr
