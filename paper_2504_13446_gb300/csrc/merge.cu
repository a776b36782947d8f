// merge.cu -- host-side merge of per-shard answers (user rows split across
// processes or GPUs).  Host code only: no CUDA call, so it also runs on hosts
// without a GPU.
//
// Exact (Def. 2): a user's rank depends on its own row and P only, so the k
// smallest (rank, user) of the union of each shard's k smallest are the
// answer of the whole user set.
//
// c-approximate (Section 4.3): each shard sends, per query, every one of its
// users whose lower-bound numerator is at most an upper estimate of that
// shard's R_up_k (rkr_query_approx_candidates).  The shard's R_up_k is at least
// the global one, so every user with r_low <= R_up_k (global) is sent; those
// include the k smallest lower and upper bounds and every user steps 2 and 3
// can return.  Steps 1-3 run again here on the union, as in rkr_query_approx.
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "common.cuh"

namespace rkr {
namespace {

rkr_status check_csr(int32_t nq, const int32_t *k, const int64_t *offs) {
  if (nq < 1) return fail(RKR_EINVAL, "nq must be >= 1");
  if (offs[0] != 0) return fail(RKR_EINVAL, "in_offs[0] must be 0");
  for (int q = 0; q < nq; ++q) {
    if (offs[q + 1] < offs[q]) return fail(RKR_EINVAL, "in_offs must be non-decreasing");
    if (k[q] < 1 || k[q] > kMaxK)
      return fail(RKR_EINVAL, "k[%d] = %d must be in [1, %d]", q, k[q], kMaxK);
    if (offs[q + 1] - offs[q] < k[q])
      return fail(RKR_EINVAL, "query %d has %lld entries, fewer than k = %d", q,
                  (long long)(offs[q + 1] - offs[q]), k[q]);
  }
  return RKR_OK;
}

}  // namespace
}  // namespace rkr

using namespace rkr;

extern "C" rkr_status rkr_merge_exact(int32_t nq, const int32_t *k, const int64_t *in_offs,
                                      const int32_t *in_users, const int32_t *in_ranks,
                                      int32_t *out_users, int32_t *out_ranks) {
  set_error("%s", "");
  if (!k || !in_offs || !in_users || !in_ranks || !out_users || !out_ranks)
    return fail(RKR_EINVAL, "null argument");
  RKR_TRY(check_csr(nq, k, in_offs));
  int64_t o = 0;
  std::vector<uint64_t> key;
  std::vector<int32_t> ids;
  for (int q = 0; q < nq; ++q) {
    key.clear();
    ids.clear();
    for (int64_t i = in_offs[q]; i < in_offs[q + 1]; ++i) {
      if (in_users[i] < 0 || in_ranks[i] < 1) return fail(RKR_EINVAL, "bad entry %lld", (long long)i);
      key.push_back(((uint64_t)(uint32_t)in_ranks[i] << 32) | (uint32_t)in_users[i]);
      ids.push_back(in_users[i]);
    }
    std::sort(ids.begin(), ids.end());
    if (std::adjacent_find(ids.begin(), ids.end()) != ids.end())
      return fail(RKR_EINVAL, "query %d lists a user twice", q);
    std::sort(key.begin(), key.end());
    for (int r = 0; r < k[q]; ++r, ++o) {
      out_users[o] = (int32_t)(key[r] & 0xffffffffu);
      out_ranks[o] = (int32_t)(key[r] >> 32);
    }
  }
  return RKR_OK;
}

extern "C" rkr_status rkr_merge_approx(int32_t nq, const int32_t *k, double c, int32_t s,
                                       const int64_t *in_offs, const int32_t *in_users,
                                       const uint32_t *in_nlow, const uint32_t *in_nup,
                                       const double *in_est, int32_t *out_users,
                                       uint32_t *out_nlow, uint32_t *out_nup, double *out_est,
                                       int32_t *out_case, int32_t *out_nc) {
  set_error("%s", "");
  if (!k || !in_offs || !in_users || !in_nlow || !in_nup || !in_est || !out_users)
    return fail(RKR_EINVAL, "null argument");
  if (!(c >= 1.0) || !isfinite(c)) return fail(RKR_EINVAL, "c must be a finite value >= 1");
  if (s < 1) return fail(RKR_EINVAL, "s must be >= 1");
  RKR_TRY(check_csr(nq, k, in_offs));
  struct E {
    uint32_t lo, up;
    int32_t u;
    double est;
  };
  std::vector<E> all, uc, tmp;
  std::vector<uint32_t> v;
  int64_t o = 0;
  for (int q = 0; q < nq; ++q) {
    all.clear();
    for (int64_t i = in_offs[q]; i < in_offs[q + 1]; ++i)
      all.push_back({in_nlow[i], in_nup[i], in_users[i], in_est[i]});
    const int kq = k[q];
    // Step 1: k-th smallest lower and upper bound numerators
    v.resize(all.size());
    for (size_t i = 0; i < all.size(); ++i) v[i] = all[i].lo;
    std::nth_element(v.begin(), v.begin() + (kq - 1), v.end());
    const uint64_t Rlo = v[kq - 1];
    for (size_t i = 0; i < all.size(); ++i) v[i] = all[i].up;
    std::nth_element(v.begin(), v.begin() + (kq - 1), v.end());
    const uint64_t Rup = v[kq - 1];
    const double lhs = c * (double)((uint64_t)s + Rlo);
    const bool caseA = lhs >= (double)((uint64_t)s + Rup);
    auto by_bounds = [](const E &a, const E &b) {
      if (a.up != b.up) return a.up < b.up;
      if (a.lo != b.lo) return a.lo < b.lo;
      return a.u < b.u;
    };
    auto emit = [&](const E &e) {
      out_users[o] = e.u;
      if (out_nlow) out_nlow[o] = e.lo;
      if (out_nup) out_nup[o] = e.up;
      if (out_est) out_est[o] = e.est;
      ++o;
    };
    int nc;
    if (caseA) {
      // Step 2, Case A: the k users with the smallest (r_up, r_low, index)
      std::partial_sort(all.begin(), all.begin() + kq, all.end(), by_bounds);
      for (int r = 0; r < kq; ++r) emit(all[r]);
      nc = kq;
    } else {
      // Case B: U_c = {r_up <= c R_low_k}; r_low > R_up_k is pruned; step 3 takes
      // the k - |U_c| smallest (r_hat, index) of the rest
      uc.clear();
      tmp.clear();
      for (const E &e : all) {
        if ((double)((uint64_t)s + e.up) <= lhs) uc.push_back(e);
        else if ((uint64_t)e.lo <= Rup) tmp.push_back(e);
      }
      std::sort(uc.begin(), uc.end(), by_bounds);
      nc = (int)std::min<size_t>(uc.size(), (size_t)kq);
      for (int r = 0; r < nc; ++r) emit(uc[r]);
      const int need = kq - nc;
      if ((int)tmp.size() < need) return fail(RKR_EINTERNAL, "query %d: too few candidates", q);
      std::partial_sort(tmp.begin(), tmp.begin() + need, tmp.end(), [](const E &a, const E &b) {
        if (a.est != b.est) return a.est < b.est;
        return a.u < b.u;
      });
      for (int r = 0; r < need; ++r) emit(tmp[r]);
    }
    if (out_case) out_case[q] = caseA ? 1 : 2;
    if (out_nc) out_nc[q] = nc;
  }
  return RKR_OK;
}
