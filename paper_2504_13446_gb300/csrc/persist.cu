// persist.cu -- saving and loading an index (and a learned pruner) as a file.
//
// The paper builds its rank table once and serves any q, k and c from it
// (Section 4.1); this file lets a built index outlive the process.
//
// Index file layout (little-endian, the host's own byte order is checked):
//   magic "RKRIDX01", u32 format version, u32 byte-order mark 0x01020304,
//   header: int64 fields (sizes, build parameters, layout constants of this
//           library), float pmax, double build_ms[8],
//   u32 number of arrays, then per array: u32 id, u32 0, u64 bytes, the bytes,
//   u64 checksum of everything before it.
// The checksum is FNV-1a over 64-bit words (the last partial word zero-padded).
// A file written by a library with other layout constants (grid columns,
// list-grid columns, level count) is refused, as is any size mismatch.
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "index.cuh"

namespace rkr {
namespace {

constexpr char kMagic[8] = {'R', 'K', 'R', 'I', 'D', 'X', '0', '1'};
constexpr char kPrunerMagic[8] = {'R', 'K', 'R', 'M', 'L', 'P', '0', '1'};
constexpr uint32_t kVersion = 2;   // 2: deep count grid and its layout constant
constexpr uint32_t kBom = 0x01020304u;
constexpr size_t kChunk = (size_t)64 << 20;

struct Hash {
  uint64_t h = 0xcbf29ce484222325ull;
  uint64_t carry = 0;
  int nc = 0;  // bytes held in carry
  void add(const void *p, size_t bytes) {
    const unsigned char *b = (const unsigned char *)p;
    size_t i = 0;
    while (nc > 0 && nc < 8 && i < bytes) {
      carry |= (uint64_t)b[i++] << (8 * nc);
      if (++nc == 8) { word(carry); carry = 0; nc = 0; }
    }
    for (; i + 8 <= bytes; i += 8) {
      uint64_t w;
      memcpy(&w, b + i, 8);
      word(w);
    }
    for (; i < bytes; ++i) {
      carry |= (uint64_t)b[i] << (8 * nc);
      if (++nc == 8) { word(carry); carry = 0; nc = 0; }
    }
  }
  void word(uint64_t w) {
    h ^= w;
    h *= 0x100000001b3ull;
  }
  uint64_t done() {
    if (nc) { word(carry); carry = 0; nc = 0; }
    return h;
  }
};

struct Header {
  int64_t n, m, d, tau, omega, s, fbounds, has_exact, floor_rank, nsamp, nlev_a, nlev_x, xg,
      lists, phn, ptile_bn, kp, list_entries, seed, sampled_pos, c_listg, c_xgrid, c_levels,
      c_maxd, dg, c_dgrid;
  float pmax;
  float pad;
  double build_ms[8];
};

struct Arr {
  uint32_t id;
  void **ptr;
  uint64_t bytes;
};

// Every device array of an index with its size; list_entries = xloff[n].
std::vector<Arr> arrays(rkr_index *x, int64_t list_entries) {
  const uint64_t n = (uint64_t)x->n, m = (uint64_t)x->m, d = (uint64_t)x->d;
  const uint64_t ns = (uint64_t)x->nsamp, kp = (uint64_t)x->Ut.kp, rb = sizeof(tc::RowBound);
  std::vector<Arr> a = {
      {1, (void **)&x->U, n * d * 4},          {2, (void **)&x->Ps, m * d * 4},
      {3, (void **)&x->perm, m * 4},           {4, (void **)&x->pnorm, m * 8},
      {5, (void **)&x->unrm, n * 4},           {6, (void **)&x->pnrm_s, m * 4},
      {7, (void **)&x->fmin, n * 8},           {8, (void **)&x->fmax, n * 8},
      {9, (void **)&x->delta, n * 8},          {10, (void **)&x->binfp, n * sizeof(BinFP)},
      {11, (void **)&x->N, n * (uint64_t)x->tau * 4},
      {12, (void **)&x->JU, n * kMaxLevels * 2}, {13, (void **)&x->JL, n * kMaxLevels * 2},
      {14, (void **)&x->S, ns * d * 4},        {15, (void **)&x->snrm, ns * 4},
      {16, (void **)&x->sw, ns * 4},           {17, (void **)&x->samp_items, ns * 4},
      {18, (void **)&x->phk, (uint64_t)x->phn * 8}, {19, (void **)&x->phv, (uint64_t)x->phn * 4},
      {20, (void **)&x->Ut.hi, n * kp * 2},    {21, (void **)&x->Ut.lo, n * kp * 2},
      {22, (void **)&x->Ut.rb1, n * rb},       {23, (void **)&x->Ut.rb3, n * rb},
      {24, (void **)&x->Pt.hi, m * kp * 2},    {25, (void **)&x->Pt.lo, m * kp * 2},
      {26, (void **)&x->Pt.rb1, m * rb},       {27, (void **)&x->Pt.rb3, m * rb},
  };
  if (x->has_exact) {
    const uint64_t xg = (uint64_t)x->xg;
    std::vector<Arr> e = {
        {30, (void **)&x->xfloor, n * 4},      {31, (void **)&x->xg0, n * 8},
        {32, (void **)&x->xdx, n * 8},         {33, (void **)&x->xbin, n * sizeof(BinFP)},
        {34, (void **)&x->XLO, n * xg * 4},    {35, (void **)&x->XHI, n * xg * 4},
        {36, (void **)&x->xlcnt, n * 4},       {37, (void **)&x->xcoff, n * (kListG + 2) * 2},
        {38, (void **)&x->ldx, n * 8},         {39, (void **)&x->lbin, n * sizeof(BinFP)},
        {40, (void **)&x->xbmax, n * 4},
        {41, (void **)&x->ptile3, ((m + 255) / 256) * rb},
        {42, (void **)&x->xlcap, n * 4},       {43, (void **)&x->xloff, (n + 1) * 8},
        {44, (void **)&x->xlist, (uint64_t)std::max<int64_t>(list_entries, 1) * 8},
        {45, (void **)&x->XJU, n * kMaxLevels * 2}, {46, (void **)&x->XJL, n * kMaxLevels * 2},
    };
    a.insert(a.end(), e.begin(), e.end());
  }
  if (x->dg > 0) {
    const uint64_t dg = (uint64_t)x->dg;
    std::vector<Arr> e = {
        {47, (void **)&x->yg0, n * 8},         {48, (void **)&x->ydx, n * 8},
        {49, (void **)&x->ybin, n * sizeof(BinFP)},
        {50, (void **)&x->DLO, n * dg * 4},    {51, (void **)&x->DHI, n * dg * 4},
    };
    a.insert(a.end(), e.begin(), e.end());
  }
  return a;
}

struct File {
  FILE *f = nullptr;
  ~File() {
    if (f) fclose(f);
  }
};

struct Pinned {
  void *p = nullptr;
  ~Pinned() {
    if (p) cudaFreeHost(p);
  }
};

rkr_status put(FILE *f, Hash &h, const void *p, size_t bytes) {
  if (fwrite(p, 1, bytes, f) != bytes) return fail(RKR_EINVAL, "write failed");
  h.add(p, bytes);
  return RKR_OK;
}

rkr_status get(FILE *f, Hash &h, void *p, size_t bytes) {
  if (fread(p, 1, bytes, f) != bytes) return fail(RKR_EINVAL, "file is truncated");
  h.add(p, bytes);
  return RKR_OK;
}

}  // namespace
}  // namespace rkr

using namespace rkr;

extern "C" rkr_status rkr_index_device_bytes(const rkr_index *idx_c, int64_t *out) {
  set_error("%s", "");
  if (!idx_c || !out) return fail(RKR_EINVAL, "null argument");
  rkr_index *idx = const_cast<rkr_index *>(idx_c);  // arrays are only listed
  int64_t list_entries = 0;
  if (idx->has_exact)
    RKR_CUDA(cudaMemcpy(&list_entries, idx->xloff + idx->n, sizeof(int64_t),
                        cudaMemcpyDeviceToHost));
  int64_t tot = 0;
  for (const Arr &a : arrays(idx, list_entries)) tot += (int64_t)a.bytes;
  // the concatenated split operands (derived, not saved)
  for (const TcSide *t : {&idx->Ut, &idx->Pt})
    if (t->cat) tot += (int64_t)t->rows * 3 * t->kp * 2;
  *out = tot;
  return RKR_OK;
}

extern "C" rkr_status rkr_index_save(const rkr_index *idx_c, const char *path) {
  set_error("%s", "");
  if (!idx_c || !path) return fail(RKR_EINVAL, "null argument");
  rkr_index *idx = const_cast<rkr_index *>(idx_c);  // arrays are only read
  int64_t list_entries = 0;
  if (idx->has_exact)
    RKR_CUDA(cudaMemcpy(&list_entries, idx->xloff + idx->n, sizeof(int64_t),
                        cudaMemcpyDeviceToHost));
  Header hd;
  memset(&hd, 0, sizeof(hd));
  hd.n = idx->n; hd.m = idx->m; hd.d = idx->d; hd.tau = idx->tau; hd.omega = idx->omega;
  hd.s = idx->s; hd.fbounds = idx->fbounds; hd.has_exact = idx->has_exact;
  hd.floor_rank = idx->floor_rank; hd.nsamp = idx->nsamp; hd.nlev_a = idx->nlev_a;
  hd.nlev_x = idx->nlev_x; hd.xg = idx->xg; hd.lists = idx->lists; hd.phn = idx->phn;
  hd.ptile_bn = idx->ptile_bn; hd.kp = idx->Ut.kp; hd.list_entries = list_entries;
  hd.seed = (int64_t)idx->seed; hd.sampled_pos = idx->sampled_pos;
  hd.c_listg = kListG; hd.c_xgrid = kXGrid; hd.c_levels = kMaxLevels; hd.c_maxd = kMaxD;
  hd.dg = idx->dg; hd.c_dgrid = kDGrid;
  hd.pmax = idx->pmax;
  for (int i = 0; i < 8; ++i) hd.build_ms[i] = idx->build_ms[i];
  File fh;
  fh.f = fopen(path, "wb");
  if (!fh.f) return fail(RKR_EINVAL, "cannot open %s for writing", path);
  Hash h;
  RKR_TRY(put(fh.f, h, kMagic, 8));
  RKR_TRY(put(fh.f, h, &kVersion, 4));
  RKR_TRY(put(fh.f, h, &kBom, 4));
  RKR_TRY(put(fh.f, h, &hd, sizeof(hd)));
  std::vector<Arr> arr = arrays(idx, list_entries);
  const uint32_t na = (uint32_t)arr.size();
  RKR_TRY(put(fh.f, h, &na, 4));
  Pinned buf;
  RKR_CUDA(cudaMallocHost(&buf.p, kChunk));
  for (const Arr &a : arr) {
    if (!*a.ptr) return fail(RKR_EINTERNAL, "index array %u is missing", a.id);
    const uint32_t zero = 0;
    RKR_TRY(put(fh.f, h, &a.id, 4));
    RKR_TRY(put(fh.f, h, &zero, 4));
    RKR_TRY(put(fh.f, h, &a.bytes, 8));
    for (uint64_t off = 0; off < a.bytes; off += kChunk) {
      const size_t b = (size_t)std::min<uint64_t>(kChunk, a.bytes - off);
      RKR_CUDA(cudaMemcpy(buf.p, (const char *)*a.ptr + off, b, cudaMemcpyDeviceToHost));
      RKR_TRY(put(fh.f, h, buf.p, b));
    }
  }
  const uint64_t sum = h.done();
  if (fwrite(&sum, 1, 8, fh.f) != 8) return fail(RKR_EINVAL, "write failed");
  if (fclose(fh.f) != 0) {
    fh.f = nullptr;
    return fail(RKR_EINVAL, "write failed");
  }
  fh.f = nullptr;
  return RKR_OK;
}

extern "C" rkr_status rkr_index_load(const char *path, rkr_index **out) {
  set_error("%s", "");
  if (!path || !out) return fail(RKR_EINVAL, "null argument");
  *out = nullptr;
  RKR_TRY(check_device());
  File fh;
  fh.f = fopen(path, "rb");
  if (!fh.f) return fail(RKR_EINVAL, "cannot open %s", path);
  Hash h;
  char magic[8];
  uint32_t ver = 0, bom = 0;
  RKR_TRY(get(fh.f, h, magic, 8));
  if (memcmp(magic, kMagic, 8) != 0) return fail(RKR_EINVAL, "%s is not an index file", path);
  RKR_TRY(get(fh.f, h, &ver, 4));
  RKR_TRY(get(fh.f, h, &bom, 4));
  if (ver != kVersion) return fail(RKR_EINVAL, "index file format %u, expected %u", ver, kVersion);
  if (bom != kBom) return fail(RKR_EINVAL, "index file has another byte order");
  Header hd;
  RKR_TRY(get(fh.f, h, &hd, sizeof(hd)));
  if (hd.c_listg != kListG || hd.c_xgrid != kXGrid || hd.c_levels != kMaxLevels ||
      hd.c_maxd != kMaxD || hd.c_dgrid != kDGrid)
    return fail(RKR_EINVAL, "index file was written with other layout constants");
  if (hd.n < 1 || hd.m < 1 || hd.d < 1 || hd.d > kMaxD || hd.tau < 2 || hd.omega < 1 ||
      hd.s < 1 || hd.nsamp < 1 || hd.kp != (hd.d + 15) / 16 * 16 || hd.phn < hd.m ||
      hd.list_entries < 0 || (hd.has_exact && hd.xg != kXGrid) ||
      (hd.dg != 0 && (hd.dg != kDGrid || hd.has_exact != 2)))
    return fail(RKR_EINVAL, "index file header is inconsistent");
  rkr_index *idx = new (std::nothrow) rkr_index();
  if (!idx) return fail(RKR_ENOMEM, "host allocation failed");
  struct Guard {
    rkr_index *x;
    ~Guard() {
      if (x) {
        index_release(x);
        delete x;
      }
    }
  } guard{idx};
  idx->n = hd.n; idx->m = hd.m; idx->d = (int)hd.d; idx->tau = (int)hd.tau;
  idx->omega = (int)hd.omega; idx->s = (int)hd.s; idx->fbounds = (int)hd.fbounds;
  idx->has_exact = (int)hd.has_exact; idx->floor_rank = (int)hd.floor_rank;
  idx->dg = (int)hd.dg;
  idx->nsamp = (int)hd.nsamp; idx->nlev_a = (int)hd.nlev_a; idx->nlev_x = (int)hd.nlev_x;
  idx->xg = (int)hd.xg; idx->lists = (int)hd.lists; idx->phn = hd.phn;
  idx->ptile_bn = (int)hd.ptile_bn; idx->seed = (uint64_t)hd.seed;
  idx->sampled_pos = (int)hd.sampled_pos; idx->pmax = hd.pmax;
  for (int i = 0; i < 8; ++i) idx->build_ms[i] = hd.build_ms[i];
  for (TcSide *t : {&idx->Ut, &idx->Pt}) {
    t->d = (int)hd.d;
    t->kp = (int)hd.kp;
    t->owned = true;
  }
  idx->Ut.rows = hd.n;
  idx->Pt.rows = hd.m;
  std::vector<Arr> arr = arrays(idx, hd.list_entries);
  uint32_t na = 0;
  RKR_TRY(get(fh.f, h, &na, 4));
  if (na != arr.size()) return fail(RKR_EINVAL, "index file holds %u arrays, expected %zu", na,
                                    arr.size());
  Pinned buf;
  RKR_CUDA(cudaMallocHost(&buf.p, kChunk));
  for (const Arr &a : arr) {
    uint32_t id = 0, zero = 0;
    uint64_t bytes = 0;
    RKR_TRY(get(fh.f, h, &id, 4));
    RKR_TRY(get(fh.f, h, &zero, 4));
    RKR_TRY(get(fh.f, h, &bytes, 8));
    if (id != a.id || bytes != a.bytes)
      return fail(RKR_EINVAL, "index file array %u (%llu bytes) where %u (%llu bytes) belongs",
                  id, (unsigned long long)bytes, a.id, (unsigned long long)a.bytes);
    if (pool_malloc_async(a.ptr, a.bytes, (cudaStream_t)0) != cudaSuccess) {
      cudaGetLastError();
      *a.ptr = nullptr;
      return fail(RKR_ENOMEM, "device allocation of %llu bytes failed",
                  (unsigned long long)a.bytes);
    }
    RKR_CUDA(cudaStreamSynchronize((cudaStream_t)0));
    for (uint64_t off = 0; off < a.bytes; off += kChunk) {
      const size_t b = (size_t)std::min<uint64_t>(kChunk, a.bytes - off);
      RKR_TRY(get(fh.f, h, buf.p, b));
      RKR_CUDA(cudaMemcpy((char *)*a.ptr + off, buf.p, b, cudaMemcpyHostToDevice));
    }
  }
  const uint64_t want = h.done();
  uint64_t sum = 0;
  if (fread(&sum, 1, 8, fh.f) != 8) return fail(RKR_EINVAL, "file is truncated");
  if (sum != want) return fail(RKR_EINVAL, "index file checksum mismatch");
  char extra;
  if (fread(&extra, 1, 1, fh.f) != 0) return fail(RKR_EINVAL, "index file has trailing bytes");
  // the concatenated split operands are derived from hi and lo, not stored
  RKR_TRY(tc_make_cat(idx->Ut, 1, (cudaStream_t)0));
  RKR_TRY(tc_make_cat(idx->Pt, 2, (cudaStream_t)0));
  RKR_CUDA(cudaStreamSynchronize((cudaStream_t)0));
  *out = idx;
  guard.x = nullptr;
  return RKR_OK;
}

// ------------------------------------------------------------ pruner

extern "C" rkr_status rkr_pruner_save(rkr_pruner *pr, const char *path) {
  set_error("%s", "");
  if (!pr || !path) return fail(RKR_EINVAL, "null argument");
  const int64_t np = rkr_pruner_nparams(pr);
  std::vector<float> p((size_t)np);
  RKR_TRY(rkr_pruner_params(pr, 0, p.data(), np));
  const int32_t FH[2] = {pruner_features(pr), pruner_hidden(pr)};
  File fh;
  fh.f = fopen(path, "wb");
  if (!fh.f) return fail(RKR_EINVAL, "cannot open %s for writing", path);
  Hash h;
  RKR_TRY(put(fh.f, h, kPrunerMagic, 8));
  RKR_TRY(put(fh.f, h, &kVersion, 4));
  RKR_TRY(put(fh.f, h, &kBom, 4));
  RKR_TRY(put(fh.f, h, FH, sizeof(FH)));
  RKR_TRY(put(fh.f, h, &np, 8));
  RKR_TRY(put(fh.f, h, p.data(), sizeof(float) * p.size()));
  const uint64_t sum = h.done();
  if (fwrite(&sum, 1, 8, fh.f) != 8) return fail(RKR_EINVAL, "write failed");
  if (fclose(fh.f) != 0) {
    fh.f = nullptr;
    return fail(RKR_EINVAL, "write failed");
  }
  fh.f = nullptr;
  return RKR_OK;
}

extern "C" rkr_status rkr_pruner_load(const char *path, rkr_pruner **out) {
  set_error("%s", "");
  if (!path || !out) return fail(RKR_EINVAL, "null argument");
  *out = nullptr;
  File fh;
  fh.f = fopen(path, "rb");
  if (!fh.f) return fail(RKR_EINVAL, "cannot open %s", path);
  Hash h;
  char magic[8];
  uint32_t ver = 0, bom = 0;
  int32_t FH[2];
  int64_t np = 0;
  RKR_TRY(get(fh.f, h, magic, 8));
  if (memcmp(magic, kPrunerMagic, 8) != 0) return fail(RKR_EINVAL, "%s is not a pruner file",
                                                       path);
  RKR_TRY(get(fh.f, h, &ver, 4));
  RKR_TRY(get(fh.f, h, &bom, 4));
  if (ver != kVersion || bom != kBom) return fail(RKR_EINVAL, "pruner file format mismatch");
  RKR_TRY(get(fh.f, h, FH, sizeof(FH)));
  RKR_TRY(get(fh.f, h, &np, 8));
  if (FH[0] < 1 || FH[0] > 1024 || FH[1] < 1 || FH[1] > 1024 || np < 1 || np > (1 << 26))
    return fail(RKR_EINVAL, "pruner file header is inconsistent");
  std::vector<float> p((size_t)np);
  RKR_TRY(get(fh.f, h, p.data(), sizeof(float) * p.size()));
  const uint64_t want = h.done();
  uint64_t sum = 0;
  if (fread(&sum, 1, 8, fh.f) != 8) return fail(RKR_EINVAL, "file is truncated");
  if (sum != want) return fail(RKR_EINVAL, "pruner file checksum mismatch");
  rkr_pruner *pr = nullptr;
  RKR_TRY(rkr_pruner_create(FH[0], FH[1], 0, &pr));
  if (rkr_pruner_nparams(pr) != np) {
    rkr_pruner_free(pr);
    return fail(RKR_EINVAL, "pruner file parameter count does not match F, H");
  }
  const rkr_status st = rkr_pruner_params(pr, 1, p.data(), np);
  if (st != RKR_OK) {
    rkr_pruner_free(pr);
    return st;
  }
  *out = pr;
  return RKR_OK;
}
