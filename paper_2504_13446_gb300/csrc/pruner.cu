// pruner.cu -- the learned pruner: a monotone rank regressor trained and run on
// the GPU.  Every matrix product (the two forward layers and the three backward
// products) runs on the tcgen05 tensor cores through the screen kernel with a
// dense epilogue (BF16 operands, FP32 accumulation in TMEM); the rest (output
// layer, masks, column sums, Adam) are small elementwise kernels.  FP32 master
// weights.
//
// Model (F non-monotone features x, the normalised score t = u.q / ||u||):
//   h1 = relu(W1 x - softplus(A) t + b1),  h2 = relu(softplus(V2) h1 + b2),
//   y  = softplus(v3) . h2 + b3  ~  log r(q, u, P).
// The weights on every path from t are <= 0 before non-decreasing activations
// and >= 0 after them, so y is non-increasing in t, as the rank of Def. 1 is.
// Loss: 0.5 * mean((y - target)^2); Adam on the raw parameters.
// Flattened parameter order: W1 (H x F), A (H), b1 (H), V2 (H x H), b2 (H), v3 (H), b3.
//
// Operand layouts (the tensor-core product D = A B^T takes both operands with K
// contiguous, K padded to a multiple of 16 with zeros): X (B x Fp), W1 (H x Fp),
// h1 (B x Hp), softplus(V2) (H x Hp) and its transpose; for the weight
// gradients the batch is K, so dz2, h1, dz1 and X are also kept transposed
// (H or Fp rows of `cap` entries, zero past the batch).
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "index.cuh"
#include "tcops.cuh"

struct rkr_pruner {
  int F = 0, H = 0, Fp = 0, Hp = 0;   // Fp, Hp: F, H rounded up to 16
  int64_t nparam = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // master, grad, Adam moments
  int64_t step = 0;
  // effective BF16 weights of the current parameters
  __nv_bfloat16 *W1b = nullptr, *W2b = nullptr, *W2t = nullptr;
  float *wt = nullptr, *w3 = nullptr;
  int *err = nullptr;                 // error word of the tensor-core products
  // batch scratch (capacity cap rows, a multiple of 16)
  int64_t cap = 0;
  __nv_bfloat16 *Xb = nullptr, *XbT = nullptr, *h1 = nullptr, *h1T = nullptr, *h2 = nullptr,
                *d2b = nullptr, *d2T = nullptr, *d1T = nullptr;
  float *z1 = nullptr, *z2 = nullptr, *y = nullptr, *dy = nullptr, *tb = nullptr, *d2 = nullptr,
        *d1 = nullptr, *tg = nullptr;
  // per-user prediction tables (rkr_pruner_invert): tab[u * tabG + g] = y(x_u, t_g),
  // tgrid[u] = (t_0, step) of user u's grid t_g = t_0 + g * step
  float *tab = nullptr;
  float2 *tgrid = nullptr;
  int tabG = 0;
  int64_t tabn = 0;
  uint64_t tab_serial = 0;          // the index they were built for
  std::vector<float> tab_R;         // and the feature projection
};

namespace rkr {
namespace {

struct Off {  // offsets of the parameter blocks in the flat vector
  int64_t W1, A, b1, V2, b2, v3, b3, n;
  Off(int F, int H) {
    W1 = 0;
    A = W1 + (int64_t)H * F;
    b1 = A + H;
    V2 = b1 + H;
    b2 = V2 + (int64_t)H * H;
    v3 = b2 + H;
    b3 = v3 + H;
    n = b3 + 1;
  }
};

__device__ __forceinline__ float softplusf(float z) {
  return z > 30.0f ? z : log1pf(expf(fminf(z, 30.0f)));
}
__device__ __forceinline__ float sigmoidf(float z) { return 1.0f / (1.0f + expf(-z)); }

// Effective weights: W1 (H x Fp) and softplus(V2) (H x Hp) in BF16 with zero
// padding, the transpose of the latter, -softplus(A) and softplus(v3) in FP32.
__global__ void k_mlp_weights(int F, int H, int Fp, int Hp, const float *__restrict__ p, Off o,
                              __nv_bfloat16 *__restrict__ W1b, __nv_bfloat16 *__restrict__ W2b,
                              __nv_bfloat16 *__restrict__ W2t, float *__restrict__ wt,
                              float *__restrict__ w3) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < (int64_t)H * Fp) {
    const int64_t r = i / Fp, c = i % Fp;
    W1b[i] = __float2bfloat16_rn(c < F ? p[o.W1 + r * F + c] : 0.0f);
  }
  if (i < (int64_t)H * Hp) {
    const int64_t r = i / Hp, c = i % Hp;
    W2b[i] = __float2bfloat16_rn(c < H ? softplusf(p[o.V2 + r * H + c]) : 0.0f);
    W2t[i] = __float2bfloat16_rn(c < H ? softplusf(p[o.V2 + c * H + r]) : 0.0f);
  }
  if (i < H) {
    wt[i] = -softplusf(p[o.A + i]);
    w3[i] = softplusf(p[o.v3 + i]);
  }
}

// Dense epilogue of a tensor-core product D (M x N): v = acc + bias[col] +
// tcol[row] * wcol[col] (each term optional); zout / fout get v (FP32), hout
// gets relu(v) or v in BF16, houtT the same transposed (houtT[col * ldt + row]).
struct EpiDense {
  static const char *name() { return "k_screen<EpiDense>"; }
  struct Thread {
    int64_t row;
  };
  static constexpr size_t kSmem = 0;
  int64_t M, N;
  int bn;
  const float *bias, *tcol, *wcol;
  int relu;
  float *zout;
  int64_t ldz;
  float *fout;
  int64_t ldf;
  __nv_bfloat16 *hout;
  int64_t ldh;
  __nv_bfloat16 *houtT;
  int64_t ldt;
  __device__ void unit_begin(char *, const tc::Unit &, int, Thread &) const {}
  __device__ void tile_begin(char *, int rb, int, int r, int, Thread &ts) const {
    ts.row = (int64_t)rb * tc::BM + r;
  }
  __device__ void chunk(char *, int, int ct, int, int col, uint32_t, const float (&v)[32],
                        Thread &ts) const {
    if (ts.row >= M) return;
    const int64_t c0 = (int64_t)ct * bn + col;
    const float tr = tcol ? tcol[ts.row] : 0.0f;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int64_t c = c0 + j;
      if (c < N) {
        float x = v[j];
        if (bias) x += bias[c];
        if (tcol) x = fmaf(tr, wcol[c], x);
        if (zout) zout[ts.row * ldz + c] = x;
        if (fout) fout[ts.row * ldf + c] = x;
        const __nv_bfloat16 h = __float2bfloat16_rn(relu ? fmaxf(x, 0.0f) : x);
        if (hout) hout[ts.row * ldh + c] = h;
        if (houtT) houtT[c * ldt + ts.row] = h;
      }
    }
  }
  __device__ void tile_end(char *, int, int, int, int, Thread &) const {}
  __device__ void unit_end(char *, const tc::Unit &, int, Thread &) const {}
};

// D = A B^T on the tensor cores: A rows of K = kp BF16 values (pitch kp), B
// likewise; the epilogue gets D's (row, column) entries.
rkr_status dense(const __nv_bfloat16 *A, int64_t M, const __nv_bfloat16 *B, int64_t N, int kp,
                 EpiDense e, int *err, cudaStream_t st) {
  constexpr int BN = 256;
  TcSide a, b;
  a.rows = M;
  a.d = kp;
  a.kp = kp;
  a.hi = a.lo = const_cast<__nv_bfloat16 *>(A);
  a.owned = false;
  b.rows = N;
  b.d = kp;
  b.kp = kp;
  b.hi = b.lo = const_cast<__nv_bfloat16 *>(B);
  b.owned = false;
  e.M = M;
  e.N = N;
  e.bn = BN;
  return launch_screen<BN, 4>(a, b, 0, row_schedule(M, N, BN), e, err, st);
}

EpiDense dense_epi() {
  EpiDense e;
  e.M = e.N = 0;
  e.bn = 256;
  e.bias = e.tcol = e.wcol = nullptr;
  e.relu = 0;
  e.zout = e.fout = nullptr;
  e.hout = e.houtT = nullptr;
  e.ldz = e.ldf = e.ldh = e.ldt = 0;
  return e;
}

// Gather a batch into X (cap x Fp) and its transpose (Fp x cap), FP32 scores and
// targets; rows [B, Bp) and columns [F, Fp) are written as zeros.
__global__ void k_mlp_batch(int64_t B, int64_t Bp, int F, int Fp, int64_t cap,
                            const int64_t *__restrict__ idx, const float *__restrict__ X,
                            const float *__restrict__ t, const float *__restrict__ target,
                            __nv_bfloat16 *__restrict__ Xb, __nv_bfloat16 *__restrict__ XbT,
                            float *__restrict__ tb, float *__restrict__ tg) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= Bp * Fp) return;
  const int64_t r = i / Fp, c = i % Fp;
  const bool live = r < B && c < F;
  const int64_t s = live ? (idx ? idx[r] : r) : 0;
  const __nv_bfloat16 x = __float2bfloat16_rn(live ? X[s * F + c] : 0.0f);
  Xb[r * Fp + c] = x;
  if (XbT) XbT[c * cap + r] = x;
  if (c == 0) {
    tb[r] = r < B ? t[idx ? idx[r] : r] : 0.0f;
    if (tg) tg[r] = r < B && target ? target[idx ? idx[r] : r] : 0.0f;
  }
}

// Gather rows of a per-user feature table: X[r] = Xu[uid[r]], tb[r] = t[r].
__global__ void k_mlp_gather(int64_t B, int F, int Fp, const int32_t *__restrict__ uid,
                             const float *__restrict__ Xu, const float *__restrict__ t,
                             __nv_bfloat16 *__restrict__ Xb, float *__restrict__ tb) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= B * Fp) return;
  const int64_t r = i / Fp, c = i % Fp;
  const int64_t u = uid[r] < 0 ? 0 : uid[r];  // invalid rows read user 0 (ignored)
  Xb[r * Fp + c] = __float2bfloat16_rn(c < F ? Xu[u * F + c] : 0.0f);
  if (c == 0) tb[r] = t[r];
}

// y[r] = w3 . h2[r] + b3 (one warp per row), and dy = (y - target) / B when asked
// (dy = 0 for the padding rows [B, cap)).
__global__ void k_mlp_out(int64_t B, int64_t cap, int H, const __nv_bfloat16 *__restrict__ h2,
                          const float *__restrict__ w3, const float *__restrict__ p, int64_t ob3,
                          float *__restrict__ y, const float *__restrict__ tg,
                          float *__restrict__ dy) {
  const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= (dy ? cap : B)) return;
  if (r >= B) {
    if (lane == 0) dy[r] = 0.0f;
    return;
  }
  float acc = 0.0f;
  for (int n = lane; n < H; n += 32) acc = fmaf(__bfloat162float(h2[r * H + n]), w3[n], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) {
    const float yy = acc + p[ob3];
    y[r] = yy;
    if (dy) dy[r] = (yy - tg[r]) / (float)B;
  }
}

// dz2 = dy[r] * w3[n] * (z2 > 0): FP32 (B x H), BF16 (cap x Hp) and transposed
// BF16 (H x cap); zero on the padding rows.
__global__ void k_mlp_dz2(int64_t B, int64_t cap, int H, int Hp, const float *__restrict__ dy,
                          const float *__restrict__ w3, const float *__restrict__ z2,
                          float *__restrict__ d2, __nv_bfloat16 *__restrict__ d2b,
                          __nv_bfloat16 *__restrict__ d2T) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= cap * H) return;
  const int64_t r = i / H, c = i % H;
  const float v = r < B && z2[i] > 0.0f ? dy[r] * w3[c] : 0.0f;
  if (r < B) d2[i] = v;
  const __nv_bfloat16 vb = __float2bfloat16_rn(v);
  d2b[r * Hp + c] = vb;
  d2T[c * cap + r] = vb;
}

// dz1 = (dz2 W2)[r, k] * (z1 > 0) in place of the product (FP32), and transposed
// BF16 (H x cap); zero on the padding rows.
__global__ void k_mlp_dz1(int64_t B, int64_t cap, int H, const float *__restrict__ z1,
                          float *__restrict__ d1, __nv_bfloat16 *__restrict__ d1T) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= cap * H) return;
  const int64_t r = i / H, c = i % H;
  const float v = r < B && z1[i] > 0.0f ? d1[i] : 0.0f;
  if (r < B) d1[i] = v;
  d1T[c * cap + r] = __float2bfloat16_rn(v);
}

// out[n] = sum_r f(D[r, n]) * rowscale[r]: f = relu when asked, rowscale = 1 when null.
__global__ void k_colsum(int64_t B, int H, const float *__restrict__ D, int relu,
                         const float *__restrict__ rowscale, float *__restrict__ out) {
  const int n = blockIdx.x;
  float acc = 0.0f;
  for (int64_t r = threadIdx.x; r < B; r += blockDim.x) {
    float v = D[r * H + n];
    if (relu) v = fmaxf(v, 0.0f);
    acc += v * (rowscale ? rowscale[r] : 1.0f);
  }
  __shared__ float red[256];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[n] = red[0];
}

// Gradients of the constrained parameters from those of the effective weights;
// db3 = sum dy.
__global__ void k_mlp_chain(int H, const float *__restrict__ p, Off o, float *__restrict__ g,
                            const float *__restrict__ dy, int64_t B) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < (int64_t)H * H) g[o.V2 + i] *= sigmoidf(p[o.V2 + i]);
  if (i < H) {
    g[o.A + i] *= -sigmoidf(p[o.A + i]);
    g[o.v3 + i] *= sigmoidf(p[o.v3 + i]);
  }
  if (i == 0) {
    float s = 0.0f;
    for (int64_t r = 0; r < B; ++r) s += dy[r];
    g[o.b3] = s;
  }
}

__global__ void k_adam(int64_t n, float *__restrict__ p, const float *__restrict__ g,
                       float *__restrict__ m, float *__restrict__ v, float lr, float b1c,
                       float b2c) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi, vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / b1c) / (sqrtf(vi / b2c) + 1e-8f);
}

int64_t round16(int64_t x) { return (x + 15) / 16 * 16; }

rkr_status ensure_cap(rkr_pruner *pr, int64_t B, cudaStream_t st) {
  B = round16(B);
  if (B <= pr->cap) return RKR_OK;
  const int H = pr->H, Fp = pr->Fp, Hp = pr->Hp;
  for (void *q : {(void *)pr->Xb, (void *)pr->XbT, (void *)pr->h1, (void *)pr->h1T,
                  (void *)pr->h2, (void *)pr->d2b, (void *)pr->d2T, (void *)pr->d1T,
                  (void *)pr->z1, (void *)pr->z2, (void *)pr->y, (void *)pr->dy, (void *)pr->tb,
                  (void *)pr->d2, (void *)pr->d1, (void *)pr->tg})
    if (q) cudaFreeAsync(q, st);
  auto al = [&](auto **q, size_t count) -> rkr_status {
    cudaError_t e = pool_malloc_async((void **)q, count * sizeof(**q), st);
    if (e != cudaSuccess) return cuda_fail(e, "pruner scratch");
    // padding entries of the operands must read as zeros
    e = cudaMemsetAsync(*q, 0, count * sizeof(**q), st);
    if (e != cudaSuccess) return cuda_fail(e, "pruner scratch");
    return RKR_OK;
  };
  RKR_TRY(al(&pr->Xb, (size_t)B * Fp));
  RKR_TRY(al(&pr->XbT, (size_t)Fp * B));
  RKR_TRY(al(&pr->h1, (size_t)B * Hp));
  RKR_TRY(al(&pr->h1T, (size_t)H * B));
  RKR_TRY(al(&pr->h2, (size_t)B * H));
  RKR_TRY(al(&pr->d2b, (size_t)B * Hp));
  RKR_TRY(al(&pr->d2T, (size_t)H * B));
  RKR_TRY(al(&pr->d1T, (size_t)H * B));
  RKR_TRY(al(&pr->z1, (size_t)B * H));
  RKR_TRY(al(&pr->z2, (size_t)B * H));
  RKR_TRY(al(&pr->d2, (size_t)B * H));
  RKR_TRY(al(&pr->d1, (size_t)B * H));
  RKR_TRY(al(&pr->y, (size_t)B));
  RKR_TRY(al(&pr->dy, (size_t)B));
  RKR_TRY(al(&pr->tb, (size_t)B));
  RKR_TRY(al(&pr->tg, (size_t)B));
  pr->cap = B;
  return RKR_OK;
}

void refresh_weights(rkr_pruner *pr, cudaStream_t st) {
  const Off o(pr->F, pr->H);
  const int64_t cnt = std::max<int64_t>((int64_t)pr->H * pr->Fp, (int64_t)pr->H * pr->Hp);
  k_mlp_weights<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(
      pr->F, pr->H, pr->Fp, pr->Hp, pr->p, o, pr->W1b, pr->W2b, pr->W2t, pr->wt, pr->w3);
  note_launch();
}

// Forward pass of the batch already gathered in Xb / tb; y in pr->y.  With
// with_grad, h1 is also kept transposed and dy formed for the backward pass.
rkr_status forward_batch(rkr_pruner *pr, int64_t B, bool with_grad, cudaStream_t st) {
  const int H = pr->H;
  const Off o(pr->F, H);
  // z1 = X W1^T + b1 + t wt^T, h1 = relu(z1)
  EpiDense e1 = dense_epi();
  e1.bias = pr->p + o.b1;
  e1.tcol = pr->tb;
  e1.wcol = pr->wt;
  e1.relu = 1;
  e1.zout = pr->z1;
  e1.ldz = H;
  e1.hout = pr->h1;
  e1.ldh = pr->Hp;
  if (with_grad) {
    e1.houtT = pr->h1T;
    e1.ldt = pr->cap;
  }
  RKR_TRY(dense(pr->Xb, B, pr->W1b, H, pr->Fp, e1, pr->err, st));
  // z2 = h1 W2^T + b2, h2 = relu(z2)
  EpiDense e2 = dense_epi();
  e2.bias = pr->p + o.b2;
  e2.relu = 1;
  e2.zout = pr->z2;
  e2.ldz = H;
  e2.hout = pr->h2;
  e2.ldh = H;
  RKR_TRY(dense(pr->h1, B, pr->W2b, H, pr->Hp, e2, pr->err, st));
  const int64_t rows = with_grad ? pr->cap : B;
  k_mlp_out<<<(unsigned)((rows * 32 + 255) / 256), 256, 0, st>>>(
      B, pr->cap, H, pr->h2, pr->w3, pr->p, o.b3, pr->y, with_grad ? pr->tg : nullptr,
      with_grad ? pr->dy : nullptr);
  note_launch();
  return RKR_OK;
}

// Backward pass of the batch of the last forward: gradients of the raw
// parameters into pr->g (same order as the flat parameter vector).  The batch
// is K of the weight-gradient products; padding rows carry zeros.
rkr_status backward_batch(rkr_pruner *pr, int64_t B, cudaStream_t st) {
  const int F = pr->F, H = pr->H;
  const Off o(F, H);
  const int64_t cap = pr->cap;
  const unsigned nb = (unsigned)((cap * H + 255) / 256);
  // dw3 = h2^T dy (the chain rule to v3 follows)
  k_colsum<<<H, 256, 0, st>>>(B, H, pr->z2, 1, pr->dy, pr->g + o.v3);
  note_launch();
  // dz2 = dy w3^T * (z2 > 0); db2 = column sums
  k_mlp_dz2<<<nb, 256, 0, st>>>(B, cap, H, pr->Hp, pr->dy, pr->w3, pr->z2, pr->d2, pr->d2b,
                                pr->d2T);
  note_launch();
  k_colsum<<<H, 256, 0, st>>>(B, H, pr->d2, 0, nullptr, pr->g + o.b2);
  note_launch();
  // dW2 = dz2^T h1 (H x H): K = the batch
  EpiDense ew2 = dense_epi();
  ew2.fout = pr->g + o.V2;
  ew2.ldf = H;
  RKR_TRY(dense(pr->d2T, H, pr->h1T, H, (int)cap, ew2, pr->err, st));
  // dh1 = dz2 W2 (B x H), then dz1 = dh1 * (z1 > 0)
  EpiDense eh1 = dense_epi();
  eh1.fout = pr->d1;
  eh1.ldf = H;
  RKR_TRY(dense(pr->d2b, B, pr->W2t, H, pr->Hp, eh1, pr->err, st));
  k_mlp_dz1<<<nb, 256, 0, st>>>(B, cap, H, pr->z1, pr->d1, pr->d1T);
  note_launch();
  // db1 = column sums; d(wt) = dz1^T t
  k_colsum<<<H, 256, 0, st>>>(B, H, pr->d1, 0, nullptr, pr->g + o.b1);
  note_launch();
  k_colsum<<<H, 256, 0, st>>>(B, H, pr->d1, 0, pr->tb, pr->g + o.A);
  note_launch();
  // dW1 = dz1^T X (H x F): K = the batch
  EpiDense ew1 = dense_epi();
  ew1.fout = pr->g + o.W1;
  ew1.ldf = F;
  RKR_TRY(dense(pr->d1T, H, pr->XbT, F, (int)cap, ew1, pr->err, st));
  // constrained parameters and db3
  const int64_t cnt = std::max<int64_t>((int64_t)H * H, 1);
  k_mlp_chain<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(H, pr->p, o, pr->g, pr->dy, B);
  note_launch();
  return RKR_OK;
}

// The products' error word: RKR_ETIMEOUT when a bounded wait gave up.
rkr_status check_err(rkr_pruner *pr, cudaStream_t st) {
  int h = 0;
  RKR_CUDA(cudaMemcpyAsync(&h, pr->err, sizeof(int), cudaMemcpyDeviceToHost, st));
  RKR_CUDA(cudaStreamSynchronize(st));
  if (h) return fail(RKR_ETIMEOUT, "pruner product wait timed out (%d)", h);
  return RKR_OK;
}

// A device view of an input array: the array itself when it is device memory,
// else a stream-ordered copy freed with the holder.
struct InDev {
  const void *p = nullptr;
  void *own = nullptr;
  cudaStream_t st = nullptr;
  rkr_status init(const void *src, size_t bytes, cudaStream_t s) {
    st = s;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, src) == cudaSuccess &&
        (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)) {
      p = src;
      return RKR_OK;
    }
    cudaGetLastError();
    cudaError_t e = pool_malloc_async(&own, bytes ? bytes : 1, s);
    if (e != cudaSuccess) return cuda_fail(e, "input staging");
    e = cudaMemcpyAsync(own, src, bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(e, "input staging copy");
    p = own;
    return RKR_OK;
  }
  ~InDev() {
    if (own) cudaFreeAsync(own, st);
  }
};

// SplitMix64-driven standard normal values (Box-Muller) for the initial weights.
uint64_t splitmix(uint64_t &x) {
  uint64_t z = (x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
double normal(uint64_t &x) {
  const double u1 = ((splitmix(x) >> 11) + 0.5) * 0x1p-53, u2 = ((splitmix(x) >> 11) + 0.5) * 0x1p-53;
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

}  // namespace

// Predictions for B pairs whose features are rows uid[r] of a per-user table Xu
// (device arrays), in chunks of the scratch capacity.
rkr_status pruner_forward_gather(rkr_pruner *pr, const float *Xu, const int32_t *uid,
                                 const float *t, int64_t B, float *y, cudaStream_t st) {
  const int64_t chunk = 1 << 16;
  RKR_TRY(ensure_cap(pr, std::min(B, chunk), st));
  refresh_weights(pr, st);
  for (int64_t a = 0; a < B; a += chunk) {
    const int64_t b = std::min(B - a, chunk);
    k_mlp_gather<<<(unsigned)((b * pr->Fp + 255) / 256), 256, 0, st>>>(b, pr->F, pr->Fp, uid + a,
                                                                       Xu, t + a, pr->Xb, pr->tb);
    note_launch();
    RKR_TRY(forward_batch(pr, b, false, st));
    RKR_CUDA(cudaMemcpyAsync(y + a, pr->y, sizeof(float) * b, cudaMemcpyDeviceToDevice, st));
  }
  return check_err(pr, st);
}

namespace {

// User u's grid: t_g = t_0 + g * step over [f_min, f_max] / ||u||, the range of
// t = u.q / ||u|| for q in P (||u|| in FP32, as the pair scores take it).
__global__ void k_tab_grid(int64_t n, int d, const float *__restrict__ U,
                           const double *__restrict__ fmin, const double *__restrict__ fmax,
                           int G, float2 *__restrict__ tg) {
  const int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (u >= n) return;
  const float *uu = U + u * d;
  float nn = 0.0f;
  for (int k = 0; k < d; ++k) nn = fmaf(uu[k], uu[k], nn);
  const float nrm = sqrtf(nn);
  float t0 = 0.0f, t1 = 0.0f;
  if (nrm > 0.0f) {
    t0 = (float)(fmin[u] / (double)nrm);
    t1 = (float)(fmax[u] / (double)nrm);
  }
  tg[u] = make_float2(t0, t1 > t0 ? (t1 - t0) / (float)(G - 1) : 0.0f);
}

// Rows of the table for users [u0, u0 + nu): row r is user u0 + r / G at t_{r % G}.
__global__ void k_tab_inputs(int64_t u0, int64_t nu, int G, const float2 *__restrict__ tg,
                             int32_t *__restrict__ uid, float *__restrict__ t) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= nu * G) return;
  const int64_t u = u0 + r / G;
  const int g = (int)(r % G);
  const float2 gr = tg[u];
  uid[r] = (int32_t)u;
  t[r] = fmaf((float)g, gr.y, gr.x);
}

// y of pair i from user uid[i]'s table at t[i]: the grid coordinate x = (t - t_0) /
// step clamped to [0, G - 1], then linear interpolation between its two grid
// points.  The network never increases with t, so neither does the table nor its
// interpolation, which lies between the two grid values around t.
__global__ void k_tab_predict(int64_t B, const int32_t *__restrict__ uid,
                              const float *__restrict__ t, const float *__restrict__ tab,
                              const float2 *__restrict__ tg, int G, float *__restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= B) return;
  const int64_t u = uid[i];
  if (u < 0) { y[i] = 0.0f; return; }
  const float2 gr = tg[u];
  float x = gr.y > 0.0f ? (t[i] - gr.x) / gr.y : 0.0f;
  x = fminf(fmaxf(x, 0.0f), (float)(G - 1));   // fmaxf also maps NaN to 0
  const int j = min((int)x, G - 2);
  const float f = x - (float)j;
  const float *row = tab + u * G;
  y[i] = fmaf(f, row[j + 1] - row[j], row[j]);
}

}  // namespace

void pruner_drop_table(rkr_pruner *pr) {
  if (pr->tab) cudaFree(pr->tab);
  if (pr->tgrid) cudaFree(pr->tgrid);
  pr->tab = nullptr;
  pr->tgrid = nullptr;
  pr->tabG = 0;
  pr->tabn = 0;
  pr->tab_serial = 0;
  pr->tab_R.clear();
}

rkr_status pruner_build_table(rkr_pruner *pr, const rkr_index *idx, const float *Xu,
                              const std::vector<float> &Rh, int G, cudaStream_t st) {
  RKR_CUDA(cudaStreamSynchronize(st));
  pruner_drop_table(pr);
  if (G == 0) return RKR_OK;
  const int64_t n = idx->n;
  note_alloc();
  RKR_CUDA(cudaMalloc((void **)&pr->tab, sizeof(float) * (size_t)n * G));
  note_alloc();
  cudaError_t e = cudaMalloc((void **)&pr->tgrid, sizeof(float2) * (size_t)n);
  if (e != cudaSuccess) {
    pruner_drop_table(pr);
    return cuda_fail(e, "pruner table allocation");
  }
  k_tab_grid<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(n, idx->d, idx->U, idx->fmin,
                                                          idx->fmax, G, pr->tgrid);
  note_launch();
  RKR_CUDA(cudaGetLastError());
  // about four million table rows per forward call
  const int64_t users = std::max<int64_t>(1, ((int64_t)1 << 22) / G);
  const int64_t rows = std::min(users, n) * G;
  DevBuf bu, bt;
  int32_t *uid;
  float *t;
  RKR_TRY(tmp_alloc(bu, &uid, rows, st));
  RKR_TRY(tmp_alloc(bt, &t, rows, st));
  for (int64_t u0 = 0; u0 < n; u0 += users) {
    const int64_t nu = std::min(users, n - u0);
    k_tab_inputs<<<(unsigned)((nu * G + 255) / 256), 256, 0, st>>>(u0, nu, G, pr->tgrid, uid, t);
    note_launch();
    rkr_status s = pruner_forward_gather(pr, Xu, uid, t, nu * G, pr->tab + u0 * G, st);
    if (s != RKR_OK) {
      cudaStreamSynchronize(st);
      pruner_drop_table(pr);
      return s;
    }
  }
  RKR_CUDA(cudaStreamSynchronize(st));
  pr->tabG = G;
  pr->tabn = n;
  pr->tab_serial = idx->serial;
  pr->tab_R = Rh;
  return RKR_OK;
}

bool pruner_table_matches(const rkr_pruner *pr, const rkr_index *idx,
                          const std::vector<float> &Rh) {
  return pr->tab && pr->tabn == idx->n && pr->tab_serial == idx->serial && pr->tab_R == Rh;
}

rkr_status pruner_table_predict(const rkr_pruner *pr, const int32_t *uid, const float *t,
                                int64_t B, float *y, cudaStream_t st) {
  if (B <= 0) return RKR_OK;
  k_tab_predict<<<(unsigned)((B + 255) / 256), 256, 0, st>>>(B, uid, t, pr->tab, pr->tgrid,
                                                             pr->tabG, y);
  note_launch();
  RKR_CUDA(cudaGetLastError());
  return RKR_OK;
}

int pruner_features(const rkr_pruner *pr) { return pr->F; }
int pruner_hidden(const rkr_pruner *pr) { return pr->H; }

}  // namespace rkr

extern "C" {

rkr_status rkr_pruner_create(int32_t F, int32_t H, uint64_t seed, rkr_pruner **out) {
  using namespace rkr;
  if (!out) return fail(RKR_EINVAL, "null output");
  if (F < 1 || F > 1024 || H < 1 || H > 1024) return fail(RKR_EINVAL, "F and H must lie in [1, 1024]");
  rkr_pruner *pr = new rkr_pruner();
  pr->F = F;
  pr->H = H;
  pr->Fp = (F + 15) / 16 * 16;
  pr->Hp = (H + 15) / 16 * 16;
  const Off o(F, H);
  pr->nparam = o.n;
  std::vector<float> init(o.n, 0.0f);
  uint64_t x = seed;
  for (int64_t i = 0; i < (int64_t)H * F; ++i) init[o.W1 + i] = (float)(normal(x) / sqrt((double)F));
  for (int i = 0; i < H; ++i) init[o.A + i] = (float)(-1.0 + 0.1 * normal(x));
  const double v2 = log(expm1(1.0 / H)), v3 = log(expm1(1.0 / sqrt((double)H)));
  for (int64_t i = 0; i < (int64_t)H * H; ++i) init[o.V2 + i] = (float)(v2 + 0.1 * normal(x));
  for (int i = 0; i < H; ++i) init[o.v3 + i] = (float)v3;
  auto al = [&](auto **q, size_t count) -> rkr_status {
    note_alloc();
    cudaError_t e = cudaMalloc((void **)q, count * sizeof(**q));
    if (e != cudaSuccess) return cuda_fail(e, "pruner allocation");
    return RKR_OK;
  };
  rkr_status s = RKR_OK;
  if (s == RKR_OK) s = al(&pr->p, o.n);
  if (s == RKR_OK) s = al(&pr->g, o.n);
  if (s == RKR_OK) s = al(&pr->m, o.n);
  if (s == RKR_OK) s = al(&pr->v, o.n);
  if (s == RKR_OK) s = al(&pr->W1b, (size_t)H * pr->Fp);
  if (s == RKR_OK) s = al(&pr->W2b, (size_t)H * pr->Hp);
  if (s == RKR_OK) s = al(&pr->W2t, (size_t)H * pr->Hp);
  if (s == RKR_OK) s = al(&pr->err, 1);
  if (s == RKR_OK) s = al(&pr->wt, (size_t)H);
  if (s == RKR_OK) s = al(&pr->w3, (size_t)H);
  if (s == RKR_OK && cudaMemcpy(pr->p, init.data(), sizeof(float) * o.n, cudaMemcpyHostToDevice) != cudaSuccess)
    s = fail(RKR_ECUDA, "pruner parameter upload failed");
  if (s == RKR_OK) {
    cudaMemset(pr->m, 0, sizeof(float) * o.n);
    cudaMemset(pr->v, 0, sizeof(float) * o.n);
    cudaMemset(pr->g, 0, sizeof(float) * o.n);
    cudaMemset(pr->err, 0, sizeof(int));
  }
  if (s != RKR_OK) {
    rkr_pruner_free(pr);
    return s;
  }
  *out = pr;
  return RKR_OK;
}

int64_t rkr_pruner_nparams(const rkr_pruner *pr) { return pr ? pr->nparam : 0; }

rkr_status rkr_pruner_params(rkr_pruner *pr, int32_t set, float *params, int64_t count) {
  using namespace rkr;
  if (!pr || !params) return fail(RKR_EINVAL, "null argument");
  if (count != pr->nparam) return fail(RKR_EINVAL, "expected %lld parameters", (long long)pr->nparam);
  cudaError_t e = set ? cudaMemcpy(pr->p, params, sizeof(float) * count, cudaMemcpyDefault)
                      : cudaMemcpy(params, pr->p, sizeof(float) * count, cudaMemcpyDefault);
  if (e != cudaSuccess) return cuda_fail(e, "rkr_pruner_params");
  if (set) {
    pr->step = 0;
    pruner_drop_table(pr);   // new weights: the tables no longer hold
  }
  return RKR_OK;
}

rkr_status rkr_pruner_forward(rkr_pruner *pr, const float *X, const float *t, int64_t B, float *y,
                              void *stream) {
  using namespace rkr;
  if (!pr || !X || !t || !y) return fail(RKR_EINVAL, "null argument");
  if (B < 1) return fail(RKR_EINVAL, "B must be >= 1");
  cudaStream_t st = (cudaStream_t)stream;
  InDev vx, vt;
  RKR_TRY(vx.init(X, sizeof(float) * B * pr->F, st));
  RKR_TRY(vt.init(t, sizeof(float) * B, st));
  X = (const float *)vx.p;
  t = (const float *)vt.p;
  const int64_t chunk = 1 << 16;
  RKR_TRY(ensure_cap(pr, std::min(B, chunk), st));
  refresh_weights(pr, st);
  for (int64_t a = 0; a < B; a += chunk) {
    const int64_t b = std::min(B - a, chunk);
    k_mlp_batch<<<(unsigned)((b * pr->Fp + 255) / 256), 256, 0, st>>>(
        b, b, pr->F, pr->Fp, pr->cap, nullptr, X + a * pr->F, t + a, nullptr, pr->Xb, nullptr,
        pr->tb, nullptr);
    note_launch();
    RKR_TRY(forward_batch(pr, b, false, st));
    RKR_CUDA(cudaMemcpyAsync(y + a, pr->y, sizeof(float) * b, cudaMemcpyDefault, st));
  }
  RKR_CUDA(cudaStreamSynchronize(st));
  return check_err(pr, st);
}

rkr_status rkr_pruner_loss_grads(rkr_pruner *pr, const float *X, const float *t,
                                 const float *target, int64_t B, float *loss, float *grads,
                                 void *stream) {
  using namespace rkr;
  if (!pr || !X || !t || !target || !grads) return fail(RKR_EINVAL, "null argument");
  if (B < 1 || B > (1 << 20)) return fail(RKR_EINVAL, "B must lie in [1, 2^20]");
  cudaStream_t st = (cudaStream_t)stream;
  InDev vx, vt, vg;
  RKR_TRY(vx.init(X, sizeof(float) * B * pr->F, st));
  RKR_TRY(vt.init(t, sizeof(float) * B, st));
  RKR_TRY(vg.init(target, sizeof(float) * B, st));
  X = (const float *)vx.p;
  t = (const float *)vt.p;
  target = (const float *)vg.p;
  RKR_TRY(ensure_cap(pr, B, st));
  refresh_weights(pr, st);
  k_mlp_batch<<<(unsigned)((pr->cap * pr->Fp + 255) / 256), 256, 0, st>>>(
      B, pr->cap, pr->F, pr->Fp, pr->cap, nullptr, X, t, target, pr->Xb, pr->XbT, pr->tb,
      pr->tg);
  note_launch();
  RKR_TRY(forward_batch(pr, B, true, st));
  RKR_TRY(backward_batch(pr, B, st));
  RKR_TRY(check_err(pr, st));
  RKR_CUDA(cudaMemcpyAsync(grads, pr->g, sizeof(float) * pr->nparam, cudaMemcpyDefault, st));
  if (loss) {
    std::vector<float> y(B), tg(B);
    RKR_CUDA(cudaMemcpyAsync(y.data(), pr->y, sizeof(float) * B, cudaMemcpyDeviceToHost, st));
    RKR_CUDA(cudaMemcpyAsync(tg.data(), pr->tg, sizeof(float) * B, cudaMemcpyDeviceToHost, st));
    RKR_CUDA(cudaStreamSynchronize(st));
    double acc = 0.0;
    for (int64_t i = 0; i < B; ++i) acc += 0.5 * ((double)y[i] - tg[i]) * ((double)y[i] - tg[i]);
    *loss = (float)(acc / B);
  }
  RKR_CUDA(cudaStreamSynchronize(st));
  return RKR_OK;
}

rkr_status rkr_pruner_train(rkr_pruner *pr, const float *X, const float *t, const float *target,
                            int64_t npairs, int32_t epochs, int32_t batch, float lr,
                            uint64_t seed, float *final_loss, void *stream) {
  using namespace rkr;
  if (!pr || !X || !t || !target) return fail(RKR_EINVAL, "null argument");
  if (npairs < 1 || epochs < 1 || batch < 1 || !(lr > 0.0f))
    return fail(RKR_EINVAL, "bad training arguments");
  cudaStream_t st = (cudaStream_t)stream;
  InDev vx, vt, vg;
  RKR_TRY(vx.init(X, sizeof(float) * npairs * pr->F, st));
  RKR_TRY(vt.init(t, sizeof(float) * npairs, st));
  RKR_TRY(vg.init(target, sizeof(float) * npairs, st));
  X = (const float *)vx.p;
  t = (const float *)vt.p;
  target = (const float *)vg.p;
  const int64_t B = std::min<int64_t>(batch, npairs);
  RKR_TRY(ensure_cap(pr, B, st));
  pruner_drop_table(pr);   // training changes the weights the tables were built from
  int64_t *perm_d = nullptr;
  RKR_CUDA(pool_malloc_async(&perm_d, sizeof(int64_t) * npairs, st));
  std::vector<int64_t> perm(npairs);
  uint64_t x = seed;
  double last = 0.0;
  for (int ep = 0; ep < epochs; ++ep) {
    for (int64_t i = 0; i < npairs; ++i) perm[i] = i;
    for (int64_t i = npairs - 1; i > 0; --i) std::swap(perm[i], perm[splitmix(x) % (uint64_t)(i + 1)]);
    RKR_CUDA(cudaMemcpyAsync(perm_d, perm.data(), sizeof(int64_t) * npairs,
                             cudaMemcpyHostToDevice, st));
    for (int64_t a = 0; a + B <= npairs; a += B) {
      refresh_weights(pr, st);
      k_mlp_batch<<<(unsigned)((pr->cap * pr->Fp + 255) / 256), 256, 0, st>>>(
          B, pr->cap, pr->F, pr->Fp, pr->cap, perm_d + a, X, t, target, pr->Xb, pr->XbT,
          pr->tb, pr->tg);
      note_launch();
      RKR_TRY(forward_batch(pr, B, true, st));
      RKR_TRY(backward_batch(pr, B, st));
      pr->step += 1;
      const float b1c = 1.0f - powf(0.9f, (float)pr->step), b2c = 1.0f - powf(0.999f, (float)pr->step);
      k_adam<<<(unsigned)((pr->nparam + 255) / 256), 256, 0, st>>>(pr->nparam, pr->p, pr->g,
                                                                   pr->m, pr->v, lr, b1c, b2c);
      note_launch();
    }
    RKR_CUDA(cudaStreamSynchronize(st));  // the host permutation is rewritten next epoch
    RKR_TRY(check_err(pr, st));
  }
  // loss of the last batch
  if (final_loss) {
    std::vector<float> y(B), tg(B);
    RKR_CUDA(cudaMemcpyAsync(y.data(), pr->y, sizeof(float) * B, cudaMemcpyDeviceToHost, st));
    RKR_CUDA(cudaMemcpyAsync(tg.data(), pr->tg, sizeof(float) * B, cudaMemcpyDeviceToHost, st));
    RKR_CUDA(cudaStreamSynchronize(st));
    for (int64_t i = 0; i < B; ++i) last += 0.5 * ((double)y[i] - tg[i]) * ((double)y[i] - tg[i]);
    *final_loss = (float)(last / B);
  }
  cudaFreeAsync(perm_d, st);
  RKR_CUDA(cudaStreamSynchronize(st));
  return RKR_OK;
}

rkr_status rkr_pruner_table(const rkr_pruner *pr, int64_t n, int32_t G, float *tab,
                            float *grid) {
  using namespace rkr;
  if (!pr || !tab || !grid) return fail(RKR_EINVAL, "null argument");
  if (!pr->tab) return fail(RKR_EINVAL, "the pruner holds no tables (rkr_pruner_invert)");
  if (n != pr->tabn || G != pr->tabG)
    return fail(RKR_EINVAL, "the tables are %lld x %d", (long long)pr->tabn, pr->tabG);
  cudaError_t e = cudaMemcpy(tab, pr->tab, sizeof(float) * (size_t)n * G, cudaMemcpyDefault);
  if (e == cudaSuccess)
    e = cudaMemcpy(grid, pr->tgrid, sizeof(float2) * (size_t)n, cudaMemcpyDefault);
  if (e != cudaSuccess) return cuda_fail(e, "rkr_pruner_table");
  return RKR_OK;
}

void rkr_pruner_free(rkr_pruner *pr) {
  if (!pr) return;
  cudaDeviceSynchronize();
  rkr::pruner_drop_table(pr);
  for (void *q : {(void *)pr->p, (void *)pr->g, (void *)pr->m, (void *)pr->v, (void *)pr->W1b,
                  (void *)pr->W2b, (void *)pr->W2t, (void *)pr->wt, (void *)pr->w3,
                  (void *)pr->err, (void *)pr->Xb, (void *)pr->XbT, (void *)pr->h1,
                  (void *)pr->h1T, (void *)pr->h2, (void *)pr->d2b, (void *)pr->d2T,
                  (void *)pr->d1T, (void *)pr->z1, (void *)pr->z2, (void *)pr->y, (void *)pr->dy,
                  (void *)pr->tb, (void *)pr->d2, (void *)pr->d1, (void *)pr->tg})
    if (q) cudaFree(q);
  delete pr;
}

}  // extern "C"
