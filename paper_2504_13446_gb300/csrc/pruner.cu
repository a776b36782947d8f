// pruner.cu -- the learned pruner: a monotone rank regressor trained and run on
// the GPU with hand-written BF16 kernels (operands rounded to BF16, FP32
// accumulation and FP32 master weights).
//
// Model (F non-monotone features x, the normalised score t = u.q / ||u||):
//   h1 = relu(W1 x - softplus(A) t + b1),  h2 = relu(softplus(V2) h1 + b2),
//   y  = softplus(v3) . h2 + b3  ~  log r(q, u, P).
// The weights on every path from t are <= 0 before non-decreasing activations
// and >= 0 after them, so y is non-increasing in t, as the rank of Def. 1 is.
// Loss: 0.5 * mean((y - target)^2); Adam on the raw parameters.
// Flattened parameter order: W1 (H x F), A (H), b1 (H), V2 (H x H), b2 (H), v3 (H), b3.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "index.cuh"

struct rkr_pruner {
  int F = 0, H = 0;
  int64_t nparam = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // master, grad, Adam moments
  int64_t step = 0;
  // effective BF16 weights of the current parameters
  __nv_bfloat16 *W1b = nullptr, *W2b = nullptr;
  float *wt = nullptr, *w3 = nullptr;
  // batch scratch (capacity cap rows)
  int64_t cap = 0;
  __nv_bfloat16 *Xb = nullptr, *h1 = nullptr, *h2 = nullptr, *d2b = nullptr, *d1b = nullptr;
  float *z1 = nullptr, *z2 = nullptr, *y = nullptr, *dy = nullptr, *tb = nullptr, *d2 = nullptr,
        *d1 = nullptr, *tg = nullptr;
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

// Effective weights: W1 and softplus(V2) in BF16, -softplus(A) and softplus(v3) in FP32.
__global__ void k_mlp_weights(int F, int H, const float *__restrict__ p, Off o,
                              __nv_bfloat16 *__restrict__ W1b, __nv_bfloat16 *__restrict__ W2b,
                              float *__restrict__ wt, float *__restrict__ w3) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < (int64_t)H * F) W1b[i] = __float2bfloat16_rn(p[o.W1 + i]);
  if (i < (int64_t)H * H) W2b[i] = __float2bfloat16_rn(softplusf(p[o.V2 + i]));
  if (i < H) {
    wt[i] = -softplusf(p[o.A + i]);
    w3[i] = softplusf(p[o.v3 + i]);
  }
}

// C[m, n] = sum_k A(m, k) B(k, n) with BF16 operands and FP32 accumulation.
// A(m, k) = A[m * sam + k * sak], B(k, n) = B[k * sbk + n * sbn].  Epilogue:
// v = acc + bias[n] + tcol[m] * wcol[n] (each term optional); zout (FP32) gets v,
// hout (BF16) gets relu(v) or v, fout (FP32) gets v.
constexpr int GT = 128, GK = 16;   // 128 x 128 output tile, K in steps of 16
__global__ void __launch_bounds__(256)
    k_gemm_bf16(int M, int N, int K, const __nv_bfloat16 *__restrict__ A, int64_t sam,
                int64_t sak, const __nv_bfloat16 *__restrict__ B, int64_t sbk, int64_t sbn,
                const float *__restrict__ bias, const float *__restrict__ tcol,
                const float *__restrict__ wcol, int relu, float *__restrict__ zout,
                __nv_bfloat16 *__restrict__ hout, float *__restrict__ fout, int64_t ldc) {
  __shared__ __align__(16) float As[GK][GT + 4];
  __shared__ __align__(16) float Bs[GK][GT + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
  // the loads run along whichever index is contiguous in memory
  const bool a_m_fast = sam == 1, b_n_fast = sbn == 1;
  float acc[8][8] = {};
  for (int k0 = 0; k0 < K; k0 += GK) {
#pragma unroll
    for (int t = 0; t < (GT * GK) / 256; ++t) {
      const int e = tid + t * 256;
      const int mm = a_m_fast ? e % GT : e / GK, kk = a_m_fast ? e / GT : e % GK;
      const int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < K) ? __bfloat162float(A[gm * sam + gk * sak]) : 0.0f;
      const int nn = b_n_fast ? e % GT : e / GK, kb = b_n_fast ? e / GT : e % GK;
      const int gn = n0 + nn, gk2 = k0 + kb;
      Bs[kb][nn] = (gn < N && gk2 < K) ? __bfloat162float(B[gk2 * sbk + gn * sbn]) : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      // rows ty*4 + {0..3} and 64 + ty*4 + {0..3}; columns likewise with tx
      const float4 a0 = *(const float4 *)&As[kk][ty * 4];
      const float4 a1 = *(const float4 *)&As[kk][64 + ty * 4];
      const float4 b0 = *(const float4 *)&Bs[kk][tx * 4];
      const float4 b1 = *(const float4 *)&Bs[kk][64 + tx * 4];
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int gm = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int gn = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
      if (gn >= N) continue;
      float v = acc[i][j];
      if (bias) v += bias[gn];
      if (tcol) v = fmaf(tcol[gm], wcol[gn], v);
      const int64_t at = (int64_t)gm * ldc + gn;
      if (zout) zout[at] = v;
      if (fout) fout[at] = v;
      if (hout) hout[at] = __float2bfloat16_rn(relu ? fmaxf(v, 0.0f) : v);
    }
  }
}

constexpr int GS = 64;   // small tile: 64 x 64 outputs, 4 x 4 per thread
__global__ void __launch_bounds__(256)
    k_gemm_bf16_small(int M, int N, int K, const __nv_bfloat16 *__restrict__ A, int64_t sam,
                int64_t sak, const __nv_bfloat16 *__restrict__ B, int64_t sbk, int64_t sbn,
                const float *__restrict__ bias, const float *__restrict__ tcol,
                const float *__restrict__ wcol, int relu, float *__restrict__ zout,
                __nv_bfloat16 *__restrict__ hout, float *__restrict__ fout, int64_t ldc) {
  __shared__ float As[GK][GS + 1], Bs[GK][GS + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * GS, n0 = blockIdx.x * GS;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += GK) {
    for (int e = threadIdx.x; e < GS * GK; e += 256) {
      const int mm = e / GK, kk = e % GK;
      const int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < K) ? __bfloat162float(A[gm * sam + gk * sak]) : 0.0f;
      const int nn = e % GS, kb = e / GS;
      const int gn = n0 + nn, gk2 = k0 + kb;
      Bs[kb][nn] = (gn < N && gk2 < K) ? __bfloat162float(B[gk2 * sbk + gn * sbn]) : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        a[i] = As[kk][ty * 4 + i];
        b[i] = Bs[kk][tx * 4 + i];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty * 4 + i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx * 4 + j;
      if (gn >= N) continue;
      float v = acc[i][j];
      if (bias) v += bias[gn];
      if (tcol) v = fmaf(tcol[gm], wcol[gn], v);
      const int64_t at = (int64_t)gm * ldc + gn;
      if (zout) zout[at] = v;
      if (fout) fout[at] = v;
      if (hout) hout[at] = __float2bfloat16_rn(relu ? fmaxf(v, 0.0f) : v);
    }
  }
}

static void gemm(int M, int N, int K, const __nv_bfloat16 *A, int64_t sam, int64_t sak,
                 const __nv_bfloat16 *B, int64_t sbk, int64_t sbn, const float *bias,
                 const float *tcol, const float *wcol, int relu, float *zout, __nv_bfloat16 *hout,
                 float *fout, int64_t ldc, cudaStream_t st) {
  // large tiles when they still give every SM a block; the gradient products
  // (small outputs, long K) keep more blocks with small tiles
  const int64_t big = (int64_t)((N + GT - 1) / GT) * ((M + GT - 1) / GT);
  if (big >= 152) {
    dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT);
    k_gemm_bf16<<<grid, 256, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, bias, tcol, wcol, relu,
                                      zout, hout, fout, ldc);
  } else {
    dim3 grid((N + GS - 1) / GS, (M + GS - 1) / GS);
    k_gemm_bf16_small<<<grid, 256, 0, st>>>(M, N, K, A, sam, sak, B, sbk, sbn, bias, tcol, wcol,
                                            relu, zout, hout, fout, ldc);
  }
  note_launch();
}

// Gather a batch: BF16 features, FP32 scores and targets.
__global__ void k_mlp_batch(int64_t B, int F, const int64_t *__restrict__ idx,
                            const float *__restrict__ X, const float *__restrict__ t,
                            const float *__restrict__ target, __nv_bfloat16 *__restrict__ Xb,
                            float *__restrict__ tb, float *__restrict__ tg) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= B * F) return;
  const int64_t r = i / F, c = i % F;
  const int64_t s = idx ? idx[r] : r;
  Xb[i] = __float2bfloat16_rn(X[s * F + c]);
  if (c == 0) {
    tb[r] = t[s];
    if (target) tg[r] = target[s];
  }
}

// Gather rows of a per-user feature table: Xb[r] = Xu[uid[r]], tb[r] = t[r].
__global__ void k_mlp_gather(int64_t B, int F, const int32_t *__restrict__ uid,
                             const float *__restrict__ Xu, const float *__restrict__ t,
                             __nv_bfloat16 *__restrict__ Xb, float *__restrict__ tb) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= B * F) return;
  const int64_t r = i / F, c = i % F;
  const int64_t u = uid[r] < 0 ? 0 : uid[r];  // invalid rows read user 0 (ignored)
  Xb[i] = __float2bfloat16_rn(Xu[u * F + c]);
  if (c == 0) tb[r] = t[r];
}

// y[r] = w3 . h2[r] + b3 (one warp per row), and dy = (y - target) / B when asked.
__global__ void k_mlp_out(int64_t B, int H, const __nv_bfloat16 *__restrict__ h2,
                          const float *__restrict__ w3, const float *__restrict__ p, int64_t ob3,
                          float *__restrict__ y, const float *__restrict__ tg,
                          float *__restrict__ dy) {
  const int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= B) return;
  float acc = 0.0f;
  for (int n = lane; n < H; n += 32) acc = fmaf(__bfloat162float(h2[r * H + n]), w3[n], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) {
    const float yy = acc + p[ob3];
    y[r] = yy;
    if (dy) dy[r] = (yy - tg[r]) / (float)B;
  }
}

// dz2 = dy[r] * w3[n] * (z2 > 0), FP32 and BF16.
__global__ void k_mlp_dz2(int64_t B, int H, const float *__restrict__ dy,
                          const float *__restrict__ w3, const float *__restrict__ z2,
                          float *__restrict__ d2, __nv_bfloat16 *__restrict__ d2b) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= B * H) return;
  const float v = z2[i] > 0.0f ? dy[i / H] * w3[i % H] : 0.0f;
  d2[i] = v;
  d2b[i] = __float2bfloat16_rn(v);
}

// dz1 = (dz2 W2)[r, k] * (z1 > 0) in place of the product, FP32 and BF16.
__global__ void k_mlp_dz1(int64_t B, int H, const float *__restrict__ z1, float *__restrict__ d1,
                          __nv_bfloat16 *__restrict__ d1b) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= B * H) return;
  const float v = z1[i] > 0.0f ? d1[i] : 0.0f;
  d1[i] = v;
  d1b[i] = __float2bfloat16_rn(v);
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

rkr_status ensure_cap(rkr_pruner *pr, int64_t B, cudaStream_t st) {
  if (B <= pr->cap) return RKR_OK;
  const int H = pr->H, F = pr->F;
  for (void *q : {(void *)pr->Xb, (void *)pr->h1, (void *)pr->h2, (void *)pr->d2b,
                  (void *)pr->d1b, (void *)pr->z1, (void *)pr->z2, (void *)pr->y, (void *)pr->dy,
                  (void *)pr->tb, (void *)pr->d2, (void *)pr->d1, (void *)pr->tg})
    if (q) cudaFreeAsync(q, st);
  auto al = [&](auto **q, size_t count) -> rkr_status {
    cudaError_t e = pool_malloc_async((void **)q, count * sizeof(**q), st);
    if (e != cudaSuccess) return cuda_fail(e, "pruner scratch");
    return RKR_OK;
  };
  RKR_TRY(al(&pr->Xb, (size_t)B * F));
  RKR_TRY(al(&pr->h1, (size_t)B * H));
  RKR_TRY(al(&pr->h2, (size_t)B * H));
  RKR_TRY(al(&pr->d2b, (size_t)B * H));
  RKR_TRY(al(&pr->d1b, (size_t)B * H));
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
  const int64_t cnt = std::max<int64_t>((int64_t)pr->H * pr->F, (int64_t)pr->H * pr->H);
  k_mlp_weights<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(pr->F, pr->H, pr->p, o, pr->W1b,
                                                                pr->W2b, pr->wt, pr->w3);
  note_launch();
}

// Forward pass of the batch already gathered in Xb / tb; y in pr->y.
void forward_batch(rkr_pruner *pr, int64_t B, bool with_grad, cudaStream_t st) {
  const int F = pr->F, H = pr->H;
  const Off o(F, H);
  // z1 = X W1^T + b1 + t wt^T, h1 = relu(z1)
  gemm((int)B, H, F, pr->Xb, F, 1, pr->W1b, 1, F, pr->p + o.b1, pr->tb, pr->wt, 1, pr->z1,
       pr->h1, nullptr, H, st);
  // z2 = h1 W2^T + b2, h2 = relu(z2)
  gemm((int)B, H, H, pr->h1, H, 1, pr->W2b, 1, H, pr->p + o.b2, nullptr, nullptr, 1, pr->z2,
       pr->h2, nullptr, H, st);
  k_mlp_out<<<(unsigned)((B * 32 + 255) / 256), 256, 0, st>>>(
      B, H, pr->h2, pr->w3, pr->p, o.b3, pr->y, with_grad ? pr->tg : nullptr,
      with_grad ? pr->dy : nullptr);
  note_launch();
}

// Backward pass of the batch of the last forward: gradients of the raw
// parameters into pr->g (same order as the flat parameter vector).
void backward_batch(rkr_pruner *pr, int64_t B, cudaStream_t st) {
  const int F = pr->F, H = pr->H;
  const Off o(F, H);
  const unsigned nb = (unsigned)((B * H + 255) / 256);
  // dw3 = h2^T dy (the chain rule to v3 follows)
  k_colsum<<<H, 256, 0, st>>>(B, H, pr->z2, 1, pr->dy, pr->g + o.v3);
  note_launch();
  // dz2 = dy w3^T * (z2 > 0); db2 = column sums
  k_mlp_dz2<<<nb, 256, 0, st>>>(B, H, pr->dy, pr->w3, pr->z2, pr->d2, pr->d2b);
  note_launch();
  k_colsum<<<H, 256, 0, st>>>(B, H, pr->d2, 0, nullptr, pr->g + o.b2);
  note_launch();
  // dW2 = dz2^T h1 (H x H)
  gemm(H, H, (int)B, pr->d2b, 1, H, pr->h1, H, 1, nullptr, nullptr, nullptr, 0, nullptr, nullptr,
       pr->g + o.V2, H, st);
  // dh1 = dz2 W2 (B x H), then dz1 = dh1 * (z1 > 0)
  gemm((int)B, H, H, pr->d2b, H, 1, pr->W2b, H, 1, nullptr, nullptr, nullptr, 0, nullptr, nullptr,
       pr->d1, H, st);
  k_mlp_dz1<<<nb, 256, 0, st>>>(B, H, pr->z1, pr->d1, pr->d1b);
  note_launch();
  // db1 = column sums; d(wt) = dz1^T t
  k_colsum<<<H, 256, 0, st>>>(B, H, pr->d1, 0, nullptr, pr->g + o.b1);
  note_launch();
  k_colsum<<<H, 256, 0, st>>>(B, H, pr->d1, 0, pr->tb, pr->g + o.A);
  note_launch();
  // dW1 = dz1^T X (H x F)
  gemm(H, F, (int)B, pr->d1b, 1, H, pr->Xb, F, 1, nullptr, nullptr, nullptr, 0, nullptr, nullptr,
       pr->g + o.W1, F, st);
  // constrained parameters and db3
  const int64_t cnt = std::max<int64_t>((int64_t)H * H, 1);
  k_mlp_chain<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(H, pr->p, o, pr->g, pr->dy, B);
  note_launch();
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
    k_mlp_gather<<<(unsigned)((b * pr->F + 255) / 256), 256, 0, st>>>(b, pr->F, uid + a, Xu,
                                                                      t + a, pr->Xb, pr->tb);
    note_launch();
    forward_batch(pr, b, false, st);
    RKR_CUDA(cudaMemcpyAsync(y + a, pr->y, sizeof(float) * b, cudaMemcpyDeviceToDevice, st));
  }
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
  if (s == RKR_OK) s = al(&pr->W1b, (size_t)H * F);
  if (s == RKR_OK) s = al(&pr->W2b, (size_t)H * H);
  if (s == RKR_OK) s = al(&pr->wt, (size_t)H);
  if (s == RKR_OK) s = al(&pr->w3, (size_t)H);
  if (s == RKR_OK && cudaMemcpy(pr->p, init.data(), sizeof(float) * o.n, cudaMemcpyHostToDevice) != cudaSuccess)
    s = fail(RKR_ECUDA, "pruner parameter upload failed");
  if (s == RKR_OK) {
    cudaMemset(pr->m, 0, sizeof(float) * o.n);
    cudaMemset(pr->v, 0, sizeof(float) * o.n);
    cudaMemset(pr->g, 0, sizeof(float) * o.n);
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
  if (set) pr->step = 0;
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
    k_mlp_batch<<<(unsigned)((b * pr->F + 255) / 256), 256, 0, st>>>(
        b, pr->F, nullptr, X + a * pr->F, t + a, nullptr, pr->Xb, pr->tb, pr->tg);
    note_launch();
    forward_batch(pr, b, false, st);
    RKR_CUDA(cudaMemcpyAsync(y + a, pr->y, sizeof(float) * b, cudaMemcpyDefault, st));
  }
  RKR_CUDA(cudaStreamSynchronize(st));
  return RKR_OK;
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
  k_mlp_batch<<<(unsigned)((B * pr->F + 255) / 256), 256, 0, st>>>(B, pr->F, nullptr, X, t,
                                                                   target, pr->Xb, pr->tb, pr->tg);
  note_launch();
  forward_batch(pr, B, true, st);
  backward_batch(pr, B, st);
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
      k_mlp_batch<<<(unsigned)((B * pr->F + 255) / 256), 256, 0, st>>>(
          B, pr->F, perm_d + a, X, t, target, pr->Xb, pr->tb, pr->tg);
      note_launch();
      forward_batch(pr, B, true, st);
      backward_batch(pr, B, st);
      pr->step += 1;
      const float b1c = 1.0f - powf(0.9f, (float)pr->step), b2c = 1.0f - powf(0.999f, (float)pr->step);
      k_adam<<<(unsigned)((pr->nparam + 255) / 256), 256, 0, st>>>(pr->nparam, pr->p, pr->g,
                                                                   pr->m, pr->v, lr, b1c, b2c);
      note_launch();
    }
    RKR_CUDA(cudaStreamSynchronize(st));  // the host permutation is rewritten next epoch
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

void rkr_pruner_free(rkr_pruner *pr) {
  if (!pr) return;
  cudaDeviceSynchronize();
  for (void *q : {(void *)pr->p, (void *)pr->g, (void *)pr->m, (void *)pr->v, (void *)pr->W1b,
                  (void *)pr->W2b, (void *)pr->wt, (void *)pr->w3, (void *)pr->Xb, (void *)pr->h1,
                  (void *)pr->h2, (void *)pr->d2b, (void *)pr->d1b, (void *)pr->z1, (void *)pr->z2,
                  (void *)pr->y, (void *)pr->dy, (void *)pr->tb, (void *)pr->d2, (void *)pr->d1,
                  (void *)pr->tg})
    if (q) cudaFree(q);
  delete pr;
}

}  // extern "C"
