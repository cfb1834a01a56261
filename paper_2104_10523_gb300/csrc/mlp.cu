// Learned path cost model: a 3-layer MLP (hidden width h, BF16 weights, FP32
// master weights and accumulation) predicting the log time of a contraction
// step from its features; training and inference run in these kernels.
//
//   z1 = x W1 + b1, a1 = relu(z1); z2 = a1 W2 + b2, a2 = relu(z2); y = a2 W3 + b3
//   loss = mean (y - t)^2, gradients by the chain rule, Adam updates of the FP32
//   master weights followed by a refresh of their BF16 copies.
//
// The paper motivates such a model (a path with more flops ran faster on the
// hardware, Sec. 4.3) but defines none.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <random>
#include <string>
#include <vector>

#include "executor.h"
#include "mlp.h"

namespace tnq {

namespace {

// ---------------------------------------------------------------- GEMM
// C[M][N] (+)= op(A)[M][K] * op(B)[K][N] (+ bias[N]); A float, B float or bf16.
// op(A)(i,k) = transA ? A[k*lda + i] : A[i*lda + k]; likewise B.
constexpr int MG_T = 64, MG_K = 16;

template <typename TB>
__global__ void __launch_bounds__(256) mlp_gemm_kernel(int M, int N, int K, const float* __restrict__ A, int lda,
                                                       int transA, const TB* __restrict__ B, int ldb, int transB,
                                                       float* __restrict__ C, int ldc, const float* __restrict__ bias,
                                                       int relu_into, float* __restrict__ R) {
  __shared__ float As[MG_K][MG_T + 1];
  __shared__ float Bs[MG_K][MG_T + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * MG_T, n0 = blockIdx.x * MG_T;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = 0; k0 < K; k0 += MG_K) {
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int idx = tid + 256 * l;
      // A tile: rows m0..m0+63, k0..k0+15
      {
        const int r = transA ? idx % MG_T : idx / MG_K, kk = transA ? idx / MG_T : idx % MG_K;
        float v = 0.f;
        if (m0 + r < M && k0 + kk < K) v = transA ? A[size_t(k0 + kk) * lda + m0 + r] : A[size_t(m0 + r) * lda + k0 + kk];
        As[kk][r] = v;
      }
      // B tile: k0..k0+15, columns n0..n0+63
      {
        const int c = transB ? idx / MG_K : idx % MG_T, kk = transB ? idx % MG_K : idx / MG_T;
        float v = 0.f;
        if (n0 + c < N && k0 + kk < K) {
          const TB b = transB ? B[size_t(n0 + c) * ldb + k0 + kk] : B[size_t(k0 + kk) * ldb + n0 + c];
          v = float(b);
        }
        Bs[kk][c] = v;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < MG_K; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = m0 + ty + 16 * i, n = n0 + tx + 16 * j;
      if (m < M && n < N) {
        float v = acc[i][j] + (bias ? bias[n] : 0.f);
        C[size_t(m) * ldc + n] = v;
        if (relu_into) R[size_t(m) * ldc + n] = fmaxf(v, 0.f);
      }
    }
}

template <typename TB>
cudaError_t gemm(cudaStream_t st, int M, int N, int K, const float* A, int lda, int tA, const TB* B, int ldb, int tB,
                 float* C, int ldc, const float* bias = nullptr, float* relu_out = nullptr) {
  dim3 grid((N + MG_T - 1) / MG_T, (M + MG_T - 1) / MG_T);
  mlp_gemm_kernel<TB><<<grid, 256, 0, st>>>(M, N, K, A, lda, tA, B, ldb, tB, C, ldc, bias, relu_out ? 1 : 0,
                                            relu_out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- elementwise
__global__ void dy_kernel(const float* y, const float* t, int B, float* dy, float* sq) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B; i += gridDim.x * blockDim.x) {
    const float d = y[i] - t[i];
    dy[i] = 2.f * d / float(B);
    sq[i] = d * d;
  }
}

// g[i] *= (z[i] > 0)
__global__ void relu_mask_kernel(float* g, const float* z, size_t n) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    if (!(z[i] > 0.f)) g[i] = 0.f;
}

// out[c] = sum over rows r < R of X[r*ld + c] (fixed row order); optionally / div
__global__ void colsum_kernel(const float* X, int R, int Cn, int ld, float* out, float scale) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < Cn; c += gridDim.x * blockDim.x) {
    float s = 0.f;
    for (int r = 0; r < R; ++r) s += X[size_t(r) * ld + c];
    out[c] = s * scale;
  }
}

__global__ void adam_kernel(float* p, const float* g, float* m, float* v, size_t n, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

__global__ void to_bf16_kernel(const float* src, __nv_bfloat16* dst, size_t n) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x)
    dst[i] = __float2bfloat16_rn(src[i]);
}

unsigned nblk(size_t n) { return unsigned(std::max<size_t>(1, std::min<size_t>((n + 255) / 256, 2048))); }

}  // namespace

// ---------------------------------------------------------------- model
size_t CostModel::n_params() const { return size_t(d_in) * h + h + size_t(h) * h + h + h + 1; }

void CostModel::layout() {
  const size_t P = n_params();
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = (off + bytes + 255) / 256 * 256;
    return o;
  };
  o_params = take(4 * P);
  o_grads = take(4 * P);
  o_m = take(4 * P);
  o_v = take(4 * P);
  o_w1b = take(2 * size_t(d_in) * h);
  o_w2b = take(2 * size_t(h) * h);
  o_w3b = take(2 * size_t(h));
  const size_t B = size_t(max_batch);
  o_x = take(4 * B * d_in);
  o_t = take(4 * B);
  o_z1 = take(4 * B * h);
  o_a1 = take(4 * B * h);
  o_z2 = take(4 * B * h);
  o_a2 = take(4 * B * h);
  o_y = take(4 * B);
  o_dy = take(4 * B);
  o_sq = take(4 * B);
  o_dz1 = take(4 * B * h);
  o_dz2 = take(4 * B * h);
  o_loss = take(8);
  ws_bytes = off;
}

// Parameter offsets (floats) inside the flat vector: W1, b1, W2, b2, W3, b3.
static void param_offsets(const CostModel& m, size_t* w1, size_t* b1, size_t* w2, size_t* b2, size_t* w3, size_t* b3) {
  *w1 = 0;
  *b1 = *w1 + size_t(m.d_in) * m.h;
  *w2 = *b1 + m.h;
  *b2 = *w2 + size_t(m.h) * m.h;
  *w3 = *b2 + m.h;
  *b3 = *w3 + m.h;
}

#define MLP_CUDA(call)                                  \
  do {                                                  \
    cudaError_t _e = (call);                            \
    if (_e != cudaSuccess) return cuda_fail(_e, #call); \
  } while (0)

static tnq_status refresh_bf16(Ctx* ctx, CostModel* m) {
  char* ws = static_cast<char*>(m->ws);
  size_t w1, b1, w2, b2, w3, b3;
  param_offsets(*m, &w1, &b1, &w2, &b2, &w3, &b3);
  const float* P = reinterpret_cast<const float*>(ws + m->o_params);
  to_bf16_kernel<<<nblk(size_t(m->d_in) * m->h), 256, 0, ctx->stream>>>(P + w1, reinterpret_cast<__nv_bfloat16*>(ws + m->o_w1b), size_t(m->d_in) * m->h);
  to_bf16_kernel<<<nblk(size_t(m->h) * m->h), 256, 0, ctx->stream>>>(P + w2, reinterpret_cast<__nv_bfloat16*>(ws + m->o_w2b), size_t(m->h) * m->h);
  to_bf16_kernel<<<nblk(m->h), 256, 0, ctx->stream>>>(P + w3, reinterpret_cast<__nv_bfloat16*>(ws + m->o_w3b), size_t(m->h));
  MLP_CUDA(cudaGetLastError());
  ctx->launches += 3;
  return TNQ_OK;
}

// Forward on B rows already in the x region; leaves y (and z/a for backward).
static tnq_status forward(Ctx* ctx, CostModel* m, int B) {
  char* ws = static_cast<char*>(m->ws);
  size_t w1, b1, w2, b2, w3, b3;
  param_offsets(*m, &w1, &b1, &w2, &b2, &w3, &b3);
  const float* P = reinterpret_cast<const float*>(ws + m->o_params);
  auto f = [&](size_t o) { return reinterpret_cast<float*>(ws + o); };
  const __nv_bfloat16* W1 = reinterpret_cast<const __nv_bfloat16*>(ws + m->o_w1b);
  const __nv_bfloat16* W2 = reinterpret_cast<const __nv_bfloat16*>(ws + m->o_w2b);
  const __nv_bfloat16* W3 = reinterpret_cast<const __nv_bfloat16*>(ws + m->o_w3b);
  const int h = m->h;
  MLP_CUDA(gemm(ctx->stream, B, h, m->d_in, f(m->o_x), m->d_in, 0, W1, h, 0, f(m->o_z1), h, P + b1, f(m->o_a1)));
  MLP_CUDA(gemm(ctx->stream, B, h, h, f(m->o_a1), h, 0, W2, h, 0, f(m->o_z2), h, P + b2, f(m->o_a2)));
  MLP_CUDA(gemm(ctx->stream, B, 1, h, f(m->o_a2), h, 0, W3, 1, 0, f(m->o_y), 1, P + b3));
  ctx->launches += 3;
  return TNQ_OK;
}

// Backward for B rows with targets in the t region; writes the gradient vector.
static tnq_status backward(Ctx* ctx, CostModel* m, int B) {
  char* ws = static_cast<char*>(m->ws);
  size_t w1, b1, w2, b2, w3, b3;
  param_offsets(*m, &w1, &b1, &w2, &b2, &w3, &b3);
  auto f = [&](size_t o) { return reinterpret_cast<float*>(ws + o); };
  float* G = f(m->o_grads);
  const __nv_bfloat16* W2 = reinterpret_cast<const __nv_bfloat16*>(ws + m->o_w2b);
  const __nv_bfloat16* W3 = reinterpret_cast<const __nv_bfloat16*>(ws + m->o_w3b);
  const int h = m->h;
  dy_kernel<<<nblk(B), 256, 0, ctx->stream>>>(f(m->o_y), f(m->o_t), B, f(m->o_dy), f(m->o_sq));
  // W3 grad = a2^T dy ; b3 grad = sum dy
  MLP_CUDA(gemm(ctx->stream, h, 1, B, f(m->o_a2), h, 1, f(m->o_dy), 1, 0, G + w3, 1));
  colsum_kernel<<<1, 32, 0, ctx->stream>>>(f(m->o_dy), B, 1, 1, G + b3, 1.f);
  // dz2 = (dy W3^T) * (z2 > 0)
  MLP_CUDA(gemm(ctx->stream, B, h, 1, f(m->o_dy), 1, 0, W3, 1, 1, f(m->o_dz2), h));
  relu_mask_kernel<<<nblk(size_t(B) * h), 256, 0, ctx->stream>>>(f(m->o_dz2), f(m->o_z2), size_t(B) * h);
  MLP_CUDA(gemm(ctx->stream, h, h, B, f(m->o_a1), h, 1, f(m->o_dz2), h, 0, G + w2, h));
  colsum_kernel<<<nblk(h), 256, 0, ctx->stream>>>(f(m->o_dz2), B, h, h, G + b2, 1.f);
  // dz1 = (dz2 W2^T) * (z1 > 0)
  MLP_CUDA(gemm(ctx->stream, B, h, h, f(m->o_dz2), h, 0, W2, h, 1, f(m->o_dz1), h));
  relu_mask_kernel<<<nblk(size_t(B) * h), 256, 0, ctx->stream>>>(f(m->o_dz1), f(m->o_z1), size_t(B) * h);
  MLP_CUDA(gemm(ctx->stream, m->d_in, h, B, f(m->o_x), m->d_in, 1, f(m->o_dz1), h, 0, G + w1, h));
  colsum_kernel<<<nblk(h), 256, 0, ctx->stream>>>(f(m->o_dz1), B, h, h, G + b1, 1.f);
  // loss = mean squared error (sum of squares in row order)
  colsum_kernel<<<1, 32, 0, ctx->stream>>>(f(m->o_sq), B, 1, 1, f(m->o_loss), 1.f / float(B));
  MLP_CUDA(cudaGetLastError());
  ctx->launches += 13;
  return TNQ_OK;
}

static tnq_status adam(Ctx* ctx, CostModel* m, float lr) {
  char* ws = static_cast<char*>(m->ws);
  m->adam_t += 1;
  const float c1 = float(1.0 - std::pow(0.9, m->adam_t)), c2 = float(1.0 - std::pow(0.999, m->adam_t));
  const size_t P = m->n_params();
  adam_kernel<<<nblk(P), 256, 0, ctx->stream>>>(reinterpret_cast<float*>(ws + m->o_params),
                                                reinterpret_cast<const float*>(ws + m->o_grads),
                                                reinterpret_cast<float*>(ws + m->o_m), reinterpret_cast<float*>(ws + m->o_v),
                                                P, lr, 0.9f, 0.999f, 1e-8f, c1, c2);
  MLP_CUDA(cudaGetLastError());
  ctx->launches++;
  return refresh_bf16(ctx, m);
}

tnq_status mlp_bind(Ctx* ctx, CostModel* m, void* ws, size_t bytes) {
  if (!ws || bytes < m->ws_bytes)
    return fail(TNQ_ERR_WORKSPACE, "cost-model workspace needs " + std::to_string(m->ws_bytes) + " bytes");
  MLP_CUDA(cudaSetDevice(ctx->device));
  m->ws = ws;
  return mlp_upload(ctx, m, m->host_params.data());
}

tnq_status mlp_upload(Ctx* ctx, CostModel* m, const float* params) {
  if (!m->ws) return fail(TNQ_ERR_WORKSPACE, "cost model has no bound workspace");
  char* ws = static_cast<char*>(m->ws);
  const size_t P = m->n_params();
  m->host_params.assign(params, params + P);
  MLP_CUDA(cudaMemcpyAsync(ws + m->o_params, params, 4 * P, cudaMemcpyHostToDevice, ctx->stream));
  MLP_CUDA(cudaMemsetAsync(ws + m->o_m, 0, 4 * P, ctx->stream));
  MLP_CUDA(cudaMemsetAsync(ws + m->o_v, 0, 4 * P, ctx->stream));
  m->adam_t = 0;
  tnq_status s = refresh_bf16(ctx, m);
  if (s != TNQ_OK) return s;
  MLP_CUDA(cudaStreamSynchronize(ctx->stream));
  return TNQ_OK;
}

tnq_status mlp_download(Ctx* ctx, CostModel* m, float* params) {
  if (!m->ws) return fail(TNQ_ERR_WORKSPACE, "cost model has no bound workspace");
  MLP_CUDA(cudaMemcpyAsync(params, static_cast<char*>(m->ws) + m->o_params, 4 * m->n_params(), cudaMemcpyDeviceToHost,
                           ctx->stream));
  MLP_CUDA(cudaStreamSynchronize(ctx->stream));
  return TNQ_OK;
}

tnq_status mlp_gradients(Ctx* ctx, CostModel* m, const float* X, const float* t, int64_t n, float* grads,
                         float* loss) {
  if (!m->ws) return fail(TNQ_ERR_WORKSPACE, "cost model has no bound workspace");
  if (n < 1 || n > m->max_batch) return fail(TNQ_ERR_INVALID_ARG, "row count must be in [1, max_batch]");
  char* ws = static_cast<char*>(m->ws);
  MLP_CUDA(cudaMemcpyAsync(ws + m->o_x, X, 4 * size_t(n) * m->d_in, cudaMemcpyHostToDevice, ctx->stream));
  MLP_CUDA(cudaMemcpyAsync(ws + m->o_t, t, 4 * size_t(n), cudaMemcpyHostToDevice, ctx->stream));
  tnq_status s = forward(ctx, m, int(n));
  if (s == TNQ_OK) s = backward(ctx, m, int(n));
  if (s != TNQ_OK) return s;
  if (grads)
    MLP_CUDA(cudaMemcpyAsync(grads, ws + m->o_grads, 4 * m->n_params(), cudaMemcpyDeviceToHost, ctx->stream));
  if (loss) MLP_CUDA(cudaMemcpyAsync(loss, ws + m->o_loss, 4, cudaMemcpyDeviceToHost, ctx->stream));
  MLP_CUDA(cudaStreamSynchronize(ctx->stream));
  return TNQ_OK;
}

tnq_status mlp_train(Ctx* ctx, CostModel* m, const float* X, const float* t, int64_t n, int epochs, int batch,
                     float lr, float* final_loss) {
  if (!m->ws) return fail(TNQ_ERR_WORKSPACE, "cost model has no bound workspace");
  if (n < 1 || epochs < 1 || batch < 1 || batch > m->max_batch)
    return fail(TNQ_ERR_INVALID_ARG, "bad training arguments (n >= 1, epochs >= 1, 1 <= batch <= max_batch)");
  char* ws = static_cast<char*>(m->ws);
  // minibatches in a seeded order per epoch; rows staged from the host per batch
  std::vector<int64_t> order(n);
  for (int64_t i = 0; i < n; ++i) order[i] = i;
  std::mt19937_64 g(m->seed ^ 0xC0FFEEULL);
  std::vector<float> xb(size_t(batch) * m->d_in), tb(batch);
  float last = 0.f;
  for (int e = 0; e < epochs; ++e) {
    std::shuffle(order.begin(), order.end(), g);
    for (int64_t s0 = 0; s0 < n; s0 += batch) {
      const int B = int(std::min<int64_t>(batch, n - s0));
      for (int r = 0; r < B; ++r) {
        const int64_t src = order[s0 + r];
        std::copy(X + src * m->d_in, X + (src + 1) * m->d_in, xb.begin() + size_t(r) * m->d_in);
        tb[r] = t[src];
      }
      MLP_CUDA(cudaMemcpyAsync(ws + m->o_x, xb.data(), 4 * size_t(B) * m->d_in, cudaMemcpyHostToDevice, ctx->stream));
      MLP_CUDA(cudaMemcpyAsync(ws + m->o_t, tb.data(), 4 * size_t(B), cudaMemcpyHostToDevice, ctx->stream));
      tnq_status s = forward(ctx, m, B);
      if (s == TNQ_OK) s = backward(ctx, m, B);
      if (s == TNQ_OK) s = adam(ctx, m, lr);
      if (s != TNQ_OK) return s;
      // the staging vectors are reused: wait for this batch's copies
      MLP_CUDA(cudaStreamSynchronize(ctx->stream));
    }
  }
  MLP_CUDA(cudaMemcpyAsync(&last, ws + m->o_loss, 4, cudaMemcpyDeviceToHost, ctx->stream));
  MLP_CUDA(cudaStreamSynchronize(ctx->stream));
  if (final_loss) *final_loss = last;
  return mlp_download(ctx, m, m->host_params.data());
}

tnq_status mlp_predict(Ctx* ctx, CostModel* m, const float* X, int64_t n, float* y) {
  if (!m->ws) return fail(TNQ_ERR_WORKSPACE, "cost model has no bound workspace");
  char* ws = static_cast<char*>(m->ws);
  const bool x_dev = false;
  (void)x_dev;
  for (int64_t s0 = 0; s0 < n; s0 += m->max_batch) {
    const int B = int(std::min<int64_t>(m->max_batch, n - s0));
    MLP_CUDA(cudaMemcpyAsync(ws + m->o_x, X + s0 * m->d_in, 4 * size_t(B) * m->d_in, cudaMemcpyHostToDevice,
                             ctx->stream));
    tnq_status s = forward(ctx, m, B);
    if (s != TNQ_OK) return s;
    MLP_CUDA(cudaMemcpyAsync(y + s0, ws + m->o_y, 4 * size_t(B), cudaMemcpyDeviceToHost, ctx->stream));
    MLP_CUDA(cudaStreamSynchronize(ctx->stream));
  }
  return TNQ_OK;
}

void mlp_init(CostModel* m) {
  // He-uniform initial weights from a seeded generator, zero biases
  const size_t P = m->n_params();
  m->host_params.assign(P, 0.f);
  size_t w1, b1, w2, b2, w3, b3;
  param_offsets(*m, &w1, &b1, &w2, &b2, &w3, &b3);
  std::mt19937_64 g(m->seed);
  auto fill = [&](size_t off, size_t count, int fan_in) {
    const double b = std::sqrt(6.0 / fan_in);
    for (size_t i = 0; i < count; ++i) m->host_params[off + i] = float((2.0 * ((g() >> 11) * (1.0 / 9007199254740992.0)) - 1.0) * b);
  };
  fill(w1, size_t(m->d_in) * m->h, m->d_in);
  fill(w2, size_t(m->h) * m->h, m->h);
  fill(w3, size_t(m->h), m->h);
}

}  // namespace tnq
