// Surrogate network for the learned energy grid: a fully connected MLP
//   x (n_in) -> [Linear -> GELU] x hidden_layers (width) -> Linear -> y (n_out)
// trained with mean-squared error and Adam, all on the GPU in hand-written kernels: a tiled FP32
// GEMM with fused bias + GELU (forward) and transposed operands (backward), column sums for the bias
// gradients, the GELU derivative, the loss and the Adam update. Inference can read a BF16 copy of
// the weights (FP32 accumulation). GELU is the tanh form 0.5 z (1 + tanh(sqrt(2/pi)(z + 0.044715 z^3))).
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/hsc_mlp.h"
#include "ctx.h"

struct hsc_mlp_ctx {
  int n_in = 0, width = 0, hidden = 0, n_out = 0, max_batch = 0, L = 0;
  std::vector<int> din, dout;
  std::vector<int64_t> woff, boff;   // offsets of W_l (din x dout, row-major) and b_l in params
  int64_t np = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  __nv_bfloat16* pb = nullptr;       // BF16 copy of the parameters (inference)
  bool pb_valid = false;
  float *Z = nullptr, *A = nullptr, *dA = nullptr, *dZ = nullptr, *y = nullptr, *loss = nullptr;
  int64_t step = 0;
};

namespace {

constexpr int TM = 64, TN = 64, TK = 16, MLP_THREADS = 256;

__device__ __forceinline__ float gelu(float z) {
  const float c = 0.7978845608028654f;
  return 0.5f * z * (1.0f + tanhf(c * (z + 0.044715f * z * z * z)));
}

__device__ __forceinline__ float gelu_grad(float z) {
  const float c = 0.7978845608028654f;
  const float t = tanhf(c * (z + 0.044715f * z * z * z));
  return 0.5f * (1.0f + t) + 0.5f * z * (1.0f - t * t) * c * (1.0f + 3.0f * 0.044715f * z * z);
}

__device__ __forceinline__ float ldv(const float* p) { return *p; }
__device__ __forceinline__ float ldv(const __nv_bfloat16* p) { return __bfloat162float(*p); }

// C[M x N] = op(A) op(B) (+ bias, GELU). TA: A stored K x M; TB: B stored N x K.
// mode 0: C = AB; 1: Z = AB + b, C = gelu(Z); 2: C = AB + b
template <bool TA, bool TB, typename TBt>
__global__ void __launch_bounds__(MLP_THREADS)
k_sgemm(int M, int N, int K, const float* A, int lda, const TBt* B, int ldb, float* C, int ldc,
        const TBt* bias, int mode, float* Zout) {
  __shared__ float As[TK][TM + 1];
  __shared__ float Bs[TK][TN + 1];
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += TK) {
    for (int i = threadIdx.x; i < TM * TK; i += MLP_THREADS) {
      int mm, kk;
      if (TA) { mm = i % TM; kk = i / TM; } else { kk = i % TK; mm = i / TK; }
      int gm = m0 + mm, gk = k0 + kk;
      float v = 0.f;
      if (gm < M && gk < K) v = TA ? A[(int64_t)gk * lda + gm] : A[(int64_t)gm * lda + gk];
      As[kk][mm] = v;
    }
    for (int i = threadIdx.x; i < TN * TK; i += MLP_THREADS) {
      int nn, kk;
      if (TB) { kk = i % TK; nn = i / TK; } else { nn = i % TN; kk = i / TN; }
      int gn = n0 + nn, gk = k0 + kk;
      float v = 0.f;
      if (gn < N && gk < K) v = TB ? ldv(&B[(int64_t)gn * ldb + gk]) : ldv(&B[(int64_t)gk * ldb + gn]);
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
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
      int r = m0 + ty * 4 + i, c = n0 + tx * 4 + j;
      if (r >= M || c >= N) continue;
      float z = acc[i][j];
      if (mode >= 1) z += ldv(&bias[c]);
      if (mode == 1) {
        if (Zout) Zout[(int64_t)r * N + c] = z;
        C[(int64_t)r * ldc + c] = gelu(z);
      } else {
        C[(int64_t)r * ldc + c] = z;
      }
    }
}

__global__ void k_gelu_back(int64_t n, const float* dA, const float* Z, float* dZ) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dZ[i] = dA[i] * gelu_grad(Z[i]);
}

// db[c] = sum_r dZ[r][c]
__global__ void k_colsum(int R, int Cc, const float* dZ, float* db) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= Cc) return;
  float s = 0.f;
  for (int r = 0; r < R; ++r) s += dZ[(int64_t)r * Cc + c];
  db[c] = s;
}

// dY = 2 (y - t) / (B n_out); loss = mean (y - t)^2 (single block reduction)
__global__ void k_mse(int n, const float* y, const float* t, float* dY, float* loss) {
  __shared__ float red[256];
  float s = 0.f;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    float d = y[i] - t[i];
    dY[i] = 2.f * d / n;
    s += d * d;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *loss = red[0] / n;
}

__global__ void k_adam(int64_t n, float* p, const float* g, float* m, float* v, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gi = g[i];
  float mi = b1 * m[i] + (1.f - b1) * gi;
  float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_to_bf16(int64_t n, const float* p, __nv_bfloat16* q) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) q[i] = __float2bfloat16(p[i]);
}

template <bool TA, bool TB, typename TBt>
cudaError_t sgemm(int M, int N, int K, const float* A, int lda, const TBt* B, int ldb, float* C,
                  int ldc, const TBt* bias, int mode, float* Z, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM);
  k_sgemm<TA, TB, TBt><<<grid, MLP_THREADS, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc, bias, mode, Z);
  return cudaGetLastError();
}

int blocks(int64_t n) { return (int)((n + 255) / 256); }

// activations of layer l (0 = input copy is not stored: A_0 is x) live at A + (l-1) * B * width
int forward(hsc_mlp_ctx* c, int B, const float* x, float* y, bool bf16, cudaStream_t s) {
  const float* in = x;
  int ld_in = c->n_in;
  for (int l = 0; l < c->L; ++l) {
    const bool last = l == c->L - 1;
    float* out = last ? y : c->A + (int64_t)l * c->max_batch * c->width;
    float* Z = last ? nullptr : c->Z + (int64_t)l * c->max_batch * c->width;
    const int mode = last ? 2 : 1;
    cudaError_t e;
    if (bf16)
      e = sgemm<false, false, __nv_bfloat16>(B, c->dout[l], c->din[l], in, ld_in, c->pb + c->woff[l],
                                             c->dout[l], out, c->dout[l], c->pb + c->boff[l], mode, Z, s);
    else
      e = sgemm<false, false, float>(B, c->dout[l], c->din[l], in, ld_in, c->p + c->woff[l],
                                     c->dout[l], out, c->dout[l], c->p + c->boff[l], mode, Z, s);
    if (e != cudaSuccess) return hsc_fail(nullptr, HSC_ERR_CUDA, cudaGetErrorString(e));
    in = out;
    ld_in = c->dout[l];
  }
  return HSC_OK;
}

}  // namespace

extern "C" int hsc_mlp_create(hsc_mlp_t* out, int32_t n_in, int32_t width, int32_t hidden_layers,
                              int32_t n_out, int32_t max_batch) {
  if (!out || n_in <= 0 || width <= 0 || hidden_layers < 1 || n_out <= 0 || max_batch <= 0)
    return hsc_fail(nullptr, HSC_ERR_ARG, "bad MLP shape");
  *out = nullptr;
  auto* c = new hsc_mlp_ctx();
  c->n_in = n_in; c->width = width; c->hidden = hidden_layers; c->n_out = n_out;
  c->max_batch = max_batch;
  c->L = hidden_layers + 1;
  for (int l = 0; l < c->L; ++l) {
    c->din.push_back(l == 0 ? n_in : width);
    c->dout.push_back(l == c->L - 1 ? n_out : width);
    c->woff.push_back(c->np);
    c->np += (int64_t)c->din[l] * c->dout[l];
    c->boff.push_back(c->np);
    c->np += c->dout[l];
  }
  const int64_t act = (int64_t)max_batch * width * hidden_layers;
  bool ok = cudaMalloc(&c->p, c->np * 4) == cudaSuccess && cudaMalloc(&c->g, c->np * 4) == cudaSuccess &&
            cudaMalloc(&c->m, c->np * 4) == cudaSuccess && cudaMalloc(&c->v, c->np * 4) == cudaSuccess &&
            cudaMalloc(&c->pb, c->np * 2) == cudaSuccess && cudaMalloc(&c->Z, act * 4) == cudaSuccess &&
            cudaMalloc(&c->A, act * 4) == cudaSuccess &&
            cudaMalloc(&c->dA, (int64_t)max_batch * std::max(width, n_out) * 4) == cudaSuccess &&
            cudaMalloc(&c->dZ, (int64_t)max_batch * std::max(width, n_out) * 4) == cudaSuccess &&
            cudaMalloc(&c->y, (int64_t)max_batch * n_out * 4) == cudaSuccess &&
            cudaMalloc(&c->loss, 4) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    hsc_mlp_destroy(c);
    return hsc_fail(nullptr, HSC_ERR_OOM, "cudaMalloc MLP");
  }
  cudaMemset(c->p, 0, c->np * 4);
  cudaMemset(c->m, 0, c->np * 4);
  cudaMemset(c->v, 0, c->np * 4);
  *out = c;
  return HSC_OK;
}

extern "C" int hsc_mlp_num_params(hsc_mlp_t c, int64_t* n) {
  if (!c || !n) return hsc_fail(nullptr, HSC_ERR_ARG, "NULL argument");
  *n = c->np;
  return HSC_OK;
}

extern "C" int hsc_mlp_set_params(hsc_mlp_t c, const float* host) {
  if (!c || !host) return hsc_fail(nullptr, HSC_ERR_ARG, "NULL argument");
  if (cudaMemcpy(c->p, host, c->np * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(c->m, 0, c->np * 4) != cudaSuccess || cudaMemset(c->v, 0, c->np * 4) != cudaSuccess)
    return hsc_fail(nullptr, HSC_ERR_CUDA, "set params");
  c->step = 0;
  c->pb_valid = false;
  return HSC_OK;
}

extern "C" int hsc_mlp_get_params(hsc_mlp_t c, float* host) {
  if (!c || !host) return hsc_fail(nullptr, HSC_ERR_ARG, "NULL argument");
  if (cudaMemcpy(host, c->p, c->np * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return hsc_fail(nullptr, HSC_ERR_CUDA, "get params");
  return HSC_OK;
}

extern "C" int hsc_mlp_forward(hsc_mlp_t c, int32_t batch, const float* x, float* y, int32_t bf16,
                               void* stream) {
  if (!c || !x || !y || batch <= 0 || batch > c->max_batch) return hsc_fail(nullptr, HSC_ERR_ARG, "bad forward arguments");
  cudaStream_t s = (cudaStream_t)stream;
  if (bf16 && !c->pb_valid) {
    k_to_bf16<<<blocks(c->np), 256, 0, s>>>(c->np, c->p, c->pb);
    c->pb_valid = true;
  }
  return forward(c, batch, x, y, bf16 != 0, s);
}

extern "C" int hsc_mlp_loss_grad(hsc_mlp_t c, int32_t batch, const float* x, const float* t,
                                 float* loss_host, float* grad_host, void* stream) {
  if (!c || !x || !t || batch <= 0 || batch > c->max_batch) return hsc_fail(nullptr, HSC_ERR_ARG, "bad training arguments");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = forward(c, batch, x, c->y, false, s);
  if (rc != HSC_OK) return rc;
  const int B = batch, W = c->width;
  k_mse<<<1, 256, 0, s>>>(B * c->n_out, c->y, t, c->dZ, c->loss);
  // backward through layers L-1 .. 0 (dZ holds the gradient w.r.t. the layer's pre-activation)
  for (int l = c->L - 1; l >= 0; --l) {
    const float* Ain = l == 0 ? x : c->A + (int64_t)(l - 1) * c->max_batch * W;
    const int din = c->din[l], dout = c->dout[l];
    cudaError_t e = sgemm<true, false, float>(din, dout, B, Ain, din, c->dZ, dout, c->g + c->woff[l], dout,
                                              nullptr, 0, nullptr, s);
    if (e != cudaSuccess) return hsc_fail(nullptr, HSC_ERR_CUDA, cudaGetErrorString(e));
    k_colsum<<<blocks(dout), 256, 0, s>>>(B, dout, c->dZ, c->g + c->boff[l]);
    if (l > 0) {
      e = sgemm<false, true, float>(B, din, dout, c->dZ, dout, c->p + c->woff[l], dout, c->dA, din,
                                    nullptr, 0, nullptr, s);
      if (e != cudaSuccess) return hsc_fail(nullptr, HSC_ERR_CUDA, cudaGetErrorString(e));
      const float* Zp = c->Z + (int64_t)(l - 1) * c->max_batch * W;
      k_gelu_back<<<blocks((int64_t)B * din), 256, 0, s>>>((int64_t)B * din, c->dA, Zp, c->dZ);
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && loss_host) e = cudaMemcpyAsync(loss_host, c->loss, 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && grad_host) e = cudaMemcpyAsync(grad_host, c->g, c->np * 4, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && (loss_host || grad_host)) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return hsc_fail(nullptr, HSC_ERR_CUDA, cudaGetErrorString(e));
  return HSC_OK;
}

extern "C" int hsc_mlp_adam(hsc_mlp_t c, float lr, float beta1, float beta2, float eps, void* stream) {
  if (!c) return hsc_fail(nullptr, HSC_ERR_ARG, "NULL MLP");
  c->step += 1;
  const float c1 = 1.f - std::pow(beta1, (float)c->step), c2 = 1.f - std::pow(beta2, (float)c->step);
  k_adam<<<blocks(c->np), 256, 0, (cudaStream_t)stream>>>(c->np, c->p, c->g, c->m, c->v, lr, beta1, beta2,
                                                          eps, c1, c2);
  c->pb_valid = false;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return hsc_fail(nullptr, HSC_ERR_CUDA, cudaGetErrorString(e));
  return HSC_OK;
}

extern "C" int hsc_mlp_destroy(hsc_mlp_t c) {
  if (!c) return HSC_OK;
  for (void* q : {(void*)c->p, (void*)c->g, (void*)c->m, (void*)c->v, (void*)c->pb, (void*)c->Z,
                  (void*)c->A, (void*)c->dA, (void*)c->dZ, (void*)c->y, (void*)c->loss})
    if (q) cudaFree(q);
  delete c;
  return HSC_OK;
}
