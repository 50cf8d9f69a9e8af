// Learned surrogate of E(theta): MLP d_in -> w -> w -> 1 with SiLU, FP32
// master weights, BF16 GEMMs on the tensor cores (tcgen05, FP32 accumulate),
// last layer and all elementwise work in FP32, Adam in FP32.
//
// A training step (x: B x d_in, targets t) runs
//   Z1 = x W1^T + b1 (GEMM),  H1 = SiLU(Z1)          -- fused epilogue
//   Z2 = H1 W2^T + b2 (GEMM), H2 = SiLU(Z2)          -- fused epilogue
//   y  = H2 w3 + b3,  dy = 2 (y - t) / B             -- FP32
//   dZ2 = dy w3^T * SiLU'(Z2);  dW2 = dZ2^T H1 (GEMM over the batch)
//   dH1 = dZ2 W2 (GEMM);  dZ1 = dH1 * SiLU'(Z1);  dW1 = dZ1^T x (GEMM)
//   dx  = dZ1 W1 (GEMM, the input gradient = surrogate gradient of E)
// GEMM operands are kept K-major: the kernels that produce H1, dZ2, dZ1 and
// the BF16 copy of x also write transposed copies for the batch-contracted
// weight gradients, and the weights keep transposed BF16 copies.
#include <cuda_bf16.h>

#include <new>

#include "gemm_tc.cuh"
#include "tnmps_internal.h"

extern "C" tnmps_status tnmps_gemm_bf16_dev(int M, int N, int K, const uint16_t *A, int lda,
                                           const uint16_t *B, int ldb, float *C, int ldc,
                                           void *stream) {
  if (M < 0 || N < 0 || K < 0 || !A || !B || !C || (K % 8) || (lda % 8) || (ldb % 8) ||
      lda < K || ldb < K || ldc < N || ((uintptr_t)A & 15) || ((uintptr_t)B & 15))
    return TNMPS_ERR_ARG;
  tcg::Operands op{A, B, M, N, K, lda, ldb, nullptr};
  tcg::EpiStore epi{C, N, ldc};
  cudaError_t e = tcg::launch(op, epi, (cudaStream_t)stream);
  return e == cudaSuccess ? TNMPS_OK : TNMPS_ERR_CUDA;
}

namespace {

__device__ __forceinline__ uint16_t bf(float x) {
  return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}
__device__ __forceinline__ float sigm(float z) { return 1.0f / (1.0f + expf(-z)); }

// bias + SiLU epilogue: Z (FP32), H as BF16 row-major (ld w) and transposed
// (ld Bp), or H as FP32 (last hidden layer)
struct EpiBiasSilu {
  const float *bias;
  float *Z;
  uint16_t *Hh, *HTh;
  float *Hf;
  int N, Bp;
  __device__ void operator()(int row, int col, const float (&v)[32]) const {
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const int c = col + j;
      if (c < N) {
        const float z = v[j] + bias[c];
        const float h = z * sigm(z);
        Z[(int64_t)row * N + c] = z;
        if (Hh) Hh[(int64_t)row * N + c] = bf(h);
        if (HTh) HTh[(int64_t)c * Bp + row] = bf(h);
        if (Hf) Hf[(int64_t)row * N + c] = h;
      }
    }
  }
};

// x (B x d) -> BF16 copy (ld d) and transposed copy (d x Bp, zero columns >= B)
__global__ void k_x_bf16(const float *x, int B, int d, int Bp, uint16_t *xh, uint16_t *xTh) {
  const int64_t n = (int64_t)Bp * d;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / d), i = (int)(e - (int64_t)b * d);
    const float v = b < B ? x[e] : 0.0f;
    if (b < B) xh[e] = bf(v);
    xTh[(int64_t)i * Bp + b] = bf(v);
  }
}

// y = H2 w3 + b3 (warp per row)
__global__ void k_last(const float *H2, const float *w3, const float *b3, int B, int w, float *y) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= B) return;
  float s = 0;
  for (int i = lane; i < w; i += 32) s += H2[(int64_t)row * w + i] * w3[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) y[row] = s + b3[0];
}

// dy = 2 (y - t) / B  (t == nullptr: dy = 1, the input-gradient pass)
__global__ void k_dy(const float *y, const float *t, int B, float *dy, float *sq) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  if (t) {
    const float r = y[b] - t[b];
    dy[b] = 2.0f * r / (float)B;
    sq[b] = r * r;
  } else {
    dy[b] = 1.0f;
  }
}

// dZ2 = dy w3^T * SiLU'(Z2), rows >= B zero (transposed copy feeds the
// batch-contracted GEMM, which runs over Bp rows)
__global__ void k_dz2(const float *dy, const float *w3, const float *Z2, int B, int Bp, int w,
                      uint16_t *dZh, uint16_t *dZTh, float *dZf) {
  const int64_t n = (int64_t)Bp * w;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / w), i = (int)(e - (int64_t)b * w);
    float g = 0;
    if (b < B) {
      const float z = Z2[e], s = sigm(z);
      g = dy[b] * w3[i] * s * (1.0f + z * (1.0f - s));
      dZh[e] = bf(g);
      dZf[e] = g;
    }
    dZTh[(int64_t)i * Bp + b] = bf(g);
  }
}

// dZ1 = dH1 * SiLU'(Z1)
__global__ void k_dz1(const float *dH1, const float *Z1, int B, int Bp, int w, uint16_t *dZh,
                      uint16_t *dZTh, float *dZf) {
  const int64_t n = (int64_t)Bp * w;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / w), i = (int)(e - (int64_t)b * w);
    float g = 0;
    if (b < B) {
      const float z = Z1[e], s = sigm(z);
      g = dH1[e] * s * (1.0f + z * (1.0f - s));
      dZh[e] = bf(g);
      dZf[e] = g;
    }
    dZTh[(int64_t)i * Bp + b] = bf(g);
  }
}

// out[c] = sum_b A[b][c] * (s ? s[b] : 1), one block per column, fixed order
__global__ void k_colsum(const float *A, const float *s, int B, int ncol, float *out) {
  const int c = blockIdx.x;
  float acc = 0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) acc += A[(int64_t)b * ncol + c] * (s ? s[b] : 1.0f);
  __shared__ float red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    out[c] = t;
  }
}

// loss = mean of sq (single block, fixed order)
__global__ void k_mean(const float *sq, int B, float *loss) {
  float acc = 0;
  for (int b = threadIdx.x; b < B; b += blockDim.x) acc += sq[b];
  __shared__ float red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    loss[0] = t / (float)B;
  }
}

// BF16 copies of W1 (w x d), W1^T (d x w), W2 (w x w), W2^T
__global__ void k_refresh(const float *W1, const float *W2, int d, int w, uint16_t *W1h,
                          uint16_t *W1Th, uint16_t *W2h, uint16_t *W2Th) {
  const int n1 = w * d, n2 = w * w;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n1 + n2; e += gridDim.x * blockDim.x) {
    if (e < n1) {
      const int o = e / d, i = e - o * d;
      const uint16_t h = bf(W1[e]);
      W1h[e] = h;
      W1Th[(int64_t)i * w + o] = h;
    } else {
      const int f = e - n1, o = f / w, i = f - o * w;
      const uint16_t h = bf(W2[f]);
      W2h[f] = h;
      W2Th[(int64_t)i * w + o] = h;
    }
  }
}

__global__ void k_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const float gg = g[e];
    const float mm = b1 * m[e] + (1.0f - b1) * gg;
    const float vv = b2 * v[e] + (1.0f - b2) * gg * gg;
    m[e] = mm;
    v[e] = vv;
    p[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
  }
}

size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

struct tnmps_mlp {
  int d = 0, w = 0, maxB = 0, Bp = 0;
  int64_t np = 0;
  cudaStream_t stream = nullptr;
  char *arena = nullptr;
  float *params, *m, *v, *grad;
  float *W1, *b1, *W2, *b2, *w3, *b3;       // views into params
  float *gW1, *gb1, *gW2, *gb2, *gw3, *gb3; // views into grad
  uint16_t *W1h, *W1Th, *W2h, *W2Th, *xh, *xTh, *H1h, *H1Th, *dZ2h, *dZ2Th, *dZ1h, *dZ1Th;
  float *Z1, *Z2, *H2, *y, *dy, *sq, *dH1, *dZ2f, *dZ1f, *loss;
  uint32_t *err;  // device flag: a GEMM's bounded wait ran out
  std::string last_error;
};

namespace {

struct MlpLayout {
  size_t total;
  std::vector<size_t> off;
};

// sizes in bytes of every buffer, in a fixed order
std::vector<size_t> mlp_sizes(int d, int w, int maxB) {
  const size_t Bp = (size_t)((maxB + 127) / 128) * 128;
  const size_t np = (size_t)w * d + w + (size_t)w * w + w + w + 1;
  return {4 * np, 4 * np, 4 * np, 4 * np,                    // params, m, v, grad
          2 * (size_t)w * d, 2 * (size_t)w * d,              // W1h, W1Th
          2 * (size_t)w * w, 2 * (size_t)w * w,              // W2h, W2Th
          2 * Bp * d, 2 * Bp * d,                            // xh, xTh
          2 * Bp * w, 2 * Bp * w,                            // H1h, H1Th
          2 * Bp * w, 2 * Bp * w, 2 * Bp * w, 2 * Bp * w,    // dZ2h, dZ2Th, dZ1h, dZ1Th
          4 * Bp * w, 4 * Bp * w, 4 * Bp * w,                // Z1, Z2, H2
          4 * Bp, 4 * Bp, 4 * Bp,                            // y, dy, sq
          4 * Bp * w, 4 * Bp * w, 4 * Bp * w, 256, 256};     // dH1, dZ2f, dZ1f, loss, err
}

cudaError_t run_forward(tnmps_mlp *m, const float *x, int B) {
  cudaStream_t s = m->stream;
  const int d = m->d, w = m->w;
  k_x_bf16<<<592, 256, 0, s>>>(x, B, d, m->Bp, m->xh, m->xTh);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  tcg::Operands o1{m->xh, m->W1h, B, w, d, d, d, m->err};
  EpiBiasSilu e1{m->b1, m->Z1, m->H1h, m->H1Th, nullptr, w, m->Bp};
  if ((e = tcg::launch(o1, e1, s)) != cudaSuccess) return e;
  tcg::Operands o2{m->H1h, m->W2h, B, w, w, w, w, m->err};
  EpiBiasSilu e2{m->b2, m->Z2, nullptr, nullptr, m->H2, w, m->Bp};
  if ((e = tcg::launch(o2, e2, s)) != cudaSuccess) return e;
  k_last<<<(B + 7) / 8, 256, 0, s>>>(m->H2, m->w3, m->b3, B, w, m->y);
  return cudaGetLastError();
}

// backward through the whole network; t == nullptr: dy = 1 (input gradient)
cudaError_t run_backward(tnmps_mlp *m, const float *t, int B, bool want_params, float *gx) {
  cudaStream_t s = m->stream;
  const int d = m->d, w = m->w, Bp = m->Bp;
  cudaError_t e;
  k_dy<<<(B + 255) / 256, 256, 0, s>>>(m->y, t, B, m->dy, m->sq);
  k_dz2<<<592, 256, 0, s>>>(m->dy, m->w3, m->Z2, B, Bp, w, m->dZ2h, m->dZ2Th, m->dZ2f);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (want_params) {
    k_colsum<<<w, 256, 0, s>>>(m->H2, m->dy, B, w, m->gw3);  // dw3 = H2^T dy
    k_colsum<<<1, 256, 0, s>>>(m->dy, nullptr, B, 1, m->gb3);
    k_colsum<<<w, 256, 0, s>>>(m->dZ2f, nullptr, B, w, m->gb2);
    tcg::Operands og{m->dZ2Th, m->H1Th, w, w, Bp, Bp, Bp, m->err};  // dW2 = dZ2^T H1
    tcg::EpiStore eg{m->gW2, w, w};
    if ((e = tcg::launch(og, eg, s)) != cudaSuccess) return e;
  }
  tcg::Operands oh{m->dZ2h, m->W2Th, B, w, w, w, w, m->err};  // dH1 = dZ2 W2
  tcg::EpiStore eh{m->dH1, w, w};
  if ((e = tcg::launch(oh, eh, s)) != cudaSuccess) return e;
  k_dz1<<<592, 256, 0, s>>>(m->dH1, m->Z1, B, Bp, w, m->dZ1h, m->dZ1Th, m->dZ1f);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (want_params) {
    k_colsum<<<w, 256, 0, s>>>(m->dZ1f, nullptr, B, w, m->gb1);
    tcg::Operands o1{m->dZ1Th, m->xTh, w, d, Bp, Bp, Bp, m->err};  // dW1 = dZ1^T x
    tcg::EpiStore e1{m->gW1, d, d};
    if ((e = tcg::launch(o1, e1, s)) != cudaSuccess) return e;
    if (t) k_mean<<<1, 256, 0, s>>>(m->sq, B, m->loss);
  }
  if (gx) {
    tcg::Operands ox{m->dZ1h, m->W1Th, B, d, w, w, w, m->err};  // dx = dZ1 W1
    tcg::EpiStore ex{gx, d, d};
    if ((e = tcg::launch(ox, ex, s)) != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

tnmps_status mfail(tnmps_mlp *m, cudaError_t e, const char *where) {
  m->last_error = std::string(where) + ": " + cudaGetErrorString(e);
  return TNMPS_ERR_CUDA;
}

}  // namespace

extern "C" {

size_t tnmps_mlp_bytes(int d_in, int width, int max_batch) {
  if (d_in < 8 || d_in % 8 || width < 8 || width % 8 || max_batch < 1) return 0;
  size_t t = 0;
  for (size_t sz : mlp_sizes(d_in, width, max_batch)) t = al(t + sz);
  return t;
}

int64_t tnmps_mlp_num_params(int d_in, int width) {
  return (int64_t)width * d_in + width + (int64_t)width * width + width + width + 1;
}

tnmps_status tnmps_mlp_init(tnmps_mlp **out, int d_in, int width, int max_batch, void *arena,
                            size_t bytes) {
  if (!out) return TNMPS_ERR_ARG;
  *out = nullptr;
  const size_t need = tnmps_mlp_bytes(d_in, width, max_batch);
  if (!need || !arena || ((uintptr_t)arena & 255)) return TNMPS_ERR_ARG;
  if (bytes < need) return TNMPS_ERR_NOMEM;
  tnmps_mlp *m = new (std::nothrow) tnmps_mlp();
  if (!m) return TNMPS_ERR_NOMEM;
  m->d = d_in;
  m->w = width;
  m->maxB = max_batch;
  m->Bp = ((max_batch + 127) / 128) * 128;
  m->np = tnmps_mlp_num_params(d_in, width);
  m->arena = (char *)arena;
  std::vector<char *> p;
  size_t o = 0;
  for (size_t sz : mlp_sizes(d_in, width, max_batch)) {
    p.push_back(m->arena + o);
    o = al(o + sz);
  }
  int i = 0;
  m->params = (float *)p[i++];
  m->m = (float *)p[i++];
  m->v = (float *)p[i++];
  m->grad = (float *)p[i++];
  m->W1h = (uint16_t *)p[i++];
  m->W1Th = (uint16_t *)p[i++];
  m->W2h = (uint16_t *)p[i++];
  m->W2Th = (uint16_t *)p[i++];
  m->xh = (uint16_t *)p[i++];
  m->xTh = (uint16_t *)p[i++];
  m->H1h = (uint16_t *)p[i++];
  m->H1Th = (uint16_t *)p[i++];
  m->dZ2h = (uint16_t *)p[i++];
  m->dZ2Th = (uint16_t *)p[i++];
  m->dZ1h = (uint16_t *)p[i++];
  m->dZ1Th = (uint16_t *)p[i++];
  m->Z1 = (float *)p[i++];
  m->Z2 = (float *)p[i++];
  m->H2 = (float *)p[i++];
  m->y = (float *)p[i++];
  m->dy = (float *)p[i++];
  m->sq = (float *)p[i++];
  m->dH1 = (float *)p[i++];
  m->dZ2f = (float *)p[i++];
  m->dZ1f = (float *)p[i++];
  m->loss = (float *)p[i++];
  m->err = (uint32_t *)p[i++];
  if (cudaMemset(m->err, 0, 4) != cudaSuccess) {
    delete m;
    return TNMPS_ERR_CUDA;
  }
  const int d = d_in, w = width;
  auto views = [&](float *base, float **W1, float **b1, float **W2, float **b2, float **w3,
                   float **b3) {
    *W1 = base;
    *b1 = *W1 + (int64_t)w * d;
    *W2 = *b1 + w;
    *b2 = *W2 + (int64_t)w * w;
    *w3 = *b2 + w;
    *b3 = *w3 + w;
  };
  views(m->params, &m->W1, &m->b1, &m->W2, &m->b2, &m->w3, &m->b3);
  views(m->grad, &m->gW1, &m->gb1, &m->gW2, &m->gb2, &m->gw3, &m->gb3);
  cudaError_t e = cudaMemsetAsync(m->arena, 0, need, m->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(m->stream);
  if (e != cudaSuccess) {
    delete m;
    return TNMPS_ERR_CUDA;
  }
  *out = m;
  return TNMPS_OK;
}

void tnmps_mlp_free(tnmps_mlp *m) { delete m; }

tnmps_status tnmps_mlp_set_stream(tnmps_mlp *m, void *stream) {
  if (!m) return TNMPS_ERR_ARG;
  m->stream = (cudaStream_t)stream;
  return TNMPS_OK;
}

tnmps_status tnmps_mlp_check(tnmps_mlp *m) {
  if (!m) return TNMPS_ERR_ARG;
  cudaError_t e = cudaStreamSynchronize(m->stream);
  uint32_t flags = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&flags, m->err, 4, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return mfail(m, e, "check");
  if (flags & TNMPS_EFLAG_TIMEOUT) {
    cudaMemset(m->err, 0, 4);
    m->last_error = "a tensor-core GEMM wait ran out; results since the last check are invalid";
    return TNMPS_ERR_TIMEOUT;
  }
  return TNMPS_OK;
}

const char *tnmps_mlp_last_error(const tnmps_mlp *m) {
  return m ? m->last_error.c_str() : "null surrogate";
}

tnmps_status tnmps_mlp_set_params(tnmps_mlp *m, const float *params_dev) {
  if (!m || !params_dev) return TNMPS_ERR_ARG;
  cudaError_t e = cudaMemcpyAsync(m->params, params_dev, 4 * (size_t)m->np,
                                  cudaMemcpyDeviceToDevice, m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->m, 0, 4 * (size_t)m->np, m->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(m->v, 0, 4 * (size_t)m->np, m->stream);
  if (e != cudaSuccess) return mfail(m, e, "set params");
  k_refresh<<<148, 256, 0, m->stream>>>(m->W1, m->W2, m->d, m->w, m->W1h, m->W1Th, m->W2h,
                                         m->W2Th);
  e = cudaGetLastError();
  return e == cudaSuccess ? TNMPS_OK : mfail(m, e, "refresh");
}

tnmps_status tnmps_mlp_get_params(tnmps_mlp *m, float *params_dev) {
  if (!m || !params_dev) return TNMPS_ERR_ARG;
  cudaError_t e = cudaMemcpyAsync(params_dev, m->params, 4 * (size_t)m->np,
                                  cudaMemcpyDeviceToDevice, m->stream);
  return e == cudaSuccess ? TNMPS_OK : mfail(m, e, "get params");
}

tnmps_status tnmps_mlp_forward(tnmps_mlp *m, const float *x_dev, int B, float *y_dev) {
  if (!m || !x_dev || !y_dev || B < 1 || B > m->maxB) return TNMPS_ERR_ARG;
  cudaError_t e = run_forward(m, x_dev, B);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(y_dev, m->y, 4 * (size_t)B, cudaMemcpyDeviceToDevice, m->stream);
  return e == cudaSuccess ? TNMPS_OK : mfail(m, e, "forward");
}

tnmps_status tnmps_mlp_backward(tnmps_mlp *m, const float *x_dev, const float *target_dev, int B,
                                float *y_dev, float *loss_dev, float *grad_params_dev,
                                float *grad_x_dev) {
  if (!m || !x_dev || B < 1 || B > m->maxB) return TNMPS_ERR_ARG;
  cudaError_t e = run_forward(m, x_dev, B);
  const bool want = target_dev != nullptr || grad_params_dev != nullptr;
  if (e == cudaSuccess) e = run_backward(m, target_dev, B, want, grad_x_dev);
  if (e == cudaSuccess && y_dev)
    e = cudaMemcpyAsync(y_dev, m->y, 4 * (size_t)B, cudaMemcpyDeviceToDevice, m->stream);
  if (e == cudaSuccess && loss_dev && target_dev)
    e = cudaMemcpyAsync(loss_dev, m->loss, 4, cudaMemcpyDeviceToDevice, m->stream);
  if (e == cudaSuccess && grad_params_dev && want)
    e = cudaMemcpyAsync(grad_params_dev, m->grad, 4 * (size_t)m->np, cudaMemcpyDeviceToDevice,
                        m->stream);
  return e == cudaSuccess ? TNMPS_OK : mfail(m, e, "backward");
}

tnmps_status tnmps_mlp_train_step(tnmps_mlp *m, const float *x_dev, const float *target_dev,
                                  int B, float lr, int step, float *loss_dev) {
  if (!m || !x_dev || !target_dev || B < 1 || B > m->maxB || step < 1) return TNMPS_ERR_ARG;
  cudaError_t e = run_forward(m, x_dev, B);
  if (e == cudaSuccess) e = run_backward(m, target_dev, B, true, nullptr);
  if (e != cudaSuccess) return mfail(m, e, "train step");
  const float b1 = 0.9f, b2 = 0.999f;
  k_adam<<<592, 256, 0, m->stream>>>(m->params, m->grad, m->m, m->v, m->np, lr, b1, b2, 1e-8f,
                                      1.0f - powf(b1, (float)step), 1.0f - powf(b2, (float)step));
  k_refresh<<<148, 256, 0, m->stream>>>(m->W1, m->W2, m->d, m->w, m->W1h, m->W1Th, m->W2h,
                                         m->W2Th);
  if (loss_dev) cudaMemcpyAsync(loss_dev, m->loss, 4, cudaMemcpyDeviceToDevice, m->stream);
  e = cudaGetLastError();
  return e == cudaSuccess ? TNMPS_OK : mfail(m, e, "adam");
}

}  // extern "C"
