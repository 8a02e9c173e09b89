// Non-GEMM kernels of the candidate-pose surrogate MLP (128 -> 256 -> 256 ->
// 256 -> 1, GELU in tanh form, BF16 weights and activations, FP32 master
// weights): the 256 -> 1 output layer's backward pass (its forward is part of
// the last training product's epilogue), column sums for the bias gradients,
// the Adam step and the BF16 weight copies. The dense
// products of training and prediction run on the 5th-generation tensor cores
// (mlp_tc.cu).
#include <cuda_bf16.h>
#include <stdint.h>

#include "mlp.h"

namespace dk {
namespace mlp {

namespace {

__device__ __forceinline__ float gelu_d(float z) { return gelu_t_grad(z); }

// Output-layer backward: y = b4 + the partial dot products (g = 0..7 in
// order); dy = 2 (y - t) / n (rows >= n: 0); dZ3 = dy w4 gelu'(Z3) (BF16);
// per-block partial sums of dW4 (H3^T dy), db4 and the loss.
__global__ void out_layer_bwd_kernel(float *y, const float *ydot, const float *b4, const float *t,
                                     int n, int rows, const __nv_bfloat16 *H3, const float *Z3,
                                     const float *w4, __nv_bfloat16 *dZ3,
                                     float *part /* [blocks][HIDDEN + 2] */) {
  const int j = threadIdx.x;  // blockDim == HIDDEN
  float dw = 0.0f, db = 0.0f, ls = 0.0f;
  for (int r = blockIdx.x; r < rows; r += gridDim.x) {
    float sum = ydot[r];
#pragma unroll
    for (int g = 1; g < 8; ++g) sum += ydot[(int64_t)g * rows + r];
    const float yr = b4[0] + sum;
    if (j == 0) y[r] = yr;
    const float e = r < n ? yr - t[r] : 0.0f;
    const float dy = 2.0f * e / (float)n;
    const int64_t o = (int64_t)r * HIDDEN + j;
    dw += __bfloat162float(H3[o]) * dy;
    dZ3[o] = __float2bfloat16_rn(dy * w4[j] * gelu_d(Z3[o]));
    if (j == 0) {
      db += dy;
      ls += e * e;
    }
  }
  float *P = part + (int64_t)blockIdx.x * (HIDDEN + 2);
  P[j] = dw;
  if (j == 0) {
    P[HIDDEN] = db;
    P[HIDDEN + 1] = ls;
  }
}

// part[b][c] = sum of X[r][c] over the rows of chunk b (chunk_rows rows each).
__global__ void colsum_part_kernel(const __nv_bfloat16 *X, int rows, int cols, int chunk_rows,
                                   float *part) {
  const int b = blockIdx.x;
  for (int c = threadIdx.x; c < cols; c += blockDim.x) {
    float s = 0.0f;
    const int r1 = min(rows, (b + 1) * chunk_rows);
    for (int r = b * chunk_rows; r < r1; ++r) s += __bfloat162float(X[(int64_t)r * cols + c]);
    part[(int64_t)b * cols + c] = s;
  }
}

// sum over b of part[b][c], one warp per column: lane l adds parts l, l + 32,
// ... in order, then a fixed shuffle tree (the same sum every run); columns
// c < split go to out[c], the others to out2[c - split].
__global__ void reduce_cols_kernel(const float *part, int blocks, int width, float *out, int split,
                                   float *out2) {
  const int c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (c >= width) return;
  float s = 0.0f;
  for (int b = lane; b < blocks; b += 32) s += part[(int64_t)b * width + c];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) {
    if (c < split) out[c] = s;
    else out2[c - split] = s;
  }
}

// Adam on FP32 masters (Kingma & Ba 2015): m = b1 m + (1-b1) g; v = b2 v +
// (1-b2) g^2; p -= lr * mhat / (sqrt(vhat) + eps), mhat = m / (1 - b1^t),
// vhat = v / (1 - b2^t); t from step_dev when given (a graph-replayed step),
// else step.
// With copies (training): the updated W1..W3 are also written as their BF16
// copies w16 [in][out] and wt16 [out][in] (what cast_weights_kernel makes).
__device__ __forceinline__ void adam_one(float *p, float *m, float *v, const float *g, int i,
                                         float lr, float b1, float b2, float eps, float c1,
                                         float c2, const WeightCopies &wc) {
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  p[i] = pi;
  if (wc.w16[0] == nullptr) return;
  int l = -1, e = 0, in = 0;
  if (i >= OFF_W1 && i < OFF_W1 + FEATURES * HIDDEN) {
    l = 0; e = i - OFF_W1; in = FEATURES;
  } else if (i >= OFF_W2 && i < OFF_W2 + HIDDEN * HIDDEN) {
    l = 1; e = i - OFF_W2; in = HIDDEN;
  } else if (i >= OFF_W3 && i < OFF_W3 + HIDDEN * HIDDEN) {
    l = 2; e = i - OFF_W3; in = HIDDEN;
  }
  if (l < 0) return;
  const __nv_bfloat16 b = __float2bfloat16_rn(pi);
  wc.w16[l][e] = b;
  wc.wt16[l][(int64_t)(e % HIDDEN) * in + e / HIDDEN] = b;
}

__global__ void adam_kernel(float *p, float *m, float *v, const float *g, int n, float lr, float b1,
                            float b2, float eps, int step, int *step_dev, WeightCopies wc,
                            int64_t *r0_dev, int64_t batch, unsigned *ticket) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  // the bias corrections 1 - b^t, once per block
  __shared__ float s_c[2];
  if (threadIdx.x == 0) {
    const float t = (float)(step_dev ? *step_dev : step);
    s_c[0] = 1.0f - powf(b1, t);
    s_c[1] = 1.0f - powf(b2, t);
  }
  __syncthreads();
  if (i < n) adam_one(p, m, v, g, i, lr, b1, b2, eps, s_c[0], s_c[1], wc);
  if (r0_dev == nullptr) return;
  // the last block to finish (every block has read the step) advances the counters
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(ticket, 1u) == gridDim.x - 1) {
      *r0_dev += batch;
      *step_dev += 1;
      *ticket = 0u;
      __threadfence();
    }
  }
}

// BF16 copies of a weight matrix W [in][out]: w16 (same layout) and wt16 [out][in].
__global__ void cast_weights_kernel(const float *W, int in, int out, __nv_bfloat16 *w16,
                                    __nv_bfloat16 *wt16) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= in * out) return;
  const int r = i / out, c = i % out;
  const __nv_bfloat16 b = __float2bfloat16_rn(W[i]);
  w16[i] = b;
  wt16[(int64_t)c * in + r] = b;
}
}  // namespace

cudaError_t out_layer_bwd(float *y, const float *ydot, const float *b4, const float *t, int n,
                          int rows, const __nv_bfloat16 *H3, const float *Z3, const float *w4,
                          __nv_bfloat16 *dZ3, float *part, int blocks, float *grad, float *loss,
                          cudaStream_t s) {
  out_layer_bwd_kernel<<<blocks, HIDDEN, 0, s>>>(y, ydot, b4, t, n, rows, H3, Z3, w4, dZ3, part);
  reduce_cols_kernel<<<(HIDDEN + 2 + 7) / 8, 256, 0, s>>>(part, blocks, HIDDEN + 2, grad,
                                                          HIDDEN + 1, loss);
  return cudaGetLastError();
}

cudaError_t colsum(const __nv_bfloat16 *X, int rows, int cols, float *out, float *scratch,
                   cudaStream_t s) {
  if (rows <= 0) return cudaMemsetAsync(out, 0, sizeof(float) * cols, s);
  const int chunks = rows < kColsumChunks ? rows : kColsumChunks;
  const int chunk_rows = (rows + chunks - 1) / chunks;
  colsum_part_kernel<<<chunks, 256, 0, s>>>(X, rows, cols, chunk_rows, scratch);
  reduce_cols_kernel<<<(cols + 7) / 8, 256, 0, s>>>(scratch, chunks, cols, out, cols, nullptr);
  return cudaGetLastError();
}

cudaError_t adam(float *p, float *m, float *v, const float *g, int n, float lr, int step,
                 int *step_dev, const WeightCopies *copies, int64_t *r0_dev, int64_t batch,
                 unsigned *ticket, cudaStream_t s) {
  if (r0_dev && (!step_dev || !ticket)) return cudaErrorInvalidValue;
  adam_kernel<<<(n + 255) / 256, 256, 0, s>>>(p, m, v, g, n, lr, 0.9f, 0.999f, 1e-8f, step,
                                              step_dev, copies ? *copies : WeightCopies{}, r0_dev,
                                              batch, ticket);
  return cudaGetLastError();
}

cudaError_t cast_weights(const float *W, int in, int out, __nv_bfloat16 *w16, __nv_bfloat16 *wt16,
                         cudaStream_t s) {
  cast_weights_kernel<<<(in * out + 255) / 256, 256, 0, s>>>(W, in, out, w16, wt16);
  return cudaGetLastError();
}

}  // namespace mlp
}  // namespace dk
