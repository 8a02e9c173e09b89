// Kernels of the BF16 surrogate MLP (mlp.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dk {
namespace mlp {

constexpr int FEATURES = 128, HIDDEN = 256;
// Packed FP32 parameters: W1[128][256], b1[256], W2[256][256], b2[256],
// W3[256][256], b3[256], W4[256], b4[1] (W stored [in][out]).
constexpr int OFF_W1 = 0;
constexpr int OFF_B1 = OFF_W1 + FEATURES * HIDDEN;
constexpr int OFF_W2 = OFF_B1 + HIDDEN;
constexpr int OFF_B2 = OFF_W2 + HIDDEN * HIDDEN;
constexpr int OFF_W3 = OFF_B2 + HIDDEN;
constexpr int OFF_B3 = OFF_W3 + HIDDEN * HIDDEN;
constexpr int OFF_W4 = OFF_B3 + HIDDEN;
constexpr int OFF_B4 = OFF_W4 + HIDDEN;
constexpr int N_PARAMS = OFF_B4 + 1;

enum { EPI_STORE_F32 = 0, EPI_BIAS_GELU = 1, EPI_GELU_BWD = 2 };

// GELU(z) = z Phi(z) = (z + |z| erf(|z| / sqrt 2)) / 2 with erf from Abramowitz &
// Stegun, Handbook of Mathematical Functions, eq. 7.1.28: erf(x) = 1 - (1 + a1 x
// + ... + a6 x^6)^-16 for x >= 0, |error| <= 3e-7 (one reciprocal, four squarings).
__device__ __forceinline__ float gelu_as(float z) {
  const float x = fabsf(z) * 0.70710678118654752f;
  float p = fmaf(4.30638e-5f, x, 2.765672e-4f);
  p = fmaf(p, x, 1.520143e-4f);
  p = fmaf(p, x, 9.2705272e-3f);
  p = fmaf(p, x, 4.22820123e-2f);
  p = fmaf(p, x, 7.05230784e-2f);
  p = fmaf(p, x, 1.0f);
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(p));
  r *= r;
  r *= r;
  r *= r;
  r *= r;  // p^-16
  return 0.5f * fmaf(fabsf(z), 1.0f - r, z);
}

// d GELU / dz with the exact erf (the backward pass of every training path).
__device__ __forceinline__ float gelu_grad(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) +
         z * 0.39894228040143268f * __expf(-0.5f * z * z);
}

struct Epilogue {
  float *c32;               // FP32 output (STORE) or pre-activation cache (BIAS_GELU), or null
  __nv_bfloat16 *c16;       // BF16 output (BIAS_GELU: activation; GELU_BWD: dZ)
  const float *bias;        // BIAS_GELU
  const float *zin;         // GELU_BWD: pre-activations
  int ldc;
  int64_t split_stride;     // STORE with split K: elements between the splits' partial outputs
};

cudaError_t out_layer(const __nv_bfloat16 *H, const float *w, const float *b, int rows, float *y,
                      cudaStream_t s);
cudaError_t out_layer_bwd(const float *y, const float *t, int n, int rows, const __nv_bfloat16 *H3,
                          const float *Z3, const float *w4, __nv_bfloat16 *dZ3, float *part,
                          int blocks, float *out, cudaStream_t s);
// out[c] = sum over rows of X[r][c]: row chunks in parallel, then a fixed-order sum
// (scratch: at least 64 * cols floats).
cudaError_t colsum(const __nv_bfloat16 *X, int rows, int cols, float *out, float *scratch,
                   cudaStream_t s);
// Adam step t = *step_dev if step_dev is given (read on the device), else step.
cudaError_t adam(float *p, float *m, float *v, const float *g, int n, float lr, int step,
                 const int *step_dev, cudaStream_t s);
cudaError_t cast_weights(const float *W, int in, int out, __nv_bfloat16 *w16, __nv_bfloat16 *wt16,
                         cudaStream_t s);

// Fused forward pass on the tensor cores (mlp_tc.cu): y[r] for rows r < n of
// X [n][128] (BF16, 16-byte aligned rows), weights wc in the tensor-core
// layout (canon_weights, canon_weight_elems() BF16 values), biases and w4,
// b4 from the packed FP32 parameters. A device-side wait that runs out sets
// *err = 1 and leaves the rows of the skipped tiles untouched.
cudaError_t canon_weights(const float *p, __nv_bfloat16 *wc, cudaStream_t s);
int canon_weight_elems();
cudaError_t fused_forward(const __nv_bfloat16 *X, int64_t n, const __nv_bfloat16 *wc,
                          const float *params, float *y, int *err, cudaStream_t s);

// Training products on the tensor cores (tcgen05, FP32 accumulator in tensor
// memory; mlp_tc.cu). C = A Bt^T with A [M][K] and Bt [256][K] BF16,
// K-major rows (lda, ldb elements, 16-byte aligned), M a multiple of 128, K
// of 64; the epilogues of gemm_nt (bias + GELU, GELU backward, FP32 store).
// *err is set if a device wait runs out (the output is then incomplete).
cudaError_t tc_gemm_nt(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *Bt, int ldb, int M,
                       int K, int epi, const Epilogue &ep, int *err, cudaStream_t s);
// C (FP32 [M][256]) = A^T B for A stored [K][M] and B stored [K][256] (the
// weight gradients): both transposed to K-major copies (at and bt, M x K and
// 256 x K BF16), K split over CTAs with FP32 partials in scratch (split x M x
// 256 floats, split <= scratch_elems / (M 256)) summed in a fixed order.
cudaError_t tc_gemm_tn_f32(const __nv_bfloat16 *A, int M, const __nv_bfloat16 *B, int K, float *C,
                           __nv_bfloat16 *at, __nv_bfloat16 *bt, float *scratch,
                           int64_t scratch_elems, int *err, cudaStream_t s);

}  // namespace mlp
}  // namespace dk
