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

// GELU in its tanh form (Hendrycks & Gimpel 2016): z (1 + tanh(u)) / 2 with
// u = sqrt(2 / pi) (z + 0.044715 z^3), the tanh on the special-function unit
// (tanh.approx.f32, relative error below 2^-11). Against the exact erf form
// z (1 + erf(z / sqrt 2)) / 2 it differs by at most 4.7e-4 (at z = 2.7,
// where GELU = 2.69) and by 2.2e-3 relative where |GELU| > 0.1: under the
// BF16 rounding of the activations it feeds (2^-8 relative). Training and
// prediction use this one definition; the FP64 reference keeps the erf form.
__device__ __forceinline__ float tanh_sfu(float x) {
  float y;
  asm("tanh.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
constexpr float kGeluC0 = 0.7978845608028654f;    // sqrt(2 / pi)
constexpr float kGeluC1 = 0.035677408136300125f;  // 0.044715 sqrt(2 / pi)
constexpr float kGeluD1 = 0.10703222440890037f;   // 3 x 0.044715 sqrt(2 / pi)
__device__ __forceinline__ float gelu_t(float z) {
  const float u = z * fmaf(kGeluC1, z * z, kGeluC0);
  const float h = 0.5f * z;
  return fmaf(h, tanh_sfu(u), h);
}

// d gelu_t / dz = (1 + t) / 2 + z (1 - t^2) u' / 2, t = tanh(u),
// u' = sqrt(2 / pi) (1 + 3 x 0.044715 z^2) (the backward pass of training).
__device__ __forceinline__ float gelu_t_grad(float z) {
  const float z2 = z * z;
  const float t = tanh_sfu(z * fmaf(kGeluC1, z2, kGeluC0));
  const float du = fmaf(kGeluD1, z2, kGeluC0);
  return fmaf(0.5f * z * du, fmaf(-t, t, 1.0f), 0.5f * (1.0f + t));
}

struct Epilogue {
  float *c32;               // FP32 output (STORE) or pre-activation cache (BIAS_GELU), or null
  __nv_bfloat16 *c16;       // BF16 output (BIAS_GELU: activation; GELU_BWD: dZ)
  const float *bias;        // BIAS_GELU
  const float *zin;         // GELU_BWD: pre-activations
  int ldc;
  int64_t split_stride;     // STORE with split K: elements between the splits' partial outputs
  __nv_bfloat16 *c16t;      // BIAS_GELU / GELU_BWD, or null: c16 transposed, [col][row]
  int64_t ldt;              // row stride of c16t (elements)
  // BIAS_GELU, or null: ydot[g][row] = sum over the 32 columns of group g of the
  // BF16 activation times w4 (the output layer's partial dot products, g < 8)
  float *ydot;
  const float *w4;
  int64_t ldy;
};

// Output-layer backward. y = b4 + the eight partial dot products ydot[g][row]
// (summed in order g = 0..7; y is written); dy = 2 (y - t) / n; dZ3 = dy w4
// gelu'(Z3); dW4, db4 into grad[0..256] and the summed squared error into
// *loss (fixed-order reductions over `blocks` partials in part).
cudaError_t out_layer_bwd(float *y, const float *ydot, const float *b4, const float *t, int n,
                          int rows, const __nv_bfloat16 *H3, const float *Z3, const float *w4,
                          __nv_bfloat16 *dZ3, float *part, int blocks, float *grad, float *loss,
                          cudaStream_t s);
// out[c] = sum over rows of X[r][c]: kColsumChunks row chunks in parallel, then a
// fixed-order sum (scratch: at least kColsumChunks * cols floats).
constexpr int kColsumChunks = 128;
cudaError_t colsum(const __nv_bfloat16 *X, int rows, int cols, float *out, float *scratch,
                   cudaStream_t s);
// BF16 copies of W1..W3 that the training products read: w16[l] [in][out], wt16[l] [out][in].
struct WeightCopies {
  __nv_bfloat16 *w16[3] = {nullptr, nullptr, nullptr};
  __nv_bfloat16 *wt16[3] = {nullptr, nullptr, nullptr};
};
// Adam step t = *step_dev if step_dev is given (read on the device), else step;
// with copies, the updated W1..W3 are also written to them (one kernel).
// With counters (r0_dev, batch), the last block to finish also advances the
// batch start and the step (the form replayed in the training graph).
cudaError_t adam(float *p, float *m, float *v, const float *g, int n, float lr, int step,
                 int *step_dev, const WeightCopies *copies, int64_t *r0_dev, int64_t batch,
                 unsigned *ticket, cudaStream_t s);
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
// C (FP32 [M][256]) = A^T B (the weight gradients) from K-major copies of
// the operands, at [M][K] (A^T) and bt [256][K] (B^T): K split over CTAs with
// FP32 partials in scratch (split x M x 256 floats, split <= scratch_elems /
// (M 256)) summed in a fixed order.
cudaError_t tc_gemm_tt_f32(const __nv_bfloat16 *at, const __nv_bfloat16 *bt, int M, int K, float *C,
                           float *scratch, int64_t scratch_elems, int *err, cudaStream_t s);
// out[c][r] = in[r][c] for in [rows][cols] BF16.
cudaError_t transpose_bf16(const __nv_bfloat16 *in, int rows, int cols, __nv_bfloat16 *out,
                           cudaStream_t s);

}  // namespace mlp
}  // namespace dk
