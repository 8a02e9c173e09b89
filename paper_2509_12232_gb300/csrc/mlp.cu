// BF16 tensor-core MLP of the candidate-pose surrogate: 128 -> 256 -> 256 ->
// 256 -> 1 with GELU (erf form), BF16 weights and activations, FP32
// accumulation, FP32 master weights (Adam). Forward, backward and the
// optimiser step are this file's kernels.
//
// The dense layers run on one GEMM kernel, C = op(A) op(B) with FP32
// accumulation on mma.sync m16n8k16 BF16 tensor-core instructions, operand
// tiles staged in shared memory by cp.async and read with ldmatrix (the
// transposed form serves the weight-gradient products). CTA tile 128 x 128 x
// 32, 8 warps of 64 x 32, double-buffered. Epilogues: FP32 store; bias +
// GELU (FP32 pre-activation kept for the backward pass, BF16 activation);
// GELU backward (dZ = dH * gelu'(Z), BF16).
#include <cuda_bf16.h>

#include "mlp.h"

namespace dk {
namespace mlp {

namespace {
constexpr int BM = 128, BN = 128, BK = 32, NTHREADS = 256;

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N));
}

template <bool TRANS>
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void *p) {
  if (TRANS)
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
  else
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float gelu(float z) { return gelu_as(z); }
__device__ __forceinline__ float gelu_d(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) +
         z * 0.39894228040143268f * __expf(-0.5f * z * z);
}

// Shared tiles. A: [BM][BK+8] (K contiguous) or [BK][BM+8] (M contiguous);
// B: [BN][BK+8] (K contiguous) or [BK][BN+8] (N contiguous). Row strides of
// 80 or 272 bytes keep ldmatrix's eight 16-byte rows on distinct banks.
template <bool AT, bool BT>
struct Tiles {
  static constexpr int A_ELEMS = AT ? BK * (BM + 8) : BM * (BK + 8);
  static constexpr int B_ELEMS = BT ? BK * (BN + 8) : BN * (BK + 8);
  __nv_bfloat16 a[2][A_ELEMS];
  __nv_bfloat16 b[2][B_ELEMS];
};

// Load the (m0, n0, k0) tiles of A and B into buffer s (512 16-byte chunks
// each: two per thread).
template <bool AT, bool BT>
__device__ __forceinline__ void load_tiles(Tiles<AT, BT> &T, int s, const __nv_bfloat16 *A, int lda,
                                           const __nv_bfloat16 *B, int ldb, int m0, int n0, int k0) {
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int c = threadIdx.x + h * NTHREADS;
    if (!AT) {
      const int row = c >> 2, col = (c & 3) * 8;
      cp_async16(&T.a[s][row * (BK + 8) + col], A + (int64_t)(m0 + row) * lda + k0 + col);
    } else {
      const int row = c >> 4, col = (c & 15) * 8;
      cp_async16(&T.a[s][row * (BM + 8) + col], A + (int64_t)(k0 + row) * lda + m0 + col);
    }
    if (!BT) {
      const int row = c >> 2, col = (c & 3) * 8;
      cp_async16(&T.b[s][row * (BK + 8) + col], B + (int64_t)(n0 + row) * ldb + k0 + col);
    } else {
      const int row = c >> 4, col = (c & 15) * 8;
      cp_async16(&T.b[s][row * (BN + 8) + col], B + (int64_t)(k0 + row) * ldb + n0 + col);
    }
  }
}

// C[M x N] = op(A) op(B):
//   AT = false: A stored [M][K] (lda); AT = true: A stored [K][M]
//   BT = false: B stored [N][K] (ldb); BT = true: B stored [K][N]
// M, N multiples of 128, K of 32 (callers pad).
template <bool AT, bool BT, int EPI>
__global__ void __launch_bounds__(NTHREADS) gemm_kernel(const __nv_bfloat16 *__restrict__ A, int lda,
                                                        const __nv_bfloat16 *__restrict__ B, int ldb,
                                                        int K, Epilogue ep) {
  __shared__ __align__(128) Tiles<AT, BT> T;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  // split K: this CTA's K range starts at blockIdx.z * K
  const int64_t kz = (int64_t)blockIdx.z * K;
  A += AT ? kz * lda : kz;
  B += BT ? kz * ldb : kz;
  if (EPI == EPI_STORE_F32) ep.c32 += (int64_t)blockIdx.z * ep.split_stride;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = warp >> 2, wn = warp & 3;  // 2 x 4 warps, 64 x 32 each
  float acc[4][4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.0f;
  const int nk = K / BK;
  load_tiles<AT, BT>(T, 0, A, lda, B, ldb, m0, n0, 0);
  cp_commit();
  for (int kt = 0; kt < nk; ++kt) {
    const int s = kt & 1;
    if (kt + 1 < nk) {
      load_tiles<AT, BT>(T, s ^ 1, A, lda, B, ldb, m0, n0, (kt + 1) * BK);
      cp_commit();
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; kk += 16) {
      uint32_t a[4][4], b[2][4];
#pragma unroll
      for (int mi = 0; mi < 4; ++mi) {
        const int mb = wm * 64 + mi * 16;
        if (!AT)
          ldsm_x4<false>(a[mi], &T.a[s][(mb + (lane & 15)) * (BK + 8) + kk + (lane >> 4) * 8]);
        else
          ldsm_x4<true>(a[mi], &T.a[s][(kk + (lane >> 4) * 8 + (lane & 7)) * (BM + 8) + mb +
                                       ((lane >> 3) & 1) * 8]);
      }
#pragma unroll
      for (int nj = 0; nj < 2; ++nj) {
        const int nb = wn * 32 + nj * 16;
        if (!BT)
          ldsm_x4<false>(b[nj], &T.b[s][(nb + (lane & 7) + (lane >> 4) * 8) * (BK + 8) + kk +
                                        ((lane >> 3) & 1) * 8]);
        else
          ldsm_x4<true>(b[nj], &T.b[s][(kk + ((lane >> 3) & 1) * 8 + (lane & 7)) * (BN + 8) + nb +
                                       (lane >> 4) * 8]);
      }
#pragma unroll
      for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
          mma_bf16(acc[mi][ni], a[mi], b[ni >> 1][(ni & 1) * 2], b[ni >> 1][(ni & 1) * 2 + 1]);
    }
    __syncthreads();
  }
  // epilogue
  const int g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int mi = 0; mi < 4; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int m = m0 + wm * 64 + mi * 16 + g + h * 8;
        const int n = n0 + wn * 32 + ni * 8 + 2 * t;
        const float v0 = acc[mi][ni][2 * h], v1 = acc[mi][ni][2 * h + 1];
        const int64_t o = (int64_t)m * ep.ldc + n;
        if (EPI == EPI_STORE_F32) {
          *reinterpret_cast<float2 *>(ep.c32 + o) = make_float2(v0, v1);
        } else if (EPI == EPI_BIAS_GELU) {
          const float z0 = v0 + ep.bias[n], z1 = v1 + ep.bias[n + 1];
          if (ep.c32) *reinterpret_cast<float2 *>(ep.c32 + o) = make_float2(z0, z1);
          *reinterpret_cast<__nv_bfloat162 *>(ep.c16 + o) = __floats2bfloat162_rn(gelu(z0), gelu(z1));
        } else {  // EPI_GELU_BWD: dZ = dH * gelu'(Z)
          const float2 z = *reinterpret_cast<const float2 *>(ep.zin + o);
          *reinterpret_cast<__nv_bfloat162 *>(ep.c16 + o) =
              __floats2bfloat162_rn(v0 * gelu_d(z.x), v1 * gelu_d(z.y));
        }
      }
}

// y[m] = b + sum_j H[m][j] w[j] (the 256 -> 1 output layer; one warp per row).
__global__ void out_layer_kernel(const __nv_bfloat16 *H, const float *w, const float *b, int rows,
                                 float *y) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= rows) return;
  const __nv_bfloat16 *h = H + (int64_t)warp * HIDDEN;
  float s = 0.0f;
#pragma unroll
  for (int j = lane; j < HIDDEN; j += 32) s += __bfloat162float(h[j]) * w[j];
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) y[warp] = s + b[0];
}

// Output-layer backward: dy = 2 (y - t) / n (rows >= n: 0); dZ3 = dy w4 gelu'(Z3) (BF16);
// per-block partial sums of dW4 (H3^T dy), db4 and the loss.
__global__ void out_layer_bwd_kernel(const float *y, const float *t, int n, int rows,
                                     const __nv_bfloat16 *H3, const float *Z3, const float *w4,
                                     __nv_bfloat16 *dZ3, float *part /* [blocks][HIDDEN + 2] */) {
  const int j = threadIdx.x;  // blockDim == HIDDEN
  float dw = 0.0f, db = 0.0f, ls = 0.0f;
  for (int r = blockIdx.x; r < rows; r += gridDim.x) {
    const float e = r < n ? y[r] - t[r] : 0.0f;
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

__global__ void reduce_parts_kernel(const float *part, int blocks, int width, float *out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= width) return;
  float s = 0.0f;
  for (int b = 0; b < blocks; ++b) s += part[(int64_t)b * width + c];
  out[c] = s;
}

// Adam on FP32 masters: m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
// p -= lr * mhat / (sqrt(vhat) + eps).
__global__ void adam_kernel(float *p, float *m, float *v, const float *g, int n, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
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

template <bool AT, bool BT, int EPI>
static cudaError_t gemm(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb, int M,
                        int N, int K, const Epilogue &ep, cudaStream_t s, int splits = 1) {
  if (M % BM || N % BN || K % (BK * splits)) return cudaErrorInvalidValue;
  dim3 grid(N / BN, M / BM, splits);
  gemm_kernel<AT, BT, EPI><<<grid, NTHREADS, 0, s>>>(A, lda, B, ldb, K / splits, ep);
  return cudaGetLastError();
}

cudaError_t gemm_nt(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *Bt, int ldb, int M, int N,
                    int K, int epi, const Epilogue &ep, cudaStream_t s) {
  switch (epi) {
    case EPI_STORE_F32: return gemm<false, false, EPI_STORE_F32>(A, lda, Bt, ldb, M, N, K, ep, s);
    case EPI_BIAS_GELU: return gemm<false, false, EPI_BIAS_GELU>(A, lda, Bt, ldb, M, N, K, ep, s);
    case EPI_GELU_BWD: return gemm<false, false, EPI_GELU_BWD>(A, lda, Bt, ldb, M, N, K, ep, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t gemm_tt_f32(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *B, int ldb, int M,
                        int N, int K, float *C, float *scratch, int64_t scratch_elems,
                        cudaStream_t s) {
  Epilogue ep{};
  ep.ldc = N;
  // enough K splits to fill the GPU (about 128 CTAs), each a multiple of BK
  const int tiles = (M / BM) * (N / BN);
  int splits = 1;
  while (splits < 64 && tiles * splits < 128 && K % (BK * splits * 2) == 0 &&
         (int64_t)splits * 2 * M * N <= scratch_elems)
    splits *= 2;
  if (splits == 1) {
    ep.c32 = C;
    return gemm<true, true, EPI_STORE_F32>(A, lda, B, ldb, M, N, K, ep, s);
  }
  ep.c32 = scratch;
  ep.split_stride = (int64_t)M * N;
  cudaError_t e = gemm<true, true, EPI_STORE_F32>(A, lda, B, ldb, M, N, K, ep, s, splits);
  if (e != cudaSuccess) return e;
  reduce_parts_kernel<<<(M * N + 255) / 256, 256, 0, s>>>(scratch, splits, M * N, C);
  return cudaGetLastError();
}

cudaError_t out_layer(const __nv_bfloat16 *H, const float *w, const float *b, int rows, float *y,
                      cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  out_layer_kernel<<<(rows * 32 + 255) / 256, 256, 0, s>>>(H, w, b, rows, y);
  return cudaGetLastError();
}

cudaError_t out_layer_bwd(const float *y, const float *t, int n, int rows, const __nv_bfloat16 *H3,
                          const float *Z3, const float *w4, __nv_bfloat16 *dZ3, float *part,
                          int blocks, float *out /* [HIDDEN + 2] */, cudaStream_t s) {
  out_layer_bwd_kernel<<<blocks, HIDDEN, 0, s>>>(y, t, n, rows, H3, Z3, w4, dZ3, part);
  reduce_parts_kernel<<<(HIDDEN + 2 + 127) / 128, 128, 0, s>>>(part, blocks, HIDDEN + 2, out);
  return cudaGetLastError();
}

cudaError_t colsum(const __nv_bfloat16 *X, int rows, int cols, float *out, float *scratch,
                   cudaStream_t s) {
  if (rows <= 0) return cudaMemsetAsync(out, 0, sizeof(float) * cols, s);
  const int chunks = rows < 64 ? rows : 64;
  const int chunk_rows = (rows + chunks - 1) / chunks;
  colsum_part_kernel<<<chunks, 256, 0, s>>>(X, rows, cols, chunk_rows, scratch);
  reduce_parts_kernel<<<(cols + 255) / 256, 256, 0, s>>>(scratch, chunks, cols, out);
  return cudaGetLastError();
}

cudaError_t adam(float *p, float *m, float *v, const float *g, int n, float lr, int step,
                 cudaStream_t s) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  adam_kernel<<<(n + 255) / 256, 256, 0, s>>>(p, m, v, g, n, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t cast_weights(const float *W, int in, int out, __nv_bfloat16 *w16, __nv_bfloat16 *wt16,
                         cudaStream_t s) {
  cast_weights_kernel<<<(in * out + 255) / 256, 256, 0, s>>>(W, in, out, w16, wt16);
  return cudaGetLastError();
}

}  // namespace mlp
}  // namespace dk
