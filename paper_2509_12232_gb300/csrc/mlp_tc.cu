// Fused forward pass of the surrogate MLP (128 -> 256 -> 256 -> 256 -> 1,
// erf-GELU after the hidden layers) on the 5th-generation tensor cores.
//
// One persistent CTA per SM (8 warps) takes tiles of 128 feature rows:
//   - the tile is stored in shared memory in the K-major "core matrix" layout
//     the tensor core reads without swizzling (8 rows x 16 bytes per 128-byte
//     block, blocks ordered by row group then by K);
//   - each layer's BF16 weights, kept in global memory in that same layout,
//     arrive by bulk asynchronous copies that complete on an mbarrier (the
//     next layer's copy runs during the current layer's epilogue);
//   - one thread issues tcgen05.mma (M = 128, N = 256, K = 16 per instruction)
//     into a 256-column FP32 accumulator in tensor memory and commits it to an
//     mbarrier;
//   - the 16 warps drain the accumulator, warp w reading lanes 32 (w mod 4) ..
//     + 31 (the lane quarter its position in the warp group may access) and
//     columns 64 (w / 4) .. + 63 with tcgen05.ld; they add the bias, apply
//     GELU, round to BF16 and store the activations in the same layout as the
//     next layer's A operand; after the third layer each thread forms a
//     quarter of its row's output (a dot product with the FP32 w4) and the
//     quarters are added. Four warps per scheduler keep the epilogue, the
//     kernel's longest phase, issuing while some wait on their loads.
// Every mbarrier wait is bounded (one second of globaltimer); a timeout sets
// *err, skips the rest of the CTA's tiles (the caller fills the output with
// NaN beforehand) and releases the tensor memory after waiting, again
// bounded, for the copies and products in flight.
#include <cuda_bf16.h>
#include <stdint.h>

#include "mlp.h"

namespace dk {
namespace mlp {

namespace {

constexpr int TM = 128;        // rows per tile (MMA M)
constexpr int kThreads = 512;  // warp w: accumulator lanes 32 (w mod 4) .., columns 64 (w / 4) ..
constexpr int kParts = kThreads / 128;  // column quarters of a row
constexpr int XH_BYTES = TM * HIDDEN * 2;       // feature tile (32 KB) or hidden tile (64 KB)
constexpr int W_BYTES = HIDDEN * HIDDEN * 2;    // one layer's weights (at most 128 KB)
constexpr int SMEM_BYTES = XH_BYTES + W_BYTES + 64 + (kParts - 1) * TM * 4 + 4 * HIDDEN * 4;
// + output partial sums of quarters 1-3, biases b1..b3 and w4
constexpr int WC_L2 = HIDDEN * FEATURES;        // element offsets of layers 2, 3 in the weights
constexpr int WC_L3 = WC_L2 + HIDDEN * HIDDEN;
constexpr int kCopyChunk = 16384;               // bytes per bulk copy
constexpr uint64_t kWaitNs = 1000000000ull;     // bound of every mbarrier wait

// Byte offset of element (r, k) of an R x K BF16 operand in the K-major
// core-matrix layout: 128-byte blocks of 8 rows x 8 elements, block (r / 8,
// k / 8) at ((r / 8) * (K / 8) + k / 8) * 128.
__host__ __device__ constexpr uint32_t canon_off(int r, int k, int K) {
  return (uint32_t)((((r >> 3) * (K >> 3) + (k >> 3)) << 7) + ((r & 7) << 4) + ((k & 7) << 1));
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

// Waits for the completion of the mbarrier phase with parity ph; false after
// kWaitNs without it.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t ph) {
  const uint64_t t0 = gtimer();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(ph)
        : "memory");
    if (done) return true;
    if (gtimer() - t0 > kWaitNs) return false;
  }
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
// generic-proxy shared-memory writes made visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Shared-memory operand descriptor, no swizzling: start address, the byte
// distance between core matrices adjacent in K (leading) and in M/N
// (stride), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N / 8 and M / 16.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}

// Issue a read of 32 consecutive accumulator columns of this thread's lane;
// the registers are valid after tmem_wait on them.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
}

// Wait for this thread's accumulator reads; ties r to the wait so that no use
// of it is scheduled before.
__device__ __forceinline__ void tmem_wait(uint32_t (&r)[32]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                 "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]),
                 "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]),
                 "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]),
                 "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]),
                 "+r"(r[30]), "+r"(r[31])
               :
               : "memory");
}

// gelu_as (mlp.h) on two activations with packed two-wide FP32 arithmetic (the same
// operations in the same order, one instruction for both lanes of a pair).
__device__ __forceinline__ float2 gelu2(float2 z) {
  const float2 az = make_float2(fabsf(z.x), fabsf(z.y));
  const float2 x = __fmul2_rn(az, make_float2(0.70710678118654752f, 0.70710678118654752f));
  float2 p = __ffma2_rn(make_float2(4.30638e-5f, 4.30638e-5f), x,
                        make_float2(2.765672e-4f, 2.765672e-4f));
  p = __ffma2_rn(p, x, make_float2(1.520143e-4f, 1.520143e-4f));
  p = __ffma2_rn(p, x, make_float2(9.2705272e-3f, 9.2705272e-3f));
  p = __ffma2_rn(p, x, make_float2(4.22820123e-2f, 4.22820123e-2f));
  p = __ffma2_rn(p, x, make_float2(7.05230784e-2f, 7.05230784e-2f));
  p = __ffma2_rn(p, x, make_float2(1.0f, 1.0f));
  float2 r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.x) : "f"(p.x));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.y) : "f"(p.y));
  r = __fmul2_rn(r, r);
  r = __fmul2_rn(r, r);
  r = __fmul2_rn(r, r);
  r = __fmul2_rn(r, r);  // p^-16
  const float2 t = __ffma2_rn(r, make_float2(-1.0f, -1.0f), make_float2(1.0f, 1.0f));
  return __fmul2_rn(make_float2(0.5f, 0.5f), __ffma2_rn(az, t, z));
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t *>(&h);
}

__global__ void __launch_bounds__(kThreads, 1)
    fused_forward_kernel(const __nv_bfloat16 *X, int64_t n, const __nv_bfloat16 *wc,
                         const float *params, float *y, int *err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  unsigned char *xh = sm;
  uint64_t *bars = reinterpret_cast<uint64_t *>(sm + XH_BYTES + W_BYTES);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2);
  float *ypart = reinterpret_cast<float *>(sm + XH_BYTES + W_BYTES + 64);
  float *s_par = ypart + (kParts - 1) * TM;  // b1, b2, b3, w4 (256 each)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quad = warp & 3, part = warp >> 2;  // accumulator lanes 32 quad.., columns 64 part..
  const uint32_t bar_w = smem_u32(&bars[0]), bar_m = smem_u32(&bars[1]);
  const uint32_t s_xh = smem_u32(xh), s_w = smem_u32(sm + XH_BYTES);
  if (tid == 0) {
    mbar_init(bar_w, 1);
    mbar_init(bar_m, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(
                     smem_u32(tslot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  for (int i = tid; i < 3 * HIDDEN; i += kThreads)
    s_par[i] = params[(i >> 8) == 0 ? OFF_B1 + i : ((i >> 8) == 1 ? OFF_B2 + i - 256 : OFF_B3 + i - 512)];
  for (int i = tid; i < HIDDEN; i += kThreads) s_par[3 * HIDDEN + i] = params[OFF_W4 + i];
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t t_lane = tmem + ((uint32_t)(32 * quad) << 16);
  const float b4 = params[OFF_B4];
  const int64_t n_tiles = (n + TM - 1) / TM;
  uint32_t ph_w = 0, ph_m = 0;
  bool ok = true, w_pending = false, m_pending = false;

  auto load_w = [&](int layer) {
    const uint32_t bytes = (layer == 0 ? FEATURES : HIDDEN) * HIDDEN * 2;
    const unsigned char *src = reinterpret_cast<const unsigned char *>(
        wc + (layer == 0 ? 0 : (layer == 1 ? WC_L2 : WC_L3)));
    if (tid == 0) {
      mbar_expect_tx(bar_w, bytes);
      for (uint32_t off = 0; off < bytes; off += kCopyChunk)
        bulk_g2s(s_w + off, src + off, kCopyChunk, bar_w);
    }
    w_pending = true;
  };

  // feature tile t: a warp moves 8 rows x 4 chunks of 16 bytes per step (full
  // 32-byte sectors) into registers, stored later in the K-major core-matrix
  // layout (K = 128); the next tile's rows are read during the last epilogue
  constexpr int kXSteps = 64 / (kThreads / 32);
  uint4 xr[kXSteps];
  auto load_x = [&](int64_t t) {
#pragma unroll
    for (int i = 0; i < kXSteps; ++i) {
      const int v = warp + (kThreads / 32) * i;
      const int row = 8 * (v & 15) + (lane & 7), chunk = 4 * (v >> 4) + (lane >> 3);
      const int64_t gr = t * TM + row;
      xr[i] = gr < n ? __ldg(reinterpret_cast<const uint4 *>(X + gr * FEATURES) + chunk)
                     : make_uint4(0, 0, 0, 0);
    }
  };
  if (blockIdx.x < n_tiles) {
    load_w(0);
    load_x(blockIdx.x);
  }
  for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
#pragma unroll
    for (int i = 0; i < kXSteps; ++i) {
      const int v = warp + (kThreads / 32) * i;
      const int row = 8 * (v & 15) + (lane & 7), chunk = 4 * (v >> 4) + (lane >> 3);
      *reinterpret_cast<uint4 *>(xh + canon_off(row, 8 * chunk, FEATURES)) = xr[i];
    }
    fence_proxy_async();
    __syncthreads();
    const int row = 32 * quad + lane;                  // this thread's row (accumulator lane)
    float yrow = part ? 0.0f : b4;
    for (int layer = 0; layer < 3 && ok; ++layer) {
      const int K = layer == 0 ? FEATURES : HIDDEN;
      // this layer's weights are in shared memory (the outcome of every wait
      // is agreed by the whole CTA, so all threads leave together)
      ok = __syncthreads_and(mbar_wait(bar_w, ph_w));
      if (!ok) break;
      w_pending = false;
      ph_w ^= 1u;
      if (tid == 0) {
        fence_after_sync();
        const uint32_t sbo = (uint32_t)K * 16;  // next 8-row group: K / 8 blocks of 128 bytes
        for (int s = 0; s < K / 16; ++s)
          mma_bf16(tmem, sdesc(s_xh + 256u * s, 128u, sbo), sdesc(s_w + 256u * s, 128u, sbo),
                   idesc_bf16(TM, HIDDEN), s > 0);
        mma_commit(bar_m);
      }
      m_pending = true;
      ok = __syncthreads_and(mbar_wait(bar_m, ph_m));  // accumulator complete; A, B buffers free
      if (!ok) break;
      m_pending = false;
      ph_m ^= 1u;
      fence_after_sync();
      // the next weights (and after the last layer the next tile's features)
      // stream in during this epilogue
      if (layer < 2) {
        load_w(layer + 1);
      } else if (t + gridDim.x < n_tiles) {
        load_w(0);
        load_x(t + gridDim.x);
      }
      // ---- epilogue: bias + GELU -> BF16 (next A operand) or the output --
      const float *bias = s_par + HIDDEN * layer;
      const float *w4 = s_par + 3 * HIDDEN;
      // two chunks of 32 columns; the read of the second is in flight while
      // the first is processed
      uint32_t ra[32], rb[32];
      auto chunk = [&](int cc, const uint32_t (&r)[32]) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float4 bl = *reinterpret_cast<const float4 *>(bias + 32 * cc + 8 * q);
          const float4 bh = *reinterpret_cast<const float4 *>(bias + 32 * cc + 8 * q + 4);
          const float bq[8] = {bl.x, bl.y, bl.z, bl.w, bh.x, bh.y, bh.z, bh.w};
          uint32_t w[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const float2 a = gelu2(__fadd2_rn(make_float2(__uint_as_float(r[8 * q + 2 * e]),
                                                          __uint_as_float(r[8 * q + 2 * e + 1])),
                                              make_float2(bq[2 * e], bq[2 * e + 1])));
            w[e] = pack_bf16(a.x, a.y);
          }
          if (layer < 2) {
            *reinterpret_cast<uint4 *>(xh + canon_off(row, 32 * cc + 8 * q, HIDDEN)) =
                make_uint4(w[0], w[1], w[2], w[3]);
          } else {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int c = 32 * cc + 8 * q + 2 * e;
              const __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162 *>(&w[e]);
              yrow = fmaf(__low2float(h), w4[c], yrow);
              yrow = fmaf(__high2float(h), w4[c + 1], yrow);
            }
          }
        }
      };
      const int c0 = 2 * part;
      tmem_ld32(t_lane + 32u * c0, ra);
      tmem_wait(ra);
      tmem_ld32(t_lane + 32u * (c0 + 1), rb);
      chunk(c0, ra);
      tmem_wait(rb);
      chunk(c0 + 1, rb);
      if (layer < 2) fence_proxy_async();
      else if (part) ypart[(part - 1) * TM + row] = yrow;
      fence_before_sync();
      __syncthreads();
    }
    if (ok && !part && t * TM + row < n)
      y[t * TM + row] = yrow + (ypart[row] + (ypart[TM + row] + ypart[2 * TM + row]));
  }
  // ---- teardown: let copies and products in flight finish, free TMEM ------
  if (w_pending) mbar_wait(bar_w, ph_w);
  if (m_pending) mbar_wait(bar_m, ph_m);
  if (!ok && lane == 0) atomicExch(err, 1);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tmem) : "memory");
}

// Layers 1-3 of the packed FP32 parameters (W stored [in][out]) as BF16
// B operands (N = 256 outputs x K inputs) in the K-major core-matrix layout.
__global__ void canon_weights_kernel(const float *p, __nv_bfloat16 *wc) {
  const int total = WC_L3 + HIDDEN * HIDDEN;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    int layer, e;
    if (i < WC_L2) {
      layer = 0;
      e = i;
    } else if (i < WC_L3) {
      layer = 1;
      e = i - WC_L2;
    } else {
      layer = 2;
      e = i - WC_L3;
    }
    const int K = layer == 0 ? FEATURES : HIDDEN;
    const int nn = e / K, k = e % K;  // output nn, input k
    const int off_w = layer == 0 ? OFF_W1 : (layer == 1 ? OFF_W2 : OFF_W3);
    const int base = layer == 0 ? 0 : (layer == 1 ? WC_L2 : WC_L3);
    wc[base + canon_off(nn, k, K) / 2] = __float2bfloat16_rn(p[off_w + k * HIDDEN + nn]);
  }
}

}  // namespace

cudaError_t canon_weights(const float *p, __nv_bfloat16 *wc, cudaStream_t s) {
  canon_weights_kernel<<<160, 256, 0, s>>>(p, wc);
  return cudaGetLastError();
}

cudaError_t fused_forward(const __nv_bfloat16 *X, int64_t n, const __nv_bfloat16 *wc,
                          const float *params, float *y, int *err, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int dev = 0, n_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fused_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             SMEM_BYTES);
  if (e != cudaSuccess) return e;
  const int64_t tiles = (n + TM - 1) / TM;
  const int grid = (int)(tiles < n_sm ? tiles : n_sm);
  fused_forward_kernel<<<grid, kThreads, SMEM_BYTES, s>>>(X, n, wc, params, y, err);
  return cudaGetLastError();
}

int canon_weight_elems() { return WC_L3 + HIDDEN * HIDDEN; }

}  // namespace mlp
}  // namespace dk
