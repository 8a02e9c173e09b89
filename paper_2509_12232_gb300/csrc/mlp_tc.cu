// Fused forward pass of the surrogate MLP (128 -> 256 -> 256 -> 256 -> 1,
// GELU after the hidden layers) on the 5th-generation tensor cores.
//
// One persistent CTA per SM takes tiles of 128 feature rows, two at a time in
// two slots, so that one slot's products run while the other slot's
// epilogue runs (the epilogue is about as long as the products):
//   - a slot's A operand (features, then each hidden layer) is a 64 KB tile
//     in shared memory in the K-major "core matrix" layout the tensor core
//     reads without swizzling (8 rows x 16 bytes per 128-byte block); its
//     accumulator is one half (256 columns) of the CTA's tensor memory;
//   - a copy warp fetches a slot's features by 2-D tensor copies once the
//     slot's last product is done, and streams the BF16 weights, kept in
//     global memory as chunks of 64 K columns (32 KB, the core-matrix layout
//     with K = 64), in the order the products use them through a ring of two
//     shared-memory stages (bulk copies completing on the stage's "full"
//     mbarrier; the products that read a stage commit to its "empty" one);
//   - an MMA warp issues, per slot and layer, tcgen05.mma (M = 128, N = 256,
//     K = 16 per instruction) into the slot's accumulator once the slot's A
//     operand is ready, and commits the layer to the slot's accumulator
//     mbarrier;
//   - 16 epilogue warps drain a finished accumulator, warp w reading lanes
//     32 (w mod 4) .. + 31 (the lane quarter its position in the warp group
//     may access) and columns 64 (w / 4) .. + 63 with tcgen05.ld: GELU,
//     rounding to BF16 and stores into the slot's A operand for the next
//     layer; then they set those columns to the next layer's bias with
//     tcgen05.st, so that the products accumulate onto it, and signal the
//     MMA warp through the slot's "A ready" mbarrier. After the third layer
//     each thread forms a quarter of its row's output (a dot product with the
//     FP32 w4) and parts 1-3 hand theirs to part 0 through shared memory.
// The hidden activations are kept doubled and W2, W3 and w4 halved (exact
// powers of two: the same roundings and products, one multiply fewer per
// activation).
// Every mbarrier wait is bounded (one second of globaltimer) and also ends
// when another role has given up; a timeout sets *err, the roles leave their
// loops (the caller fills the output with NaN beforehand), and the tensor
// memory is released after the copies and products in flight are waited for.
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "mlp.h"

namespace dk {
namespace mlp {

namespace {

constexpr int TM = 128;                       // rows per tile (MMA M)
#ifndef DOCK_MLP_EPI_WARPS
#define DOCK_MLP_EPI_WARPS 16
#endif
constexpr int kEpiWarps = DOCK_MLP_EPI_WARPS; // a multiple of 4
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kMmaWarp = kEpiWarps, kCopyWarp = kEpiWarps + 1;
constexpr int kThreads = kEpiThreads + 64;    // + the MMA warp and the weight-copy warp
constexpr int kParts = kEpiWarps / 4;         // column parts of a row: warp w takes lanes
                                              // 32 (w mod 4).. and part w / 4 of the columns
constexpr int kPartChunks = HIDDEN / 32 / kParts;  // 32-column accumulator reads per part
// Registers per thread: each of the SM's four schedulers holds a quarter of
// the register file, and the warps are spread over them round robin.
constexpr int kMaxRegs = (16384 / (32 * ((kEpiWarps + 2 + 3) / 4))) / 8 * 8;
constexpr int ACT_BYTES = TM * HIDDEN * 2;    // one slot's A operand (64 KB)
constexpr int KC = 64;                        // K columns of one weight chunk
constexpr int WCH_ELEMS = HIDDEN * KC;        // BF16 values of a chunk (32 KB)
constexpr int WCH_BYTES = 2 * WCH_ELEMS;
constexpr int kStages = 2;                    // weight chunks in shared memory
// mbarriers: weight stages full / empty, slot accumulators complete, slot A
// operands ready, slot features landed, slot A operand free (its last
// product done), output partials full / empty, products drained at the end
constexpr int B_WFULL = 0, B_WEMPTY = kStages, B_ACC = 2 * kStages, B_ACT = B_ACC + 2,
              B_XF = B_ACT + 2, B_AFREE = B_XF + 2, B_YFULL = B_AFREE + 2,
              B_YEMPTY = B_YFULL + 2, B_FIN = B_YEMPTY + 2, N_BARS = B_FIN + 1;
constexpr int X_BYTES = TM * FEATURES * 2;    // one feature tile (32 KB)
constexpr int OFF_WST = 2 * ACT_BYTES;
constexpr int OFF_BAR = OFF_WST + kStages * WCH_BYTES;
constexpr int kBarBytes = (8 * N_BARS + 8 + 127) / 128 * 128;
constexpr int OFF_YP = OFF_BAR + kBarBytes;         // barriers, TMEM address, abort flag
constexpr int OFF_PAR = OFF_YP + 2 * (kParts - 1) * TM * 4;  // output partials of parts >= 1
constexpr int SMEM_BYTES = OFF_PAR + 4 * HIDDEN * 4;         // + biases b1..b3 and w4
static_assert(8 * N_BARS + 8 <= kBarBytes, "barrier block");
static_assert(SMEM_BYTES <= 227 * 1024, "shared memory");
constexpr int WC_L2 = HIDDEN * FEATURES;      // weight values of layer 1 (and of 1 + 2: WC_L3)
constexpr int WC_L3 = WC_L2 + HIDDEN * HIDDEN;
constexpr uint64_t kWaitNs = 1000000000ull;   // bound of every mbarrier wait

// First chunk of layer `layer` (0-2) in the chunked weight array.
__host__ __device__ constexpr int wchunk0(int layer) {
  return layer == 0 ? 0 : (layer == 1 ? FEATURES / KC : (FEATURES + HIDDEN) / KC);
}

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

// mbar_wait that also gives up once *abort is set (another role of the CTA
// has given up).
__device__ __forceinline__ bool mbar_wait_ab(uint32_t bar, uint32_t ph, const volatile int *abort) {
  uint64_t t0 = 0;
  for (uint32_t k = 0;; ++k) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(ph)
        : "memory");
    if (done) return true;
    if ((k & 15) == 0) {  // the clock and the flag every 16 polls
      if (k == 0) t0 = gtimer();
      else if (*abort || gtimer() - t0 > kWaitNs) return false;
    }
  }
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// Tiled 2-D tensor copy of box (x, y) of the tensor map into shared memory.
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, int x, int y,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
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

// Write 32 consecutive accumulator columns of this thread's lane.
__device__ __forceinline__ void tmem_st32(uint32_t taddr, const uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31, %32};" ::"r"(taddr),
      "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
      "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]),
      "r"(r[15]), "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]),
      "r"(r[22]), "r"(r[23]), "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]),
      "r"(r[29]), "r"(r[30]), "r"(r[31])
      : "memory");
}

__device__ __forceinline__ void tmem_wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// gelu_t (mlp.h) on two activations: packed two-wide FP32 arithmetic (the same
// operations in the same order, one instruction for both) around two tanh
// on the special-function unit.
__device__ __forceinline__ float2 gelu2(float2 z) {
  const float2 z2 = __fmul2_rn(z, z);
  const float2 t = __ffma2_rn(make_float2(kGeluC1, kGeluC1), z2, make_float2(kGeluC0, kGeluC0));
  const float2 u = __fmul2_rn(z, t);
  const float2 th = make_float2(tanh_sfu(u.x), tanh_sfu(u.y));
  const float2 h = __fmul2_rn(make_float2(0.5f, 0.5f), z);
  return __ffma2_rn(h, th, h);
}

// Twice gelu2, z (1 + tanh(u)) in one fused multiply-add: the same value
// scaled by 2 exactly (one multiply fewer). The fused forward pass keeps its
// hidden activations scaled by 2 and the weights that read them (W2, W3, w4)
// scaled by 1/2, powers of two that leave every BF16 rounding and every
// product unchanged.
__device__ __forceinline__ float2 gelu2_twice(float2 z) {
  const float2 z2 = __fmul2_rn(z, z);
  const float2 t = __ffma2_rn(make_float2(kGeluC1, kGeluC1), z2, make_float2(kGeluC0, kGeluC0));
  const float2 u = __fmul2_rn(z, t);
  const float2 th = make_float2(tanh_sfu(u.x), tanh_sfu(u.y));
  return __ffma2_rn(z, th, z);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t *>(&h);
}

__global__ void __maxnreg__(kMaxRegs)
    fused_forward_kernel(const __grid_constant__ CUtensorMap tmx, int64_t n,
                         const __nv_bfloat16 *wc, const float *params, float *y, int *err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  uint64_t *bars = reinterpret_cast<uint64_t *>(sm + OFF_BAR);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + OFF_BAR + 8 * N_BARS);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(sm + OFF_BAR + 8 * N_BARS + 4);
  float *ypart = reinterpret_cast<float *>(sm + OFF_YP);   // [slot][part - 1][row]
  float *s_par = reinterpret_cast<float *>(sm + OFF_PAR);  // b1, b2, b3, w4 / 2 (256 each)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  auto bar = [&](int i) { return smem_u32(&bars[i]); };
  const uint32_t s_act = smem_u32(sm), s_wst = smem_u32(sm + OFF_WST);
  if (tid == 0) {
    for (int i = 0; i < kStages; ++i) {
      mbar_init(bar(B_WFULL + i), 1);
      mbar_init(bar(B_WEMPTY + i), 1);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(bar(B_ACC + s), 1);
      mbar_init(bar(B_ACT + s), kEpiWarps);
      mbar_init(bar(B_XF + s), 1);
      mbar_init(bar(B_AFREE + s), 1);
      mbar_init(bar(B_YFULL + s), kEpiWarps - 4);  // warps of parts >= 1
      mbar_init(bar(B_YEMPTY + s), 4);             // warps of part 0
    }
    mbar_init(bar(B_FIN), 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(
                     smem_u32(tslot))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  for (int i = tid; i < 3 * HIDDEN; i += kThreads)
    s_par[i] = params[(i >> 8) == 0 ? OFF_B1 + i : ((i >> 8) == 1 ? OFF_B2 + i - 256 : OFF_B3 + i - 512)];
  for (int i = tid; i < HIDDEN; i += kThreads) s_par[3 * HIDDEN + i] = 0.5f * params[OFF_W4 + i];
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;
  const int64_t n_tiles = (n + TM - 1) / TM, G = gridDim.x;
  // this CTA's tiles blockIdx.x + i G, i < n_local; tile i goes to slot i mod 2
  const int n_local = blockIdx.x < n_tiles ? (int)((n_tiles - 1 - blockIdx.x) / G + 1) : 0;
  bool ok = true;
  auto fail = [&]() {
    ok = false;
    *abort_flag = 1;
  };

  if (warp == kCopyWarp) {
    // ---- features and weight chunks in the order the products use them ----
    if (lane == 0) {
      int g = 0;                       // weight chunks issued
      int x_issued[2] = {0, 0};        // feature tiles issued per slot
      uint32_t ph_free[2] = {0u, 0u};
      for (int i0 = 0; i0 < n_local && ok; i0 += 2)
        for (int layer = 0; layer < 3 && ok; ++layer)
          for (int s = 0; s < 2 && ok && i0 + s < n_local; ++s) {
            if (layer == 0) {
              // the tile's features into the slot once its previous tile's
              // last product is done: one 2 KB box (8 K values x 128 rows)
              // per K block, which is the core-matrix layout with the K
              // blocks 2 KB apart
              if (i0 > 0) {
                if (!mbar_wait_ab(bar(B_AFREE + s), ph_free[s], abort_flag)) {
                  fail();
                  break;
                }
                ph_free[s] ^= 1u;
              }
              const int row0 = (int)((blockIdx.x + (int64_t)(i0 + s) * G) * TM);
              mbar_expect_tx(bar(B_XF + s), X_BYTES);
              for (int c = 0; c < FEATURES / 8; ++c)
                tma_load_2d(s_act + s * ACT_BYTES + c * (TM * 16), &tmx, 8 * c, row0, bar(B_XF + s));
              ++x_issued[s];
            }
            const int nch = (layer ? HIDDEN : FEATURES) / KC;
            for (int c = 0; c < nch; ++c, ++g) {
              const int st = g % kStages;
              if (g >= kStages &&
                  !mbar_wait_ab(bar(B_WEMPTY + st), (uint32_t)((g / kStages) - 1) & 1u, abort_flag)) {
                fail();
                break;
              }
              mbar_expect_tx(bar(B_WFULL + st), WCH_BYTES);
              bulk_g2s(s_wst + st * WCH_BYTES, wc + (int64_t)(wchunk0(layer) + c) * WCH_ELEMS,
                       WCH_BYTES, bar(B_WFULL + st));
            }
          }
      // the last copies into each stage and slot land before the CTA ends
      for (int k = 1; k <= kStages && k <= g; ++k)
        mbar_wait(bar(B_WFULL + (g - k) % kStages), (uint32_t)((g - k) / kStages) & 1u);
      for (int s = 0; s < 2; ++s)
        if (x_issued[s] > 0) mbar_wait(bar(B_XF + s), (uint32_t)(x_issued[s] - 1) & 1u);
    }
  } else if (warp == kMmaWarp) {
    // ---- products: per slot and layer, once the slot's A operand is ready --
    if (lane == 0) {
      int g = 0;  // chunks consumed
      uint32_t ph_act[2] = {0u, 0u}, ph_x[2] = {0u, 0u};
      bool issued = false;
      for (int i0 = 0; i0 < n_local && ok; i0 += 2)
        for (int layer = 0; layer < 3 && ok; ++layer)
          for (int s = 0; s < 2 && ok && i0 + s < n_local; ++s) {
            // layer 0: the features have landed; every layer: the epilogue
            // has read the accumulator, set it to this layer's bias and (layers
            // 1-2) written this layer's A operand
            if (layer == 0) {
              if (!mbar_wait_ab(bar(B_XF + s), ph_x[s], abort_flag)) {
                fail();
                break;
              }
              ph_x[s] ^= 1u;
            }
            if (!mbar_wait_ab(bar(B_ACT + s), ph_act[s], abort_flag)) {
              fail();
              break;
            }
            ph_act[s] ^= 1u;
            fence_after_sync();
            const int K = layer ? HIDDEN : FEATURES;
            // A operand: features with K blocks 2 KB apart and row groups 128 B
            // apart; hidden layers with K blocks 128 B and row groups K * 16 B
            const uint32_t a0 = s_act + s * ACT_BYTES;
            const uint32_t lbo_a = layer ? 128u : TM * 16u, sbo_a = layer ? (uint32_t)K * 16 : 128u;
            const uint32_t d = tmem + 256u * s;
            for (int c = 0; c < K / KC; ++c, ++g) {
              const int st = g % kStages;
              if (!mbar_wait_ab(bar(B_WFULL + st), (uint32_t)(g / kStages) & 1u, abort_flag)) {
                fail();
                break;
              }
              fence_after_sync();
#pragma unroll
              for (int j = 0; j < KC / 16; ++j)
                mma_bf16(d, sdesc(a0 + 2u * lbo_a * (c * (KC / 16) + j), lbo_a, sbo_a),
                         sdesc(s_wst + st * WCH_BYTES + 256u * j, 128u, (KC / 8) * 128u),
                         idesc_bf16(TM, HIDDEN), 1u);  // onto the bias
              mma_commit(bar(B_WEMPTY + st));
              issued = true;
            }
            if (ok) {
              if (layer == 2) mma_commit(bar(B_AFREE + s));  // the slot may take new features
              mma_commit(bar(B_ACC + s));
            }
          }
      // the products in flight finish before the tensor memory is released
      if (issued) {
        mma_commit(bar(B_FIN));
        mbar_wait(bar(B_FIN), 0u);
      }
    }
  } else {
    // ---- epilogue warps -----------------------------------------------------
    const int quad = warp & 3, part = warp >> 2;  // lanes 32 quad.., column part `part`
    const int row = 32 * quad + lane;             // this thread's row (accumulator lane)
    const uint32_t t_lane = tmem + ((uint32_t)(32 * quad) << 16);
    const float b4 = params[OFF_B4];
    uint32_t ph_acc[2] = {0u, 0u};
    int y_use[2] = {0, 0};
    const int c0 = kPartChunks * part;
    // this thread's accumulator columns of slot s set to the bias of layer
    // `layer` (the products then accumulate onto it)
    auto preload_bias = [&](int s, int layer) {
      const float *b = s_par + HIDDEN * layer;
      const uint32_t ta = t_lane + 256u * s;
#pragma unroll
      for (int k = 0; k < kPartChunks; ++k) {
        uint32_t r[32];
#pragma unroll
        for (int j = 0; j < 32; j += 4) {
          const float4 v = *reinterpret_cast<const float4 *>(b + 32 * (c0 + k) + j);
          r[j] = __float_as_uint(v.x);
          r[j + 1] = __float_as_uint(v.y);
          r[j + 2] = __float_as_uint(v.z);
          r[j + 3] = __float_as_uint(v.w);
        }
        tmem_st32(ta + 32u * (c0 + k), r);
      }
      tmem_wait_st();
    };
    // A operand ready (a hidden layer written, the accumulator read and set
    // to the next bias)
    auto signal_act = [&](int s) {
      fence_proxy_async();
      fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_ACT + s));
    };
    for (int s = 0; s < 2 && s < n_local; ++s) {
      preload_bias(s, 0);
      signal_act(s);
    }
    for (int i0 = 0; i0 < n_local && ok; i0 += 2)
      for (int layer = 0; layer < 3 && ok; ++layer)
        for (int s = 0; s < 2 && ok && i0 + s < n_local; ++s) {
          const int i = i0 + s;
          const int64_t t = blockIdx.x + (int64_t)i * G;
          if (!__all_sync(0xffffffffu, mbar_wait_ab(bar(B_ACC + s), ph_acc[s], abort_flag))) {
            fail();
            break;
          }
          ph_acc[s] ^= 1u;
          fence_after_sync();
          const bool next = layer == 2 && i + 2 < n_local;
          // ---- GELU (the bias is in the accumulator) -> BF16 (next A operand)
          // ---- or the output ----------------------------------------------
          unsigned char *act = sm + s * ACT_BYTES;
          const float *w4 = s_par + 3 * HIDDEN;
          float yrow = part ? 0.0f : b4;
          // two chunks of 32 columns; the read of the second is in flight
          // while the first is processed
          uint32_t ra[32], rb[32];
          auto chunk = [&](int cc, const uint32_t (&r)[32]) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              uint32_t w[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                const float2 a = gelu2_twice(make_float2(__uint_as_float(r[8 * q + 2 * e]),
                                                         __uint_as_float(r[8 * q + 2 * e + 1])));
                w[e] = pack_bf16(a.x, a.y);
              }
              if (layer < 2) {
                *reinterpret_cast<uint4 *>(act + canon_off(row, 32 * cc + 8 * q, HIDDEN)) =
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
          const uint32_t ta = t_lane + 256u * s;
          tmem_ld32(ta + 32u * c0, ra);
          tmem_wait(ra);
#pragma unroll
          for (int k = 0; k < kPartChunks; k += 2) {
            if (k + 1 < kPartChunks) tmem_ld32(ta + 32u * (c0 + k + 1), rb);
            chunk(c0 + k, ra);
            if (k + 1 < kPartChunks) {
              tmem_wait(rb);
              if (k + 2 < kPartChunks) tmem_ld32(ta + 32u * (c0 + k + 2), ra);
              chunk(c0 + k + 1, rb);
              if (k + 2 < kPartChunks) tmem_wait(ra);
            }
          }
          if (layer < 2) {
            preload_bias(s, layer + 1);
            signal_act(s);
            continue;
          }
          // ---- output: parts >= 1 hand their partial dot products to part 0 -
          float *yp = ypart + s * (kParts - 1) * TM;
          const int u = y_use[s]++;
          if (part) {
            if (u > 0 &&
                !__all_sync(0xffffffffu, mbar_wait_ab(bar(B_YEMPTY + s), (uint32_t)(u - 1) & 1u,
                                                      abort_flag))) {
              fail();
              break;
            }
            yp[(part - 1) * TM + row] = yrow;
            __syncwarp();
            if (lane == 0) mbar_arrive(bar(B_YFULL + s));
          } else {
            if (!__all_sync(0xffffffffu,
                            mbar_wait_ab(bar(B_YFULL + s), (uint32_t)u & 1u, abort_flag))) {
              fail();
              break;
            }
            float rest = yp[(kParts - 2) * TM + row];
#pragma unroll
            for (int q = kParts - 3; q >= 0; --q) rest = yp[q * TM + row] + rest;
            if (t * TM + row < n) y[t * TM + row] = yrow + rest;
            __syncwarp();
            if (lane == 0) mbar_arrive(bar(B_YEMPTY + s));
          }
          if (next) {  // the accumulator may take the next tile
            preload_bias(s, 0);
            signal_act(s);
          }
        }
  }
  // ---- teardown: copies and products in flight have finished; free TMEM ---
  if (!ok && lane == 0) atomicExch(err, 1);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
}

// ---------------------------------------------------------------------------
// Training products on tcgen05: C[M][256] = A[M][K] Bt[256][K]^T.
// CTA (blockIdx.x, split blockIdx.y, column quarter blockIdx.z) computes rows
// m0 .. m0 + 127 and columns 64 z .. + 63 over its K range in chunks of 64
// (four quarters per row block give a 4,096-row batch 128 CTAs): one thread
// streams the chunks of A (128 x 64) and Bt (its 64 rows x 64) by 2-D tensor
// copies into a ring of four stages and issues four MMAs (M 128, N 64, K 16)
// per chunk into the 64-column FP32 accumulator, committing each chunk to its
// stage's "empty" mbarrier, after which the stage takes the chunk four ahead.
// The epilogue reads the accumulator with tcgen05.ld: warp w takes lanes
// 32 (w mod 4) .. + 31 and columns 32 (w / 4) .. + 31. Every mbarrier wait
// is bounded as in the
// forward kernel; a timeout sets *err and the CTA writes nothing.
// ---------------------------------------------------------------------------
// The transposed copy c16t[c][r] (row stride ldt) of a thread's 32 BF16
// values h (row r, columns col..col+31): the lanes of a warp hold 32
// consecutive rows, so each column is one 64-byte store per warp.
__device__ __forceinline__ void store_transposed(const Epilogue &ep, const uint32_t (&h)[16],
                                                 int64_t row, int col) {
  if (ep.c16t == nullptr) return;
  unsigned short *t = reinterpret_cast<unsigned short *>(ep.c16t);
#pragma unroll
  for (int k = 0; k < 32; ++k)
    t[(int64_t)(col + k) * ep.ldt + row] =
        (unsigned short)((k & 1) ? (h[k >> 1] >> 16) : (h[k >> 1] & 0xffffu));
}

constexpr int GK = 64;                     // K per chunk
constexpr int GA_BYTES = 128 * GK * 2;     // A chunk: 16 KB
constexpr int GN = 64;                     // columns per CTA (4 CTAs across 256 columns)
constexpr int GB_BYTES = GN * GK * 2;      // Bt chunk: 8 KB
constexpr int G_STAGE = GA_BYTES + GB_BYTES;
constexpr int G_STAGES = 4;                // chunks in flight
constexpr int G_SMEM = G_STAGES * G_STAGE + 128;
constexpr int G_THREADS = 256;

template <int EPI>
__global__ void __launch_bounds__(G_THREADS, 2)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tma, const __grid_constant__ CUtensorMap tmb,
                   int k_split, Epilogue ep, int *err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  // mbarriers: stage full [G_STAGES], stage empty [G_STAGES], products done
  uint64_t *bars = reinterpret_cast<uint64_t *>(sm + G_STAGES * G_STAGE);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2 * G_STAGES + 1);
  int *s_ok = reinterpret_cast<int *>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t m0 = (int64_t)blockIdx.x * 128;
  const int k0 = blockIdx.y * k_split;
  const int n0 = GN * blockIdx.z;
  const int nc = k_split / GK;
  auto bar = [&](int i) { return smem_u32(&bars[i]); };
  const int B_FULL = 0, B_EMPTY = G_STAGES, B_DONE = 2 * G_STAGES;
  if (tid == 0) {
    for (int i = 0; i < 2 * G_STAGES + 1; ++i) mbar_init(bar(i), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tslot)), "n"(GN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  const uint32_t tmem = *tslot;
  bool ok = nc > 0;
  if (tid == 0) {
    // One thread streams the chunks (tensor copies: a box of 8 K values x the
    // operand's rows per K block, which lands as the core-matrix layout with
    // K blocks 2 KB (A) or 1 KB (Bt) apart and row groups 128 B apart) and
    // issues the products; a stage is refilled once its products are done.
    auto load = [&](int c) {
      const int st = c % G_STAGES;
      const uint32_t sa = smem_u32(sm + st * G_STAGE), sb = sa + GA_BYTES;
      const int kk = k0 + c * GK;
      mbar_expect_tx(bar(B_FULL + st), G_STAGE);
#pragma unroll
      for (int kb = 0; kb < GK / 8; ++kb) {
        tma_load_2d(sa + kb * (128 * 16), &tma, kk + 8 * kb, (int)m0, bar(B_FULL + st));
        tma_load_2d(sb + kb * (GN * 16), &tmb, kk + 8 * kb, n0, bar(B_FULL + st));
      }
    };
    int loaded = 0, used = 0;
    for (; ok && loaded < nc && loaded < G_STAGES; ++loaded) load(loaded);
    for (int c = 0; c < nc && ok; ++c) {
      const int st = c % G_STAGES;
      if (!mbar_wait(bar(B_FULL + st), (uint32_t)(c / G_STAGES) & 1u)) {
        ok = false;
        break;
      }
      used = c + 1;
      fence_after_sync();
      const uint32_t sa = smem_u32(sm + st * G_STAGE), sb = sa + GA_BYTES;
#pragma unroll
      for (int q = 0; q < GK / 16; ++q)
        mma_bf16(tmem, sdesc(sa + 2u * (128 * 16) * q, 128u * 16, 128u),
                 sdesc(sb + 2u * (GN * 16) * q, GN * 16u, 128u), idesc_bf16(128, GN),
                 (c > 0 || q > 0) ? 1u : 0u);
      mma_commit(bar(B_EMPTY + st));
      // refill the stage of chunk c - 1 once its products are done
      if (c >= 1 && loaded < nc) {
        const int pc = c - 1;
        if (!mbar_wait(bar(B_EMPTY + pc % G_STAGES), (uint32_t)(pc / G_STAGES) & 1u)) {
          ok = false;
          break;
        }
        load(loaded++);
      }
    }
    // the products issued so far, then the copies not consumed, finish
    if (used > 0) mma_commit(bar(B_DONE));
    if (!ok) {
      if (used > 0) mbar_wait(bar(B_DONE), 0u);
      for (int c = used; c < loaded; ++c)
        mbar_wait(bar(B_FULL + c % G_STAGES), (uint32_t)(c / G_STAGES) & 1u);
    }
    *s_ok = ok ? 1 : 0;
  }
  __syncthreads();
  ok = *s_ok != 0;
  if (ok) ok = __syncthreads_and(mbar_wait(bar(B_DONE), 0u));
  if (ok) {
    fence_after_sync();
    const int quad = warp & 3, half = warp >> 2;
    const int64_t row = m0 + 32 * quad + lane;
    const uint32_t t_lane = tmem + ((uint32_t)(32 * quad) << 16);
#pragma unroll 1
    for (int cc = 0; cc < GN / 64; ++cc) {
      const int tcol = (GN / 2) * half + 32 * cc, col = n0 + tcol;
      uint32_t r[32];
      tmem_ld32(t_lane + (uint32_t)tcol, r);
      tmem_wait(r);
      const int64_t o = row * ep.ldc + col;
      if (EPI == EPI_STORE_F32) {
        float4 *dst = reinterpret_cast<float4 *>(ep.c32 + (int64_t)blockIdx.y * ep.split_stride + o);
#pragma unroll
        for (int j = 0; j < 8; ++j)
          dst[j] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                               __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
      } else if (EPI == EPI_BIAS_GELU) {
        uint32_t h[16];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float4 b = *reinterpret_cast<const float4 *>(ep.bias + col + 4 * j);
          const float z0 = __uint_as_float(r[4 * j]) + b.x, z1 = __uint_as_float(r[4 * j + 1]) + b.y;
          const float z2 = __uint_as_float(r[4 * j + 2]) + b.z, z3 = __uint_as_float(r[4 * j + 3]) + b.w;
          if (ep.c32) reinterpret_cast<float4 *>(ep.c32 + o)[j] = make_float4(z0, z1, z2, z3);
          const float2 g01 = gelu2(make_float2(z0, z1)), g23 = gelu2(make_float2(z2, z3));
          h[2 * j] = pack_bf16(g01.x, g01.y);
          h[2 * j + 1] = pack_bf16(g23.x, g23.y);
        }
        uint4 *dst = reinterpret_cast<uint4 *>(ep.c16 + o);
#pragma unroll
        for (int j = 0; j < 4; ++j) dst[j] = make_uint4(h[4 * j], h[4 * j + 1], h[4 * j + 2], h[4 * j + 3]);
        store_transposed(ep, h, row, col);
        if (ep.ydot) {  // the output layer's partial dot product over these 32 columns
          float d = 0.0f;
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const __nv_bfloat162 hv = *reinterpret_cast<const __nv_bfloat162 *>(&h[k]);
            d = fmaf(__low2float(hv), __ldg(ep.w4 + col + 2 * k), d);
            d = fmaf(__high2float(hv), __ldg(ep.w4 + col + 2 * k + 1), d);
          }
          ep.ydot[(int64_t)(col >> 5) * ep.ldy + row] = d;
        }
      } else {  // EPI_GELU_BWD: dZ = dH gelu'(Z)
        uint32_t h[16];
        const float4 *zin = reinterpret_cast<const float4 *>(ep.zin + o);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float4 z = zin[j];
          h[2 * j] = pack_bf16(__uint_as_float(r[4 * j]) * gelu_t_grad(z.x),
                               __uint_as_float(r[4 * j + 1]) * gelu_t_grad(z.y));
          h[2 * j + 1] = pack_bf16(__uint_as_float(r[4 * j + 2]) * gelu_t_grad(z.z),
                                   __uint_as_float(r[4 * j + 3]) * gelu_t_grad(z.w));
        }
        uint4 *dst = reinterpret_cast<uint4 *>(ep.c16 + o);
#pragma unroll
        for (int j = 0; j < 4; ++j) dst[j] = make_uint4(h[4 * j], h[4 * j + 1], h[4 * j + 2], h[4 * j + 3]);
        store_transposed(ep, h, row, col);
      }
    }
  }
  // ---- teardown (the producing thread has waited for its work in flight) ---
  if (!ok && tid == 0 && nc > 0) atomicExch(err, 1);
  fence_before_sync();
  __syncthreads();
  fence_after_sync();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(GN)
                 : "memory");
}

// out [cols][rows] = in [rows][cols]^T (BF16; 32 x 32 tiles through shared memory).
__global__ void transpose_bf16_kernel(const __nv_bfloat16 *in, int rows, int cols,
                                      __nv_bfloat16 *out) {
  __shared__ __nv_bfloat16 t[32][33];
  const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int r = r0 + i, c = c0 + threadIdx.x;
    if (r < rows && c < cols) t[i][threadIdx.x] = in[(int64_t)r * cols + c];
  }
  __syncthreads();
  for (int i = threadIdx.y; i < 32; i += blockDim.y) {
    const int c = c0 + i, r = r0 + threadIdx.x;
    if (r < rows && c < cols) out[(int64_t)c * rows + r] = t[threadIdx.x][i];
  }
}

// out[c] = sum of the `parts` partials in order 0, 1, ... (fixed order).
__global__ void sum_parts_kernel(const float *part, int parts, int64_t width, float *out) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= width) return;
  float s = 0.0f;
  for (int b = 0; b < parts; ++b) s += part[(int64_t)b * width + c];
  out[c] = s;
}

// Layers 1-3 of the packed FP32 parameters (W stored [in][out]) as BF16
// B operands (N = 256 outputs x K inputs) in chunks of KC input columns, each
// chunk in the K-major core-matrix layout with K = KC; layer l's chunks
// start at chunk wchunk0(l).
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
    // W2, W3 halved: they read activations kept doubled (gelu2_twice)
    const float w = p[off_w + k * HIDDEN + nn];
    wc[(wchunk0(layer) + k / KC) * WCH_ELEMS + canon_off(nn, k % KC, KC) / 2] =
        __float2bfloat16_rn(layer == 0 ? w : 0.5f * w);
  }
}

}  // namespace

cudaError_t canon_weights(const float *p, __nv_bfloat16 *wc, cudaStream_t s) {
  canon_weights_kernel<<<160, 256, 0, s>>>(p, wc);
  return cudaGetLastError();
}

// cuTensorMapEncodeTiled from the driver, found once through the runtime.
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

cudaError_t fused_forward(const __nv_bfloat16 *X, int64_t n, const __nv_bfloat16 *wc,
                          const float *params, float *y, int *err, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  // 32-bit row coordinates in the tensor copies; 16-byte aligned rows
  if (n > (int64_t)INT32_MAX - TM || (reinterpret_cast<uintptr_t>(X) & 15u) != 0)
    return cudaErrorInvalidValue;
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  // X [n][128] BF16 as a 2-D tensor; a box is 8 features x 128 rows (2 KB),
  // rows past n read as zero
  CUtensorMap map;
  const cuuint64_t dims[2] = {(cuuint64_t)FEATURES, (cuuint64_t)n};
  const cuuint64_t strides[1] = {(cuuint64_t)FEATURES * 2};
  const cuuint32_t box[2] = {8u, (cuuint32_t)TM};
  const cuuint32_t estr[2] = {1u, 1u};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(X), dims, strides,
          box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  int dev = 0, n_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(fused_forward_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             SMEM_BYTES);
  if (e != cudaSuccess) return e;
  const int64_t tiles = (n + TM - 1) / TM;
  const int grid = (int)(tiles < n_sm ? tiles : n_sm);
  fused_forward_kernel<<<grid, kThreads, SMEM_BYTES, s>>>(map, n, wc, params, y, err);
  return cudaGetLastError();
}

int canon_weight_elems() { return WC_L3 + HIDDEN * HIDDEN; }

template <int EPI>
static cudaError_t tc_gemm_launch(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *Bt,
                                  int ldb, int M, int k_split, int splits, const Epilogue &ep,
                                  int *err, cudaStream_t s) {
  // the shared-memory attribute once per device (also keeps it out of graph captures)
  static bool attr_set[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || !attr_set[dev]) {
    e = cudaFuncSetAttribute(tc_gemm_kernel<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             G_SMEM);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) attr_set[dev] = true;
  }
  // A [M][K] and Bt [256][K] (row strides lda, ldb) as 2-D tensors; a box is
  // 8 K values x 128 (A) or 64 (Bt) rows
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  if ((reinterpret_cast<uintptr_t>(A) & 15u) || (reinterpret_cast<uintptr_t>(Bt) & 15u))
    return cudaErrorInvalidValue;
  const cuuint64_t K = (cuuint64_t)k_split * splits;
  CUtensorMap ma, mb;
  const cuuint64_t da[2] = {K, (cuuint64_t)M}, db[2] = {K, (cuuint64_t)HIDDEN};
  const cuuint64_t sa[1] = {(cuuint64_t)lda * 2}, sb[1] = {(cuuint64_t)ldb * 2};
  const cuuint32_t ba[2] = {8u, 128u}, bb[2] = {8u, (cuuint32_t)GN}, es[2] = {1u, 1u};
  if (enc(&ma, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(A), da, sa, ba, es,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
      enc(&mb, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16 *>(Bt), db, sb, bb, es,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  tc_gemm_kernel<EPI><<<dim3(M / 128, splits, HIDDEN / GN), G_THREADS, G_SMEM, s>>>(
      ma, mb, k_split, ep, err);
  return cudaGetLastError();
}

cudaError_t tc_gemm_nt(const __nv_bfloat16 *A, int lda, const __nv_bfloat16 *Bt, int ldb, int M,
                       int K, int epi, const Epilogue &ep, int *err, cudaStream_t s) {
  if (M <= 0) return cudaSuccess;
  if (M % 128 || K % GK || K <= 0 || lda % 8 || ldb % 8) return cudaErrorInvalidValue;
  switch (epi) {
    case EPI_STORE_F32: return tc_gemm_launch<EPI_STORE_F32>(A, lda, Bt, ldb, M, K, 1, ep, err, s);
    case EPI_BIAS_GELU: return tc_gemm_launch<EPI_BIAS_GELU>(A, lda, Bt, ldb, M, K, 1, ep, err, s);
    case EPI_GELU_BWD: return tc_gemm_launch<EPI_GELU_BWD>(A, lda, Bt, ldb, M, K, 1, ep, err, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t transpose_bf16(const __nv_bfloat16 *in, int rows, int cols, __nv_bfloat16 *out,
                           cudaStream_t s) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  transpose_bf16_kernel<<<dim3((cols + 31) / 32, (rows + 31) / 32), dim3(32, 8), 0, s>>>(in, rows,
                                                                                       cols, out);
  return cudaGetLastError();
}

cudaError_t tc_gemm_tt_f32(const __nv_bfloat16 *at, const __nv_bfloat16 *bt, int M, int K, float *C,
                           float *scratch, int64_t scratch_elems, int *err, cudaStream_t s) {
  if (M <= 0) return cudaSuccess;
  if (M % 128 || K % GK || K <= 0) return cudaErrorInvalidValue;
  // enough K splits to give about 128 CTAs, each a multiple of the chunk
  int splits = 1;
  const int tiles = (M / 128) * (HIDDEN / GN);
  while (splits < 64 && tiles * splits < 128 && K % (GK * splits * 2) == 0 &&
         (int64_t)splits * 2 * M * HIDDEN <= scratch_elems)
    splits *= 2;
  Epilogue ep{};
  ep.ldc = HIDDEN;
  ep.c32 = splits > 1 ? scratch : C;
  ep.split_stride = (int64_t)M * HIDDEN;
  cudaError_t e = tc_gemm_launch<EPI_STORE_F32>(at, K, bt, K, M, K / splits, splits, ep, err, s);
  if (e != cudaSuccess || splits == 1) return e;
  const int64_t w = (int64_t)M * HIDDEN;
  sum_parts_kernel<<<(unsigned)((w + 255) / 256), 256, 0, s>>>(scratch, splits, w, C);
  return cudaGetLastError();
}

}  // namespace mlp
}  // namespace dk
