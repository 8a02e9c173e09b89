// The learned pre-screen of candidate poses: an MLP 128 -> 256 -> 256 -> 256
// -> 1 (GELU) on per-pose features, trained on the GPU by the kernels of
// mlp.cu on (features, exact score) pairs that the exact scorer produces.
// C ABI: dock_surrogate_* in include/dock.h.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <random>
#include <vector>

#include "handles.h"
#include "mlp.h"
#include "nvtx_range.h"

using namespace dk;
using dk::mlp::FEATURES;
using dk::mlp::HIDDEN;
using dk::mlp::N_PARAMS;

static int sfail(int st, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vset_error(st, fmt, ap);
  va_end(ap);
  return st;
}

#define SCU(call)                                                                   \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      int st_ = e_ == cudaErrorMemoryAllocation ? DOCK_ENOMEM : DOCK_ECUDA;         \
      return sfail(st_, "%s failed: %s", #call, cudaGetErrorString(e_));            \
    }                                                                               \
  } while (0)

namespace {
constexpr int kMaxTrainBatch = 65536;

// SplitMix64 output mix (Steele, Lea & Flood, OOPSLA 2014).
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Training visits its n rows in the order r -> pi(r): a keyed bijection of
// [0, n), a balanced four-round Feistel network on 2h-bit words (4^h >= n;
// Luby & Rackoff) with round keys K_i = mix64(seed + (i + 1) golden-ratio
// increment) and round function mix64(R ^ K_i) mod 2^h, restricted to
// [0, n) by cycle walking (Black & Rogaway): a value >= n is encrypted
// again. Each row's source is computed where it is gathered, so no order
// array is drawn on the host or copied.
struct TrainOrder {
  uint64_t n, mask, K[4];
  int h;
};

static TrainOrder make_train_order(uint64_t seed, uint64_t n) {
  TrainOrder o;
  o.n = n;
  o.h = 1;
  while ((1ULL << (2 * o.h)) < n) ++o.h;
  o.mask = (1ULL << o.h) - 1;
  for (int i = 0; i < 4; ++i) {
    uint64_t z = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    o.K[i] = z ^ (z >> 31);
  }
  return o;
}

__device__ __forceinline__ uint64_t train_row(const TrainOrder &o, uint64_t r) {
  uint64_t x = r;
  // a cycle of the permutation of [0, 4^h) through x returns below n
  for (uint64_t walk = 0; walk <= (o.mask + 1) * (o.mask + 1); ++walk) {
    uint64_t L = x >> o.h, R = x & o.mask;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const uint64_t t = L ^ (mix64(R ^ o.K[i]) & o.mask);
      L = R;
      R = t;
    }
    x = (L << o.h) | R;
    if (x < o.n) return x;
  }
  return o.n;  // unreachable: the row is then skipped (zeros)
}

// order[i] = pi(i) for i < n: the run's order of the training rows, made
// once so that a step's gather reads it instead of walking the permutation.
__global__ void train_order_kernel(TrainOrder o, int64_t n, int64_t *order) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    order[i] = (int64_t)train_row(o, (uint64_t)i);
}

// Gathers `rows` rows (r < rows_valid real, the rest zero) into the batch:
// row r is training row order[r0 + r] when order is given, else row r.
__global__ void gather_rows_kernel(const __nv_bfloat16 *X, const float *t, const int64_t *order,
                                   int64_t r0, const int64_t *r0_dev, int64_t n_src,
                                   int rows,
                                   int rows_valid, __nv_bfloat16 *Xb, float *tb, float t_mean,
                                   float t_inv_std, float t_clip) {
  // one warp per row: 128 bf16 = 256 bytes = 32 lanes x 8 bytes
  const int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (r >= rows) return;
  if (r0_dev) r0 = *r0_dev;  // graph-replayed step: the batch start lives on the device
  uint2 v = make_uint2(0, 0);
  float tv = 0.0f;
  if (r < rows_valid) {
    const int64_t src = order ? order[r0 + r] : r;
    if (src < n_src) {
      v = reinterpret_cast<const uint2 *>(X + src * FEATURES)[lane];
      if (t) tv = (fminf(t[src], t_clip) - t_mean) * t_inv_std;
    }
  }
  reinterpret_cast<uint2 *>(Xb + (int64_t)r * FEATURES)[lane] = v;
  if (lane == 0 && tb) tb[r] = tv;
}

// The device counters of a graph-replayed training step.
__global__ void set_counters_kernel(int64_t *r0, int64_t r0_value, int *step, int step_value) {
  *r0 = r0_value;
  *step = step_value;
}

// mean and sum of squares of min(t, clip) (double accumulation, one block)
__global__ void target_stats_kernel(const float *t, int64_t n, float clip, double *out) {
  __shared__ double s1[256], s2[256];
  double a = 0.0, b = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = fminf(t[i], clip);
    a += v;
    b += v * v;
  }
  s1[threadIdx.x] = a;
  s2[threadIdx.x] = b;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s1[threadIdx.x] += s1[threadIdx.x + o];
      s2[threadIdx.x] += s2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = s1[0];
    out[1] = s2[0];
  }
}

__global__ void destandardize_kernel(const float *y, int n, float mean, float std, float *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = y[i] * std + mean;
}
}  // namespace

struct dock_surrogate {
  int device = 0;
  float *p = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;   // FP32 masters, Adam, grads
  __nv_bfloat16 *w16[3] = {nullptr, nullptr, nullptr};            // W1..W3 [in][out]
  __nv_bfloat16 *wt16[3] = {nullptr, nullptr, nullptr};           // W1..W3 [out][in]
  // batch workspace
  int cap = 0;
  __nv_bfloat16 *X = nullptr, *H[3] = {nullptr, nullptr, nullptr}, *dZ[3] = {nullptr, nullptr, nullptr};
  float *Z[3] = {nullptr, nullptr, nullptr}, *y = nullptr, *t = nullptr, *part = nullptr,
        *outg = nullptr;
  // K-major copies of a weight gradient's operands (activations^T, dZ^T):
  // H_0^T, H_1^T and dZ_0^T, dZ_1^T written by the epilogues that make them,
  // X^T and dZ_2^T by transposes (into at, bt)
  __nv_bfloat16 *at = nullptr, *bt = nullptr;
  __nv_bfloat16 *Ht[2] = {nullptr, nullptr}, *dZt[2] = {nullptr, nullptr};
  double *stats = nullptr;
  int step = 0;
  int64_t *d_r0 = nullptr;  // batch start and Adam step of a graph-replayed training step
  int *d_step = nullptr;
  cudaStream_t ts = nullptr;  // training runs (and its step graph is captured) on this stream
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // the backward pass's weight gradients (ts_w[l], one stream per layer, each
  // with its own split-K scratch) and bias gradients (ts_c) run
  // beside its chain of input gradients, forked and joined by events
  cudaStream_t ts_w[3] = {nullptr, nullptr, nullptr}, ts_c = nullptr;
  cudaEvent_t ev_dz[3] = {nullptr, nullptr, nullptr}, ev_w[3] = {nullptr, nullptr, nullptr},
              ev_c = nullptr, ev_x = nullptr;
  float *cpart = nullptr;  // column-sum partials of the bias gradients
  int64_t *order = nullptr;  // the training rows' order for the current run
  int64_t order_cap = 0;
  float t_mean = 0.0f, t_std = 1.0f, t_clip = 1e30f;
  // weights of the fused tensor-core forward pass (refreshed lazily after the
  // FP32 masters change) and its device error flag
  __nv_bfloat16 *wc = nullptr;
  bool wc_valid = false;
  int *err = nullptr;
  float *wpart = nullptr;  // split-K partial weight gradients, one region per layer
  float *ydot = nullptr;   // the output layer's partial dot products [8][rows]
  unsigned *ticket = nullptr;  // blocks of a replayed step's Adam kernel that are done
  ~dock_surrogate() {
    for (float *q : {p, m, v, g, y, t, part, outg}) if (q) cudaFree(q);
    if (wc) cudaFree(wc);
    if (err) cudaFree(err);
    if (wpart) cudaFree(wpart);
    if (ydot) cudaFree(ydot);
    if (ticket) cudaFree(ticket);
    if (d_r0) cudaFree(d_r0);
    if (d_step) cudaFree(d_step);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    for (cudaEvent_t e : {ev_dz[0], ev_dz[1], ev_dz[2], ev_w[0], ev_w[1], ev_w[2], ev_c, ev_x})
      if (e) cudaEventDestroy(e);
    if (ts) cudaStreamDestroy(ts);
    for (cudaStream_t q : {ts_w[0], ts_w[1], ts_w[2]}) if (q) cudaStreamDestroy(q);
    if (ts_c) cudaStreamDestroy(ts_c);
    if (cpart) cudaFree(cpart);
    if (order) cudaFree(order);
    for (int l = 0; l < 3; ++l) {
      if (w16[l]) cudaFree(w16[l]);
      if (wt16[l]) cudaFree(wt16[l]);
      if (H[l]) cudaFree(H[l]);
      if (dZ[l]) cudaFree(dZ[l]);
      if (Z[l]) cudaFree(Z[l]);
    }
    if (X) cudaFree(X);
    if (at) cudaFree(at);
    if (bt) cudaFree(bt);
    for (int l = 0; l < 2; ++l) {
      if (Ht[l]) cudaFree(Ht[l]);
      if (dZt[l]) cudaFree(dZt[l]);
    }
    if (stats) cudaFree(stats);
  }
};

static const int kIn[3] = {FEATURES, HIDDEN, HIDDEN};
static const int kOffW[3] = {mlp::OFF_W1, mlp::OFF_W2, mlp::OFF_W3};
static const int kOffB[3] = {mlp::OFF_B1, mlp::OFF_B2, mlp::OFF_B3};
static const int kBwdBlocks = 512;
// split-K partials of one layer's weight gradient: 16 splits of 256 x 256 or
// 32 of 128 x 256 (128 CTAs per product); one region per layer
static const int64_t kWpartElems = 16 * HIDDEN * HIDDEN;

static int ensure_workspace(dock_surrogate *S, int rows) {
  if (rows <= S->cap) return DOCK_OK;
  if (S->X) cudaFree(S->X);
  if (S->at) cudaFree(S->at);
  if (S->bt) cudaFree(S->bt);
  S->at = S->bt = nullptr;
  for (int l = 0; l < 2; ++l) {
    if (S->Ht[l]) cudaFree(S->Ht[l]);
    if (S->dZt[l]) cudaFree(S->dZt[l]);
    S->Ht[l] = S->dZt[l] = nullptr;
  }
  for (int l = 0; l < 3; ++l) {
    if (S->H[l]) cudaFree(S->H[l]);
    if (S->dZ[l]) cudaFree(S->dZ[l]);
    if (S->Z[l]) cudaFree(S->Z[l]);
    S->H[l] = S->dZ[l] = nullptr;
    S->Z[l] = nullptr;
  }
  for (float **q : {&S->y, &S->t, &S->ydot}) {
    if (*q) cudaFree(*q);
    *q = nullptr;
  }
  S->cap = 0;
  SCU(cudaMalloc(&S->X, sizeof(__nv_bfloat16) * (size_t)rows * FEATURES));
  SCU(cudaMalloc(&S->at, sizeof(__nv_bfloat16) * (size_t)rows * HIDDEN));
  SCU(cudaMalloc(&S->bt, sizeof(__nv_bfloat16) * (size_t)rows * HIDDEN));
  for (int l = 0; l < 2; ++l) {
    SCU(cudaMalloc(&S->Ht[l], sizeof(__nv_bfloat16) * (size_t)rows * HIDDEN));
    SCU(cudaMalloc(&S->dZt[l], sizeof(__nv_bfloat16) * (size_t)rows * HIDDEN));
  }
  for (int l = 0; l < 3; ++l) {
    SCU(cudaMalloc(&S->H[l], sizeof(__nv_bfloat16) * (size_t)rows * HIDDEN));
    SCU(cudaMalloc(&S->dZ[l], sizeof(__nv_bfloat16) * (size_t)rows * HIDDEN));
    SCU(cudaMalloc(&S->Z[l], sizeof(float) * (size_t)rows * HIDDEN));
  }
  SCU(cudaMalloc(&S->y, sizeof(float) * rows));
  SCU(cudaMalloc(&S->ydot, sizeof(float) * 8 * (size_t)rows));
  SCU(cudaMalloc(&S->t, sizeof(float) * rows));
  S->cap = rows;
  return DOCK_OK;
}

static int refresh_bf16(dock_surrogate *S, cudaStream_t s) {
  for (int l = 0; l < 3; ++l)
    SCU(mlp::cast_weights(S->p + kOffW[l], kIn[l], HIDDEN, S->w16[l], S->wt16[l], s));
  S->wc_valid = false;
  return DOCK_OK;
}

// Forward pass of `rows` rows already in S->X (rows a multiple of 128), the
// three hidden layers on the tensor cores (tcgen05). keep = true keeps FP32
// pre-activations for the backward pass.
static int forward(dock_surrogate *S, int rows, bool keep, cudaStream_t s) {
  const __nv_bfloat16 *in = S->X;
  for (int l = 0; l < 3; ++l) {
    mlp::Epilogue ep{};
    ep.c32 = keep ? S->Z[l] : nullptr;
    ep.c16 = S->H[l];
    ep.c16t = keep && l < 2 ? S->Ht[l] : nullptr;  // the next layer's weight gradient reads H_l^T
    ep.ldt = rows;
    if (l == 2) {  // the output layer as eight partial dot products per row
      ep.ydot = S->ydot;
      ep.w4 = S->p + mlp::OFF_W4;
      ep.ldy = rows;
    }
    ep.bias = S->p + kOffB[l];
    ep.ldc = HIDDEN;
    SCU(mlp::tc_gemm_nt(in, kIn[l], S->wt16[l], kIn[l], rows, kIn[l], mlp::EPI_BIAS_GELU, ep,
                        S->err, s));
    in = S->H[l];
  }
  return DOCK_OK;
}

// Gradients of loss = mean over the first n rows of (y - t)^2 into S->g
// (rows >= n padded: contribute nothing). Needs forward(keep = true). The
// chain dZ_2 -> dZ_1 -> dZ_0 runs on s; each layer's weight gradient (on
// ts_w[l]) and bias gradient (on ts_c) start once its dZ is written, and s waits
// for both before it returns (also inside a captured step graph).
static int backward(dock_surrogate *S, int rows, int n, cudaStream_t s) {
  // X^T for the first layer's weight gradient, on its side stream while the
  // input-gradient chain runs (X is final once the forward pass is queued)
  SCU(cudaEventRecord(S->ev_x, s));
  SCU(cudaStreamWaitEvent(S->ts_w[0], S->ev_x, 0));
  SCU(mlp::transpose_bf16(S->X, rows, FEATURES, S->at, S->ts_w[0]));
  // dW4 and db4 straight into the gradient, the loss into outg[HIDDEN + 1]
  SCU(mlp::out_layer_bwd(S->y, S->ydot, S->p + mlp::OFF_B4, S->t, n, rows, S->H[2], S->Z[2],
                         S->p + mlp::OFF_W4, S->dZ[2], S->part, kBwdBlocks, S->g + mlp::OFF_W4,
                         S->outg + HIDDEN + 1, s));
  for (int l = 2; l >= 0; --l) {
    SCU(cudaEventRecord(S->ev_dz[l], s));
    SCU(cudaStreamWaitEvent(S->ts_w[l], S->ev_dz[l], 0));
    SCU(cudaStreamWaitEvent(S->ts_c, S->ev_dz[l], 0));
    // dW_l = act_in^T dZ_l (tensor cores, K = rows split over CTAs) from
    // K-major copies: H_{l-1}^T and dZ_l^T from the epilogues, X^T (above) and
    // dZ_2^T transposed here
    const __nv_bfloat16 *at = l ? S->Ht[l - 1] : S->at, *bt = l < 2 ? S->dZt[l] : S->bt;
    if (l == 2) SCU(mlp::transpose_bf16(S->dZ[2], rows, HIDDEN, S->bt, S->ts_w[2]));
    SCU(mlp::tc_gemm_tt_f32(at, bt, kIn[l], rows, S->g + kOffW[l], S->wpart + l * kWpartElems,
                            kWpartElems, S->err, S->ts_w[l]));
    // db_l = column sums of dZ_l
    SCU(mlp::colsum(S->dZ[l], rows, HIDDEN, S->g + kOffB[l], S->cpart, S->ts_c));
    if (l) {
      // dZ_{l-1} = (dZ_l W_l^T) * gelu'(Z_{l-1})
      mlp::Epilogue ep{};
      ep.c16 = S->dZ[l - 1];
      ep.c16t = S->dZt[l - 1];
      ep.ldt = rows;
      ep.zin = S->Z[l - 1];
      ep.ldc = HIDDEN;
      SCU(mlp::tc_gemm_nt(S->dZ[l], HIDDEN, S->w16[l], HIDDEN, rows, HIDDEN, mlp::EPI_GELU_BWD,
                          ep, S->err, s));
    }
  }
  for (int l = 0; l < 3; ++l) SCU(cudaEventRecord(S->ev_w[l], S->ts_w[l]));
  SCU(cudaEventRecord(S->ev_c, S->ts_c));
  for (int l = 0; l < 3; ++l) SCU(cudaStreamWaitEvent(s, S->ev_w[l], 0));
  SCU(cudaStreamWaitEvent(s, S->ev_c, 0));
  return DOCK_OK;
}

// Waits for the stream; DOCK_EDEVICE (flag cleared) if a tensor-core kernel's
// bounded device wait ran out since the last check.
static int check_device_flag(dock_surrogate *S, cudaStream_t s, const char *what) {
  int flag = 0;
  SCU(cudaMemcpyAsync(&flag, S->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  SCU(cudaStreamSynchronize(s));
  if (flag) {
    SCU(cudaMemsetAsync(S->err, 0, sizeof(int), s));
    return sfail(DOCK_EDEVICE, "%s: a device wait ran out (results incomplete)", what);
  }
  return DOCK_OK;
}

extern "C" int dock_surrogate_create(uint64_t seed, void *stream, dock_surrogate **out) {
  if (!out) return sfail(DOCK_EINVAL, "dock_surrogate_create: NULL out");
  *out = nullptr;
  std::unique_ptr<dock_surrogate> S(new dock_surrogate());
  SCU(cudaGetDevice(&S->device));
  cudaStream_t s = (cudaStream_t)stream;
  for (float **q : {&S->p, &S->m, &S->v, &S->g}) SCU(cudaMalloc(q, sizeof(float) * N_PARAMS));
  SCU(cudaMalloc(&S->part, sizeof(float) * kBwdBlocks * (HIDDEN + 2)));
  SCU(cudaMalloc(&S->outg, sizeof(float) * (HIDDEN + 2)));
  SCU(cudaMalloc(&S->stats, sizeof(double) * 2));
  for (int l = 0; l < 3; ++l) {
    SCU(cudaMalloc(&S->w16[l], sizeof(__nv_bfloat16) * kIn[l] * HIDDEN));
    SCU(cudaMalloc(&S->wt16[l], sizeof(__nv_bfloat16) * kIn[l] * HIDDEN));
  }
  SCU(cudaMalloc(&S->wc, sizeof(__nv_bfloat16) * mlp::canon_weight_elems()));
  SCU(cudaMalloc(&S->wpart, sizeof(float) * 3 * kWpartElems));
  SCU(cudaMalloc(&S->ticket, sizeof(unsigned)));
  SCU(cudaMemsetAsync(S->ticket, 0, sizeof(unsigned), s));
  SCU(cudaMalloc(&S->err, sizeof(int)));
  SCU(cudaMalloc(&S->d_r0, sizeof(int64_t)));
  SCU(cudaStreamCreateWithFlags(&S->ts, cudaStreamNonBlocking));
  for (int l = 0; l < 3; ++l) SCU(cudaStreamCreateWithFlags(&S->ts_w[l], cudaStreamNonBlocking));
  SCU(cudaStreamCreateWithFlags(&S->ts_c, cudaStreamNonBlocking));
  for (cudaEvent_t *e : {&S->ev_dz[0], &S->ev_dz[1], &S->ev_dz[2], &S->ev_w[0], &S->ev_w[1],
                         &S->ev_w[2], &S->ev_c, &S->ev_x})
    SCU(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  SCU(cudaMalloc(&S->cpart, sizeof(float) * mlp::kColsumChunks * HIDDEN));
  SCU(cudaEventCreateWithFlags(&S->ev_in, cudaEventDisableTiming));
  SCU(cudaEventCreateWithFlags(&S->ev_out, cudaEventDisableTiming));
  SCU(cudaMalloc(&S->d_step, sizeof(int)));
  SCU(cudaMemsetAsync(S->err, 0, sizeof(int), s));
  // He-normal weights, zero biases (host draw from the seed, one upload)
  std::vector<float> h(N_PARAMS, 0.0f);
  std::mt19937_64 rng(seed);
  for (int l = 0; l < 3; ++l) {
    std::normal_distribution<float> nd(0.0f, std::sqrt(2.0f / kIn[l]));
    for (int i = 0; i < kIn[l] * HIDDEN; ++i) h[kOffW[l] + i] = nd(rng);
  }
  std::normal_distribution<float> nd4(0.0f, std::sqrt(1.0f / HIDDEN));
  for (int i = 0; i < HIDDEN; ++i) h[mlp::OFF_W4 + i] = nd4(rng);
  SCU(cudaMemcpyAsync(S->p, h.data(), sizeof(float) * N_PARAMS, cudaMemcpyHostToDevice, s));
  SCU(cudaMemsetAsync(S->m, 0, sizeof(float) * N_PARAMS, s));
  SCU(cudaMemsetAsync(S->v, 0, sizeof(float) * N_PARAMS, s));
  int st = refresh_bf16(S.get(), s);
  if (st != DOCK_OK) return st;
  SCU(cudaStreamSynchronize(s));
  *out = S.release();
  return DOCK_OK;
}

extern "C" void dock_surrogate_destroy(dock_surrogate *S) { delete S; }

extern "C" int dock_surrogate_set_params(dock_surrogate *S, const float *params, float t_mean,
                                         float t_std, float t_clip, void *stream) {
  if (!S || !params) return sfail(DOCK_EINVAL, "dock_surrogate_set_params: NULL argument");
  if (!(t_std > 0.0f)) return sfail(DOCK_EINVAL, "dock_surrogate_set_params: t_std <= 0");
  SCU(cudaSetDevice(S->device));
  cudaStream_t s = (cudaStream_t)stream;
  SCU(cudaMemcpyAsync(S->p, params, sizeof(float) * N_PARAMS, cudaMemcpyHostToDevice, s));
  S->t_mean = t_mean;
  S->t_std = t_std;
  S->t_clip = t_clip;
  int st = refresh_bf16(S, s);
  if (st != DOCK_OK) return st;
  SCU(cudaStreamSynchronize(s));
  return DOCK_OK;
}

extern "C" int dock_surrogate_get_params(const dock_surrogate *S, float *params, float *t_mean,
                                         float *t_std, float *t_clip) {
  if (!S) return sfail(DOCK_EINVAL, "dock_surrogate_get_params: NULL surrogate");
  SCU(cudaSetDevice(S->device));
  if (params) SCU(cudaMemcpy(params, S->p, sizeof(float) * N_PARAMS, cudaMemcpyDeviceToHost));
  if (t_mean) *t_mean = S->t_mean;
  if (t_std) *t_std = S->t_std;
  if (t_clip) *t_clip = S->t_clip;
  return DOCK_OK;
}

int dk_surrogate_predict_raw(dock_surrogate *S, const uint16_t *features, int64_t n, float *out,
                             int destandardize, cudaStream_t s) {
  if (n <= 0) return DOCK_OK;
  const __nv_bfloat16 *F = reinterpret_cast<const __nv_bfloat16 *>(features);
  if (!S->wc_valid) {
    SCU(mlp::canon_weights(S->p, S->wc, s));
    S->wc_valid = true;
  }
  SCU(cudaMemsetAsync(out, 0xFF, sizeof(float) * n, s));  // NaN in rows a failed tile skips
  SCU(mlp::fused_forward(F, n, S->wc, S->p, out, S->err, s));
  if (destandardize) {
    destandardize_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, (int)n, S->t_mean,
                                                                      S->t_std, out);
    SCU(cudaGetLastError());
  }
  return DOCK_OK;
}

extern "C" int dock_surrogate_predict(dock_surrogate *S, const uint16_t *features, int64_t n,
                                      float *out, void *stream) {
  const dk::NvtxRange nvtx_range("dock_surrogate_predict");
  if (!S || (n > 0 && (!features || !out))) return sfail(DOCK_EINVAL, "dock_surrogate_predict: NULL");
  if (n < 0 || n > INT32_MAX) return sfail(DOCK_EINVAL, "dock_surrogate_predict: n out of range");
  if ((reinterpret_cast<uintptr_t>(features) & 15) != 0)
    return sfail(DOCK_EINVAL, "dock_surrogate_predict: features not 16-byte aligned");
  SCU(cudaSetDevice(S->device));
  cudaStream_t s = (cudaStream_t)stream;
  int st = dk_surrogate_predict_raw(S, features, n, out, 1, s);
  if (st != DOCK_OK) return st;
  int flag = 0;
  SCU(cudaMemcpyAsync(&flag, S->err, sizeof(int), cudaMemcpyDeviceToHost, s));
  SCU(cudaStreamSynchronize(s));
  if (flag) {
    SCU(cudaMemsetAsync(S->err, 0, sizeof(int), s));
    return sfail(DOCK_EDEVICE, "dock_surrogate_predict: a device wait ran out (rows left NaN)");
  }
  return DOCK_OK;
}

extern "C" int dock_surrogate_gradients(dock_surrogate *S, const uint16_t *features,
                                        const float *targets, int32_t n, float *grad, float *loss,
                                        void *stream) {
  const dk::NvtxRange nvtx_range("dock_surrogate_gradients");
  if (!S || !features || !targets || !grad) return sfail(DOCK_EINVAL, "dock_surrogate_gradients: NULL");
  if (n < 1 || n > kMaxTrainBatch) return sfail(DOCK_EINVAL, "dock_surrogate_gradients: n %d", n);
  SCU(cudaSetDevice(S->device));
  cudaStream_t s = (cudaStream_t)stream;
  const int rows = (n + 127) / 128 * 128;
  int st = ensure_workspace(S, rows);
  if (st != DOCK_OK) return st;
  // targets used as given (identity standardisation)
  gather_rows_kernel<<<(rows * 32 + 255) / 256, 256, 0, s>>>(
      reinterpret_cast<const __nv_bfloat16 *>(features), targets, nullptr, 0, nullptr, n,
      rows, n, S->X, S->t, 0.0f, 1.0f, 3.0e38f);
  SCU(cudaGetLastError());
  if ((st = forward(S, rows, true, s)) != DOCK_OK) return st;
  if ((st = backward(S, rows, n, s)) != DOCK_OK) return st;
  SCU(cudaMemcpyAsync(grad, S->g, sizeof(float) * N_PARAMS, cudaMemcpyDeviceToDevice, s));
  if ((st = check_device_flag(S, s, "dock_surrogate_gradients")) != DOCK_OK) return st;
  if (loss) {
    SCU(cudaStreamSynchronize(s));
    float ls = 0.0f;
    SCU(cudaMemcpy(&ls, S->outg + HIDDEN + 1, sizeof(float), cudaMemcpyDeviceToHost));
    *loss = ls / n;
  }
  return DOCK_OK;
}

extern "C" int dock_surrogate_train(dock_surrogate *S, const uint16_t *features, const float *scores,
                                    int64_t n, const dock_train_params *tp, float *loss_per_epoch,
                                    void *stream) {
  const dk::NvtxRange nvtx_range("dock_surrogate_train");
  if (!S || !features || !scores || !tp) return sfail(DOCK_EINVAL, "dock_surrogate_train: NULL");
  if (n < 2 || tp->epochs < 1 || tp->batch < 128 || tp->batch > kMaxTrainBatch || tp->batch % 128 ||
      !(tp->lr > 0.0f))
    return sfail(DOCK_EINVAL, "dock_surrogate_train: bad sizes or learning rate");
  SCU(cudaSetDevice(S->device));
  // the work runs on the surrogate's own stream, ordered after the caller's
  // stream and before its later work (a graph can be captured there even
  // when the caller passes the legacy default stream)
  cudaStream_t caller = (cudaStream_t)stream, s = S->ts;
  SCU(cudaEventRecord(S->ev_in, caller));
  SCU(cudaStreamWaitEvent(s, S->ev_in, 0));
  int st = ensure_workspace(S, tp->batch);
  if (st != DOCK_OK) return st;
  // target standardisation over the training set: min(score, clip), then mean / std
  const float clip = tp->score_clip;
  target_stats_kernel<<<1, 256, 0, s>>>(scores, n, clip, S->stats);
  SCU(cudaGetLastError());
  double st2[2];
  SCU(cudaMemcpyAsync(st2, S->stats, sizeof st2, cudaMemcpyDeviceToHost, s));
  SCU(cudaStreamSynchronize(s));
  const double mean = st2[0] / n, var = std::max(st2[1] / n - mean * mean, 1e-12);
  S->t_mean = (float)mean;
  S->t_std = (float)std::sqrt(var);
  S->t_clip = clip;
  // one order of the rows for the run, keyed by the seed (the same every epoch)
  const TrainOrder ord = make_train_order(tp->seed, (uint64_t)n);
  if (S->order_cap < n) {
    if (S->order) cudaFree(S->order);
    S->order = nullptr;
    S->order_cap = 0;
    SCU(cudaMalloc(&S->order, sizeof(int64_t) * (size_t)n));
    S->order_cap = n;
  }
  train_order_kernel<<<152 * 8, 256, 0, s>>>(ord, n, S->order);
  SCU(cudaGetLastError());
  const __nv_bfloat16 *F = reinterpret_cast<const __nv_bfloat16 *>(features);
  const int B = tp->batch;
  const int64_t steps_per_epoch = (n + B - 1) / B;
  // one training step: gather, forward, backward, Adam, BF16 weight copies.
  // dev: the batch start and the Adam step are read from the device counters
  // (the form captured in a CUDA graph; the graph's last kernel advances them)
  auto step_body = [&](int64_t r0, int valid, bool dev) -> int {
    const int rows = (valid + 127) / 128 * 128;
    gather_rows_kernel<<<(rows * 32 + 255) / 256, 256, 0, s>>>(
        F, scores, S->order, r0, dev ? S->d_r0 : nullptr, n, rows, valid, S->X, S->t, S->t_mean,
        1.0f / S->t_std, clip);
    SCU(cudaGetLastError());
    int rc;
    if ((rc = forward(S, rows, true, s)) != DOCK_OK) return rc;
    if ((rc = backward(S, rows, valid, s)) != DOCK_OK) return rc;
    // Adam writes the BF16 copies the next step's products read
    mlp::WeightCopies wcp;
    for (int l = 0; l < 3; ++l) {
      wcp.w16[l] = S->w16[l];
      wcp.wt16[l] = S->wt16[l];
    }
    // replayed form: Adam's last block also advances the batch start and the step
    SCU(mlp::adam(S->p, S->m, S->v, S->g, N_PARAMS, tp->lr, S->step + 1, dev ? S->d_step : nullptr,
                  &wcp, dev ? S->d_r0 : nullptr, B, S->ticket, s));
    S->wc_valid = false;  // the prediction's tensor-core layout is rebuilt when next needed
    return DOCK_OK;
  };
  // full batches replay one captured graph of the step (captured at the first)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  auto release = [&]() {
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    gexec = nullptr;
    graph = nullptr;
  };
  for (int ep = 0; ep < tp->epochs; ++ep) {
    double ep_loss = 0.0;
    for (int64_t b = 0; b < steps_per_epoch; ++b) {
      const int64_t r0 = b * B;
      const int valid = (int)std::min<int64_t>(B, n - r0);
      if (valid == B) {
        if (b == 0 || !gexec) {  // counters for this epoch's run of full batches
          set_counters_kernel<<<1, 1, 0, s>>>(S->d_r0, r0, S->d_step, S->step + 1);
          SCU(cudaGetLastError());
        }
        if (!gexec) {
          SCU(cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
          st = step_body(r0, valid, true);
          cudaError_t ce = cudaStreamEndCapture(s, &graph);
          if (st != DOCK_OK) {
            release();
            return st;
          }
          if (ce == cudaSuccess) ce = cudaGraphInstantiate(&gexec, graph, 0);
          if (ce != cudaSuccess) {
            release();
            return sfail(DOCK_ECUDA, "dock_surrogate_train: step graph: %s", cudaGetErrorString(ce));
          }
        }
        cudaError_t le = cudaGraphLaunch(gexec, s);
        if (le != cudaSuccess) {
          release();
          return sfail(DOCK_ECUDA, "dock_surrogate_train: %s", cudaGetErrorString(le));
        }
        ++S->step;
      } else {
        if ((st = step_body(r0, valid, false)) != DOCK_OK) {
          release();
          return st;
        }
        ++S->step;
      }
      if (loss_per_epoch && (b == steps_per_epoch - 1 || (b & 63) == 0)) {
        float ls = 0.0f;
        cudaError_t ce = cudaMemcpyAsync(&ls, S->outg + HIDDEN + 1, sizeof(float),
                                         cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        if (ce != cudaSuccess) {
          release();
          return sfail(DOCK_ECUDA, "dock_surrogate_train: %s", cudaGetErrorString(ce));
        }
        ep_loss = ls / valid;
      }
    }
    if (loss_per_epoch) loss_per_epoch[ep] = (float)ep_loss;
  }
  release();
  SCU(cudaEventRecord(S->ev_out, s));
  SCU(cudaStreamWaitEvent(caller, S->ev_out, 0));
  return check_device_flag(S, s, "dock_surrogate_train");
}
