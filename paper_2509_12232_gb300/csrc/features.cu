// Surrogate pre-screen kernels: pose features of given genotypes or of GA
// candidates, per-ligand top-k of the predictions, and the mu + lambda merge
// of population and exactly scored candidates.
#include <cuda_bf16.h>

#include "surrogate_kernels.h"
#include "pose.cuh"

namespace dk {

namespace {
constexpr int kFeatL = 8;         // lanes per pose
constexpr int kFeatThreads = 128;
constexpr int kFeatSlots = kFeatThreads / kFeatL;
constexpr int kFeatApl = DOCK_MAX_ATOMS / kFeatL;
// shared feature rows kFeatRow floats apart: the rows of the four poses of a
// warp start 8 banks apart, so a warp's lane-indexed writes do not collide
constexpr int kFeatRow = DOCK_N_FEATURES + 8;

__device__ __forceinline__ float sel16(const float (&g)[DOCK_MAX_GENES], int j) {
  float v = 0.0f;
#pragma unroll
  for (int jj = 0; jj < DOCK_MAX_TORSIONS; ++jj)
    if (jj == j) v = g[7 + jj];
  return v;
}

// Features of the pose in `slot` by the 8 lanes of a group, into the
// group's shared row f[128] (FP32), deterministic: the (type, shell) counts
// by integer shared-memory atomics (exact in any order), the shell sums of q
// and |q| per lane in atom order, then over the lanes by a fixed shuffle tree.
__device__ __forceinline__ void pose_features(const float (&g)[DOCK_MAX_GENES], const LigView &V,
                                              const float4 *slot, int lane, unsigned gmask,
                                              float cx, float cy, float cz, float radius, float *f) {
  const float inv_w = 8.0f / radius;
  int *hist = reinterpret_cast<int *>(f);  // f[0..55] hold the counts until converted
#pragma unroll
  for (int i = 0; i < 7; ++i) hist[i * 8 + lane] = 0;
  __syncwarp(gmask);
  float qs[8], aqs[8];
#pragma unroll
  for (int s = 0; s < 8; ++s) qs[s] = aqs[s] = 0.0f;
  for (int a = lane; a < V.n; a += kFeatL) {
    const float4 p = slot[a];
    const float dx = p.x - cx, dy = p.y - cy, dz = p.z - cz;
    const int sh = min((int)(sqrtf(dx * dx + dy * dy + dz * dz) * inv_w), 7);
    const int t = V.types[a];
    if (t < 7) atomicAdd(&hist[t * 8 + sh], 1);
    const float q = __ldg(&V.atoms[a].w);
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      if (sh == s) {
        qs[s] += q;
        aqs[s] += fabsf(q);
      }
    }
  }
  // lane s ends with shell s's sums (the same tree for every shell)
  float myq = 0.0f, myaq = 0.0f;
#pragma unroll
  for (int s = 0; s < 8; ++s) {
    float v = qs[s], av = aqs[s];
#pragma unroll
    for (int o = 1; o < kFeatL; o <<= 1) {
      v += __shfl_xor_sync(gmask, v, o);
      av += __shfl_xor_sync(gmask, av, o);
    }
    if (s == lane) {
      myq = v;
      myaq = av;
    }
  }
  __syncwarp(gmask);
#pragma unroll
  for (int i = 0; i < 7; ++i) f[i * 8 + lane] = (float)hist[i * 8 + lane] * 0.125f;
  f[56 + lane] = myq;
  f[64 + lane] = myaq;
  // torsions: lane j writes slots j and j + 8
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int j = lane + h * 8;
    float s = 0.0f, c = 0.0f;
    if (j < V.k) sincosf(sel16(g, j), &s, &c);
    f[72 + 2 * j] = s;
    f[73 + 2 * j] = c;
  }
  if (lane == 0) {
    float qw = g[3], qx = g[4], qy = g[5], qz = g[6];
    const float inv = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
    qw *= inv; qx *= inv; qy *= inv; qz *= inv;
    f[104] = 1.f - 2.f * (qy * qy + qz * qz); f[105] = 2.f * (qx * qy - qw * qz);
    f[106] = 2.f * (qx * qz + qw * qy);       f[107] = 2.f * (qx * qy + qw * qz);
    f[108] = 1.f - 2.f * (qx * qx + qz * qz); f[109] = 2.f * (qy * qz - qw * qx);
    f[110] = 2.f * (qx * qz - qw * qy);       f[111] = 2.f * (qy * qz + qw * qx);
    f[112] = 1.f - 2.f * (qx * qx + qy * qy);
    f[113] = g[0] / radius;
    f[114] = g[1] / radius;
    f[115] = g[2] / radius;
    f[116] = (float)V.n / 100.0f;
    f[117] = (float)V.k / 16.0f;
  }
  if (lane >= 1 && lane <= 7) f[117 + lane] = 0.0f;  // 118..124
  if (lane < 3) f[125 + lane] = 0.0f;               // 125..127
}

struct FeatArgs {
  const LigInfo *ligs;
  const float4 *atoms;
  const uint8_t *types;
  const float *pair_rec;
  const TorInfo *tors;
  const uint8_t *moves;
  GridView grid;
  float cx, cy, cz, radius;
  int32_t n_ligands;
  // given genotypes
  int32_t pop_csr;
  const int32_t *pose_ligand;
  const float *genos;            // [n][DOCK_MAX_GENES]
  int64_t n_poses;
  float *scores;                 // optional exact scores
  // GA candidates
  int32_t pop, candidates, gen;
  uint64_t seed, thr_cross, thr_mut;
  const float *geno_prev;
  const float *score_prev;
  const int64_t *geno_off;
  float *cand_geno;              // [n_ligands * candidates][DOCK_MAX_GENES]
  __nv_bfloat16 *features;       // [rows][128]
};

template <bool FROM_GA>
__global__ void __launch_bounds__(kFeatThreads) feat_kernel(const FeatArgs A) {
  __shared__ float4 s_col[slots_bytes(kFeatThreads, kFeatL, kFeatApl) / 16];
  __shared__ __align__(16) float s_f[kFeatSlots][kFeatRow];
  const int lane = threadIdx.x & (kFeatL - 1), slot = threadIdx.x / kFeatL;
  int lig;
  int64_t row;
  float g[DOCK_MAX_GENES];
  if (FROM_GA) {
    lig = blockIdx.y;
    const int c = blockIdx.x * kFeatSlots + slot;
    if (c >= A.candidates) return;
    row = (int64_t)lig * A.candidates + c;
    const LigInfo li = A.ligs[lig];
    ga_child_group<kFeatL>(g, li.k, A.pop, A.geno_prev + A.geno_off[lig],
                           A.score_prev + (int64_t)lig * A.pop, A.thr_cross, A.thr_mut, A.seed,
                           li.ligand_id, (uint32_t)A.gen, (uint32_t)c, lane,
                           group_mask<kFeatL>());
    float *out = A.cand_geno + row * DOCK_MAX_GENES;
#pragma unroll
    for (int e = 0; e < DOCK_MAX_GENES; ++e)
      if ((e & (kFeatL - 1)) == lane) out[e] = g[e];
  } else {
    row = (int64_t)blockIdx.x * kFeatSlots + slot;
    if (row >= A.n_poses) return;
    const float *src;
    if (A.pop_csr > 0) {
      lig = (int)(row / A.pop_csr);
      src = A.genos + A.geno_off[lig] + (row % A.pop_csr) * (7 + A.ligs[lig].k);
    } else {
      lig = A.pose_ligand[row];
      if (lig < 0 || lig >= A.n_ligands) {
        if (A.scores && lane == 0) A.scores[row] = __int_as_float(0x7fc00000);
        return;
      }
      src = A.genos + row * DOCK_MAX_GENES;
    }
    const int G = 7 + A.ligs[lig].k;
#pragma unroll
    for (int e = 0; e < DOCK_MAX_GENES; ++e) g[e] = e < G ? src[e] : 0.0f;
  }
  const LigInfo li = A.ligs[lig];
  const LigView V = lig_view(li, A.atoms, A.types, A.pair_rec, A.tors);
  const unsigned gmask = group_mask<kFeatL>();
  float4 *sl = s_col + slot * slot_stride(kFeatL, kFeatApl);
  apply_pose<kFeatL>(g, V, A.moves, A.cx, A.cy, A.cz, sl, lane, gmask);
  float *f = s_f[slot];
  pose_features(g, V, sl, lane, gmask, A.cx, A.cy, A.cz, A.radius, f);
  __syncwarp(gmask);
  // 128 values -> BF16: lane l converts the four-value chunks l + 8 m (one
  // 16-byte shared read each, the group's eight reads on distinct banks) and
  // stores them as 8-byte pieces (64 contiguous bytes per group and m)
  __nv_bfloat16 *out = A.features + row * DOCK_N_FEATURES;
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int c = lane + 8 * m;
    const float4 v = *reinterpret_cast<const float4 *>(f + 4 * c);
    const __nv_bfloat162 h0 = __floats2bfloat162_rn(v.x, v.y), h1 = __floats2bfloat162_rn(v.z, v.w);
    reinterpret_cast<uint2 *>(out)[c] = make_uint2(*reinterpret_cast<const uint32_t *>(&h0),
                                                   *reinterpret_cast<const uint32_t *>(&h1));
  }
  if (!FROM_GA && A.scores) {
    const float sc = score_posed<kFeatL>(V, A.grid, sl, lane, gmask, nullptr);
    if (lane == 0) A.scores[row] = sc;
  }
}

// Bitonic sort of n (power of two) u64 keys in shared memory, ascending.
__device__ void bitonic_sort(unsigned long long *k, int n) {
  for (int size = 2; size <= n; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      __syncthreads();
      for (int i = threadIdx.x; i < n / 2; i += blockDim.x) {
        const int lo = 2 * i - (i & (stride - 1)), hi = lo + stride;
        const bool up = (lo & size) == 0;
        const unsigned long long a = k[lo], b = k[hi];
        if ((a > b) == up) {
          k[lo] = b;
          k[hi] = a;
        }
      }
    }
  __syncthreads();
}

__device__ __forceinline__ unsigned long long pkey(float s, uint32_t low) {
  return ((unsigned long long)score_key(s) << 32) | low;
}

// Per ligand: the `keep` candidates with the lowest predicted score (ties by
// index); their genotypes are gathered into kept_geno and kept_lig.
__global__ void topk_kernel(const float *pred, int candidates, int n2, int keep, const float *cand_geno,
                            float *kept_geno, int32_t *kept_lig) {
  extern __shared__ unsigned long long keys[];
  const int lig = blockIdx.x;
  for (int i = threadIdx.x; i < n2; i += blockDim.x)
    keys[i] = i < candidates ? pkey(pred[(int64_t)lig * candidates + i], (uint32_t)i) : ~0ull;
  bitonic_sort(keys, n2);
  for (int e = threadIdx.x; e < keep * DOCK_MAX_GENES; e += blockDim.x) {
    const int r = e / DOCK_MAX_GENES, gi = e % DOCK_MAX_GENES;
    const int c = (int)(keys[r] & 0xffffffffull);
    kept_geno[((int64_t)lig * keep + r) * DOCK_MAX_GENES + gi] =
        cand_geno[((int64_t)lig * candidates + c) * DOCK_MAX_GENES + gi];
  }
  for (int r = threadIdx.x; r < keep; r += blockDim.x) kept_lig[(int64_t)lig * keep + r] = lig;
}

// mu + lambda: the new population of each ligand is the best `pop` of the
// population (origin 0) and the kept candidates (origin 1) by exact score,
// ties by origin then index.
__global__ void merge_kernel(const float *geno_prev, const float *score_prev, const int64_t *geno_off,
                             const LigInfo *ligs, int pop, const float *kept_geno,
                             const float *kept_score, int keep, int n2, float *geno_next,
                             float *score_next) {
  extern __shared__ unsigned long long keys[];
  const int lig = blockIdx.x;
  const int G = 7 + ligs[lig].k;
  for (int i = threadIdx.x; i < n2; i += blockDim.x) {
    unsigned long long k = ~0ull;
    if (i < pop) k = pkey(score_prev[(int64_t)lig * pop + i], (uint32_t)i);
    else if (i < pop + keep)
      k = pkey(kept_score[(int64_t)lig * keep + (i - pop)], 0x80000000u | (uint32_t)(i - pop));
    keys[i] = k;
  }
  bitonic_sort(keys, n2);
  const float *gp = geno_prev + geno_off[lig];
  float *gn = geno_next + geno_off[lig];
  for (int e = threadIdx.x; e < pop * G; e += blockDim.x) {
    const int r = e / G, gi = e % G;
    const uint32_t low = (uint32_t)(keys[r] & 0xffffffffull);
    const int idx = (int)(low & 0x7fffffffu);
    gn[e] = (low & 0x80000000u) ? kept_geno[((int64_t)lig * keep + idx) * DOCK_MAX_GENES + gi]
                                : gp[(int64_t)idx * G + gi];
  }
  for (int r = threadIdx.x; r < pop; r += blockDim.x) {
    const uint32_t low = (uint32_t)(keys[r] & 0xffffffffull);
    const int idx = (int)(low & 0x7fffffffu);
    score_next[(int64_t)lig * pop + r] = (low & 0x80000000u) ? kept_score[(int64_t)lig * keep + idx]
                                                             : score_prev[(int64_t)lig * pop + idx];
  }
}

int pow2_at_least(int n) {
  int p = 1;
  while (p < n) p <<= 1;
  return p;
}
}  // namespace

cudaError_t launch_features(const FeatureLaunch &F, cudaStream_t s) {
  FeatArgs A{};
  A.ligs = F.ligs;
  A.atoms = F.atoms;
  A.types = F.types;
  A.pair_rec = F.pair_rec;
  A.tors = F.tors;
  A.moves = F.moves;
  A.grid = F.grid;
  A.cx = F.cx; A.cy = F.cy; A.cz = F.cz; A.radius = F.radius;
  A.n_ligands = F.n_ligands;
  A.pop_csr = F.pop_csr;
  A.pose_ligand = F.pose_ligand;
  A.genos = F.genos;
  A.n_poses = F.n_poses;
  A.scores = F.scores;
  A.pop = F.pop;
  A.candidates = F.candidates;
  A.gen = F.gen;
  A.seed = F.seed;
  A.thr_cross = F.thr_cross;
  A.thr_mut = F.thr_mut;
  A.geno_prev = F.geno_prev;
  A.score_prev = F.score_prev;
  A.geno_off = F.geno_off;
  A.cand_geno = F.cand_geno;
  A.features = reinterpret_cast<__nv_bfloat16 *>(F.features);
  if (F.from_ga) {
    if (F.n_ligands == 0 || F.candidates == 0) return cudaSuccess;
    dim3 grid((F.candidates + kFeatSlots - 1) / kFeatSlots, F.n_ligands);
    feat_kernel<true><<<grid, kFeatThreads, 0, s>>>(A);
  } else {
    if (F.n_poses == 0) return cudaSuccess;
    feat_kernel<false><<<(unsigned)((F.n_poses + kFeatSlots - 1) / kFeatSlots), kFeatThreads, 0, s>>>(A);
  }
  return cudaGetLastError();
}

cudaError_t launch_topk(const float *pred, int n_ligands, int candidates, int keep,
                        const float *cand_geno, float *kept_geno, int32_t *kept_lig, cudaStream_t s) {
  if (n_ligands == 0) return cudaSuccess;
  const int n2 = pow2_at_least(candidates);
  const int smem = n2 * 8;
  cudaError_t e = cudaFuncSetAttribute(topk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  topk_kernel<<<n_ligands, 1024, smem, s>>>(pred, candidates, n2, keep, cand_geno, kept_geno, kept_lig);
  return cudaGetLastError();
}

cudaError_t launch_merge(const float *geno_prev, const float *score_prev, const int64_t *geno_off,
                         const LigInfo *ligs, int n_ligands, int pop, const float *kept_geno,
                         const float *kept_score, int keep, float *geno_next, float *score_next,
                         cudaStream_t s) {
  if (n_ligands == 0) return cudaSuccess;
  const int n2 = pow2_at_least(pop + keep);
  const int smem = n2 * 8;
  cudaError_t e = cudaFuncSetAttribute(merge_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  merge_kernel<<<n_ligands, 1024, smem, s>>>(geno_prev, score_prev, geno_off, ligs, pop, kept_geno,
                                             kept_score, keep, n2, geno_next, score_next);
  return cudaGetLastError();
}

}  // namespace dk
