// Fused GA step + pose application + FP32 scoring (the docking hot path).
//
// One persistent kernel per search generation covers a whole batch of ligands
// of uneven size. Work items are (ligand, tile of poses) pulled from an atomic
// queue in largest-first order. A pose is handled by a group of L lanes
// (L = 1, 2, 4 or 8, chosen per ligand from its atom count) that all hold the
// pose's genotype in registers; its posed coordinates live in shared memory
// as three planes [atom][pose slot]. Per pose:
//   GA step (Section V, "genetic algorithm ... similar to AutoDock") or the
//   generation-0 draw,
//   Algorithm 1: rigid rotation + translation, then torsions in tree order,
//   Algorithm 2: inter-energy by trilinear lookup in the per-type maps and
//   intra-energy over the included pairs, each lane summing with Kahan
//   compensation, then a shuffle tree with TwoSum across the L lanes.
#include "device_common.cuh"

namespace dk {

// Coordinate planes: L * atoms_per_lane rows (atoms) by SP columns (pose
// slots). For L > 1 the row stride SP is an odd multiple of 32 / L, so the L
// lanes of a group reading consecutive atoms of one pose hit disjoint banks;
// rows * SP <= atoms_per_lane * (threads + 32) for every L.
__host__ __device__ __forceinline__ int plane_stride(int threads, int L) {
  const int S = threads / L;
  if (L == 1) return S;
  const int w = 32 / L;
  return ((S / w) & 1) ? S : S + w;
}

int search_smem_bytes(int threads, int atoms_per_lane) {
  return 3 * atoms_per_lane * (threads + 32) * (int)sizeof(float);
}

struct LigView {
  const float4 *atoms;      // this ligand's atoms
  const uint8_t *types;
  const uint32_t *pair_idx;
  const float4 *pair_coef;
  const TorInfo *tors;
  int n, k, n_pairs;
};

__device__ __forceinline__ LigView lig_view(const LigInfo &li, const float4 *atoms,
                                            const uint8_t *types, const uint32_t *pair_idx,
                                            const float4 *pair_coef, const TorInfo *tors) {
  LigView v;
  v.atoms = atoms + li.atom_off;
  v.types = types + li.atom_off;
  v.pair_idx = pair_idx + li.pair_off;
  v.pair_coef = pair_coef + li.pair_off;
  v.tors = tors + li.tors_off;
  v.n = li.n;
  v.k = li.k;
  v.n_pairs = li.n_pairs;
  return v;
}

// Pose one genotype and score it with a group of L lanes. Coordinates of the
// pose go to column `slot` of the smem planes (row stride SP). Every lane of
// the group returns the same score.
__device__ __forceinline__ float pose_and_score(const float (&g)[DOCK_MAX_GENES], const LigView &V,
                                                const uint8_t *moves, const GridView &G, float cx,
                                                float cy, float cz, float *sx, float *sy,
                                                float *sz, int SP, int slot, int lane, int L,
                                                unsigned gmask, float *coords_out) {
  // ---- Algorithm 1: rigid motion about the ligand centroid ----------------
  float qw = g[3], qx = g[4], qy = g[5], qz = g[6];
  float inv = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
  qw *= inv; qx *= inv; qy *= inv; qz *= inv;
  const float r00 = 1.f - 2.f * (qy * qy + qz * qz), r01 = 2.f * (qx * qy - qw * qz),
              r02 = 2.f * (qx * qz + qw * qy);
  const float r10 = 2.f * (qx * qy + qw * qz), r11 = 1.f - 2.f * (qx * qx + qz * qz),
              r12 = 2.f * (qy * qz - qw * qx);
  const float r20 = 2.f * (qx * qz - qw * qy), r21 = 2.f * (qy * qz + qw * qx),
              r22 = 1.f - 2.f * (qx * qx + qy * qy);
  const float tx = cx + g[0], ty = cy + g[1], tz = cz + g[2];
  for (int a = lane; a < V.n; a += L) {
    float4 p = __ldg(V.atoms + a);
    sx[a * SP + slot] = r00 * p.x + r01 * p.y + r02 * p.z + tx;
    sy[a * SP + slot] = r10 * p.x + r11 * p.y + r12 * p.z + ty;
    sz[a * SP + slot] = r20 * p.x + r21 * p.y + r22 * p.z + tz;
  }
  __syncwarp(gmask);
  // ---- torsions root to leaf, each about the current bond axis ------------
#pragma unroll
  for (int j = 0; j < DOCK_MAX_TORSIONS; ++j) {
    if (j < V.k) {
      const TorInfo T = V.tors[j];
      const float ax = sx[T.a * SP + slot], ay = sy[T.a * SP + slot], az = sz[T.a * SP + slot];
      float ux = sx[T.b * SP + slot] - ax, uy = sy[T.b * SP + slot] - ay,
            uz = sz[T.b * SP + slot] - az;
      const float il = rsqrtf(ux * ux + uy * uy + uz * uz);
      ux *= il; uy *= il; uz *= il;
      float s, c;
      __sincosf(g[7 + j], &s, &c);
      const float oc = 1.f - c;
      const float m00 = c + ux * ux * oc, m01 = ux * uy * oc - uz * s, m02 = ux * uz * oc + uy * s;
      const float m10 = uy * ux * oc + uz * s, m11 = c + uy * uy * oc, m12 = uy * uz * oc - ux * s;
      const float m20 = uz * ux * oc - uy * s, m21 = uz * uy * oc + ux * s, m22 = c + uz * uz * oc;
      const uint8_t *mv = moves + T.move_off;
      for (int m = lane; m < T.n_move; m += L) {
        const int at = mv[m];
        const float vx = sx[at * SP + slot] - ax, vy = sy[at * SP + slot] - ay,
                    vz = sz[at * SP + slot] - az;
        sx[at * SP + slot] = ax + m00 * vx + m01 * vy + m02 * vz;
        sy[at * SP + slot] = ay + m10 * vx + m11 * vy + m12 * vz;
        sz[at * SP + slot] = az + m20 * vx + m21 * vy + m22 * vz;
      }
      __syncwarp(gmask);
    }
  }
  // ---- Algorithm 2: inter-energy by grid lookup ----------------------------
  Kahan acc;
#pragma unroll 2
  for (int a = lane; a < V.n; a += L) {
    const float x = sx[a * SP + slot], y = sy[a * SP + slot], z = sz[a * SP + slot];
    float e;
    if (!grid_energy(G, V.types[a], __ldg(&V.atoms[a].w), x, y, z, e)) e = kEout;
    acc.add(e);
    if (coords_out) {
      coords_out[3 * a] = x;
      coords_out[3 * a + 1] = y;
      coords_out[3 * a + 2] = z;
    }
  }
  // ---- intra-energy over the included pairs --------------------------------
  for (int p = lane; p < V.n_pairs; p += L) {
    const uint32_t idx = __ldg(V.pair_idx + p);
    const float4 coef = __ldg(V.pair_coef + p);
    const int i = idx & 255, j = (idx >> 8) & 255;
    const float dx = sx[i * SP + slot] - sx[j * SP + slot];
    const float dy = sy[i * SP + slot] - sy[j * SP + slot];
    const float dz = sz[i * SP + slot] - sz[j * SP + slot];
    acc.add(pair_energy(dx * dx + dy * dy + dz * dz, coef, (idx >> 16) & 1));
  }
  // ---- combine the group's compensated sums --------------------------------
  float s = acc.s, c = acc.c;
  for (int off = 1; off < L; off <<= 1) {
    const float so = __shfl_xor_sync(gmask, s, off);
    const float co = __shfl_xor_sync(gmask, c, off);
    float t, e;
    two_sum(s, so, t, e);
    s = t;
    c = __fsub_rn(__fadd_rn(c, co), e);
  }
  __syncwarp(gmask);
  return __fsub_rn(s, c);
}

__device__ __forceinline__ unsigned group_mask(int L) {
  if (L >= 32) return 0xffffffffu;
  const unsigned base = (threadIdx.x & 31) & ~(unsigned)(L - 1);
  return ((1u << L) - 1u) << base;
}

__global__ void __launch_bounds__(128, 6) search_kernel(const SearchArgs A) {
  extern __shared__ float smem[];
  __shared__ int s_item;
  const int T = blockDim.x;
  const int plane = A.atoms_per_lane * (T + 32);
  float *sx = smem, *sy = smem + plane, *sz = smem + 2 * plane;
  for (;;) {
    if (threadIdx.x == 0) {
      int it = (int)atomicAdd(A.counter, 1u);
      if (A.deadline != nullptr && it < A.n_items && globaltimer_ns() > *A.deadline) {
        atomicExch(A.status, (int)DOCK_ETIMEOUT);
        it = A.n_items;
      }
      s_item = it;
    }
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= A.n_items) break;
    const Item item = A.items[it];
    const int L = item.lanes;
    const int S = T / L;
    const int SP = plane_stride(T, L);
    const int lane = threadIdx.x & (L - 1);
    const int slot = threadIdx.x / L;
    const int ind = item.first_div * S + slot;
    if (ind >= A.pop) continue;
    const LigInfo li = A.ligs[item.lig];
    const int G = 7 + li.k;
    const int64_t goff = A.geno_off[item.lig];
    const int64_t soff = (int64_t)item.lig * A.pop;
    float g[DOCK_MAX_GENES];
    if (A.gen == 0) {
      ga_init(g, li.k, A.radius, A.seed, li.ligand_id, (uint32_t)ind);
    } else if (ind == 0) {
      int best = (int)(A.best_prev[item.lig] & 0xffffffffull);
      if (best >= A.pop) best = 0;  // previous generation stopped by its deadline
      const float *src = A.geno_prev + goff + (int64_t)best * G;
#pragma unroll
      for (int e = 0; e < DOCK_MAX_GENES; ++e) g[e] = e < G ? src[e] : 0.0f;
    } else {
      ga_child(g, li.k, A.pop, A.geno_prev + goff, A.score_prev + soff, A.thr_cross, A.thr_mut,
               A.seed, li.ligand_id, (uint32_t)A.gen, (uint32_t)ind);
    }
    float *gout = A.geno_next + goff + (int64_t)ind * G;
#pragma unroll
    for (int e = 0; e < DOCK_MAX_GENES; ++e)
      if (e < G && (e & (L - 1)) == lane) gout[e] = g[e];
    const LigView V = lig_view(li, A.atoms, A.types, A.pair_idx, A.pair_coef, A.tors);
    const float score = pose_and_score(g, V, A.moves, A.grid, A.cx, A.cy, A.cz, sx, sy, sz, SP,
                                       slot, lane, L, group_mask(L), nullptr);
    if (lane == 0) {
      A.score_next[soff + ind] = score;
      const unsigned long long key =
          ((unsigned long long)score_key(score) << 32) | (unsigned long long)(uint32_t)ind;
      atomicMin(&A.best_next[item.lig], key);
    }
  }
}

static cudaError_t configure_search() {
  // called outside stream capture (from the occupancy query) before any launch
  return cudaFuncSetAttribute(search_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              200 * 1024);
}

cudaError_t search_occupancy(int threads, int smem, int *blocks_per_sm) {
  cudaError_t e = configure_search();
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, search_kernel, threads, smem);
}

cudaError_t launch_search(const SearchArgs &a, int blocks, int threads, cudaStream_t s) {
  const int smem = search_smem_bytes(threads, a.atoms_per_lane);
  search_kernel<<<blocks, threads, smem, s>>>(a);
  return cudaGetLastError();
}

// Writes globaltimer + timeout: the absolute deadline the search kernels test.
__global__ void set_deadline_kernel(uint64_t *deadline, uint64_t timeout_ns) {
  *deadline = globaltimer_ns() + timeout_ns;
}

cudaError_t launch_set_deadline(uint64_t *deadline, uint64_t timeout_ns, cudaStream_t s) {
  set_deadline_kernel<<<1, 1, 0, s>>>(deadline, timeout_ns);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Scoring of caller-given poses: a group of a.lanes lanes per pose, each group
// with its own ligand.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) score_kernel(const ScoreArgs A) {
  extern __shared__ float smem[];
  const int T = blockDim.x, L = A.lanes, S = T / L, SP = plane_stride(T, L);
  const int plane = A.atoms_per_lane * (T + 32);
  float *sx = smem, *sy = smem + plane, *sz = smem + 2 * plane;
  const int lane = threadIdx.x & (L - 1), slot = threadIdx.x / L;
  const int64_t pose = (int64_t)blockIdx.x * S + slot;
  if (pose >= A.n_poses) return;
  const int lig = A.pose_ligand[pose];
  if (lig < 0 || lig >= A.n_ligands) {
    if (lane == 0) A.scores[pose] = __int_as_float(0x7fc00000);
    return;
  }
  const LigInfo li = A.ligs[lig];
  float g[DOCK_MAX_GENES];
  const float *src = A.genos + pose * DOCK_MAX_GENES;
#pragma unroll
  for (int e = 0; e < DOCK_MAX_GENES; ++e) g[e] = e < 7 + li.k ? src[e] : 0.0f;
  const LigView V = lig_view(li, A.atoms, A.types, A.pair_idx, A.pair_coef, A.tors);
  float *co = A.coords ? A.coords + pose * (DOCK_MAX_ATOMS * 3) : nullptr;
  const float score = pose_and_score(g, V, A.moves, A.grid, A.cx, A.cy, A.cz, sx, sy, sz, SP,
                                     slot, lane, L, group_mask(L), co);
  if (lane == 0) A.scores[pose] = score;
}

cudaError_t launch_score(const ScoreArgs &a, cudaStream_t s) {
  const int threads = 128;
  const int S = threads / a.lanes;
  const int64_t blocks = (a.n_poses + S - 1) / S;
  if (blocks == 0) return cudaSuccess;
  const int smem = search_smem_bytes(threads, a.atoms_per_lane);
  cudaError_t e = cudaFuncSetAttribute(score_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       smem);
  if (e != cudaSuccess) return e;
  score_kernel<<<(unsigned)blocks, threads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace dk
