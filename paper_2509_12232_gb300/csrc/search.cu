// Fused GA step + pose application + FP32 scoring (the docking hot path).
//
// One persistent kernel per search generation covers a whole batch of ligands
// of uneven size. Work items are (ligand, tile of poses) pulled from an atomic
// queue in largest-first order (the next item is fetched while the current
// one runs). A pose is handled by a group of L lanes (L = 1, 2, 4 or 8, chosen
// per ligand from its atom count) that all hold the pose's genotype in
// registers; its posed coordinates live in shared memory as float4 rows
// [atom][pose slot]. Per pose:
//   GA step (Section V, "genetic algorithm ... similar to AutoDock") or the
//   generation-0 draw,
//   Algorithm 1: rigid rotation + translation, then torsions in tree order,
//   Algorithm 2: inter-energy by trilinear lookup in the per-type maps and
//   intra-energy over the included pairs, interleaved so each atom's grid
//   loads are in flight while a share of the pairs is computed; each lane
//   keeps a Kahan-compensated sum (pair terms added in blocks of four), then
//   a shuffle tree with TwoSum combines the L lanes.
#include "device_common.cuh"

namespace dk {

// Coordinate rows: L * atoms_per_lane rows (atoms) by SP float4 columns (pose
// slots). For L > 1 the stride SP is an odd multiple of 8 / L, so each
// quarter-warp phase of a 16-byte shared load (2, 4 or 8 lanes of consecutive
// atoms) touches distinct bank groups; rows * SP <= atoms_per_lane * (T + 8).
__host__ __device__ __forceinline__ int plane_stride(int threads, int L) {
  const int S = threads / L;
  if (L == 1) return S;
  const int w = 8 / L;
  return ((S / w) & 1) ? S : S + w;
}

int search_smem_bytes(int threads, int atoms_per_lane) {
  return atoms_per_lane * (threads + 8) * (int)sizeof(float4);
}

struct LigView {
  const float4 *atoms;      // this ligand's atoms (centred) + charge
  const uint8_t *types;
  const float *pair_rec;    // 8 floats per pair
  const TorInfo *tors;
  int n, k, n_pairs;
};

__device__ __forceinline__ LigView lig_view(const LigInfo &li, const float4 *atoms,
                                            const uint8_t *types, const float *pair_rec,
                                            const TorInfo *tors) {
  LigView v;
  v.atoms = atoms + li.atom_off;
  v.types = types + li.atom_off;
  v.pair_rec = pair_rec + (int64_t)li.pair_off * 8;
  v.tors = tors + li.tors_off;
  v.n = li.n;
  v.k = li.k;
  v.n_pairs = li.n_pairs;
  return v;
}

// Pair terms in row-major pair order: the coordinates of atom i stay in
// registers while consecutive pairs of a lane share it.
struct PairWalker {
  const LigView &V;
  const float4 *col;
  int SP;
  int last_i = -1;
  float4 ci;
  __device__ __forceinline__ PairWalker(const LigView &v, const float4 *c, int sp)
      : V(v), col(c), SP(sp) {}
  __device__ __forceinline__ float term(int p) {
    float rec[8];
    ld8(V.pair_rec + (int64_t)p * 8, rec);
    const uint32_t ij = __float_as_uint(rec[6]);
    const int i = (int)(ij & 0xffffu);
    if (i != last_i) {
      ci = col[i * SP];
      last_i = i;
    }
    const float4 b = col[(int)(ij >> 16) * SP];
    const float dx = ci.x - b.x, dy = ci.y - b.y, dz = ci.z - b.z;
    return pair_energy(dx * dx + dy * dy + dz * dz, rec);
  }
};

// Pose one genotype and score it with a group of L lanes. The pose's
// coordinates are column `col` (stride SP) of the shared rows. Every lane of
// the group returns the same score.
__device__ __forceinline__ float pose_and_score(const float (&g)[DOCK_MAX_GENES], const LigView &V,
                                                const uint8_t *moves, const GridView &G, float cx,
                                                float cy, float cz, float4 *col, int SP, int lane,
                                                int L, unsigned gmask, float *coords_out) {
  // ---- Algorithm 1: rigid motion about the ligand centroid ----------------
  float qw = g[3], qx = g[4], qy = g[5], qz = g[6];
  const float inv = rsqrt_ftz(qw * qw + qx * qx + qy * qy + qz * qz);
  qw *= inv; qx *= inv; qy *= inv; qz *= inv;
  const float r00 = 1.f - 2.f * (qy * qy + qz * qz), r01 = 2.f * (qx * qy - qw * qz),
              r02 = 2.f * (qx * qz + qw * qy);
  const float r10 = 2.f * (qx * qy + qw * qz), r11 = 1.f - 2.f * (qx * qx + qz * qz),
              r12 = 2.f * (qy * qz - qw * qx);
  const float r20 = 2.f * (qx * qz - qw * qy), r21 = 2.f * (qy * qz + qw * qx),
              r22 = 1.f - 2.f * (qx * qx + qy * qy);
  const float tx = cx + g[0], ty = cy + g[1], tz = cz + g[2];
  for (int a = lane; a < V.n; a += L) {
    const float4 p = __ldg(V.atoms + a);
    col[a * SP] = make_float4(r00 * p.x + r01 * p.y + r02 * p.z + tx,
                              r10 * p.x + r11 * p.y + r12 * p.z + ty,
                              r20 * p.x + r21 * p.y + r22 * p.z + tz, 0.0f);
  }
  __syncwarp(gmask);
  // ---- torsions root to leaf, each about the current bond axis ------------
#pragma unroll
  for (int j = 0; j < DOCK_MAX_TORSIONS; ++j) {
    if (j < V.k) {
      const TorInfo T = V.tors[j];
      const float4 pa = col[T.a * SP], pb = col[T.b * SP];
      float ux = pb.x - pa.x, uy = pb.y - pa.y, uz = pb.z - pa.z;
      const float il = rsqrt_ftz(ux * ux + uy * uy + uz * uz);
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
        const float4 p = col[at * SP];
        const float vx = p.x - pa.x, vy = p.y - pa.y, vz = p.z - pa.z;
        col[at * SP] = make_float4(pa.x + m00 * vx + m01 * vy + m02 * vz,
                                   pa.y + m10 * vx + m11 * vy + m12 * vz,
                                   pa.z + m20 * vx + m21 * vy + m22 * vz, 0.0f);
      }
      __syncwarp(gmask);
    }
  }
  // ---- Algorithm 2: each grid lookup (inter-energy of one atom) is issued,
  // ---- a share of the intra pairs runs while its loads are in flight, then
  // ---- the lookup is interpolated ------------------------------------------
  Kahan acc;
  PairWalker W(V, col, SP);
  const int na = V.n > lane ? (V.n - lane + L - 1) / L : 0;               // atoms lane + k L
  const int np_l = V.n_pairs > lane ? (V.n_pairs - lane + L - 1) / L : 0;  // pairs lane + m L
  int m = 0;
  for (int k = 0; k < na; ++k) {
    const int a = lane + k * L;
    const float4 pa = col[a * SP];
    const Lookup lk = grid_issue(G, V.types[a], __ldg(&V.atoms[a].w), pa.x, pa.y, pa.z);
    if (coords_out) {
      coords_out[3 * a] = pa.x;
      coords_out[3 * a + 1] = pa.y;
      coords_out[3 * a + 2] = pa.z;
    }
    const int m_end = (int)(((int64_t)(k + 1) * np_l) / na);
    for (; m + 3 < m_end; m += 4) {
      const int p = lane + m * L;
      const float e0 = W.term(p), e1 = W.term(p + L);
      const float e2 = W.term(p + 2 * L), e3 = W.term(p + 3 * L);
      acc.add((e0 + e1) + (e2 + e3));
    }
    for (; m < m_end; ++m) acc.add(W.term(lane + m * L));
    acc.add(grid_finish(lk));
  }
  for (; m < np_l; ++m) acc.add(W.term(lane + m * L));
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

__device__ __forceinline__ int fetch_item(const SearchArgs &A) {
  int it = (int)atomicAdd(A.counter, 1u);
  if (A.deadline != nullptr && it < A.n_items && globaltimer_ns() > *A.deadline) {
    atomicExch(A.status, (int)DOCK_ETIMEOUT);
    it = A.n_items;
  }
  return it;
}

__global__ void __launch_bounds__(128, 5) search_kernel(const SearchArgs A) {
  extern __shared__ float4 smem4[];
  __shared__ int s_item;
  const int T = blockDim.x;
  if (threadIdx.x == 0) s_item = fetch_item(A);
  __syncthreads();
  for (;;) {
    const int it = s_item;
    __syncthreads();
    if (it >= A.n_items) break;
    int next = 0;
    if (threadIdx.x == 0) next = fetch_item(A);  // overlaps with this item
    const Item item = A.items[it];
    const int L = item.lanes;
    const int S = T / L;
    const int SP = plane_stride(T, L);
    const int lane = threadIdx.x & (L - 1);
    const int slot = threadIdx.x / L;
    const int ind = item.first_div * S + slot;
    if (ind < A.pop) {
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
      const LigView V = lig_view(li, A.atoms, A.types, A.pair_rec, A.tors);
      const float score = pose_and_score(g, V, A.moves, A.grid, A.cx, A.cy, A.cz, smem4 + slot, SP,
                                         lane, L, group_mask(L), nullptr);
      if (lane == 0) {
        A.score_next[soff + ind] = score;
        const unsigned long long key =
            ((unsigned long long)score_key(score) << 32) | (unsigned long long)(uint32_t)ind;
        atomicMin(&A.best_next[item.lig], key);
      }
    }
    if (threadIdx.x == 0) s_item = next;
    __syncthreads();
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
  extern __shared__ float4 smem4[];
  const int T = blockDim.x, L = A.lanes, S = T / L, SP = plane_stride(T, L);
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
  const LigView V = lig_view(li, A.atoms, A.types, A.pair_rec, A.tors);
  float *co = A.coords ? A.coords + pose * (DOCK_MAX_ATOMS * 3) : nullptr;
  const float score = pose_and_score(g, V, A.moves, A.grid, A.cx, A.cy, A.cz, smem4 + slot, SP,
                                     lane, L, group_mask(L), co);
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
