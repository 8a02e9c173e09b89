// Fused GA step + pose application + FP32 scoring (the docking hot path).
//
// One persistent kernel per search generation covers a whole batch of ligands
// of uneven size. Work items are (ligand, tile of poses) pulled from an atomic
// queue in largest-first order (the next item is fetched while the current
// one runs). A pose is handled by a group of L lanes (L = 1, 2, 4 or 8, chosen
// per ligand from its atom count; one launch per L, the launches of a
// generation running concurrently) that all hold the pose's genotype in
// registers; its posed coordinates live in the pose's shared-memory slot as
// float4 rows, one per atom. L is a compile-time constant of the per-item
// code path. Per pose:
//   GA step (Section V, "genetic algorithm ... similar to AutoDock") or the
//   generation-0 draw,
//   Algorithm 1: rigid rotation + translation, then torsions in tree order,
//   Algorithm 2: inter-energy by trilinear lookup in the per-type maps and
//   intra-energy over the included pairs, interleaved so each atom's grid
//   loads are in flight while a share of the pairs is computed; each lane
//   keeps a Kahan-compensated sum (pair terms added in blocks of four), then
//   a shuffle tree with TwoSum combines the L lanes.
#include <algorithm>

#include "pose.cuh"

namespace dk {

int search_smem_bytes(int threads, int atoms_per_lane) {
  int b = 0;
  for (int L = 1; L <= 8; L <<= 1) b = std::max(b, slots_bytes(threads, L, atoms_per_lane));
  return b;
}

__device__ __forceinline__ int fetch_item(const SearchArgs &A) {
  int it = (int)atomicAdd(A.counter, 1u);
#ifdef DOCK_CHECKED
  if (it < A.n_items && *(volatile int32_t *)A.status != 0) it = A.n_items;  // a check failed
#endif
  if (A.deadline != nullptr && it < A.n_items && globaltimer_ns() > *A.deadline) {
    atomicExch(A.status, (int)DOCK_ETIMEOUT);
    it = A.n_items;
  }
  return it;
}

// One work item for the pose slot of this thread, L lanes per pose; PW: the
// inter-energy is the pairwise sum over the protein cell list (no maps).
template <int L, bool PW>
__device__ __forceinline__ void search_item(const SearchArgs &A, const Item &item, float4 *smem4) {
  const int S = blockDim.x / L;
  const int lane = threadIdx.x & (L - 1);
  const int slot = threadIdx.x / L;
  const int ind = item.first_div * S + slot;
  if (ind >= A.pop) return;
  const unsigned gmask = group_mask<L>();
  if (!DK_OK(item.lig >= 0 && item.lig < A.bounds.ligands, A.status, 12)) return;
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
    ga_child_group<L>(g, li.k, A.pop, A.geno_prev + goff, A.score_prev + soff, A.thr_cross,
                      A.thr_mut, A.seed, li.ligand_id, (uint32_t)A.gen, (uint32_t)ind, lane,
                      gmask);
  }
  float *gout = A.geno_next + goff + (int64_t)ind * G;
#pragma unroll
  for (int e = 0; e < DOCK_MAX_GENES; ++e)
    if (e < G && (e & (L - 1)) == lane) gout[e] = g[e];
  const LigView V = lig_view(li, A.atoms, A.types, A.pair_rec, A.tors, DK_BOUNDS(A),
                             slot_stride(L, A.atoms_per_lane));
  float4 *sl = smem4 + slot * slot_stride(L, A.atoms_per_lane);
  float score;
  if constexpr (PW) {
    apply_pose<L>(g, V, A.moves, A.cx, A.cy, A.cz, sl, lane, gmask);
    score = score_posed_pw<L>(V, A.pw, sl, lane, gmask, A.pw.tpair, A.pw.tsv);
  } else {
    score = pose_and_score<L>(g, V, A.moves, A.grid, A.cx, A.cy, A.cz, sl, lane, gmask, nullptr);
  }
  if (lane == 0) {
    A.score_next[soff + ind] = score;
    const unsigned long long key =
        ((unsigned long long)score_key(score) << 32) | (unsigned long long)(uint32_t)ind;
    atomicMin(&A.best_next[item.lig], key);
  }
}

// One launch per lanes-per-pose group: all its items have L lanes per pose.
template <int L, bool PW = false>
__global__ void __launch_bounds__(128, 5) search_kernel(const SearchArgs A) {
  extern __shared__ float4 smem4[];
  __shared__ int s_item;
  if (threadIdx.x == 0) s_item = fetch_item(A);
  __syncthreads();
  for (;;) {
    const int it = s_item;
    __syncthreads();
    if (it >= A.n_items) break;
    int next = 0;
    if (threadIdx.x == 0) next = fetch_item(A);  // overlaps with this item
    search_item<L, PW>(A, A.items[it], smem4);
    if (threadIdx.x == 0) s_item = next;
    __syncthreads();
  }
}

template <int L, bool PW = false>
static cudaError_t search_occupancy_l(int threads, int smem, int *blocks_per_sm) {
  // called outside stream capture before any launch of the instantiation
  cudaError_t e = cudaFuncSetAttribute(search_kernel<L, PW>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, search_kernel<L, PW>, threads,
                                                       smem);
}

cudaError_t search_occupancy(int threads, int L, int atoms_per_lane, int *blocks_per_sm,
                             bool pairwise) {
  const int smem = slots_bytes(threads, L, atoms_per_lane);
  if (pairwise) {
    switch (L) {
      case 1: return search_occupancy_l<1, true>(threads, smem, blocks_per_sm);
      case 2: return search_occupancy_l<2, true>(threads, smem, blocks_per_sm);
      case 4: return search_occupancy_l<4, true>(threads, smem, blocks_per_sm);
      case 8: return search_occupancy_l<8, true>(threads, smem, blocks_per_sm);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (L) {
    case 1: return search_occupancy_l<1>(threads, smem, blocks_per_sm);
    case 2: return search_occupancy_l<2>(threads, smem, blocks_per_sm);
    case 4: return search_occupancy_l<4>(threads, smem, blocks_per_sm);
    case 8: return search_occupancy_l<8>(threads, smem, blocks_per_sm);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_search(const SearchArgs &a, int blocks, int threads, int L, cudaStream_t s,
                          bool pairwise) {
  const int smem = slots_bytes(threads, L, a.atoms_per_lane);
  if (pairwise) {
    switch (L) {
      case 1: search_kernel<1, true><<<blocks, threads, smem, s>>>(a); break;
      case 2: search_kernel<2, true><<<blocks, threads, smem, s>>>(a); break;
      case 4: search_kernel<4, true><<<blocks, threads, smem, s>>>(a); break;
      case 8: search_kernel<8, true><<<blocks, threads, smem, s>>>(a); break;
      default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
  }
  switch (L) {
    case 1: search_kernel<1><<<blocks, threads, smem, s>>>(a); break;
    case 2: search_kernel<2><<<blocks, threads, smem, s>>>(a); break;
    case 4: search_kernel<4><<<blocks, threads, smem, s>>>(a); break;
    case 8: search_kernel<8><<<blocks, threads, smem, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
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
template <int L>
__device__ __forceinline__ void score_one(const ScoreArgs &A, float4 *smem4) {
  const int S = blockDim.x / L;
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
  const LigView V = lig_view(li, A.atoms, A.types, A.pair_rec, A.tors, DK_BOUNDS(A),
                             slot_stride(L, A.atoms_per_lane));
  float *co = A.coords ? A.coords + pose * (DOCK_MAX_ATOMS * 3) : nullptr;
  float4 *sl = smem4 + slot * slot_stride(L, A.atoms_per_lane);
  const float score = pose_and_score<L>(g, V, A.moves, A.grid, A.cx, A.cy, A.cz, sl, lane,
                                        group_mask<L>(), co);
  if (lane == 0) A.scores[pose] = score;
}

__global__ void __launch_bounds__(128) score_kernel(const ScoreArgs A) {
  extern __shared__ float4 smem4[];
  switch (A.lanes) {
    case 1: score_one<1>(A, smem4); break;
    case 2: score_one<2>(A, smem4); break;
    case 4: score_one<4>(A, smem4); break;
    default: score_one<8>(A, smem4); break;
  }
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
