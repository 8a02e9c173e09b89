// Scoring of caller-given poses with the pairwise inter-energy: every protein
// atom within the 8 A cutoff of a ligand atom enters through the pair terms
// (Algorithm 2's inter loop over nearby protein atoms, the sum the grid maps
// of Section V approximate), plus the intra-energy; FP32 with compensated
// sums. Protein atoms come from the cell list of cutoff_ranges: at most nine
// rows of 8 A y-z cells per ligand atom, each trimmed in x (1 A cells) to the
// chord of the cutoff sphere.
#include "pose.cuh"

namespace dk {

namespace {

constexpr int kPwL = 8;  // lanes per pose
constexpr int kPwThreads = 128;
constexpr int kPwApl = DOCK_MAX_ATOMS / kPwL;

__global__ void __launch_bounds__(kPwThreads) score_pairwise_kernel(const PairwiseArgs A) {
  __shared__ float4 s_col[slots_bytes(kPwThreads, kPwL, kPwApl) / 16];
  __shared__ float4 s_tp[DOCK_MAX_TYPES * DOCK_MAX_TYPES];
  __shared__ float2 s_sv[DOCK_MAX_TYPES];
  const int T = A.pw.n_types;
  for (int i = threadIdx.x; i < T * T; i += blockDim.x) s_tp[i] = A.pw.tpair[i];
  for (int i = threadIdx.x; i < T; i += blockDim.x) s_sv[i] = A.pw.tsv[i];
  __syncthreads();
  const int lane = threadIdx.x & (kPwL - 1), slot = threadIdx.x / kPwL;
  const int64_t pose = (int64_t)blockIdx.x * (kPwThreads / kPwL) + slot;
  if (pose >= A.n_poses) return;
  const int lig = A.pose_ligand[pose];
  if (lig < 0 || lig >= A.n_ligands) {
    if (lane == 0) A.scores[pose] = __int_as_float(0x7fc00000);
    return;
  }
  const unsigned gmask = group_mask<kPwL>();
  const LigInfo li = A.ligs[lig];
  float g[DOCK_MAX_GENES];
  const float *src = A.genos + pose * DOCK_MAX_GENES;
#pragma unroll
  for (int e = 0; e < DOCK_MAX_GENES; ++e) g[e] = e < 7 + li.k ? src[e] : 0.0f;
  const LigView V = lig_view(li, A.atoms, A.types, A.pair_rec, A.tors, DK_BOUNDS(A),
                             slot_stride(kPwL, kPwApl));
  float4 *sl = s_col + slot * slot_stride(kPwL, kPwApl);
  apply_pose<kPwL>(g, V, A.moves, A.cx, A.cy, A.cz, sl, lane, gmask);
  const float score = score_posed_pw<kPwL>(V, A.pw, sl, lane, gmask, s_tp, s_sv);
  if (lane == 0) A.scores[pose] = score;
}

}  // namespace

cudaError_t launch_score_pairwise(const PairwiseArgs &a, cudaStream_t s) {
  const int per_block = kPwThreads / kPwL;
  const int64_t blocks = (a.n_poses + per_block - 1) / per_block;
  if (blocks == 0) return cudaSuccess;
  score_pairwise_kernel<<<(unsigned)blocks, kPwThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace dk
