// Scoring of caller-given poses with the pairwise inter-energy: every protein
// atom within the 8 A cutoff of a ligand atom enters through the pair terms
// (Algorithm 2's inter loop over nearby protein atoms, the sum the grid maps
// of Section V approximate), plus the intra-energy; FP32 with compensated
// sums. Protein atoms come from a cell list with 8 A cells (cells ordered x
// fastest, so the three x-neighbours of a cell are one contiguous atom range:
// nine ranges per ligand atom).
#include "pose.cuh"

namespace dk {

namespace {

constexpr int kPwL = 8;  // lanes per pose
constexpr int kPwThreads = 128;
constexpr int kPwApl = DOCK_MAX_ATOMS / kPwL;

// Inclusive cell range [lo, hi] of the cells within one cell of coordinate u
// (cell units) on an axis of d cells; empty (lo > hi) far outside.
__device__ __forceinline__ void cell_range(float u, int d, int &lo, int &hi) {
  const float c = floorf(fminf(fmaxf(u, -4.0f), (float)d + 4.0f));
  lo = max((int)c - 1, 0);
  hi = min((int)c + 1, d - 1);
}

__global__ void __launch_bounds__(kPwThreads) score_pairwise_kernel(const PairwiseArgs A) {
  __shared__ float4 s_col[slots_bytes(kPwThreads, kPwL, kPwApl) / 16];
  __shared__ float4 s_tp[DOCK_MAX_TYPES * DOCK_MAX_TYPES];
  __shared__ float2 s_sv[DOCK_MAX_TYPES];
  const int T = A.n_types;
  for (int i = threadIdx.x; i < T * T; i += blockDim.x) s_tp[i] = A.tpair[i];
  for (int i = threadIdx.x; i < T; i += blockDim.x) s_sv[i] = A.tsv[i];
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
  const LigView V = lig_view(li, A.atoms, A.types, A.pair_rec, A.tors);
  float4 *sl = s_col + slot * slot_stride(kPwL, kPwApl);
  apply_pose<kPwL>(g, V, A.moves, A.cx, A.cy, A.cz, sl, lane, gmask);
  // ---- intra pairs (as in the grid scorer) ---------------------------------
  Kahan acc;
  if (lane == 0) acc.add(V.intra_const);
  PairWalker<kPwL> W(V, sl, lane);
  const int np_l = V.n_pairs > lane ? (V.n_pairs - lane + kPwL - 1) / kPwL : 0;
  int m = 0;
  for (; m + 3 < np_l; m += 4) {
    const float e0 = W.term(m), e1 = W.term(m + 1), e2 = W.term(m + 2), e3 = W.term(m + 3);
    acc.add((e0 + e1) + (e2 + e3));
  }
  for (; m < np_l; ++m) acc.add(W.term(m));
  // ---- inter: every protein atom within the cutoff --------------------------
  const float kElec = (float)((double)kWElec * kCoulomb);
  for (int a = lane; a < V.n; a += kPwL) {
    const float4 p = sl[a];
    const int ti = V.types[a];
    const float qi = __ldg(&V.atoms[a].w);
    const float qe = kElec * qi;
    const float si = kWSol * (s_sv[ti].x + (float)kQasp * fabsf(qi));  // W_sol S_i
    const float vi = kWSol * s_sv[ti].y;                               // W_sol V_i
    int x0, x1, y0, y1, z0, z1;
    cell_range((p.x - A.lox) * A.inv_cs, A.dx, x0, x1);
    cell_range((p.y - A.loy) * A.inv_cs, A.dy, y0, y1);
    cell_range((p.z - A.loz) * A.inv_cs, A.dz, z0, z1);
    Kahan ai;
    for (int cz = z0; cz <= z1; ++cz)
      for (int cy = y0; cy <= y1; ++cy) {
        if (x0 > x1) break;
        const int row = (cz * A.dy + cy) * A.dx;
        const int j1 = __ldg(A.cell_start + row + x1 + 1);
        for (int j = __ldg(A.cell_start + row + x0); j < j1; ++j) {
          const float4 b = __ldg(A.cprot + j);
          const float dx = p.x - b.x, dy = p.y - b.y, dz = p.z - b.z;
          const float r2 = dx * dx + dy * dy + dz * dz;
          if (r2 < kCutoff2) {
            const float4 ex = __ldg(A.cext + j);  // {S_j, V_j, type, 0}
            const float4 c = s_tp[ti * T + (int)ex.z];
            const float rec[8] = {c.x, c.y, c.z, c.w, qe * b.w, fmaf(si, ex.y, ex.x * vi),
                                  0.0f, 0.0f};
            ai.add(pair_energy(r2, rec));
          }
        }
      }
    acc.add(ai.value());
  }
  // ---- combine the group's compensated sums --------------------------------
  float s = acc.s, c = acc.c;
#pragma unroll
  for (int off = 1; off < kPwL; off <<= 1) {
    const float so = __shfl_xor_sync(gmask, s, off);
    const float co = __shfl_xor_sync(gmask, c, off);
    float t, e;
    two_sum(s, so, t, e);
    s = t;
    c = __fsub_rn(__fadd_rn(c, co), e);
  }
  if (lane == 0) A.scores[pose] = __fsub_rn(s, c);
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
