// Device functions of the pose (Algorithm 1) and score (Algorithm 2) shared
// by the search, scoring and feature kernels.
#pragma once

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

// Algorithm 1 for one genotype by a group of L lanes: the posed coordinates
// go to column `col` (stride SP) of the shared rows.
__device__ __forceinline__ void apply_pose(const float (&g)[DOCK_MAX_GENES], const LigView &V,
                                           const uint8_t *moves, float cx, float cy, float cz,
                                           float4 *col, int SP, int lane, int L, unsigned gmask) {
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
}

// Algorithm 2 for the posed ligand in column `col`: every lane of the group
// returns the same FP32 score.
__device__ __forceinline__ float score_posed(const LigView &V, const GridView &G, float4 *col, int SP,
                                             int lane, int L, unsigned gmask, float *coords_out) {
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

__device__ __forceinline__ float pose_and_score(const float (&g)[DOCK_MAX_GENES], const LigView &V,
                                                const uint8_t *moves, const GridView &G, float cx,
                                                float cy, float cz, float4 *col, int SP, int lane,
                                                int L, unsigned gmask, float *coords_out) {
  apply_pose(g, V, moves, cx, cy, cz, col, SP, lane, L, gmask);
  return score_posed(V, G, col, SP, lane, L, gmask, coords_out);
}

__device__ __forceinline__ unsigned group_mask(int L) {
  if (L >= 32) return 0xffffffffu;
  const unsigned base = (threadIdx.x & 31) & ~(unsigned)(L - 1);
  return ((1u << L) - 1u) << base;
}

}  // namespace dk
