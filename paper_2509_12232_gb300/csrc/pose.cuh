// Device functions of the pose (Algorithm 1) and score (Algorithm 2) shared
// by the search, scoring and feature kernels. L, the number of lanes that
// share a pose, is a template parameter (1, 2, 4 or 8).
#pragma once

#include "device_common.cuh"

namespace dk {

// Coordinate slots in shared memory: pose slot s owns float4 rows
// [s * SS, s * SS + L * apl), atom a at row a (byte offset 16 a), with
// SS = (L * apl rounded up to 8) + (L mod 8). The 16-byte loads of a
// quarter warp (8 / L slots x L lanes reading consecutive atoms of their own
// slot) then fall on distinct bank groups.
__host__ __device__ constexpr int slot_stride(int L, int apl) {
  return ((L * apl + 7) & ~7) + (L & 7);
}

__host__ __device__ constexpr int slots_bytes(int threads, int L, int apl) {
  return (threads / L) * slot_stride(L, apl) * 16;
}

struct LigView {
  const float4 *atoms;      // this ligand's atoms (centred) + charge
  const uint8_t *types;
  const float *pair_rec;    // 4 floats per pair
  const TorInfo *tors;
  int n, k, n_pairs;
  float intra_const;  // energy of the pose-invariant pairs
#ifdef DOCK_CHECKED
  int32_t *word;      // status word of the call
  int64_t moves;      // moved-atom entries of the set
  int rows;           // float4 rows of the pose slot
#endif
};

// b, slot_rows: array sizes for the bounds-checked build (unused otherwise);
// there a ligand whose rows do not fit its arrays or its slot gets no work.
__device__ __forceinline__ LigView lig_view(const LigInfo &li, const float4 *atoms,
                                            const uint8_t *types, const float *pair_rec,
                                            const TorInfo *tors, const Bounds *b = nullptr,
                                            int slot_rows = 0) {
  LigView v;
  v.atoms = atoms + li.atom_off;
  v.types = types + li.atom_off;
  v.pair_rec = pair_rec + (int64_t)li.pair_off * 4;
  v.tors = tors + li.tors_off;
  v.n = li.n;
  v.k = li.k;
  v.n_pairs = li.n_pairs;
  v.intra_const = li.intra_const;
#ifdef DOCK_CHECKED
  // without bounds (callers outside the checked kernels) every check passes
  v.word = b ? b->word : nullptr;
  v.moves = b ? b->moves : INT64_MAX;
  v.rows = b ? slot_rows : (1 << 20);
  if (b) {
    const bool ok = DK_OK((int64_t)li.atom_off + li.n <= b->atoms && li.atom_off >= 0, v.word, 1) &&
                    DK_OK((int64_t)li.pair_off + li.n_pairs <= b->pairs && li.pair_off >= 0,
                          v.word, 2) &&
                    DK_OK((int64_t)li.tors_off + li.k <= b->tors && li.tors_off >= 0, v.word, 3) &&
                    DK_OK(li.n <= slot_rows && li.k <= DOCK_MAX_TORSIONS, v.word, 4);
    if (!ok) v.n = v.k = v.n_pairs = 0;
  }
#endif
  return v;
}

__device__ __forceinline__ float4 slot_row(const float4 *slot, uint32_t byte_off) {
  return *reinterpret_cast<const float4 *>(reinterpret_cast<const char *>(slot) + byte_off);
}

// Pair terms of one lane, pairs lane, lane + L, ... of the row-ordered list:
// consecutive pairs of a lane mostly share atom i, whose coordinates (and
// scaled charge, in w) stay in registers. The 16-byte record carries the byte
// offsets of both atoms in the slot.
template <int L>
struct PairWalker {
  const float *rec;  // this lane's first record
  const float4 *slot;
  uint32_t last_i = 0xffffffffu;
  float4 ci;
#ifdef DOCK_CHECKED
  const LigView *V;
  int lane;
  __device__ __forceinline__ PairWalker(const LigView &v, const float4 *s, int ln)
      : rec(v.pair_rec + ln * 4), slot(s), V(&v), lane(ln) {}
#else
  __device__ __forceinline__ PairWalker(const LigView &v, const float4 *s, int lane)
      : rec(v.pair_rec + lane * 4), slot(s) {}
#endif
  // m: the lane's pair counter (pair lane + m L)
  __device__ __forceinline__ float term(int m) {
#ifdef DOCK_CHECKED
    const bool in = DK_OK(lane + m * L < V->n_pairs, V->word, 5);
    const float4 r = ld4(rec + (in ? m * (4 * L) : -lane * 4));
    uint32_t oij = __float_as_uint(r.x);
    if (!DK_OK((oij & 0xffffu) < 16u * V->rows && (oij >> 16) < 16u * V->rows, V->word, 6))
      oij = 0;
#else
    const float4 r = ld4(rec + m * (4 * L));
    const uint32_t oij = __float_as_uint(r.x);
#endif
    const uint32_t oi = oij & 0xffffu;
    if (oi != last_i) {
      ci = slot_row(slot, oi);
      last_i = oi;
    }
    const float4 b = slot_row(slot, oij >> 16);
    const float dx = ci.x - b.x, dy = ci.y - b.y, dz = ci.z - b.z;
    return pair_energy16(dx * dx + dy * dy + dz * dz, r.y, r.z, r.w, ci.w * b.w);
  }
};

// Algorithm 1 for one genotype by a group of L lanes: the posed coordinates
// go to the pose's slot.
template <int L>
__device__ __forceinline__ void apply_pose(const float (&g)[DOCK_MAX_GENES], const LigView &V,
                                           const uint8_t *moves, float cx, float cy, float cz,
                                           float4 *slot, int lane, unsigned gmask) {
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
  // w of a row: the atom's charge scaled by sqrt(W_elec 332.06363), so that a
  // pair's qq is the product of its two rows' w
  const float kq = kChargeScale;
  for (int a = lane; a < V.n; a += L) {
    const float4 p = __ldg(V.atoms + a);
    slot[a] = make_float4(r00 * p.x + r01 * p.y + r02 * p.z + tx,
                          r10 * p.x + r11 * p.y + r12 * p.z + ty,
                          r20 * p.x + r21 * p.y + r22 * p.z + tz, kq * p.w);
  }
  __syncwarp(gmask);
  // ---- torsions root to leaf, each about the current bond axis ------------
  // (a rolled loop keeps the code small; the angle is picked from the
  // register genotype by selects, not by a dynamic index)
#pragma unroll 1
  for (int j = 0; j < V.k; ++j) {
    {
      TorInfo T = V.tors[j];
#ifdef DOCK_CHECKED
      if (!DK_OK(T.a < V.n && T.b < V.n && T.move_off >= 0 && T.n_move >= 0 &&
                     (int64_t)T.move_off + T.n_move <= V.moves, V.word, 7)) {
        T.a = T.b = 0;
        T.n_move = 0;
      }
#endif
      const float4 pa = slot[T.a], pb = slot[T.b];
      float ux = pb.x - pa.x, uy = pb.y - pa.y, uz = pb.z - pa.z;
      const float il = rsqrt_ftz(ux * ux + uy * uy + uz * uz);
      ux *= il; uy *= il; uz *= il;
      float theta = g[7];
#pragma unroll
      for (int q = 1; q < DOCK_MAX_TORSIONS; ++q) theta = j == q ? g[7 + q] : theta;
      float s, c;
      __sincosf(theta, &s, &c);
      const float oc = 1.f - c;
      const float m00 = c + ux * ux * oc, m01 = ux * uy * oc - uz * s, m02 = ux * uz * oc + uy * s;
      const float m10 = uy * ux * oc + uz * s, m11 = c + uy * uy * oc, m12 = uy * uz * oc - ux * s;
      const float m20 = uz * ux * oc - uy * s, m21 = uz * uy * oc + ux * s, m22 = c + uz * uz * oc;
      const uint8_t *mv = moves + T.move_off;
      for (int m = lane; m < T.n_move; m += L) {
        int at = mv[m];
#ifdef DOCK_CHECKED
        if (!DK_OK(at < V.n, V.word, 8)) at = 0;
#endif
        const float4 p = slot[at];
        const float vx = p.x - pa.x, vy = p.y - pa.y, vz = p.z - pa.z;
        slot[at] = make_float4(pa.x + m00 * vx + m01 * vy + m02 * vz,
                               pa.y + m10 * vx + m11 * vy + m12 * vz,
                               pa.z + m20 * vx + m21 * vy + m22 * vz, p.w);
      }
      __syncwarp(gmask);
    }
  }
}

// Algorithm 2 for the posed ligand in `slot`: every lane of the group returns
// the same FP32 score.
template <int L>
__device__ __forceinline__ float score_posed(const LigView &V, const GridView &G,
                                             const float4 *slot, int lane, unsigned gmask,
                                             float *coords_out) {
  // ---- Algorithm 2: each grid lookup (inter-energy of one atom) is issued,
  // ---- a share of the intra pairs (whole blocks of four) runs while its
  // ---- loads are in flight, then the lookup is interpolated ----------------
  Kahan acc;
  if (lane == 0) acc.add(V.intra_const);
  PairWalker<L> W(V, slot, lane);
  const int na = V.n > lane ? (V.n - lane + L - 1) / L : 0;               // atoms lane + k L
  const int np_l = V.n_pairs > lane ? (V.n_pairs - lane + L - 1) / L : 0;  // pairs lane + m L
  const int ppa = na > 0 ? (((np_l + na - 1) / na) + 3) & ~3 : 0;          // pairs per atom
  int m = 0;
  for (int k = 0; k < na; ++k) {
    const int a = lane + k * L;
    const float4 pa = slot[a];
#ifdef DOCK_CHECKED
    const Lookup lk = grid_issue(G, V.types[a], __ldg(&V.atoms[a].w), pa.x, pa.y, pa.z, V.word);
#else
    const Lookup lk = grid_issue(G, V.types[a], __ldg(&V.atoms[a].w), pa.x, pa.y, pa.z);
#endif
    if (coords_out) {
      coords_out[3 * a] = pa.x;
      coords_out[3 * a + 1] = pa.y;
      coords_out[3 * a + 2] = pa.z;
    }
    const int m_end = min(np_l, m + ppa);
    for (; m + 7 < m_end; m += 8) {
      const float e0 = W.term(m), e1 = W.term(m + 1), e2 = W.term(m + 2), e3 = W.term(m + 3);
      const float e4 = W.term(m + 4), e5 = W.term(m + 5), e6 = W.term(m + 6), e7 = W.term(m + 7);
      acc.add(((e0 + e1) + (e2 + e3)) + ((e4 + e5) + (e6 + e7)));
    }
    if (m + 3 < m_end) {
      const float e0 = W.term(m), e1 = W.term(m + 1);
      const float e2 = W.term(m + 2), e3 = W.term(m + 3);
      acc.add((e0 + e1) + (e2 + e3));
      m += 4;
    }
    acc.add(grid_finish(lk));
  }
  for (; m < np_l; ++m) acc.add(W.term(m));
  // ---- combine the group's compensated sums --------------------------------
  float s = acc.s, c = acc.c;
#pragma unroll
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

// The pairwise inter-energy of this lane's atoms (lane, lane + L, ...): every
// protein atom within the 8 A cutoff through the pair terms (Algorithm 2's
// inter loop over nearby protein atoms), found through cutoff_ranges. tp /
// sv: the type-pair and per-type tables (in shared or global memory).
template <int L>
__device__ __forceinline__ void pairwise_inter(const LigView &V, const PwView &W,
                                               const float4 *slot, int lane, const float4 *tp,
                                               const float2 *sv, Kahan &acc) {
  const float kElec = (float)((double)kWElec * kCoulomb);
  const int T = W.n_types;
  for (int a = lane; a < V.n; a += L) {
    const float4 p = slot[a];
    const int ti = V.types[a];
    const float qi = __ldg(&V.atoms[a].w);
    const float qe = kElec * qi;
    const float2 svi = sv[ti];
    const float si = (float)kWSol * (svi.x + (float)kQasp * fabsf(qi));  // W_sol S_i
    const float vi = (float)kWSol * svi.y;                               // W_sol V_i
    Kahan ai;
    cutoff_ranges(W.cells, p.x, p.y, p.z, kCutoffSearch2, [&](int j0, int j1) {
#ifdef DOCK_CHECKED
      if (!DK_OK(j0 >= 0 && j0 <= j1 && j1 <= W.n_atoms, V.word, 10)) j1 = j0 = 0;
#endif
      for (int j = j0; j < j1; ++j) {
        const float4 b = __ldg(W.cprot + j);
        const float dx = p.x - b.x, dy = p.y - b.y, dz = p.z - b.z;
        const float r2 = dx * dx + dy * dy + dz * dz;
        if (r2 < kCutoff2) {
          const float4 ex = __ldg(W.cext + j);  // {S_j, V_j, type, 0}
          int tj = (int)ex.z;
#ifdef DOCK_CHECKED
          if (!DK_OK(tj >= 0 && tj < T && ti < T, V.word, 11)) tj = 0;
#endif
          const float4 c = tp[ti * T + tj];
          const float rec[8] = {c.x, c.y, c.z, c.w, qe * b.w, fmaf(si, ex.y, ex.x * vi),
                                0.0f, 0.0f};
          ai.add(pair_energy(r2, rec));
        }
      }
    });
    acc.add(ai.value());
  }
}

// Algorithm 2 with the pairwise inter-energy (no maps) for the posed ligand in
// `slot`: intra pairs as in score_posed, then pairwise_inter; every lane of
// the group returns the same FP32 score.
template <int L>
__device__ __forceinline__ float score_posed_pw(const LigView &V, const PwView &W,
                                                const float4 *slot, int lane, unsigned gmask,
                                                const float4 *tp, const float2 *sv) {
  Kahan acc;
  if (lane == 0) acc.add(V.intra_const);
  PairWalker<L> Wk(V, slot, lane);
  const int np_l = V.n_pairs > lane ? (V.n_pairs - lane + L - 1) / L : 0;
  int m = 0;
  for (; m + 3 < np_l; m += 4) {
    const float e0 = Wk.term(m), e1 = Wk.term(m + 1), e2 = Wk.term(m + 2), e3 = Wk.term(m + 3);
    acc.add((e0 + e1) + (e2 + e3));
  }
  for (; m < np_l; ++m) acc.add(Wk.term(m));
  pairwise_inter<L>(V, W, slot, lane, tp, sv, acc);
  float s = acc.s, c = acc.c;
#pragma unroll
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

template <int L>
__device__ __forceinline__ float pose_and_score(const float (&g)[DOCK_MAX_GENES], const LigView &V,
                                                const uint8_t *moves, const GridView &G, float cx,
                                                float cy, float cz, float4 *slot, int lane,
                                                unsigned gmask, float *coords_out) {
  apply_pose<L>(g, V, moves, cx, cy, cz, slot, lane, gmask);
  return score_posed<L>(V, G, slot, lane, gmask, coords_out);
}

template <int L>
__device__ __forceinline__ unsigned group_mask() {
  if (L >= 32) return 0xffffffffu;
  const unsigned base = (threadIdx.x & 31) & ~(unsigned)(L - 1);
  return ((1u << L) - 1u) << base;
}

}  // namespace dk
