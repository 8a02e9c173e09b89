// Best-pose bookkeeping and FP64 rescoring.
//
// After the last generation each ligand's DOCK_N_BEST individuals by
// (FP32 score, index) are re-posed and rescored in FP64 (the paper fixes
// scoring to float for speed and notes AutoDock also supports double,
// Section VII "Software"); one warp rescores one pose. The FP64 path
// interpolates the FP32 maps in FP64 and evaluates the intra pair terms in
// FP64 from the per-type parameters.
#include "device_common.cuh"

namespace dk {

// ---- FP64 pair terms ----------------------------------------------------------
__device__ __forceinline__ double pow_int(double x, int n) {
  double r = 1.0;
  for (int i = 0; i < n; ++i) r *= x;
  return r;
}

__device__ double pair_energy64(const dock_type_params *P, int ti, int tj, double qi, double qj,
                                double r) {
  if (!(r < 8.0)) return 0.0;
  if (r < 0.5) r = 0.5;
  const int ri = P[ti].hb_role, rj = P[tj].hb_role;
  const bool hb = (ri == 1 && rj == 2) || (ri == 2 && rj == 1);
  double disp;
  if (hb) {
    const int acc = ri == 2 ? ti : tj;
    const double R = P[acc].hb_R, e = P[acc].hb_eps, s = R / r;
    disp = 5.0 * e * pow_int(s, 12) - 6.0 * e * pow_int(s, 10);
    disp = (disp > kEmax ? kEmax : disp) * (double)kWHb;
  } else {
    const double R = 0.5 * ((double)P[ti].Rii + (double)P[tj].Rii);
    const double e = sqrt((double)P[ti].eps * (double)P[tj].eps), s = R / r;
    disp = e * pow_int(s, 12) - 2.0 * e * pow_int(s, 6);
    disp = (disp > kEmax ? kEmax : disp) * (double)kWVdw;
  }
  const double diel = kDielA + kDielB / (1.0 + kDielK * exp(-kDielLambda * kDielB * r));
  const double elec = (double)kWElec * kCoulomb * qi * qj / (diel * r);
  const double si = (double)P[ti].solpar + kQasp * fabs(qi);
  const double sj = (double)P[tj].solpar + kQasp * fabs(qj);
  const double des = (double)kWSol * (si * (double)P[tj].vol + sj * (double)P[ti].vol) *
                     exp(-r * r / (2.0 * kSigma * kSigma));
  return disp + elec + des;
}

// Sum of the pair terms of ligand l's pose-invariant pairs at its input
// geometry, one warp per ligand; lane-strided partial sums combined by a
// fixed shuffle tree.
__global__ void intra_const_kernel(LigInfo *ligs, int n_ligands, const float4 *atoms_raw,
                                   const uint8_t *types, const uint32_t *pair_idx,
                                   const dock_type_params *params) {
  const int l = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (l >= n_ligands) return;
  const LigInfo li = ligs[l];
  const float4 *at = atoms_raw + li.atom_off;
  const uint8_t *ty = types + li.atom_off;
  double e = 0.0;
  for (int p = li.n_pairs + lane; p < li.n_pairs_all; p += 32) {
    const uint32_t idx = pair_idx[li.pair_off + p];
    const int i = idx & 255, j = (idx >> 8) & 255;
    const double dx = (double)at[i].x - (double)at[j].x, dy = (double)at[i].y - (double)at[j].y,
                 dz = (double)at[i].z - (double)at[j].z;
    e += pair_energy64(params, ty[i], ty[j], (double)at[i].w, (double)at[j].w,
                       sqrt(dx * dx + dy * dy + dz * dz));
  }
  for (int off = 16; off > 0; off >>= 1) e += __shfl_xor_sync(0xffffffffu, e, off);
  if (lane == 0) ligs[l].intra_const = (float)e;
}

cudaError_t launch_intra_const(LigInfo *ligs, int n_ligands, const float4 *atoms_raw,
                               const uint8_t *types, const uint32_t *pair_idx,
                               const dock_type_params *params, cudaStream_t s) {
  if (n_ligands == 0) return cudaSuccess;
  const int per_block = 8;
  intra_const_kernel<<<(n_ligands + per_block - 1) / per_block, 32 * per_block, 0, s>>>(
      ligs, n_ligands, atoms_raw, types, pair_idx, params);
  return cudaGetLastError();
}

struct GridView64 {
  const float4 *maps;
  int n;
  double ox, oy, oz, h;
};

__device__ bool grid_energy64(const GridView64 &G, int t, double q, double x, double y, double z,
                              double &e) {
  const double u[3] = {(x - G.ox) / G.h, (y - G.oy) / G.h, (z - G.oz) / G.h};
  int i0[3];
  double f[3];
  for (int m = 0; m < 3; ++m) {
    if (!(u[m] >= 0.0 && u[m] <= (double)(G.n - 1))) return false;
    i0[m] = (int)floor(u[m]);
    if (i0[m] > G.n - 2) i0[m] = G.n - 2;
    f[m] = u[m] - i0[m];
  }
  double acc = 0.0;
  for (int c = 0; c < 8; ++c) {
    const int dx = c & 1, dy = (c >> 1) & 1, dz = (c >> 2) & 1;
    const float4 v = G.maps[(((int64_t)t * G.n + i0[2] + dz) * G.n + i0[1] + dy) * G.n + i0[0] + dx];
    const double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
    acc += w * ((double)v.x + q * (double)v.y + fabs(q) * (double)v.z);
  }
  e = acc;
  return true;
}

// FP64 pairwise inter-energy of this lane's atoms (lane, lane + 32, ...):
// every protein atom within the cutoff of the cell list, the pair terms in
// FP64 (the no-grid search's rescoring).
__device__ double pairwise_inter64(const Fp64Args &F, const float4 *atoms, const uint8_t *types,
                                   int n, const double *xyz) {
  const PwView &W = F.pw;
  const CellGrid &C = W.cells;
  // the cell ranges of cutoff_ranges, bounds in FP64 (margin as there)
  const double rc2 = (double)kCutoffSearch2;
  auto span = [](double u, int d, int &lo, int &hi) {
    const double c = floor(fmin(fmax(u, -4.0), (double)d + 4.0));
    lo = max((int)c - 1, 0);
    hi = min((int)c + 1, d - 1);
  };
  double e = 0.0;
  for (int a = threadIdx.x & 31; a < n; a += 32) {
    const double x = xyz[3 * a], y = xyz[3 * a + 1], z = xyz[3 * a + 2];
    const double ux = (x - (double)C.lox) / (double)kCellX;
    int y0, y1, z0, z1;
    span((y - (double)C.loy) / (double)kCellYZ, C.dy, y0, y1);
    span((z - (double)C.loz) / (double)kCellYZ, C.dz, z0, z1);
    for (int cz = z0; cz <= z1; ++cz) {
      const double zl = (double)C.loz + cz * (double)kCellYZ;
      const double dzv = fmax(fmax(zl - z, z - (zl + (double)kCellYZ)), 0.0);
      for (int cy = y0; cy <= y1; ++cy) {
        const double yl = (double)C.loy + cy * (double)kCellYZ;
        const double dyv = fmax(fmax(yl - y, y - (yl + (double)kCellYZ)), 0.0);
        const double d2 = dyv * dyv + dzv * dzv;
        if (!(d2 < rc2)) continue;
        const double h = sqrt(rc2 - d2) / (double)kCellX;
        const int xa = max((int)floor(fmin(fmax(ux - h, -1.0), (double)C.dx)), 0);
        const int xb = min((int)floor(fmin(fmax(ux + h, -1.0), (double)C.dx)), C.dx - 1);
        if (xa > xb) continue;
        const int row = (cz * C.dy + cy) * C.dx;
        const int j1 = C.cell_start[row + xb + 1];
        for (int j = C.cell_start[row + xa]; j < j1; ++j) {
          const float4 b = W.cprot[j];
          const double dx = x - (double)b.x, dy = y - (double)b.y, dz = z - (double)b.z;
          const double r = sqrt(dx * dx + dy * dy + dz * dz);
          if (r < 8.0)
            e += pair_energy64(F.params, types[a], (int)W.cext[j].z, (double)atoms[a].w,
                               (double)b.w, r);
        }
      }
    }
  }
  return e;
}

// Pose + score of one genotype in FP64 by one warp. xyz: smem [128][3].
__device__ double pose_score_fp64_warp(const float *geno, const LigInfo &li, const Fp64Args &F,
                                       const GridView64 &G, const double *cent, double *xyz) {
  const int lane = threadIdx.x & 31;
  const float4 *atoms = F.atoms + li.atom_off;
  const uint8_t *types = F.types + li.atom_off;
  double q[4] = {geno[3], geno[4], geno[5], geno[6]};
  const double nq = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  const double w = q[0] / nq, x = q[1] / nq, y = q[2] / nq, z = q[3] / nq;
  const double R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z),     2 * (x * z + w * y),
                       2 * (x * y + w * z),     1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                       2 * (x * z - w * y),     2 * (y * z + w * x),     1 - 2 * (x * x + y * y)};
  const double t[3] = {F.cx + (double)geno[0], F.cy + (double)geno[1], F.cz + (double)geno[2]};
  for (int a = lane; a < li.n; a += 32) {
    const float4 p = atoms[a];  // raw input coordinates
    const double v[3] = {(double)p.x - cent[0], (double)p.y - cent[1], (double)p.z - cent[2]};
    for (int m = 0; m < 3; ++m)
      xyz[3 * a + m] = R[3 * m] * v[0] + R[3 * m + 1] * v[1] + R[3 * m + 2] * v[2] + t[m];
  }
  __syncwarp();
  for (int j = 0; j < li.k; ++j) {
    const TorInfo T = F.tors[li.tors_off + j];
    const double a0 = xyz[3 * T.a], a1 = xyz[3 * T.a + 1], a2 = xyz[3 * T.a + 2];
    double u0 = xyz[3 * T.b] - a0, u1 = xyz[3 * T.b + 1] - a1, u2 = xyz[3 * T.b + 2] - a2;
    const double len = sqrt(u0 * u0 + u1 * u1 + u2 * u2);
    u0 /= len; u1 /= len; u2 /= len;
    double s, c;
    sincos((double)geno[7 + j], &s, &c);
    for (int m = lane; m < T.n_move; m += 32) {
      const int at = F.moves[T.move_off + m];
      const double p0 = xyz[3 * at] - a0, p1 = xyz[3 * at + 1] - a1, p2 = xyz[3 * at + 2] - a2;
      const double d = u0 * p0 + u1 * p1 + u2 * p2;
      const double c0 = u1 * p2 - u2 * p1, c1 = u2 * p0 - u0 * p2, c2 = u0 * p1 - u1 * p0;
      xyz[3 * at] = a0 + p0 * c + c0 * s + u0 * d * (1.0 - c);
      xyz[3 * at + 1] = a1 + p1 * c + c1 * s + u1 * d * (1.0 - c);
      xyz[3 * at + 2] = a2 + p2 * c + c2 * s + u2 * d * (1.0 - c);
    }
    __syncwarp();
  }
  double e = 0.0;
  if (F.pairwise) {
    e = pairwise_inter64(F, atoms, types, li.n, xyz);
  } else {
    for (int a = lane; a < li.n; a += 32) {
      double v;
      if (grid_energy64(G, types[a], (double)atoms[a].w, xyz[3 * a], xyz[3 * a + 1], xyz[3 * a + 2],
                        v))
        e += v;
      else
        e += (double)kEout;
    }
  }
  for (int p = lane; p < li.n_pairs_all; p += 32) {
    const uint32_t idx = F.pair_idx[li.pair_off + p];
    const int i = idx & 255, j = (idx >> 8) & 255;
    const double dx = xyz[3 * i] - xyz[3 * j], dy = xyz[3 * i + 1] - xyz[3 * j + 1],
                 dz = xyz[3 * i + 2] - xyz[3 * j + 2];
    e += pair_energy64(F.params, types[i], types[j], (double)atoms[i].w, (double)atoms[j].w,
                       sqrt(dx * dx + dy * dy + dz * dz));
  }
  for (int off = 16; off > 0; off >>= 1) e += __shfl_xor_sync(0xffffffffu, e, off);
  __syncwarp();
  return e;
}

__host__ __device__ __forceinline__ GridView64 grid64(const Fp64Args &F) {
  GridView64 G;
  G.maps = F.grid.maps;
  G.n = F.grid.n;
  G.h = F.h;
  return G;
}

struct FinalArgs {
  Fp64Args f;
  GridView64 g64;
  const double *centroids;   // [n_ligands][3]
  int pop;
  const int64_t *geno_off;
  const float *genos;
  const float *scores;
  const int32_t *lig_status;
  const int32_t *status;
  uint64_t exact_evals, surrogate_evals;
  const unsigned long long *extra_evals;  // optional [n_ligands] (local-search probes)
  dock_result *out;
};

// One CTA (256 threads) per ligand: best 8 by (score, index), then FP64.
__global__ void __launch_bounds__(256) finalize_kernel(const FinalArgs A) {
  __shared__ unsigned long long s_red[8];
  __shared__ int s_best[DOCK_N_BEST];
  __shared__ double s_xyz[8][DOCK_MAX_ATOMS * 3];
  __shared__ double s_e64[DOCK_N_BEST];
  const int lig = blockIdx.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const float *sc = A.scores + (int64_t)lig * A.pop;
  // thread-local sorted best 8 keys
  unsigned long long best[DOCK_N_BEST];
#pragma unroll
  for (int r = 0; r < DOCK_N_BEST; ++r) best[r] = ~0ull;
  for (int i = tid; i < A.pop; i += blockDim.x) {
    unsigned long long key = ((unsigned long long)score_key(sc[i]) << 32) | (unsigned)i;
#pragma unroll
    for (int r = 0; r < DOCK_N_BEST; ++r) {
      if (key < best[r]) {
        const unsigned long long t = best[r];
        best[r] = key;
        key = t;
      }
    }
  }
  for (int r = 0; r < DOCK_N_BEST; ++r) {
    unsigned long long m = best[0];
    for (int off = 16; off > 0; off >>= 1) {
      const unsigned long long o = __shfl_xor_sync(0xffffffffu, m, off);
      m = o < m ? o : m;
    }
    if (lane == 0) s_red[warp] = m;
    __syncthreads();
    unsigned long long g = s_red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) g = s_red[w] < g ? s_red[w] : g;
    if (best[0] == g && g != ~0ull) {  // unique owner (keys carry the index)
#pragma unroll
      for (int q = 0; q < DOCK_N_BEST - 1; ++q) best[q] = best[q + 1];
      best[DOCK_N_BEST - 1] = ~0ull;
    }
    if (tid == 0) s_best[r] = g == ~0ull ? -1 : (int)(g & 0xffffffffull);
    __syncthreads();
  }
  const LigInfo li = A.f.ligs[lig];
  const int G = 7 + li.k;
  if (warp < DOCK_N_BEST) {
    const int bi = s_best[warp];
    double e = __longlong_as_double(0x7ff8000000000000ULL);
    if (bi >= 0) {
      const float *geno = A.genos + A.geno_off[lig] + (int64_t)bi * G;
      e = pose_score_fp64_warp(geno, li, A.f, A.g64, A.centroids + 3 * lig, s_xyz[warp]);
    }
    if (lane == 0) s_e64[warp] = e;
  }
  __syncthreads();
  dock_result *R = A.out + lig;
  if (tid == 0) {
    R->ligand_id = li.ligand_id;
    R->n_genes = G;
    int st = A.lig_status ? A.lig_status[lig] : 0;
    if (*A.status != 0) st = *A.status;
    R->status = st;
    R->exact_evals = A.exact_evals + (A.extra_evals ? A.extra_evals[lig] : 0ull);
    R->surrogate_evals = A.surrogate_evals;
  }
  if (tid < DOCK_N_BEST) {
    const int bi = s_best[tid];
    R->best_index[tid] = bi;
    R->best_fp32[tid] = bi >= 0 ? sc[bi] : __int_as_float(0x7fc00000);
    R->best_fp64[tid] = s_e64[tid];
  }
  for (int e = tid; e < DOCK_N_BEST * DOCK_MAX_GENES; e += blockDim.x) {
    const int r = e / DOCK_MAX_GENES, gi = e % DOCK_MAX_GENES;
    const int bi = s_best[r];
    R->genotype[r][gi] = (bi >= 0 && gi < G) ? A.genos[A.geno_off[lig] + (int64_t)bi * G + gi] : 0.0f;
  }
}

// One warp per ligand: the minimum of (score key << 32) | index.
__global__ void best_keys_kernel(const float *scores, int n_ligands, int pop,
                                 unsigned long long *best) {
  const int lig = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (lig >= n_ligands) return;  // whole warps
  const int lane = threadIdx.x & 31;
  const float *sc = scores + (int64_t)lig * pop;
  unsigned long long k = ~0ull;
  for (int i = lane; i < pop; i += 32) {
    const unsigned long long c = ((unsigned long long)score_key(sc[i]) << 32) | (uint32_t)i;
    k = c < k ? c : k;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long c = __shfl_xor_sync(0xffffffffu, k, o);
    k = c < k ? c : k;
  }
  if (lane == 0) best[lig] = k;
}

cudaError_t launch_best_keys(const float *scores, int n_ligands, int pop,
                             unsigned long long *best, cudaStream_t s) {
  if (n_ligands == 0) return cudaSuccess;
  best_keys_kernel<<<(n_ligands + 7) / 8, 256, 0, s>>>(scores, n_ligands, pop, best);
  return cudaGetLastError();
}

cudaError_t launch_finalize_impl(const Fp64Args &f, const double *centroids, int n_ligands, int pop,
                                 const int64_t *geno_off, const float *genos, const float *scores,
                                 const int32_t *lig_status, const int32_t *status,
                                 uint64_t exact_evals, uint64_t surrogate_evals,
                                 const unsigned long long *extra_evals, double ox, double oy,
                                 double oz, dock_result *out, cudaStream_t s) {
  if (n_ligands == 0) return cudaSuccess;
  FinalArgs A;
  A.f = f;
  A.g64 = grid64(f);
  A.g64.ox = ox; A.g64.oy = oy; A.g64.oz = oz;
  A.centroids = centroids;
  A.pop = pop;
  A.geno_off = geno_off;
  A.genos = genos;
  A.scores = scores;
  A.lig_status = lig_status;
  A.status = status;
  A.exact_evals = exact_evals;
  A.surrogate_evals = surrogate_evals;
  A.extra_evals = extra_evals;
  A.out = out;
  finalize_kernel<<<n_ligands, 256, 0, s>>>(A);
  return cudaGetLastError();
}

// FP64 scoring of caller-given poses: one warp per pose.
struct Score64Args {
  Fp64Args f;
  GridView64 g64;
  const double *centroids;
  const int32_t *pose_ligand;
  int n_ligands;
  const float *genos;
  int64_t n_poses;
  double *out;
};

__global__ void __launch_bounds__(128) score64_kernel(const Score64Args A) {
  __shared__ double s_xyz[4][DOCK_MAX_ATOMS * 3];
  const int warp = threadIdx.x >> 5;
  const int64_t pose = (int64_t)blockIdx.x * 4 + warp;
  if (pose >= A.n_poses) return;
  const int lig = A.pose_ligand[pose];
  if (lig < 0 || lig >= A.n_ligands) {
    if ((threadIdx.x & 31) == 0) A.out[pose] = __longlong_as_double(0x7ff8000000000000ULL);
    return;
  }
  const LigInfo li = A.f.ligs[lig];
  const double e = pose_score_fp64_warp(A.genos + pose * DOCK_MAX_GENES, li, A.f, A.g64,
                                        A.centroids + 3 * lig, s_xyz[warp]);
  if ((threadIdx.x & 31) == 0) A.out[pose] = e;
}

cudaError_t launch_score_fp64_impl(const Fp64Args &f, const double *centroids, double ox, double oy,
                                   double oz, const int32_t *pose_ligand, int n_ligands,
                                   const float *genos, int64_t n_poses, double *out, cudaStream_t s) {
  if (n_poses == 0) return cudaSuccess;
  Score64Args A;
  A.f = f;
  A.g64 = grid64(f);
  A.g64.ox = ox; A.g64.oy = oy; A.g64.oz = oz;
  A.centroids = centroids;
  A.pose_ligand = pose_ligand;
  A.n_ligands = n_ligands;
  A.genos = genos;
  A.n_poses = n_poses;
  A.out = out;
  score64_kernel<<<(unsigned)((n_poses + 3) / 4), 128, 0, s>>>(A);
  return cudaGetLastError();
}

}  // namespace dk
