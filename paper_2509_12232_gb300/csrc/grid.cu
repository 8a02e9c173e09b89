// Grid-map construction (Section V: the inter-energy is memoised in 3-D maps
// around the fixed protein, one per ligand atom type, as AutoGrid does).
//
// One thread per node, nodes tiled 8 x 8 x 4 per block; the 8 x 4 nodes of a
// warp walk the atom ranges of cutoff_ranges_box over their bounding box (at
// most nine rows of 8 A y-z cells, each trimmed in x to the chord of the
// cutoff sphere), so their loops and loads stay uniform.
// A float32 distance test prefilters, the kept pairs are evaluated and summed
// in FP64 and the node values are rounded to FP32 once:
//   M_t = sum_j min(c12 r^-12 - c6 r^-6 - c10 r^-10, w EMAX) + W_sol (solpar_t V_j + S_j V_t) g(r)
//   E   = sum_j W_elec 332.06363 q_j / (eps(r) r)
//   D   = sum_j W_sol 0.01097 V_j g(r),          g(r) = exp(-r^2 / (2 sigma^2))
// with the type-pair coefficients c12, c6, c10 (weight w folded in; 12-10 form
// for donor-acceptor pairs) from an FP64 table, r floored at 0.5 A, pairs at
// r >= 8 A skipped and M_t capped at EMAX.
// Layout: float4 {M_t, E, D, 0} in [t][z][y][x] order.
#include "device_common.cuh"

namespace dk {

namespace {

__global__ void __launch_bounds__(256) grid_build_kernel(const GridBuildArgs A) {
  __shared__ double4 s_coef[DOCK_MAX_TYPES * DOCK_MAX_TYPES];  // {c12, c6, c10, w EMAX}
  __shared__ double2 s_sv[DOCK_MAX_TYPES];                      // {solpar, vol}
  const int T = A.n_types;
  const int tid = threadIdx.x + blockDim.x * (threadIdx.y + blockDim.y * threadIdx.z);
  for (int i = tid; i < T * T; i += 256) s_coef[i] = A.coef[i];
  for (int i = tid; i < T; i += 256) s_sv[i] = A.tsv[i];
  __syncthreads();
  const int ix = blockIdx.x * blockDim.x + threadIdx.x;
  const int iy = blockIdx.y * blockDim.y + threadIdx.y;
  const int iz = blockIdx.z * blockDim.z + threadIdx.z;
  // the nodes of this warp (8 x 4 x 1 of the 8 x 8 x 4 block) share one cell
  // walk over their bounding box: uniform ranges, broadcast loads
  const int wy = blockIdx.y * 8 + ((tid >> 5) & 1) * 4;
  const float bxl = (float)(A.ox + (blockIdx.x * 8) * A.h);
  const float bxh = (float)(A.ox + (blockIdx.x * 8 + 7) * A.h);
  const float byl = (float)(A.oy + wy * A.h), byh = (float)(A.oy + (wy + 3) * A.h);
  const float bz = (float)(A.oz + iz * A.h);
  if (ix >= A.n || iy >= A.n || iz >= A.n) return;
  const double px = A.ox + ix * A.h, py = A.oy + iy * A.h, pz = A.oz + iz * A.h;
  const float pxf = (float)px, pyf = (float)py, pzf = (float)pz;
  double m[DOCK_MAX_TYPES];
#pragma unroll
  for (int t = 0; t < DOCK_MAX_TYPES; ++t) m[t] = 0.0;
  double E = 0.0, D = 0.0;
  const double inv2s2 = 1.0 / (2.0 * kSigma * kSigma);
  const double kE = (double)kWElec * kCoulomb, kD = (double)kWSol * kQasp;
  cutoff_ranges_box(A.cells, bxl, bxh, byl, byh, bz, bz, kCutoffSearch2, [&](int j0, int j1) {
    for (int j = j0; j < j1; ++j) {
      const float4 p = __ldg(A.cprot + j);
      const float dxf = pxf - p.x, dyf = pyf - p.y, dzf = pzf - p.z;
      if (dxf * dxf + dyf * dyf + dzf * dzf > 64.5f) continue;
      const double dx = px - (double)p.x, dy = py - (double)p.y, dz = pz - (double)p.z;
      const double r2 = dx * dx + dy * dy + dz * dz;
      if (!(r2 < 64.0)) continue;
      const double r2c = r2 < 0.25 ? 0.25 : r2;  // r floored at 0.5 A
      const double r = sqrt(r2c);
      const double ir2 = 1.0 / r2c, ir4 = ir2 * ir2, ir6 = ir4 * ir2;
      const double ir10 = ir6 * ir4, ir12 = ir6 * ir6;
      const float4 ex = __ldg(A.cext + j);  // {S_j, V_j, type, 0}
      const int tj = (int)ex.z;
      const double qj = p.w, vj = ex.y;
      const double g = exp(-r2c * inv2s2);
      const double aj = (double)kWSol * vj * g, bj = (double)kWSol * (double)ex.x * g;
#pragma unroll
      for (int t = 0; t < DOCK_MAX_TYPES; ++t) {
        if (t < T) {
          const double4 c = s_coef[t * T + tj];
          const double raw = c.x * ir12 - c.y * ir6 - c.z * ir10;
          m[t] += (raw > c.w ? c.w : raw) + s_sv[t].x * aj + s_sv[t].y * bj;
        }
      }
      const double diel = kDielA + kDielB / (1.0 + kDielK * exp(-kDielLambda * kDielB * r));
      E += kE * qj / (diel * r);
      D += kD * vj * g;
    }
  });
  const int64_t nn = (int64_t)A.n * A.n * A.n;
  const int64_t node = ((int64_t)iz * A.n + iy) * A.n + ix;
  A.fpm[node] = make_float2((float)(E + D), (float)(E - D));
#pragma unroll
  for (int t = 0; t < DOCK_MAX_TYPES; ++t) {
    if (t < T) {
      const double mt = m[t] > kEmax ? kEmax : m[t];
      A.maps[(int64_t)t * nn + node] = make_float4((float)mt, (float)E, (float)D, 0.0f);
    }
  }
}
}  // namespace

cudaError_t launch_grid_build_impl(const GridBuildArgs &A, cudaStream_t s) {
  const dim3 blk(8, 8, 4);
  const dim3 grd((A.n + 7) / 8, (A.n + 7) / 8, (A.n + 3) / 4);
  grid_build_kernel<<<grd, blk, 0, s>>>(A);
  return cudaGetLastError();
}

// (x, y)-cell records for the FP32 scorer: record (t, sign, z, y, x) holds
// {M_t, F} at (x, y), (x+1, y), (x, y+1), (x+1, y+1); F = E + D for sign 0 and
// E - D for sign 1.
__global__ void xycell_maps_kernel(const float4 *maps, const float2 *fpm, int n_types, int n,
                                   float *xycell) {
  const int64_t nc = n - 1, plane = (int64_t)nc * nc, vol = (int64_t)n * n * n;
  const int64_t total = (int64_t)n_types * 2 * n * plane;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < total;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ix = c % nc, iy = (c / nc) % nc, iz = (c / plane) % n, tsg = c / (plane * n);
    const int t = (int)(tsg >> 1), sg = (int)(tsg & 1);
    float v[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int64_t node = (iz * n + iy + (k >> 1)) * n + ix + (k & 1);
      const float2 f = fpm[node];
      v[2 * k] = maps[(int64_t)t * vol + node].x;
      v[2 * k + 1] = sg ? f.y : f.x;
    }
    float4 *o = reinterpret_cast<float4 *>(xycell + c * 8);
    o[0] = make_float4(v[0], v[1], v[2], v[3]);
    o[1] = make_float4(v[4], v[5], v[6], v[7]);
  }
}

cudaError_t launch_xycell_maps(const float4 *maps, const float2 *fpm, int n_types, int n,
                               float *xycell, cudaStream_t s) {
  xycell_maps_kernel<<<152 * 8, 256, 0, s>>>(maps, fpm, n_types, n, xycell);
  return cudaGetLastError();
}

}  // namespace dk
