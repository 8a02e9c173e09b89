// Grid-map construction (Section V: the inter-energy is memoised in 3-D maps
// around the fixed protein, one per ligand atom type, as AutoGrid does).
//
// One thread per node. Protein atoms stream through shared memory in tiles;
// a float32 distance test prefilters, the kept pairs are evaluated and summed
// in FP64 and the node values are rounded to FP32 once:
//   M_t = sum_j w min(disp_raw(t, t_j, r), EMAX) + W_sol (solpar_t V_j + S_j V_t) g(r)
//   E   = sum_j W_elec 332.06363 q_j / (eps(r) r)
//   D   = sum_j W_sol 0.01097 V_j g(r),          g(r) = exp(-r^2 / (2 sigma^2))
// with r floored at 0.5 A and pairs at r >= 8 A skipped; M_t capped at EMAX.
// Layout: float4 {M_t, E, D, 0} in [t][z][y][x] order.
#include "device_common.cuh"

namespace dk {

namespace {
constexpr int kTile = 256;

__device__ __forceinline__ double ipow64(double x, int n) {
  double r = 1.0;
  for (int i = 0; i < n; ++i) r *= x;
  return r;
}

struct GridBuildArgs {
  const float4 *prot;
  const uint8_t *ptype;
  int n_prot;
  const dock_type_params *params;
  int n_types;
  int n;
  double ox, oy, oz, h;
  float4 *maps;
  float2 *fpm;   // per node {E + D, E - D}, rounded once from FP64
};

__global__ void __launch_bounds__(256) grid_build_kernel(const GridBuildArgs A) {
  __shared__ float4 s_atom[kTile];
  __shared__ uint8_t s_type[kTile];
  __shared__ dock_type_params s_par[DOCK_MAX_TYPES];
  const int T = A.n_types;
  if (threadIdx.x < T) s_par[threadIdx.x] = A.params[threadIdx.x];
  const int64_t nn = (int64_t)A.n * A.n * A.n;
  const int64_t node = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = node < nn;
  const int ix = (int)(node % A.n), iy = (int)((node / A.n) % A.n), iz = (int)(node / ((int64_t)A.n * A.n));
  const double px = A.ox + ix * A.h, py = A.oy + iy * A.h, pz = A.oz + iz * A.h;
  const float pxf = (float)px, pyf = (float)py, pzf = (float)pz;
  double m[DOCK_MAX_TYPES];
#pragma unroll
  for (int t = 0; t < DOCK_MAX_TYPES; ++t) m[t] = 0.0;
  double E = 0.0, D = 0.0;
  const double inv2s2 = 1.0 / (2.0 * kSigma * kSigma);
  for (int base = 0; base < A.n_prot; base += kTile) {
    __syncthreads();
    const int cnt = min(kTile, A.n_prot - base);
    if (threadIdx.x < cnt) {
      s_atom[threadIdx.x] = A.prot[base + threadIdx.x];
      s_type[threadIdx.x] = A.ptype[base + threadIdx.x];
    }
    __syncthreads();
    if (!active) continue;
    for (int a = 0; a < cnt; ++a) {
      const float4 p = s_atom[a];
      const float dxf = pxf - p.x, dyf = pyf - p.y, dzf = pzf - p.z;
      if (dxf * dxf + dyf * dyf + dzf * dzf > 64.5f) continue;
      const double dx = px - (double)p.x, dy = py - (double)p.y, dz = pz - (double)p.z;
      double r = sqrt(dx * dx + dy * dy + dz * dz);
      if (!(r < 8.0)) continue;
      if (r < 0.5) r = 0.5;
      const int tj = s_type[a];
      const double qj = p.w;
      const double g = exp(-r * r * inv2s2);
      const double sj = (double)s_par[tj].solpar + kQasp * fabs(qj);
      const double vj = s_par[tj].vol;
      const int rj = s_par[tj].hb_role;
#pragma unroll
      for (int t = 0; t < DOCK_MAX_TYPES; ++t) {
        if (t < T) {
          const int rt = s_par[t].hb_role;
          double disp;
          if ((rt == 1 && rj == 2) || (rt == 2 && rj == 1)) {
            const int acc = rt == 2 ? t : tj;
            const double R = s_par[acc].hb_R, e = s_par[acc].hb_eps, s = R / r;
            disp = 5.0 * e * ipow64(s, 12) - 6.0 * e * ipow64(s, 10);
            disp = (disp > kEmax ? kEmax : disp) * (double)kWHb;
          } else {
            const double R = 0.5 * ((double)s_par[t].Rii + (double)s_par[tj].Rii);
            const double e = sqrt((double)s_par[t].eps * (double)s_par[tj].eps), s = R / r;
            disp = e * ipow64(s, 12) - 2.0 * e * ipow64(s, 6);
            disp = (disp > kEmax ? kEmax : disp) * (double)kWVdw;
          }
          m[t] += disp + (double)kWSol * ((double)s_par[t].solpar * vj + sj * (double)s_par[t].vol) * g;
        }
      }
      const double diel = kDielA + kDielB / (1.0 + kDielK * exp(-kDielLambda * kDielB * r));
      E += (double)kWElec * kCoulomb * qj / (diel * r);
      D += (double)kWSol * kQasp * vj * g;
    }
  }
  if (!active) return;
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

cudaError_t launch_grid_build_impl(const float4 *prot, const uint8_t *ptype, int n_prot,
                                   const dock_type_params *params_dev, int n_types, int n,
                                   double ox, double oy, double oz, double h, float4 *maps,
                                   float2 *fpm, cudaStream_t s) {
  GridBuildArgs A;
  A.prot = prot;
  A.ptype = ptype;
  A.n_prot = n_prot;
  A.params = params_dev;
  A.n_types = n_types;
  A.n = n;
  A.ox = ox; A.oy = oy; A.oz = oz; A.h = h;
  A.maps = maps;
  A.fpm = fpm;
  const int64_t nn = (int64_t)n * n * n;
  const int threads = 256;
  grid_build_kernel<<<(unsigned)((nn + threads - 1) / threads), threads, 0, s>>>(A);
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
