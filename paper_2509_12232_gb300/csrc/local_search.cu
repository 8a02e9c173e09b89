// Solis-Wets local search: the Lamarckian variant of AutoDock's GA (Morris et
// al. 1998; the random search with bias of Solis & Wets 1981). The paper's own
// search has none (Section V); this refines chosen individuals with the same
// pose (Algorithm 1) and score (Algorithm 2) as the search kernel.
//
// One chain (one individual) per group of L lanes, chains pulled from a queue
// so that chains of very different lengths balance across the GPU. The
// chain's genotype x, bias b, displacement xi and probe y live in shared
// memory next to the pose's coordinate slot; lane l owns genes l, l + L, ...
// (their normals, bias and probe arithmetic), and every lane reads the whole
// probe to pose and score it. All genotype arithmetic is correctly rounded
// FP32, so a chain is bit-exact with the CPU oracle given the same scores.
#include <algorithm>

#include "pose.cuh"

namespace dk {

namespace {

constexpr uint32_t kLsGenBit = 0x80000000u;  // generation word of the local search's counters
constexpr int kGeneStride = 24;              // floats per gene vector in shared memory

__device__ __forceinline__ float ls_sigma(int e) { return e < 3 ? 1.0f : (e < 7 ? 0.1f : 0.5f); }

// N(0, 1) draw of gene e at iteration t: Irwin-Hall sum of the twelve 16-bit
// halves of words 0-5 of one Philox block (slot 64 t + e), exact in float.
__device__ __forceinline__ float ls_normal(uint64_t seed, uint64_t lig_id, uint32_t gen,
                                           uint32_t ind, uint32_t t, int e) {
  const Words8 w = rng_words<true>(seed, lig_id, gen, ind, 64u * t + (uint32_t)e);
  int32_t S = 0;
#pragma unroll
  for (int k = 0; k < 6; ++k) S += (int32_t)(w.w[k] & 0xffffu) + (int32_t)(w.w[k] >> 16);
  return __fmul_rn((float)(S - 6 * 65536), 0x1p-16f);
}

__device__ __forceinline__ float nan_to_inf(float v) {
  return v != v ? __int_as_float(0x7f800000) : v;
}

// the mutation's torsion wrap (one turn at most)
__device__ __forceinline__ float wrap_gene(float v, int e) {
  if (e >= 7) {
    if (v > kPiF) v = __fsub_rn(v, kTwoPiF);
    else if (v < -kPiF) v = __fadd_rn(v, kTwoPiF);
  }
  return v;
}

// Poses and scores the probe Y (its quaternion renormalised first and
// written back, so that an accepted probe is stored as scored).
template <int L>
__device__ __forceinline__ float ls_probe(float *Y, int G, const LigView &V, const LsArgs &A,
                                          float4 *sl, int lane, unsigned gmask) {
  float g[DOCK_MAX_GENES];
#pragma unroll
  for (int e = 0; e < DOCK_MAX_GENES; ++e) g[e] = e < G ? Y[e] : 0.0f;
  quat_normalize(g[3], g[4], g[5], g[6]);
  __syncwarp(gmask);
  if (lane == 0) {
    Y[3] = g[3];
    Y[4] = g[4];
    Y[5] = g[5];
    Y[6] = g[6];
  }
  return pose_and_score<L>(g, V, A.moves, A.grid, A.cx, A.cy, A.cz, sl, lane, gmask, nullptr);
}

// State of one chain, held identically by the lanes of its group.
struct Chain {
  int phase;      // 0: score the start, 1: probe x + xi, 2: probe x - xi
  int t, succ, fail, ev;
  float f, f0, f1, rho;
};

// One loop turn of a chain: build and score one probe, then (after the
// forward probe succeeded, or after the backward probe) the iteration's
// outcome: bias update, acceptance, rho schedule.
template <int L>
__device__ __forceinline__ void ls_turn(const LsArgs &A, const LigView &V, int G, uint64_t lig_id,
                                        uint32_t ind, Chain &c, float *X, float *B, float *XI,
                                        float *Y, float4 *sl, int lane, unsigned gmask,
                                        float *trace) {
  if (c.phase == 1) {
    const uint32_t gen = A.gen | kLsGenBit;
    for (int e = lane; e < G; e += L) {
      const float z = ls_normal(A.seed, lig_id, gen, ind, (uint32_t)c.t, e);
      const float xi = __fadd_rn(B[e], __fmul_rn(__fmul_rn(c.rho, ls_sigma(e)), z));
      XI[e] = xi;
      Y[e] = wrap_gene(__fadd_rn(X[e], xi), e);
    }
  } else if (c.phase == 2) {
    for (int e = lane; e < G; e += L) Y[e] = wrap_gene(__fsub_rn(X[e], XI[e]), e);
  }
  __syncwarp(gmask);
  const float v = ls_probe<L>(Y, G, V, A, sl, lane, gmask);
  if (c.phase == 0) {
    c.f0 = v;
    c.f = nan_to_inf(v);
    c.phase = 1;
    return;
  }
  ++c.ev;
  if (c.phase == 1) {
    c.f1 = v;
    if (!(v < c.f)) {
      c.phase = 2;
      return;
    }
  }
  const bool ok = v < c.f, fwd = c.phase == 1;
  if (ok) c.f = v;
  for (int e = lane; e < G; e += L) {
    if (ok) X[e] = Y[e];
    const float b = B[e], xi = XI[e];
    B[e] = fwd ? __fadd_rn(__fmul_rn(0.2f, b), __fmul_rn(0.4f, xi))
               : (ok ? __fsub_rn(b, __fmul_rn(0.4f, xi)) : __fmul_rn(0.5f, b));
  }
  __syncwarp(gmask);
  if (trace != nullptr && lane == 0) {
    trace[2 + 2 * c.t] = c.f1;
    trace[3 + 2 * c.t] = fwd ? __int_as_float(0x7fc00000) : v;
  }
  if (ok) {
    ++c.succ;
    c.fail = 0;
  } else {
    ++c.fail;
    c.succ = 0;
  }
  if (c.succ >= A.max_succ) {
    c.rho = __fmul_rn(2.0f, c.rho);
    c.succ = 0;
  } else if (c.fail >= A.max_fail) {
    c.rho = __fmul_rn(0.5f, c.rho);
    c.fail = 0;
  }
  ++c.t;
  c.phase = 1;
}

// Index of the r-th set bit of bits[0..words).
__device__ __forceinline__ int nth_set_bit(const uint32_t *bits, int words, uint32_t r) {
  for (int w = 0; w < words; ++w) {
    uint32_t b = bits[w];
    const uint32_t n = (uint32_t)__popc(b);
    if (r < n) {
      for (uint32_t k = 0; k < r; ++k) b &= b - 1u;
      return w * 32 + __ffs(b) - 1;
    }
    r -= n;
  }
  return -1;
}

// Chains run by lane groups; a group whose chain ends takes the next one
// (batch: the next selected individual of the warp's ligand; standalone: the
// group's next pose), so the groups of a warp keep scoring probes of the same
// ligand side by side. Every turn scores at most one probe per group through
// one call site.
template <int L>
__global__ void __launch_bounds__(128, 4) ls_kernel(const LsArgs A) {
  extern __shared__ float4 smem4[];
  const int lane = threadIdx.x & (L - 1), slot = threadIdx.x / L, S = blockDim.x / L;
  const unsigned gmask = group_mask<L>();
  const int ss = slot_stride(L, A.atoms_per_lane);
  float4 *sl = smem4 + slot * ss;
  float *X = reinterpret_cast<float *>(smem4 + S * ss) + slot * 4 * kGeneStride;
  float *B = X + kGeneStride, *XI = B + kGeneStride, *Y = XI + kGeneStride;
  const int trace_w = 2 + 2 * A.max_its;
  const bool batch = A.units != nullptr;
  // standalone: this group's poses p0, p0 + stride, ...
  int64_t next_p = (int64_t)blockIdx.x * S + slot;
  const int64_t stride = (int64_t)gridDim.x * S;
  // the current ligand (per warp in batch mode, per group standalone)
  int lig = 0, G = 7;
  LigView V{};
  uint64_t lig_id = 0;
  const uint32_t *bits = nullptr;
  uint32_t count = 0;
  // the current chain
  Chain c{};
  int64_t ind = 0;
  float *gp = nullptr, *tr = nullptr;
  bool active = false, exhausted = batch;  // batch: no unit yet
  for (;;) {
    // (every lane of the warp reaches this point each turn: the vote is uniform)
    if (batch && __all_sync(0xffffffffu, exhausted)) {
      // ---- the warp takes its next unit (a ligand) -------------------------
      int u = 0;
      if ((threadIdx.x & 31) == 0) {
        u = (int)atomicAdd(A.counter, 1u);
        if (A.deadline != nullptr && u < A.n_units && globaltimer_ns() > *A.deadline) {
          atomicExch(A.status, (int)DOCK_ETIMEOUT);
          u = A.n_units;
        }
#ifdef DOCK_CHECKED
        if (u < A.n_units && *(volatile int32_t *)A.status != 0) u = A.n_units;  // a check failed
#endif
      }
      u = __shfl_sync(0xffffffffu, u, 0);
      if (u >= A.n_units) break;
      lig = A.units[u];
      if (!DK_OK(lig >= 0 && lig < A.bounds.ligands, A.status, 13)) lig = 0;
      const LigInfo li = A.ligs[lig];
      G = 7 + li.k;
      V = lig_view(li, A.atoms, A.types, A.pair_rec, A.tors, DK_BOUNDS(A), ss);
      lig_id = li.ligand_id;
      bits = A.sel_bits + (int64_t)lig * A.sel_words;
      count = A.sel_count[lig];
      exhausted = false;
    }
    // ---- finish a chain that is over; take the next one -------------------
    for (;;) {
      if (active && c.phase == 1 && (c.t >= A.max_its || c.rho < A.rho_lb)) {
        for (int e = lane; e < G; e += L) gp[e] = X[e];
        if (lane == 0) {
          if (batch) {
            A.score[(int64_t)lig * A.pop + ind] = c.f;
            const unsigned long long key =
                ((unsigned long long)score_key(c.f) << 32) | (unsigned long long)(uint32_t)ind;
            atomicMin(&A.best[lig], key);
            atomicAdd(&A.evals[lig], (unsigned long long)c.ev);
          } else {
            A.scores[ind] = c.f;
            if (A.pose_evals) A.pose_evals[ind] = (uint32_t)c.ev;
          }
          if (tr != nullptr) {
            tr[0] = c.f0;
            tr[1] = (float)c.t;
          }
        }
        __syncwarp(gmask);
        active = false;
      }
      if (active || exhausted) break;
      if (batch) {
        uint32_t r = 0;
        if (lane == 0) r = atomicAdd(A.chain_ctr + lig, 1u);
        r = __shfl_sync(gmask, r, 0, L);
        if (r >= count) {
          exhausted = true;
          break;
        }
        ind = nth_set_bit(bits, A.sel_words, r);
        if (!DK_OK(ind >= 0 && ind < A.pop, A.status, 14)) ind = 0;
        gp = A.geno + A.geno_off[lig] + ind * G;
        c.f0 = A.score[(int64_t)lig * A.pop + ind];
        c.f = nan_to_inf(c.f0);
        c.phase = 1;
        tr = A.trace ? A.trace + ((int64_t)lig * A.pop + ind) * trace_w : nullptr;
      } else {
        ind = next_p;
        next_p += stride;
        if (ind >= A.n_poses) {
          exhausted = true;
          break;
        }
        lig = A.pose_ligand[ind];
        if (lig < 0 || lig >= A.n_ligands) {
          if (lane == 0) A.scores[ind] = __int_as_float(0x7fc00000);
          continue;
        }
        const LigInfo li = A.ligs[lig];
        G = 7 + li.k;
        V = lig_view(li, A.atoms, A.types, A.pair_rec, A.tors, DK_BOUNDS(A), ss);
        lig_id = li.ligand_id;
        gp = A.genos + ind * DOCK_MAX_GENES;
        c.phase = 0;
        tr = A.trace ? A.trace + ind * trace_w : nullptr;
      }
      c.t = c.succ = c.fail = c.ev = 0;
      c.rho = A.rho;
      for (int e = lane; e < G; e += L) {
        X[e] = gp[e];
        Y[e] = gp[e];
        B[e] = 0.0f;
      }
      __syncwarp(gmask);
      active = true;
    }
    if (!batch && !__any_sync(0xffffffffu, active)) break;
    if (active)
      ls_turn<L>(A, V, G, lig_id, (uint32_t)ind, c, X, B, XI, Y, sl, lane, gmask, tr);
  }
}

// Selection bits of all generations: warp w covers individuals 32 j .. 32 j + 31
// of ligand l in generation g, w = (g n_ligands + l) words + j.
__global__ void ls_select_kernel(const LigInfo *ligs, int n_ligands, int pop, int words, int gens,
                                 uint64_t seed, uint64_t thr, uint32_t *bits, uint32_t *count) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_words = (int64_t)gens * n_ligands * words;
  if (w >= n_words) return;  // whole warps (blockDim is a multiple of 32)
  const int j = (int)(w % words);
  const int64_t gl = w / words;
  const int l = (int)(gl % n_ligands), g = (int)(gl / n_ligands);
  const int ind = j * 32 + (threadIdx.x & 31);
  bool sel = false;
  if (ind < pop) {
    const Words8 r = rng_words(seed, ligs[l].ligand_id, (uint32_t)g | kLsGenBit, (uint32_t)ind, 63);
    sel = (uint64_t)r.w[0] < thr;
  }
  const unsigned m = __ballot_sync(0xffffffffu, sel);
  if ((threadIdx.x & 31) == 0) {
    bits[w] = m;
    if (m) atomicAdd(count + gl, (uint32_t)__popc(m));
  }
}

template <int L>
cudaError_t ls_occupancy_l(int threads, int smem, int *blocks_per_sm) {
  cudaError_t e =
      cudaFuncSetAttribute(ls_kernel<L>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, ls_kernel<L>, threads, smem);
}

}  // namespace

int ls_smem_bytes(int threads, int L, int atoms_per_lane) {
  return slots_bytes(threads, L, atoms_per_lane) + (threads / L) * 4 * kGeneStride * 4;
}

cudaError_t ls_occupancy(int threads, int L, int atoms_per_lane, int *blocks_per_sm) {
  const int smem = ls_smem_bytes(threads, L, atoms_per_lane);
  switch (L) {
    case 1: return ls_occupancy_l<1>(threads, smem, blocks_per_sm);
    case 2: return ls_occupancy_l<2>(threads, smem, blocks_per_sm);
    case 4: return ls_occupancy_l<4>(threads, smem, blocks_per_sm);
    case 8: return ls_occupancy_l<8>(threads, smem, blocks_per_sm);
    case 16: return ls_occupancy_l<16>(threads, smem, blocks_per_sm);
    case 32: return ls_occupancy_l<32>(threads, smem, blocks_per_sm);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_ls_select(const LigInfo *ligs, int n_ligands, int pop, int gens, uint64_t seed,
                             uint64_t thr_ls, uint32_t *sel_bits, uint32_t *sel_count,
                             cudaStream_t s) {
  const int words = (pop + 31) / 32;
  const int64_t n_words = (int64_t)gens * n_ligands * words;
  cudaError_t e = cudaMemsetAsync(sel_count, 0, sizeof(uint32_t) * (size_t)gens * n_ligands, s);
  if (e != cudaSuccess || n_words == 0) return e;
  const int64_t blocks = (n_words * 32 + 255) / 256;
  ls_select_kernel<<<(unsigned)blocks, 256, 0, s>>>(ligs, n_ligands, pop, words, gens, seed, thr_ls,
                                                     sel_bits, sel_count);
  return cudaGetLastError();
}

cudaError_t launch_ls(const LsArgs &a, int blocks, int threads, int L, cudaStream_t s) {
  const int smem = ls_smem_bytes(threads, L, a.atoms_per_lane);
  switch (L) {
    case 1: ls_kernel<1><<<blocks, threads, smem, s>>>(a); break;
    case 2: ls_kernel<2><<<blocks, threads, smem, s>>>(a); break;
    case 4: ls_kernel<4><<<blocks, threads, smem, s>>>(a); break;
    case 8: ls_kernel<8><<<blocks, threads, smem, s>>>(a); break;
    case 16: ls_kernel<16><<<blocks, threads, smem, s>>>(a); break;
    case 32: ls_kernel<32><<<blocks, threads, smem, s>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace dk
