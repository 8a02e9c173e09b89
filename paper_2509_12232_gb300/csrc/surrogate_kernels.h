// Launchers of the surrogate pre-screen kernels (features.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dock_internal.h"

namespace dk {

struct FeatureLaunch {
  const LigInfo *ligs;
  const float4 *atoms;
  const uint8_t *types;
  const float *pair_rec;
  const TorInfo *tors;
  const uint8_t *moves;
  GridView grid;
  float cx, cy, cz, radius;
  int32_t n_ligands;
  bool from_ga;
  // given genotypes (from_ga = false): rows [n][DOCK_MAX_GENES] with pose_ligand,
  // or, when pop_csr > 0, whole populations in the search's CSR layout
  // (row r = ligand r / pop_csr, individual r % pop_csr, via geno_off)
  int32_t pop_csr;
  const int32_t *pose_ligand;
  const float *genos;
  int64_t n_poses;
  float *scores;
  // GA candidates (from_ga = true)
  int32_t pop, candidates, gen;
  uint64_t seed, thr_cross, thr_mut;
  const float *geno_prev;
  const float *score_prev;
  const int64_t *geno_off;
  float *cand_geno;
  uint16_t *features;
};

cudaError_t launch_features(const FeatureLaunch &F, cudaStream_t s);
cudaError_t launch_topk(const float *pred, int n_ligands, int candidates, int keep,
                        const float *cand_geno, float *kept_geno, int32_t *kept_lig, cudaStream_t s);
cudaError_t launch_merge(const float *geno_prev, const float *score_prev, const int64_t *geno_off,
                         const LigInfo *ligs, int n_ligands, int pop, const float *kept_geno,
                         const float *kept_score, int keep, float *geno_next, float *score_next,
                         cudaStream_t s);

}  // namespace dk
