// Internal types shared by the library's translation units (host + device).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dock.h"

namespace dk {

// Per-ligand record, pop-independent (built by dock_load_ligands).
// Included intra pairs come in two runs: the n_pairs pairs whose distance the
// torsions change (pair_rec and pair_idx), then n_pairs_all - n_pairs pairs
// whose distance no pose changes (pair_idx only: every torsion that separates
// the two atoms has one of them on its axis). Their energy is one constant per
// ligand, intra_const, summed in FP64 on the device by dock_load_ligands.
struct LigInfo {
  int32_t atom_off;   // first atom in the atom arrays
  int32_t n;          // atoms
  int32_t k;          // torsions
  int32_t pair_off;   // first included intra pair
  int32_t n_pairs;    // pairs evaluated per pose
  int32_t tors_off;   // first torsion record
  int32_t n_pairs_all;  // all included pairs (FP64 path)
  float intra_const;    // energy of the pose-invariant pairs
  uint64_t ligand_id;
};

// Sizes of the arrays the hot kernels index, and the device word in which a
// bounds-checked build (compiled with DOCK_CHECKED) records its first failed
// index check as kCheckBase - site (the host then reports DOCK_EDEVICE). The
// normal build carries the struct but tests nothing.
constexpr int32_t kCheckBase = -1000;
struct Bounds {
  int32_t *word;           // status word of the call (NULL: checks not recorded)
  int64_t atoms, pairs;    // atom rows, FP32 pair records of the ligand set
  int64_t tors, moves;     // torsion records, moved-atom entries
  int32_t ligands;
  int32_t tex_elems;       // 16-byte elements of the map records
  int32_t prot_atoms;      // protein atoms of the cell list
  int32_t slot_rows;       // float4 rows of one pose's shared-memory slot
};

// One rotatable bond: rotate atoms moves[move_off .. move_off + n_move) about
// the axis parent(b) = a -> b.
struct TorInfo {
  int32_t move_off;
  int16_t n_move;
  uint8_t a, b;
};

// A work item of the search kernel: poses [first, first + count) of ligand lig,
// run with `lanes` lanes per pose.
struct Item {
  int32_t lig;
  int16_t first_div;  // first pose / slots (tile index)
  int8_t lanes;       // lanes per pose: 1, 2, 4, 8
  int8_t pad;
};

// pair_idx (u32, FP64 path): bits 0-7 atom i, 8-15 atom j, 16 H-bond flag.
// pair_rec (FP32 path): 4 floats per pair, 16-byte aligned:
// {bits(16 i | 16 j << 16), c12, cb, ds} (atoms' byte offsets in a pose's
// coordinate slot; weights folded in; cb = c6 for a 12-6 pair and -c10 for a
// 12-10 H-bond pair) for
// E = min(c12 r^-12 - c6 r^-6 - c10 r^-10, w EMAX) + qq / (eps(r) r) + ds exp(-r^2 / 2 sigma^2);
// qq comes from the scaled charges the pose slots carry.

struct GridView {
  const float4 *maps;   // [n_types][n][n][n] {M_t, E, D, 0}
  const float *xycell;  // [n_types][2][n][n-1][n-1] (x, y)-cell records, 8 floats, 32-byte
                        // aligned: {M, F} at (x,y), (x+1,y), (x,y+1), (x+1,y+1) with
                        // F = E + D (sign 0, for q >= 0) or E - D (sign 1, q < 0), so
                        // M + q E + |q| D = M + q F
  int32_t n;            // nodes per axis
  float ox, oy, oz;     // origin
  float inv_h;
  float gx, gy, gz;     // -origin / h: grid coordinate u = x inv_h + g
  int32_t plane_elems;  // 16-byte elements of one z plane of records, 2 (n-1)^2
  int32_t n_types;
  int32_t tex_elems;    // 16-byte elements of all records, 2 n_types 2 n (n-1)^2
};

// Protein atoms by cell: cells are kCellX wide in x and kCellYZ in y and z
// (x fastest); the atoms of cell c are [cell_start[c], cell_start[c + 1]).
// A row (cy, cz) is dx consecutive cells, so any x interval of a row is one
// contiguous atom range; the fine x cells let a lookup keep only the cells
// that meet the chord of the cutoff sphere.
constexpr float kCellX = 1.0f, kCellYZ = 8.0f;
struct CellGrid {
  const int32_t *cell_start;
  float lox, loy, loz;  // corner of cell (0, 0, 0)
  int32_t dx, dy, dz;
};

// The protein for the pairwise inter-energy: atoms sorted by cell, cprot {x,
// y, z, q}, cext {S_j = solpar + 0.01097 |q|, V_j, type, 0}.
struct PwView {
  const float4 *cprot, *cext;
  CellGrid cells;
  const float4 *tpair;      // [T][T] {c12, c6, c10, cap} weights folded in
  const float2 *tsv;        // [T] {solpar, vol}
  int32_t n_types;
  int32_t n_atoms;          // protein atoms in cprot / cext
};

struct SearchArgs {
  // ligands
  const LigInfo *ligs;
  const float4 *atoms;      // {x, y, z, q}, centred on the ligand centroid
  const uint8_t *types;
  const float *pair_rec;
  const TorInfo *tors;
  const uint8_t *moves;
  const int64_t *geno_off;  // [n_ligands]
  // work queue
  const Item *items;
  int32_t n_items;
  uint32_t *counter;        // this generation's queue counter (starts at 0)
  int32_t atoms_per_lane;   // smem capacity: lanes * atoms_per_lane >= n
  // pocket
  GridView grid;
  float cx, cy, cz;         // pocket centre
  float radius;
  // GA
  int32_t pop;
  int32_t gen;
  uint64_t seed;
  uint64_t thr_cross, thr_mut;
  const float *geno_prev;
  float *geno_next;
  const float *score_prev;
  float *score_next;
  const unsigned long long *best_prev;  // [n_ligands] best key of gen-1
  unsigned long long *best_next;        // [n_ligands] best key of gen (init ~0)
  // control
  int32_t *status;          // device status word
  int32_t *lig_status;      // [n_ligands]
  const uint64_t *deadline;  // device globaltimer deadline, NULL = none
  PwView pw;                // the protein of the pairwise inter-energy (no-grid search)
  Bounds bounds;
};

// Solis-Wets refinement (local_search.cu). Batch mode (units != nullptr):
// after a generation's search launch; the individuals drawn for refinement
// are the set bits of sel_bits (one bit mask of pop bits per ligand, built
// for every generation by launch_ls_select), their number sel_count. A unit
// is a ligand: the warp that takes it runs that ligand's chains, its lane
// groups pulling them one by one from the ligand's chain counter (several
// units per ligand share it). Standalone mode: pose p of genos / scores,
// ligand pose_ligand[p], scored first.
struct LsArgs {
  const LigInfo *ligs;
  const float4 *atoms;
  const uint8_t *types;
  const float *pair_rec;
  const TorInfo *tors;
  const uint8_t *moves;
  GridView grid;
  float cx, cy, cz;
  int32_t atoms_per_lane;
  int32_t max_its, max_succ, max_fail;
  float rho, rho_lb;
  uint64_t seed;
  uint32_t gen;
  // batch mode
  const int32_t *units;           // ligand of each warp unit
  int32_t n_units;
  uint32_t *counter;              // unit queue counter (starts at 0)
  const uint32_t *sel_bits;       // [n_ligands][pop / 32 rounded up] of this generation
  const uint32_t *sel_count;      // [n_ligands]
  uint32_t *chain_ctr;            // [n_ligands] chains taken (starts at 0)
  int32_t sel_words;
  const int64_t *geno_off;
  float *geno;                    // the generation's population (CSR)
  float *score;                   // [n_ligands][pop]
  int32_t pop;
  unsigned long long *best;       // [n_ligands] best key of the generation
  unsigned long long *evals;      // [n_ligands] probes scored
  int32_t *status;
  const uint64_t *deadline;
  // standalone mode
  const int32_t *pose_ligand;
  int32_t n_ligands;
  int64_t n_poses;
  float *genos;                   // [n_poses][DOCK_MAX_GENES]
  float *scores;
  uint32_t *pose_evals;           // optional [n_poses]
  // optional trace rows of 2 + 2 max_its floats: batch [n_ligands * pop],
  // standalone [n_poses]
  float *trace;
  Bounds bounds;
};
// Selection bits and counts of generations [0, gens) (counts zeroed first):
// bit i of ligand l, generation g is set when individual i is refined.
cudaError_t launch_ls_select(const LigInfo *ligs, int n_ligands, int pop, int gens, uint64_t seed,
                             uint64_t thr_ls, uint32_t *sel_bits, uint32_t *sel_count,
                             cudaStream_t s);
cudaError_t ls_occupancy(int threads, int L, int atoms_per_lane, int *blocks_per_sm);
int ls_smem_bytes(int threads, int L, int atoms_per_lane);
cudaError_t launch_ls(const LsArgs &a, int blocks, int threads, int L, cudaStream_t s);

struct ScoreArgs {
  const LigInfo *ligs;
  const float4 *atoms;
  const uint8_t *types;
  const float *pair_rec;
  const TorInfo *tors;
  const uint8_t *moves;
  GridView grid;
  float cx, cy, cz;
  const int32_t *pose_ligand;
  int32_t n_ligands;        // pose_ligand entries outside [0, n_ligands) score NaN
  const float *genos;       // [n_poses][DOCK_MAX_GENES]
  int64_t n_poses;
  float *scores;
  float *coords;            // optional
  int32_t lanes;            // lanes per pose
  int32_t atoms_per_lane;
  Bounds bounds;
};

// Pairwise scoring of caller-given poses (pairwise.cu): the ScoreArgs inputs
// plus the protein cell list and the type tables.
struct PairwiseArgs {
  const LigInfo *ligs;
  const float4 *atoms;
  const uint8_t *types;
  const float *pair_rec;
  const TorInfo *tors;
  const uint8_t *moves;
  float cx, cy, cz;
  const int32_t *pose_ligand;
  int32_t n_ligands;        // pose_ligand entries outside [0, n_ligands) score NaN
  const float *genos;       // [n_poses][DOCK_MAX_GENES]
  int64_t n_poses;
  float *scores;
  PwView pw;
  Bounds bounds;
};
cudaError_t launch_score_pairwise(const PairwiseArgs &a, cudaStream_t s);

// FP64 rescoring / scoring inputs (type table in FP32 as given).
struct Fp64Args {
  const LigInfo *ligs;
  const float4 *atoms;             // raw input coordinates + charge
  const uint8_t *types;
  const uint32_t *pair_idx;
  const TorInfo *tors;
  const uint8_t *moves;
  GridView grid;
  double h;                        // grid spacing (exact)
  double cx, cy, cz;
  const dock_type_params *params;  // device [n_types]
  int32_t pairwise;                // 1: inter-energy by the pairwise sum over pw
  PwView pw;
};

// Launchers (defined in the .cu files).
// Grid maps from the protein cell list (grid.cu).
struct GridBuildArgs {
  const float4 *cprot, *cext;  // cell-sorted protein atoms, as in PwView
  CellGrid cells;
  const double4 *coef;         // [T][T] {c12, c6, c10, w EMAX}, weights folded in
  const double2 *tsv;          // [T] {solpar, vol}
  int32_t n_types, n;
  double ox, oy, oz, h;
  float4 *maps;
  float2 *fpm;                 // per node {E + D, E - D}, rounded once from FP64
};
cudaError_t launch_grid_build_impl(const GridBuildArgs &A, cudaStream_t s);
// Energy of each ligand's pose-invariant pairs (FP64 sum, stored rounded to
// FP32 in ligs[l].intra_const); one warp per ligand.
cudaError_t launch_intra_const(LigInfo *ligs, int n_ligands, const float4 *atoms_raw,
                               const uint8_t *types, const uint32_t *pair_idx,
                               const dock_type_params *params, cudaStream_t s);

// One launch of the search kernel instantiated for L lanes per pose; every
// item of a.items has a.items[i].lanes == L.
cudaError_t launch_search(const SearchArgs &a, int blocks, int threads, int L, cudaStream_t s,
                          bool pairwise = false);
cudaError_t launch_score(const ScoreArgs &a, cudaStream_t s);
// Best key ((score key << 32) | index, the search kernel's atomicMin key) of
// each ligand's population scores [n_ligands][pop]: a resumed search's
// elitism reads it for the saved generation.
cudaError_t launch_best_keys(const float *scores, int n_ligands, int pop,
                             unsigned long long *best, cudaStream_t s);
cudaError_t launch_finalize_impl(const Fp64Args &f, const double *centroids, int n_ligands, int pop,
                                 const int64_t *geno_off, const float *genos, const float *scores,
                                 const int32_t *lig_status, const int32_t *status,
                                 uint64_t exact_evals, uint64_t surrogate_evals,
                                 const unsigned long long *extra_evals, double ox, double oy,
                                 double oz, dock_result *out, cudaStream_t s);
cudaError_t launch_score_fp64_impl(const Fp64Args &f, const double *centroids, double ox, double oy,
                                   double oz, const int32_t *pose_ligand, int n_ligands,
                                   const float *genos, int64_t n_poses, double *out, cudaStream_t s);
int search_smem_bytes(int threads, int atoms_per_lane);
cudaError_t launch_xycell_maps(const float4 *maps, const float2 *fpm, int n_types, int n,
                               float *xycell, cudaStream_t s);

}  // namespace dk
