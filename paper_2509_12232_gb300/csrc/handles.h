// Library-internal definitions of the opaque handles of include/dock.h and
// small host helpers shared by the C-ABI translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>

#include <vector>

#include "dock_internal.h"

struct dock_surrogate;
// Inference of the surrogate (surrogate.cu): out[i] = prediction of row i.
int dk_surrogate_predict_raw(dock_surrogate *S, const uint16_t *features, int64_t n, float *out,
                             int destandardize, cudaStream_t s);

namespace dk {
// Records the message returned by dock_last_error() for this thread; returns st.
int vset_error(int st, const char *fmt, va_list ap);
cudaError_t search_occupancy(int threads, int L, int atoms_per_lane, int *blocks_per_sm,
                             bool pairwise = false);
cudaError_t launch_set_deadline(uint64_t *deadline, uint64_t timeout_ns, cudaStream_t s);
}  // namespace dk

using namespace dk;

template <typename T>
inline cudaError_t dalloc(T **p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc((void **)p, count * sizeof(T));
}

template <typename T>
inline void dfree(T *&p) {
  if (p) cudaFree((void *)p);
  p = nullptr;
}

struct dock_pocket {
  int device = 0;
  int n_types = 0;
  std::vector<dock_type_params> params;
  dock_type_params *d_params = nullptr;
  int n_prot = 0;
  float4 *d_maps = nullptr;
  float *d_xycell = nullptr;  // (x, y)-cell records of the FP32 scorer
  float2 *d_fpm = nullptr;    // per node {E + D, E - D}
  int n = 0;
  double ox = 0, oy = 0, oz = 0, h = 0;
  float center[3] = {0, 0, 0};
  float radius = 0;
  // protein cell list and type tables of the pairwise scorer
  float4 *d_cprot = nullptr, *d_cext = nullptr, *d_tpair = nullptr;
  float2 *d_tsv = nullptr;
  int32_t *d_cell_start = nullptr;
  float cell_lo[3] = {0, 0, 0};
  int cell_dims[3] = {1, 1, 1};
  ~dock_pocket() {
    dfree(d_cprot);
    dfree(d_cext);
    dfree(d_tpair);
    dfree(d_tsv);
    dfree(d_cell_start);
    dfree(d_params);
    dfree(d_maps);
    dfree(d_xycell);
    dfree(d_fpm);
  }
};

inline GridView grid_view(const dock_pocket *p) {
  GridView g;
  g.maps = p->d_maps;
  g.xycell = p->d_xycell;
  g.n = p->n;
  g.ox = (float)p->ox;
  g.oy = (float)p->oy;
  g.oz = (float)p->oz;
  g.inv_h = (float)(1.0 / p->h);
  g.gx = (float)(-p->ox / p->h);
  g.gy = (float)(-p->oy / p->h);
  g.gz = (float)(-p->oz / p->h);
  g.plane_elems = 2 * (p->n - 1) * (p->n - 1);
  g.n_types = p->n_types;
  g.tex_elems = 4 * p->n_types * p->n * (p->n - 1) * (p->n - 1);
  return g;
}

inline CellGrid cell_grid(const dock_pocket *p) {
  CellGrid c;
  c.cell_start = p->d_cell_start;
  c.lox = p->cell_lo[0];
  c.loy = p->cell_lo[1];
  c.loz = p->cell_lo[2];
  c.dx = p->cell_dims[0];
  c.dy = p->cell_dims[1];
  c.dz = p->cell_dims[2];
  return c;
}

inline PwView pw_view(const dock_pocket *p) {
  PwView w;
  w.cprot = p->d_cprot;
  w.cext = p->d_cext;
  w.cells = cell_grid(p);
  w.tpair = p->d_tpair;
  w.tsv = p->d_tsv;
  w.n_types = p->n_types;
  w.n_atoms = p->n_prot;
  return w;
}

struct Workspace {
  size_t geno_cap = 0, score_cap = 0, best_cap = 0, item_cap = 0, gen_cap = 0, lig_cap = 0;
  float *geno[2] = {nullptr, nullptr};
  float *score[2] = {nullptr, nullptr};
  unsigned long long *best = nullptr;  // [generations][n_ligands]
  uint32_t *counters = nullptr;        // [generations]
  Item *items = nullptr;
  int64_t *geno_off = nullptr;
  int32_t *status = nullptr;           // [1] + deadline slot
  uint64_t *deadline = nullptr;
  int32_t *lig_status = nullptr;
  dock_result *results = nullptr;
  unsigned long long *ls_evals = nullptr;  // [n_ligands] local-search probes
  // Lamarckian search: selection bits [gens][n_ligands][pop/32], counts and
  // chain counters [gens][n_ligands], warp units (ligand per unit)
  size_t ls_bits_cap = 0, ls_count_cap = 0, ls_units_cap = 0;
  uint32_t *ls_bits = nullptr, *ls_count = nullptr, *ls_chain = nullptr;
  int32_t *ls_units = nullptr;
  // surrogate mode: candidates, their features and predictions, kept candidates
  size_t sur_cap = 0, kept_cap = 0;
  float *cand_geno = nullptr, *pred = nullptr, *kept_geno = nullptr, *kept_score = nullptr;
  uint16_t *feats = nullptr;
  int32_t *kept_lig = nullptr;
  size_t feat_off_cap = 0;
  int64_t *feat_off = nullptr;  // genotype offsets for dock_features_population
  // side streams and events: the per-lanes-per-pose launches of a generation
  // run concurrently, forked from the caller's stream and joined back
  cudaStream_t side[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t fork = nullptr, join[3] = {nullptr, nullptr, nullptr};
  // Host-to-device tables of dock_batch and the device-to-host reads of
  // dock_results go through `io`, a stream of their own: a copy from or to
  // pageable host memory on the caller's stream would wait for everything
  // queued there (the previous search, or a later one), stalling the host
  // while the GPU drains. up_* hold the bytes each table last received, so a
  // repeated search on the same set copies nothing.
  cudaStream_t io = nullptr;
  cudaEvent_t io_done = nullptr;
  std::vector<uint8_t> up_goff, up_items, up_units;
  // cached graph
  cudaGraphExec_t graph = nullptr;
  std::vector<uint8_t> graph_key;
  ~Workspace() {
    for (int i = 0; i < 2; ++i) {
      dfree(geno[i]);
      dfree(score[i]);
    }
    dfree(best);
    dfree(counters);
    dfree(items);
    dfree(geno_off);
    dfree(status);
    dfree(deadline);
    dfree(lig_status);
    dfree(results);
    dfree(ls_evals);
    dfree(ls_bits);
    dfree(ls_count);
    dfree(ls_chain);
    dfree(ls_units);
    dfree(cand_geno);
    dfree(pred);
    dfree(feats);
    dfree(kept_geno);
    dfree(kept_score);
    dfree(kept_lig);
    dfree(feat_off);
    if (graph) cudaGraphExecDestroy(graph);
    for (int i = 0; i < 3; ++i) {
      if (side[i]) cudaStreamDestroy(side[i]);
      if (join[i]) cudaEventDestroy(join[i]);
    }
    if (fork) cudaEventDestroy(fork);
    if (io) cudaStreamDestroy(io);
    if (io_done) cudaEventDestroy(io_done);
  }
};

struct dock_ligands {
  int device = 0;
  int n_ligands = 0;
  int max_atoms = 0;
  int tuned_threads = 0, tuned_apl = 0;  // launch shape chosen by dock_autotune (0: defaults)
  bool profiling = false;                 // time each generation's launch (autotuner)
  std::vector<LigInfo> info;
  LigInfo *d_info = nullptr;
  float4 *d_atoms = nullptr;      // centred
  float4 *d_atoms_raw = nullptr;  // input coordinates
  double *d_centroid = nullptr;
  uint8_t *d_types = nullptr;
  uint32_t *d_pair_idx = nullptr;
  float *d_pair_rec = nullptr;
  TorInfo *d_tors = nullptr;
  uint8_t *d_moves = nullptr;
  int32_t *d_check = nullptr;  // index-check word of calls without a status word (checked build)
  int64_t total_pair_slots = 0;  // pair_idx / pair_rec entries (all included pairs)
  int64_t total_pairs = 0, total_atoms = 0, total_tors = 0, total_moved = 0, h2d_bytes = 0;
  Workspace ws;
  ~dock_ligands() {
    dfree(d_info);
    dfree(d_atoms);
    dfree(d_atoms_raw);
    dfree(d_centroid);
    dfree(d_types);
    dfree(d_pair_idx);
    dfree(d_pair_rec);
    dfree(d_tors);
    dfree(d_moves);
    dfree(d_check);
  }
};

// Array sizes of a (pocket, ligand set) for the bounds-checked build; word is
// the status word the call's kernels record a failed check in.
inline Bounds bounds_of(const dock_pocket *p, const dock_ligands *l, int32_t *word) {
  Bounds b;
  b.word = word;
  b.atoms = l->total_atoms;
  b.pairs = l->total_pair_slots;
  b.tors = l->total_tors;
  b.moves = l->total_moved;
  b.ligands = l->n_ligands;
  b.tex_elems = 4 * p->n_types * p->n * (p->n - 1) * (p->n - 1);
  b.prot_atoms = p->n_prot;
  b.slot_rows = 0;
  return b;
}

inline uint64_t prob_threshold(float p) {
  double t = (double)p * 4294967296.0;
  if (!(t > 0)) t = 0;
  if (t > 4294967296.0) t = 4294967296.0;
  return (uint64_t)t;
}

// Lanes per pose of an n-atom ligand: the smallest L in {1, 2, 4, 8} with
// L * atoms_per_lane >= n (or the forced value).
inline int lanes_for(int n, int apl, int forced) {
  if (forced) return forced;
  int L = 1;
  while (L * apl < n && L < 8) L <<= 1;
  return L;
}
