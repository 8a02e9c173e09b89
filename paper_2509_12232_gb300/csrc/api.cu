// C ABI of the docking library: pocket and ligand set preparation, the
// batched search (one persistent kernel per generation, optionally captured
// as a CUDA graph), results and pose scoring. See include/dock.h.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>
#include <thread>
#include <vector>

#include "dock_internal.h"
#include "surrogate_kernels.h"
#include "handles.h"
#include "nvtx_range.h"


using namespace dk;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
// Message of the last failed call on this thread (fixed storage: recording an
// error allocates nothing).
static thread_local char g_err[512];

int dk::vset_error(int st, const char *fmt, va_list ap) {
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  return st;
}

static int fail(int st, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vset_error(st, fmt, ap);
  va_end(ap);
  return st;
}

// Solis-Wets settings other than the rate (dock_ls_params).
static int check_ls_params(const dock_ls_params *ls, const char *who) {
  if (ls->max_its < 1 || ls->max_its > DOCK_LS_MAX_ITS || ls->max_succ < 1 || ls->max_fail < 1 ||
      !(ls->rho > 0.0f) || !std::isfinite(ls->rho) || !std::isfinite(ls->rho_lb))
    return fail(DOCK_EINVAL, "%s: local search needs 1 <= max_its <= %d, max_succ, max_fail >= 1, "
                             "finite rho > 0 and finite rho_lb", who, DOCK_LS_MAX_ITS);
  return DOCK_OK;
}

#define CU(call)                                                                     \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      int st_ = e_ == cudaErrorMemoryAllocation ? DOCK_ENOMEM : DOCK_ECUDA;          \
      return fail(st_, "%s failed: %s", #call, cudaGetErrorString(e_));              \
    }                                                                                \
  } while (0)

extern "C" const char *dock_last_error(void) { return g_err; }

extern "C" const char *dock_version(void) {
  return "gb300-dock 0.1 (sm_103a, Philox4x64-10 GA, FP32 Kahan scoring, FP64 rescoring)";
}


// AutoDock4 free-energy constants for the host-side pair coefficients.
static const double kHWVdw = 0.1662, kHWHb = 0.1209, kHWElec = 0.1406, kHWSol = 0.1322;
static const double kHCoulomb = 332.06363, kHQasp = 0.01097, kHEmax = 1.0e5;

// Dispersion coefficients of a type pair with the weight folded in: a
// donor-acceptor pair takes the 12-10 H-bond form with R and eps of the
// acceptor (c6 = 0), any other the 12-6 form with the combined R and eps
// (c10 = 0); w is the term's weight (the raw value is capped at EMAX before it).
static void pair_coeffs(const dock_type_params *tp, int ti, int tj, double &c12, double &c6,
                        double &c10, double &w) {
  const bool hb = (tp[ti].hb_role == 1 && tp[tj].hb_role == 2) ||
                  (tp[ti].hb_role == 2 && tp[tj].hb_role == 1);
  c6 = c10 = 0.0;
  if (hb) {
    const int acc = tp[ti].hb_role == 2 ? ti : tj;
    const double R = tp[acc].hb_R, e = tp[acc].hb_eps;
    w = kHWHb;
    c12 = w * 5.0 * e * std::pow(R, 12);
    c10 = w * 6.0 * e * std::pow(R, 10);
  } else {
    const double R = 0.5 * ((double)tp[ti].Rii + (double)tp[tj].Rii);
    const double e = std::sqrt((double)tp[ti].eps * (double)tp[tj].eps);
    w = kHWVdw;
    c12 = w * e * std::pow(R, 12);
    c6 = w * 2.0 * e * std::pow(R, 6);
  }
}

// ---------------------------------------------------------------------------
// pocket
// ---------------------------------------------------------------------------


extern "C" int dock_create_pocket(const dock_pocket_desc *d, void *stream, dock_pocket **out) {
  const dk::NvtxRange nvtx_range("dock_create_pocket");
  if (!d || !out) return fail(DOCK_EINVAL, "dock_create_pocket: NULL argument");
  *out = nullptr;
  if (d->n_types < 1 || d->n_types > DOCK_MAX_TYPES || !d->params)
    return fail(DOCK_EINVAL, "dock_create_pocket: n_types %d out of range", d->n_types);
  if (!(d->spacing > 0.0f) || !(d->radius > 0.0f))
    return fail(DOCK_EINVAL, "dock_create_pocket: spacing and radius must be > 0");
  if (d->n_atoms < 0 || (d->n_atoms > 0 && (!d->x || !d->y || !d->z || !d->q || !d->type)))
    return fail(DOCK_EINVAL, "dock_create_pocket: bad protein arrays");
  for (int t = 0; t < d->n_types; ++t) {
    const dock_type_params &p = d->params[t];
    if (p.hb_role < 0 || p.hb_role > 2 || !(p.Rii > 0) || !(p.eps >= 0))
      return fail(DOCK_EINVAL, "dock_create_pocket: bad parameters for type %d", t);
  }
  for (int i = 0; i < d->n_atoms; ++i) {
    if (d->type[i] >= d->n_types) return fail(DOCK_EINVAL, "protein atom %d: type out of range", i);
    if (!std::isfinite(d->x[i]) || !std::isfinite(d->y[i]) || !std::isfinite(d->z[i]) ||
        !std::isfinite(d->q[i]))
      return fail(DOCK_EINVAL, "protein atom %d: non-finite value", i);
  }
  const double n_f = std::floor(2.0 * (double)d->radius / (double)d->spacing + 1e-9) + 1.0;
  if (n_f < 2 || n_f > 1024) return fail(DOCK_EINVAL, "grid of %g nodes per axis", n_f);
  dock_pocket *P = new dock_pocket();
  std::unique_ptr<dock_pocket> guard(P);
  CU(cudaGetDevice(&P->device));
  P->n_types = d->n_types;
  P->params.assign(d->params, d->params + d->n_types);
  P->n_prot = d->n_atoms;
  P->n = (int)n_f;
  P->h = d->spacing;
  const double half = 0.5 * (P->n - 1) * P->h;
  P->ox = (double)d->center[0] - half;
  P->oy = (double)d->center[1] - half;
  P->oz = (double)d->center[2] - half;
  for (int m = 0; m < 3; ++m) P->center[m] = d->center[m];
  P->radius = d->radius;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nodes = (size_t)P->n * P->n * P->n;
  CU(dalloc(&P->d_params, P->n_types));
  CU(cudaMemcpyAsync(P->d_params, P->params.data(), sizeof(dock_type_params) * P->n_types,
                     cudaMemcpyHostToDevice, s));
  // ---- protein atoms by cell (kCellX in x, kCellYZ in y and z) and the
  // ---- type-pair tables (grid build and pairwise scorer) ----------------------
  std::vector<float4> cprot((size_t)d->n_atoms), cext((size_t)d->n_atoms);
  std::vector<int32_t> cell_start;
  {
    const double cs3[3] = {kCellX, kCellYZ, kCellYZ};
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int m = 0; m < 3; ++m) {
      const float *c = m == 0 ? d->x : (m == 1 ? d->y : d->z);
      lo[m] = d->n_atoms ? c[0] : 0.0;
      hi[m] = lo[m];
      for (int i = 1; i < d->n_atoms; ++i) {
        lo[m] = std::min(lo[m], (double)c[i]);
        hi[m] = std::max(hi[m], (double)c[i]);
      }
      P->cell_lo[m] = (float)(lo[m] - 0.5);
      const double dm = std::floor((hi[m] - (double)P->cell_lo[m]) / cs3[m]) + 1.0;
      if (dm > 4096) return fail(DOCK_EINVAL, "dock_create_pocket: protein extent too large");
      P->cell_dims[m] = (int)dm;
    }
    const int64_t ncell = (int64_t)P->cell_dims[0] * P->cell_dims[1] * P->cell_dims[2];
    if (ncell > (1 << 26)) return fail(DOCK_EINVAL, "dock_create_pocket: too many cells");
    std::vector<int32_t> cell_of((size_t)d->n_atoms);
    cell_start.assign((size_t)ncell + 1, 0);
    for (int i = 0; i < d->n_atoms; ++i) {
      int ci[3];
      const float c3[3] = {d->x[i], d->y[i], d->z[i]};
      for (int m = 0; m < 3; ++m)
        ci[m] = std::min(P->cell_dims[m] - 1,
                         std::max(0, (int)std::floor(((double)c3[m] - P->cell_lo[m]) / cs3[m])));
      cell_of[i] = (ci[2] * P->cell_dims[1] + ci[1]) * P->cell_dims[0] + ci[0];
      ++cell_start[(size_t)cell_of[i] + 1];
    }
    for (int64_t c = 0; c < ncell; ++c) cell_start[(size_t)c + 1] += cell_start[(size_t)c];
    std::vector<int32_t> fill(cell_start.begin(), cell_start.end() - 1);
    for (int i = 0; i < d->n_atoms; ++i) {
      const int dst = fill[(size_t)cell_of[i]]++;
      const dock_type_params &tq = P->params[d->type[i]];
      cprot[dst] = make_float4(d->x[i], d->y[i], d->z[i], d->q[i]);
      cext[dst] = make_float4((float)((double)tq.solpar + kHQasp * std::fabs((double)d->q[i])),
                              tq.vol, (float)d->type[i], 0.0f);
    }
  }
  std::vector<float4> tpair((size_t)P->n_types * P->n_types);
  std::vector<double4> gcoef((size_t)P->n_types * P->n_types);
  std::vector<float2> tsv((size_t)P->n_types);
  std::vector<double2> gtsv((size_t)P->n_types);
  for (int ti = 0; ti < P->n_types; ++ti) {
    tsv[ti] = make_float2(P->params[ti].solpar, P->params[ti].vol);
    gtsv[ti] = make_double2(P->params[ti].solpar, P->params[ti].vol);
    for (int tj = 0; tj < P->n_types; ++tj) {
      double c12, c6, c10, w;
      pair_coeffs(P->params.data(), ti, tj, c12, c6, c10, w);
      tpair[(size_t)ti * P->n_types + tj] =
          make_float4((float)c12, (float)c6, (float)c10, (float)(w * kHEmax));
      gcoef[(size_t)ti * P->n_types + tj] = make_double4(c12, c6, c10, w * kHEmax);
    }
  }
  CU(dalloc(&P->d_cprot, std::max<size_t>(1, cprot.size())));
  CU(dalloc(&P->d_cext, std::max<size_t>(1, cext.size())));
  CU(dalloc(&P->d_cell_start, cell_start.size()));
  CU(dalloc(&P->d_tpair, tpair.size()));
  CU(dalloc(&P->d_tsv, tsv.size()));
  if (d->n_atoms) {
    CU(cudaMemcpyAsync(P->d_cprot, cprot.data(), sizeof(float4) * cprot.size(), cudaMemcpyHostToDevice, s));
    CU(cudaMemcpyAsync(P->d_cext, cext.data(), sizeof(float4) * cext.size(), cudaMemcpyHostToDevice, s));
  }
  CU(cudaMemcpyAsync(P->d_cell_start, cell_start.data(), sizeof(int32_t) * cell_start.size(),
                     cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(P->d_tpair, tpair.data(), sizeof(float4) * tpair.size(), cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(P->d_tsv, tsv.data(), sizeof(float2) * tsv.size(), cudaMemcpyHostToDevice, s));
  double4 *d_gcoef = nullptr;
  double2 *d_gtsv = nullptr;
  CU(dalloc(&d_gcoef, gcoef.size()));
  CU(dalloc(&d_gtsv, gtsv.size()));
  std::unique_ptr<double4, void (*)(double4 *)> gcoef_guard(d_gcoef, [](double4 *q) { dfree(q); });
  std::unique_ptr<double2, void (*)(double2 *)> gtsv_guard(d_gtsv, [](double2 *q) { dfree(q); });
  CU(cudaMemcpyAsync(d_gcoef, gcoef.data(), sizeof(double4) * gcoef.size(), cudaMemcpyHostToDevice, s));
  CU(cudaMemcpyAsync(d_gtsv, gtsv.data(), sizeof(double2) * gtsv.size(), cudaMemcpyHostToDevice, s));
  // ---- grid maps ---------------------------------------------------------------
  CU(dalloc(&P->d_maps, nodes * P->n_types));
  CU(dalloc(&P->d_xycell, (size_t)P->n_types * 2 * P->n * (P->n - 1) * (P->n - 1) * 8));
  CU(dalloc(&P->d_fpm, nodes));
  {
    GridBuildArgs G;
    G.cprot = P->d_cprot;
    G.cext = P->d_cext;
    G.cells = cell_grid(P);
    G.coef = d_gcoef;
    G.tsv = d_gtsv;
    G.n_types = P->n_types;
    G.n = P->n;
    G.ox = P->ox;
    G.oy = P->oy;
    G.oz = P->oz;
    G.h = P->h;
    G.maps = P->d_maps;
    G.fpm = P->d_fpm;
    CU(launch_grid_build_impl(G, s));
  }
  CU(launch_xycell_maps(P->d_maps, P->d_fpm, P->n_types, P->n, P->d_xycell, s));
  {
    const size_t n4 = (size_t)P->n_types * 2 * P->n * (P->n - 1) * (P->n - 1) * 2;
    // the scorers index the records' 16-byte elements with 32-bit integers
    if (n4 > (size_t)INT32_MAX)
      return fail(DOCK_EINVAL, "dock_create_pocket: %zu grid records exceed 2^30", n4 / 2);
  }
  // the tables above are freed on return: wait for the kernels that read them
  CU(cudaStreamSynchronize(s));
  *out = guard.release();
  return DOCK_OK;
}

extern "C" void dock_pocket_destroy(dock_pocket *p) { delete p; }

extern "C" int dock_pocket_grid(const dock_pocket *p, int32_t *n, float origin[3],
                                const void **maps) {
  if (!p) return fail(DOCK_EINVAL, "dock_pocket_grid: NULL pocket");
  if (n) *n = p->n;
  if (origin) {
    origin[0] = (float)p->ox;
    origin[1] = (float)p->oy;
    origin[2] = (float)p->oz;
  }
  if (maps) *maps = p->d_maps;
  return DOCK_OK;
}

// ---------------------------------------------------------------------------
// ligands
// ---------------------------------------------------------------------------


namespace {
struct LigHost {
  std::vector<uint32_t> pair_idx;  // pairs the poses change, then the pose-invariant ones
  int n_var = 0;                   // pairs the poses change
  std::vector<float> pair_rec;   // 8 per pair the poses change
  std::vector<TorInfo> tors;   // move_off relative to this ligand's moves
  std::vector<uint8_t> moves;
  double cent[3];
  std::string err;
};

// Topology and pair coefficients of ligand l (see dock_load_ligands in dock.h).
// Weighted dispersion coefficients {c12, c6, c10, w} of every type pair (one
// table per dock_load_ligands call).
struct TypePairTable {
  int T = 0;
  std::vector<double> c;  // [T][T][4]
  explicit TypePairTable(const dock_pocket *P) : T(P->n_types), c((size_t)T * T * 4) {
    for (int ti = 0; ti < T; ++ti)
      for (int tj = 0; tj < T; ++tj) {
        double *q = &c[((size_t)ti * T + tj) * 4];
        pair_coeffs(P->params.data(), ti, tj, q[0], q[1], q[2], q[3]);
      }
  }
  const double *at(int ti, int tj) const { return &c[((size_t)ti * T + tj) * 4]; }
};

void prepare_ligand(const dock_ligand_batch *b, const dock_pocket *P, const TypePairTable &TP, int l,
                    LigHost &H) {
  const int a0 = b->atom_off[l], n = b->atom_off[l + 1] - a0;
  const int t0 = b->tors_off[l], k = b->tors_off[l + 1] - t0;
  char msg[160];
  if (n < 1 || n > DOCK_MAX_ATOMS) {
    snprintf(msg, sizeof msg, "ligand %d: %d atoms (1..%d)", l, n, DOCK_MAX_ATOMS);
    H.err = msg;
    return;
  }
  if (k < 0 || k > DOCK_MAX_TORSIONS) {
    snprintf(msg, sizeof msg, "ligand %d: %d torsions (0..%d)", l, k, DOCK_MAX_TORSIONS);
    H.err = msg;
    return;
  }
  const int16_t *par = b->parent + a0;
  for (int i = 0; i < n; ++i) {
    if ((i == 0 && par[i] != -1) || (i > 0 && (par[i] < 0 || par[i] >= i))) {
      snprintf(msg, sizeof msg, "ligand %d: atom %d has parent %d (need parent < index)", l, i, par[i]);
      H.err = msg;
      return;
    }
    if (b->type[a0 + i] >= P->n_types) {
      snprintf(msg, sizeof msg, "ligand %d: atom %d type out of range", l, i);
      H.err = msg;
      return;
    }
    if (!std::isfinite(b->x[a0 + i]) || !std::isfinite(b->y[a0 + i]) ||
        !std::isfinite(b->z[a0 + i]) || !std::isfinite(b->q[a0 + i])) {
      snprintf(msg, sizeof msg, "ligand %d: atom %d non-finite", l, i);
      H.err = msg;
      return;
    }
  }
  std::vector<uint8_t> rot((size_t)n, 0);
  for (int j = 0; j < k; ++j) {
    const int bb = b->tors_b[t0 + j];
    if (bb <= 0 || bb >= n || (j > 0 && b->tors_b[t0 + j - 1] >= bb)) {
      snprintf(msg, sizeof msg, "ligand %d: torsion %d child atom %d invalid or out of order", l, j, bb);
      H.err = msg;
      return;
    }
    rot[bb] = 1;
  }
  // centroid and children
  double c[3] = {0, 0, 0};
  for (int i = 0; i < n; ++i) {
    c[0] += b->x[a0 + i];
    c[1] += b->y[a0 + i];
    c[2] += b->z[a0 + i];
  }
  for (int m = 0; m < 3; ++m) H.cent[m] = c[m] / n;
  std::vector<std::vector<int>> kids((size_t)n);
  for (int i = 1; i < n; ++i) kids[par[i]].push_back(i);
  // atoms moved by each torsion: the subtree below b (b itself stays on the axis)
  for (int j = 0; j < k; ++j) {
    const int bb = b->tors_b[t0 + j];
    TorInfo T;
    T.move_off = (int32_t)H.moves.size();
    std::vector<int> stack(kids[bb].begin(), kids[bb].end());
    while (!stack.empty()) {
      const int a = stack.back();
      stack.pop_back();
      H.moves.push_back((uint8_t)a);
      for (int ch : kids[a]) stack.push_back(ch);
    }
    // ascending atom order: the L lanes then rotate mostly consecutive rows
    std::sort(H.moves.begin() + T.move_off, H.moves.end());
    T.n_move = (int16_t)(H.moves.size() - T.move_off);
    T.a = (uint8_t)par[bb];
    T.b = (uint8_t)bb;
    H.tors.push_back(T);
  }
  // rigid fragments: a rotatable bond starts a new fragment
  std::vector<int> frag((size_t)n, 0);
  int nf = 0;
  for (int i = 1; i < n; ++i) frag[i] = rot[i] ? ++nf : frag[par[i]];
  // bond distances by BFS from every atom
  std::vector<uint8_t> dist((size_t)n * n, 255);
  std::vector<int> queue((size_t)n);
  for (int s0 = 0; s0 < n; ++s0) {
    uint8_t *d = &dist[(size_t)s0 * n];
    int qh = 0, qt = 0;
    queue[qt++] = s0;
    d[s0] = 0;
    while (qh < qt) {
      const int a = queue[qh++];
      auto visit = [&](int v) {
        if (d[v] == 255) {
          d[v] = (uint8_t)std::min(254, d[a] + 1);
          queue[qt++] = v;
        }
      };
      if (a > 0) visit(par[a]);
      for (int ch : kids[a]) visit(ch);
    }
  }
  // a pair's distance changes with a torsion that moves one of its atoms and
  // not the other, unless the other lies on the torsion's axis
  std::vector<uint8_t> moved((size_t)k * n, 0);
  for (int t = 0; t < k; ++t)
    for (int m = 0; m < H.tors[t].n_move; ++m) moved[(size_t)t * n + H.moves[H.tors[t].move_off + m]] = 1;
  auto pose_invariant = [&](int i, int j) {
    for (int t = 0; t < k; ++t) {
      const uint8_t mi = moved[(size_t)t * n + i], mj = moved[(size_t)t * n + j];
      if (mi == mj) continue;
      const int still = mi ? j : i;
      if (still != H.tors[t].a && still != H.tors[t].b) return false;
    }
    return true;
  };
  std::vector<uint32_t> inv_idx;
  const dock_type_params *tp = P->params.data();
  // Row order of the per-pose pairs: rows i ascending; within a row the j are
  // permuted so that the pairs at list positions p of one aligned window of 4
  // (2, 8) have distinct j mod 4 (2, 8) where the row allows it. A pose's L
  // lanes read the atoms of pairs p .. p + L - 1 together, and distinct j
  // mod L keep those 16-byte shared-memory rows on distinct bank groups. The
  // residues taken in the current windows are kept as bitmasks; the first j
  // with the lowest clash cost (L = 4 first, then 2, then 8) is placed next.
  // The pose-invariant pairs (the FP64 constant's) keep plain row order.
  std::vector<int> row, order;
  uint32_t used4 = 0, used2 = 0, used8 = 0;
  auto cost = [&](int j) {
    return 100 * (int)((used4 >> (j & 3)) & 1u) + 10 * (int)((used2 >> (j & 1)) & 1u) +
           (int)((used8 >> (j & 7)) & 1u);
  };
  for (int i = 0; i < n; ++i) {
    row.clear();
    for (int j = i + 1; j < n; ++j) {
      if (dist[(size_t)i * n + j] <= 3 || frag[i] == frag[j]) continue;
      if (!pose_invariant(i, j)) {
        row.push_back(j);
        continue;
      }
      const bool hb = (tp[b->type[a0 + i]].hb_role == 1 && tp[b->type[a0 + j]].hb_role == 2) ||
                      (tp[b->type[a0 + i]].hb_role == 2 && tp[b->type[a0 + j]].hb_role == 1);
      inv_idx.push_back((uint32_t)i | ((uint32_t)j << 8) | ((uint32_t)(hb ? 1 : 0) << 16));
    }
    while (!row.empty()) {
      const int pos = (int)(order.size() / 2);
      if (pos % 4 == 0) used4 = 0;
      if (pos % 2 == 0) used2 = 0;
      if (pos % 8 == 0) used8 = 0;
      size_t best = 0;
      int best_c = cost(row[0]);
      for (size_t r = 1; r < row.size() && best_c > 0; ++r) {
        const int c = cost(row[r]);
        if (c < best_c) {
          best_c = c;
          best = r;
        }
      }
      const int j = row[best];
      used4 |= 1u << (j & 3);
      used2 |= 1u << (j & 1);
      used8 |= 1u << (j & 7);
      order.push_back(j);
      order.push_back(i);  // kept in pairs: order[2 p] = j, order[2 p + 1] = i
      row.erase(row.begin() + (long)best);
    }
  }
  H.pair_rec.reserve(order.size() * 2);
  H.pair_idx.reserve(order.size() / 2 + inv_idx.size());
  for (size_t p = 0; p < order.size() / 2; ++p) {
    {
      const int j = order[2 * p], i = order[2 * p + 1];
      const int ti = b->type[a0 + i], tj = b->type[a0 + j];
      const double qi = b->q[a0 + i], qj = b->q[a0 + j];
      const bool hb = (tp[ti].hb_role == 1 && tp[tj].hb_role == 2) ||
                      (tp[ti].hb_role == 2 && tp[tj].hb_role == 1);
      const double *cw = TP.at(ti, tj);
      const double c12 = cw[0], c6 = cw[1], c10 = cw[2], w = cw[3];
      const double si = (double)tp[ti].solpar + kHQasp * std::fabs(qi);
      const double sj = (double)tp[tj].solpar + kHQasp * std::fabs(qj);
      H.pair_idx.push_back((uint32_t)i | ((uint32_t)j << 8) | ((uint32_t)(hb ? 1 : 0) << 16));
      (void)w;
      const uint32_t oij = (16u * (uint32_t)i) | ((16u * (uint32_t)j) << 16);
      float oijf;
      std::memcpy(&oijf, &oij, 4);
      const float rec[4] = {oijf, (float)c12, hb ? (float)-c10 : (float)c6,
                            (float)(kHWSol * (si * tp[tj].vol + sj * tp[ti].vol))};
      H.pair_rec.insert(H.pair_rec.end(), rec, rec + 4);
    }
  }
  H.n_var = (int)H.pair_idx.size();
  H.pair_idx.insert(H.pair_idx.end(), inv_idx.begin(), inv_idx.end());
}

template <typename F>
void parallel_for(int n, F f) {
  int nt = (int)std::min<unsigned>(std::max(1u, std::thread::hardware_concurrency()), 64u);
  if (n < 64) nt = 1;
  std::atomic<int> next(0);
  auto work = [&]() {
    for (;;) {
      const int i = next.fetch_add(4);
      if (i >= n) break;
      for (int j = i; j < std::min(n, i + 4); ++j) f(j);
    }
  };
  std::vector<std::thread> th;
  for (int t = 1; t < nt; ++t) th.emplace_back(work);
  work();
  for (auto &t : th) t.join();
}
}  // namespace

// The bounds-checked build's report for calls without a status word of their
// own (scoring, pairwise scoring, standalone local search): waits for the
// stream and reads the ligand set's check word. A no-op in the normal build.
static int checked_report(dock_ligands *L, cudaStream_t s, const char *what) {
#ifdef DOCK_CHECKED
  int32_t w = 0;
  CU(cudaMemcpyAsync(&w, L->d_check, sizeof w, cudaMemcpyDeviceToHost, s));
  CU(cudaStreamSynchronize(s));
  if (w != 0) {
    CU(cudaMemsetAsync(L->d_check, 0, sizeof w, s));
    return fail(DOCK_EDEVICE, "%s: bounds check failed at site %d", what, kCheckBase - w);
  }
#else
  (void)L;
  (void)s;
  (void)what;
#endif
  return DOCK_OK;
}

extern "C" int dock_load_ligands(const dock_pocket *P, const dock_ligand_batch *b, void *stream,
                                 dock_ligands **out) {
  const dk::NvtxRange nvtx_range("dock_load_ligands");
  if (!P || !b || !out) return fail(DOCK_EINVAL, "dock_load_ligands: NULL argument");
  *out = nullptr;
  const int nl = b->n_ligands;
  if (nl < 0) return fail(DOCK_EINVAL, "dock_load_ligands: n_ligands < 0");
  if (nl > 0 && (!b->atom_off || !b->tors_off || !b->x || !b->y || !b->z || !b->q || !b->type ||
                 !b->parent || !b->ligand_id || (!b->tors_b && b->tors_off[nl] > 0)))
    return fail(DOCK_EINVAL, "dock_load_ligands: NULL array");
  if (nl > 0 && (b->atom_off[0] != 0 || b->tors_off[0] != 0))
    return fail(DOCK_EINVAL, "dock_load_ligands: offsets must start at 0");
  for (int l = 0; l < nl; ++l)
    if (b->atom_off[l + 1] < b->atom_off[l] || b->tors_off[l + 1] < b->tors_off[l])
      return fail(DOCK_EINVAL, "dock_load_ligands: offsets decrease at ligand %d", l);
  std::vector<LigHost> H((size_t)nl);
  const TypePairTable TP(P);
  parallel_for(nl, [&](int l) { prepare_ligand(b, P, TP, l, H[l]); });
  for (int l = 0; l < nl; ++l)
    if (!H[l].err.empty()) return fail(DOCK_EINVAL, "dock_load_ligands: %s", H[l].err.c_str());
  dock_ligands *L = new dock_ligands();
  std::unique_ptr<dock_ligands> guard(L);
  CU(cudaGetDevice(&L->device));
  L->n_ligands = nl;
  L->info.resize((size_t)nl);
  const int n_atoms = nl ? b->atom_off[nl] : 0;
  int64_t np = 0, nvar = 0, nm = 0, nt = 0;
  for (int l = 0; l < nl; ++l) {
    LigInfo &I = L->info[l];
    I.atom_off = b->atom_off[l];
    I.n = b->atom_off[l + 1] - b->atom_off[l];
    I.k = b->tors_off[l + 1] - b->tors_off[l];
    I.pair_off = (int32_t)np;
    I.n_pairs = H[l].n_var;
    I.n_pairs_all = (int32_t)H[l].pair_idx.size();
    I.intra_const = 0.0f;  // set on the device below
    I.tors_off = (int32_t)nt;
    I.ligand_id = b->ligand_id[l];
    for (auto &T : H[l].tors) T.move_off += (int32_t)nm;
    np += I.n_pairs_all;
    nvar += I.n_pairs;
    nm += (int64_t)H[l].moves.size();
    nt += I.k;
    L->max_atoms = std::max(L->max_atoms, I.n);
  }
  if (np > INT32_MAX || nm > INT32_MAX) return fail(DOCK_EINVAL, "dock_load_ligands: batch too large");
  L->total_pairs = nvar;
  L->total_pair_slots = np;
  std::vector<float4> atoms((size_t)n_atoms), raw((size_t)n_atoms);
  std::vector<double> cent((size_t)nl * 3);
  std::vector<uint32_t> pidx((size_t)np);
  // records of the per-pose pairs at their pair offsets; the slots of the
  // pose-invariant pairs are zeroed per ligand below (no serial fill)
  std::unique_ptr<float[]> prec(new float[(size_t)np * 4]);
  std::vector<TorInfo> tors((size_t)nt);
  std::vector<uint8_t> moves((size_t)nm);
  parallel_for(nl, [&](int l) {
    const LigInfo &I = L->info[l];
    for (int i = 0; i < I.n; ++i) {
      const int a = I.atom_off + i;
      raw[a] = make_float4(b->x[a], b->y[a], b->z[a], b->q[a]);
      atoms[a] = make_float4((float)(b->x[a] - H[l].cent[0]), (float)(b->y[a] - H[l].cent[1]),
                             (float)(b->z[a] - H[l].cent[2]), b->q[a]);
    }
    for (int m = 0; m < 3; ++m) cent[(size_t)l * 3 + m] = H[l].cent[m];
    std::copy(H[l].pair_idx.begin(), H[l].pair_idx.end(), pidx.begin() + I.pair_off);
    std::copy(H[l].pair_rec.begin(), H[l].pair_rec.end(), prec.get() + (size_t)I.pair_off * 4);
    std::fill(prec.get() + ((size_t)I.pair_off + I.n_pairs) * 4,
              prec.get() + ((size_t)I.pair_off + I.n_pairs_all) * 4, 0.0f);
    std::copy(H[l].tors.begin(), H[l].tors.end(), tors.begin() + I.tors_off);
    if (!H[l].tors.empty())
      std::copy(H[l].moves.begin(), H[l].moves.end(), moves.begin() + H[l].tors[0].move_off);
  });
  cudaStream_t s = (cudaStream_t)stream;
  CU(dalloc(&L->d_info, (size_t)nl));
  CU(dalloc(&L->d_atoms, (size_t)n_atoms));
  CU(dalloc(&L->d_atoms_raw, (size_t)n_atoms));
  CU(dalloc(&L->d_centroid, (size_t)nl * 3));
  CU(dalloc(&L->d_types, (size_t)n_atoms));
  CU(dalloc(&L->d_pair_idx, (size_t)np));
  CU(dalloc(&L->d_pair_rec, (size_t)np * 4));
  CU(dalloc(&L->d_tors, (size_t)nt));
  CU(dalloc(&L->d_moves, (size_t)nm));
  auto up = [&](void *dst, const void *src, size_t bytes) -> cudaError_t {
    return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s) : cudaSuccess;
  };
  CU(up(L->d_info, L->info.data(), sizeof(LigInfo) * nl));
  CU(up(L->d_atoms, atoms.data(), sizeof(float4) * n_atoms));
  CU(up(L->d_atoms_raw, raw.data(), sizeof(float4) * n_atoms));
  CU(up(L->d_centroid, cent.data(), sizeof(double) * cent.size()));
  CU(up(L->d_types, b->type, (size_t)n_atoms));
  CU(up(L->d_pair_idx, pidx.data(), sizeof(uint32_t) * np));
  CU(up(L->d_pair_rec, prec.get(), sizeof(float) * 4 * np));
  CU(up(L->d_tors, tors.data(), sizeof(TorInfo) * nt));
  CU(up(L->d_moves, moves.data(), (size_t)nm));
  CU(dalloc(&L->d_check, 1));
  CU(cudaMemsetAsync(L->d_check, 0, sizeof(int32_t), s));
  CU(launch_intra_const(L->d_info, nl, L->d_atoms_raw, L->d_types, L->d_pair_idx, P->d_params, s));
  CU(cudaStreamSynchronize(s));
  L->total_atoms = n_atoms;
  L->total_tors = nt;
  L->total_moved = nm;
  L->h2d_bytes = (int64_t)(sizeof(LigInfo) * nl + 2 * sizeof(float4) * n_atoms + sizeof(double) * 3 * nl +
                           n_atoms + (sizeof(uint32_t) + 4 * sizeof(float)) * np + sizeof(TorInfo) * nt + nm);
  *out = guard.release();
  return DOCK_OK;
}

extern "C" int dock_ligands_info(const dock_ligands *L, int32_t *n_ligands, int64_t *n_atoms,
                                 int64_t *n_pairs, int64_t *n_torsions, int64_t *n_moved,
                                 int64_t *h2d_bytes) {
  if (!L) return fail(DOCK_EINVAL, "dock_ligands_info: NULL ligands");
  if (n_ligands) *n_ligands = L->n_ligands;
  if (n_atoms) *n_atoms = L->total_atoms;
  if (n_pairs) *n_pairs = L->total_pairs;
  if (n_torsions) *n_torsions = L->total_tors;
  if (n_moved) *n_moved = L->total_moved;
  if (h2d_bytes) *h2d_bytes = L->h2d_bytes;
  return DOCK_OK;
}

extern "C" void dock_ligands_destroy(dock_ligands *l) { delete l; }

// ---------------------------------------------------------------------------
// search
// ---------------------------------------------------------------------------
struct dock_job {
  dock_ligands *L = nullptr;
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  int n_ligands = 0, pop = 0, generations = 0;
  int final_buf = 0;
  // optional per-launch timing of the search kernels
  std::vector<cudaEvent_t> ev;
  ~dock_job() {
    if (done) cudaEventDestroy(done);
    for (auto e : ev) cudaEventDestroy(e);
  }
};


// The launches of one search generation, one per lanes-per-pose group (items
// [begin, begin + count) of the item list): the first on q, the others on the
// workspace's side streams, forked from q and joined back, so a group's CTAs
// take over SMs as the previous group's queue drains.
struct LaunchGroup {
  int32_t L, begin, count, blocks;
  int32_t ls_begin, ls_count, ls_blocks;  // local-search units of the group
  int32_t ls_L, ls_apl;                   // lanes per chain, shared-memory atoms per lane
};

// One group's launches of generation a.gen on stream st: its search launch,
// then, with ls (Lamarckian search), its Solis-Wets launch over the same items
// (queue counters i and 4 + i of the generation).
static cudaError_t enqueue_group(const SearchArgs &a, const std::vector<LaunchGroup> &groups,
                                 size_t i, int threads, cudaStream_t st, const LsArgs *ls,
                                 bool pairwise) {
  SearchArgs b = a;
  b.items = a.items + groups[i].begin;
  b.n_items = groups[i].count;
  b.counter = a.counter + i;
  cudaError_t r = launch_search(b, groups[i].blocks, threads, groups[i].L, st, pairwise);
  if (r != cudaSuccess || ls == nullptr) return r;
  if (groups[i].ls_count == 0) return r;
  LsArgs c = *ls;
  const int64_t gl = (int64_t)a.gen * c.n_ligands;
  c.units = ls->units + groups[i].ls_begin;
  c.n_units = groups[i].ls_count;
  c.counter = a.counter + 4 + i;
  c.gen = (uint32_t)a.gen;
  c.sel_bits = ls->sel_bits + gl * c.sel_words;
  c.sel_count = ls->sel_count + gl;
  c.chain_ctr = ls->chain_ctr + gl;
  c.atoms_per_lane = groups[i].ls_apl;
  c.geno = a.geno_next;
  c.score = a.score_next;
  c.best = a.best_next;
  return launch_ls(c, groups[i].ls_blocks, threads, groups[i].ls_L, st);
}

// The launches of one generation, every group forked from q onto the
// workspace's side streams and joined back, so a group's CTAs take over SMs as
// the previous group's queue drains.
static cudaError_t enqueue_search(Workspace &W, const SearchArgs &a, const std::vector<LaunchGroup> &groups,
                                  int threads, cudaStream_t q, const LsArgs *ls = nullptr,
                                  bool pairwise = false) {
  cudaError_t e = cudaSuccess;
  if (groups.empty()) return cudaSuccess;
  if (groups.size() == 1) return enqueue_group(a, groups, 0, threads, q, ls, pairwise);
  if ((e = cudaEventRecord(W.fork, q)) != cudaSuccess) return e;
  for (size_t i = 1; i < groups.size(); ++i) {
    if ((e = cudaStreamWaitEvent(W.side[i - 1], W.fork, 0)) != cudaSuccess) return e;
    if ((e = enqueue_group(a, groups, i, threads, W.side[i - 1], ls, pairwise)) != cudaSuccess)
      return e;
    if ((e = cudaEventRecord(W.join[i - 1], W.side[i - 1])) != cudaSuccess) return e;
  }
  if ((e = enqueue_group(a, groups, 0, threads, q, ls, pairwise)) != cudaSuccess) return e;
  for (size_t i = 1; i < groups.size(); ++i)
    if ((e = cudaStreamWaitEvent(q, W.join[i - 1], 0)) != cudaSuccess) return e;
  return cudaSuccess;
}

// Launch configuration of the search kernel: threads per CTA and the smem
// capacity in atoms per lane; a ligand of n atoms runs with the smallest
// L in {1, 2, 4, 8} with L * atoms_per_lane >= n.
struct LaunchCfg {
  int threads = 128;
  int atoms_per_lane = 16;
};


extern "C" int dock_batch(dock_pocket *P, dock_ligands *L, const dock_search_params *sp, void *stream,
                          dock_job **out) {
  const dk::NvtxRange nvtx_range("dock_batch");
  if (!P || !L || !sp || !out) return fail(DOCK_EINVAL, "dock_batch: NULL argument");
  *out = nullptr;
  if (sp->pop < 2 || sp->pop > DOCK_MAX_POP) return fail(DOCK_EINVAL, "dock_batch: pop %d", sp->pop);
  if (sp->generations < 1) return fail(DOCK_EINVAL, "dock_batch: generations %d", sp->generations);
  if (!(sp->p_cross >= 0 && sp->p_cross <= 1 && sp->p_mut >= 0 && sp->p_mut <= 1))
    return fail(DOCK_EINVAL, "dock_batch: probabilities out of [0, 1]");
  const bool sur = sp->mode == DOCK_MODE_SURROGATE;
  if (sp->mode != DOCK_MODE_PLAIN && !sur) return fail(DOCK_EINVAL, "dock_batch: mode %d", sp->mode);
  if (sur && (!sp->surrogate || sp->candidates < 1 || sp->candidates > DOCK_MAX_CANDIDATES ||
              sp->keep < 1 || sp->keep > sp->candidates || sp->pop + sp->keep > 16384))
    return fail(DOCK_EINVAL, "dock_batch: surrogate mode needs a surrogate, 1 <= keep <= "
                             "candidates <= %d and pop + keep <= 16384", DOCK_MAX_CANDIDATES);
  if (sp->inter != DOCK_INTER_GRID && sp->inter != DOCK_INTER_PAIRWISE)
    return fail(DOCK_EINVAL, "dock_batch: inter %d", sp->inter);
  const bool pairwise = sp->inter == DOCK_INTER_PAIRWISE;
  if (pairwise && (sur || sp->ls.rate != 0.0f))
    return fail(DOCK_EINVAL, "dock_batch: the pairwise inter-energy needs the plain GA");
  const bool resume = sp->resume_genotypes != nullptr;
  if (resume && (sur || sp->ls.rate != 0.0f || !sp->resume_scores || sp->resume_from < 0 ||
                 sp->resume_from > sp->generations - 2))
    return fail(DOCK_EINVAL, "dock_batch: resume needs the plain GA without local search, "
                             "scores, and 0 <= resume_from <= generations - 2");
  const int forced = sp->lanes_per_pose;
  if (forced != 0 && forced != 1 && forced != 2 && forced != 4 && forced != 8)
    return fail(DOCK_EINVAL, "dock_batch: lanes_per_pose %d", forced);
  if (!(sp->ls.rate >= 0.0f && sp->ls.rate <= 1.0f))
    return fail(DOCK_EINVAL, "dock_batch: ls.rate out of [0, 1]");
  const bool lamarck = sp->ls.rate > 0.0f;
  if (lamarck && sur) return fail(DOCK_EINVAL, "dock_batch: local search needs the plain mode");
  if (lamarck) {
    const int st = check_ls_params(&sp->ls, "dock_batch");
    if (st != DOCK_OK) return st;
  }
  CU(cudaSetDevice(L->device));
  cudaStream_t s = (cudaStream_t)stream;
  const int nl = L->n_ligands, pop = sp->pop, gens = sp->generations;
  LaunchCfg cfg;
  if (L->tuned_threads) {
    cfg.threads = L->tuned_threads;
    cfg.atoms_per_lane = L->tuned_apl;
  }
  if (const char *e = getenv("DOCK_THREADS")) cfg.threads = atoi(e);
  if (const char *e = getenv("DOCK_ATOMS_PER_LANE")) cfg.atoms_per_lane = atoi(e);
  if (forced) cfg.atoms_per_lane = std::max(cfg.atoms_per_lane, (L->max_atoms + forced - 1) / forced);
  if (L->max_atoms > 8 * cfg.atoms_per_lane) cfg.atoms_per_lane = (L->max_atoms + 7) / 8;
  if (cfg.threads < 32 || cfg.threads > 128 || (cfg.threads & (cfg.threads - 1)) || cfg.atoms_per_lane < 1)
    return fail(DOCK_EINVAL, "dock_batch: launch shape %d threads x %d atoms per lane", cfg.threads,
                cfg.atoms_per_lane);
  // keep the coordinate planes within the shared memory an SM offers
  while (search_smem_bytes(cfg.threads, cfg.atoms_per_lane) > 200 * 1024 && cfg.threads > 32)
    cfg.threads >>= 1;
  if (search_smem_bytes(cfg.threads, cfg.atoms_per_lane) > 200 * 1024)
    return fail(DOCK_EINVAL, "dock_batch: ligands too large for the requested lanes per pose");
  Workspace &W = L->ws;
  // genotype offsets and work items (largest first)
  std::vector<int64_t> goff((size_t)nl);
  int64_t total_genes = 0;
  for (int l = 0; l < nl; ++l) {
    goff[l] = total_genes;
    total_genes += (int64_t)pop * (7 + L->info[l].k);
  }
  struct Keyed {
    float cost;
    Item it;
  };
  std::vector<Keyed> items;
  for (int l = 0; l < nl; ++l) {
    const LigInfo &I = L->info[l];
    const int Ln = lanes_for(I.n, cfg.atoms_per_lane, forced);
    const int S = cfg.threads / Ln;
    const int tiles = (pop + S - 1) / S;
    const float cost = (float)(I.n_pairs + 6 * I.n + 12 * I.k) / Ln + 60.0f;
    for (int t = 0; t < tiles; ++t) items.push_back({cost, Item{l, (int16_t)t, (int8_t)Ln, 0}});
  }
  // grouped by lanes per pose (one launch per group), largest first in a group
  std::stable_sort(items.begin(), items.end(), [](const Keyed &a, const Keyed &b) {
    return a.it.lanes != b.it.lanes ? a.it.lanes > b.it.lanes : a.cost > b.cost;
  });
  std::vector<Item> host_items(items.size());
  for (size_t i = 0; i < items.size(); ++i) host_items[i] = items[i].it;
  std::vector<LaunchGroup> groups;
  for (size_t i = 0; i < host_items.size(); ++i) {
    if (groups.empty() || groups.back().L != host_items[i].lanes)
      groups.push_back(LaunchGroup{host_items[i].lanes, (int32_t)i, 0, 0});
    ++groups.back().count;
  }
  // local-search units: each ligand of a group R times (R warps share its
  // chains, about three chains per lane group), largest ligands first
  std::vector<int32_t> host_units;
  // lanes per chain (at least the search group's): more lanes shorten a
  // chain's sequence of probes, the longest of which bounds a generation
  int ls_lanes = 16;
  if (const char *e = getenv("DOCK_LS_LANES")) ls_lanes = atoi(e);
  // chains a lane group is expected to run one after another (sets how many
  // warps share a ligand's chains)
  double ls_chains = 2.0;
  if (const char *e = getenv("DOCK_LS_CHAINS")) ls_chains = std::max(0.25, atof(e));
  if (ls_lanes != 0 && ls_lanes != 1 && ls_lanes != 2 && ls_lanes != 4 && ls_lanes != 8 &&
      ls_lanes != 16 && ls_lanes != 32)
    return fail(DOCK_EINVAL, "dock_batch: DOCK_LS_LANES %d", ls_lanes);
  if (lamarck) {
    for (LaunchGroup &gr : groups) {
      gr.ls_L = std::max(gr.L, ls_lanes);
      gr.ls_apl = (gr.L * cfg.atoms_per_lane + gr.ls_L - 1) / gr.ls_L;
      const int gpw = 32 / gr.ls_L;
      const double expect = (double)sp->ls.rate * pop;
      const int R = std::max(1, (int)std::ceil(expect / (ls_chains * gpw)));
      gr.ls_begin = (int32_t)host_units.size();
      int last = -1;
      for (int i = gr.begin; i < gr.begin + gr.count; ++i) {
        const int l = host_items[i].lig;
        if (l == last) continue;  // items of a ligand are adjacent (same cost)
        last = l;
        for (int r = 0; r < R; ++r) host_units.push_back(l);
      }
      gr.ls_count = (int32_t)host_units.size() - gr.ls_begin;
    }
  } else {
    for (LaunchGroup &gr : groups) gr.ls_begin = gr.ls_count = gr.ls_L = gr.ls_apl = 0;
  }
  const size_t n_scores = (size_t)nl * pop;
  // workspace: grown on demand and reused by later batches on this ligand set
  if ((size_t)total_genes > W.geno_cap || !W.geno[0]) {
    dfree(W.geno[0]);
    dfree(W.geno[1]);
    W.geno_cap = 0;
    CU(dalloc(&W.geno[0], (size_t)total_genes));
    CU(dalloc(&W.geno[1], (size_t)total_genes));
    W.geno_cap = (size_t)total_genes;
  }
  if (n_scores > W.score_cap || !W.score[0]) {
    dfree(W.score[0]);
    dfree(W.score[1]);
    W.score_cap = 0;
    CU(dalloc(&W.score[0], n_scores));
    CU(dalloc(&W.score[1], n_scores));
    W.score_cap = n_scores;
  }
  if ((size_t)gens * nl > W.best_cap || !W.best) {
    dfree(W.best);
    W.best_cap = 0;
    CU(dalloc(&W.best, (size_t)gens * nl));
    W.best_cap = (size_t)gens * nl;
  }
  if ((size_t)gens * 8 > W.gen_cap || !W.counters) {
    dfree(W.counters);
    W.gen_cap = 0;
    CU(dalloc(&W.counters, (size_t)gens * 8));
    W.gen_cap = (size_t)gens * 8;
  }
  if (groups.size() > 1 && !W.fork) {
    for (int i = 0; i < 3; ++i) {
      CU(cudaStreamCreateWithFlags(&W.side[i], cudaStreamNonBlocking));
      CU(cudaEventCreateWithFlags(&W.join[i], cudaEventDisableTiming));
    }
    CU(cudaEventCreateWithFlags(&W.fork, cudaEventDisableTiming));
  }
  if (!W.io) {
    CU(cudaStreamCreateWithFlags(&W.io, cudaStreamNonBlocking));
    CU(cudaEventCreateWithFlags(&W.io_done, cudaEventDisableTiming));
  }
  // buffers allocated by this call: no queued work can be reading them
  bool fresh_items = false, fresh_goff = false, fresh_units = false;
  if (host_items.size() > W.item_cap || !W.items) {
    dfree(W.items);
    W.item_cap = 0;
    CU(dalloc(&W.items, host_items.size()));
    W.item_cap = host_items.size();
    fresh_items = true;
  }
  if ((size_t)nl > W.lig_cap || !W.geno_off) {
    fresh_goff = true;
    dfree(W.geno_off);
    dfree(W.lig_status);
    dfree(W.results);
    W.lig_cap = 0;
    dfree(W.ls_evals);
    CU(dalloc(&W.geno_off, (size_t)nl));
    CU(dalloc(&W.lig_status, (size_t)nl));
    CU(dalloc(&W.results, (size_t)nl));
    CU(dalloc(&W.ls_evals, (size_t)nl));
    W.lig_cap = (size_t)nl;
  }
  if (!W.status) CU(dalloc(&W.status, 1));
  if (!W.deadline) CU(dalloc(&W.deadline, 1));
  const int sel_words = (pop + 31) / 32;
  if (lamarck) {
    const size_t nb = (size_t)gens * nl * sel_words, nc = (size_t)gens * nl;
    if (nb > W.ls_bits_cap || !W.ls_bits) {
      dfree(W.ls_bits);
      W.ls_bits_cap = 0;
      CU(dalloc(&W.ls_bits, nb));
      W.ls_bits_cap = nb;
    }
    if (nc > W.ls_count_cap || !W.ls_count) {
      dfree(W.ls_count);
      dfree(W.ls_chain);
      W.ls_count_cap = 0;
      CU(dalloc(&W.ls_count, nc));
      CU(dalloc(&W.ls_chain, nc));
      W.ls_count_cap = nc;
    }
    if (host_units.size() > W.ls_units_cap || !W.ls_units) {
      dfree(W.ls_units);
      W.ls_units_cap = 0;
      CU(dalloc(&W.ls_units, host_units.size()));
      W.ls_units_cap = host_units.size();
      fresh_units = true;
    }
  }
  // The host tables: one the device already holds is not copied again; one
  // going into a buffer allocated above is copied on the io stream, which s
  // then waits for; a changed one in a buffer that searches queued on s may
  // still read is copied on s, after them.
  bool io_used = false;
  auto upload = [&](void *dst, const void *src, size_t bytes, std::vector<uint8_t> &last,
                    bool fresh) -> cudaError_t {
    const uint8_t *b = static_cast<const uint8_t *>(src);
    if (!fresh && last.size() == bytes && (bytes == 0 || memcmp(last.data(), b, bytes) == 0))
      return cudaSuccess;
    last.clear();  // unknown until the copy is queued
    if (bytes) {
      const cudaError_t e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, fresh ? W.io : s);
      if (e != cudaSuccess) return e;
      io_used |= fresh;
    }
    last.assign(b, b + bytes);
    return cudaSuccess;
  };
  if (lamarck)
    CU(upload(W.ls_units, host_units.data(), sizeof(int32_t) * host_units.size(), W.up_units,
              fresh_units));
  CU(upload(W.geno_off, goff.data(), sizeof(int64_t) * nl, W.up_goff, fresh_goff));
  CU(upload(W.items, host_items.data(), sizeof(Item) * host_items.size(), W.up_items, fresh_items));
  if (io_used) {
    CU(cudaEventRecord(W.io_done, W.io));
    CU(cudaStreamWaitEvent(s, W.io_done, 0));
  }
  int n_sm = 0;
  CU(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, L->device));
  for (LaunchGroup &gr : groups) {
    int per_sm = 0;
    CU(search_occupancy(cfg.threads, gr.L, cfg.atoms_per_lane, &per_sm, pairwise));
    if (per_sm < 1) return fail(DOCK_EINVAL, "dock_batch: launch shape does not fit an SM");
    gr.blocks = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * n_sm, gr.count));
    gr.ls_blocks = 0;
    if (lamarck && gr.ls_count > 0) {
      // one warp per unit
      CU(ls_occupancy(cfg.threads, gr.ls_L, gr.ls_apl, &per_sm));
      if (per_sm < 1) return fail(DOCK_EINVAL, "dock_batch: launch shape does not fit an SM");
      const int64_t need = (gr.ls_count + cfg.threads / 32 - 1) / (cfg.threads / 32);
      gr.ls_blocks = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * n_sm, need));
    }
  }

  dock_job *J = new dock_job();
  std::unique_ptr<dock_job> jguard(J);
  J->L = L;
  J->stream = s;
  J->n_ligands = nl;
  J->pop = pop;
  J->generations = gens;
  J->final_buf = (gens - 1) & 1;
  CU(cudaEventCreateWithFlags(&J->done, cudaEventDisableTiming));
  const bool profile = getenv("DOCK_PROFILE_LAUNCHES") != nullptr || L->profiling;

  SearchArgs A;
  A.ligs = L->d_info;
  A.atoms = L->d_atoms;
  A.types = L->d_types;
  A.pair_rec = L->d_pair_rec;
  A.tors = L->d_tors;
  A.moves = L->d_moves;
  A.geno_off = W.geno_off;
  A.items = W.items;
  A.n_items = (int32_t)host_items.size();
  A.atoms_per_lane = cfg.atoms_per_lane;
  A.grid = grid_view(P);
  A.cx = P->center[0];
  A.cy = P->center[1];
  A.cz = P->center[2];
  A.radius = P->radius;
  A.pop = pop;
  A.seed = sp->seed;
  A.thr_cross = prob_threshold(sp->p_cross);
  A.thr_mut = prob_threshold(sp->p_mut);
  A.status = W.status;
  A.lig_status = W.lig_status;
  A.deadline = sp->timeout_ns ? W.deadline : nullptr;
  A.pw = pw_view(P);
  A.bounds = bounds_of(P, L, W.status);

  LsArgs LA{};
  if (lamarck) {
    LA.ligs = L->d_info;
    LA.atoms = L->d_atoms;
    LA.types = L->d_types;
    LA.pair_rec = L->d_pair_rec;
    LA.tors = L->d_tors;
    LA.moves = L->d_moves;
    LA.grid = grid_view(P);
    LA.cx = P->center[0];
    LA.cy = P->center[1];
    LA.cz = P->center[2];
    LA.atoms_per_lane = cfg.atoms_per_lane;
    LA.max_its = sp->ls.max_its;
    LA.max_succ = sp->ls.max_succ;
    LA.max_fail = sp->ls.max_fail;
    LA.rho = sp->ls.rho;
    LA.rho_lb = sp->ls.rho_lb;
    LA.seed = sp->seed;
    LA.units = W.ls_units;
    LA.sel_bits = W.ls_bits;
    LA.sel_count = W.ls_count;
    LA.chain_ctr = W.ls_chain;
    LA.sel_words = sel_words;
    LA.n_ligands = nl;
    LA.geno_off = W.geno_off;
    LA.pop = pop;
    LA.evals = W.ls_evals;
    LA.status = W.status;
    LA.bounds = bounds_of(P, L, W.status);
    LA.deadline = A.deadline;
  }

  Fp64Args F;
  F.ligs = L->d_info;
  F.atoms = L->d_atoms_raw;
  F.types = L->d_types;
  F.pair_idx = L->d_pair_idx;
  F.tors = L->d_tors;
  F.moves = L->d_moves;
  F.grid = grid_view(P);
  F.h = P->h;
  F.cx = P->center[0];
  F.cy = P->center[1];
  F.cz = P->center[2];
  F.params = P->d_params;
  F.pairwise = pairwise ? 1 : 0;
  F.pw = pw_view(P);

  const int C = sur ? sp->candidates : 0, K = sur ? sp->keep : 0;
  if (sur) {
    const size_t rows = (size_t)nl * C, kept = (size_t)nl * K;
    if (rows > W.sur_cap || !W.cand_geno) {
      dfree(W.cand_geno);
      dfree(W.pred);
      dfree(W.feats);
      W.sur_cap = 0;
      CU(dalloc(&W.cand_geno, rows * DOCK_MAX_GENES));
      CU(dalloc(&W.pred, rows));
      CU(dalloc(&W.feats, rows * DOCK_N_FEATURES));
      W.sur_cap = rows;
    }
    if (kept > W.kept_cap || !W.kept_geno) {
      dfree(W.kept_geno);
      dfree(W.kept_score);
      dfree(W.kept_lig);
      W.kept_cap = 0;
      CU(dalloc(&W.kept_geno, kept * DOCK_MAX_GENES));
      CU(dalloc(&W.kept_score, kept));
      CU(dalloc(&W.kept_lig, kept));
      W.kept_cap = kept;
    }
  }
  FeatureLaunch FL{};
  FL.ligs = L->d_info;
  FL.atoms = L->d_atoms;
  FL.types = L->d_types;
  FL.pair_rec = L->d_pair_rec;
  FL.tors = L->d_tors;
  FL.moves = L->d_moves;
  FL.grid = grid_view(P);
  FL.cx = P->center[0];
  FL.cy = P->center[1];
  FL.cz = P->center[2];
  FL.radius = P->radius;
  FL.n_ligands = nl;
  FL.from_ga = true;
  FL.pop = pop;
  FL.candidates = C;
  FL.seed = sp->seed;
  FL.thr_cross = A.thr_cross;
  FL.thr_mut = A.thr_mut;
  FL.geno_off = W.geno_off;
  FL.cand_geno = W.cand_geno;
  FL.features = W.feats;
  ScoreArgs KS{};
  KS.ligs = L->d_info;
  KS.atoms = L->d_atoms;
  KS.types = L->d_types;
  KS.pair_rec = L->d_pair_rec;
  KS.tors = L->d_tors;
  KS.moves = L->d_moves;
  KS.grid = grid_view(P);
  KS.cx = P->center[0];
  KS.cy = P->center[1];
  KS.cz = P->center[2];
  KS.pose_ligand = W.kept_lig;
  KS.n_ligands = nl;
  KS.genos = W.kept_geno;
  KS.n_poses = (int64_t)nl * K;
  KS.scores = W.kept_score;
  KS.coords = nullptr;
  KS.lanes = 8;
  KS.atoms_per_lane = DOCK_MAX_ATOMS / 8;
  KS.bounds = bounds_of(P, L, W.status);

  // One surrogate generation g >= 1: candidates + features, prediction, top
  // `keep`, exact scores of the kept, mu + lambda merge into generation g.
  auto surrogate_generation = [&](int g, cudaStream_t q) -> int {
    FeatureLaunch f = FL;
    f.gen = g;
    f.geno_prev = W.geno[(g + 1) & 1];
    f.score_prev = W.score[(g + 1) & 1];
    CU(launch_features(f, q));
    const int pst = dk_surrogate_predict_raw(sp->surrogate, W.feats, (int64_t)nl * C, W.pred, 0, q);
    if (pst != DOCK_OK) return pst;
    CU(launch_topk(W.pred, nl, C, K, W.cand_geno, W.kept_geno, W.kept_lig, q));
    CU(launch_score(KS, q));
    CU(launch_merge(W.geno[(g + 1) & 1], W.score[(g + 1) & 1], W.geno_off, L->d_info, nl, pop,
                    W.kept_geno, W.kept_score, K, W.geno[g & 1], W.score[g & 1], q));
    return DOCK_OK;
  };

  const int g_first = resume ? sp->resume_from + 1 : 0;  // first generation this call runs
  // The groups hold disjoint ligands and every buffer a generation writes is
  // indexed by ligand (genotypes, scores, best keys, Solis-Wets selections and
  // chain counters), so unless a whole generation is copied out (traces) or
  // timed, each group can run its generations on its own stream, the streams
  // joined once, before the finalize: one group's tail (the last items of a
  // generation, the longest Solis-Wets chains) then overlaps the others' next
  // generations instead of idling SMs at a join per generation. That pays
  // where tails are a sizeable share of a generation: with local search, or
  // when a persistent CTA takes few items per generation (1,000 ligands of
  // 10-60 atoms x 1,024 poses: about 30; 62.0 vs 62.9 ms per search). With
  // hundreds per CTA (100,000 ligands of 8-100 atoms x 512 poses: about 600)
  // the tails are negligible and groups that stay in step share the SMs
  // better (1,500 vs 1,541 ms per search with free-running groups).
  int64_t most_per_block = 0;
  for (const LaunchGroup &gr : groups)
    most_per_block = std::max<int64_t>(most_per_block, gr.count / std::max(gr.blocks, 1));
  const bool free_run = groups.size() > 1 && !sur && !profile && !sp->trace_genotypes &&
                        !sp->trace_scores && (lamarck || most_per_block < 128);
  auto enqueue = [&](cudaStream_t q) -> int {
    CU(cudaMemsetAsync(W.counters, 0, sizeof(uint32_t) * gens * 8, q));
    if (lamarck) {
      CU(cudaMemsetAsync(W.ls_evals, 0, sizeof(unsigned long long) * (size_t)nl, q));
      CU(cudaMemsetAsync(W.ls_chain, 0, sizeof(uint32_t) * (size_t)gens * nl, q));
      // which individuals each generation refines (drawn up front: no data dependence)
      CU(launch_ls_select(L->d_info, nl, pop, gens, sp->seed, prob_threshold(sp->ls.rate), W.ls_bits,
                          W.ls_count, q));
    }
    CU(cudaMemsetAsync(W.best, 0xFF, sizeof(unsigned long long) * (size_t)gens * nl, q));
    CU(cudaMemsetAsync(W.status, 0, sizeof(int32_t), q));
    CU(cudaMemsetAsync(W.lig_status, 0, sizeof(int32_t) * (size_t)nl, q));
    if (sp->timeout_ns) CU(launch_set_deadline(W.deadline, sp->timeout_ns, q));
    if (resume) {
      // the saved generation becomes the previous one of the first generation run
      const int g = sp->resume_from;
      if (total_genes)
        CU(cudaMemcpyAsync(W.geno[g & 1], sp->resume_genotypes, sizeof(float) * total_genes,
                           cudaMemcpyDeviceToDevice, q));
      if (n_scores)
        CU(cudaMemcpyAsync(W.score[g & 1], sp->resume_scores, sizeof(float) * n_scores,
                           cudaMemcpyDeviceToDevice, q));
      CU(launch_best_keys(W.score[g & 1], nl, pop, W.best + (size_t)g * nl, q));
    }
    auto gen_args = [&](int g) {
      SearchArgs a = A;
      a.gen = g;
      a.counter = W.counters + (size_t)g * 8;  // 4 search + 4 local-search queues
      a.geno_prev = W.geno[(g + 1) & 1];
      a.geno_next = W.geno[g & 1];
      a.score_prev = W.score[(g + 1) & 1];
      a.score_next = W.score[g & 1];
      a.best_prev = g ? W.best + (size_t)(g - 1) * nl : nullptr;
      a.best_next = W.best + (size_t)g * nl;
      return a;
    };
    auto gen_ls = [&](int g) {
      LsArgs la = LA;
      if (lamarck && sp->trace_ls)
        la.trace = sp->trace_ls + (size_t)g * n_scores * (size_t)(2 + 2 * sp->ls.max_its);
      return la;
    };
    if (free_run) {
      // each group runs all its generations on its own stream; one join
      CU(cudaEventRecord(W.fork, q));
      for (size_t i = 1; i < groups.size(); ++i) CU(cudaStreamWaitEvent(W.side[i - 1], W.fork, 0));
      for (int g = g_first; g < gens; ++g) {
        const SearchArgs a = gen_args(g);
        const LsArgs la = gen_ls(g);
        for (size_t i = 0; i < groups.size(); ++i)
          CU(enqueue_group(a, groups, i, cfg.threads, i ? W.side[i - 1] : q,
                           lamarck ? &la : nullptr, pairwise));
      }
      for (size_t i = 1; i < groups.size(); ++i) {
        CU(cudaEventRecord(W.join[i - 1], W.side[i - 1]));
        CU(cudaStreamWaitEvent(q, W.join[i - 1], 0));
      }
    }
    for (int g = free_run ? gens : g_first; g < gens; ++g) {
      const SearchArgs a = gen_args(g);
      if (sur && g > 0) {
        const int st2 = surrogate_generation(g, q);
        if (st2 != DOCK_OK) return st2;
      } else {
        const LsArgs la = gen_ls(g);
        if (profile) {
          cudaEvent_t e0, e1;
          CU(cudaEventCreate(&e0));
          CU(cudaEventCreate(&e1));
          J->ev.push_back(e0);
          J->ev.push_back(e1);
          CU(cudaEventRecord(e0, q));
          CU(enqueue_search(W, a, groups, cfg.threads, q, lamarck ? &la : nullptr, pairwise));
          CU(cudaEventRecord(e1, q));
        } else {
          CU(enqueue_search(W, a, groups, cfg.threads, q, lamarck ? &la : nullptr, pairwise));
        }
      }
      if (sp->trace_genotypes && total_genes)
        CU(cudaMemcpyAsync(sp->trace_genotypes + (size_t)g * total_genes, W.geno[g & 1],
                           sizeof(float) * total_genes, cudaMemcpyDeviceToDevice, q));
      if (sp->trace_scores && n_scores)
        CU(cudaMemcpyAsync(sp->trace_scores + (size_t)g * n_scores, W.score[g & 1],
                           sizeof(float) * n_scores, cudaMemcpyDeviceToDevice, q));
    }
    CU(launch_finalize_impl(F, L->d_centroid, nl, pop, W.geno_off, W.geno[(gens - 1) & 1],
                            W.score[(gens - 1) & 1], W.lig_status, W.status,
                            sur ? (uint64_t)pop + (uint64_t)(gens - 1) * K
                                : (uint64_t)pop * (uint64_t)(gens - g_first),
                            sur ? (uint64_t)(gens - 1) * C : 0, lamarck ? W.ls_evals : nullptr,
                            P->ox, P->oy, P->oz, W.results, q));
    return DOCK_OK;
  };

  if (sp->use_graph && !profile && !sur && s != nullptr) {
    // graph key: everything the captured launches depend on
    std::vector<uint8_t> key;
    auto put = [&](const void *p, size_t n) {
      const uint8_t *c = (const uint8_t *)p;
      key.insert(key.end(), c, c + n);
    };
    put(&A, sizeof A);
    put(&F, sizeof F);
    put(&gens, sizeof gens);
    put(groups.data(), sizeof(LaunchGroup) * groups.size());
    put(&cfg, sizeof cfg);
    put(&sp->trace_genotypes, sizeof(void *));
    put(&sp->trace_scores, sizeof(void *));
    put(&sp->ls, sizeof sp->ls);
    put(&sp->trace_ls, sizeof(void *));
    put(&sp->inter, sizeof sp->inter);
    put(&sp->resume_genotypes, sizeof(void *));
    put(&sp->resume_scores, sizeof(void *));
    put(&g_first, sizeof g_first);
    const void *bufs[11] = {W.geno[0], W.geno[1], W.score[0], W.score[1], W.best, W.results,
                            W.ls_evals, W.ls_bits, W.ls_count, W.ls_chain, W.ls_units};
    put(bufs, sizeof bufs);
    if (!W.graph || key != W.graph_key) {
      if (W.graph) {
        cudaGraphExecDestroy(W.graph);
        W.graph = nullptr;
      }
      cudaGraph_t graph;
      CU(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      int est = enqueue(s);
      cudaError_t ce = cudaStreamEndCapture(s, &graph);
      if (est != DOCK_OK) {
        if (ce == cudaSuccess) cudaGraphDestroy(graph);
        return est;
      }
      CU(ce);
      cudaError_t ie = cudaGraphInstantiate(&W.graph, graph, 0);
      cudaGraphDestroy(graph);
      CU(ie);
      W.graph_key = key;
    }
    CU(cudaGraphLaunch(W.graph, s));
  } else {
    int est = enqueue(s);
    if (est != DOCK_OK) return est;
  }
  CU(cudaEventRecord(J->done, s));
  *out = jguard.release();
  return DOCK_OK;
}

extern "C" int dock_results(dock_job *J, dock_result *out, int32_t cap, uint64_t timeout_ns) {
  const dk::NvtxRange nvtx_range("dock_results");
  if (!J) return fail(DOCK_EINVAL, "dock_results: NULL job");
  if (cap < 0 || (cap > 0 && !out)) return fail(DOCK_EINVAL, "dock_results: bad output buffer");
  CU(cudaSetDevice(J->L->device));
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    cudaError_t q = cudaEventQuery(J->done);
    if (q == cudaSuccess) break;
    if (q != cudaErrorNotReady) return fail(DOCK_ECUDA, "dock_results: %s", cudaGetErrorString(q));
    const uint64_t el = (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
                            std::chrono::steady_clock::now() - t0).count();
    if (timeout_ns && el > timeout_ns) return fail(DOCK_ETIMEOUT, "dock_results: job still running");
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
  // read on the workspace's own stream: a copy on the legacy default stream
  // would also wait for any search queued there after this job
  Workspace &W = J->L->ws;
  int32_t status = 0;
  CU(cudaMemcpyAsync(&status, W.status, sizeof status, cudaMemcpyDeviceToHost, W.io));
  const int n = std::min(cap, J->n_ligands);
  if (n > 0)
    CU(cudaMemcpyAsync(out, W.results, sizeof(dock_result) * n, cudaMemcpyDeviceToHost, W.io));
  CU(cudaStreamSynchronize(W.io));
  if (status == DOCK_ETIMEOUT) return fail(DOCK_ETIMEOUT, "dock_results: device deadline exceeded");
  if (status <= kCheckBase)
    return fail(DOCK_EDEVICE, "dock_results: bounds check failed at site %d", kCheckBase - status);
  if (status != 0) return fail(DOCK_EDEVICE, "dock_results: device status %d", status);
  return DOCK_OK;
}

extern "C" int dock_job_population(const dock_job *J, const float **genos, const float **scores) {
  if (!J) return fail(DOCK_EINVAL, "dock_job_population: NULL job");
  if (genos) *genos = J->L->ws.geno[J->final_buf];
  if (scores) *scores = J->L->ws.score[J->final_buf];
  return DOCK_OK;
}

// Sum of the device times of the search-kernel launches of a job enqueued with
// DOCK_PROFILE_LAUNCHES set in the environment (waits for the job).
extern "C" int dock_job_kernel_time(const dock_job *J, double *ms_total, int32_t *launches) {
  if (!J) return fail(DOCK_EINVAL, "dock_job_kernel_time: NULL job");
  CU(cudaEventSynchronize(J->done));
  double tot = 0;
  for (size_t i = 0; i + 1 < J->ev.size(); i += 2) {
    float ms = 0;
    CU(cudaEventElapsedTime(&ms, J->ev[i], J->ev[i + 1]));
    tot += ms;
  }
  if (ms_total) *ms_total = tot;
  if (launches) *launches = (int32_t)(J->ev.size() / 2);
  return DOCK_OK;
}

extern "C" void dock_job_destroy(dock_job *J) { delete J; }

// ---------------------------------------------------------------------------
// scoring of given poses
// ---------------------------------------------------------------------------
extern "C" int dock_score(dock_pocket *P, dock_ligands *L, const int32_t *pose_ligand,
                          const float *genos, int64_t n_poses, float *scores, double *scores64,
                          float *coords, int32_t fp64, void *stream) {
  const dk::NvtxRange nvtx_range("dock_score");
  if (!P || !L) return fail(DOCK_EINVAL, "dock_score: NULL pocket or ligands");
  if (n_poses < 0) return fail(DOCK_EINVAL, "dock_score: n_poses < 0");
  if (n_poses == 0) return DOCK_OK;
  if (!pose_ligand || !genos || (fp64 ? !scores64 : !scores))
    return fail(DOCK_EINVAL, "dock_score: NULL device buffer");
  CU(cudaSetDevice(L->device));
  cudaStream_t s = (cudaStream_t)stream;
  if (fp64) {
    Fp64Args F;
    F.ligs = L->d_info;
    F.atoms = L->d_atoms_raw;
    F.types = L->d_types;
    F.pair_idx = L->d_pair_idx;
    F.tors = L->d_tors;
    F.moves = L->d_moves;
    F.grid = grid_view(P);
    F.h = P->h;
    F.cx = P->center[0];
    F.cy = P->center[1];
    F.cz = P->center[2];
    F.params = P->d_params;
    F.pairwise = 0;
    F.pw = pw_view(P);
    CU(launch_score_fp64_impl(F, L->d_centroid, P->ox, P->oy, P->oz, pose_ligand, L->n_ligands, genos,
                              n_poses, scores64, s));
    return DOCK_OK;
  }
  ScoreArgs A;
  A.ligs = L->d_info;
  A.atoms = L->d_atoms;
  A.types = L->d_types;
  A.pair_rec = L->d_pair_rec;
  A.tors = L->d_tors;
  A.moves = L->d_moves;
  A.grid = grid_view(P);
  A.cx = P->center[0];
  A.cy = P->center[1];
  A.cz = P->center[2];
  A.pose_ligand = pose_ligand;
  A.n_ligands = L->n_ligands;
  A.genos = genos;
  A.n_poses = n_poses;
  A.scores = scores;
  A.coords = coords;
  A.lanes = 8;
  A.atoms_per_lane = DOCK_MAX_ATOMS / 8;
  A.bounds = bounds_of(P, L, L->d_check);
  CU(launch_score(A, s));
  return checked_report(L, s, "dock_score");
}

extern "C" int dock_local_search(dock_pocket *P, dock_ligands *L, const dock_ls_params *ls,
                                 uint64_t seed, uint32_t generation, const int32_t *pose_ligand,
                                 int64_t n_poses, float *genos, float *scores, float *trace,
                                 uint32_t *evals, void *stream) {
  const dk::NvtxRange nvtx_range("dock_local_search");
  if (!P || !L || !ls) return fail(DOCK_EINVAL, "dock_local_search: NULL argument");
  if (n_poses < 0) return fail(DOCK_EINVAL, "dock_local_search: n_poses < 0");
  const int st = check_ls_params(ls, "dock_local_search");
  if (st != DOCK_OK) return st;
  if (n_poses > 0xffffffffll) return fail(DOCK_EINVAL, "dock_local_search: n_poses >= 2^32");
  if (n_poses == 0) return DOCK_OK;
  if (!pose_ligand || !genos || !scores)
    return fail(DOCK_EINVAL, "dock_local_search: NULL device buffer");
  CU(cudaSetDevice(L->device));
  cudaStream_t s = (cudaStream_t)stream;
  LsArgs A{};
  A.ligs = L->d_info;
  A.atoms = L->d_atoms;
  A.types = L->d_types;
  A.pair_rec = L->d_pair_rec;
  A.tors = L->d_tors;
  A.moves = L->d_moves;
  A.grid = grid_view(P);
  A.cx = P->center[0];
  A.cy = P->center[1];
  A.cz = P->center[2];
  A.atoms_per_lane = DOCK_MAX_ATOMS / 8;
  A.max_its = ls->max_its;
  A.max_succ = ls->max_succ;
  A.max_fail = ls->max_fail;
  A.rho = ls->rho;
  A.rho_lb = ls->rho_lb;
  A.seed = seed;
  A.gen = generation;
  A.units = nullptr;
  A.pose_ligand = pose_ligand;
  A.n_ligands = L->n_ligands;
  A.n_poses = n_poses;
  A.genos = genos;
  A.scores = scores;
  A.pose_evals = evals;
  A.trace = trace;
  A.bounds = bounds_of(P, L, L->d_check);
  const int threads = 128, lanes = 8;
  int per_sm = 0, n_sm = 0;
  CU(ls_occupancy(threads, lanes, A.atoms_per_lane, &per_sm));
  CU(cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, L->device));
  if (per_sm < 1) return fail(DOCK_EINVAL, "dock_local_search: launch shape does not fit an SM");
  const int64_t need = (n_poses + threads / lanes - 1) / (threads / lanes);
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * n_sm, need));
  CU(launch_ls(A, blocks, threads, lanes, s));
  return checked_report(L, s, "dock_local_search");
}

extern "C" int dock_score_pairwise(dock_pocket *P, dock_ligands *L, const int32_t *pose_ligand,
                                   const float *genos, int64_t n_poses, float *scores, void *stream) {
  const dk::NvtxRange nvtx_range("dock_score_pairwise");
  if (!P || !L) return fail(DOCK_EINVAL, "dock_score_pairwise: NULL pocket or ligands");
  if (n_poses < 0) return fail(DOCK_EINVAL, "dock_score_pairwise: n_poses < 0");
  if (n_poses == 0) return DOCK_OK;
  if (!pose_ligand || !genos || !scores)
    return fail(DOCK_EINVAL, "dock_score_pairwise: NULL device buffer");
  CU(cudaSetDevice(L->device));
  PairwiseArgs A;
  A.ligs = L->d_info;
  A.atoms = L->d_atoms;
  A.types = L->d_types;
  A.pair_rec = L->d_pair_rec;
  A.tors = L->d_tors;
  A.moves = L->d_moves;
  A.cx = P->center[0];
  A.cy = P->center[1];
  A.cz = P->center[2];
  A.pose_ligand = pose_ligand;
  A.n_ligands = L->n_ligands;
  A.genos = genos;
  A.n_poses = n_poses;
  A.scores = scores;
  A.pw = pw_view(P);
  A.bounds = bounds_of(P, L, L->d_check);
  CU(launch_score_pairwise(A, (cudaStream_t)stream));
  return checked_report(L, (cudaStream_t)stream, "dock_score_pairwise");
}

extern "C" int dock_features(dock_pocket *P, dock_ligands *L, const int32_t *pose_ligand,
                             const float *genotypes, int64_t n_poses, uint16_t *features,
                             float *scores, void *stream) {
  const dk::NvtxRange nvtx_range("dock_features");
  if (!P || !L) return fail(DOCK_EINVAL, "dock_features: NULL pocket or ligands");
  if (n_poses < 0) return fail(DOCK_EINVAL, "dock_features: n_poses < 0");
  if (n_poses == 0) return DOCK_OK;
  if (!pose_ligand || !genotypes || !features) return fail(DOCK_EINVAL, "dock_features: NULL buffer");
  CU(cudaSetDevice(L->device));
  FeatureLaunch F{};
  F.ligs = L->d_info;
  F.atoms = L->d_atoms;
  F.types = L->d_types;
  F.pair_rec = L->d_pair_rec;
  F.tors = L->d_tors;
  F.moves = L->d_moves;
  F.grid = grid_view(P);
  F.cx = P->center[0];
  F.cy = P->center[1];
  F.cz = P->center[2];
  F.radius = P->radius;
  F.n_ligands = L->n_ligands;
  F.from_ga = false;
  F.pose_ligand = pose_ligand;
  F.genos = genotypes;
  F.n_poses = n_poses;
  F.scores = scores;
  F.features = features;
  CU(launch_features(F, (cudaStream_t)stream));
  return DOCK_OK;
}

extern "C" int dock_features_population(dock_pocket *P, dock_ligands *L, int32_t pop,
                                        const float *genotypes, uint16_t *features, float *scores,
                                        void *stream) {
  if (!P || !L || !genotypes || !features)
    return fail(DOCK_EINVAL, "dock_features_population: NULL argument");
  if (pop < 1 || pop > DOCK_MAX_POP) return fail(DOCK_EINVAL, "dock_features_population: pop %d", pop);
  CU(cudaSetDevice(L->device));
  cudaStream_t s = (cudaStream_t)stream;
  const int nl = L->n_ligands;
  if (nl == 0) return DOCK_OK;
  std::vector<int64_t> goff((size_t)nl);
  int64_t tot = 0;
  for (int l = 0; l < nl; ++l) {
    goff[l] = tot;
    tot += (int64_t)pop * (7 + L->info[l].k);
  }
  Workspace &W = L->ws;
  if ((size_t)nl > W.feat_off_cap || !W.feat_off) {
    dfree(W.feat_off);
    W.feat_off_cap = 0;
    CU(dalloc(&W.feat_off, (size_t)nl));
    W.feat_off_cap = (size_t)nl;
  }
  CU(cudaMemcpyAsync(W.feat_off, goff.data(), sizeof(int64_t) * nl, cudaMemcpyHostToDevice, s));
  FeatureLaunch F{};
  F.ligs = L->d_info;
  F.atoms = L->d_atoms;
  F.types = L->d_types;
  F.pair_rec = L->d_pair_rec;
  F.tors = L->d_tors;
  F.moves = L->d_moves;
  F.grid = grid_view(P);
  F.cx = P->center[0];
  F.cy = P->center[1];
  F.cz = P->center[2];
  F.radius = P->radius;
  F.n_ligands = nl;
  F.from_ga = false;
  F.pop_csr = pop;
  F.genos = genotypes;
  F.geno_off = W.feat_off;
  F.n_poses = (int64_t)nl * pop;
  F.scores = scores;
  F.features = features;
  CU(launch_features(F, s));
  // the offsets buffer is reused by later calls: finish before returning
  CU(cudaStreamSynchronize(s));
  return DOCK_OK;
}

// ---------------------------------------------------------------------------
// autotuner
// ---------------------------------------------------------------------------
extern "C" int dock_autotune(dock_pocket *P, dock_ligands *L, const dock_search_params *sp,
                             void *stream, dock_tune_table *table) {
  const dk::NvtxRange nvtx_range("dock_autotune");
  if (!P || !L || !sp || !table) return fail(DOCK_EINVAL, "dock_autotune: NULL argument");
  if (sp->mode != DOCK_MODE_PLAIN || sp->lanes_per_pose != 0)
    return fail(DOCK_EINVAL, "dock_autotune: tunes the plain search with lanes_per_pose = 0");
  CU(cudaSetDevice(L->device));
  // candidate shapes: CTA threads x shared-memory atoms per lane
  static const int kThreads[] = {64, 128};
  static const int kApl[] = {8, 12, 16, 24, 32};
  dock_tune_table T;
  memset(&T, 0, sizeof T);
  const int old_t = L->tuned_threads, old_a = L->tuned_apl;
  dock_search_params q = *sp;
  q.generations = std::min(std::max(sp->generations, 2), 4);
  q.use_graph = 0;
  q.trace_genotypes = nullptr;
  q.trace_scores = nullptr;
  q.timeout_ns = 0;
  q.ls.rate = 0.0f;  // the launch shape of the search kernel alone (grid or pairwise inter)
  q.trace_ls = nullptr;
  for (int ti = 0; ti < 2; ++ti)
    for (int ai = 0; ai < 5; ++ai) {
      const int apl = kApl[ai], thr = kThreads[ti];
      if (8 * apl < L->max_atoms || search_smem_bytes(thr, apl) > 200 * 1024) continue;
      L->tuned_threads = thr;
      L->tuned_apl = apl;
      L->profiling = true;
      // time generations >= 1 (GA steps) of a short search, best of two runs
      double best = 1e30;
      for (int rep = 0; rep < 2; ++rep) {
        dock_job *J = nullptr;
        L->profiling = true;
        int st = dock_batch(P, L, &q, stream, &J);
        if (st != DOCK_OK) {
          L->profiling = false;
          L->tuned_threads = old_t;
          L->tuned_apl = old_a;
          return st;
        }
        double ms = 0;
        int32_t n = 0;
        st = dock_job_kernel_time(J, &ms, &n);
        dock_job_destroy(J);
        L->profiling = false;
        if (st != DOCK_OK) {
          L->tuned_threads = old_t;
          L->tuned_apl = old_a;
          return st;
        }
        if (n > 0) best = std::min(best, ms / n);
      }
      if (T.n < DOCK_TUNE_MAX) {
        T.threads[T.n] = thr;
        T.atoms_per_lane[T.n] = apl;
        T.ms_per_generation[T.n] = (float)best;
        ++T.n;
      }
    }
  L->tuned_threads = old_t;
  L->tuned_apl = old_a;
  if (T.n == 0) return fail(DOCK_EINVAL, "dock_autotune: no launch shape fits these ligands");
  // the pick: fastest measured shape, ties to the earlier entry
  T.best = 0;
  for (int i = 1; i < T.n; ++i)
    if (T.ms_per_generation[i] < T.ms_per_generation[T.best]) T.best = i;
  L->tuned_threads = T.threads[T.best];
  L->tuned_apl = T.atoms_per_lane[T.best];
  *table = T;
  return DOCK_OK;
}
