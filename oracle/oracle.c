/*
 * Plain FP64 CPU oracle for the muDock docking hot path.
 *
 * TEST INFRASTRUCTURE ONLY. Tests, the package's smoke check and the
 * benchmark's CPU-baseline leg may call this code; the CUDA product path
 * never does. It shares no code, header or table with the CUDA library.
 *
 * What it computes, in the paper's order:
 *   Algorithm 1 (Section V): translate and rotate the ligand, then rotate the
 *     fragment below each rotatable bond.
 *   Algorithm 2 (Section V): score = inter-energy (per ligand atom, lookup in
 *     the per-atom-type grid maps built "as AutoGrid does") + intra-energy
 *     (per ligand atom pair) with electrostatic, van der Waals, hydrogen-bond
 *     and desolvation terms.
 *   Section V: a genetic algorithm without local search proposes the poses.
 *   Optionally, the Lamarckian variant of AutoDock's search that the paper
 *   leaves out: Solis-Wets local search on a share of each generation.
 * The paper prints no formulas or constants. The energy terms follow the
 * AutoDock4 free-energy function the paper names as its equivalent
 * (Section V, citing AutoDock4): 12-6 dispersion/repulsion, 12-10 hydrogen
 * bond, Coulomb with the Mehler-Solmajer distance-dependent dielectric, and
 * Gaussian charge-dependent desolvation. The GA operators are a reading of
 * "similar to the genetic algorithm used by AutoDock".
 *
 * Floating point: energies, poses and grids are FP64. The GA works on FP32
 * genotypes with only correctly rounded single-precision operations (the
 * paper fixes the precision to float, Section VII "Software"), so it is
 * written in float here; compile with -ffp-contract=off.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- AutoDock4 free-energy constants (force-field literature) ---------- */
#define W_VDW 0.1662
#define W_HB 0.1209
#define W_ELEC 0.1406
#define W_SOL 0.1322
#define COULOMB 332.06363
#define QASP 0.01097
#define SIGMA_SOL 3.6
#define DIEL_A (-8.5525)
#define DIEL_EPS0 78.4
#define DIEL_K 7.7839
#define DIEL_LAMBDA 0.003627
/* ---- readings of what the paper leaves open ---------------------------- */
#define CUTOFF 8.0   /* non-bonded cutoff, Angstrom                        */
#define RMIN 0.5     /* distances floored here                              */
#define EMAX 1.0e5   /* cap on a pair's raw 12-6 / 12-10 value and on M_t   */
#define EOUT 1000.0  /* energy of a ligand atom outside the grid box        */
#define HB_DONOR 1
#define HB_ACCEPTOR 2

typedef struct {
  int32_t n_types;
  const float *Rii, *eps, *vol, *solpar, *hb_R, *hb_eps;
  const int32_t *hb_role;
} orc_params;

typedef struct {
  int32_t n;
  const float *x, *y, *z, *q;
  const uint8_t *type;
  const int16_t *parent;
  int32_t k;
  const int16_t *tors_b;
} orc_ligand;

typedef struct {
  int32_t n_atoms;
  const float *x, *y, *z, *q;
  const uint8_t *type;
  double center[3];
  double radius, spacing;
} orc_pocket;

typedef struct {
  int32_t nx, ny, nz, n_types;
  double ox, oy, oz, h;
  double *maps; /* [n_types + 2][nz][ny][nx]: M_0..M_{T-1}, E, D */
} orc_grid;

/* ======================================================================= */
/* Energy terms of one atom pair                                           */
/* ======================================================================= */

/* Mehler-Solmajer sigmoidal dielectric eps(r) = A + B / (1 + k exp(-lambda B r)),
 * B = eps0 - A. */
double orc_dielectric(double r) {
  const double B = DIEL_EPS0 - DIEL_A;
  return DIEL_A + B / (1.0 + DIEL_K * exp(-DIEL_LAMBDA * B * r));
}

static int is_hb_pair(const orc_params *p, int ti, int tj) {
  return (p->hb_role[ti] == HB_DONOR && p->hb_role[tj] == HB_ACCEPTOR) ||
         (p->hb_role[ti] == HB_ACCEPTOR && p->hb_role[tj] == HB_DONOR);
}

static double ipow(double x, int n) {
  double r = 1.0;
  for (int i = 0; i < n; ++i) r *= x;
  return r;
}

/* Raw (unweighted, uncapped) dispersion-repulsion of a pair at distance r:
 * 12-10 for a donor-acceptor pair (well -eps_hb at hb_R of the acceptor),
 * else 12-6 (well -eps_ij at R_ij = (Rii + Rjj)/2, eps_ij = sqrt(eps_i eps_j)). */
double orc_disp_raw(const orc_params *p, int ti, int tj, double r) {
  if (is_hb_pair(p, ti, tj)) {
    int acc = p->hb_role[ti] == HB_ACCEPTOR ? ti : tj;
    double R = p->hb_R[acc], e = p->hb_eps[acc];
    double s = R / r;
    return 5.0 * e * ipow(s, 12) - 6.0 * e * ipow(s, 10);
  } else {
    double R = 0.5 * ((double)p->Rii[ti] + (double)p->Rii[tj]);
    double e = sqrt((double)p->eps[ti] * (double)p->eps[tj]);
    double s = R / r;
    return e * ipow(s, 12) - 2.0 * e * ipow(s, 6);
  }
}

/* The four weighted terms of a ligand-ligand or ligand-protein pair:
 * out[0] dispersion-repulsion / H-bond, out[1] electrostatic, out[2]
 * desolvation, out[3] their sum. Zero at r >= CUTOFF; r floored at RMIN. */
void orc_pair_terms(const orc_params *p, int ti, int tj, double qi, double qj, double r,
                    double out[4]) {
  out[0] = out[1] = out[2] = out[3] = 0.0;
  if (!(r < CUTOFF)) return;
  if (r < RMIN) r = RMIN;
  double w = is_hb_pair(p, ti, tj) ? W_HB : W_VDW;
  double raw = orc_disp_raw(p, ti, tj, r);
  if (raw > EMAX) raw = EMAX;
  out[0] = w * raw;
  out[1] = W_ELEC * COULOMB * qi * qj / (orc_dielectric(r) * r);
  double si = (double)p->solpar[ti] + QASP * fabs(qi);
  double sj = (double)p->solpar[tj] + QASP * fabs(qj);
  out[2] = W_SOL * (si * (double)p->vol[tj] + sj * (double)p->vol[ti]) *
           exp(-r * r / (2.0 * SIGMA_SOL * SIGMA_SOL));
  out[3] = out[0] + out[1] + out[2];
}

/* ======================================================================= */
/* Ligand topology: fragments moved by each torsion, included intra pairs   */
/* ======================================================================= */

/* 1 if atom i lies in the subtree rooted at b (i != b), walking parents. */
static int below(const int16_t *parent, int i, int b) {
  for (int a = parent[i]; a >= 0; a = parent[a])
    if (a == b) return 1;
  return 0;
}

/* moves[j*n + i] = 1 if torsion j (bond parent[b_j] -> b_j) moves atom i.
 * pairs: included intra pairs (i < j): more than three bonds apart and not
 * in the same rigid fragment (no rotatable bond on the path). Returns the
 * number of pairs, or -1 on bad topology. */
int orc_topology(const orc_ligand *L, uint8_t *moves, int32_t *pairs) {
  int n = L->n, k = L->k;
  for (int i = 0; i < n; ++i) {
    int pa = L->parent[i];
    if ((i == 0 && pa != -1) || (i > 0 && (pa < 0 || pa >= i))) return -1;
  }
  for (int j = 0; j < k; ++j) {
    int b = L->tors_b[j];
    if (b <= 0 || b >= n) return -1;
    if (j > 0 && L->tors_b[j - 1] >= b) return -1;
    for (int i = 0; i < n; ++i) moves[j * n + i] = (uint8_t)below(L->parent, i, b);
  }
  /* rotatable flag per child atom */
  uint8_t *rot = (uint8_t *)calloc((size_t)n, 1);
  for (int j = 0; j < k; ++j) rot[L->tors_b[j]] = 1;
  /* bond distance and rotatable-on-path via the tree path through the
   * lowest common ancestor */
  int *depth = (int *)malloc(sizeof(int) * (size_t)n);
  for (int i = 0; i < n; ++i) depth[i] = i == 0 ? 0 : depth[L->parent[i]] + 1;
  int np = 0;
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      int a = i, b = j, d = 0, crosses = 0;
      while (a != b) {
        if (depth[a] >= depth[b]) {
          crosses |= rot[a];
          a = L->parent[a];
        } else {
          crosses |= rot[b];
          b = L->parent[b];
        }
        ++d;
      }
      if (d > 3 && crosses) {
        pairs[2 * np] = i;
        pairs[2 * np + 1] = j;
        ++np;
      }
    }
  free(rot);
  free(depth);
  return np;
}

/* ======================================================================= */
/* Pose (Algorithm 1)                                                       */
/* ======================================================================= */

/* Rotation matrix of the unit quaternion q = (w, x, y, z) (normalised here). */
void orc_quat_matrix(const double q_in[4], double R[9]) {
  double n = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
  double w = q_in[0] / n, x = q_in[1] / n, y = q_in[2] / n, z = q_in[3] / n;
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* Rotate point v about the axis through a with unit direction u by theta
 * (right-hand rule), Rodrigues' formula. */
static void rodrigues(const double a[3], const double u[3], double c, double s, double v[3]) {
  double p[3] = {v[0] - a[0], v[1] - a[1], v[2] - a[2]};
  double d = u[0] * p[0] + u[1] * p[1] + u[2] * p[2];
  double cr[3] = {u[1] * p[2] - u[2] * p[1], u[2] * p[0] - u[0] * p[2], u[0] * p[1] - u[1] * p[0]};
  for (int m = 0; m < 3; ++m) v[m] = a[m] + p[m] * c + cr[m] * s + u[m] * d * (1.0 - c);
}

static void apply_torsion(const orc_ligand *L, const uint8_t *moves, int j, double theta,
                          double *xyz) {
  int n = L->n, b = L->tors_b[j], a = L->parent[b];
  double pa[3] = {xyz[3 * a], xyz[3 * a + 1], xyz[3 * a + 2]};
  double u[3] = {xyz[3 * b] - pa[0], xyz[3 * b + 1] - pa[1], xyz[3 * b + 2] - pa[2]};
  double len = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  u[0] /= len; u[1] /= len; u[2] /= len;
  double c = cos(theta), s = sin(theta);
  for (int i = 0; i < n; ++i)
    if (moves[j * n + i]) rodrigues(pa, u, c, s, &xyz[3 * i]);
}

/* Posed coordinates xyz[3n] of genotype g = [t(3), q(4), theta(k)].
 * The input coordinates are taken about their centroid c_lig:
 * rigid x' = R(q)(x - c_lig) + center + t. order 0: rigid motion, then the
 * torsions root to leaf on the current coordinates (Algorithm 1's order);
 * 1: torsions root to leaf on the input frame, then the rigid motion;
 * 2: torsions leaf to root on the input frame, then the rigid motion. */
void orc_pose(const orc_ligand *L, const uint8_t *moves, const float *g, const double center[3],
              int order, double *xyz) {
  int n = L->n;
  double c[3] = {0, 0, 0};
  for (int i = 0; i < n; ++i) { c[0] += L->x[i]; c[1] += L->y[i]; c[2] += L->z[i]; }
  c[0] /= n; c[1] /= n; c[2] /= n;
  double q[4] = {g[3], g[4], g[5], g[6]}, R[9];
  orc_quat_matrix(q, R);
  double t[3] = {center[0] + g[0], center[1] + g[1], center[2] + g[2]};
  for (int i = 0; i < n; ++i) {
    xyz[3 * i] = L->x[i] - c[0];
    xyz[3 * i + 1] = L->y[i] - c[1];
    xyz[3 * i + 2] = L->z[i] - c[2];
  }
  if (order == 1)
    for (int j = 0; j < L->k; ++j) apply_torsion(L, moves, j, g[7 + j], xyz);
  if (order == 2)
    for (int j = L->k - 1; j >= 0; --j) apply_torsion(L, moves, j, g[7 + j], xyz);
  for (int i = 0; i < n; ++i) {
    double v[3] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
    for (int m = 0; m < 3; ++m)
      xyz[3 * i + m] = R[3 * m] * v[0] + R[3 * m + 1] * v[1] + R[3 * m + 2] * v[2] + t[m];
  }
  if (order == 0)
    for (int j = 0; j < L->k; ++j) apply_torsion(L, moves, j, g[7 + j], xyz);
}

/* ======================================================================= */
/* Scoring (Algorithm 2)                                                    */
/* ======================================================================= */

/* Intra-energy: sum of the pair terms over the included pairs.
 * *margin (if given) = min over included pairs of |r - CUTOFF|. */
double orc_intra(const orc_ligand *L, const orc_params *p, const int32_t *pairs, int np,
                 const double *xyz, double *margin) {
  double e = 0.0, m = INFINITY, t[4];
  for (int s = 0; s < np; ++s) {
    int i = pairs[2 * s], j = pairs[2 * s + 1];
    double dx = xyz[3 * i] - xyz[3 * j], dy = xyz[3 * i + 1] - xyz[3 * j + 1],
           dz = xyz[3 * i + 2] - xyz[3 * j + 2];
    double r = sqrt(dx * dx + dy * dy + dz * dz);
    orc_pair_terms(p, L->type[i], L->type[j], L->q[i], L->q[j], r, t);
    e += t[3];
    if (fabs(r - CUTOFF) < m) m = fabs(r - CUTOFF);
  }
  if (margin) *margin = m;
  return e;
}

/* Inter-energy, pairwise form: every ligand atom against every protein atom. */
double orc_inter_pairwise(const orc_ligand *L, const orc_params *p, const orc_pocket *P,
                          const double *xyz) {
  double e = 0.0, t[4];
  for (int i = 0; i < L->n; ++i)
    for (int j = 0; j < P->n_atoms; ++j) {
      double dx = xyz[3 * i] - P->x[j], dy = xyz[3 * i + 1] - P->y[j], dz = xyz[3 * i + 2] - P->z[j];
      double r = sqrt(dx * dx + dy * dy + dz * dz);
      orc_pair_terms(p, L->type[i], P->type[j], L->q[i], P->q[j], r, t);
      e += t[3];
    }
  return e;
}

/* Grid geometry: n = floor(2R/h) + 1 nodes per axis, centred on the pocket. */
void orc_grid_geometry(const orc_pocket *P, int32_t n_types, orc_grid *G) {
  int n = (int)floor(2.0 * P->radius / P->spacing + 1e-9) + 1;
  G->nx = G->ny = G->nz = n;
  G->n_types = n_types;
  G->h = P->spacing;
  double half = 0.5 * (n - 1) * P->spacing;
  G->ox = P->center[0] - half;
  G->oy = P->center[1] - half;
  G->oz = P->center[2] - half;
}

/* Value of every map at node p: for a probe of type t, charge q,
 * inter(p) = M_t(p) + q E(p) + |q| D(p), with
 *   M_t = sum_j w min(disp_raw, EMAX) + W_SOL (solpar_t V_j + S_j V_t) g(r)
 *   E   = sum_j W_ELEC COULOMB q_j / (eps(r) r)
 *   D   = sum_j W_SOL QASP V_j g(r),       g(r) = exp(-r^2 / 2 sigma^2),
 * which splits the pair terms exactly; M_t is then capped at EMAX. */
static void grid_node(const orc_pocket *P, const orc_params *p, int T, double px, double py,
                      double pz, double *vals) {
  for (int t = 0; t < T + 2; ++t) vals[t] = 0.0;
  for (int j = 0; j < P->n_atoms; ++j) {
    double dx = px - P->x[j], dy = py - P->y[j], dz = pz - P->z[j];
    double r = sqrt(dx * dx + dy * dy + dz * dz);
    if (!(r < CUTOFF)) continue;
    if (r < RMIN) r = RMIN;
    int tj = P->type[j];
    double qj = P->q[j];
    double g = exp(-r * r / (2.0 * SIGMA_SOL * SIGMA_SOL));
    double sj = (double)p->solpar[tj] + QASP * fabs(qj);
    for (int t = 0; t < T; ++t) {
      double w = is_hb_pair(p, t, tj) ? W_HB : W_VDW;
      double raw = orc_disp_raw(p, t, tj, r);
      if (raw > EMAX) raw = EMAX;
      vals[t] += w * raw + W_SOL * ((double)p->solpar[t] * p->vol[tj] + sj * p->vol[t]) * g;
    }
    vals[T] += W_ELEC * COULOMB * qj / (orc_dielectric(r) * r);
    vals[T + 1] += W_SOL * QASP * (double)p->vol[tj] * g;
  }
  for (int t = 0; t < T; ++t)
    if (vals[t] > EMAX) vals[t] = EMAX;
}

typedef struct {
  const orc_pocket *P;
  const orc_params *p;
  orc_grid *G;
  int z0, z1;
} grid_job;

static void *grid_worker(void *arg) {
  grid_job *J = (grid_job *)arg;
  orc_grid *G = J->G;
  int T = G->n_types;
  size_t plane = (size_t)G->nx * G->ny, vol = plane * G->nz;
  double vals[64];
  for (int k = J->z0; k < J->z1; ++k)
    for (int jy = 0; jy < G->ny; ++jy)
      for (int i = 0; i < G->nx; ++i) {
        grid_node(J->P, J->p, T, G->ox + i * G->h, G->oy + jy * G->h, G->oz + k * G->h, vals);
        size_t node = (size_t)k * plane + (size_t)jy * G->nx + i;
        for (int t = 0; t < T + 2; ++t) G->maps[(size_t)t * vol + node] = vals[t];
      }
  return NULL;
}

/* Build all maps (G->maps must hold (T+2)*nx*ny*nz doubles). */
void orc_grid_build(const orc_pocket *P, const orc_params *p, orc_grid *G, int n_threads) {
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  pthread_t th[256];
  grid_job jobs[256];
  for (int t = 0; t < n_threads; ++t) {
    jobs[t].P = P; jobs[t].p = p; jobs[t].G = G;
    jobs[t].z0 = (int)((long)G->nz * t / n_threads);
    jobs[t].z1 = (int)((long)G->nz * (t + 1) / n_threads);
    pthread_create(&th[t], NULL, grid_worker, &jobs[t]);
  }
  for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
}

/* Trilinear interpolation of one map at (x, y, z). Returns 0 and sets *v
 * when inside the box [o, o + (n-1) h] on every axis (faces included), else
 * returns 1. The cell index is clamped to n-2 so the far face is inside. */
int orc_trilinear(const orc_grid *G, const double *map, double x, double y, double z, double *v) {
  double u[3] = {(x - G->ox) / G->h, (y - G->oy) / G->h, (z - G->oz) / G->h};
  int n[3] = {G->nx, G->ny, G->nz}, i0[3];
  double f[3];
  for (int m = 0; m < 3; ++m) {
    if (!(u[m] >= 0.0 && u[m] <= (double)(n[m] - 1))) return 1;
    i0[m] = (int)floor(u[m]);
    if (i0[m] > n[m] - 2) i0[m] = n[m] - 2;
    f[m] = u[m] - i0[m];
  }
  double acc = 0.0;
  for (int dz = 0; dz < 2; ++dz)
    for (int dy = 0; dy < 2; ++dy)
      for (int dx = 0; dx < 2; ++dx) {
        double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
        size_t node = ((size_t)(i0[2] + dz) * G->ny + (i0[1] + dy)) * G->nx + (i0[0] + dx);
        acc += w * map[node];
      }
  *v = acc;
  return 0;
}

/* Inter-energy by grid lookup ("nearby" = inside the grid box):
 * M_t + q E + |q| D per inside atom, EOUT per outside atom.
 * *margin (if given) = min distance of any atom to a box face. */
double orc_inter_grid(const orc_ligand *L, const orc_grid *G, const double *xyz, double *margin) {
  size_t vol = (size_t)G->nx * G->ny * G->nz;
  int T = G->n_types;
  double e = 0.0, m = INFINITY;
  double lo[3] = {G->ox, G->oy, G->oz};
  double hi[3] = {G->ox + (G->nx - 1) * G->h, G->oy + (G->ny - 1) * G->h, G->oz + (G->nz - 1) * G->h};
  for (int i = 0; i < L->n; ++i) {
    const double *x = &xyz[3 * i];
    for (int a = 0; a < 3; ++a) {
      if (fabs(x[a] - lo[a]) < m) m = fabs(x[a] - lo[a]);
      if (fabs(x[a] - hi[a]) < m) m = fabs(x[a] - hi[a]);
    }
    double vm, ve, vd;
    if (orc_trilinear(G, G->maps + (size_t)L->type[i] * vol, x[0], x[1], x[2], &vm)) {
      e += EOUT;
      continue;
    }
    orc_trilinear(G, G->maps + (size_t)T * vol, x[0], x[1], x[2], &ve);
    orc_trilinear(G, G->maps + (size_t)(T + 1) * vol, x[0], x[1], x[2], &vd);
    double q = L->q[i];
    e += vm + q * ve + fabs(q) * vd;
  }
  if (margin) *margin = m;
  return e;
}

/* Score many poses of one ligand (grid form). Any output may be NULL.
 * inter/intra/margin are per pose; xyz is [n_poses][n][3]. Returns the
 * number of included pairs, or -1 on bad topology. */
int orc_score_poses(const orc_ligand *L, const orc_params *p, const orc_grid *G,
                    const double center[3], const float *genos, int n_genes, int64_t n_poses,
                    double *score, double *inter, double *intra, double *margin, double *xyz_out) {
  int n = L->n;
  uint8_t *moves = (uint8_t *)malloc((size_t)(L->k > 0 ? L->k : 1) * n);
  int32_t *pairs = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n * (n - 1) + 2));
  double *xyz = (double *)malloc(sizeof(double) * 3 * (size_t)n);
  int np = orc_topology(L, moves, pairs);
  if (np >= 0)
    for (int64_t s = 0; s < n_poses; ++s) {
      orc_pose(L, moves, genos + s * n_genes, center, 0, xyz);
      double m1, m2;
      double ei = orc_inter_grid(L, G, xyz, &m1);
      double ea = orc_intra(L, p, pairs, np, xyz, &m2);
      if (score) score[s] = ei + ea;
      if (inter) inter[s] = ei;
      if (intra) intra[s] = ea;
      if (margin) margin[s] = m1 < m2 ? m1 : m2;
      if (xyz_out) memcpy(xyz_out + s * 3 * n, xyz, sizeof(double) * 3 * n);
    }
  free(moves);
  free(pairs);
  free(xyz);
  return np;
}

/* ======================================================================= */
/* Counter-based RNG: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11)      */
/* ======================================================================= */
static void mulhilo64(uint64_t a, uint64_t b, uint64_t *hi, uint64_t *lo) {
  __uint128_t p = (__uint128_t)a * b;
  *hi = (uint64_t)(p >> 64);
  *lo = (uint64_t)p;
}

void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3], k0 = key[0], k1 = key[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t hi0, lo0, hi1, lo1;
    mulhilo64(0xD2E7470EE14C6C93ULL, c0, &hi0, &lo0);
    mulhilo64(0xCA5A826395121157ULL, c2, &hi1, &lo1);
    uint64_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    k0 += 0x9E3779B97F4A7C15ULL;
    k1 += 0xBB67AE8584CAA73BULL;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Eight 32-bit words of one block: counter (slot, individual, generation,
 * ligand id), key (seed, 0); word 2i is the low half of output i. */
void orc_rng_words(uint64_t seed, uint64_t lig, uint32_t gen, uint32_t ind, uint32_t slot,
                   uint32_t w[8]) {
  uint64_t ctr[4] = {slot, ind, gen, lig}, key[2] = {seed, 0}, o[4];
  orc_philox4x64(ctr, key, o);
  for (int i = 0; i < 4; ++i) {
    w[2 * i] = (uint32_t)o[i];
    w[2 * i + 1] = (uint32_t)(o[i] >> 32);
  }
}

/* Irwin-Hall normal deviate from the first 12 words of slots (s, s+1):
 * z = (sum of the top 24 bits of each word - 6 * 2^24) * 2^-24. */
float orc_normal(uint64_t seed, uint64_t lig, uint32_t gen, uint32_t ind, uint32_t s) {
  uint32_t a[8], b[8];
  orc_rng_words(seed, lig, gen, ind, s, a);
  orc_rng_words(seed, lig, gen, ind, s + 1, b);
  int64_t S = 0;
  for (int i = 0; i < 8; ++i) S += a[i] >> 8;
  for (int i = 0; i < 4; ++i) S += b[i] >> 8;
  float z = (float)(S - 6 * (int64_t)16777216);
  return z * 0x1p-24f;
}

static float u24(uint32_t w) { return (float)(w >> 8) * 0x1p-24f; }

/* ======================================================================= */
/* Genetic algorithm (reading of "similar to AutoDock's GA", Section V)     */
/* All genotype arithmetic is correctly rounded FP32.                        */
/* ======================================================================= */
#define PI_F 3.14159265358979323846f
#define TWO_PI_F 6.28318530717958647692f

static uint64_t prob_threshold(float p) {
  double t = (double)p * 4294967296.0;
  if (t < 0) t = 0;
  if (t > 4294967296.0) t = 4294967296.0;
  return (uint64_t)t;
}

static void quat_normalize(float *q) {
  float n2 = q[0] * q[0];
  n2 = n2 + q[1] * q[1];
  n2 = n2 + q[2] * q[2];
  n2 = n2 + q[3] * q[3];
  float n = sqrtf(n2);
  if (!(n > 0.0f)) {
    q[0] = 1.0f; q[1] = q[2] = q[3] = 0.0f;
    return;
  }
  for (int m = 0; m < 4; ++m) q[m] = q[m] / n;
}

/* Generation 0: translation uniform in [-R/2, R/2)^3 around the pocket
 * centre (slot 0), quaternion of four normals normalised (slots 1..8),
 * torsions uniform in [-pi, pi) (slots 9, 10). */
void orc_ga_init(int k, int P, float radius, uint64_t seed, uint64_t lig, float *geno) {
  int G = 7 + k;
  float half = 0.5f * radius;
  for (int i = 0; i < P; ++i) {
    float *g = geno + (size_t)i * G;
    uint32_t w[8];
    orc_rng_words(seed, lig, 0, (uint32_t)i, 0, w);
    for (int m = 0; m < 3; ++m) {
      float t = u24(w[m]) * radius;
      g[m] = t - half;
    }
    for (int m = 0; m < 4; ++m) g[3 + m] = orc_normal(seed, lig, 0, (uint32_t)i, 1 + 2 * m);
    quat_normalize(g + 3);
    for (int j = 0; j < k; ++j) {
      orc_rng_words(seed, lig, 0, (uint32_t)i, 9 + j / 8, w);
      float t = u24(w[j % 8]) * TWO_PI_F;
      g[7 + j] = t - PI_F;
    }
  }
}

static int better(const float *s, int a, int b) {
  float sa = s[a] != s[a] ? INFINITY : s[a];
  float sb = s[b] != s[b] ? INFINITY : s[b];
  return sa < sb || (sa == sb && a < b);
}

/* Block index of gene g: translation x, y, z are blocks 0-2, the quaternion
 * is block 3, torsion j is block 4 + j. */
static int gene_block(int g) { return g < 3 ? g : (g < 7 ? 3 : g - 3); }

/* One generation: individual 0 is the best of the previous generation
 * (elitism 1); individual i >= 1 = tournament(2) winners A, B -> two-point
 * crossover on blocks with probability p_cross -> per-gene mutation with
 * probability p_mut, adding sigma * N(0,1) (1 A, 0.1, 0.5 rad). */
/* Child `ind` of the population `prev` (scores `score`): tournaments A, B,
 * crossover, mutation, as described above. */
static void ga_child_one(int k, int P, uint64_t tc, uint64_t tm, uint64_t seed, uint64_t lig,
                         uint32_t gen, uint32_t ind, const float *prev, const float *score,
                         float *c) {
  int G = 7 + k, B = 4 + k;
  uint32_t w[8];
  orc_rng_words(seed, lig, gen, ind, 0, w);
  int a1 = (int)(((uint64_t)w[0] * (uint64_t)P) >> 32), a2 = (int)(((uint64_t)w[1] * (uint64_t)P) >> 32);
  int b1 = (int)(((uint64_t)w[2] * (uint64_t)P) >> 32), b2 = (int)(((uint64_t)w[3] * (uint64_t)P) >> 32);
  int pa = better(score, a1, a2) ? a1 : a2;
  int pb = better(score, b1, b2) ? b1 : b2;
  int lo = 0, hi = 0;
  if ((uint64_t)w[4] < tc) {
    int c1 = (int)(((uint64_t)w[5] * (uint64_t)(B + 1)) >> 32);
    int c2 = (int)(((uint64_t)w[6] * (uint64_t)(B + 1)) >> 32);
    lo = c1 < c2 ? c1 : c2;
    hi = c1 < c2 ? c2 : c1;
  }
  for (int g = 0; g < G; ++g) {
    int blk = gene_block(g);
    c[g] = (blk >= lo && blk < hi) ? prev[(size_t)pb * G + g] : prev[(size_t)pa * G + g];
  }
  int qmut = 0;
  for (int g = 0; g < G; ++g) {
    uint32_t m[8];
    orc_rng_words(seed, lig, gen, ind, 1 + g / 8, m);
    if ((uint64_t)m[g % 8] >= tm) continue;
    float z = orc_normal(seed, lig, gen, ind, 4 + 2 * g);
    float sigma = g < 3 ? 1.0f : (g < 7 ? 0.1f : 0.5f);
    float d = sigma * z;
    c[g] = c[g] + d;
    if (g >= 3 && g < 7) qmut = 1;
    if (g >= 7) {
      if (c[g] > PI_F) c[g] = c[g] - TWO_PI_F;
      else if (c[g] < -PI_F) c[g] = c[g] + TWO_PI_F;
    }
  }
  if (qmut) quat_normalize(c + 3);
}

/* One generation: individual 0 is the best of the previous generation
 * (elitism 1); individual i >= 1 = tournament(2) winners A, B -> two-point
 * crossover on blocks with probability p_cross -> per-gene mutation with
 * probability p_mut, adding sigma * N(0,1) (1 A, 0.1, 0.5 rad). */
void orc_ga_step(int k, int P, float p_cross, float p_mut, uint64_t seed, uint64_t lig,
                 uint32_t gen, const float *prev, const float *score, float *next) {
  int G = 7 + k;
  uint64_t tc = prob_threshold(p_cross), tm = prob_threshold(p_mut);
  int best = 0;
  for (int i = 1; i < P; ++i)
    if (better(score, i, best)) best = i;
  memcpy(next, prev + (size_t)best * G, sizeof(float) * G);
  for (int i = 1; i < P; ++i)
    ga_child_one(k, P, tc, tm, seed, lig, gen, (uint32_t)i, prev, score, next + (size_t)i * G);
}

/* n children 0..n-1 of a population (candidates of the pre-screened search;
 * child c uses the counters of individual c). */
void orc_ga_children(int k, int P, int n, float p_cross, float p_mut, uint64_t seed, uint64_t lig,
                     uint32_t gen, const float *prev, const float *score, float *out) {
  uint64_t tc = prob_threshold(p_cross), tm = prob_threshold(p_mut);
  for (int c = 0; c < n; ++c)
    ga_child_one(k, P, tc, tm, seed, lig, gen, (uint32_t)c, prev, score, out + (size_t)c * (7 + k));
}

/* ======================================================================= */
/* Solis-Wets local search: the Lamarckian variant of the GA. The paper's   */
/* search has none (Section V); AutoDock's Lamarckian GA (Morris et al.      */
/* 1998, in the paper's references) refines a share of each generation with  */
/* the random search with bias of Solis & Wets (1981, Math. Oper. Res. 6).   */
/* Readings, one step per iteration t of one individual x with score f:      */
/*   step_e = (rho * sigma_e) * N(0,1), sigma = the mutation scales (1 A,    */
/*     0.1 per quaternion component, 0.5 rad per torsion);                   */
/*   xi = b + step; probe x + xi; if its score is lower, accept it and set   */
/*     b = 0.2 b + 0.4 xi; otherwise probe x - xi; if that is lower, accept   */
/*     it and set b = b - 0.4 xi; otherwise b = 0.5 b;                       */
/*   an accepted probe counts a success (failures reset), else a failure     */
/*     (successes reset); max_succ successes in a row double rho, max_fail    */
/*     failures in a row halve it (counter reset);                           */
/*   stop after max_its iterations or when rho < rho_lb.                     */
/* A probe wraps torsions as the mutation does and renormalises the         */
/* quaternion. NaN scores count as +inf. Genotype arithmetic is correctly    */
/* rounded FP32 as in the GA. Random numbers: the GA's Philox counters with  */
/* the generation word OR 2^31. The normal of gene e at iteration t is the   */
/* Irwin-Hall sum of the twelve 16-bit halves of words 0-5 of slot 64 t + e,  */
/* (sum - 6 * 2^16) * 2^-16 (exact in float, variance 1); whether an         */
/* individual is refined in a generation is decided by word 0 of slot 63     */
/* against the rate.                                                         */
/* ======================================================================= */
typedef struct {
  float rate;                    /* probability an individual is refined      */
  int32_t max_its, max_succ, max_fail;
  float rho, rho_lb;
} orc_ls_params;

/* objective of a probe: it = iteration, which = 0 forward / 1 backward */
typedef float (*orc_objective)(const float *g, int32_t it, int32_t which, void *ctx);

#define LS_GEN_BIT 0x80000000u

int orc_ls_selected(float rate, uint64_t seed, uint64_t lig, uint32_t gen, uint32_t ind) {
  uint32_t w[8];
  orc_rng_words(seed, lig, gen | LS_GEN_BIT, ind, 63, w);
  return (uint64_t)w[0] < prob_threshold(rate);
}

static float gene_sigma(int e) { return e < 3 ? 1.0f : (e < 7 ? 0.1f : 0.5f); }

/* the local search's normal of gene e at iteration t (see above) */
float orc_ls_normal(uint64_t seed, uint64_t lig, uint32_t gen, uint32_t ind, uint32_t t, int e) {
  uint32_t w[8];
  orc_rng_words(seed, lig, gen | LS_GEN_BIT, ind, 64u * t + (uint32_t)e, w);
  int32_t S = 0;
  for (int k = 0; k < 6; ++k) S += (int32_t)(w[k] & 0xffffu) + (int32_t)(w[k] >> 16);
  return (float)(S - 6 * 65536) * 0x1p-16f;
}

static float nan_to_inf(float v) { return v != v ? INFINITY : v; }

/* y = x + xi (dir > 0) or x - xi (dir < 0), torsions wrapped, quaternion
 * renormalised */
static void ls_probe(int G, const float *x, const float *xi, int dir, float *y) {
  for (int e = 0; e < G; ++e) {
    y[e] = dir > 0 ? x[e] + xi[e] : x[e] - xi[e];
    if (e >= 7) {
      if (y[e] > PI_F) y[e] = y[e] - TWO_PI_F;
      else if (y[e] < -PI_F) y[e] = y[e] + TWO_PI_F;
    }
  }
  quat_normalize(y + 3);
}

/* Refines x (in/out, 7 + k genes) with score *f (in/out); returns the number
 * of objective evaluations, the iterations run in *its. */
int orc_solis_wets(int k, const orc_ls_params *p, uint64_t seed, uint64_t lig, uint32_t gen,
                   uint32_t ind, float *x, float *f, orc_objective obj, void *ctx, int32_t *its) {
  int G = 7 + k, evals = 0, succ = 0, fail = 0, t;
  float b[32], xi[32], y[32];
  float rho = p->rho, fx = nan_to_inf(*f);
  for (int e = 0; e < G; ++e) b[e] = 0.0f;
  for (t = 0; t < p->max_its && !(rho < p->rho_lb); ++t) {
    for (int e = 0; e < G; ++e) {
      float z = orc_ls_normal(seed, lig, gen, ind, (uint32_t)t, e);
      float step = (rho * gene_sigma(e)) * z;
      xi[e] = b[e] + step;
    }
    int ok = 0;
    ls_probe(G, x, xi, +1, y);
    float f1 = nan_to_inf(obj(y, t, 0, ctx));
    ++evals;
    if (f1 < fx) {
      memcpy(x, y, sizeof(float) * G);
      fx = f1;
      ok = 1;
      for (int e = 0; e < G; ++e) b[e] = 0.2f * b[e] + 0.4f * xi[e];
    } else {
      ls_probe(G, x, xi, -1, y);
      float f2 = nan_to_inf(obj(y, t, 1, ctx));
      ++evals;
      if (f2 < fx) {
        memcpy(x, y, sizeof(float) * G);
        fx = f2;
        ok = 1;
        for (int e = 0; e < G; ++e) b[e] = b[e] - 0.4f * xi[e];
      } else {
        for (int e = 0; e < G; ++e) b[e] = 0.5f * b[e];
      }
    }
    if (ok) {
      ++succ;
      fail = 0;
    } else {
      ++fail;
      succ = 0;
    }
    if (succ >= p->max_succ) {
      rho = 2.0f * rho;
      succ = 0;
    } else if (fail >= p->max_fail) {
      rho = 0.5f * rho;
      fail = 0;
    }
  }
  *f = fx;
  if (its) *its = t;
  return evals;
}

/* ======================================================================= */
/* Whole search for a set of ligands (free-run: the oracle's own scores,     */
/* rounded to float, drive selection), pthreads with a shared ligand index   */
/* as in the paper's node-level work stealing (Section IV, Section VII).     */
/* ======================================================================= */
typedef struct {
  int32_t pop, generations;
  float p_cross, p_mut;
  uint64_t seed;
  orc_ls_params ls;  /* rate 0: GA only (the paper's search) */
} orc_search;

typedef struct {
  int32_t n_ligands;
  const int32_t *atom_off, *tors_off;
  const float *x, *y, *z, *q;
  const uint8_t *type;
  const int16_t *parent, *tors_b;
  const uint64_t *ligand_id;
} orc_batch;

typedef struct {
  const orc_batch *b;
  const orc_params *p;
  const orc_grid *G;
  const orc_pocket *P;
  const orc_search *s;
  float *final_geno;    /* [n_ligands][pop][23] */
  float *final_score;   /* [n_ligands][pop]      */
  double *best64;       /* [n_ligands][8]         */
  int32_t *best_idx;    /* [n_ligands][8]         */
  volatile int next;
  pthread_mutex_t mu;
} dock_ctx;

/* objective of the oracle's own search: the FP64 score rounded to float */
typedef struct {
  const orc_ligand *L;
  const orc_params *p;
  const orc_grid *G;
  const orc_pocket *P;
  const uint8_t *moves;
  const int32_t *pairs;
  int np;
  double *xyz;
  double last;
} ls_ctx;

static float ls_objective(const float *g, int32_t it, int32_t which, void *ctx) {
  ls_ctx *X = (ls_ctx *)ctx;
  (void)it;
  (void)which;
  orc_pose(X->L, X->moves, g, X->P->center, 0, X->xyz);
  X->last = orc_inter_grid(X->L, X->G, X->xyz, NULL) + orc_intra(X->L, X->p, X->pairs, X->np, X->xyz, NULL);
  return (float)X->last;
}

static void dock_one(dock_ctx *C, int l) {
  const orc_batch *b = C->b;
  orc_ligand L = {b->atom_off[l + 1] - b->atom_off[l], b->x + b->atom_off[l], b->y + b->atom_off[l],
                  b->z + b->atom_off[l], b->q + b->atom_off[l], b->type + b->atom_off[l],
                  b->parent + b->atom_off[l], b->tors_off[l + 1] - b->tors_off[l],
                  b->tors_b + b->tors_off[l]};
  int P = C->s->pop, G = 7 + L.k, n = L.n;
  uint64_t lig = b->ligand_id[l];
  float *ga = (float *)malloc(sizeof(float) * (size_t)P * G);
  float *gb = (float *)malloc(sizeof(float) * (size_t)P * G);
  float *sc = (float *)malloc(sizeof(float) * (size_t)P);
  double *s64 = (double *)malloc(sizeof(double) * (size_t)P);
  uint8_t *moves = (uint8_t *)malloc((size_t)(L.k > 0 ? L.k : 1) * n);
  int32_t *pairs = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n * (n - 1) + 2));
  double *xyz = (double *)malloc(sizeof(double) * 3 * (size_t)n);
  int np = orc_topology(&L, moves, pairs);
  orc_ga_init(L.k, P, (float)C->P->radius, C->s->seed, lig, ga);
  for (int gen = 0; gen < C->s->generations; ++gen) {
    if (gen > 0) {
      orc_ga_step(L.k, P, C->s->p_cross, C->s->p_mut, C->s->seed, lig, (uint32_t)gen, ga, sc, gb);
      float *t = ga; ga = gb; gb = t;
    }
    for (int i = 0; i < P; ++i) {
      orc_pose(&L, moves, ga + (size_t)i * G, C->P->center, 0, xyz);
      s64[i] = orc_inter_grid(&L, C->G, xyz, NULL) + orc_intra(&L, C->p, pairs, np, xyz, NULL);
      sc[i] = (float)s64[i];
    }
    if (C->s->ls.rate > 0.0f) {
      /* Lamarckian step: the selected individuals are refined in place */
      ls_ctx X = {&L, C->p, C->G, C->P, moves, pairs, np, xyz, 0.0};
      for (int i = 0; i < P; ++i) {
        if (!orc_ls_selected(C->s->ls.rate, C->s->seed, lig, (uint32_t)gen, (uint32_t)i)) continue;
        orc_solis_wets(L.k, &C->s->ls, C->s->seed, lig, (uint32_t)gen, (uint32_t)i,
                       ga + (size_t)i * G, sc + i, ls_objective, &X, NULL);
        orc_pose(&L, moves, ga + (size_t)i * G, C->P->center, 0, xyz);
        s64[i] = orc_inter_grid(&L, C->G, xyz, NULL) + orc_intra(&L, C->p, pairs, np, xyz, NULL);
      }
    }
  }
  for (int i = 0; i < P; ++i) {
    memcpy(C->final_geno + ((size_t)l * P + i) * 23, ga + (size_t)i * G, sizeof(float) * G);
    C->final_score[(size_t)l * P + i] = sc[i];
  }
  /* best 8 by (FP32 score, index); their FP64 scores */
  int chosen[8];
  for (int r = 0; r < 8; ++r) {
    int bi = -1;
    for (int i = 0; i < P; ++i) {
      int used = 0;
      for (int u = 0; u < r; ++u) used |= chosen[u] == i;
      if (used) continue;
      if (bi < 0 || better(sc, i, bi)) bi = i;
    }
    chosen[r] = bi;
    C->best_idx[(size_t)l * 8 + r] = bi;
    C->best64[(size_t)l * 8 + r] = bi >= 0 ? s64[bi] : NAN;
  }
  (void)np;
  free(ga); free(gb); free(sc); free(s64); free(moves); free(pairs); free(xyz);
}

static void *dock_worker(void *arg) {
  dock_ctx *C = (dock_ctx *)arg;
  for (;;) {
    pthread_mutex_lock(&C->mu);
    int l = C->next++;
    pthread_mutex_unlock(&C->mu);
    if (l >= C->b->n_ligands) break;
    dock_one(C, l);
  }
  return NULL;
}

void orc_dock_batch(const orc_batch *b, const orc_params *p, const orc_pocket *P, const orc_grid *G,
                    const orc_search *s, int n_threads, float *final_geno, float *final_score,
                    double *best64, int32_t *best_idx) {
  dock_ctx C;
  C.b = b; C.p = p; C.G = G; C.P = P; C.s = s;
  C.final_geno = final_geno; C.final_score = final_score; C.best64 = best64; C.best_idx = best_idx;
  C.next = 0;
  pthread_mutex_init(&C.mu, NULL);
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  pthread_t th[256];
  for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, dock_worker, &C);
  for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
  pthread_mutex_destroy(&C.mu);
}
