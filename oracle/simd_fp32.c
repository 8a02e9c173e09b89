/*
 * FP32 CPU docking search in the style the paper measures (Section IV and
 * Section VII): single-precision data in structure-of-arrays form, the inner
 * loops over atoms and atom pairs written for the compiler's
 * auto-vectoriser (#pragma omp simd, built with -O3 -ffast-math
 * -fopenmp-simd: vector exp and sqrt come from the C library's vector math
 * functions), one ligand per thread with a shared work index (the paper's
 * node-level work stealing).
 *
 * A BASELINE, NOT THE ORACLE: it runs beside the FP64 oracle as a second,
 * fairer CPU reference point for the benchmark (context only), and is test
 * infrastructure like the rest of this directory. The GA is the oracle's
 * own (orc_ga_init / orc_ga_step, linked from oracle.c), so given this path's
 * FP32 scores its genotypes are the oracle's replay of them bit for bit; the
 * pose and score are re-written here in FP32:
 *   Algorithm 1: rigid motion about the ligand centroid, then each torsion
 *     about its current bond axis (root to leaf), Rodrigues' formula;
 *   Algorithm 2: inter-energy by trilinear lookup in FP32 copies of the
 *     per-type maps (M_t + q E + |q| D, E_out outside the box) and
 *     intra-energy over the included pairs with the AutoDock4 terms (12-6
 *     or 12-10 capped at 1e5 weighted, Coulomb with the Mehler-Solmajer
 *     dielectric, Gaussian desolvation), r floored at 0.5 A, cutoff 8 A.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- layouts shared with oracle.c ---------------------------------------- */
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
  double *maps;
} orc_grid;

typedef struct {
  int32_t n_ligands;
  const int32_t *atom_off, *tors_off;
  const float *x, *y, *z, *q;
  const uint8_t *type;
  const int16_t *parent, *tors_b;
  const uint64_t *ligand_id;
} orc_batch;

int orc_topology(const orc_ligand *L, uint8_t *moves, int32_t *pairs);
void orc_ga_init(int k, int P, float radius, uint64_t seed, uint64_t lig, float *geno);
void orc_ga_step(int k, int P, float p_cross, float p_mut, uint64_t seed, uint64_t lig,
                 uint32_t gen, const float *prev, const float *score, float *next);

/* ---- AutoDock4 constants (as in the oracle) ------------------------------- */
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
#define EMAX 1.0e5
#define EOUT 1000.0f

/* ---- FP32 maps ------------------------------------------------------------- */
typedef struct {
  int n[3], T;
  float o[3], inv_h;
  float *maps; /* [T + 2][nz][ny][nx] */
} grid32;

/* ---- one ligand in SoA form, pair coefficients with the weights folded in - */
typedef struct {
  int n, k, np;
  float *x, *y, *z, *q;   /* centred input coordinates */
  int *type;
  float *px, *py, *pz;    /* posed coordinates */
  int *pi, *pj;           /* included pairs */
  float *c12, *c6, *c10, *cap, *qq, *ds;
  int *ta, *tb, *mv_off, *mv_n, *mv; /* torsion axes and moved atoms */
} lig32;

static int hb_pair(const orc_params *p, int a, int b) {
  return (p->hb_role[a] == 1 && p->hb_role[b] == 2) || (p->hb_role[a] == 2 && p->hb_role[b] == 1);
}

static void lig32_free(lig32 *S) {
  void *ptr[] = {S->x, S->y, S->z, S->q, S->type, S->px, S->py, S->pz, S->pi, S->pj, S->c12,
                 S->c6, S->c10, S->cap, S->qq, S->ds, S->ta, S->tb, S->mv_off, S->mv_n, S->mv};
  for (size_t i = 0; i < sizeof ptr / sizeof ptr[0]; ++i) free(ptr[i]);
}

/* SoA copy of a ligand, its included pairs with their FP32 coefficients and
 * its moved-atom lists; returns -1 on a bad topology. */
static int lig32_build(lig32 *S, const orc_ligand *L, const orc_params *p, const double center[3]) {
  memset(S, 0, sizeof *S);
  const int n = L->n, k = L->k;
  S->n = n;
  S->k = k;
  uint8_t *moves = (uint8_t *)malloc((size_t)(k > 0 ? k : 1) * n);
  int32_t *pairs = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n * (n - 1) + 2));
  const int np = orc_topology(L, moves, pairs);
  if (np < 0) {
    free(moves);
    free(pairs);
    return -1;
  }
  S->np = np;
#define ALLOC(f, t, c) S->f = (t *)malloc(sizeof(t) * (size_t)((c) > 0 ? (c) : 1))
  ALLOC(x, float, n); ALLOC(y, float, n); ALLOC(z, float, n); ALLOC(q, float, n);
  ALLOC(type, int, n); ALLOC(px, float, n); ALLOC(py, float, n); ALLOC(pz, float, n);
  ALLOC(pi, int, np); ALLOC(pj, int, np); ALLOC(c12, float, np); ALLOC(c6, float, np);
  ALLOC(c10, float, np); ALLOC(cap, float, np); ALLOC(qq, float, np); ALLOC(ds, float, np);
  ALLOC(ta, int, k); ALLOC(tb, int, k); ALLOC(mv_off, int, k); ALLOC(mv_n, int, k);
  ALLOC(mv, int, k * n);
#undef ALLOC
  double c[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < n; ++i) {
    c[0] += L->x[i];
    c[1] += L->y[i];
    c[2] += L->z[i];
  }
  for (int m = 0; m < 3; ++m) c[m] /= n;
  for (int i = 0; i < n; ++i) {
    S->x[i] = (float)(L->x[i] - c[0]);
    S->y[i] = (float)(L->y[i] - c[1]);
    S->z[i] = (float)(L->z[i] - c[2]);
    S->q[i] = L->q[i];
    S->type[i] = L->type[i];
  }
  (void)center;
  for (int s = 0; s < np; ++s) {
    const int i = pairs[2 * s], j = pairs[2 * s + 1], ti = L->type[i], tj = L->type[j];
    S->pi[s] = i;
    S->pj[s] = j;
    if (hb_pair(p, ti, tj)) {
      const int acc = p->hb_role[ti] == 2 ? ti : tj;
      const double R = p->hb_R[acc], e = p->hb_eps[acc];
      S->c12[s] = (float)(W_HB * 5.0 * e * pow(R, 12));
      S->c10[s] = (float)(W_HB * 6.0 * e * pow(R, 10));
      S->c6[s] = 0.0f;
      S->cap[s] = (float)(W_HB * EMAX);
    } else {
      const double R = 0.5 * ((double)p->Rii[ti] + (double)p->Rii[tj]);
      const double e = sqrt((double)p->eps[ti] * (double)p->eps[tj]);
      S->c12[s] = (float)(W_VDW * e * pow(R, 12));
      S->c6[s] = (float)(W_VDW * 2.0 * e * pow(R, 6));
      S->c10[s] = 0.0f;
      S->cap[s] = (float)(W_VDW * EMAX);
    }
    S->qq[s] = (float)(W_ELEC * COULOMB * (double)L->q[i] * (double)L->q[j]);
    const double si = (double)p->solpar[ti] + QASP * fabs((double)L->q[i]);
    const double sj = (double)p->solpar[tj] + QASP * fabs((double)L->q[j]);
    S->ds[s] = (float)(W_SOL * (si * (double)p->vol[tj] + sj * (double)p->vol[ti]));
  }
  int off = 0;
  for (int j = 0; j < k; ++j) {
    S->tb[j] = L->tors_b[j];
    S->ta[j] = L->parent[L->tors_b[j]];
    S->mv_off[j] = off;
    for (int i = 0; i < n; ++i)
      if (moves[j * n + i]) S->mv[off++] = i;
    S->mv_n[j] = off - S->mv_off[j];
  }
  free(moves);
  free(pairs);
  return 0;
}

/* Algorithm 1 in FP32 for genotype g (translation, quaternion w x y z, torsions). */
static void pose32(lig32 *S, const float *g, const float center[3]) {
  float qw = g[3], qx = g[4], qy = g[5], qz = g[6];
  const float inv = 1.0f / sqrtf(qw * qw + qx * qx + qy * qy + qz * qz);
  qw *= inv; qx *= inv; qy *= inv; qz *= inv;
  const float r00 = 1 - 2 * (qy * qy + qz * qz), r01 = 2 * (qx * qy - qw * qz), r02 = 2 * (qx * qz + qw * qy);
  const float r10 = 2 * (qx * qy + qw * qz), r11 = 1 - 2 * (qx * qx + qz * qz), r12 = 2 * (qy * qz - qw * qx);
  const float r20 = 2 * (qx * qz - qw * qy), r21 = 2 * (qy * qz + qw * qx), r22 = 1 - 2 * (qx * qx + qy * qy);
  const float tx = center[0] + g[0], ty = center[1] + g[1], tz = center[2] + g[2];
  const int n = S->n;
  float *restrict px = S->px, *restrict py = S->py, *restrict pz = S->pz;
  const float *restrict x = S->x, *restrict y = S->y, *restrict z = S->z;
#pragma omp simd
  for (int a = 0; a < n; ++a) {
    px[a] = r00 * x[a] + r01 * y[a] + r02 * z[a] + tx;
    py[a] = r10 * x[a] + r11 * y[a] + r12 * z[a] + ty;
    pz[a] = r20 * x[a] + r21 * y[a] + r22 * z[a] + tz;
  }
  for (int j = 0; j < S->k; ++j) {
    const int a = S->ta[j], b = S->tb[j];
    const float ax = px[a], ay = py[a], az = pz[a];
    float ux = px[b] - ax, uy = py[b] - ay, uz = pz[b] - az;
    const float il = 1.0f / sqrtf(ux * ux + uy * uy + uz * uz);
    ux *= il; uy *= il; uz *= il;
    const float c = cosf(g[7 + j]), s = sinf(g[7 + j]), oc = 1.0f - c;
    const int *restrict mv = S->mv + S->mv_off[j];
    const int m_n = S->mv_n[j];
#pragma omp simd
    for (int m = 0; m < m_n; ++m) {  /* moved atoms are distinct */
      const int at = mv[m];
      const float vx = px[at] - ax, vy = py[at] - ay, vz = pz[at] - az;
      const float d = (ux * vx + uy * vy + uz * vz) * oc;
      px[at] = ax + vx * c + (uy * vz - uz * vy) * s + ux * d;
      py[at] = ay + vy * c + (uz * vx - ux * vz) * s + uy * d;
      pz[at] = az + vz * c + (ux * vy - uy * vx) * s + uz * d;
    }
  }
}

/* Algorithm 2 in FP32 for the posed ligand. */
static float score32(const lig32 *S, const grid32 *G) {
  const int n = S->n, T = G->T, nx = G->n[0], ny = G->n[1], nz = G->n[2];
  const size_t vol = (size_t)nx * ny * nz;
  const float *restrict maps = G->maps;
  const float *restrict px = S->px, *restrict py = S->py, *restrict pz = S->pz;
  float inter = 0.0f;
#pragma omp simd reduction(+ : inter)
  for (int a = 0; a < n; ++a) {
    const float ux = (px[a] - G->o[0]) * G->inv_h, uy = (py[a] - G->o[1]) * G->inv_h,
                uz = (pz[a] - G->o[2]) * G->inv_h;
    const int inside = ux >= 0.0f && ux <= (float)(nx - 1) && uy >= 0.0f && uy <= (float)(ny - 1) &&
                       uz >= 0.0f && uz <= (float)(nz - 1);
    float e = EOUT;
    if (inside) {
      int ix = (int)ux, iy = (int)uy, iz = (int)uz;
      ix = ix > nx - 2 ? nx - 2 : ix;
      iy = iy > ny - 2 ? ny - 2 : iy;
      iz = iz > nz - 2 ? nz - 2 : iz;
      const float fx = ux - ix, fy = uy - iy, fz = uz - iz;
      const size_t b0 = ((size_t)iz * ny + iy) * nx + ix;
      const size_t d1 = 1, dy = (size_t)nx, dz = (size_t)nx * ny;
      const float q = S->q[a], aq = fabsf(q);
      const size_t base[3] = {(size_t)S->type[a] * vol, (size_t)T * vol, (size_t)(T + 1) * vol};
      float v[3];
      for (int m = 0; m < 3; ++m) {
        const float *M = maps + base[m] + b0;
        const float c00 = M[0] + fx * (M[d1] - M[0]), c10 = M[dy] + fx * (M[dy + d1] - M[dy]);
        const float c01 = M[dz] + fx * (M[dz + d1] - M[dz]);
        const float c11 = M[dz + dy] + fx * (M[dz + dy + d1] - M[dz + dy]);
        const float c0 = c00 + fy * (c10 - c00), c1 = c01 + fy * (c11 - c01);
        v[m] = c0 + fz * (c1 - c0);
      }
      e = v[0] + q * v[1] + aq * v[2];
    }
    inter += e;
  }
  const float lamB = (float)(DIEL_LAMBDA * (DIEL_EPS0 - DIEL_A)), dA = (float)DIEL_A;
  const float dB = (float)(DIEL_EPS0 - DIEL_A), dK = (float)DIEL_K;
  const float isig = (float)(1.0 / (2.0 * SIGMA_SOL * SIGMA_SOL));
  const int np = S->np;
  const int *restrict pi = S->pi, *restrict pj = S->pj;
  float intra = 0.0f;
#pragma omp simd reduction(+ : intra)
  for (int s = 0; s < np; ++s) {
    const float dx = px[pi[s]] - px[pj[s]], dy = py[pi[s]] - py[pj[s]], dz = pz[pi[s]] - pz[pj[s]];
    const float r2 = dx * dx + dy * dy + dz * dz;
    const float r2c = r2 > 0.25f ? r2 : 0.25f;
    const float r = sqrtf(r2c);
    const float i2 = 1.0f / r2c, i6 = i2 * i2 * i2;
    float disp = i6 * (S->c12[s] * i6 - S->c6[s] - S->c10[s] * i2 * i2);
    disp = disp < S->cap[s] ? disp : S->cap[s];
    const float eps = dA + dB / (1.0f + dK * expf(-lamB * r));
    const float e = disp + S->qq[s] / (eps * r) + S->ds[s] * expf(-r2c * isig);
    intra += r2 < 64.0f ? e : 0.0f;
  }
  return inter + intra;
}

static void grid32_from(grid32 *G32, const orc_grid *G) {
  G32->n[0] = G->nx;
  G32->n[1] = G->ny;
  G32->n[2] = G->nz;
  G32->T = G->n_types;
  G32->o[0] = (float)G->ox;
  G32->o[1] = (float)G->oy;
  G32->o[2] = (float)G->oz;
  G32->inv_h = (float)(1.0 / G->h);
  const size_t count = (size_t)(G->n_types + 2) * G->nx * G->ny * G->nz;
  G32->maps = (float *)malloc(sizeof(float) * count);
  for (size_t i = 0; i < count; ++i) G32->maps[i] = (float)G->maps[i];
}

/* FP32 scores of n given poses of one ligand (genotypes of n_genes floats). */
int cpu32_score_poses(const orc_ligand *L, const orc_params *p, const orc_grid *G,
                      const double center[3], const float *genos, int n_genes, int64_t n,
                      float *out) {
  lig32 S;
  if (lig32_build(&S, L, p, center) < 0) return -1;
  grid32 G32;
  grid32_from(&G32, G);
  const float c[3] = {(float)center[0], (float)center[1], (float)center[2]};
  for (int64_t i = 0; i < n; ++i) {
    pose32(&S, genos + i * n_genes, c);
    out[i] = score32(&S, &G32);
  }
  free(G32.maps);
  lig32_free(&S);
  return 0;
}

typedef struct {
  const orc_batch *b;
  const orc_params *p;
  const orc_pocket *P;
  const grid32 *G;
  int pop, gens;
  float p_cross, p_mut;
  uint64_t seed;
  float *final_score;   /* [n_ligands][pop] */
  int32_t *best_idx;    /* [n_ligands] */
  float *trace_geno;    /* optional, ligand 0: [gens][pop][7 + k] */
  float *trace_score;   /* optional, ligand 0: [gens][pop] */
  int next;
  pthread_mutex_t mu;
} cpu32_ctx;

static void dock_one32(cpu32_ctx *C, int l) {
  const orc_batch *b = C->b;
  const orc_ligand L = {b->atom_off[l + 1] - b->atom_off[l], b->x + b->atom_off[l],
                        b->y + b->atom_off[l], b->z + b->atom_off[l], b->q + b->atom_off[l],
                        b->type + b->atom_off[l], b->parent + b->atom_off[l],
                        b->tors_off[l + 1] - b->tors_off[l], b->tors_b + b->tors_off[l]};
  lig32 S;
  if (lig32_build(&S, &L, C->p, C->P->center) < 0) return;
  const int P = C->pop, G = 7 + L.k;
  const uint64_t lig = b->ligand_id[l];
  const float c[3] = {(float)C->P->center[0], (float)C->P->center[1], (float)C->P->center[2]};
  float *ga = (float *)malloc(sizeof(float) * (size_t)P * G);
  float *gb = (float *)malloc(sizeof(float) * (size_t)P * G);
  float *sc = (float *)malloc(sizeof(float) * (size_t)P);
  orc_ga_init(L.k, P, (float)C->P->radius, C->seed, lig, ga);
  for (int gen = 0; gen < C->gens; ++gen) {
    if (gen > 0) {
      orc_ga_step(L.k, P, C->p_cross, C->p_mut, C->seed, lig, (uint32_t)gen, ga, sc, gb);
      float *t = ga;
      ga = gb;
      gb = t;
    }
    for (int i = 0; i < P; ++i) {
      pose32(&S, ga + (size_t)i * G, c);
      sc[i] = score32(&S, C->G);
    }
    if (l == 0 && C->trace_geno) {
      memcpy(C->trace_geno + (size_t)gen * P * G, ga, sizeof(float) * (size_t)P * G);
      memcpy(C->trace_score + (size_t)gen * P, sc, sizeof(float) * (size_t)P);
    }
  }
  int best = 0;
  for (int i = 1; i < P; ++i) {
    const float a = sc[i] != sc[i] ? INFINITY : sc[i], o = sc[best] != sc[best] ? INFINITY : sc[best];
    if (a < o) best = i;
  }
  memcpy(C->final_score + (size_t)l * P, sc, sizeof(float) * (size_t)P);
  C->best_idx[l] = best;
  free(ga);
  free(gb);
  free(sc);
  lig32_free(&S);
}

static void *cpu32_worker(void *arg) {
  cpu32_ctx *C = (cpu32_ctx *)arg;
  for (;;) {
    pthread_mutex_lock(&C->mu);
    const int l = C->next++;
    pthread_mutex_unlock(&C->mu);
    if (l >= C->b->n_ligands) break;
    dock_one32(C, l);
  }
  return NULL;
}

/* The plain GA search of a ligand set with FP32 scoring on n_threads host
 * threads: final population scores and the best individual per ligand;
 * trace_geno / trace_score (optional) record ligand 0's generations. */
void cpu32_dock_batch(const orc_batch *b, const orc_params *p, const orc_pocket *P,
                      const orc_grid *G, int pop, int gens, float p_cross, float p_mut,
                      uint64_t seed, int n_threads, float *final_score, int32_t *best_idx,
                      float *trace_geno, float *trace_score) {
  grid32 G32;
  grid32_from(&G32, G);
  cpu32_ctx C;
  C.b = b; C.p = p; C.P = P; C.G = &G32;
  C.pop = pop; C.gens = gens; C.p_cross = p_cross; C.p_mut = p_mut; C.seed = seed;
  C.final_score = final_score; C.best_idx = best_idx;
  C.trace_geno = trace_geno; C.trace_score = trace_score;
  C.next = 0;
  pthread_mutex_init(&C.mu, NULL);
  if (n_threads < 1) n_threads = 1;
  if (n_threads > 256) n_threads = 256;
  pthread_t th[256];
  for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, cpu32_worker, &C);
  for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
  pthread_mutex_destroy(&C.mu);
  free(G32.maps);
}
