/*
 * Plain FP64 oracle of the learned surrogate that pre-screens candidate
 * poses: an MLP 128 -> 256 -> 256 -> 256 -> 1 with GELU on per-pose
 * features, trained on (features, exact score) pairs.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.c). The paper itself has no learned
 * component; these functions compute the surrogate as designed here:
 *
 * Features of one posed ligand (128 values, in this order):
 *   [0, 56)    atom counts / 8 per (type t < 7, radial shell s < 8) around the
 *              pocket centre, shell width R/8, the last shell open: index 8 t + s
 *   [56, 64)   sum of charges per shell
 *   [64, 72)   sum of |charge| per shell
 *   [72, 104)  sin, cos of torsion j (index 72 + 2 j, 73 + 2 j), 0 for j >= k
 *   [104, 113) rotation matrix of the normalised quaternion, row-major
 *   [113, 116) translation gene / R
 *   116: n / 100, 117: k / 16, [118, 128) zero.
 *
 * MLP: h1 = gelu(x W1 + b1), h2 = gelu(h1 W2 + b2), h3 = gelu(h2 W3 + b3),
 * y = h3 W4 + b4, gelu(z) = z (1 + erf(z / sqrt 2)) / 2. Parameters are packed
 * W1[128][256], b1[256], W2[256][256], b2[256], W3[256][256], b3[256],
 * W4[256], b4 (W stored [in][out]). Loss = mean over the batch of (y - t)^2.
 *
 * Training (per pocket, on (features, exact score) pairs):
 *   target t = (min(score, clip) - mean) / std, mean and std of min(score,
 *   clip) over the training set;
 *   rows visited in one fixed order per run (orc_train_order, a keyed
 *   bijection of [0, n)) in batches, the same order every epoch;
 *   per batch one Adam step (Kingma & Ba, ICLR 2015, Algorithm 1):
 *     m = b1 m + (1 - b1) g,  v = b2 v + (1 - b2) g^2,
 *     p = p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps),
 *   with lr 1e-3, b1 0.9, b2 0.999, eps 1e-8 and t the step count from 1.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
  int32_t n;
  const float *x, *y, *z, *q;
  const uint8_t *type;
  const int16_t *parent;
  int32_t k;
  const int16_t *tors_b;
} sur_ligand; /* same layout as the oracle's orc_ligand */

#define NF 128
#define NH 256
#define N_PARAMS (NF * NH + NH + NH * NH + NH + NH * NH + NH + NH + 1)

void orc_quat_matrix(const double q_in[4], double R[9]);

void orc_features(const sur_ligand *L, const double *xyz, const double center[3],
                  const float *geno, double radius, double *f) {
  for (int i = 0; i < NF; ++i) f[i] = 0.0;
  const double w = radius / 8.0;
  for (int a = 0; a < L->n; ++a) {
    double dx = xyz[3 * a] - center[0], dy = xyz[3 * a + 1] - center[1], dz = xyz[3 * a + 2] - center[2];
    double d = sqrt(dx * dx + dy * dy + dz * dz);
    int s = (int)floor(d / w);
    if (s > 7) s = 7;
    int t = L->type[a];
    if (t < 7) f[8 * t + s] += 1.0 / 8.0;
    f[56 + s] += L->q[a];
    f[64 + s] += fabs((double)L->q[a]);
  }
  for (int j = 0; j < L->k && j < 16; ++j) {
    f[72 + 2 * j] = sin((double)geno[7 + j]);
    f[73 + 2 * j] = cos((double)geno[7 + j]);
  }
  double q[4] = {geno[3], geno[4], geno[5], geno[6]}, R[9];
  orc_quat_matrix(q, R);
  for (int m = 0; m < 9; ++m) f[104 + m] = R[m];
  for (int m = 0; m < 3; ++m) f[113 + m] = (double)geno[m] / radius;
  f[116] = L->n / 100.0;
  f[117] = L->k / 16.0;
}

static double gelu(double z) { return 0.5 * z * (1.0 + erf(z / sqrt(2.0))); }
static double gelu_d(double z) {
  return 0.5 * (1.0 + erf(z / sqrt(2.0))) + z * exp(-0.5 * z * z) / sqrt(2.0 * M_PI);
}

typedef struct {
  const double *W1, *b1, *W2, *b2, *W3, *b3, *W4, *b4;
} mlp_view;

static mlp_view view(const double *p) {
  mlp_view v;
  v.W1 = p; p += NF * NH;
  v.b1 = p; p += NH;
  v.W2 = p; p += NH * NH;
  v.b2 = p; p += NH;
  v.W3 = p; p += NH * NH;
  v.b3 = p; p += NH;
  v.W4 = p; p += NH;
  v.b4 = p;
  return v;
}

/* z[j] = b[j] + sum_i x[i] W[i][j] */
static void dense(const double *x, int nin, const double *W, const double *b, int nout, double *z) {
  for (int j = 0; j < nout; ++j) z[j] = b[j];
  for (int i = 0; i < nin; ++i)
    for (int j = 0; j < nout; ++j) z[j] += x[i] * W[i * nout + j];
}

/* Forward pass for n rows of X (n x 128); Y gets n outputs. */
void orc_mlp_forward(const double *params, int n, const double *X, double *Y) {
  mlp_view v = view(params);
  double z1[NH], h1[NH], z2[NH], h2[NH], z3[NH], h3[NH];
  for (int r = 0; r < n; ++r) {
    dense(X + (size_t)r * NF, NF, v.W1, v.b1, NH, z1);
    for (int j = 0; j < NH; ++j) h1[j] = gelu(z1[j]);
    dense(h1, NH, v.W2, v.b2, NH, z2);
    for (int j = 0; j < NH; ++j) h2[j] = gelu(z2[j]);
    dense(h2, NH, v.W3, v.b3, NH, z3);
    for (int j = 0; j < NH; ++j) h3[j] = gelu(z3[j]);
    double y = v.b4[0];
    for (int j = 0; j < NH; ++j) y += h3[j] * v.W4[j];
    Y[r] = y;
  }
}

/* Gradient of loss = (1/n) sum (y_r - t_r)^2 with respect to every
 * parameter (same packing as params); returns the loss. */
double orc_mlp_backward(const double *params, int n, const double *X, const double *T, double *grad) {
  mlp_view v = view(params);
  memset(grad, 0, sizeof(double) * N_PARAMS);
  mlp_view g = view(grad);
  double *gW1 = (double *)g.W1, *gb1 = (double *)g.b1, *gW2 = (double *)g.W2, *gb2 = (double *)g.b2;
  double *gW3 = (double *)g.W3, *gb3 = (double *)g.b3, *gW4 = (double *)g.W4, *gb4 = (double *)g.b4;
  double z1[NH], h1[NH], z2[NH], h2[NH], z3[NH], h3[NH], d3[NH], d2[NH], d1[NH];
  double loss = 0.0;
  for (int r = 0; r < n; ++r) {
    const double *x = X + (size_t)r * NF;
    dense(x, NF, v.W1, v.b1, NH, z1);
    for (int j = 0; j < NH; ++j) h1[j] = gelu(z1[j]);
    dense(h1, NH, v.W2, v.b2, NH, z2);
    for (int j = 0; j < NH; ++j) h2[j] = gelu(z2[j]);
    dense(h2, NH, v.W3, v.b3, NH, z3);
    for (int j = 0; j < NH; ++j) h3[j] = gelu(z3[j]);
    double y = v.b4[0];
    for (int j = 0; j < NH; ++j) y += h3[j] * v.W4[j];
    double e = y - T[r];
    loss += e * e;
    double dy = 2.0 * e / n;
    gb4[0] += dy;
    for (int j = 0; j < NH; ++j) {
      gW4[j] += h3[j] * dy;
      d3[j] = dy * v.W4[j] * gelu_d(z3[j]);
    }
    for (int j = 0; j < NH; ++j) gb3[j] += d3[j];
    for (int i = 0; i < NH; ++i) {
      double s = 0.0;
      for (int j = 0; j < NH; ++j) {
        gW3[i * NH + j] += h2[i] * d3[j];
        s += v.W3[i * NH + j] * d3[j];
      }
      d2[i] = s * gelu_d(z2[i]);
    }
    for (int j = 0; j < NH; ++j) gb2[j] += d2[j];
    for (int i = 0; i < NH; ++i) {
      double s = 0.0;
      for (int j = 0; j < NH; ++j) {
        gW2[i * NH + j] += h1[i] * d2[j];
        s += v.W2[i * NH + j] * d2[j];
      }
      d1[i] = s * gelu_d(z1[i]);
    }
    for (int j = 0; j < NH; ++j) gb1[j] += d1[j];
    for (int i = 0; i < NF; ++i)
      for (int j = 0; j < NH; ++j) gW1[i * NH + j] += x[i] * d1[j];
  }
  return loss / n;
}

int orc_mlp_n_params(void) { return N_PARAMS; }

/* ======================================================================= */
/* Training: Adam step and the order of the training rows                   */
/* ======================================================================= */

/* One Adam step (Kingma & Ba 2015, Algorithm 1) on n parameters in FP64;
 * t is the step number (1 for the first step). */
void orc_adam_step(double *p, double *m, double *v, const double *g, int64_t n, double lr,
                   double b1, double b2, double eps, int t) {
  const double c1 = 1.0 - pow(b1, t), c2 = 1.0 - pow(b2, t);
  for (int64_t i = 0; i < n; ++i) {
    m[i] = b1 * m[i] + (1.0 - b1) * g[i];
    v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
    const double mh = m[i] / c1, vh = v[i] / c2;
    p[i] -= lr * mh / (sqrt(vh) + eps);
  }
}

/* SplitMix64 output mix (Steele, Lea & Flood, OOPSLA 2014). */
static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* The order in which training visits its n rows: row r of the visit is
 * out[r] = pi(r), pi a bijection of [0, n) keyed by seed. pi is a balanced
 * four-round Feistel network on 2h-bit words (4^h the smallest power of four
 * >= n; Luby & Rackoff 1988), round i mapping (L, R) to
 * (R, L xor (mix64(R xor K_i) mod 2^h)) with K_i = mix64(seed + (i + 1)
 * 0x9E3779B97F4A7C15), restricted to [0, n) by cycle walking (Black &
 * Rogaway 2002): values >= n are encrypted again until one falls below n. */
uint64_t orc_train_order_one(uint64_t seed, uint64_t n, uint64_t r) {
  int h = 1;
  while ((1ULL << (2 * h)) < n) ++h;
  const uint64_t mask = (1ULL << h) - 1;
  uint64_t K[4];
  for (int i = 0; i < 4; ++i) K[i] = mix64(seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ULL);
  uint64_t x = r;
  do {
    uint64_t L = x >> h, R = x & mask;
    for (int i = 0; i < 4; ++i) {
      const uint64_t t = L ^ (mix64(R ^ K[i]) & mask);
      L = R;
      R = t;
    }
    x = (L << h) | R;
  } while (x >= n);
  return x;
}

void orc_train_order(uint64_t seed, int64_t n, int64_t *out) {
  for (int64_t r = 0; r < n; ++r) out[r] = (int64_t)orc_train_order_one(seed, (uint64_t)n, (uint64_t)r);
}
