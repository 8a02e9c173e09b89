/*
 * dock.h - C ABI of the GB300 docking library (libdock.so).
 *
 * The library runs the data-parallel hot path of the muDock method
 * (arXiv 2509.12232, Section V): for every candidate pose of every ligand,
 * inside a genetic-algorithm search, apply the pose (Algorithm 1: translate,
 * rotate, then rotate the fragment below each rotatable bond) and score it
 * (Algorithm 2: inter-energy by lookup in per-atom-type grid maps built once
 * per protein, plus pairwise intra-energy of the ligand).
 *
 * Conventions for every call:
 *  - Plain C types only. Pointers documented as "host" are read (or written)
 *    before the call returns; the caller keeps ownership. Pointers documented
 *    as "device" are CUDA device pointers that must stay valid until the work
 *    enqueued by the call has finished on its stream.
 *  - Objects returned through an out-pointer (dock_pocket, dock_ligands,
 *    dock_job) own their device memory; free them with the matching
 *    *_destroy call. Destroy calls accept NULL.
 *  - stream is a cudaStream_t passed as void* (NULL = legacy default stream).
 *  - Every call returns a dock_status; on failure dock_last_error() gives a
 *    message for the calling thread. No C++ exception crosses the ABI.
 *  - There is no CPU fallback: without a usable CUDA device the calls return
 *    DOCK_ECUDA.
 *  - The library uses the CUDA device that is current on the calling thread
 *    when the object is created; later calls on that object switch to it.
 */
#ifndef DOCK_H
#define DOCK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DOCK_OK = 0,
  DOCK_EINVAL = -1,   /* invalid argument or input data                     */
  DOCK_ENOMEM = -2,   /* device or host allocation failed                   */
  DOCK_ECUDA = -3,    /* CUDA runtime error (no device, launch failure ...) */
  DOCK_ETIMEOUT = -4, /* host wait or device deadline exceeded              */
  DOCK_EDEVICE = -5,  /* a kernel reported an error through its status word */
  DOCK_ENOTIMPL = -6  /* feature not built                                  */
} dock_status;

#define DOCK_MAX_ATOMS 128     /* heavy atoms per ligand                     */
#define DOCK_MAX_TORSIONS 16   /* rotatable bonds per ligand                 */
#define DOCK_MAX_GENES 23      /* 3 translation + 4 quaternion + torsions    */
#define DOCK_MAX_TYPES 16      /* atom types in the parameter table          */
#define DOCK_MAX_POP 4096      /* individuals per ligand                     */
#define DOCK_N_BEST 8          /* best poses rescored in FP64 per ligand     */

/* Per-atom-type force-field parameters (AutoDock4 free-energy form that the
 * paper's scoring is "functionally equivalent" to, Section V).
 * Rii: like-pair vdW well distance (A); eps: well depth (kcal/mol);
 * vol: atomic volume (A^3); solpar: atomic solvation parameter;
 * hb_role: 0 none, 1 H-bond donor, 2 H-bond acceptor; hb_R / hb_eps: the
 * 12-10 well of a donor-acceptor pair, read from the acceptor's row. */
typedef struct {
  float Rii, eps, vol, solpar, hb_R, hb_eps;
  int32_t hb_role;
} dock_type_params;

/* ------------------------------------------------------------------------ */
/* Pocket: protein + grid maps (Section V, "we precompute different 3D maps  */
/* around the protein, as AutoGrid does", one map per ligand atom type).     */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t n_atoms;               /* protein atoms, >= 0                        */
  const float *x, *y, *z, *q;    /* host, [n_atoms] coordinates (A), charges   */
  const uint8_t *type;           /* host, [n_atoms], each < n_types            */
  float center[3];               /* pocket centre: grid centre, pose origin    */
  float radius;                  /* cavity radius R: the grid has floor(2R/h)+1
                                    nodes per axis, centred on center          */
  float spacing;                 /* grid spacing h (A), e.g. 0.375             */
  int32_t n_types;               /* 1..DOCK_MAX_TYPES                          */
  const dock_type_params *params;/* host, [n_types]                            */
} dock_pocket_desc;

typedef struct dock_pocket dock_pocket;

/* Copies the protein to the device and builds the grid maps there: for every
 * node and ligand type t, M_t (12-6 / 12-10 and type-dependent desolvation),
 * E (electrostatic potential) and D (charge desolvation), so that a ligand
 * atom of type t and charge q at a node scores M_t + q E + |q| D. Work is
 * enqueued on stream; the call synchronises it before returning.
 * Errors: DOCK_EINVAL (NULL pointers, n_types out of range, spacing <= 0,
 * radius <= 0, a type >= n_types), DOCK_ENOMEM, DOCK_ECUDA. */
int dock_create_pocket(const dock_pocket_desc *desc, void *stream, dock_pocket **out);
void dock_pocket_destroy(dock_pocket *pocket);

/* Grid geometry of a pocket: nodes per axis and origin (the node with index
 * (0,0,0)). Maps are float4 {M_t, E, D, 0} in [n_types][n][n][n] order (x
 * fastest); *maps_device receives the device pointer (owned by the pocket). */
int dock_pocket_grid(const dock_pocket *pocket, int32_t *n_per_axis, float origin[3],
                     const void **maps_device);

/* ------------------------------------------------------------------------ */
/* Ligands (Algorithm 1 input "Ligand"): CSR over a batch.                   */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t n_ligands;             /* >= 0                                        */
  const int32_t *atom_off;       /* host [n_ligands+1]; ligand l owns atoms
                                    atom_off[l] .. atom_off[l+1]-1, 1..128 each */
  const float *x, *y, *z, *q;    /* host [atom_off[n_ligands]]                  */
  const uint8_t *type;           /* host, each < the pocket's n_types           */
  const int16_t *parent;         /* host, ligand-local bond tree: atom 0 is the
                                    root (-1), every other atom i has
                                    0 <= parent[i] < i                          */
  const int32_t *tors_off;       /* host [n_ligands+1]; <= 16 per ligand        */
  const int16_t *tors_b;         /* host: child atom b of each rotatable bond
                                    (parent[b], b), strictly increasing within a
                                    ligand (ancestors before descendants)      */
  const uint64_t *ligand_id;     /* host [n_ligands]: keys the RNG streams      */
} dock_ligand_batch;

typedef struct dock_ligands dock_ligands;

/* Validates the batch, derives per ligand the atoms moved by each torsion,
 * the included intra pairs (more than three bonds apart, with a rotatable bond
 * on the path between them) and their pair coefficients, centres each ligand
 * on its centroid, and uploads all of it. The pocket supplies the parameter
 * table. Synchronises stream before returning.
 * Errors: DOCK_EINVAL (bad sizes, parent order, torsion list, types),
 * DOCK_ENOMEM, DOCK_ECUDA. */
int dock_load_ligands(const dock_pocket *pocket, const dock_ligand_batch *batch, void *stream,
                      dock_ligands **out);
void dock_ligands_destroy(dock_ligands *ligands);

/* Sizes of a loaded ligand set, for work accounting: totals over its ligands
 * of atoms, intra pairs evaluated per pose (the included pairs whose distance
 * a pose can change; the others, where every torsion separating the two atoms
 * has one of them on its axis, are summed once per ligand at load time),
 * torsions and torsion-moved atoms (sum over torsions of the atoms each one
 * rotates), and the bytes dock_load_ligands copied to the device. Any output
 * may be NULL. */
int dock_ligands_info(const dock_ligands *ligands, int32_t *n_ligands, int64_t *n_atoms,
                      int64_t *n_pairs, int64_t *n_torsions, int64_t *n_moved,
                      int64_t *h2d_bytes);

/* Genotype layout used by every call below: ligand l with k_l torsions has
 * G_l = 7 + k_l genes [tx, ty, tz, qw, qx, qy, qz, theta_1 .. theta_k]; the
 * population of ligand l starts at float offset geno_off[l] = sum over l' < l
 * of pop * G_l', individual i at geno_off[l] + i * G_l. Scores of ligand l,
 * individual i are at l * pop + i. */

/* ------------------------------------------------------------------------ */
/* Search (Section V: GA without local search; fitness = score)               */
/* ------------------------------------------------------------------------ */
typedef struct dock_surrogate dock_surrogate;

/* Solis-Wets local search: the Lamarckian variant of AutoDock's GA (Morris
 * et al. 1998, in the paper's references; the random search with bias of
 * Solis & Wets 1981). The paper's own search has none (Section V). One
 * iteration on genotype x with score f: step_e = (rho sigma_e) N(0,1) with
 * the mutation scales sigma (1 A, 0.1, 0.5 rad); xi = b + step; probe x + xi,
 * accepted if its score is lower (b = 0.2 b + 0.4 xi), else probe x - xi,
 * accepted if lower (b = b - 0.4 xi), else b = 0.5 b; max_succ successes in a
 * row double rho, max_fail failures in a row halve it; the search ends after
 * max_its iterations or once rho < rho_lb. Probes wrap torsions as the
 * mutation does and renormalise the quaternion; NaN scores count as +inf;
 * genotype arithmetic is correctly rounded FP32 (bit-exact with the CPU
 * oracle given the same scores). Random numbers: the GA's Philox counters
 * with the generation word OR 2^31 (the normal of iteration t, gene e is the
 * Irwin-Hall sum of the twelve 16-bit halves of words 0-5 of slot 64 t + e;
 * the selection draw is word 0 of slot 63). */
typedef struct {
  float rate;                    /* dock_batch: probability that an individual
                                    is refined after scoring, every generation
                                    (0 = the paper's GA without local search;
                                    AutoDock: 0.06); ignored by
                                    dock_local_search (every pose is refined)  */
  int32_t max_its;               /* iterations per refinement, 1..DOCK_LS_MAX_ITS
                                    (AutoDock: 300)                            */
  int32_t max_succ, max_fail;    /* >= 1 (AutoDock: 4 and 4)                   */
  float rho, rho_lb;             /* initial step scale and the stop threshold,
                                    finite, rho > 0 (AutoDock: 1.0, 0.01)       */
} dock_ls_params;

#define DOCK_LS_MAX_ITS 10000

typedef struct {
  int32_t pop;                   /* individuals per ligand, 2..DOCK_MAX_POP     */
  int32_t generations;           /* scoring passes, >= 1 (generation 0 = init)  */
  float p_cross;                 /* two-point block crossover probability       */
  float p_mut;                   /* per-gene mutation probability               */
  uint64_t seed;                 /* Philox4x64-10 key                           */
  int32_t lanes_per_pose;        /* 0 = pick by ligand size (autotune table);
                                    else 1, 2, 4 or 8 lanes of a warp per pose   */
  int32_t use_graph;             /* 1: capture the generation launches in a CUDA
                                    graph and launch it; 0: plain launches      */
  uint64_t timeout_ns;           /* device deadline for the whole search from its
                                    first kernel (0 = none); exceeding it stops
                                    the work loops and flags DOCK_ETIMEOUT      */
  float *trace_genotypes;        /* optional device [generations][total genes]:
                                    every generation's population              */
  float *trace_scores;           /* optional device [generations][n_ligands*pop]*/
  int32_t mode;                  /* DOCK_MODE_PLAIN or DOCK_MODE_SURROGATE        */
  int32_t candidates;            /* surrogate: candidates per ligand and
                                    generation, <= DOCK_MAX_CANDIDATES           */
  int32_t keep;                  /* surrogate: candidates kept for exact scoring
                                    (1..candidates), merged (mu + lambda) with the
                                    population by exact score                   */
  dock_surrogate *surrogate;     /* surrogate: the trained network                */
  dock_ls_params ls;             /* plain mode only: ls.rate > 0 makes the search
                                    Lamarckian (Solis-Wets on the selected
                                    individuals of every generation, generation 0
                                    included; the refined genotype and score
                                    replace the individual before the next
                                    generation's selection); rate 0 = no local
                                    search                                      */
  float *trace_ls;               /* optional device [generations][n_ligands*pop]
                                    [2 + 2 ls.max_its]: for each refined
                                    individual its score before refinement, the
                                    iterations run, then per iteration the
                                    scores of the probes x + xi and x - xi (NaN
                                    when not evaluated); rows of individuals not
                                    refined are not written                     */
  int32_t inter;                 /* DOCK_INTER_GRID: inter-energy by trilinear
                                    lookup in the pocket's maps (Algorithm 2);
                                    DOCK_INTER_PAIRWISE: the pairwise sum over
                                    every protein atom within the cutoff, no
                                    maps (plain GA only; the best 8 are
                                    rescored with the FP64 pairwise sum)        */
  const float *resume_genotypes; /* optional device: a saved population, that of
                                    generation resume_from, in the layout of one
                                    generation of trace_genotypes; the search
                                    then runs generations resume_from + 1 ..
                                    generations - 1 only, bit-identical to the
                                    search that saved it (the GA's random
                                    numbers depend on seed, ligand, generation
                                    and individual alone; the trace arrays get
                                    the generations run). Plain GA without local
                                    search; NULL = start from generation 0      */
  const float *resume_scores;    /* device [n_ligands*pop]: that population's
                                    FP32 scores (trace_scores of the generation) */
  int32_t resume_from;           /* 0 .. generations - 2 (with resume_genotypes) */
} dock_search_params;

#define DOCK_INTER_GRID 0
#define DOCK_INTER_PAIRWISE 1

#define DOCK_MODE_PLAIN 0
#define DOCK_MODE_SURROGATE 1
#define DOCK_MAX_CANDIDATES 8192

typedef struct dock_job dock_job;

/* Enqueues the whole search for every ligand on stream and returns at once:
 * generation 0 draws the population, each later generation runs one GA step
 * (tournament selection, crossover, mutation, elitism 1) fused with pose
 * application and FP32 scoring with compensated (Kahan) sums; after the last
 * generation the best DOCK_N_BEST individuals of each ligand are re-posed and
 * rescored in FP64. The pocket and ligands must outlive the job.
 * Errors: DOCK_EINVAL, DOCK_ENOMEM, DOCK_ECUDA. */
/* With mode = DOCK_MODE_SURROGATE each generation after the first draws
 * `candidates` children per ligand by the same GA operators, ranks them by the
 * surrogate's predicted score from their features, scores the best `keep`
 * exactly (FP32) and keeps the best pop of population and kept candidates by
 * exact score (ties: population first, then index); every reported score is
 * exact. */
/* Environment overrides of the launch shape, for tuning and benchmarking (read
 * at each call; unset = dock_autotune's pick for these ligands, else 128
 * threads x 16 atoms per lane): DOCK_THREADS (CTA threads, a power of two in
 * 32..128), DOCK_ATOMS_PER_LANE (shared-memory atoms per lane; raised to fit
 * the largest ligand in 8 lanes), DOCK_LS_LANES (lanes per Solis-Wets chain:
 * 0, 1, 2, 4, 8, 16 or 32, at least the search's lanes per pose; default 16)
 * and DOCK_LS_CHAINS (chains a lane group runs one after another; raised to at
 * least 0.25; default 2). DOCK_THREADS or DOCK_LS_LANES outside those values
 * fails with DOCK_EINVAL. None changes what is computed, only which lanes sum
 * which terms and so the rounding of the FP32 sums. */
int dock_batch(dock_pocket *pocket, dock_ligands *ligands, const dock_search_params *params,
               void *stream, dock_job **out);

typedef struct {
  uint64_t ligand_id;
  int32_t n_genes;               /* G_l                                          */
  int32_t status;                /* DOCK_OK, or DOCK_ETIMEOUT for this ligand    */
  float best_fp32[DOCK_N_BEST];  /* FP32 scores of the best individuals, sorted
                                    by (score, index)                           */
  double best_fp64[DOCK_N_BEST]; /* the same poses rescored in FP64               */
  int32_t best_index[DOCK_N_BEST];/* their index in the final population          */
  float genotype[DOCK_N_BEST][DOCK_MAX_GENES];
  uint64_t exact_evals;          /* exact FP32 scorings done for this ligand
                                    (local-search probes included)              */
  uint64_t surrogate_evals;      /* surrogate evaluations (0 in plain mode)       */
} dock_result;

/* Waits (polling, at most timeout_ns; 0 = no limit) for the job, then copies
 * min(cap, n_ligands) results in input order to out (host).
 * Errors: DOCK_ETIMEOUT (still running: call again later), DOCK_EDEVICE (a
 * kernel set its status word), DOCK_ECUDA, DOCK_EINVAL. */
int dock_results(dock_job *job, dock_result *out, int32_t cap, uint64_t timeout_ns);

/* Device pointer of the job's final population (genotypes, scores) in the
 * layout above; valid until dock_job_destroy. */
int dock_job_population(const dock_job *job, const float **genotypes, const float **scores);
void dock_job_destroy(dock_job *job);

/* ------------------------------------------------------------------------ */
/* Scoring of given poses (Algorithm 1 then Algorithm 2, no search).         */
/* ------------------------------------------------------------------------ */
/* pose_ligand: device [n_poses] ligand index of each pose; genotypes: device
 * [n_poses][DOCK_MAX_GENES] (genes beyond G_l ignored); scores: device
 * [n_poses] FP32 output; coords: optional device [n_poses][DOCK_MAX_ATOMS][3]
 * posed coordinates (atoms beyond n_l untouched). fp64 = 1 scores in FP64 on
 * the GPU (the rescoring path) and writes scores64 (device [n_poses]) instead
 * of scores. Asynchronous on stream.
 * Errors: DOCK_EINVAL, DOCK_ECUDA. */
int dock_score(dock_pocket *pocket, dock_ligands *ligands, const int32_t *pose_ligand,
               const float *genotypes, int64_t n_poses, float *scores, double *scores64,
               float *coords, int32_t fp64, void *stream);

/* Scores (device FP32 [n_poses]) of caller-given poses with the pairwise
 * inter-energy: for every ligand atom, every protein atom within the 8 A
 * cutoff through the same pair terms as the intra pairs (the sum the grid maps
 * approximate; Algorithm 2's inter loop over nearby protein atoms, Section V),
 * plus the intra-energy. There is no grid box and no outside penalty, so the
 * score is invariant under a rigid motion of protein and ligand together.
 * FP32 with compensated sums; pose_ligand and genotypes as for dock_score;
 * pose_ligand entries outside [0, n_ligands) score NaN. Asynchronous on stream. */
int dock_score_pairwise(dock_pocket *pocket, dock_ligands *ligands, const int32_t *pose_ligand,
                        const float *genotypes, int64_t n_poses, float *scores, void *stream);

/* Solis-Wets refinement (see dock_ls_params) of caller-given poses: pose i
 * (ligand pose_ligand[i], genotype genotypes[i], layout as for dock_score) is
 * scored, then refined with the random-number counters of individual i of
 * generation `generation` of a search with `seed`; the refined genotype
 * replaces genotypes[i] (genes beyond G_l untouched) and its FP32 score is
 * written to scores[i]. Eight lanes per pose. trace: optional device
 * [n_poses][2 + 2 ls->max_its] as for dock_search_params.trace_ls. evals:
 * optional device [n_poses] uint32 probes scored. A pose whose pose_ligand
 * entry is outside [0, n_ligands) keeps its genotype and scores NaN.
 * Asynchronous on stream.
 * Errors: DOCK_EINVAL, DOCK_ECUDA. */
int dock_local_search(dock_pocket *pocket, dock_ligands *ligands, const dock_ls_params *ls,
                      uint64_t seed, uint32_t generation, const int32_t *pose_ligand,
                      int64_t n_poses, float *genotypes, float *scores, float *trace,
                      uint32_t *evals, void *stream);

/* ------------------------------------------------------------------------ */
/* Search without device allocation                                          */
/* ------------------------------------------------------------------------ */
/* The paper has no counterpart to this call; it serves callers that cannot
 * allocate GPU memory while they run: code whose device memory belongs to
 * another framework's pool, or that runs under a rule forbidding
 * cudaMalloc/cudaFree after start-up (every other search call here allocates
 * its working buffers on first use). dock_batch_noalloc runs the same plain
 * search as dock_batch (same kernels, same genotypes and scores for the same
 * seed; work items are queued in input order instead of largest first, and
 * no CUDA graph is used) and writes one dock_result per ligand to `results`,
 * a caller-owned device buffer of n_ligands records. All its working buffers
 * (populations, scores, per-generation best keys, queue counters, work
 * items, status words) live in one fixed device array of
 * DOCK_NOALLOC_SCRATCH_BYTES inside the library, which every GPU that loads
 * the library holds until the process exits. The call allocates nothing:
 * no cudaMalloc, cudaFree, host heap or allocating library routine.
 *  - Limits: at most DOCK_NOALLOC_MAX_LIGANDS ligands, and the search's
 *    buffers (about 8 bytes per gene of the population, 8 per pose score
 *    and 8 per ligand and generation) must fit the array; larger requests
 *    return DOCK_EINVAL with the bytes needed in dock_last_error().
 *    lanes_per_pose must be 0; use_graph is ignored.
 *  - The first call on a device looks up the array's device address with
 *    that device current; make that first call before any stream capture.
 *  - Every call shares the array and leaves its contents behind (each call
 *    clears what must start at zero). Calls that overlap on the GPU (other
 *    streams, other host threads) race on it: serialise them.
 *  - Asynchronous on stream: synchronise it before reading `results`. A
 *    device deadline (timeout_ns) shows as status DOCK_ETIMEOUT in the
 *    result records.
 * Errors: DOCK_EINVAL, DOCK_ECUDA. */
#define DOCK_NOALLOC_SCRATCH_BYTES (8u * 1024u * 1024u)
#define DOCK_NOALLOC_MAX_LIGANDS 64
int dock_batch_noalloc(dock_pocket *pocket, dock_ligands *ligands, const dock_search_params *params,
                       dock_result *results, void *stream);

/* ------------------------------------------------------------------------ */
/* Learned pre-screen (not in the paper: an MLP surrogate of the exact score) */
/* ------------------------------------------------------------------------ */
/* Per-pose features (128 values, BF16, row-major [pose][128]):
 *   [0, 56)    atom counts / 8 per (type t < 7, radial shell s < 8) around the
 *              pocket centre, shell width R/8 (last shell open): 8 t + s
 *   [56, 64)   sum of charges per shell; [64, 72) sum of |charge| per shell
 *   [72, 104)  sin, cos of torsion j at 72 + 2j, 73 + 2j (0 for j >= k)
 *   [104, 113) rotation matrix of the quaternion, row-major
 *   [113, 116) translation gene / R; 116: n / 100; 117: k / 16; rest 0.
 * Values are computed in FP32 and rounded to BF16 (round to nearest even).
 * The network is MLP 128 -> 256 -> 256 -> 256 -> 1 with GELU in its tanh form
 * (within 4.7e-4 of the erf form, under the BF16 rounding of the activations):
 * BF16 weights and activations, FP32 accumulation on the tensor cores, FP32
 * master weights; parameters packed as W1[128][256], b1[256], W2[256][256],
 * b2[256], W3[256][256], b3[256], W4[256], b4 (W stored [in][out]). */
#define DOCK_N_FEATURES 128
#define DOCK_MLP_N_PARAMS 164865

/* Poses the given genotypes (same layout as dock_score) and writes their
 * features (device BF16 [n_poses][128], as uint16_t) and, when scores is not
 * NULL, their exact FP32 scores. Asynchronous on stream.
 * Errors: DOCK_EINVAL (NULL buffers, pocket with more than 7 types), DOCK_ECUDA. */
int dock_features(dock_pocket *pocket, dock_ligands *ligands, const int32_t *pose_ligand,
                  const float *genotypes, int64_t n_poses, uint16_t *features, float *scores,
                  void *stream);

/* The same for whole populations in the search's genotype layout
 * (dock_batch's trace or population buffers: ligand l, individual i at
 * geno_off[l] + i * G_l for the given pop): row r = ligand r / pop,
 * individual r % pop; features [n_ligands * pop][128], scores optional.
 * Synchronises stream before returning. */
int dock_features_population(dock_pocket *pocket, dock_ligands *ligands, int32_t pop,
                             const float *genotypes, uint16_t *features, float *scores,
                             void *stream);

typedef struct {
  int32_t epochs;      /* passes over the training set                        */
  int32_t batch;       /* rows per step, a multiple of 128, <= 65536 (4096)    */
  float lr;            /* Adam learning rate (1e-3); beta 0.9 / 0.999, eps 1e-8 */
  float score_clip;    /* targets are min(score, clip), standardised by their
                          mean and standard deviation over the training set    */
  uint64_t seed;       /* order of the rows: batch position r visits row
                          pi(r), pi a bijection of [0, n) keyed by seed (a
                          four-round Feistel network on 2h-bit words, 4^h >= n,
                          round function the SplitMix64 mix of R xor
                          mix(seed + (i + 1) 0x9E3779B97F4A7C15) mod 2^h,
                          cycle-walked into [0, n)); the same every epoch     */
} dock_train_params;

/* Creates a network with He-normal weights drawn from seed and zero biases. */
int dock_surrogate_create(uint64_t seed, void *stream, dock_surrogate **out);
void dock_surrogate_destroy(dock_surrogate *surrogate);
/* Host copies of the FP32 master parameters (DOCK_MLP_N_PARAMS) and of the
 * target standardisation (prediction = output * t_std + t_mean). */
int dock_surrogate_set_params(dock_surrogate *surrogate, const float *params, float t_mean,
                              float t_std, float t_clip, void *stream);
int dock_surrogate_get_params(const dock_surrogate *surrogate, float *params, float *t_mean,
                              float *t_std, float *t_clip);
/* Predicted scores (device FP32 [n]) of device BF16 features [n][128] (16-byte
 * aligned), by the fused tensor-core forward pass. Returns once the scores are
 * written; DOCK_EDEVICE if a device-side wait ran out (those rows are NaN). */
int dock_surrogate_predict(dock_surrogate *surrogate, const uint16_t *features, int64_t n,
                           float *out, void *stream);
/* Gradient (device FP32, packed like the parameters) of
 * mean over n rows of (output - target)^2, targets used as given; n <= 65536.
 * *loss (host, optional) receives the loss; waits for the stream. */
int dock_surrogate_gradients(dock_surrogate *surrogate, const uint16_t *features,
                             const float *targets, int32_t n, float *grad, float *loss,
                             void *stream);
/* Trains with Adam (Kingma & Ba 2015: m, v with bias correction by step
 * count t from 1; FP32 masters, moments and update) on (features [n][128]
 * BF16, exact scores [n]) device arrays, one step per batch of the row order
 * above; loss_per_epoch (host, optional, [epochs]) gets the loss of each
 * epoch's last batch in standardised units. Waits for the stream. */
int dock_surrogate_train(dock_surrogate *surrogate, const uint16_t *features,
                         const float *scores, int64_t n, const dock_train_params *params,
                         float *loss_per_epoch, void *stream);

/* ------------------------------------------------------------------------ */
/* Autotuner of the search kernel's launch shape                             */
/* ------------------------------------------------------------------------ */
#define DOCK_TUNE_MAX 16
typedef struct {
  int32_t n;                               /* shapes measured                */
  int32_t threads[DOCK_TUNE_MAX];          /* CTA threads                    */
  int32_t atoms_per_lane[DOCK_TUNE_MAX];   /* shared-memory atoms per lane   */
  float ms_per_generation[DOCK_TUNE_MAX];  /* device time of one GA generation
                                              (best of two short searches)    */
  int32_t best;                            /* index of the chosen shape       */
} dock_tune_table;

/* Times the plain search (with the inter-energy params->inter names; no local
 * search) on this ligand set for each candidate launch shape
 * (CTA threads in {64, 128} x shared-memory atoms per lane in {8 .. 32}; a
 * ligand of n atoms then runs with the smallest L in {1, 2, 4, 8} lanes per
 * pose with L * atoms_per_lane >= n), picks the fastest (ties to the earlier
 * shape), records the table and keeps the pick on the ligand set: later
 * dock_batch calls with lanes_per_pose = 0 use it. Runs short searches
 * (min(max(generations, 2), 4) generations) on stream and waits for them;
 * results do not depend on the shape beyond FP32 summation order.
 * Errors: DOCK_EINVAL (surrogate mode, forced lanes, or an invalid inter),
 * DOCK_ENOMEM, DOCK_ECUDA. */
int dock_autotune(dock_pocket *pocket, dock_ligands *ligands, const dock_search_params *params,
                  void *stream, dock_tune_table *table);

/* Profiling aid: device time of the search-kernel launches of a job enqueued
 * while the environment variable DOCK_PROFILE_LAUNCHES was set (CUDA events
 * around each generation's launch on the job's stream; no graph). Waits for
 * the job. *ms_total = summed milliseconds, *launches = number of launches
 * (0 when the job was not profiled). */
int dock_job_kernel_time(const dock_job *job, double *ms_total, int32_t *launches);

/* Measurement aid (the paper has no counterpart): the device's FP32
 * fused-multiply-add rate (*fp32_tflops, TFLOP/s, FMA = 2 flops) and its
 * special-function rate (*mufu_tops, ex2 per second in units of 1e12), each
 * measured by a kernel of independent dependency chains on every SM, timed
 * with events on stream (best of three after a warm-up run); the rooflines
 * of the scoring kernels divide by these instead of unit counts times the
 * clock. Allocates and frees 4 bytes; waits for stream. Errors: DOCK_EINVAL
 * (NULL output), DOCK_ENOMEM, DOCK_ECUDA. */
int dock_measure_peaks(double *fp32_tflops, double *mufu_tops, void *stream);

const char *dock_last_error(void);

/* Library build string (architecture, version). */
const char *dock_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DOCK_H */
