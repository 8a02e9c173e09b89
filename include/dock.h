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
 * of atoms, included intra pairs, torsions and torsion-moved atoms (sum over
 * torsions of the atoms each one rotates), and the bytes dock_load_ligands
 * copied to the device. Any output may be NULL. */
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
} dock_search_params;

typedef struct dock_job dock_job;

/* Enqueues the whole search for every ligand on stream and returns at once:
 * generation 0 draws the population, each later generation runs one GA step
 * (tournament selection, crossover, mutation, elitism 1) fused with pose
 * application and FP32 scoring with compensated (Kahan) sums; after the last
 * generation the best DOCK_N_BEST individuals of each ligand are re-posed and
 * rescored in FP64. The pocket and ligands must outlive the job.
 * Errors: DOCK_EINVAL, DOCK_ENOMEM, DOCK_ECUDA. */
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
  uint64_t exact_evals;          /* exact FP32 scorings done for this ligand      */
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

/* Profiling aid: device time of the search-kernel launches of a job enqueued
 * while the environment variable DOCK_PROFILE_LAUNCHES was set (CUDA events
 * around each generation's launch on the job's stream; no graph). Waits for
 * the job. *ms_total = summed milliseconds, *launches = number of launches
 * (0 when the job was not profiled). */
int dock_job_kernel_time(const dock_job *job, double *ms_total, int32_t *launches);

const char *dock_last_error(void);

/* Library build string (architecture, version). */
const char *dock_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DOCK_H */
