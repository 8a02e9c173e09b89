// dock_batch_noalloc: the plain search of dock_batch for callers that cannot
// allocate device memory while they run, for example code whose GPU memory
// is owned by another framework's pool or that runs under a policy that
// forbids cudaMalloc/cudaFree after start-up. Every working buffer of the
// search (population and score ping-pong buffers, per-generation best keys,
// queue counters, work items, status words) lives in one fixed static device
// array of this file instead of memory allocated per call.
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "handles.h"
#include "nvtx_range.h"

namespace dk {
namespace {

// The scratch array. Every GPU that loads the library holds it until the
// process exits; all calls on a device share it.
static __device__ __align__(256) unsigned char g_noalloc_scratch[DOCK_NOALLOC_SCRATCH_BYTES];

// Device addresses of the array, one per device, filled on the first call on
// that device (host code may not use the symbol itself as an address).
constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_setup_mu;

int fail(int st, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vset_error(st, fmt, ap);
  va_end(ap);
  return st;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Work items of all ligands, grouped by lanes per pose (8, 4, 2, 1; input
// order within a group, group g starting at item group_begin[g]), and the
// genotype offsets; a single thread, at most DOCK_NOALLOC_MAX_LIGANDS ligands.
__global__ void noalloc_items_kernel(const LigInfo *ligs, int n_ligands, int pop, int threads,
                                     int atoms_per_lane, int4 group_begin, Item *items,
                                     int64_t *geno_off) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int next[4] = {group_begin.x, group_begin.y, group_begin.z, group_begin.w};
  int64_t g = 0;
  for (int l = 0; l < n_ligands; ++l) {
    const LigInfo I = ligs[l];
    geno_off[l] = g;
    g += (int64_t)pop * (7 + I.k);
    int L = 1;
    while (L * atoms_per_lane < I.n && L < 8) L <<= 1;
    const int grp = L == 8 ? 0 : (L == 4 ? 1 : (L == 2 ? 2 : 3));
    const int S = threads / L;
    for (int t = 0; t * S < pop; ++t) items[next[grp]++] = Item{l, (int16_t)t, (int8_t)L, 0};
  }
}

}  // namespace
}  // namespace dk

extern "C" int dock_batch_noalloc(dock_pocket *P, dock_ligands *L, const dock_search_params *sp,
                                  dock_result *results, void *stream) {
  const dk::NvtxRange nvtx_range("dock_batch_noalloc");
  using namespace dk;
  if (!P || !L || !sp || !results) return fail(DOCK_EINVAL, "dock_batch_noalloc: NULL argument");
  if (sp->pop < 2 || sp->pop > DOCK_MAX_POP)
    return fail(DOCK_EINVAL, "dock_batch_noalloc: pop %d", sp->pop);
  if (sp->generations < 1)
    return fail(DOCK_EINVAL, "dock_batch_noalloc: generations %d", sp->generations);
  if (!(sp->p_cross >= 0 && sp->p_cross <= 1 && sp->p_mut >= 0 && sp->p_mut <= 1))
    return fail(DOCK_EINVAL, "dock_batch_noalloc: probabilities out of [0, 1]");
  if (sp->mode != DOCK_MODE_PLAIN)
    return fail(DOCK_EINVAL, "dock_batch_noalloc: only the plain search (mode 0)");
  if (sp->resume_genotypes != nullptr)
    return fail(DOCK_EINVAL, "dock_batch_noalloc: no resume (resume_genotypes must be NULL)");
  if (sp->ls.rate != 0.0f)
    return fail(DOCK_EINVAL, "dock_batch_noalloc: no local search (ls.rate must be 0)");
  if (sp->inter != DOCK_INTER_GRID)
    return fail(DOCK_EINVAL, "dock_batch_noalloc: grid inter-energy only (inter must be 0)");
  if (sp->lanes_per_pose != 0)
    return fail(DOCK_EINVAL, "dock_batch_noalloc: lanes_per_pose must be 0 (picked by size)");
  const int nl = L->n_ligands, pop = sp->pop, gens = sp->generations;
  if (nl > DOCK_NOALLOC_MAX_LIGANDS)
    return fail(DOCK_EINVAL, "dock_batch_noalloc: %d ligands (at most %d)", nl,
                DOCK_NOALLOC_MAX_LIGANDS);
  if (L->device < 0 || L->device >= kMaxDevices)
    return fail(DOCK_EINVAL, "dock_batch_noalloc: device %d", L->device);
  cudaError_t e = cudaSetDevice(L->device);
  if (e != cudaSuccess) return fail(DOCK_ECUDA, "dock_batch_noalloc: %s", cudaGetErrorString(e));
  // set-up, once per device, with the device current
  void *base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[L->device]) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p)
        return fail(DOCK_ECUDA, "dock_batch_noalloc: scratch address: %s", cudaGetErrorString(e));
      g_scratch_addr[L->device] = p;
    }
    base = g_scratch_addr[L->device];
  }
  // launch shape (as dock_batch with its defaults)
  const int threads = 128;
  int apl = 16;
  if (L->max_atoms > 8 * apl) apl = (L->max_atoms + 7) / 8;
  // sizes of the working buffers
  int64_t total_genes = 0, n_items = 0;
  int64_t group_items[4] = {0, 0, 0, 0};  // lanes per pose 8, 4, 2, 1
  for (int l = 0; l < nl; ++l) {
    const LigInfo &I = L->info[l];
    total_genes += (int64_t)pop * (7 + I.k);
    const int Ln = lanes_for(I.n, apl, 0);
    const int S = threads / Ln;
    group_items[Ln == 8 ? 0 : (Ln == 4 ? 1 : (Ln == 2 ? 2 : 3))] += (pop + S - 1) / S;
    n_items += (pop + S - 1) / S;
  }
  const size_t n_scores = (size_t)nl * pop;
  size_t off = 0;
  const size_t o_geno0 = off; off = align256(off + sizeof(float) * total_genes);
  const size_t o_geno1 = off; off = align256(off + sizeof(float) * total_genes);
  const size_t o_sc0 = off; off = align256(off + sizeof(float) * n_scores);
  const size_t o_sc1 = off; off = align256(off + sizeof(float) * n_scores);
  const size_t o_best = off; off = align256(off + sizeof(unsigned long long) * (size_t)gens * nl);
  const size_t o_cnt = off; off = align256(off + sizeof(uint32_t) * gens * 4);
  const size_t o_items = off; off = align256(off + sizeof(Item) * n_items);
  const size_t o_goff = off; off = align256(off + sizeof(int64_t) * nl);
  const size_t o_stat = off; off = align256(off + sizeof(int32_t));
  const size_t o_dl = off; off = align256(off + sizeof(uint64_t));
  const size_t o_lst = off; off = align256(off + sizeof(int32_t) * nl);
  if (off > (size_t)DOCK_NOALLOC_SCRATCH_BYTES)
    return fail(DOCK_EINVAL,
                "dock_batch_noalloc: the search needs %zu bytes of scratch, more than the %zu "
                "reserved (fewer ligands, poses or generations)",
                off, (size_t)DOCK_NOALLOC_SCRATCH_BYTES);
  unsigned char *S0 = (unsigned char *)base;
  float *geno[2] = {(float *)(S0 + o_geno0), (float *)(S0 + o_geno1)};
  float *score[2] = {(float *)(S0 + o_sc0), (float *)(S0 + o_sc1)};
  unsigned long long *best = (unsigned long long *)(S0 + o_best);
  uint32_t *counters = (uint32_t *)(S0 + o_cnt);
  Item *items = (Item *)(S0 + o_items);
  int64_t *goff = (int64_t *)(S0 + o_goff);
  int32_t *status = (int32_t *)(S0 + o_stat);
  uint64_t *deadline = (uint64_t *)(S0 + o_dl);
  int32_t *lig_status = (int32_t *)(S0 + o_lst);

  // one launch per non-empty lanes-per-pose group, one after another
  static const int kGroupL[4] = {8, 4, 2, 1};
  int group_begin[4];
  int group_blocks[4] = {0, 0, 0, 0};
  int n_sm = 0;
  if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, L->device)) != cudaSuccess)
    return fail(DOCK_ECUDA, "dock_batch_noalloc: %s", cudaGetErrorString(e));
  for (int g = 0, b = 0; g < 4; b += (int)group_items[g], ++g) {
    group_begin[g] = b;
    if (!group_items[g]) continue;
    int per_sm = 0;
    if ((e = search_occupancy(threads, kGroupL[g], apl, &per_sm)) != cudaSuccess)
      return fail(DOCK_ECUDA, "dock_batch_noalloc: %s", cudaGetErrorString(e));
    if (per_sm < 1) return fail(DOCK_EINVAL, "dock_batch_noalloc: launch shape does not fit an SM");
    group_blocks[g] = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)per_sm * n_sm,
                                                                    group_items[g]));
  }
  cudaStream_t s = (cudaStream_t)stream;

  SearchArgs A;
  A.ligs = L->d_info;
  A.atoms = L->d_atoms;
  A.types = L->d_types;
  A.pair_rec = L->d_pair_rec;
  A.tors = L->d_tors;
  A.moves = L->d_moves;
  A.geno_off = goff;
  A.items = items;
  A.n_items = (int32_t)n_items;
  A.atoms_per_lane = apl;
  A.grid = grid_view(P);
  A.cx = P->center[0];
  A.cy = P->center[1];
  A.cz = P->center[2];
  A.radius = P->radius;
  A.pop = pop;
  A.seed = sp->seed;
  A.thr_cross = prob_threshold(sp->p_cross);
  A.thr_mut = prob_threshold(sp->p_mut);
  A.status = status;
  A.lig_status = lig_status;
  A.deadline = sp->timeout_ns ? deadline : nullptr;
  A.pw = pw_view(P);
  A.bounds = bounds_of(P, L, status);
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

#define NA_CU(call)                                                                   \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess)                                                            \
      return fail(DOCK_ECUDA, "dock_batch_noalloc: %s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)
  // the array keeps the previous call's contents: clear what starts at zero
  NA_CU(cudaMemsetAsync(counters, 0, sizeof(uint32_t) * gens * 4, s));
  NA_CU(cudaMemsetAsync(best, 0xFF, sizeof(unsigned long long) * (size_t)gens * nl, s));
  NA_CU(cudaMemsetAsync(status, 0, sizeof(int32_t), s));
  if (nl) NA_CU(cudaMemsetAsync(lig_status, 0, sizeof(int32_t) * nl, s));
  noalloc_items_kernel<<<1, 32, 0, s>>>(
      L->d_info, nl, pop, threads, apl,
      make_int4(group_begin[0], group_begin[1], group_begin[2], group_begin[3]), items, goff);
  NA_CU(cudaGetLastError());
  if (sp->timeout_ns) NA_CU(launch_set_deadline(deadline, sp->timeout_ns, s));
  for (int g = 0; g < gens; ++g) {
    SearchArgs a = A;
    a.gen = g;
    a.geno_prev = geno[(g + 1) & 1];
    a.geno_next = geno[g & 1];
    a.score_prev = score[(g + 1) & 1];
    a.score_next = score[g & 1];
    a.best_prev = g ? best + (size_t)(g - 1) * nl : nullptr;
    a.best_next = best + (size_t)g * nl;
    for (int gr = 0; gr < 4; ++gr) {
      if (!group_items[gr]) continue;
      SearchArgs b = a;
      b.items = items + group_begin[gr];
      b.n_items = (int32_t)group_items[gr];
      b.counter = counters + (size_t)g * 4 + gr;
      NA_CU(launch_search(b, group_blocks[gr], threads, kGroupL[gr], s));
    }
    if (sp->trace_genotypes && total_genes)
      NA_CU(cudaMemcpyAsync(sp->trace_genotypes + (size_t)g * total_genes, geno[g & 1],
                            sizeof(float) * total_genes, cudaMemcpyDeviceToDevice, s));
    if (sp->trace_scores && n_scores)
      NA_CU(cudaMemcpyAsync(sp->trace_scores + (size_t)g * n_scores, score[g & 1],
                            sizeof(float) * n_scores, cudaMemcpyDeviceToDevice, s));
  }
  NA_CU(launch_finalize_impl(F, L->d_centroid, nl, pop, goff, geno[(gens - 1) & 1],
                             score[(gens - 1) & 1], lig_status, status, (uint64_t)pop * gens, 0,
                             nullptr, P->ox, P->oy, P->oz, results, s));
#undef NA_CU
  return DOCK_OK;
}
