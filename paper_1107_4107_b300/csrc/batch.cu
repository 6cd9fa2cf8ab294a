// Batched persistent launch: many parameter sets (eps, h) with uneven ensemble
// sizes and step counts advanced by one CUDA-graph launch, in compensated FP32
// (FP32C) or double-float (DF64, DF64F).
//
// Plan (host): the run is cut into epochs of roughly equal GPU work; in epoch
// e every set that still has steps left advances min(len_e, remaining) steps.
// An epoch is a list of (set, number of tiles, steps) entries sorted by the
// cost of one tile (longest first), so work items (set, tile) are never
// stored: item k of the epoch maps to an entry by its tile prefix sum.
// Kernel: one persistent launch per epoch, grid = resident blocks; items are
// popped with an atomic counter (no waits of any kind), the next one fetched
// while the current tile runs, and the set's argument block and coefficients
// are staged in shared memory.  FP32C hands out warp-sized items (each warp
// its own tile of 32 * TPT trajectories and its own slot, no block barrier);
// the double-float kernel hands out block-sized ones (thread 0 fills the
// block's second slot, one barrier per item) -- each the faster of the two
// for its kernel.  Every tile runs the same per-trajectory code as the
// single-ensemble kernels (run32.cuh, rundf.cuh), so batched and unbatched
// trajectories are bit-identical.  The graph: one
// memset of the epoch counters, the epoch launches in order, and a final
// kernel that advances the per-set step bases so that a replay continues
// every set where the previous one stopped.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "kernels.cuh"
#include "run32.cuh"
#include "rundf.cuh"

struct arnold_ctx;   // defined in api.cu

namespace arnold {

void fp32_tab(Tab32* tb);
void df_tab(TabDF* tb);
// Accessors into arnold_ctx (api.cu).
int ctx_run_args(arnold_ctx* c, RunArgs32* ra, StepCoef* sc, const float2** scf, const float4** scd);
void ctx_add_steps(arnold_ctx* c, long long s);
long long ctx_steps(arnold_ctx* c);

namespace {

struct EpochEntry {     // one active set in one epoch
  int set;
  int nsteps;           // steps of this epoch for the set
  long long step0_rel;  // epoch start relative to the run start
  long long tile_end;   // inclusive prefix of tiles up to this entry
};

struct EpochDesc {
  int first;            // first entry
  int count;            // entries
  long long tiles;      // items of the epoch
};

// Locate item `item` of an epoch: its entry (set, steps) and tile index --
// the first entry whose tile prefix exceeds the item, by bisection (the
// prefixes increase; <= 4096 entries, so at most 12 probes).
__device__ __forceinline__ const EpochEntry& find_entry(const EpochEntry* __restrict__ entries, const EpochDesc& ep,
                                                       long long item, long long& t_idx) {
  int lo = ep.first, hi = ep.first + ep.count - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (entries[mid].tile_end <= item) lo = mid + 1;
    else hi = mid;
  }
  t_idx = item - (lo > ep.first ? entries[lo - 1].tile_end : 0);
  return entries[lo];
}

// FP32C hands out work per warp: a work item is one warp's tile (32 * TPT
// trajectories of one set), so no warp ever waits for another.  Each warp has
// its own shared slot for the set's argument block and coefficients.
constexpr int kMaxWarps = 8;   // blocks of at most 256 threads

// Copy set `set`'s argument block and coefficients into this warp's slot, the
// 32 lanes moving 4-byte words in turn; ends with the warp synchronised.
template <typename C>
__device__ __forceinline__ void stage_set(const RunArgs32* __restrict__ sets, const C* __restrict__ coefs, int set,
                                          RunArgs32* ra, C* cf, int lane) {
  static_assert(sizeof(RunArgs32) % 4 == 0 && sizeof(C) % 4 == 0, "argument blocks are whole words");
  const unsigned* s1 = reinterpret_cast<const unsigned*>(sets + set);
  unsigned* d1 = reinterpret_cast<unsigned*>(ra);
  for (int k = lane; k < (int)(sizeof(RunArgs32) / 4); k += 32) d1[k] = s1[k];
  const unsigned* s2 = reinterpret_cast<const unsigned*>(coefs + set);
  unsigned* d2 = reinterpret_cast<unsigned*>(cf);
  for (int k = lane; k < (int)(sizeof(C) / 4); k += 32) d2[k] = s2[k];
  __syncwarp();
}

// Lane 0 takes the next item off the epoch's counter; every lane gets it.
__device__ __forceinline__ int next_item(int* counter, int lane) {
  int item = 0;
  if (lane == 0) item = atomicAdd(counter, 1);
  return __shfl_sync(0xFFFFFFFFu, item, 0);
}

// Thread 0: pop the next work item into shared slot `slot` and stage its set's
// arguments and step coefficients beside it (the double-float kernel's
// block-sized items).  A block works on slot it & 1 in iteration it while
// thread 0 fills the other slot, which every thread last read before the
// barrier that opened iteration it; the barrier that opens iteration it + 1
// publishes it.  So each item costs one barrier, and the atomic's latency
// overlaps the tile's run.
template <typename C>
__device__ __forceinline__ void pop_item(int* counter, const EpochDesc& ep, const EpochEntry* __restrict__ entries,
                                         const RunArgs32* __restrict__ sets, const C* __restrict__ coefs,
                                         long long* s_item, RunArgs32* s_ra, C* s_cf, int slot) {
  const long long item = atomicAdd(counter, 1);
  s_item[slot] = item;
  if (item < ep.tiles) {
    long long t_idx;
    const int set = find_entry(entries, ep, item, t_idx).set;
    s_ra[slot] = sets[set];
    s_cf[slot] = coefs[set];
  }
}

// FP32C: warp-sized items (measured against block-sized ones: no barrier
// stalls, issue 83.8 -> 85.0 %, 1 % faster).  Register cap: two resident
// blocks of 256 threads per SM.
template <int M, bool TAN, int TPT>
__global__ void __launch_bounds__(256, 2) k_batch_fp32c(const RunArgs32* __restrict__ sets,
                                                     const Coef32* __restrict__ coefs,
                                                     const long long* __restrict__ base,
                                                     const EpochEntry* __restrict__ entries, EpochDesc ep,
                                                     int* __restrict__ counter, const float2* __restrict__ scf,
                                                     Tab32 tb) {
  extern __shared__ __align__(16) unsigned char smem[];
  float2* ssc = reinterpret_cast<float2*>(smem);
  __shared__ RunArgs32 s_ra[kMaxWarps];
  __shared__ Coef32 s_cf[kMaxWarps];
  for (int k = threadIdx.x; k <= tb.jmax; k += blockDim.x) ssc[k] = scf[k];
  __syncthreads();   // the table; the only block-wide barrier
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  RunArgs32& ra = s_ra[warp];
  Coef32& cf = s_cf[warp];
  int item = next_item(counter, lane);
  while (item < ep.tiles) {
    int next = 0;   // fetched now: the atomic's latency hides behind this tile
    if (lane == 0) next = atomicAdd(counter, 1);
    long long t_idx;
    const EpochEntry& en = find_entry(entries, ep, item, t_idx);
    stage_set(sets, coefs, en.set, &ra, &cf, lane);
    long long idx[TPT];
    int valid = 0;
    const long long i0 = t_idx * (32LL * TPT);
#pragma unroll
    for (int r = 0; r < TPT; ++r) {
      const long long i = i0 + lane + 32LL * r;
      const bool ok = i < ra.n;
      idx[r] = ok ? i : ra.n - 1;
      valid |= ok ? (1 << r) : 0;
    }
    if (valid) run_traj32<M, TAN, false, TPT>(ra, cf, idx, valid, base[en.set] + en.step0_rel, en.nsteps, ssc, tb);
    __syncwarp();   // every lane is done with the slot before it is restaged
    item = __shfl_sync(0xFFFFFFFFu, next, 0);
  }
}

// The double-float modes (one trajectory per thread; FAST = DF64F): a work item
// is one block's tile, popped by thread 0 into the other of two shared slots
// while the block runs the current one (one barrier per item).  Measured
// against warp-sized items for this kernel: 0.7 % faster (its items are long,
// and a quarter as many of them need staging).
template <int M, bool TAN, bool FAST>
__global__ void __launch_bounds__(256, 2) k_batch_df(const RunArgs32* __restrict__ sets,
                                                     const CoefDF* __restrict__ coefs,
                                                     const long long* __restrict__ base,
                                                     const EpochEntry* __restrict__ entries, EpochDesc ep,
                                                     int* __restrict__ counter, const float4* __restrict__ scd,
                                                     TabDF tb) {
  extern __shared__ __align__(16) unsigned char smem[];
  float4* stab = reinterpret_cast<float4*>(smem);
  __shared__ long long s_item[2];
  __shared__ RunArgs32 s_ra[2];
  __shared__ CoefDF s_cf[2];
  for (int k = threadIdx.x; k <= tb.mask; k += blockDim.x) stab[k] = scd[k];
  if (threadIdx.x == 0) pop_item(counter, ep, entries, sets, coefs, s_item, s_ra, s_cf, 0);
  for (int it = 0;; ++it) {
    __syncthreads();
    const int slot = it & 1;
    const long long item = s_item[slot];
    if (item >= ep.tiles) break;
    if (threadIdx.x == 0) pop_item(counter, ep, entries, sets, coefs, s_item, s_ra, s_cf, slot ^ 1);
    long long t_idx;
    const EpochEntry& en = find_entry(entries, ep, item, t_idx);
    const RunArgs32& ra = s_ra[slot];
    const long long i = t_idx * blockDim.x + threadIdx.x;
    if (i < ra.n) run_traj_df<M, TAN, FAST>(ra, s_cf[slot], i, base[en.set] + en.step0_rel, en.nsteps, stab, tb);
  }
}

__global__ void k_batch_advance(long long* base, const long long* steps, int n_sets) {
  for (int s = threadIdx.x; s < n_sets; s += blockDim.x) base[s] += steps[s];
}

template <int M, bool TAN, int TPT>
cudaError_t launch_epoch(int grid, int block, size_t smem, cudaStream_t st, const RunArgs32* sets, const Coef32* coefs,
                         const long long* base, const EpochEntry* entries, const EpochDesc& ep, int* counter,
                         const float2* scf, const Tab32& tb) {
  k_batch_fp32c<M, TAN, TPT><<<grid, block, smem, st>>>(sets, coefs, base, entries, ep, counter, scf, tb);
  return cudaGetLastError();
}

template <int M, bool TAN, int TPT>
int blocks_per_sm(int block, size_t smem) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_fp32c<M, TAN, TPT>, block, smem) != cudaSuccess)
    return 1;
  return nb > 0 ? nb : 1;
}

template <int M, bool TAN, bool FAST>
cudaError_t launch_epoch_df(int grid, int block, size_t smem, cudaStream_t st, const RunArgs32* sets,
                            const CoefDF* coefs, const long long* base, const EpochEntry* entries, const EpochDesc& ep,
                            int* counter, const float4* scd, const TabDF& tb) {
  k_batch_df<M, TAN, FAST><<<grid, block, smem, st>>>(sets, coefs, base, entries, ep, counter, scd, tb);
  return cudaGetLastError();
}

template <int M, bool TAN, bool FAST>
int blocks_per_sm_df(int block, size_t smem) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_df<M, TAN, FAST>, block, smem) != cudaSuccess)
    return 1;
  return nb > 0 ? nb : 1;
}

}  // namespace

}  // namespace arnold

using namespace arnold;

struct arnold_batch {
  int n_sets = 0;
  int scheme = 0, precision = ARNOLD_FP32C, tangent = 1, device = 0;
  arnold_batch_tuning tune{};
  cudaStream_t stream = nullptr;
  std::vector<arnold_batch_set> sets;
  std::vector<arnold_ctx*> ctx;
  RunArgs32* d_sets = nullptr;
  void* d_coefs = nullptr;      // Coef32[n_sets] (FP32C) or CoefDF[n_sets] (DF64, DF64F)
  long long* d_base = nullptr;
  long long* d_steps = nullptr;
  EpochEntry* d_entries = nullptr;
  int* d_counters = nullptr;
  std::vector<EpochDesc> epochs;
  const float2* scf = nullptr;  // FP32 sincos table (FP32C)
  const float4* scd = nullptr;  // double-float sincos table (DF64, DF64F)
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long launches = 0;
  long long total_steps = 0;    // map steps per run
  long long items = 0;
};

namespace {

int bstatus(cudaError_t e) {
  if (e == cudaSuccess) return ARNOLD_OK;
  if (e == cudaErrorMemoryAllocation) return ARNOLD_ENOMEM;
  return ARNOLD_ECUDA;
}

int kicks_of(int scheme) {
  return scheme == ARNOLD_SCHEME_YOSHIDA6A ? 7 : (scheme == ARNOLD_SCHEME_TRIPLEJUMP6 ? 9 : 1);
}

bool is_df(int precision) { return precision == ARNOLD_DF64 || precision == ARNOLD_DF64F; }

// Shared memory of one block: the mode's sincos table.
size_t table_smem(int precision) {
  if (is_df(precision)) {
    TabDF tb;
    df_tab(&tb);
    return (size_t)(tb.mask + 1) * sizeof(float4);
  }
  Tab32 tb;
  fp32_tab(&tb);
  return (size_t)(tb.jmax + 1) * sizeof(float2);
}

cudaError_t launch_any(const arnold_batch* b, int grid, size_t smem, const EpochDesc& ep, int* counter) {
  const int M = kicks_of(b->scheme);
  const bool T = b->tangent;
  const int B = b->tune.block_size;
  if (is_df(b->precision)) {
    TabDF tb;
    df_tab(&tb);
    const bool F = b->precision == ARNOLD_DF64F;
    const CoefDF* cf = (const CoefDF*)b->d_coefs;
#define ARNOLD_BATCH_LAUNCH_DF(MM, TT, FF)                                                                         \
  if (M == MM && T == TT && F == FF)                                                                               \
    return launch_epoch_df<MM, TT, FF>(grid, B, smem, b->stream, b->d_sets, cf, b->d_base, b->d_entries, ep, counter, \
                                       b->scd, tb);
    ARNOLD_BATCH_LAUNCH_DF(7, true, true)
    ARNOLD_BATCH_LAUNCH_DF(7, false, true)
    ARNOLD_BATCH_LAUNCH_DF(7, true, false)
    ARNOLD_BATCH_LAUNCH_DF(7, false, false)
    ARNOLD_BATCH_LAUNCH_DF(9, true, true)
    ARNOLD_BATCH_LAUNCH_DF(9, false, true)
    ARNOLD_BATCH_LAUNCH_DF(9, true, false)
    ARNOLD_BATCH_LAUNCH_DF(9, false, false)
    ARNOLD_BATCH_LAUNCH_DF(1, true, true)
    ARNOLD_BATCH_LAUNCH_DF(1, false, true)
    ARNOLD_BATCH_LAUNCH_DF(1, true, false)
    ARNOLD_BATCH_LAUNCH_DF(1, false, false)
#undef ARNOLD_BATCH_LAUNCH_DF
    return cudaErrorInvalidValue;
  }
  Tab32 tb;
  fp32_tab(&tb);
  const int P = b->tune.traj_per_thread;
  const Coef32* cf = (const Coef32*)b->d_coefs;
#define ARNOLD_BATCH_LAUNCH(MM, TT, PP)                                                                            \
  if (M == MM && T == TT && P == PP)                                                                               \
    return launch_epoch<MM, TT, PP>(grid, B, smem, b->stream, b->d_sets, cf, b->d_base, b->d_entries, ep, counter, \
                                    b->scf, tb);
  ARNOLD_BATCH_LAUNCH(7, true, 1)
  ARNOLD_BATCH_LAUNCH(7, true, 2)
  ARNOLD_BATCH_LAUNCH(7, false, 1)
  ARNOLD_BATCH_LAUNCH(7, false, 2)
  ARNOLD_BATCH_LAUNCH(9, true, 1)
  ARNOLD_BATCH_LAUNCH(9, true, 2)
  ARNOLD_BATCH_LAUNCH(9, false, 1)
  ARNOLD_BATCH_LAUNCH(9, false, 2)
  ARNOLD_BATCH_LAUNCH(1, true, 1)
  ARNOLD_BATCH_LAUNCH(1, true, 2)
  ARNOLD_BATCH_LAUNCH(1, false, 1)
  ARNOLD_BATCH_LAUNCH(1, false, 2)
#undef ARNOLD_BATCH_LAUNCH
  return cudaErrorInvalidValue;
}

int occupancy_any(const arnold_batch* b, size_t smem) {
  const int M = kicks_of(b->scheme);
  const bool T = b->tangent;
  const int B = b->tune.block_size;
  if (is_df(b->precision)) {
    const bool F = b->precision == ARNOLD_DF64F;
#define ARNOLD_BATCH_OCC_DF(MM, TT, FF) \
  if (M == MM && T == TT && F == FF) return blocks_per_sm_df<MM, TT, FF>(B, smem);
    ARNOLD_BATCH_OCC_DF(7, true, true)
    ARNOLD_BATCH_OCC_DF(7, false, true)
    ARNOLD_BATCH_OCC_DF(7, true, false)
    ARNOLD_BATCH_OCC_DF(7, false, false)
    ARNOLD_BATCH_OCC_DF(9, true, true)
    ARNOLD_BATCH_OCC_DF(9, false, true)
    ARNOLD_BATCH_OCC_DF(9, true, false)
    ARNOLD_BATCH_OCC_DF(9, false, false)
    ARNOLD_BATCH_OCC_DF(1, true, true)
    ARNOLD_BATCH_OCC_DF(1, false, true)
    ARNOLD_BATCH_OCC_DF(1, true, false)
    ARNOLD_BATCH_OCC_DF(1, false, false)
#undef ARNOLD_BATCH_OCC_DF
    return 1;
  }
  const int P = b->tune.traj_per_thread;
#define ARNOLD_BATCH_OCC(MM, TT, PP) \
  if (M == MM && T == TT && P == PP) return blocks_per_sm<MM, TT, PP>(B, smem);
  ARNOLD_BATCH_OCC(7, true, 1)
  ARNOLD_BATCH_OCC(7, true, 2)
  ARNOLD_BATCH_OCC(7, false, 1)
  ARNOLD_BATCH_OCC(7, false, 2)
  ARNOLD_BATCH_OCC(9, true, 1)
  ARNOLD_BATCH_OCC(9, true, 2)
  ARNOLD_BATCH_OCC(9, false, 1)
  ARNOLD_BATCH_OCC(9, false, 2)
  ARNOLD_BATCH_OCC(1, true, 1)
  ARNOLD_BATCH_OCC(1, true, 2)
  ARNOLD_BATCH_OCC(1, false, 1)
  ARNOLD_BATCH_OCC(1, false, 2)
#undef ARNOLD_BATCH_OCC
  return 1;
}

void free_batch(arnold_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  void* ptrs[] = {b->d_sets, b->d_coefs, b->d_base, b->d_steps, b->d_entries, b->d_counters};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (arnold_ctx* c : b->ctx) arnold_destroy(c);
}

}  // namespace

extern "C" {

void arnold_batch_tuning_default(arnold_batch_tuning* t) {
  if (!t) return;
  t->block_size = 256;
  t->traj_per_thread = 1;
  t->renorm_every = 100;
  t->epoch_ms = 200;
}

int arnold_batch_create(const arnold_batch_set* sets, int n_sets, int scheme, int precision, int tangent,
                        const arnold_batch_tuning* tuning, int device, void* cuda_stream, arnold_batch** out) {
  if (out) *out = nullptr;
  if (!out || !sets || n_sets <= 0 || n_sets > 4096 || scheme < 0 || scheme > 2 || (tangent != 0 && tangent != 1))
    return ARNOLD_EINVAL;
  if (precision != ARNOLD_FP32C && precision != ARNOLD_DF64 && precision != ARNOLD_DF64F) return ARNOLD_EINVAL;
  arnold_batch_tuning tu;
  arnold_batch_tuning_default(&tu);
  if (tuning) tu = *tuning;
  if (tu.block_size < 32 || tu.block_size > 256 || tu.block_size % 32 || (tu.traj_per_thread != 1 && tu.traj_per_thread != 2) ||
      tu.renorm_every < 1 || tu.epoch_ms < 1)
    return ARNOLD_EINVAL;
  if (is_df(precision) && tu.traj_per_thread != 1) return ARNOLD_EINVAL;
  for (int s = 0; s < n_sets; ++s) {
    const arnold_batch_set& q = sets[s];
    if (!(q.h != 0.0) || q.G <= 0 || q.G > (1 << 20) || q.n_steps < 0 || q.n_steps > (1LL << 40) ||
        !(q.E > 2.0 * fabs(q.eps)))
      return ARNOLD_EINVAL;
  }
  arnold_batch* b = new (std::nothrow) arnold_batch();
  if (!b) return ARNOLD_ENOMEM;
  b->n_sets = n_sets;
  b->scheme = scheme;
  b->precision = precision;
  b->tangent = tangent;
  b->device = device;
  b->tune = tu;
  b->stream = (cudaStream_t)cuda_stream;
  b->sets.assign(sets, sets + n_sets);
  int st = ARNOLD_OK;
  std::vector<RunArgs32> hra(n_sets);
  std::vector<Coef32> hcf(n_sets);
  std::vector<CoefDF> hcd(n_sets);
  std::vector<long long> hsteps(n_sets);
  for (int s = 0; s < n_sets && st == ARNOLD_OK; ++s) {
    arnold_params p;
    arnold_params_default(&p);
    p.eps = sets[s].eps;
    p.h = sets[s].h;
    p.scheme = scheme;
    p.precision = precision;
    p.tangent = tangent;
    p.renorm_every = tu.renorm_every;
    arnold_ctx* c = nullptr;
    st = arnold_create(&p, sets[s].G * sets[s].G, device, cuda_stream, &c);
    if (st) break;
    b->ctx.push_back(c);
    StepCoef sc;
    st = ctx_run_args(c, &hra[s], &sc, &b->scf, &b->scd);
    hcf[s] = coef32_from(sc);
    hcd[s] = coef_df_from(sc);
    hsteps[s] = sets[s].n_steps;
  }
  cudaError_t e = cudaSuccess;
  if (st == ARNOLD_OK) {
    const size_t cbytes = is_df(precision) ? sizeof(CoefDF) : sizeof(Coef32);
    const void* hc = is_df(precision) ? (const void*)hcd.data() : (const void*)hcf.data();
    e = cudaMalloc(&b->d_sets, sizeof(RunArgs32) * n_sets);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_coefs, cbytes * n_sets);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_base, sizeof(long long) * n_sets);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_steps, sizeof(long long) * n_sets);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_sets, hra.data(), sizeof(RunArgs32) * n_sets, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_coefs, hc, cbytes * n_sets, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_steps, hsteps.data(), sizeof(long long) * n_sets, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->d_base, 0, sizeof(long long) * n_sets);
    st = bstatus(e);
  }
  // ---- epoch plan ----
  std::vector<EpochEntry> entries;
  if (st == ARNOLD_OK) {
    // one warp's trajectories (FP32C) or one block's (double-float): see the kernels
    const long long tile = is_df(precision) ? (long long)tu.block_size : 32LL * tu.traj_per_thread;
    // map-steps/s estimates of each mode (7 kicks per step), for the epoch length only
    const double rate7 = precision == ARNOLD_FP32C ? 2.0e10 : (precision == ARNOLD_DF64F ? 1.1e10 : 7.0e9);
    const double rate = rate7 * 7.0 / kicks_of(scheme);
    const double target = rate * tu.epoch_ms * 1e-3;          // map steps per epoch
    long long done = 0, max_steps = 0;
    for (auto& q : b->sets) max_steps = std::max(max_steps, (long long)q.n_steps);
    for (auto& q : b->sets) b->total_steps += q.G * q.G * q.n_steps;
    while (done < max_steps) {
      double active_n = 0.0;
      for (auto& q : b->sets)
        if (q.n_steps > done) active_n += (double)(q.G * q.G);
      long long len = (long long)(target / active_n);
      len = std::max(16LL, std::min(len, 1LL << 30));
      len = std::min(len, max_steps - done);
      std::vector<EpochEntry> ep;
      for (int s = 0; s < n_sets; ++s) {
        if (sets[s].n_steps <= done) continue;
        EpochEntry en;
        en.set = s;
        en.nsteps = (int)std::min(len, (long long)sets[s].n_steps - done);
        en.step0_rel = done;
        en.tile_end = ((long long)sets[s].G * sets[s].G + tile - 1) / tile;   // tiles of this set, for now
        ep.push_back(en);
      }
      // longest tile first: cost of one tile = steps * trajectories in a tile (all full but the last)
      std::stable_sort(ep.begin(), ep.end(), [](const EpochEntry& a, const EpochEntry& b2) { return a.nsteps > b2.nsteps; });
      EpochDesc d;
      d.first = (int)entries.size();
      d.count = (int)ep.size();
      long long acc = 0;
      for (auto& en : ep) {
        acc += en.tile_end;
        en.tile_end = acc;
        entries.push_back(en);
      }
      d.tiles = acc;
      b->items += acc;
      b->epochs.push_back(d);
      done += len;
    }
    e = cudaMalloc(&b->d_entries, sizeof(EpochEntry) * std::max<size_t>(1, entries.size()));
    if (e == cudaSuccess && !entries.empty())
      e = cudaMemcpy(b->d_entries, entries.data(), sizeof(EpochEntry) * entries.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counters, sizeof(int) * std::max<size_t>(1, b->epochs.size()));
    st = bstatus(e);
  }
  if (st != ARNOLD_OK) {
    free_batch(b);
    delete b;
    return st;
  }
  *out = b;
  return ARNOLD_OK;
}

void arnold_batch_destroy(arnold_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  cudaStreamSynchronize(b->stream);
  free_batch(b);
  delete b;
}

int arnold_batch_init(arnold_batch* b) {
  if (!b) return ARNOLD_EINVAL;
  for (int s = 0; s < b->n_sets; ++s) {
    const int st = arnold_init_grid(b->ctx[s], b->sets[s].G, 0, b->sets[s].E, b->sets[s].seed, nullptr);
    if (st) return st;
  }
  cudaError_t e = cudaSetDevice(b->device);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_base, 0, sizeof(long long) * b->n_sets, b->stream);
  b->launches += b->n_sets;
  return bstatus(e);
}

int arnold_batch_run(arnold_batch* b) {
  if (!b) return ARNOLD_EINVAL;
  cudaError_t e = cudaSetDevice(b->device);
  if (e != cudaSuccess) return bstatus(e);
  if (!b->exec) {
    const size_t smem = table_smem(b->precision);
    int sms = 148;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    const int grid = sms * occupancy_any(b, smem);
    // capture on a private stream so that the caller's stream state is untouched
    cudaStream_t cs;
    e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e != cudaSuccess) return bstatus(e);
    cudaStream_t keep = b->stream;
    b->stream = cs;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_counters, 0, sizeof(int) * std::max<size_t>(1, b->epochs.size()), cs);
    for (size_t k = 0; k < b->epochs.size() && e == cudaSuccess; ++k)
      e = launch_any(b, grid, smem, b->epochs[k], b->d_counters + k);
    if (e == cudaSuccess) {
      k_batch_advance<<<1, 256, 0, cs>>>(b->d_base, b->d_steps, b->n_sets);
      e = cudaGetLastError();
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
    b->graph = g;
    b->stream = keep;
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return bstatus(e);
  }
  e = cudaGraphLaunch(b->exec, b->stream);
  if (e != cudaSuccess) return bstatus(e);
  b->launches += (long long)b->epochs.size() + 2;
  for (int s = 0; s < b->n_sets; ++s) ctx_add_steps(b->ctx[s], b->sets[s].n_steps);
  return ARNOLD_OK;
}

int arnold_batch_indicator(arnold_batch* b, int set, int kind, void* out, int ptr_kind) {
  if (!b || set < 0 || set >= b->n_sets) return ARNOLD_EINVAL;
  return arnold_indicator(b->ctx[set], kind, out, ptr_kind);
}

int arnold_batch_stats(arnold_batch* b, int set, arnold_stats* out) {
  if (!b || set < 0 || set >= b->n_sets) return ARNOLD_EINVAL;
  return arnold_stats_compute(b->ctx[set], out);
}

int arnold_batch_info(const arnold_batch* b, int64_t* epochs, int64_t* items, int64_t* map_steps_per_run) {
  if (!b) return ARNOLD_EINVAL;
  if (epochs) *epochs = (int64_t)b->epochs.size();
  if (items) *items = b->items;
  if (map_steps_per_run) *map_steps_per_run = b->total_steps;
  return ARNOLD_OK;
}

int arnold_batch_sync(arnold_batch* b) {
  if (!b) return ARNOLD_EINVAL;
  cudaError_t e = cudaSetDevice(b->device);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) return bstatus(e);
  for (arnold_ctx* c : b->ctx) {
    const int st = arnold_sync(c);
    if (st) return st;
  }
  return ARNOLD_OK;
}

int64_t arnold_batch_launch_count(const arnold_batch* b) { return b ? b->launches : -1; }

}  // extern "C"
