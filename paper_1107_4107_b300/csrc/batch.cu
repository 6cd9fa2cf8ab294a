// Batched persistent launch: many parameter sets (eps, h) with uneven ensemble
// sizes and step counts advanced by one CUDA-graph launch (compensated FP32).
//
// Plan (host): the run is cut into epochs of roughly equal GPU work; in epoch
// e every set that still has steps left advances min(len_e, remaining) steps.
// An epoch is a list of (set, number of tiles, steps) entries sorted by the
// cost of one tile (longest first), so work items (set, tile) are never
// stored: item k of the epoch maps to an entry by its tile prefix sum.
// Kernel: one persistent launch per epoch, grid = resident blocks; each block
// pops items with an atomic counter (no waits of any kind), loads the set's
// arguments and runs its tile with the same per-trajectory code as the
// single-ensemble kernel (run32.cuh), so batched and unbatched trajectories
// are bit-identical.  The graph: one memset of the epoch counters, the epoch
// launches in order, and a final kernel that advances the per-set step bases
// so that a replay continues every set where the previous one stopped.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "kernels.cuh"
#include "run32.cuh"

struct arnold_ctx;   // defined in api.cu

namespace arnold {

void fp32_tab(Tab32* tb);
// Accessors into arnold_ctx (api.cu).
int ctx_run_args32(arnold_ctx* c, RunArgs32* ra, Coef32* cf, const float2** scf);
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

// Register cap: two resident blocks of 256 threads per SM.
template <int M, bool TAN, int TPT>
__global__ void __launch_bounds__(256, 2) k_batch_fp32c(const RunArgs32* __restrict__ sets,
                                                     const Coef32* __restrict__ coefs,
                                                     const long long* __restrict__ base,
                                                     const EpochEntry* __restrict__ entries, EpochDesc ep,
                                                     int* __restrict__ counter, const float2* __restrict__ scf,
                                                     Tab32 tb) {
  extern __shared__ __align__(16) unsigned char smem[];
  float2* ssc = reinterpret_cast<float2*>(smem);
  __shared__ long long s_item;
  __shared__ Coef32 s_cf;
  for (int k = threadIdx.x; k <= tb.jmax; k += blockDim.x) ssc[k] = scf[k];
  const long long tile = (long long)blockDim.x * TPT;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const long long item = s_item;
    if (item >= ep.tiles) break;
    int e = ep.first;
    while (entries[e].tile_end <= item) ++e;   // <= 64 entries, sorted prefix
    const EpochEntry en = entries[e];
    const long long prev_end = e > ep.first ? entries[e - 1].tile_end : 0;
    const long long t_idx = item - prev_end;
    const RunArgs32& ra = sets[en.set];
    // the set's coefficients, staged in shared memory for the whole block
    {
      const float* src = reinterpret_cast<const float*>(coefs + en.set);
      float* dst = reinterpret_cast<float*>(&s_cf);
      for (int k = threadIdx.x; k < (int)(sizeof(Coef32) / sizeof(float)); k += blockDim.x) dst[k] = src[k];
    }
    __syncthreads();
    const Coef32& cf = s_cf;
    long long idx[TPT];
    int valid = 0;
    const long long i0 = t_idx * tile;
#pragma unroll
    for (int r = 0; r < TPT; ++r) {
      const long long i = i0 + threadIdx.x + (long long)r * blockDim.x;
      const bool ok = i < ra.n;
      idx[r] = ok ? i : ra.n - 1;
      valid |= ok ? (1 << r) : 0;
    }
    if (valid) run_traj32<M, TAN, false, TPT>(ra, cf, idx, valid, base[en.set] + en.step0_rel, en.nsteps, ssc, tb);
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

}  // namespace

}  // namespace arnold

using namespace arnold;

struct arnold_batch {
  int n_sets = 0;
  int scheme = 0, tangent = 1, device = 0;
  arnold_batch_tuning tune{};
  cudaStream_t stream = nullptr;
  std::vector<arnold_batch_set> sets;
  std::vector<arnold_ctx*> ctx;
  RunArgs32* d_sets = nullptr;
  Coef32* d_coefs = nullptr;
  long long* d_base = nullptr;
  long long* d_steps = nullptr;
  EpochEntry* d_entries = nullptr;
  int* d_counters = nullptr;
  std::vector<EpochDesc> epochs;
  const float2* scf = nullptr;
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

cudaError_t launch_any(const arnold_batch* b, int grid, size_t smem, const EpochDesc& ep, int* counter,
                       const Tab32& tb) {
  const int M = b->scheme == ARNOLD_SCHEME_YOSHIDA6A ? 7 : (b->scheme == ARNOLD_SCHEME_TRIPLEJUMP6 ? 9 : 1);
  const bool T = b->tangent;
  const int P = b->tune.traj_per_thread;
  const int B = b->tune.block_size;
#define ARNOLD_BATCH_LAUNCH(MM, TT, PP)                                                                            \
  if (M == MM && T == TT && P == PP)                                                                               \
    return launch_epoch<MM, TT, PP>(grid, B, smem, b->stream, b->d_sets, b->d_coefs, b->d_base, b->d_entries, ep, \
                                    counter, b->scf, tb);
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
  const int M = b->scheme == ARNOLD_SCHEME_YOSHIDA6A ? 7 : (b->scheme == ARNOLD_SCHEME_TRIPLEJUMP6 ? 9 : 1);
  const bool T = b->tangent;
  const int P = b->tune.traj_per_thread;
  const int B = b->tune.block_size;
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

int arnold_batch_create(const arnold_batch_set* sets, int n_sets, int scheme, int tangent,
                        const arnold_batch_tuning* tuning, int device, void* cuda_stream, arnold_batch** out) {
  if (out) *out = nullptr;
  if (!out || !sets || n_sets <= 0 || n_sets > 4096 || scheme < 0 || scheme > 2 || (tangent != 0 && tangent != 1))
    return ARNOLD_EINVAL;
  arnold_batch_tuning tu;
  arnold_batch_tuning_default(&tu);
  if (tuning) tu = *tuning;
  if (tu.block_size < 32 || tu.block_size > 256 || tu.block_size % 32 || (tu.traj_per_thread != 1 && tu.traj_per_thread != 2) ||
      tu.renorm_every < 1 || tu.epoch_ms < 1)
    return ARNOLD_EINVAL;
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
  b->tangent = tangent;
  b->device = device;
  b->tune = tu;
  b->stream = (cudaStream_t)cuda_stream;
  b->sets.assign(sets, sets + n_sets);
  int st = ARNOLD_OK;
  std::vector<RunArgs32> hra(n_sets);
  std::vector<Coef32> hcf(n_sets);
  std::vector<long long> hsteps(n_sets);
  for (int s = 0; s < n_sets && st == ARNOLD_OK; ++s) {
    arnold_params p;
    arnold_params_default(&p);
    p.eps = sets[s].eps;
    p.h = sets[s].h;
    p.scheme = scheme;
    p.precision = ARNOLD_FP32C;
    p.tangent = tangent;
    p.renorm_every = tu.renorm_every;
    arnold_ctx* c = nullptr;
    st = arnold_create(&p, sets[s].G * sets[s].G, device, cuda_stream, &c);
    if (st) break;
    b->ctx.push_back(c);
    st = ctx_run_args32(c, &hra[s], &hcf[s], &b->scf);
    hsteps[s] = sets[s].n_steps;
  }
  cudaError_t e = cudaSuccess;
  if (st == ARNOLD_OK) {
    e = cudaMalloc(&b->d_sets, sizeof(RunArgs32) * n_sets);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_coefs, sizeof(Coef32) * n_sets);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_base, sizeof(long long) * n_sets);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_steps, sizeof(long long) * n_sets);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_sets, hra.data(), sizeof(RunArgs32) * n_sets, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_coefs, hcf.data(), sizeof(Coef32) * n_sets, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_steps, hsteps.data(), sizeof(long long) * n_sets, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(b->d_base, 0, sizeof(long long) * n_sets);
    st = bstatus(e);
  }
  // ---- epoch plan ----
  std::vector<EpochEntry> entries;
  if (st == ARNOLD_OK) {
    const long long tile = (long long)tu.block_size * tu.traj_per_thread;
    const int m = scheme == ARNOLD_SCHEME_YOSHIDA6A ? 7 : (scheme == ARNOLD_SCHEME_TRIPLEJUMP6 ? 9 : 1);
    const double rate = 2.0e10 * 7.0 / m;                     // map-steps/s, FP32C estimate
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
    Tab32 tb;
    fp32_tab(&tb);
    const size_t smem = (size_t)(tb.jmax + 1) * sizeof(float2);
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
      e = launch_any(b, grid, smem, b->epochs[k], b->d_counters + k, tb);
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
