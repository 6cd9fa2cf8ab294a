// Ensemble statistics of the per-trajectory indicators, and the pipe probe.
//
// Statistics (an ensemble statistic like the density F of Sec. IV): a
// histogram of log10 chi over [-8, 1) in 200 bins, the chaotic count, the
// maximum energy error and Welford mean / second moment of each momentum
// component.  Pass 1: every block reduces a grid-stride share of the
// trajectories (shared-memory histogram; per-thread Welford accumulators
// merged by a fixed warp-shuffle tree, then across the block's warps) into one
// partial in the context's scratch.
// Pass 2: the partials are merged in block order, so the result is
// deterministic.
#include <math.h>

#include "kernels.cuh"

namespace arnold {

namespace {

constexpr int kStatsThreads = 256;

struct Acc {
  double cnt, mean[3], m2[3], demax;
  unsigned long long chaotic, under, over;
};

__device__ __forceinline__ void acc_zero(Acc& a) {
  a.cnt = 0.0;
  for (int c = 0; c < 3; ++c) { a.mean[c] = 0.0; a.m2[c] = 0.0; }
  a.demax = 0.0;
  a.chaotic = a.under = a.over = 0;
}

// Chan-Golub-LeVeque merge of two Welford accumulators.
__device__ __forceinline__ void merge(Acc& a, const Acc& b) {
  const double n = a.cnt + b.cnt;
  if (b.cnt > 0.0) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double d = b.mean[c] - a.mean[c];
      a.mean[c] = a.mean[c] + d * (b.cnt / n);
      a.m2[c] = a.m2[c] + b.m2[c] + d * d * (a.cnt * b.cnt / n);
    }
    a.cnt = n;
  }
  a.demax = fmax(a.demax, b.demax);
  a.chaotic += b.chaotic;
  a.under += b.under;
  a.over += b.over;
}

// Lane l merges lane l + o for o = 16, 8, 4, 2, 1 (a fixed tree, so the result
// does not depend on timing); lane 0 ends with the warp's accumulator.
__device__ __forceinline__ void warp_merge(Acc& a) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    Acc b;
    b.cnt = __shfl_down_sync(0xffffffffu, a.cnt, o);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      b.mean[c] = __shfl_down_sync(0xffffffffu, a.mean[c], o);
      b.m2[c] = __shfl_down_sync(0xffffffffu, a.m2[c], o);
    }
    b.demax = __shfl_down_sync(0xffffffffu, a.demax, o);
    b.chaotic = __shfl_down_sync(0xffffffffu, a.chaotic, o);
    b.under = __shfl_down_sync(0xffffffffu, a.under, o);
    b.over = __shfl_down_sync(0xffffffffu, a.over, o);
    if ((threadIdx.x & 31) + o < 32) merge(a, b);
  }
}

__global__ void __launch_bounds__(kStatsThreads) k_stats_partial(long long n, const double* __restrict__ chi,
                                                                 const double* __restrict__ dE,
                                                                 const double* __restrict__ p, double threshold,
                                                                 StatsPartial* __restrict__ partials) {
  __shared__ unsigned int hist[ARNOLD_HIST_BINS];
  __shared__ Acc red[kStatsThreads / 32];
  for (int k = threadIdx.x; k < ARNOLD_HIST_BINS; k += blockDim.x) hist[k] = 0;
  __syncthreads();
  Acc a;
  acc_zero(a);
  const double scale = (double)ARNOLD_HIST_BINS / 9.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double x = chi[i];
    if (x > threshold) a.chaotic++;
    if (!(x > 0.0)) {
      a.under++;
    } else {
      const double uu = (log10(x) - (-8.0)) * scale;
      if (uu < 0.0) a.under++;
      else if (uu >= (double)ARNOLD_HIST_BINS) a.over++;
      else atomicAdd(&hist[(int)floor(uu)], 1u);
    }
    if (dE) a.demax = fmax(a.demax, dE[i]);
    a.cnt += 1.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double xv = p[c * n + i];
      const double d = xv - a.mean[c];
      a.mean[c] += d / a.cnt;
      a.m2[c] += d * (xv - a.mean[c]);
    }
  }
  warp_merge(a);
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  if ((threadIdx.x & 31) == 0) red[warp] = a;
  __syncthreads();
  if (warp == 0) {   // the warps' accumulators, merged by the same tree
    Acc w;
    if (threadIdx.x < nwarps) w = red[threadIdx.x];
    else acc_zero(w);
    warp_merge(w);
    if (threadIdx.x == 0) red[0] = w;
  }
  __syncthreads();
  StatsPartial& out = partials[blockIdx.x];
  for (int k = threadIdx.x; k < ARNOLD_HIST_BINS; k += blockDim.x) out.hist[k] = hist[k];
  if (threadIdx.x == 0) {
    const Acc& r = red[0];
    out.under = r.under;
    out.over = r.over;
    out.chaotic = r.chaotic;
    out.n = (unsigned long long)r.cnt;
    out.dE_max = r.demax;
    for (int c = 0; c < 3; ++c) { out.mean[c] = r.mean[c]; out.m2[c] = r.m2[c]; }
  }
}

__global__ void k_stats_merge(const StatsPartial* __restrict__ partials, int np, StatsPartial* __restrict__ out) {
  for (int k = threadIdx.x; k < ARNOLD_HIST_BINS; k += blockDim.x) {
    unsigned long long s = 0;
    for (int b = 0; b < np; ++b) s += partials[b].hist[k];
    out->hist[k] = s;
  }
  if (threadIdx.x == 0) {
    Acc a;
    acc_zero(a);
    for (int b = 0; b < np; ++b) {
      Acc x;
      x.cnt = (double)partials[b].n;
      for (int c = 0; c < 3; ++c) { x.mean[c] = partials[b].mean[c]; x.m2[c] = partials[b].m2[c]; }
      x.demax = partials[b].dE_max;
      x.chaotic = partials[b].chaotic;
      x.under = partials[b].under;
      x.over = partials[b].over;
      merge(a, x);
    }
    out->n = (unsigned long long)a.cnt;
    out->under = a.under;
    out->over = a.over;
    out->chaotic = a.chaotic;
    out->dE_max = a.demax;
    for (int c = 0; c < 3; ++c) { out->mean[c] = a.mean[c]; out->m2[c] = a.m2[c]; }
  }
}

// ------------------------------------------------------------------ probe ---
// Eight independent dependency chains per thread; the compiler keeps them.
template <int KIND>
__global__ void k_probe(int iters, double* sink) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double d[8];
  float f[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) { d[k] = 1.0 + t * 1e-9 + k; f[k] = 1.0f + t * 1e-7f + k; }
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (KIND == 0) d[k] = fma(d[k], 0.999999, 1e-7);
      if (KIND == 1) f[k] = fmaf(f[k], 0.99999f, 1e-5f);
      if (KIND == 2) f[k] = __sinf(f[k]);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += d[k] + (double)f[k];
  sink[t] = s;
}

}  // namespace

cudaError_t launch_stats(long long n, const double* chi, const double* dE, const double* p, double threshold,
                         StatsPartial* partials, int grid, StatsPartial* out, cudaStream_t st) {
  k_stats_partial<<<grid, kStatsThreads, 0, st>>>(n, chi, dE, p, threshold, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_stats_merge<<<1, 256, 0, st>>>(partials, grid, out);
  return cudaGetLastError();
}

cudaError_t launch_probe(int kind, int grid, int block, int iters, double* sink, cudaStream_t st) {
  if (kind == 0) k_probe<0><<<grid, block, 0, st>>>(iters, sink);
  else if (kind == 1) k_probe<1><<<grid, block, 0, st>>>(iters, sink);
  else if (kind == 2) k_probe<2><<<grid, block, 0, st>>>(iters, sink);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace arnold
