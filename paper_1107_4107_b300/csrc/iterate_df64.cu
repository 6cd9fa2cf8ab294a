// DF64 ensemble propagator: FP64-grade trajectories on the FP32 pipes.  The
// FAST instances (the DF64F mode) take their sines and cosines from
// sincos_df_fast (~3e-10) and keep everything else double-float.
//
// Same composite step and state layout as the compensated-FP32 path (float
// pairs for angles and momenta, exact TwoProd/TwoSum drifts), but every kick
// is evaluated in double-float (step_df.cuh): table sincos with the reduced
// argument kept as a pair and the force products split exactly, so the map
// is followed to ~1e-16 per operation like the FP64 kernel.  The tangent
// vector is double-float too (pair components and coefficients, TwoSum
// accumulation): on a regular orbit the tangent map is a shear whose growth
// an FP32 tangent biases.  Its norm and log at renormalisation are FP64.
#include "kernels.cuh"
#include "rundf.cuh"

namespace arnold {

namespace {

// The substep loop is not unrolled: a double-float kick is ~350 instructions,
// and seven unrolled copies overflow the instruction cache (ncu: issue stalls
// on instruction fetch); the loop reads its coefficients from shared memory.
template <int M, bool TAN, bool FAST>
__global__ void __launch_bounds__(256) k_iterate_df64(IterArgs a, TabDF tb, CoefDF cfg) {
  extern __shared__ __align__(16) unsigned char smem[];
  float4* stab = reinterpret_cast<float4*>(smem);
  __shared__ CoefDF cf;
  for (int k = threadIdx.x; k <= tb.mask; k += blockDim.x) stab[k] = a.scd[k];
  if (threadIdx.x == 0) cf = cfg;
  __syncthreads();
  RunArgs32 ra;
  ra.s = a.s;
  ra.f = a.f;
  ra.n = a.n;
  ra.R = a.R;
  ra.W = a.W;
  ra.h = a.h;
  ra.eps = a.eps;
  ra.flags = a.flags;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (long long)gridDim.x * blockDim.x)
    run_traj_df<M, TAN, FAST>(ra, cf, i, a.step0, a.nsteps, stab, tb);
}

template <int M, bool TAN, bool FAST>
cudaError_t launch_one(const IterArgs& a, const TabDF& tb, const CoefDF& cf, int block, int grid, cudaStream_t st) {
  const size_t smem = (size_t)(tb.mask + 1) * sizeof(float4);
  k_iterate_df64<M, TAN, FAST><<<grid, block, smem, st>>>(a, tb, cf);
  return cudaGetLastError();
}

template <int M, bool TAN, bool FAST>
int occ_one(const TabDF& tb, int block) {
  int nb = 0;
  const size_t smem = (size_t)(tb.mask + 1) * sizeof(float4);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_iterate_df64<M, TAN, FAST>, block, smem) != cudaSuccess)
    return 1;
  return nb > 0 ? nb : 1;
}

template <bool FAST>
cudaError_t launch_scheme(const IterArgs& a, const TabDF& tb, const CoefDF& cf, int scheme, bool tangent, int block,
                          int grid, cudaStream_t st) {
  switch (scheme) {
    case ARNOLD_SCHEME_YOSHIDA6A:
      return tangent ? launch_one<7, true, FAST>(a, tb, cf, block, grid, st)
                     : launch_one<7, false, FAST>(a, tb, cf, block, grid, st);
    case ARNOLD_SCHEME_TRIPLEJUMP6:
      return tangent ? launch_one<9, true, FAST>(a, tb, cf, block, grid, st)
                     : launch_one<9, false, FAST>(a, tb, cf, block, grid, st);
    case ARNOLD_SCHEME_LEAPFROG2:
      return tangent ? launch_one<1, true, FAST>(a, tb, cf, block, grid, st)
                     : launch_one<1, false, FAST>(a, tb, cf, block, grid, st);
  }
  return cudaErrorInvalidValue;
}

template <bool FAST>
int occ_scheme(const TabDF& tb, int scheme, bool tangent, int block) {
  switch (scheme) {
    case ARNOLD_SCHEME_YOSHIDA6A: return tangent ? occ_one<7, true, FAST>(tb, block) : occ_one<7, false, FAST>(tb, block);
    case ARNOLD_SCHEME_TRIPLEJUMP6:
      return tangent ? occ_one<9, true, FAST>(tb, block) : occ_one<9, false, FAST>(tb, block);
    default: return tangent ? occ_one<1, true, FAST>(tb, block) : occ_one<1, false, FAST>(tb, block);
  }
}

template <bool FAST>
__global__ void k_debug_sincos_df(const double* x, double* s, double* c, long long n, const float4* tab, TabDF tb) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    Pair p;
    p.hi = __double2float_rn(x[i]);
    p.lo = __double2float_rn(x[i] - (double)p.hi);
    Pair ss, cc;
    if (FAST) sincos_df_fast(p, tab, tb, ss, cc);
    else sincos_df(p, tab, tb, ss, cc);
    s[i] = (double)ss.hi + (double)ss.lo;
    c[i] = (double)cc.hi + (double)cc.lo;
  }
}

}  // namespace

void df_tab(TabDF* tb);

cudaError_t launch_debug_sincos_df(const double* x, double* s, double* c, long long n, const float4* scd, bool fast,
                                   cudaStream_t st) {
  TabDF tb;
  df_tab(&tb);
  long long g = (n + 255) / 256;
  const int grid = (int)(g > 4096 ? 4096 : (g < 1 ? 1 : g));
  if (fast) k_debug_sincos_df<true><<<grid, 256, 0, st>>>(x, s, c, n, scd, tb);
  else k_debug_sincos_df<false><<<grid, 256, 0, st>>>(x, s, c, n, scd, tb);
  return cudaGetLastError();
}

cudaError_t launch_iterate_df64(const IterArgs& a, int scheme, bool tangent, bool fast, int block, int grid,
                                cudaStream_t st) {
  TabDF tb;
  df_tab(&tb);
  const CoefDF cf = coef_df_from(a.cf);
  return fast ? launch_scheme<true>(a, tb, cf, scheme, tangent, block, grid, st)
              : launch_scheme<false>(a, tb, cf, scheme, tangent, block, grid, st);
}

int df64_blocks_per_sm(int scheme, bool tangent, bool fast, int block) {
  TabDF tb;
  df_tab(&tb);
  return fast ? occ_scheme<true>(tb, scheme, tangent, block) : occ_scheme<false>(tb, scheme, tangent, block);
}

}  // namespace arnold
