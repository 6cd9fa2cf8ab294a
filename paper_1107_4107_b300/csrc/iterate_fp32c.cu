// Compensated-FP32 ensemble propagator (the throughput path on B300, whose
// FP32 pipe issues ~74x more FMAs per second than its FP64 pipe).
//
// Same composite step as the FP64 kernel (Sec. III reading: symmetric
// composition of drift-kick-drift leapfrogs), in the rotated coordinates
// u = x + y, v = x - y (see arnold_internal.cuh), with:
//  * every angle and momentum a float pair (hi, lo), value hi + lo;
//  * drift: the increment s * (q_hi + q_lo) formed as an exact product
//    (Dekker/FMA TwoProd) plus the cross terms, added with Knuth's TwoSum;
//    the step size s itself is a float pair;
//  * kick: the increment (FP32 force) added with TwoSum into the pair;
//  * sincos by lookup in an exactly periodic FP32 table (Tang's method,
//    N = 2048, sin r ~ r, cos r ~ 1 - r^2/2, neglected terms < 7e-10) at the
//    reduced argument ((hi - j D1) - j D2 - j D3) + lo, so angles need no
//    reduction before a kick and the low word reaches the force;
//  * pairs renormalised (Fast2Sum) once per composite step, and the angles
//    reduced exactly (2 pi as three floats, TwoSum) once any exceeds 64 rad,
//    laps counted in int32;
//  * tangent vector in plain FP32; its renormalisation logs accumulated in
//    FP64 every R steps, when the energy error is sampled in FP64 as well.
// Variant REDUCE64: that reduction is done by widening the pair to FP64,
// subtracting k times the FP64 2pi and splitting back (the FP64 reduction).
#include <math.h>

#include "run32.cuh"

namespace arnold {

namespace {

template <int M, bool TAN, bool REDUCE64>
__global__ void __launch_bounds__(256) k_iterate_fp32c(IterArgs a, Tab32 tb) {
  extern __shared__ __align__(16) unsigned char smem[];
  float2* ssc = reinterpret_cast<float2*>(smem);
  for (int k = threadIdx.x; k <= tb.jmax; k += blockDim.x) ssc[k] = a.scf[k];
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
  const Coef32 cf = coef32_from(a.cf);
  const long long n = a.n;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const long long idx[1] = {i};
    run_traj32<M, TAN, REDUCE64, 1>(ra, cf, idx, 1, a.step0, a.nsteps, ssc, tb);
  }
}

template <int M, bool TAN, bool R64>
cudaError_t launch_one(const IterArgs& a, const Tab32& tb, int block, int grid, cudaStream_t st) {
  const size_t smem = (size_t)(tb.jmax + 1) * sizeof(float2);
  k_iterate_fp32c<M, TAN, R64><<<grid, block, smem, st>>>(a, tb);
  return cudaGetLastError();
}

template <bool R64>
cudaError_t launch_scheme(const IterArgs& a, const Tab32& tb, int scheme, bool tangent, int block, int grid,
                          cudaStream_t st) {
  switch (scheme) {
    case ARNOLD_SCHEME_YOSHIDA6A:
      return tangent ? launch_one<7, true, R64>(a, tb, block, grid, st) : launch_one<7, false, R64>(a, tb, block, grid, st);
    case ARNOLD_SCHEME_TRIPLEJUMP6:
      return tangent ? launch_one<9, true, R64>(a, tb, block, grid, st) : launch_one<9, false, R64>(a, tb, block, grid, st);
    case ARNOLD_SCHEME_LEAPFROG2:
      return tangent ? launch_one<1, true, R64>(a, tb, block, grid, st) : launch_one<1, false, R64>(a, tb, block, grid, st);
  }
  return cudaErrorInvalidValue;
}

__global__ void k_debug_sincos32(const double* x, double* s, double* c, long long n, const float2* sc, Tab32 tb) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    Pair p;
    p.hi = __double2float_rn(x[i]);
    p.lo = __double2float_rn(x[i] - (double)p.hi);
    float ss, cc;
    sincos_tab32(p, sc, tb, ss, cc);
    s[i] = ss;
    c[i] = cc;
  }
}

}  // namespace

// Table geometry shared with the host table builder (api.cu).
void fp32_tab(Tab32* tb);

cudaError_t launch_iterate_fp32c_v(const IterArgs& a, int scheme, bool tangent, bool reduce64, int block, int grid,
                                   cudaStream_t st) {
  Tab32 tb;
  fp32_tab(&tb);
  return reduce64 ? launch_scheme<true>(a, tb, scheme, tangent, block, grid, st)
                  : launch_scheme<false>(a, tb, scheme, tangent, block, grid, st);
}

cudaError_t launch_iterate_fp32c(const IterArgs& a, int scheme, bool tangent, int block, int grid, cudaStream_t st) {
  return launch_iterate_fp32c_v(a, scheme, tangent, false, block, grid, st);
}

int fp32c_blocks_per_sm(int scheme, bool tangent, int block) {
  Tab32 tb;
  fp32_tab(&tb);
  const size_t smem = (size_t)(tb.jmax + 1) * sizeof(float2);
  int nb = 0;
  cudaError_t e = cudaSuccess;
  switch (scheme) {
    case ARNOLD_SCHEME_YOSHIDA6A:
      e = tangent ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_iterate_fp32c<7, true, false>, block, smem)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_iterate_fp32c<7, false, false>, block, smem);
      break;
    case ARNOLD_SCHEME_TRIPLEJUMP6:
      e = tangent ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_iterate_fp32c<9, true, false>, block, smem)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_iterate_fp32c<9, false, false>, block, smem);
      break;
    default:
      e = tangent ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_iterate_fp32c<1, true, false>, block, smem)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_iterate_fp32c<1, false, false>, block, smem);
  }
  if (e != cudaSuccess || nb < 1) return 1;
  return nb;
}

cudaError_t launch_debug_sincos32(const double* x, double* s, double* c, long long n, const float2* scf,
                                  cudaStream_t st) {
  Tab32 tb;
  fp32_tab(&tb);
  long long g = (n + 255) / 256;
  int grid = (int)(g > 4096 ? 4096 : (g < 1 ? 1 : g));
  k_debug_sincos32<<<grid, 256, 0, st>>>(x, s, c, n, scf, tb);
  return cudaGetLastError();
}

}  // namespace arnold
