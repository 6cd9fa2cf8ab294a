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
//  * mod-2pi reduction after each drift against 2pi as a float pair
//    (hi - C_hi is exact by Sterbenz' lemma), laps counted in int32;
//  * pairs renormalised (Fast2Sum) once per composite step;
//  * sincos by table lookup in FP32 (Tang's method, N = 2048,
//    sin r ~ r, cos r ~ 1 - r^2/2 for |r| <= pi/2048; neglected terms
//    < 7e-10) at the reduced argument (hi - theta_j) + lo, so the low word
//    of the angle reaches the force;
//  * tangent vector in plain FP32; its renormalisation logs accumulated in
//    FP64 every R steps, when the energy error is sampled in FP64 as well.
// Variant REDUCE64: the wrap is done by widening the pair to FP64,
// subtracting the FP64 2pi and splitting back (the FP64 reduction).
#include <math.h>

#include "step32.cuh"

namespace arnold {

namespace {

template <int M, bool TAN, bool REDUCE64>
__global__ void __launch_bounds__(256) k_iterate_fp32c(IterArgs a, Tab32 tb) {
  extern __shared__ __align__(16) unsigned char smem[];
  float2* ssc = reinterpret_cast<float2*>(smem);
  for (int k = threadIdx.x; k <= tb.jmax; k += blockDim.x) ssc[k] = a.scf[k];
  __syncthreads();

  const long long n = a.n;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    Traj32 t;
    t.u = {a.f.hi[i], a.f.lo[i]};
    t.v = {a.f.hi[n + i], a.f.lo[n + i]};
    t.z = {a.f.hi[2 * n + i], a.f.lo[2 * n + i]};
    t.qu = {a.f.hi[3 * n + i], a.f.lo[3 * n + i]};
    t.qv = {a.f.hi[4 * n + i], a.f.lo[4 * n + i]};
    t.pz = {a.f.hi[5 * n + i], a.f.lo[5 * n + i]};
    if (TAN) {
      t.du = a.f.tg[i];
      t.dv = a.f.tg[n + i];
      t.dz = a.f.tg[2 * n + i];
      t.dqu = a.f.tg[3 * n + i];
      t.dqv = a.f.tg[4 * n + i];
      t.dpz = a.f.tg[5 * n + i];
    }
    t.lu = a.s.lap[i];
    t.lv = a.s.lap[n + i];
    t.lz = a.s.lap[2 * n + i];
    double logsum = TAN ? a.s.logsum[i] : 0.0;
    double demax = a.s.demax[i];
    int to_renorm = a.R - (int)(a.step0 % a.R);
    long long to_window = a.W > 0 ? a.W - a.step0 % a.W : 0;
    int bad = 0;

#pragma unroll 1
    for (int s = 0; s < a.nsteps; ++s) {
      drift32<TAN, REDUCE64>(t, a.cf.sig_hi[0], a.cf.sig_lo[0]);
#pragma unroll
      for (int k = 0; k < M; ++k) {
        kick32<TAN>(t, a.cf.k2f[k], a.cf.k4f[k], ssc, tb);
        drift32<TAN, REDUCE64>(t, a.cf.sig_hi[k + 1], a.cf.sig_lo[k + 1]);
      }
      renorm(t.u); renorm(t.v); renorm(t.z);
      renorm(t.qu); renorm(t.qv); renorm(t.pz);
      if (--to_renorm == 0) {
        to_renorm = a.R;
        if (TAN) {
          const float n2 = 0.5f * (t.du * t.du + t.dv * t.dv) + t.dz * t.dz +
                           0.5f * (t.dqu * t.dqu + t.dqv * t.dqv) + t.dpz * t.dpz;
          logsum += 0.5 * (double)__logf(n2);
          const float inv = rsqrtf(n2);
          t.du *= inv; t.dv *= inv; t.dz *= inv;
          t.dqu *= inv; t.dqv *= inv; t.dpz *= inv;
          if (!(n2 > 0.0f) || !isfinite(n2)) bad = 1;
        }
        float su, cu, sv, cv, sz, cz;
        sincos_tab32(t.u, ssc, tb, su, cu);
        sincos_tab32(t.v, ssc, tb, sv, cv);
        sincos_tab32(t.z, ssc, tb, sz, cz);
        const double kin = 0.25 * (pair_sq_d(t.qu) + pair_sq_d(t.qv)) + 0.5 * pair_sq_d(t.pz);
        const double H = kin + a.eps * (double)((cu + cv) * (cz * cz));
        const double dE = fabs(H - a.s.e0[i]);
        demax = fmax(demax, dE);
        if (!isfinite(dE)) bad = 1;
      }
      if (a.W > 0 && --to_window == 0) {
        to_window = a.W;
        const double inv_dt = 1.0 / ((double)a.W * a.h);
        const double dU = (((double)t.u.hi + (double)t.u.lo) - a.s.ref[i]) + kTwoPi * (double)(t.lu - a.s.lapref[i]);
        const double dV =
            (((double)t.v.hi + (double)t.v.lo) - a.s.ref[n + i]) + kTwoPi * (double)(t.lv - a.s.lapref[n + i]);
        const double dZ =
            (((double)t.z.hi + (double)t.z.lo) - a.s.ref[2 * n + i]) + kTwoPi * (double)(t.lz - a.s.lapref[2 * n + i]);
        a.s.V[i] = 0.5 * (dU + dV) * inv_dt;
        a.s.V[n + i] = 0.5 * (dU - dV) * inv_dt;
        a.s.V[2 * n + i] = dZ * inv_dt;
        a.s.ref[i] = (double)t.u.hi + (double)t.u.lo;
        a.s.ref[n + i] = (double)t.v.hi + (double)t.v.lo;
        a.s.ref[2 * n + i] = (double)t.z.hi + (double)t.z.lo;
        a.s.lapref[i] = t.lu; a.s.lapref[n + i] = t.lv; a.s.lapref[2 * n + i] = t.lz;
      }
    }

    a.f.hi[i] = t.u.hi;          a.f.lo[i] = t.u.lo;
    a.f.hi[n + i] = t.v.hi;      a.f.lo[n + i] = t.v.lo;
    a.f.hi[2 * n + i] = t.z.hi;  a.f.lo[2 * n + i] = t.z.lo;
    a.f.hi[3 * n + i] = t.qu.hi; a.f.lo[3 * n + i] = t.qu.lo;
    a.f.hi[4 * n + i] = t.qv.hi; a.f.lo[4 * n + i] = t.qv.lo;
    a.f.hi[5 * n + i] = t.pz.hi; a.f.lo[5 * n + i] = t.pz.lo;
    if (TAN) {
      a.f.tg[i] = t.du;
      a.f.tg[n + i] = t.dv;
      a.f.tg[2 * n + i] = t.dz;
      a.f.tg[3 * n + i] = t.dqu;
      a.f.tg[4 * n + i] = t.dqv;
      a.f.tg[5 * n + i] = t.dpz;
      a.s.logsum[i] = logsum;
    }
    a.s.lap[i] = t.lu;
    a.s.lap[n + i] = t.lv;
    a.s.lap[2 * n + i] = t.lz;
    a.s.demax[i] = demax;
    if (bad) atomicOr(a.flags, kFlagNonFinite);
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
void fp32_table_geometry(float* d, float* inv_d, int* jmax);

cudaError_t launch_iterate_fp32c_v(const IterArgs& a, int scheme, bool tangent, bool reduce64, int block, int grid,
                                   cudaStream_t st) {
  Tab32 tb;
  fp32_table_geometry(&tb.d, &tb.inv_d, &tb.jmax);
  return reduce64 ? launch_scheme<true>(a, tb, scheme, tangent, block, grid, st)
                  : launch_scheme<false>(a, tb, scheme, tangent, block, grid, st);
}

cudaError_t launch_iterate_fp32c(const IterArgs& a, int scheme, bool tangent, int block, int grid, cudaStream_t st) {
  return launch_iterate_fp32c_v(a, scheme, tangent, false, block, grid, st);
}

int fp32c_blocks_per_sm(int scheme, bool tangent, int block) {
  Tab32 tb;
  fp32_table_geometry(&tb.d, &tb.inv_d, &tb.jmax);
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
  fp32_table_geometry(&tb.d, &tb.inv_d, &tb.jmax);
  long long g = (n + 255) / 256;
  int grid = (int)(g > 4096 ? 4096 : (g < 1 ? 1 : g));
  k_debug_sincos32<<<grid, 256, 0, st>>>(x, s, c, n, scf, tb);
  return cudaGetLastError();
}

}  // namespace arnold
