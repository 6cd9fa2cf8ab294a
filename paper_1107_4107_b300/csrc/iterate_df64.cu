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
#include "run32.cuh"
#include "step_df.cuh"

namespace arnold {

namespace {

struct CoefDF {
  float sh[10], sl[10];   // drifts as float pairs
  Pair k2[9];             // 2 tau eps as pairs
};

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
  const float hf = (float)a.h;
  const long long n = a.n;
  auto pd = [](const Pair& p) { return (double)p.hi + (double)p.lo; };
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    TrajDF t;
    t.u = {a.f.hi[i], a.f.lo[i]};
    t.v = {a.f.hi[n + i], a.f.lo[n + i]};
    t.z = {a.f.hi[2 * n + i], a.f.lo[2 * n + i]};
    t.qu = {a.f.hi[3 * n + i], a.f.lo[3 * n + i]};
    t.qv = {a.f.hi[4 * n + i], a.f.lo[4 * n + i]};
    t.pz = {a.f.hi[5 * n + i], a.f.lo[5 * n + i]};
    if (TAN) {
      t.du = {a.f.tg[i], a.f.tg_lo[i]};
      t.dv = {a.f.tg[n + i], a.f.tg_lo[n + i]};
      t.dz = {a.f.tg[2 * n + i], a.f.tg_lo[2 * n + i]};
      t.dqu = {a.f.tg[3 * n + i], a.f.tg_lo[3 * n + i]};
      t.dqv = {a.f.tg[4 * n + i], a.f.tg_lo[4 * n + i]};
      t.dpz = {a.f.tg[5 * n + i], a.f.tg_lo[5 * n + i]};
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
      drift_df<TAN>(t, cf.sh[0], cf.sl[0]);
#pragma unroll 1
      for (int k = 0; k < M; ++k) {
        kick_df<TAN, FAST>(t, cf.k2[k], stab, tb);
        drift_df<TAN>(t, cf.sh[k + 1], cf.sl[k + 1]);
      }
      end_step_df<TAN>(t, tb);
      if (--to_renorm == 0) {
        to_renorm = a.R;
        if (TAN) {   // norm and log in FP64 (once per R steps)
          const double w0 = pd(t.du), w1 = pd(t.dv), w2 = pd(t.dz), w3 = pd(t.dqu), w4 = pd(t.dqv), w5 = pd(t.dpz);
          const double n2 = 0.5 * (w0 * w0 + w1 * w1) + w2 * w2 + 0.5 * (w3 * w3 + w4 * w4) + w5 * w5;
          const double l = 0.5 * log(n2);
          logsum += l;
          if (a.s.megno) megno_update(a.s.megno, n, i, (a.step0 + s + 1) / a.R, l);
          // rescale by 1/|w| to double-float accuracy: whatever norm the factor
          // leaves enters the next log, so an FP32 factor (~1e-7) would add up
          // over the renormalisations
          const double inv = rsqrt(n2);
          const float ih = __double2float_rn(inv);
          const Pair iv = {ih, __double2float_rn(inv - (double)ih)};
          Pair* w[6] = {&t.du, &t.dv, &t.dz, &t.dqu, &t.dqv, &t.dpz};
#pragma unroll
          for (int c = 0; c < 6; ++c) *w[c] = df_mul(*w[c], iv);
          if (!(n2 > 0.0) || !isfinite(n2)) bad = 1;
        }
        const double kin = 0.25 * (pair_sq_d(t.qu) + pair_sq_d(t.qv)) + 0.5 * pair_sq_d(t.pz);
        const double dE = fabs(kin + a.eps * potential_df(t, stab, tb) - a.s.e0[i]);
        demax = fmax(demax, dE);
        if (!isfinite(dE)) bad = 1;
        // angles start a step below 12 rad and move at most h |q| within it (the
        // drift weights' partial sums stay in [0, 1]): below 21 < 25 rad, the
        // table's exact index range, while h |q| <= 9
        const float qmax = fmaxf(fmaxf(fabsf(t.qu.hi), fabsf(t.qv.hi)), fabsf(t.pz.hi));
        if (qmax * fabsf(hf) > 9.0f) atomicOr(a.flags, kFlagRange);
        if (a.s.left) {
          const double qu = pd(t.qu), qv = pd(t.qv);
          if (!inside_patch(0.5 * (qu + qv), 0.5 * (qu - qv), pd(t.pz), a.s.patch)) a.s.left[i] = 1;
        }
      }
      if (a.W > 0 && --to_window == 0) {
        to_window = a.W;
        close_window32(ra, i, t, (a.step0 + s + 1) / a.W);
      }
    }
    a.f.hi[i] = t.u.hi;          a.f.lo[i] = t.u.lo;
    a.f.hi[n + i] = t.v.hi;      a.f.lo[n + i] = t.v.lo;
    a.f.hi[2 * n + i] = t.z.hi;  a.f.lo[2 * n + i] = t.z.lo;
    a.f.hi[3 * n + i] = t.qu.hi; a.f.lo[3 * n + i] = t.qu.lo;
    a.f.hi[4 * n + i] = t.qv.hi; a.f.lo[4 * n + i] = t.qv.lo;
    a.f.hi[5 * n + i] = t.pz.hi; a.f.lo[5 * n + i] = t.pz.lo;
    if (TAN) {
      a.f.tg[i] = t.du.hi;          a.f.tg_lo[i] = t.du.lo;
      a.f.tg[n + i] = t.dv.hi;      a.f.tg_lo[n + i] = t.dv.lo;
      a.f.tg[2 * n + i] = t.dz.hi;  a.f.tg_lo[2 * n + i] = t.dz.lo;
      a.f.tg[3 * n + i] = t.dqu.hi; a.f.tg_lo[3 * n + i] = t.dqu.lo;
      a.f.tg[4 * n + i] = t.dqv.hi; a.f.tg_lo[4 * n + i] = t.dqv.lo;
      a.f.tg[5 * n + i] = t.dpz.hi; a.f.tg_lo[5 * n + i] = t.dpz.lo;
      a.s.logsum[i] = logsum;
    }
    a.s.lap[i] = t.lu;
    a.s.lap[n + i] = t.lv;
    a.s.lap[2 * n + i] = t.lz;
    a.s.demax[i] = demax;
    if (bad) atomicOr(a.flags, kFlagNonFinite);
  }
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

CoefDF coef_df(const StepCoef& c) {
  CoefDF r;
  for (int k = 0; k < 10; ++k) { r.sh[k] = c.sig_hi[k]; r.sl[k] = c.sig_lo[k]; }
  for (int k = 0; k < 9; ++k) {
    r.k2[k].hi = (float)c.k2[k];
    r.k2[k].lo = (float)(c.k2[k] - (double)r.k2[k].hi);
  }
  return r;
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
  const CoefDF cf = coef_df(a.cf);
  return fast ? launch_scheme<true>(a, tb, cf, scheme, tangent, block, grid, st)
              : launch_scheme<false>(a, tb, cf, scheme, tangent, block, grid, st);
}

int df64_blocks_per_sm(int scheme, bool tangent, bool fast, int block) {
  TabDF tb;
  df_tab(&tb);
  return fast ? occ_scheme<true>(tb, scheme, tangent, block) : occ_scheme<false>(tb, scheme, tangent, block);
}

}  // namespace arnold
