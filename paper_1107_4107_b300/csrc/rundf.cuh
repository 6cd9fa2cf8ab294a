// The double-float per-trajectory run (load state, n composite steps with
// renormalisation / energy sampling / window closing, store state), shared by
// the single-ensemble DF64 kernel and the batched persistent kernel, so both
// compute bit-identical trajectories.  FAST selects the ~3e-10 sincos of the
// DF64F mode; everything else is double-float (step_df.cuh).
#pragma once
#include "run32.cuh"
#include "step_df.cuh"

namespace arnold {

// Step coefficients of one ensemble in double-float: drifts and kicks as
// float pairs.
struct CoefDF {
  float sh[10], sl[10];   // drifts sigma_k = sh + sl
  Pair k2[9];             // 2 tau_k eps
};

inline CoefDF coef_df_from(const StepCoef& c) {
  CoefDF r;
  for (int k = 0; k < 10; ++k) { r.sh[k] = c.sig_hi[k]; r.sl[k] = c.sig_lo[k]; }
  for (int k = 0; k < 9; ++k) {
    r.k2[k].hi = (float)c.k2[k];
    r.k2[k].lo = (float)(c.k2[k] - (double)r.k2[k].hi);
  }
  return r;
}

// Largest h |q| per composite step a double-float run accepts.  Angles start a
// step below 12 rad (end_step_df) and move at most h |q| within it (the drift
// weights' partial sums stay in [0, 1] for all three schemes), so they stay
// below 172 rad: the reduction then removes at most 28 < 64 whole turns, for
// which k c1 and k c2 (18-bit parts of 2 pi) are exact products, and the
// table index |j| < 2^22 keeps x - j d1 exact.  Beyond it the run sets the
// range flag (ARNOLD_ERANGE).
constexpr float kDfMaxStepAngle = 160.0f;

// Advance trajectory i of the ensemble by nsteps composite steps starting at
// global step step0.
template <int M, bool TAN, bool FAST>
__device__ __forceinline__ void run_traj_df(const RunArgs32& a, const CoefDF& cf, long long i, long long step0,
                                            int nsteps, const float4* stab, const TabDF& tb) {
  const long long n = a.n;
  const float hf = (float)a.h;
  auto pd = [](const Pair& p) { return (double)p.hi + (double)p.lo; };
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
  int to_renorm = a.R - (int)(step0 % a.R);
  long long to_window = a.W > 0 ? a.W - step0 % a.W : 0;
  int bad = 0;
#pragma unroll 1
  for (int s = 0; s < nsteps; ++s) {
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
        if (a.s.megno) megno_update(a.s.megno, n, i, (step0 + s + 1) / a.R, l);
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
      const float qmax = fmaxf(fmaxf(fabsf(t.qu.hi), fabsf(t.qv.hi)), fabsf(t.pz.hi));
      if (qmax * fabsf(hf) > kDfMaxStepAngle) atomicOr(a.flags, kFlagRange);
      if (a.s.left) {
        const double qu = pd(t.qu), qv = pd(t.qv);
        if (!inside_patch(0.5 * (qu + qv), 0.5 * (qu - qv), pd(t.pz), a.s.patch)) a.s.left[i] = 1;
      }
    }
    if (a.W > 0 && --to_window == 0) {
      to_window = a.W;
      close_window32(a, i, t, (step0 + s + 1) / a.W);
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

}  // namespace arnold
