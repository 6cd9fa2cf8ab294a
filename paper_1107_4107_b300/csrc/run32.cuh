// The compensated-FP32 per-trajectory run (load state, n composite steps with
// renormalisation / energy sampling / window closing, store state), shared by
// the single-ensemble kernel and the batched persistent kernel so both compute
// bit-identical trajectories.  TPT trajectories per thread are advanced
// interleaved (substep by substep) for instruction-level parallelism.
#pragma once
#include "step32.cuh"

namespace arnold {

// What one run needs from its ensemble (a subset of IterArgs).
struct RunArgs32 {
  Fp64State s;
  Fp32cState f;
  long long n;       // trajectories in the ensemble (SoA stride)
  int R;             // renormalisation / energy-sampling interval
  long long W;       // window (0 = none)
  double h, eps;
  int* flags;
};

// Step coefficients of one ensemble in FP32 (drifts as float pairs).
struct Coef32 {
  float sh[10], sl[10], k2[9];
};

__host__ __device__ inline Coef32 coef32_from(const StepCoef& c) {
  Coef32 r;
  for (int k = 0; k < 10; ++k) { r.sh[k] = c.sig_hi[k]; r.sl[k] = c.sig_lo[k]; }
  for (int k = 0; k < 9; ++k) r.k2[k] = c.k2f[k];
  return r;
}

template <bool TAN>
__device__ __forceinline__ void load32(const RunArgs32& a, long long i, Traj32& t, double& logsum, double& demax) {
  const long long n = a.n;
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
  logsum = TAN ? a.s.logsum[i] : 0.0;
  demax = a.s.demax[i];
}

template <bool TAN>
__device__ __forceinline__ void store32(const RunArgs32& a, long long i, const Traj32& t, double logsum, double demax) {
  const long long n = a.n;
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
}

// Renormalisation of the tangent (FP64 log accumulation, MEGNO sums of the
// j-th renormalisation when enabled) and FP64 energy sample.  `own` is false
// for a padding slot that repeats another thread's trajectory: it must not
// update the MEGNO sums a second time.
template <bool TAN>
__device__ __forceinline__ void renorm_sample32(const RunArgs32& a, long long i, Traj32& t, double& logsum,
                                                double& demax, int& bad, const float2* ssc, const Tab32& tb,
                                                long long j, bool own) {
  if (TAN) {
    // norm and log in FP64 (once per R steps), rescale in FP32
    const double du = t.du, dv = t.dv, dz = t.dz, dqu = t.dqu, dqv = t.dqv, dpz = t.dpz;
    const double n2 = 0.5 * (du * du + dv * dv) + dz * dz + 0.5 * (dqu * dqu + dqv * dqv) + dpz * dpz;
    const double l = 0.5 * log(n2);
    logsum += l;
    if (a.s.megno && own) megno_update(a.s.megno, a.n, i, j, l);
    const float inv = rsqrtf(__double2float_rn(n2));
    t.du *= inv; t.dv *= inv; t.dz *= inv;
    t.dqu *= inv; t.dqv *= inv; t.dpz *= inv;
    if (!(n2 > 0.0) || !(n2 <= 3.4e38)) bad |= 1;   // NaN, zero, or beyond FP32 (the factor)
  }
  // angles move at most h |q| within a step (the drift weights' partial sums stay in
  // [0, 1]) and each drift adds at most 0.8 h |q|: with h |q| <= 400 they stay in
  // [624, 2448] rad, above every increment and inside the table's exact range
  const float qmax = fmaxf(fmaxf(fabsf(t.qu.hi), fabsf(t.qv.hi)), fabsf(t.pz.hi));
  if (qmax * fabsf((float)a.h) > 400.0f) bad |= 2;
  float su, cu, sv, cv, sz, cz;
  sincos_tab32(t.u, ssc, tb, su, cu);
  sincos_tab32(t.v, ssc, tb, sv, cv);
  sincos_tab32(t.z, ssc, tb, sz, cz);
  const double kin = 0.25 * (pair_sq_d(t.qu) + pair_sq_d(t.qv)) + 0.5 * pair_sq_d(t.pz);
  const double H = kin + a.eps * (double)((cu + cv) * (cz * cz));
  const double dE = fabs(H - a.s.e0[i]);
  demax = fmax(demax, dE);
  if (!isfinite(dE)) bad |= 1;
  if (a.s.left) {
    const double qu = (double)t.qu.hi + (double)t.qu.lo, qv = (double)t.qv.hi + (double)t.qv.lo;
    if (!inside_patch(0.5 * (qu + qv), 0.5 * (qu - qv), (double)t.pz.hi + (double)t.pz.lo, a.s.patch)) a.s.left[i] = 1;
  }
}

// Close averaging window w (counted from the clock reset) of V (Sec. IV) for
// trajectory i.
template <typename T>   // Traj32 or TrajDF: angle pairs and laps
__device__ __forceinline__ void close_window32(const RunArgs32& a, long long i, const T& t, long long w) {
  const long long n = a.n;
  const double inv_dt = 1.0 / ((double)a.W * a.h);
  const double u = (double)t.u.hi + (double)t.u.lo, v = (double)t.v.hi + (double)t.v.lo,
               z = (double)t.z.hi + (double)t.z.lo;
  const double dU = (u - a.s.ref[i]) + kTwoPi * (double)(t.lu - a.s.lapref[i]);
  const double dV = (v - a.s.ref[n + i]) + kTwoPi * (double)(t.lv - a.s.lapref[n + i]);
  const double dZ = (z - a.s.ref[2 * n + i]) + kTwoPi * (double)(t.lz - a.s.lapref[2 * n + i]);
  const double vx = 0.5 * (dU + dV) * inv_dt, vy = 0.5 * (dU - dV) * inv_dt, vz = dZ * inv_dt;
  a.s.V[i] = vx;
  a.s.V[n + i] = vy;
  a.s.V[2 * n + i] = vz;
  snapshot_v(a.s, n, i, w, vx, vy, vz);
  a.s.ref[i] = u;
  a.s.ref[n + i] = v;
  a.s.ref[2 * n + i] = z;
  a.s.lapref[i] = t.lu;
  a.s.lapref[n + i] = t.lv;
  a.s.lapref[2 * n + i] = t.lz;
}

// Advance TPT trajectories idx[r] (valid if bit r of `valid` is set) by nsteps
// composite steps starting at global step step0.
template <int M, bool TAN, bool R64, int TPT>
__device__ __forceinline__ void run_traj32(const RunArgs32& a, const Coef32& cf, const long long* idx, int valid,
                                           long long step0, int nsteps, const float2* ssc, const Tab32& tb) {
  Traj32 t[TPT];
  double logsum[TPT], demax[TPT];
#pragma unroll
  for (int r = 0; r < TPT; ++r) load32<TAN>(a, idx[r], t[r], logsum[r], demax[r]);
  int to_renorm = a.R - (int)(step0 % a.R);
  long long to_window = a.W > 0 ? a.W - step0 % a.W : 0;
  int bad = 0;
#pragma unroll 1
  for (int s = 0; s < nsteps; ++s) {
#pragma unroll
    for (int r = 0; r < TPT; ++r) drift32<TAN, true>(t[r], cf.sh[0], cf.sl[0]);
#pragma unroll
    for (int k = 0; k < M; ++k) {
#pragma unroll
      for (int r = 0; r < TPT; ++r) kick32<TAN>(t[r], cf.k2[k], ssc, tb);
#pragma unroll
      for (int r = 0; r < TPT; ++r) drift32<TAN, true>(t[r], cf.sh[k + 1], cf.sl[k + 1]);
    }
#pragma unroll
    for (int r = 0; r < TPT; ++r) end_step32<R64>(t[r], tb);
    if (--to_renorm == 0) {
      to_renorm = a.R;
#pragma unroll
      for (int r = 0; r < TPT; ++r)
        renorm_sample32<TAN>(a, idx[r], t[r], logsum[r], demax[r], bad, ssc, tb, (step0 + s + 1) / a.R,
                             (valid >> r) & 1);
    }
    if (a.W > 0 && --to_window == 0) {
      to_window = a.W;
#pragma unroll
      for (int r = 0; r < TPT; ++r)
        if (valid & (1 << r)) close_window32(a, idx[r], t[r], (step0 + s + 1) / a.W);
    }
  }
#pragma unroll
  for (int r = 0; r < TPT; ++r)
    if (valid & (1 << r)) store32<TAN>(a, idx[r], t[r], logsum[r], demax[r]);
  if (bad & 1) atomicOr(a.flags, kFlagNonFinite);
  if (bad & 2) atomicOr(a.flags, kFlagRange);
}

}  // namespace arnold
