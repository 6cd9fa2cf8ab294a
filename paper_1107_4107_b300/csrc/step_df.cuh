// Double-float ("DF64") building blocks: FP64-grade arithmetic on the FP32
// pipes.  A value is a float pair (hi, lo) with |lo| <= ulp(hi)/2 after
// renormalisation (about 48 significant bits); products use the exact FMA
// split (Dekker / Ogita-Rump-Oishi TwoProd) and sums Knuth's TwoSum, so each
// operation is correct to ~2^-47 relative.  The B300 issues FP32 FMAs 74x
// faster than FP64 ones, so the whole kick (sincos, force) in double-float
// costs a fraction of the native FP64 kick.
#pragma once
#include "step32.cuh"

namespace arnold {

// Sincos table of the DF64 path: theta_j = 2 pi j / 2048, entry j holds
// (sin hi, sin lo, cos hi, cos lo) rounded from long-double libm; the step
// D = 2 pi / 2048 is split d1 (11 significant bits, its last bit 2^-19) + d2 +
// d3 (59 bits in all).  x.hi - j d1 is then exact for any |x| < 2^22 D: both
// are multiples of min(ulp(x.hi), 2^-19) and their difference is below D.
// Angles are reduced once they pass 12 rad at the end of a step, so within a
// step |x| < 12 + h |q| (h |q| <= kDfMaxStepAngle, checked at renormalisation).
struct TabDF {
  float inv_d, d1, d2, d3;
  int mask;          // 2047
  float inv2pi, c1, c2, c3;
};

__device__ __forceinline__ Pair df_mul(const Pair& a, const Pair& b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  Pair r;
  fast_two_sum(p, e, r.hi, r.lo);
  return r;
}

// Product without the final renormalisation: (p, e) with |e| up to ~2 ulp(p),
// for products that feed another product or an accumulation.
__device__ __forceinline__ Pair df_mul_u(const Pair& a, const Pair& b) {
  Pair r;
  r.hi = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -r.hi);
  e = fmaf(a.hi, b.lo, e);
  r.lo = fmaf(a.lo, b.hi, e);
  return r;
}

// a + b without the final renormalisation: (s, e) with |e| up to ~ulp(s), for
// sums that only feed products (df_mul_u multiplies both words, so an
// unnormalised low word costs no accuracy there).
__device__ __forceinline__ Pair df_add_u(const Pair& a, const Pair& b) {
  Pair r;
  float e;
  two_sum(a.hi, b.hi, r.hi, e);
  r.lo = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  return r;
}

// x += inc (both pairs), keeping x's low word for the next renormalisation.
__device__ __forceinline__ void df_acc(Pair& x, const Pair& inc) {
  float s, e;
  two_sum(x.hi, inc.hi, s, e);
  x.hi = s;
  x.lo = __fadd_rn(x.lo, __fadd_rn(e, inc.lo));
}

// sin and cos of the pair x to a few units of the pair's last place (~1e-14
// for values near 1; Tang's table method in double-float): x = theta_j + r,
// r formed exactly as a pair, sin r - r and
// cos r - 1 from their Taylor terms (r^3/6, r^5/120 in FP32, r^2/2 as a pair,
// r^4/24 in FP32; |r| <= 1.6e-3 so the next terms are < 1e-19), then
// sin x = S + C (r + u) + S cm and cos x = C - S (r + u) + C cm with the large
// products split exactly and the small ones gathered in FP32.
__device__ __forceinline__ void sincos_df(const Pair& x, const float4* __restrict__ tab, const TabDF& tb, Pair& s,
                                          Pair& c) {
  const float t = fmaf(x.hi, tb.inv_d, 12582912.0f);
  const float jf = __fsub_rn(t, 12582912.0f);
  const int j = (__float_as_int(t) - 0x4B400000) & tb.mask;
  const float r1 = fmaf(-jf, tb.d1, x.hi);                 // exact
  const float p = __fmul_rn(jf, tb.d2);
  const float pe = fmaf(jf, tb.d2, -p);                     // exact error of jf * d2
  float a, ae, rh, be;
  two_sum(r1, -p, a, ae);                                  // exact
  two_sum(a, x.lo, rh, be);                                // exact: the low word joins before rounding
  float rl = fmaf(-jf, tb.d3, __fadd_rn(be, __fsub_rn(ae, pe)));
  fast_two_sum(rh, rl, rh, rl);
  const float r2h = __fmul_rn(rh, rh);
  const float r2e = fmaf(2.0f * rh, rl, fmaf(rh, rh, -r2h));
  const float r3 = __fmul_rn(r2h, rh);
  const float u = __fmul_rn(r3, fmaf(r2h, 1.0f / 120.0f, -1.0f / 6.0f));   // sin r - r
  const float cmh = -0.5f * r2h;                                           // cos r - 1 (leading, exact)
  const float cml = fmaf(__fmul_rn(r2h, r2h), 1.0f / 24.0f, -0.5f * r2e);
  const float4 e = tab[j];   // (S hi, S lo, C hi, C lo)
  const float rlu = __fadd_rn(rl, u);
  {
    const float pa = __fmul_rn(e.z, rh), ea = fmaf(e.z, rh, -pa);        // C_h r_h
    const float pb = __fmul_rn(e.x, cmh), eb = fmaf(e.x, cmh, -pb);      // S_h cm_h
    float s1, e1, s2, e2;
    two_sum(e.x, pa, s1, e1);
    two_sum(s1, pb, s2, e2);
    float sm = __fadd_rn(__fadd_rn(e1, e2), __fadd_rn(ea, eb));
    sm = __fadd_rn(sm, e.y);
    sm = fmaf(e.z, rlu, sm);
    sm = fmaf(e.w, rh, sm);
    sm = fmaf(e.x, cml, sm);
    sm = fmaf(e.y, cmh, sm);
    fast_two_sum(s2, sm, s.hi, s.lo);
  }
  {
    const float pa = __fmul_rn(e.x, rh), ea = fmaf(e.x, rh, -pa);        // S_h r_h
    const float pb = __fmul_rn(e.z, cmh), eb = fmaf(e.z, cmh, -pb);      // C_h cm_h
    float c1, f1, c2, f2;
    two_sum(e.z, -pa, c1, f1);
    two_sum(c1, pb, c2, f2);
    float sm = __fadd_rn(__fadd_rn(f1, f2), __fsub_rn(eb, ea));
    sm = __fadd_rn(sm, e.w);
    sm = fmaf(-e.x, rlu, sm);
    sm = fmaf(-e.y, rh, sm);
    sm = fmaf(e.z, cml, sm);
    sm = fmaf(e.w, cmh, sm);
    fast_two_sum(c2, sm, c.hi, c.lo);
  }
}

// sin and cos of the pair x to ~3e-10 absolute (the "DF64F" mode): the same
// table, but the reduced argument r = x - theta_j in FP32 (one rounding per
// FMA at |r| <= D/2, ~1e-10), sin r - r = -r^3/6 folded into r, and the small
// terms C (r - r^3/6) + S cm and C cm - S (r - r^3/6) (|.| <= 1.6e-3) in FP32,
// joined to the table's pair (S, C) by Fast2Sum.  The error is that of r and of
// the small terms' rounding; the products and sums that use the result stay
// double-float.
__device__ __forceinline__ void sincos_df_fast(const Pair& x, const float4* __restrict__ tab, const TabDF& tb,
                                               Pair& s, Pair& c) {
  const float t = fmaf(x.hi, tb.inv_d, 12582912.0f);
  const float jf = __fsub_rn(t, 12582912.0f);
  const int j = (__float_as_int(t) - 0x4B400000) & tb.mask;
  float r = fmaf(-jf, tb.d1, x.hi);                         // exact
  r = fmaf(-jf, tb.d2, r);
  r = fmaf(-jf, tb.d3, r);
  r = __fadd_rn(r, x.lo);
  const float cm = __fmul_rn(-0.5f, __fmul_rn(r, r));      // cos r - 1 (r^4/24 < 3e-13 dropped)
  const float rs = fmaf(__fmul_rn(r, 0.333333343f), cm, r); // r - r^3/6 = sin r (r^5/120 < 1e-16 dropped)
  const float4 e = tab[j];   // (S hi, S lo, C hi, C lo)
  const float qs = fmaf(e.z, rs, __fmul_rn(e.x, cm));
  const float qc = fmaf(-e.x, rs, __fmul_rn(e.z, cm));
  // |qs|, |qc| <= |r| + |cm| < 1.55e-3 < sin(2 pi / 2048) = 3.07e-3 <= |S|, |C|
  // for every entry but the four where S or C is zero or a rounding of zero
  // (below 1e-19), so Fast2Sum is exact there and elsewhere loses at most that
  // 1e-19, far below the 3e-10 bound (measured: 5 % faster than TwoSum).
  float h, l;
  fast_two_sum(e.x, qs, h, l);
  s = {h, __fadd_rn(l, e.y)};
  fast_two_sum(e.z, qc, h, l);
  c = {h, __fadd_rn(l, e.w)};
}

// State of one DF64 trajectory: phase-space state and tangent as float pairs
// (~48 bits each), laps as integers.
struct TrajDF {
  Pair u, v, z, qu, qv, pz;
  Pair du, dv, dz, dqu, dqv, dpz;
  int lu, lv, lz;
};

__device__ __forceinline__ Pair df_neg(const Pair& a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ Pair df_scale2(const Pair& a, float m) { return {m * a.hi, m * a.lo}; }   // m = +-2: exact

// Drift in double-float: the state as in the FP32C path (TwoSum, s a float
// pair), the tangent dX += s dP as double-float products accumulated with
// TwoSum.
template <bool TAN>
__device__ __forceinline__ void drift_df(TrajDF& t, float sh, float sl) {
  drift_comp<false>(t.u, sh, sl, t.qu);
  drift_comp<false>(t.v, sh, sl, t.qv);
  drift_comp<false>(t.z, sh, sl, t.pz);
  if (TAN) {
    const Pair s = {sh, sl};
    df_acc(t.du, df_mul_u(s, t.dqu));
    df_acc(t.dv, df_mul_u(s, t.dqv));
    df_acc(t.dz, df_mul_u(s, t.dpz));
  }
}

// Kick in double-float: q_u += G s_u, q_v += G s_v, p_z += Sp A with
// G = (k2 c_z) c_z, Sp = (k2 c_z) s_z, A = c_u + c_v (k2 = 2 tau eps as a
// pair).  The tangent update (the Hessian of Eq. 2 applied to the tangent) is
// double-float as well, coefficients and accumulation: on a regular orbit the
// tangent map is a shear, and FP32 coefficients or FP32 accumulation bias its
// growth over 1e6 steps (the chi field then drifts by percents).  FAST takes
// the sines and cosines from sincos_df_fast (~3e-10) instead of sincos_df.
template <bool TAN, bool FAST = false>
__device__ __forceinline__ void kick_df(TrajDF& t, const Pair& k2, const float4* tab, const TabDF& tb) {
  Pair su, cu, sv, cv, sz, cz;
  if (FAST) {
    sincos_df_fast(t.u, tab, tb, su, cu);
    sincos_df_fast(t.v, tab, tb, sv, cv);
    sincos_df_fast(t.z, tab, tb, sz, cz);
  } else {
    sincos_df(t.u, tab, tb, su, cu);
    sincos_df(t.v, tab, tb, sv, cv);
    sincos_df(t.z, tab, tb, sz, cz);
  }
  const Pair kc = df_mul_u(k2, cz);
  const Pair G = df_mul_u(kc, cz);    // k2 c_z^2
  const Pair Sp = df_mul_u(kc, sz);   // k2 s_z c_z
  const Pair A = df_add_u(cu, cv);   // feeds products only
  df_acc(t.qu, df_mul_u(G, su));
  df_acc(t.qv, df_mul_u(G, sv));
  df_acc(t.pz, df_mul_u(Sp, A));
  if (TAN) {
    const Pair Gu = df_mul_u(G, cu), Gv = df_mul_u(G, cv);
    const Pair Yu = df_mul_u(Sp, su), Yv = df_mul_u(Sp, sv);
    const Pair Z = df_mul_u(A, df_add_u(df_scale2(G, 2.0f), df_neg(k2)));   // A (k4 c_z^2 - k2), k4 = 2 k2
    const Pair m2dz = df_scale2(t.dz, -2.0f);
    df_acc(t.dqu, df_mul_u(Gu, t.du));
    df_acc(t.dqu, df_mul_u(Yu, m2dz));
    df_acc(t.dqv, df_mul_u(Gv, t.dv));
    df_acc(t.dqv, df_mul_u(Yv, m2dz));
    df_acc(t.dpz, df_mul_u(Z, t.dz));
    df_acc(t.dpz, df_mul_u(df_neg(Yu), t.du));
    df_acc(t.dpz, df_mul_u(df_neg(Yv), t.dv));
  }
}

// Potential (Eq. 2) in double-float, returned as FP64.
template <typename T>
__device__ __forceinline__ double potential_df(const T& t, const float4* tab, const TabDF& tb) {
  Pair su, cu, sv, cv, sz, cz;
  sincos_df(t.u, tab, tb, su, cu);
  sincos_df(t.v, tab, tb, sv, cv);
  sincos_df(t.z, tab, tb, sz, cz);
  const double A = ((double)cu.hi + (double)cu.lo) + ((double)cv.hi + (double)cv.lo);
  const double c = (double)cz.hi + (double)cz.lo;
  return A * (c * c);
}

}  // namespace arnold

namespace arnold {

// End of a DF64 step: renormalise every pair, and once an angle passes 12 rad
// remove whole turns from the angles (exactly, 2 pi as three floats: k c1 and
// k c2 are exact for |k| < 64 turns, and angles stay below 12 + h |q| < 172 rad
// while h |q| <= kDfMaxStepAngle, checked at renormalisation, ERANGE
// otherwise).
__device__ __forceinline__ void reduce_angle_df(Pair& x, int& lap, const TabDF& tb) {
  const float t = fmaf(x.hi, tb.inv2pi, 12582912.0f);
  const float kf = __fsub_rn(t, 12582912.0f);
  const int k = __float_as_int(t) - 0x4B400000;
  const float h1 = fmaf(-kf, tb.c1, x.hi);
  float s, e;
  two_sum(h1, __fmul_rn(-kf, tb.c2), s, e);
  const float lo = fmaf(-kf, tb.c3, __fadd_rn(x.lo, e));
  fast_two_sum(s, lo, x.hi, x.lo);
  lap += k;
}

template <bool TAN>
__device__ __forceinline__ void end_step_df(TrajDF& t, const TabDF& tb) {
  renorm(t.qu); renorm(t.qv); renorm(t.pz);
  renorm(t.u); renorm(t.v); renorm(t.z);
  if (TAN) {
    renorm(t.du); renorm(t.dv); renorm(t.dz);
    renorm(t.dqu); renorm(t.dqv); renorm(t.dpz);
  }
  const int big = max(max(__float_as_int(t.u.hi) & 0x7FFFFFFF, __float_as_int(t.v.hi) & 0x7FFFFFFF),
                      __float_as_int(t.z.hi) & 0x7FFFFFFF);
  if (big > 0x41400000) {   // |angle| > 12
    reduce_angle_df(t.u, t.lu, tb);
    reduce_angle_df(t.v, t.lv, tb);
    reduce_angle_df(t.z, t.lz, tb);
  }
}

}  // namespace arnold
