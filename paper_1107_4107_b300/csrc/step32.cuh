// Compensated-FP32 building blocks (float pairs, TwoSum/TwoProd updates,
// exact float-pair mod-2pi reduction, FP32 periodic-table sincos, drift/kick)
// shared by the iterate, batch and adjoint kernels so that recomputed states
// are bit-identical.
#pragma once
#include "devmath.cuh"

namespace arnold {

struct Pair { float hi, lo; };

struct Traj32 {
  Pair u, v, z, qu, qv, pz;
  float du, dv, dz, dqu, dqv, dpz;
  int lu, lv, lz;
};

// Knuth TwoSum: s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Fast2Sum (|a| >= |b| or a == 0): s + e == a + b exactly.
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ void renorm(Pair& p) { fast_two_sum(p.hi, p.lo, p.hi, p.lo); }

// x += inc (inc a plain float): TwoSum, error folded into lo.
__device__ __forceinline__ void add_comp(Pair& x, float inc) {
  float s, e;
  two_sum(x.hi, inc, s, e);
  x.hi = s;
  x.lo = __fadd_rn(x.lo, e);
}

// x += s * q with s = (sh, sl), q a pair: exact leading product + cross terms.
// FAST: the angle is known to outweigh the increment (|x.hi| >= |p|), as for
// FP32C angles held in [kWinLo, kWinHi), so Fast2Sum is exact; otherwise TwoSum.
template <bool FAST>
__device__ __forceinline__ void drift_comp(Pair& x, float sh, float sl, const Pair& q) {
  const float p = __fmul_rn(sh, q.hi);
  float e = fmaf(sh, q.hi, -p);          // exact error of the product
  e = fmaf(sh, q.lo, e);
  e = fmaf(sl, q.hi, e);
  float s, t;
  if (FAST) fast_two_sum(x.hi, p, s, t);
  else two_sum(x.hi, p, s, t);
  x.hi = s;
  x.lo = __fadd_rn(x.lo, __fadd_rn(t, e));
}

// FP32 table sincos (Tang's method) with an exactly periodic table:
// theta_j = j D, D = 2 pi / 2048, table[j mod 2048] = (sin, cos)(2 pi j / 2048)
// rounded from long-double libm.  D is split D1 + D2 + D3 (D1 with 7
// significant bits, so j D1 is exact for |j| < 2^17) and the reduced argument
// r = ((hi - j D1) - j D2 - j D3) + lo is formed with one rounding per FMA at
// |r| <= D/2; angles therefore need no reduction before a kick as long as
// |hi| < 2^17 D ~ 400.  sin r ~ r, cos r ~ 1 - r^2/2 (neglected terms < 7e-10).
// 2 pi = C1 + C2 + C3 (C1, C2 with 18 significant bits) serves the exact
// reduction below.
struct Tab32 {
  float inv_d;       // 1 / D
  float d1, d2, d3;  // D = d1 + d2 + d3
  int jmax;          // 2047: last table index and index mask
  float inv2pi;      // 1 / (2 pi)
  float c1, c2, c3;  // 2 pi = c1 + c2 + c3
};

__device__ __forceinline__ void sincos_tab32(const Pair& x, const float2* __restrict__ sc, const Tab32& tb, float& s,
                                             float& c) {
  const float t = fmaf(x.hi, tb.inv_d, 12582912.0f);       // 1.5 * 2^23: rint(hi / D) in the low bits
  const float jf = __fsub_rn(t, 12582912.0f);
  const int j = (__float_as_int(t) - 0x4B400000) & tb.jmax;
  float r = fmaf(-jf, tb.d1, x.hi);                          // exact
  r = fmaf(-jf, tb.d2, r);
  r = fmaf(-jf, tb.d3, r);
  r = __fadd_rn(r, x.lo);
  const float2 e = sc[j];
  const float cm = __fmul_rn(-0.5f, __fmul_rn(r, r));
  s = fmaf(e.y, r, fmaf(e.x, cm, e.x));
  c = fmaf(-e.x, r, fmaf(e.y, cm, e.y));
}

// FP32C angles are held in the window [kWinLo, kWinHi) rad (any angle is
// one modulo 2 pi): there every angle outweighs its drift increment (|s q| <
// 400 per step, checked at renormalisation), so drifts add with Fast2Sum, and
// the table sincos stays exact (j d1 exact below 3217 rad).  An angle that
// leaves the window is brought back near kWinMid by whole turns.
constexpr float kWinLo = 1024.0f, kWinHi = 2048.0f, kWinMid = 1536.0f;

// x += k * 2 pi exactly, 2 pi = C1 + C2 + C3 (14, 16 bits and the rest), |k| < 256:
// k C1 and k C2 are exact products, two TwoSums keep both additions exact, so
// the only rounding is at the level of lo.
__device__ __forceinline__ void add_turns32(Pair& x, float kf, const Tab32& tb) {
  float s, e, s2, e2;
  two_sum(x.hi, __fmul_rn(kf, tb.c1), s, e);
  two_sum(s, __fmul_rn(kf, tb.c2), s2, e2);
  const float lo = fmaf(kf, tb.c3, __fadd_rn(__fadd_rn(x.lo, e), e2));
  fast_two_sum(s2, lo, x.hi, x.lo);
}

// Bring an angle pair back to within pi of kWinMid, laps -= k for the k turns
// added.  REDUCE64 variant: the same in FP64 (widen, add k * 2pi, split).
template <bool REDUCE64>
__device__ __forceinline__ void reduce_angle(Pair& x, int& lap, const Tab32& tb) {
  if (REDUCE64) {
    const double d = (double)x.hi + (double)x.lo;
    const double k = rint(((double)kWinMid - d) * (1.0 / kTwoPi));
    const double r = fma(k, kTwoPi, d);
    x.hi = __double2float_rn(r);
    x.lo = __double2float_rn(r - (double)x.hi);
    lap -= (int)k;
  } else {
    const float t = fmaf(__fsub_rn(kWinMid, x.hi), tb.inv2pi, 12582912.0f);   // kWinMid - hi: exact
    const float kf = __fsub_rn(t, 12582912.0f);
    add_turns32(x, kf, tb);
    lap -= __float_as_int(t) - 0x4B400000;
  }
}

template <bool REDUCE64>
__device__ __forceinline__ void end_step32(Traj32& t, const Tab32& tb) {
  renorm(t.u); renorm(t.v); renorm(t.z);
  renorm(t.qu); renorm(t.qv); renorm(t.pz);
  // outside [kWinLo, kWinHi): (bits - bits(1024)) as unsigned >= bits(2048) - bits(1024)
  const unsigned int lo_bits = 0x44800000u, span = 0x00800000u;
  const bool out = (unsigned int)(__float_as_int(t.u.hi) - lo_bits) >= span ||
                   (unsigned int)(__float_as_int(t.v.hi) - lo_bits) >= span ||
                   (unsigned int)(__float_as_int(t.z.hi) - lo_bits) >= span;
  if (out) {
    reduce_angle<REDUCE64>(t.u, t.lu, tb);
    reduce_angle<REDUCE64>(t.v, t.lv, tb);
    reduce_angle<REDUCE64>(t.z, t.lz, tb);
  }
}

template <bool TAN, bool FAST = false>
__device__ __forceinline__ void drift32(Traj32& t, float sh, float sl) {
  drift_comp<FAST>(t.u, sh, sl, t.qu);
  drift_comp<FAST>(t.v, sh, sl, t.qv);
  drift_comp<FAST>(t.z, sh, sl, t.pz);
  if (TAN) {
    t.du = fmaf(sh, t.dqu, t.du);
    t.dv = fmaf(sh, t.dqv, t.dv);
    t.dz = fmaf(sh, t.dpz, t.dz);
  }
}

template <bool TAN>
__device__ __forceinline__ void kick32(Traj32& t, float k2, const float2* sc, const Tab32& tb) {
  float su, cu, sv, cv, sz, cz;
  sincos_tab32(t.u, sc, tb, su, cu);
  sincos_tab32(t.v, sc, tb, sv, cv);
  sincos_tab32(t.z, sc, tb, sz, cz);
  const float kc = k2 * cz;
  const float G = kc * cz;    // k2 c_z^2
  const float Sp = kc * sz;   // k2 s_z c_z
  const float A = cu + cv;
  add_comp(t.qu, G * su);
  add_comp(t.qv, G * sv);
  add_comp(t.pz, Sp * A);
  if (TAN) {
    const float Gu = G * cu, Gv = G * cv;
    const float Yu = Sp * su, Yv = Sp * sv;
    const float Z = A * fmaf(2.0f, G, -k2);   // A (k4 c_z^2 - k2), k4 = 2 k2
    const float m2dz = -2.0f * t.dz;
    t.dqu = fmaf(Gu, t.du, t.dqu);
    t.dqu = fmaf(Yu, m2dz, t.dqu);
    t.dqv = fmaf(Gv, t.dv, t.dqv);
    t.dqv = fmaf(Yv, m2dz, t.dqv);
    t.dpz = fmaf(Z, t.dz, t.dpz);
    t.dpz = fmaf(-Yu, t.du, t.dpz);
    t.dpz = fmaf(-Yv, t.dv, t.dpz);
  }
}

__device__ __forceinline__ double pair_sq_d(const Pair& p) {
  const double d = (double)p.hi + (double)p.lo;
  return d * d;
}

}  // namespace arnold
