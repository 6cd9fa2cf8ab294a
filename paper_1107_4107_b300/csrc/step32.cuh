// Compensated-FP32 building blocks (float pairs, TwoSum/TwoProd updates,
// float-pair mod-2pi wraps, FP32 table sincos, drift/kick) shared by the
// iterate and adjoint kernels so that recomputed states are bit-identical.
#pragma once
#include "devmath.cuh"

namespace arnold {

constexpr float kC2PiHi = 6.28318548202514648438f;        // float nearest 2pi
constexpr float kC2PiLo = -1.74845553146951715462e-07f;   // 2pi - kC2PiHi, rounded
constexpr int kC2PiHiBits = 0x40C90FDB;

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
__device__ __forceinline__ void drift_comp(Pair& x, float sh, float sl, const Pair& q) {
  const float p = __fmul_rn(sh, q.hi);
  float e = fmaf(sh, q.hi, -p);          // exact error of the product
  e = fmaf(sh, q.lo, e);
  e = fmaf(sl, q.hi, e);
  float s, t;
  two_sum(x.hi, p, s, t);
  x.hi = s;
  x.lo = __fadd_rn(x.lo, __fadd_rn(t, e));
}

template <bool REDUCE64>
__device__ __forceinline__ void wrap_pair(Pair& x, int& lap) {
  const int b = __float_as_int(x.hi);
  if (b >= kC2PiHiBits || b < 0) {
#pragma unroll 1
    for (int it = 0; it < 4096; ++it) {
      const int bb = __float_as_int(x.hi);
      if (bb >= kC2PiHiBits) {
        if (REDUCE64) {
          const double d = ((double)x.hi + (double)x.lo) - kTwoPi;
          x.hi = __double2float_rn(d);
          x.lo = __double2float_rn(d - (double)x.hi);
        } else {
          x.hi = __fsub_rn(x.hi, kC2PiHi);   // exact (Sterbenz)
          x.lo = __fsub_rn(x.lo, kC2PiLo);
        }
        lap += 1;
      } else if (bb < 0) {
        if (REDUCE64) {
          const double d = ((double)x.hi + (double)x.lo) + kTwoPi;
          x.hi = __double2float_rn(d);
          x.lo = __double2float_rn(d - (double)x.hi);
        } else {
          float s, e;
          two_sum(x.hi, kC2PiHi, s, e);
          x.hi = s;
          x.lo = __fadd_rn(x.lo, __fadd_rn(e, kC2PiLo));
        }
        lap -= 1;
      } else {
        break;
      }
    }
  }
}

// FP32 table sincos of the pair value hi + lo, hi in [-D/2, 2pi + D/2].
struct Tab32 {
  float inv_d;     // 1 / D
  float d;         // D (12 significant bits: j * D exact in FP32)
  int jmax;        // last table index
};

__device__ __forceinline__ void sincos_tab32(const Pair& x, const float2* __restrict__ sc, const Tab32& tb, float& s,
                                             float& c) {
  const float t = fmaf(x.hi, tb.inv_d, 12582912.0f);       // 1.5 * 2^23
  const float jf = __fsub_rn(t, 12582912.0f);
  int j = __float_as_int(t) - 0x4B400000;
  j = min(max(j, 0), tb.jmax);
  const float r = __fadd_rn(fmaf(-jf, tb.d, x.hi), x.lo);   // (hi - theta_j) exact, then + lo
  const float2 e = sc[j];
  const float cm = __fmul_rn(-0.5f, __fmul_rn(r, r));
  s = fmaf(e.y, r, fmaf(e.x, cm, e.x));
  c = fmaf(-e.x, r, fmaf(e.y, cm, e.y));
}

template <bool TAN, bool REDUCE64>
__device__ __forceinline__ void drift32(Traj32& t, float sh, float sl) {
  drift_comp(t.u, sh, sl, t.qu);
  drift_comp(t.v, sh, sl, t.qv);
  drift_comp(t.z, sh, sl, t.pz);
  wrap_pair<REDUCE64>(t.u, t.lu);
  wrap_pair<REDUCE64>(t.v, t.lv);
  wrap_pair<REDUCE64>(t.z, t.lz);
  if (TAN) {
    t.du = fmaf(sh, t.dqu, t.du);
    t.dv = fmaf(sh, t.dqv, t.dv);
    t.dz = fmaf(sh, t.dpz, t.dz);
  }
}

template <bool TAN>
__device__ __forceinline__ void kick32(Traj32& t, float k2, float k4, const float2* sc, const Tab32& tb) {
  float su, cu, sv, cv, sz, cz;
  sincos_tab32(t.u, sc, tb, su, cu);
  sincos_tab32(t.v, sc, tb, sv, cv);
  sincos_tab32(t.z, sc, tb, sz, cz);
  const float g = cz * cz;
  const float sh = sz * cz;
  const float G = k2 * g;
  const float Sp = k2 * sh;
  const float A = cu + cv;
  add_comp(t.qu, G * su);
  add_comp(t.qv, G * sv);
  add_comp(t.pz, Sp * A);
  if (TAN) {
    const float Gu = G * cu, Gv = G * cv;
    const float Yu = Sp * su, Yv = Sp * sv;
    const float Z = A * fmaf(k4, g, -k2);
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
