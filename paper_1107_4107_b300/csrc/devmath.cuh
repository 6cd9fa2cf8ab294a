// Device math shared by the kernels of libarnold: angle wrapping and sincos.
#pragma once
#include <cstring>
#include "arnold_internal.cuh"

namespace arnold {

// Bring an FP64 angle into [0, 2pi), one lap of the FP64 constant 2pi at a
// time, counting laps.  The range tests compare the IEEE bit pattern as a
// signed integer (an FP64 compare costs two DFMA slots on this part; the
// integer compare is free).  A value just below 0 that rounds up to 2pi on
// the way back lands on 0 with the lap undone.  At most 4096 laps per call.
__device__ __forceinline__ void wrap_angle(double& u, int& lap) {
  long long b = __double_as_longlong(u);
  if (b >= kTwoPiBits || b < 0) {
#pragma unroll 1
    for (int it = 0; it < 4096; ++it) {
      b = __double_as_longlong(u);
      if (b >= kTwoPiBits) { u -= kTwoPi; lap += 1; }
      else if (b < 0) { u += kTwoPi; lap -= 1; }
      else break;
    }
  }
}

// Bit views of FP64 / FP32 values, usable on the host as well (the sincos
// below is checked against long-double libm by a host harness).
__host__ __device__ __forceinline__ unsigned long long f64_bits(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long b;
  memcpy(&b, &x, 8);
  return b;
#endif
}
__host__ __device__ __forceinline__ double f64_from_bits(unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double x;
  memcpy(&x, &b, 8);
  return x;
#endif
}
__host__ __device__ __forceinline__ unsigned int f32_bits(float x) {
#ifdef __CUDA_ARCH__
  return __float_as_uint(x);
#else
  unsigned int b;
  memcpy(&b, &x, 4);
  return b;
#endif
}
__host__ __device__ __forceinline__ float f32_from_bits(unsigned int b) {
#ifdef __CUDA_ARCH__
  return __uint_as_float(b);
#else
  float x;
  memcpy(&x, &b, 4);
  return x;
#endif
}

// x = hi + lo + e with hi the leading 24 significand bits of x and lo the
// next 23 (both truncated toward zero), |e| < 2^-46 |x|, from the IEEE bits
// with integer and FP32 operations only (an FP64 -> FP32 conversion costs an
// FP64 issue slot on this part).  lo = 0 for |x| < 2^-80, hi = 0 for
// |x| < 2^-126.
__host__ __device__ __forceinline__ void split_f64(double x, float& hi, float& lo) {
  const unsigned long long b = f64_bits(x);
  const unsigned int h = (unsigned int)(b >> 32), l = (unsigned int)b;
  const int e = (int)((h >> 20) & 0x7FFu);
  const unsigned int sign = h & 0x80000000u;
  const unsigned int mh = ((h & 0xFFFFFu) << 3) | (l >> 29);
  hi = e > 896 ? f32_from_bits(sign | ((unsigned int)(e - 896) << 23) | mh) : 0.0f;
  // the next 23 significand bits as an exact FP32 integer, scaled by 2^(e - 1069)
  const float m = f32_from_bits(0x4B000000u | ((l & 0x1FFFFFFFu) >> 6)) - 8388608.0f;
  const float scale = f32_from_bits((unsigned int)(e > 942 ? e - 942 : 1) << 23);
  lo = e > 942 ? f32_from_bits(f32_bits(m * scale) ^ sign) : 0.0f;
}

// The FP64 value of a normalised float pair (|b| <= ulp(a) / 2), assembled in
// 64-bit integer arithmetic: a's significand at bits 52..29, b's aligned
// below it and added or subtracted, one normalising shift.  Bits of b below
// a's 53-bit window are dropped (error < 1 ulp of the result).
__host__ __device__ __forceinline__ double pair_to_f64(float a, float b) {
  const unsigned int ua = f32_bits(a), ub = f32_bits(b);
  const int ea = (int)((ua >> 23) & 0xFFu), eb = (int)((ub >> 23) & 0xFFu);
  const unsigned long long A = (unsigned long long)((ua & 0x7FFFFFu) | 0x800000u) << 29;
  const int k = ea - eb;
  const unsigned long long mb = (ub & 0x7FFFFFu) | 0x800000u;
  // b's significand in units of a's 53-bit window (selects, no branches)
  const int kl = (k >= 0 && k <= 29) ? 29 - k : 0, kr = k <= 29 ? 0 : (k < 53 ? k - 29 : 63);
  unsigned long long B = (mb << kl) >> kr;
  B = (eb != 0 && k >= 24) ? B : 0ULL;
  const unsigned long long M0 = ((ua ^ ub) & 0x80000000u) ? A - B : A + B;
  const bool up = (M0 >> 53) != 0, down = (M0 >> 52) == 0;
  const unsigned long long M = up ? M0 >> 1 : (down ? M0 << 1 : M0);
  const unsigned long long E = (unsigned long long)(ea + 896 + (up ? 1 : 0) - (down ? 1 : 0));
  const double d = f64_from_bits(((unsigned long long)(ua & 0x80000000u) << 32) | (E << 52) |
                                 (M & 0xFFFFFFFFFFFFFULL));
  return ea != 0 ? d : 0.0;
}

__host__ __device__ __forceinline__ int clz64(unsigned long long v) {
#ifdef __CUDA_ARCH__
  return __clzll((long long)v);
#else
  return v ? __builtin_clzll(v) : 64;
#endif
}

// r = x - t as a float pair (rh, rl), for t >= 0 and t = 0 or x / t in
// [1/4, 4] (then r is exact in FP64, Sterbenz): the significands are aligned
// and subtracted in 64-bit integers and the difference cut into its leading
// 24 and next 23 bits (truncated; |error| < 2^-46 |r|), with no FP64
// instruction.  |r| < 2^-126 gives rh = 0, |r| < 2^-80 gives rl = 0.
__host__ __device__ __forceinline__ void reduce_pair(double x, double t, float& rh, float& rl) {
  const unsigned long long bx = f64_bits(x), bt = f64_bits(t);
  const int ex = (int)((bx >> 52) & 0x7FFu), et = (int)(bt >> 52);
  const unsigned long long mx = (bx & 0xFFFFFFFFFFFFFULL) | (ex ? 0x10000000000000ULL : 0ULL);
  const unsigned long long mt = (bt & 0xFFFFFFFFFFFFFULL) | (et ? 0x10000000000000ULL : 0ULL);
  const int ex1 = ex ? ex : 1, et1 = et ? et : 1;    // subnormals share the exponent of 2^-1022
  const int e0 = (mt == 0 || ex1 < et1) ? ex1 : et1;
  const int sx = ex1 - e0, st = et1 - e0;          // 0..2 when both are non-zero
  // magnitudes shifted as unsigned (< 2^61), then signed
  const long long ax = (long long)(mx << (sx < 8 ? sx : 8));
  const long long R = ((bx >> 63) ? -ax : ax) - (mt == 0 ? 0LL : (long long)(mt << (st < 8 ? st : 8)));
  const unsigned int sign = R < 0 ? 0x80000000u : 0u;
  const unsigned long long U = (unsigned long long)(R < 0 ? -R : R);
  const int lz = clz64(U);
  const unsigned long long top = U << (lz & 63);
  const int p = 63 - lz + e0;                       // r = 1.xxx * 2^(p - 1075)
  const int fh = p - 948, fl = p - 994;             // FP32 exponent fields of rh and of rl's unit
  rh = (U != 0 && fh >= 1) ? f32_from_bits(sign | ((unsigned int)fh << 23) | ((unsigned int)(top >> 40) & 0x7FFFFFu))
                           : 0.0f;
  const float m = f32_from_bits(0x4B000000u | ((unsigned int)(top >> 17) & 0x7FFFFFu)) - 8388608.0f;
  const float sc = f32_from_bits((unsigned int)(fl >= 1 ? fl : 1) << 23);
  rl = (U != 0 && fl >= 1) ? f32_from_bits(f32_bits(m * sc) ^ sign) : 0.0f;
}

// 2x and -2x exactly, by an exponent increment (and a sign flip) on the
// IEEE bits: integer operations instead of an FP64 multiply.  Zero and
// subnormal x (|x| < 2^-1022) give x and -x.
__host__ __device__ __forceinline__ double times2(double x) {
  const unsigned long long b = f64_bits(x);
  return ((b >> 52) & 0x7FFu) ? f64_from_bits(b + (1ULL << 52)) : x;
}
__host__ __device__ __forceinline__ double neg_times2(double x) {
  const unsigned long long b = f64_bits(x) ^ 0x8000000000000000ULL;
  return ((b >> 52) & 0x7FFu) ? f64_from_bits(b + (1ULL << 52)) : f64_from_bits(b);
}

// Knuth's TwoSum on FP32 (host and device; the build keeps FP32 operations
// uncontracted).
__host__ __device__ __forceinline__ void tsum32(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// FP64 sincos for x in [0, 2pi] by table lookup (Tang, "Table-lookup
// algorithms for elementary functions", 1991): x = theta_j + r with
// |r| <= D/2 ~ 7.7e-4, theta_j = j D exact, so r = x - theta_j is exact
// (formed as a float pair in integer arithmetic), and
//   sin x = S + ds,  ds = C (r + sm) + S cm,
//   cos x = C + dc,  dc = C cm - S (r + sm),
// with sm = sin r - r = -r^3/6 + r^5/120 (next term < 3e-22; r^3/6 as a
// float pair) and
// cm = cos r - 1 = -r^2/2 + r^4/24 (next term < 3e-22).  Only the two final
// additions run in FP64 (2 FP64 instructions; the FP64 pipe is 1/74 of the
// FP32 one here).  The corrections |ds|, |dc| <= 7.7e-4 are formed in
// double-float arithmetic on the FP32 pipes from integer splits of r, S and C
// (relative error ~2^-46, i.e. < 1e-17 absolute) and joined back to FP64 in
// integer arithmetic, so the result keeps FP64 accuracy (the final rounding
// dominates: <= ~1.3e-16).  The index j comes from a truncated FP32 copy of
// x built with integer operations; j is clamped to the table.
__host__ __device__ __forceinline__ void sincos_tab64(double x, const double2* __restrict__ sc,
                                                      const double* __restrict__ th, double& s, double& c) {
  const float kInvD = (float)(kTabN / kTwoPi);
  int hi = (int)(f64_bits(x) >> 32);
  hi = hi > 0x38000000 ? hi : 0x38000000;               // x < 2^-126 (or negative) -> index 0
  const float xf = f32_from_bits((unsigned int)(hi - 0x38000000) << 3);   // FP32 bits from the FP64 bits
  const float t = fmaf(xf, kInvD, 12582912.0f);         // 1.5 * 2^23: round-to-nearest integer in the low bits
  int j = (int)f32_bits(t) - 0x4B400000;
  j = j < 0 ? 0 : (j > kTabN ? kTabN : j);
  const double2 e = sc[j];
  float rh, rl, Sh, Sl, Ch, Cl;
  reduce_pair(x, th[j], rh, rl);                         // r = x - theta_j, exact, no FP64 slot
  split_f64(e.x, Sh, Sl);
  split_f64(e.y, Ch, Cl);
  const float r2h = rh * rh;
  const float r2l = fmaf(rh + rh, rl, fmaf(rh, rh, -r2h));
  const float cmh = -0.5f * r2h;                                        // exact
  const float cml = fmaf(r2h * r2h, 1.0f / 24.0f, -0.5f * r2l);
  // sin r - r = -r^3/6 + r^5/120 with r^3/6 as a pair (1/6 = k6h + k6l)
  constexpr float k6h = 0.16666667163372039794921875f;       // 1/6 rounded to FP32
  constexpr float k6l = -4.96705373128255208333e-09f;         // 1/6 - k6h
  const float r3 = r2h * rh;
  const float r3e = fmaf(r2h, rl, fmaf(r2l, rh, fmaf(r2h, rh, -r3)));
  const float q = r3 * k6h;
  const float qe = fmaf(r3, k6l, fmaf(r3e, k6h, fmaf(r3, k6h, -q)));
  const float smh = -q;
  const float sml = fmaf(r3 * r2h, 1.0f / 120.0f, -qe);
  // C r and S r as pairs (TwoProd), S cm and C cm as pairs.  For j = 0 the
  // C r = r term is left to the FP64 sum (sin x = x + (sin r - r)), which
  // keeps sin x relatively accurate near 0.
  const bool j0 = j == 0;
  const float rhc = j0 ? 0.0f : rh, rlc = j0 ? 0.0f : rl;
  const float cr = Ch * rhc, cre = fmaf(Cl, rhc, fmaf(Ch, rlc, fmaf(Ch, rhc, -cr)));
  const float sr = Sh * rh, sre = fmaf(Sl, rh, fmaf(Sh, rl, fmaf(Sh, rh, -sr)));
  const float scm = Sh * cmh, scme = fmaf(Sl, cmh, fmaf(Sh, cml, fmaf(Sh, cmh, -scm)));
  const float ccm = Ch * cmh, ccme = fmaf(Cl, cmh, fmaf(Ch, cml, fmaf(Ch, cmh, -ccm)));
  float a, ae, b, be, dh, dl;
  tsum32(cr, scm, a, ae);
  tsum32(a, Ch * smh, b, be);
  tsum32(b, (((ae + be) + cre) + scme) + Ch * sml, dh, dl);
  s = (j0 ? x : e.x) + pair_to_f64(dh, dl);
  tsum32(ccm, -sr, a, ae);
  tsum32(a, ((ae + ccme) - sre) - Sh * (smh + sml), dh, dl);
  c = e.y + pair_to_f64(dh, dl);
  // x < 2^-60 (the pair would flush r = x): sin x = x, cos x = 1, exact in
  // FP64; selected with an integer test, no FP64 instruction.
  const bool tiny = (f64_bits(x) >> 52) < 963u;
  s = tiny ? x : s;
  c = tiny ? 1.0 : c;
}

// Copy the FP64 sincos tables into shared memory (whole block participates).
__device__ __forceinline__ void load_tab64(const double2* __restrict__ gsc, const double* __restrict__ gth,
                                           double2* ssc, double* sth) {
  for (int k = threadIdx.x; k < kTabEntries; k += blockDim.x) {
    ssc[k] = gsc[k];
    sth[k] = gth[k];
  }
  __syncthreads();
}

// SplitMix64 output number k (0-based) of the stream seeded with `seed`
// (Steele, Lea & Flood 2014; published finaliser constants).
__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed, unsigned long long k) {
  unsigned long long z = seed + (k + 1ULL) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Uniform angle in [0, 2pi): (r >> 11) * 2^-53 * 2pi, the same IEEE
// operations as the host generator.
__device__ __forceinline__ double uniform_angle(unsigned long long r) {
  double u = __dmul_rn((double)(r >> 11), 1.1102230246251565404236316680908203125e-16);
  return __dmul_rn(u, kTwoPi);
}

}  // namespace arnold
