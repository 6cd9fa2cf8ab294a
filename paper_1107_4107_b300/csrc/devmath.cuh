// Device math shared by the kernels of libarnold: angle wrapping and sincos.
#pragma once
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

// FP64 sincos for x in [0, 2pi] by table lookup (Tang, "Table-lookup
// algorithms for elementary functions", 1991): x = theta_j + r with
// |r| <= D/2 ~ 7.7e-4, sin x = S cos r + C sin r, cos x = C cos r - S sin r,
// with Taylor polynomials sin r = r - r^3/6 (next term < 3e-18) and
// cos r - 1 = -r^2/2 + r^4/24 (next term < 3e-22).  10 FP64 instructions.
// The index j is taken from a truncated FP32 copy of x built with integer
// operations, so it costs no FP64 slot; j is clamped to the table.
__device__ __forceinline__ void sincos_tab64(double x, const double2* __restrict__ sc,
                                             const double* __restrict__ th, double& s, double& c) {
  constexpr float kInvD = (float)(kTabN / kTwoPi);
  int hi = __double2hiint(x);
  hi = max(hi, 0x38000000);                            // x < 2^-126 (or negative) -> index 0
  float xf = __int_as_float((hi - 0x38000000) << 3);   // FP32 exponent/mantissa from the FP64 bits
  float t = fmaf(xf, kInvD, 12582912.0f);              // 1.5 * 2^23: round-to-nearest integer in the low bits
  int j = __float_as_int(t) - 0x4B400000;
  j = min(max(j, 0), kTabN);
  const double2 e = sc[j];
  const double r = x - th[j];
  const double r2 = r * r;
  const double sr = fma(r2 * r, -1.0 / 6.0, r);
  const double cm = r2 * fma(r2, 1.0 / 24.0, -0.5);
  s = fma(e.y, sr, fma(e.x, cm, e.x));
  c = fma(-e.x, sr, fma(e.y, cm, e.y));
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
