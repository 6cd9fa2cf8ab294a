// Host-side check of the FP64 sincos building blocks of the CUDA path
// (paper_1107_4107_b300/csrc/devmath.cuh), compiled by nvcc for the host:
//   pair_to_f64   vs the exact sum (double)a + (double)b of normalised float pairs
//   split_f64     |hi + lo - x| <= 2^-46 |x|
//   reduce_pair   vs split_f64(x - t) when x - t is exact (Sterbenz)
//   sincos_tab64  vs long-double libm over [0, 2pi], table edges, tiny x
// Prints one JSON line of the worst errors; exit status 0.
#include <cmath>
#include <cstdio>
#include <random>
#include "../paper_1107_4107_b300/csrc/devmath.cuh"
using namespace arnold;

int main() {
  std::mt19937_64 g(20111107);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  std::uniform_int_distribution<int> X(-70, 8);
  double pair_err = 0.0, split_err = 0.0;
  for (long i = 0; i < 4000000; ++i) {
    const double v = ldexp(U(g), X(g));
    const float a = (float)v;
    const float b = (i % 5 == 0) ? 0.0f : (float)(v - (double)a);
    const double ref = (double)a + (double)b;
    const double got = pair_to_f64(a, b);
    if (ref != 0.0) pair_err = fmax(pair_err, fabs(got - ref) / fabs(ref));
    float h, l;
    split_f64(v, h, l);
    if (fabs(v) >= ldexp(1.0, -79)) split_err = fmax(split_err, fabs(((double)h + (double)l) - v) / fabs(v));   // documented range: lo = 0 below 2^-80
  }
  // the FP64 table exactly as the library builds it
  const double D0 = kTwoPi / (double)kTabN;
  unsigned long long bits;
  memcpy(&bits, &D0, 8);
  bits &= ~((1ULL << 14) - 1ULL);
  double D;
  memcpy(&D, &bits, 8);
  static double2 sc[kTabEntries];
  static double th[kTabEntries];
  for (int j = 0; j < kTabEntries; ++j) {
    th[j] = (double)j * D;
    sc[j].x = (double)sinl((long double)th[j]);
    sc[j].y = (double)cosl((long double)th[j]);
  }
  long reduce_mismatch = 0;
  double sin_err = 0.0, cos_err = 0.0, tiny_rel = 0.0;
  auto check = [&](double x) {
    double s, c;
    sincos_tab64(x, sc, th, s, c);
    sin_err = fmax(sin_err, (double)fabsl((long double)s - sinl((long double)x)));
    cos_err = fmax(cos_err, (double)fabsl((long double)c - cosl((long double)x)));
  };
  std::uniform_real_distribution<double> A(0.0, kTwoPi);
  for (long i = 0; i < 2000000; ++i) {
    const double x = A(g);
    check(x);
    const int j = (int)std::lround(x / D);
    if (j >= 1 && j <= kTabN) {
      float a, b, c, d;
      reduce_pair(x, th[j], a, b);
      split_f64(x - th[j], c, d);
      if (f32_bits(a) != f32_bits(c) || f32_bits(b) != f32_bits(d)) ++reduce_mismatch;
    }
  }
  for (int j = 0; j < kTabEntries; ++j)
    for (double f : {0.0, 0.5, -0.5, 0.4999999, -0.4999999, 1e-9, -1e-9}) {
      const double x = th[j] + f * D;
      if (x >= 0.0 && x <= kTwoPi) check(x);
    }
  // near 0 (table index 0) sin x keeps a small relative error as well
  std::uniform_real_distribution<double> L(-330.0, -3.12);   // x < D/2: table index 0
  for (long i = 0; i < 200000; ++i) {
    const double x = i < 8 ? (double[]){5e-324, 1e-300, 1e-40, 1e-30, 1e-20, 1e-10, 1e-5, 7.6e-4}[i] : pow(10.0, L(g));
    check(x);
    double s, c;
    sincos_tab64(x, sc, th, s, c);
    tiny_rel = fmax(tiny_rel, (double)(fabsl((long double)s - sinl((long double)x)) / sinl((long double)x)));
  }
  printf("{\"pair_to_f64_rel\": %.3e, \"split_f64_rel\": %.3e, \"reduce_pair_mismatch\": %ld, "
         "\"sin_abs\": %.3e, \"cos_abs\": %.3e, \"tiny_sin_rel\": %.3e}\n",
         pair_err, split_err, reduce_mismatch, sin_err, cos_err, tiny_rel);
  return 0;
}
