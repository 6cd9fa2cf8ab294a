// Set-up and read-out kernels: initial conditions (paper Sec. IV), state
// conversion between the paper's (X, P) and the rotated coordinates, and the
// per-trajectory indicators (FTLE, V, energy error, class).
#include <math.h>

#include "devmath.cuh"
#include "kernels.cuh"

namespace arnold {

namespace {

// Reduce an arbitrary angle into [0, 2pi); returns the laps removed.
__device__ __forceinline__ int reduce_any(double& x) {
  const double k = floor(x * (1.0 / kTwoPi));
  x = fma(-k, kTwoPi, x);
  int lap = (int)k;
  wrap_angle(x, lap);   // fix a rounding step over either end
  return lap;
}

// From reduced x, y in [0, 2pi) to reduced u = x + y, v = x - y and their laps.
__device__ __forceinline__ void to_uv(double x, double y, double& u, double& v, int& lu, int& lv) {
  u = x + y;
  v = x - y;
  lu = 0;
  lv = 0;
  wrap_angle(u, lu);
  wrap_angle(v, lv);
}

// Common tail of the two initialisers: energy reference, tangent, bookkeeping.
__device__ __forceinline__ void init_common(const InitArgs& a, long long i, double u, double v, double z, double qu,
                                            double qv, double pz, int lu, int lv, int lz) {
  const long long n = a.n;
  double su, cu, sv, cv, sz, cz;
  sincos_tab64(u, a.sc, a.th, su, cu);
  sincos_tab64(v, a.sc, a.th, sv, cv);
  sincos_tab64(z, a.sc, a.th, sz, cz);
  const double e0 = 0.25 * (qu * qu + qv * qv) + 0.5 * (pz * pz) + a.eps * ((cu + cv) * (cz * cz));
  if (a.s.st) {
    a.s.st[i] = u; a.s.st[n + i] = v; a.s.st[2 * n + i] = z;
    a.s.st[3 * n + i] = qu; a.s.st[4 * n + i] = qv; a.s.st[5 * n + i] = pz;
  }
  if (a.f.hi) {
    const double vals[6] = {u, v, z, qu, qv, pz};
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      Pair x;
      x.hi = __double2float_rn(vals[c]);
      x.lo = __double2float_rn(vals[c] - (double)x.hi);
      if (c < 3 && a.window_turns) add_turns32(x, (float)a.window_turns, a.tab32);   // exact
      a.f.hi[c * n + i] = x.hi;
      a.f.lo[c * n + i] = x.lo;
    }
  }
  const int T = a.window_turns;   // laps debited for the turns added (0 unless FP32C)
  a.s.lap[i] = lu - T; a.s.lap[n + i] = lv - T; a.s.lap[2 * n + i] = lz - T;
  a.s.lapref[i] = lu; a.s.lapref[n + i] = lv; a.s.lapref[2 * n + i] = lz;
  a.s.ref[i] = u; a.s.ref[n + i] = v; a.s.ref[2 * n + i] = z;
  a.s.e0[i] = e0;
  a.s.p0[i] = 0.5 * (qu + qv); a.s.p0[n + i] = 0.5 * (qu - qv); a.s.p0[2 * n + i] = pz;
  a.s.demax[i] = 0.0;
  if (a.s.logsum) a.s.logsum[i] = 0.0;
  if (a.s.megno) { a.s.megno[i] = 0.0; a.s.megno[n + i] = 0.0; }
  a.s.V[i] = 0.0; a.s.V[n + i] = 0.0; a.s.V[2 * n + i] = 0.0;
  if (a.s.left) a.s.left[i] = 0;
  if (a.tangent) {
    double w[6];
    if (a.w_in) {
#pragma unroll
      for (int c = 0; c < 6; ++c) w[c] = a.w_in[c * n + i];
    } else {
      const double c0 = 0.40824829046386301637;   // 1/sqrt(6)
#pragma unroll
      for (int c = 0; c < 6; ++c) w[c] = c0;
    }
    double n2 = 0.0;
#pragma unroll
    for (int c = 0; c < 6; ++c) n2 += w[c] * w[c];
    const double inv = 1.0 / sqrt(n2);
    const double t6[6] = {(w[0] + w[1]) * inv, (w[0] - w[1]) * inv, w[2] * inv,
                          (w[3] + w[4]) * inv, (w[3] - w[4]) * inv, w[5] * inv};
#pragma unroll
    for (int c = 0; c < 6; ++c) {
      if (a.s.tg) a.s.tg[c * n + i] = t6[c];
      if (a.f.tg) {
        const float hi = __double2float_rn(t6[c]);
        a.f.tg[c * n + i] = hi;
        if (a.f.tg_lo) a.f.tg_lo[c * n + i] = __double2float_rn(t6[c] - (double)hi);
      }
    }
  }
}

// One trajectory from the paper's (X, P): angles reduced, rotated coordinates,
// and for shell modes the fixed-energy momentum (Sec. IV): mode 1 scales the
// unit direction (px, py, pz) to |P| = sqrt(2 (E - eps Hp)), mode 2 sets
// p_z = +sqrt(2 (E - eps Hp) - p_x^2 - p_y^2).
__device__ __forceinline__ void set_one(const InitArgs& a, long long i, double x, double y, double z, double px,
                                        double py, double pz, int mode) {
  reduce_any(x);
  reduce_any(y);
  const int lz = reduce_any(z);
  double u, v;
  int lu, lv;
  to_uv(x, y, u, v, lu, lv);
  if (mode) {   // fixed-energy initial momenta (Sec. IV)
    double su, cu, sv, cv, sz, cz;
    sincos_tab64(u, a.sc, a.th, su, cu);
    sincos_tab64(v, a.sc, a.th, sv, cv);
    sincos_tab64(z, a.sc, a.th, sz, cz);
    const double hp = (cu + cv) * (cz * cz);
    if (mode == 1) {          // P = sqrt(2 (E - eps Hp)) * unit direction
      const double r = 2.0 * (a.E - a.eps * hp);
      const double m = sqrt(r);
      if (!(r >= 0.0)) atomicOr(a.flags, kFlagNonFinite);
      px *= m; py *= m; pz *= m;
    } else {                  // p_z = +sqrt(2 (E - eps Hp) - p_x^2 - p_y^2)
      const double r = 2.0 * (a.E - a.eps * hp) - px * px - py * py;
      pz = sqrt(r);
      if (!(r >= 0.0)) atomicOr(a.flags, kFlagNonFinite);
    }
  }
  // the parity of lu + lv carries the pi offset of x and y; displacements
  // are measured from here, so earlier laps of x and y are not kept
  init_common(a, i, u, v, z, px + py, px - py, pz, lu, lv, lz);
}

__global__ void k_set_state(InitArgs a) {
  const long long n = a.n;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    set_one(a, i, a.x_in[i], a.x_in[n + i], a.x_in[2 * n + i], a.p_in[i], a.p_in[n + i], a.p_in[2 * n + i],
            a.shell_mode);
}

// ---- initial conditions drawn on the device (Sec. IV, Figs. 2-4) ----------
// Candidate t draws SplitMix64(seed) counters 5t .. 5t+4, as the host generator
// does: three angles uniform on the torus, then two uniforms for the momentum.

__device__ __forceinline__ double uniform01_dev(unsigned long long r) {
  return __dmul_rn((double)(r >> 11), 1.1102230246251565404236316680908203125e-16);
}

// Sphere ensemble (Figs. 2-3): direction with cos theta uniform in
// [cos_lo, cos_hi] and phi uniform in [phi_lo, phi_hi]; |P| from the energy.
__global__ void k_init_sphere(InitArgs a, unsigned long long offset, double cos_lo, double cos_hi, double phi_lo,
                              double phi_hi) {
  const long long n = a.n;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const unsigned long long c = 5ULL * (offset + (unsigned long long)i);
    const double x = uniform_angle(splitmix64(a.seed, c));
    const double y = uniform_angle(splitmix64(a.seed, c + 1));
    const double z = uniform_angle(splitmix64(a.seed, c + 2));
    const double u = uniform01_dev(splitmix64(a.seed, c + 3));
    const double w = uniform01_dev(splitmix64(a.seed, c + 4));
    const double ct = cos_lo + (cos_hi - cos_lo) * u;
    const double ph = phi_lo + (phi_hi - phi_lo) * w;
    const double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double sp, cp;
    sincos(ph, &sp, &cp);
    set_one(a, i, x, y, z, st * cp, st * sp, ct, 1);
  }
}

// Gaussian cloud of Fig. 4: (p_x, p_y) = centre + sigma r (cos 2 pi u2, sin 2 pi u2),
// r = sqrt(-2 ln u1), u1 in (0, 1] (Box-Muller); p_z from the energy.  Returns
// whether the energy condition has a real p_z, and the candidate's values.
struct Cand { double x, y, z, px, py; };

__device__ __forceinline__ bool gauss_candidate(const InitArgs& a, unsigned long long t, double cx, double cy,
                                                double sigma, Cand& k) {
  const unsigned long long c = 5ULL * t;
  k.x = uniform_angle(splitmix64(a.seed, c));
  k.y = uniform_angle(splitmix64(a.seed, c + 1));
  k.z = uniform_angle(splitmix64(a.seed, c + 2));
  const double u1 = 1.0 - uniform01_dev(splitmix64(a.seed, c + 3));
  const double u2 = uniform01_dev(splitmix64(a.seed, c + 4));
  const double r = sqrt(-2.0 * log(u1));
  double s2, c2;
  sincos(kTwoPi * u2, &s2, &c2);
  k.px = cx + sigma * r * c2;
  k.py = cy + sigma * r * s2;
  // the energy condition as set_one evaluates it (the same angles, the same
  // rotated-coordinate sincos), so "valid" here means a real p_z there
  double x = k.x, y = k.y, u, v;
  int lu, lv;
  to_uv(x, y, u, v, lu, lv);
  double su, cu, sv, cv, sz, cz;
  sincos_tab64(u, a.sc, a.th, su, cu);
  sincos_tab64(v, a.sc, a.th, sv, cv);
  sincos_tab64(k.z, a.sc, a.th, sz, cz);
  const double hp = (cu + cv) * (cz * cz);
  return 2.0 * (a.E - a.eps * hp) - k.px * k.px - k.py * k.py >= 0.0;
}

constexpr int kDrawBlock = 256;

// Pass 1: valid candidates among t0 + [b * 256, (b + 1) * 256), per block.
__global__ void __launch_bounds__(kDrawBlock) k_gauss_count(InitArgs a, unsigned long long t0, double cx, double cy,
                                                            double sigma, int* counts) {
  __shared__ int s_warp[kDrawBlock / 32];
  Cand k;
  const bool ok = gauss_candidate(a, t0 + (unsigned long long)blockIdx.x * kDrawBlock + threadIdx.x, cx, cy, sigma, k);
  const unsigned int m = __ballot_sync(0xFFFFFFFFu, ok);
  if ((threadIdx.x & 31) == 0) s_warp[threadIdx.x >> 5] = __popc(m);
  __syncthreads();
  if (threadIdx.x == 0) {
    int s = 0;
    for (int w = 0; w < kDrawBlock / 32; ++w) s += s_warp[w];
    counts[blockIdx.x] = s;
  }
}

// Pass 2 (one block): exclusive prefix of the block counts, starting at the
// number already kept (*have), in block order; *have becomes the new total.
__global__ void __launch_bounds__(1024) k_gauss_scan(const int* counts, int nb, long long* offs, long long* have) {
  __shared__ long long s_part[1024];
  const int per = (nb + 1023) / 1024;
  const int lo = threadIdx.x * per, hi = min(nb, lo + per);
  long long s = 0;
  for (int b = lo; b < hi; ++b) s += counts[b];
  s_part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {   // 1024 partial sums: a plain sequential prefix, once
    long long acc = *have;
    for (int k = 0; k < 1024; ++k) {
      const long long v = s_part[k];
      s_part[k] = acc;
      acc += v;
    }
    *have = acc;
  }
  __syncthreads();
  long long acc = s_part[threadIdx.x];
  for (int b = lo; b < hi; ++b) {
    offs[b] = acc;
    acc += counts[b];
  }
}

// Pass 3: each valid candidate goes to slot offs[block] + its rank within the
// block (candidate order), while slots remain; the candidate that fills the
// last slot records its index + 1 in *drawn.
__global__ void __launch_bounds__(kDrawBlock) k_gauss_place(InitArgs a, unsigned long long t0, double cx, double cy,
                                                            double sigma, const long long* offs,
                                                            unsigned long long* drawn) {
  __shared__ int s_warp[kDrawBlock / 32];
  const unsigned long long t = t0 + (unsigned long long)blockIdx.x * kDrawBlock + threadIdx.x;
  Cand k;
  const bool ok = gauss_candidate(a, t, cx, cy, sigma, k);
  const unsigned int m = __ballot_sync(0xFFFFFFFFu, ok);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) s_warp[warp] = __popc(m);
  __syncthreads();
  int before = 0;
  for (int w = 0; w < warp; ++w) before += s_warp[w];
  before += __popc(m & ((1u << lane) - 1u));
  const long long slot = offs[blockIdx.x] + before;
  if (ok && slot < a.n) {
    set_one(a, slot, k.x, k.y, k.z, k.px, k.py, 0.0, 2);
    if (slot == a.n - 1) *drawn = t + 1;
  }
}

// Grid-slice initial conditions (Sec. IV): see arnold_init_grid in arnold.h.
__global__ void k_init_grid(InitArgs a) {
  const long long n = a.n;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const long long tg = a.row0 * a.G + i;
    const long long col = tg % a.G, row = tg / a.G;
    const double ui = __ddiv_rn(__dadd_rn((double)col, 0.5), (double)a.G);
    const double uj = __ddiv_rn(__dadd_rn((double)row, 0.5), (double)a.G);
    const double px = __dmul_rn(__dsub_rn(__dmul_rn(2.0, ui), 1.0), a.half_width);
    const double py = __dmul_rn(__dsub_rn(__dmul_rn(2.0, uj), 1.0), a.half_width);
    const unsigned long long c = 3ULL * (unsigned long long)tg;
    const double x = uniform_angle(splitmix64(a.seed, c));
    const double y = uniform_angle(splitmix64(a.seed, c + 1));
    const double z = uniform_angle(splitmix64(a.seed, c + 2));
    double u, v;
    int lu, lv;
    to_uv(x, y, u, v, lu, lv);
    double su, cu, sv, cv, sz, cz;
    sincos_tab64(u, a.sc, a.th, su, cu);
    sincos_tab64(v, a.sc, a.th, sv, cv);
    sincos_tab64(z, a.sc, a.th, sz, cz);
    const double hp = (cu + cv) * (cz * cz);           // Eq. 2 = cos x cos y (1 + cos 2z)
    const double r = 2.0 * (a.E - a.eps * hp) - px * px - py * py;
    const double pz = sqrt(r);                          // NaN if r < 0 (excluded by the grid half-width)
    if (!(r >= 0.0)) atomicOr(a.flags, kFlagNonFinite);
    if (a.raw_out) {   // the generated values, for bit-exact tests
      a.raw_out[i] = x; a.raw_out[n + i] = y; a.raw_out[2 * n + i] = z;
      a.raw_out[3 * n + i] = px; a.raw_out[4 * n + i] = py; a.raw_out[5 * n + i] = pz;
    }
    init_common(a, i, u, v, z, px + py, px - py, pz, lu, lv, 0);
  }
}

// ---------------------------------------------------------------- readout ---
__device__ __forceinline__ double reduce_pi_parity(double half, int par) {
  // half in (-pi, 2pi): add pi when the lap parity is odd, then wrap
  double x = par ? half + kPi : half;
  int dummy = 0;
  wrap_angle(x, dummy);
  return x;
}

__device__ __forceinline__ double load_pair(const Fp32cState& f, long long k) {
  return (double)f.hi[k] + (double)f.lo[k];
}

// The indicator of one trajectory: `v` holds its value in each output row
// (3 for X, P, dX, V; 6 for the tangent; 1 otherwise), `b` the byte of the
// u8 kinds.  Only the arrays the kind needs are read.
__device__ __forceinline__ void indicator_one(const ReadArgs& a, long long i, double* v, unsigned char& b) {
  const long long n = a.n;
  double u = 0.0, vv = 0.0, z = 0.0, qu = 0.0, qv = 0.0, pz = 0.0;
  int lu = 0, lv = 0, lz = 0;
  auto load_state = [&]() {
    if (a.fp32c) {
      u = load_pair(a.f, i); vv = load_pair(a.f, n + i); z = load_pair(a.f, 2 * n + i);
      qu = load_pair(a.f, 3 * n + i); qv = load_pair(a.f, 4 * n + i); pz = load_pair(a.f, 5 * n + i);
    } else {
      u = a.s.st[i]; vv = a.s.st[n + i]; z = a.s.st[2 * n + i];
      qu = a.s.st[3 * n + i]; qv = a.s.st[4 * n + i]; pz = a.s.st[5 * n + i];
    }
    lu = a.s.lap[i]; lv = a.s.lap[n + i]; lz = a.s.lap[2 * n + i];
    if (a.fp32c) {   // pair states keep angles unreduced between exact reductions: bring them into [0, 2pi)
      lu += reduce_any(u);
      lv += reduce_any(vv);
      lz += reduce_any(z);
    }
  };
  auto load_tangent = [&](double* w) {
    for (int c = 0; c < 6; ++c)
      w[c] = a.fp32c ? (double)a.f.tg[c * n + i] + (a.f.tg_lo ? (double)a.f.tg_lo[c * n + i] : 0.0)
                     : a.s.tg[c * n + i];
  };
  switch (a.kind) {
    case ARNOLD_IND_X: {
      load_state();
      const int par = (lu + lv) & 1;
      v[0] = reduce_pi_parity(0.5 * (u + vv), par);
      v[1] = reduce_pi_parity(0.5 * (u - vv), par);
      v[2] = z;
      break;
    }
    case ARNOLD_IND_P:
      load_state();
      v[0] = 0.5 * (qu + qv);
      v[1] = 0.5 * (qu - qv);
      v[2] = pz;
      break;
    case ARNOLD_IND_DX:
    case ARNOLD_IND_V:
    case ARNOLD_IND_VDEV: {
      if (a.kind != ARNOLD_IND_DX && a.W > 0) {
        v[0] = a.s.V[i]; v[1] = a.s.V[n + i]; v[2] = a.s.V[2 * n + i];
      } else {
        load_state();
        const double dU = (u - a.s.ref[i]) + kTwoPi * (double)(lu - a.s.lapref[i]);
        const double dV = (vv - a.s.ref[n + i]) + kTwoPi * (double)(lv - a.s.lapref[n + i]);
        const double dZ = (z - a.s.ref[2 * n + i]) + kTwoPi * (double)(lz - a.s.lapref[2 * n + i]);
        const double sc = a.kind == ARNOLD_IND_DX ? 1.0 : 1.0 / a.t;
        v[0] = 0.5 * (dU + dV) * sc;
        v[1] = 0.5 * (dU - dV) * sc;
        v[2] = dZ * sc;
      }
      if (a.kind == ARNOLD_IND_VDEV) {   // |V - P(0)|: regular cells keep V near their initial momentum
        const double ex = v[0] - a.s.p0[i], ey = v[1] - a.s.p0[n + i], ez = v[2] - a.s.p0[2 * n + i];
        v[0] = sqrt(ex * ex + ey * ey + ez * ez);
        v[1] = v[2] = 0.0;
      }
      break;
    }
    case ARNOLD_IND_TANGENT: {
      double w[6];
      load_tangent(w);
      v[0] = 0.5 * (w[0] + w[1]);
      v[1] = 0.5 * (w[0] - w[1]);
      v[2] = w[2];
      v[3] = 0.5 * (w[3] + w[4]);
      v[4] = 0.5 * (w[3] - w[4]);
      v[5] = w[5];
      break;
    }
    case ARNOLD_IND_LOGSUM:
      v[0] = a.s.logsum[i];
      break;
    case ARNOLD_IND_MEGNO:      // <Y>_m = Ysum / m (0 before the first renormalisation)
      v[0] = a.m > 0 ? a.s.megno[n + i] / (double)a.m : 0.0;
      break;
    case ARNOLD_IND_MEGNO_Y:    // Y_m = 2 S / m
      v[0] = a.m > 0 ? 2.0 * a.s.megno[i] / (double)a.m : 0.0;
      break;
    case ARNOLD_IND_LEFT:
      b = a.s.left ? a.s.left[i] : 0;
      break;
    case ARNOLD_IND_DE_MAX:
      v[0] = a.s.demax[i];
      break;
    case ARNOLD_IND_DE: {
      load_state();
      double su, cu, sv, cv, sz, cz;
      sincos_tab64(u, a.sc, a.th, su, cu);
      sincos_tab64(vv, a.sc, a.th, sv, cv);
      sincos_tab64(z, a.sc, a.th, sz, cz);
      const double H = 0.25 * (qu * qu + qv * qv) + 0.5 * (pz * pz) + a.eps * ((cu + cv) * (cz * cz));
      v[0] = fabs(H - a.s.e0[i]);
      break;
    }
    case ARNOLD_IND_CHI:
    case ARNOLD_IND_CLASS: {
      double w[6];
      load_tangent(w);
      const double n2 = 0.5 * (w[0] * w[0] + w[1] * w[1]) + w[2] * w[2] + 0.5 * (w[3] * w[3] + w[4] * w[4]) +
                        w[5] * w[5];
      const double chi = (a.s.logsum[i] + 0.5 * log(n2)) / a.t;
      v[0] = chi;
      b = chi > a.threshold ? 1 : 0;
      break;
    }
  }
}

// Values of trajectories i and i + 1 in one SoA row: a 16-byte (or 2-byte)
// vector store when both exist and the address is aligned (a row starts at
// r n, so an odd n misaligns every other row), scalar stores otherwise.
__device__ __forceinline__ void put2(double* row, long long i, bool two, double x0, double x1) {
  double* p = row + i;
  if (two && (reinterpret_cast<unsigned long long>(p) & 15ULL) == 0) {
    *reinterpret_cast<double2*>(p) = make_double2(x0, x1);
  } else {
    p[0] = x0;
    if (two) p[1] = x1;
  }
}
__device__ __forceinline__ void put2(unsigned char* row, long long i, bool two, unsigned char x0,
                                     unsigned char x1) {
  unsigned char* p = row + i;
  if (two && (reinterpret_cast<unsigned long long>(p) & 1ULL) == 0) {
    *reinterpret_cast<uchar2*>(p) = make_uchar2(x0, x1);
  } else {
    p[0] = x0;
    if (two) p[1] = x1;
  }
}

// Read-out: each thread computes two consecutive trajectories and writes them
// with vector stores, so a warp writes 512 contiguous bytes of every f64 row.
__global__ void k_indicator(ReadArgs a) {
  const long long n = a.n;
  const int rows = (a.kind == ARNOLD_IND_TANGENT) ? 6
                   : (a.kind == ARNOLD_IND_X || a.kind == ARNOLD_IND_P || a.kind == ARNOLD_IND_DX ||
                      a.kind == ARNOLD_IND_V) ? 3 : 1;
  const bool bytes = a.kind == ARNOLD_IND_CLASS || a.kind == ARNOLD_IND_LEFT;
  for (long long i = 2 * ((long long)blockIdx.x * blockDim.x + threadIdx.x); i < n;
       i += 2 * (long long)gridDim.x * blockDim.x) {
    const bool two = i + 1 < n;
    double v0[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, v1[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    unsigned char b0 = 0, b1 = 0;
    indicator_one(a, i, v0, b0);
    if (two) indicator_one(a, i + 1, v1, b1);
    if (bytes) {
      put2((unsigned char*)a.out, i, two, b0, b1);
    } else {
#pragma unroll
      for (int r = 0; r < 6; ++r)
        if (r < rows) put2((double*)a.out + r * n, i, two, v0[r], v1[r]);
    }
  }
}

__global__ void k_debug_sincos(const double* x, double* s, double* c, long long n, const double2* sc,
                               const double* th) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double ss, cc;
    sincos_tab64(x[i], sc, th, ss, cc);
    s[i] = ss;
    c[i] = cc;
  }
}

// Density of V on the momentum sphere (Sec. IV, F of Figs. 2-4): counts of the
// direction of V in n_cos x n_phi equal-width cells of cos theta and phi over
// the patch; directions outside the patch, and (filtered) trajectories that
// left the tracked area, are not counted.
__global__ void k_vhist(long long n, const double* V, const unsigned char* left, int filtered, double c0, double c1,
                        double f0, double f1, int n_cos, int n_phi, unsigned long long* counts) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    if (filtered && left && left[i]) continue;
    const double vx = V[i], vy = V[n + i], vz = V[2 * n + i];
    const double m = sqrt(vx * vx + vy * vy + vz * vz);
    const double c = vz / m;
    double phi = atan2(vy, vx);
    if (phi < 0.0) phi += kTwoPi;
    if (!(c >= c0 && c <= c1 && phi >= f0 && phi <= f1)) continue;
    int a = (int)((c - c0) / (c1 - c0) * n_cos);
    int b = (int)((phi - f0) / (f1 - f0) * n_phi);
    a = min(max(a, 0), n_cos - 1);
    b = min(max(b, 0), n_phi - 1);
    atomicAdd(&counts[(long long)a * n_phi + b], 1ULL);
  }
}

}  // namespace

cudaError_t launch_vhist(long long n, const double* V, const unsigned char* left, int filtered, const double* p4,
                         int n_cos, int n_phi, unsigned long long* counts, int grid, cudaStream_t st) {
  k_vhist<<<grid, 256, 0, st>>>(n, V, left, filtered, p4[0], p4[1], p4[2], p4[3], n_cos, n_phi, counts);
  return cudaGetLastError();
}

cudaError_t launch_set_state(const InitArgs& a, int grid, int block, cudaStream_t st) {
  k_set_state<<<grid, block, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_init_sphere(const InitArgs& a, unsigned long long offset, const double* patch4, int grid,
                               cudaStream_t st) {
  k_init_sphere<<<grid, 256, 0, st>>>(a, offset, patch4[0], patch4[1], patch4[2], patch4[3]);
  return cudaGetLastError();
}

cudaError_t launch_gauss_chunk(const InitArgs& a, unsigned long long t0, int nb, double cx, double cy, double sigma,
                               int* counts, long long* offs, long long* have, unsigned long long* drawn,
                               cudaStream_t st) {
  k_gauss_count<<<nb, kDrawBlock, 0, st>>>(a, t0, cx, cy, sigma, counts);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_gauss_scan<<<1, 1024, 0, st>>>(counts, nb, offs, have);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_gauss_place<<<nb, kDrawBlock, 0, st>>>(a, t0, cx, cy, sigma, offs, drawn);
  return cudaGetLastError();
}

cudaError_t launch_init_grid(const InitArgs& a, int grid, int block, cudaStream_t st) {
  k_init_grid<<<grid, block, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_indicator(const ReadArgs& a, int grid, int block, cudaStream_t st) {
  k_indicator<<<grid, block, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_debug_sincos64(const double* x, double* s, double* c, long long n, const double2* sc,
                                  const double* th, cudaStream_t st) {
  long long g = (n + 255) / 256;
  int grid = (int)(g > 4096 ? 4096 : (g < 1 ? 1 : g));
  k_debug_sincos<<<grid, 256, 0, st>>>(x, s, c, n, sc, th);
  return cudaGetLastError();
}

}  // namespace arnold
