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

__global__ void k_set_state(InitArgs a) {
  const long long n = a.n;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double x = a.x_in[i], y = a.x_in[n + i], z = a.x_in[2 * n + i];
    reduce_any(x);
    reduce_any(y);
    const int lz = reduce_any(z);
    double u, v;
    int lu, lv;
    to_uv(x, y, u, v, lu, lv);
    double px = a.p_in[i], py = a.p_in[n + i], pz = a.p_in[2 * n + i];
    if (a.shell_mode) {   // fixed-energy initial momenta (Sec. IV)
      double su, cu, sv, cv, sz, cz;
      sincos_tab64(u, a.sc, a.th, su, cu);
      sincos_tab64(v, a.sc, a.th, sv, cv);
      sincos_tab64(z, a.sc, a.th, sz, cz);
      const double hp = (cu + cv) * (cz * cz);
      if (a.shell_mode == 1) {          // P = sqrt(2 (E - eps Hp)) * unit direction
        const double r = 2.0 * (a.E - a.eps * hp);
        const double m = sqrt(r);
        if (!(r >= 0.0)) atomicOr(a.flags, kFlagNonFinite);
        px *= m; py *= m; pz *= m;
      } else {                          // p_z = +sqrt(2 (E - eps Hp) - p_x^2 - p_y^2)
        const double r = 2.0 * (a.E - a.eps * hp) - px * px - py * py;
        pz = sqrt(r);
        if (!(r >= 0.0)) atomicOr(a.flags, kFlagNonFinite);
      }
    }
    // the parity of lu + lv carries the pi offset of x and y; displacements
    // are measured from here, so earlier laps of x and y are not kept
    init_common(a, i, u, v, z, px + py, px - py, pz, lu, lv, lz);
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
    case ARNOLD_IND_V: {
      if (a.kind == ARNOLD_IND_V && a.W > 0) {
        v[0] = a.s.V[i]; v[1] = a.s.V[n + i]; v[2] = a.s.V[2 * n + i];
        break;
      }
      load_state();
      const double dU = (u - a.s.ref[i]) + kTwoPi * (double)(lu - a.s.lapref[i]);
      const double dV = (vv - a.s.ref[n + i]) + kTwoPi * (double)(lv - a.s.lapref[n + i]);
      const double dZ = (z - a.s.ref[2 * n + i]) + kTwoPi * (double)(lz - a.s.lapref[2 * n + i]);
      const double sc = a.kind == ARNOLD_IND_V ? 1.0 / a.t : 1.0;
      v[0] = 0.5 * (dU + dV) * sc;
      v[1] = 0.5 * (dU - dV) * sc;
      v[2] = dZ * sc;
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
