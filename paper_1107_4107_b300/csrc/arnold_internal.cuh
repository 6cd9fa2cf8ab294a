// Internal definitions shared by the kernels and the C-ABI layer of libarnold.
//
// State layout in HBM (structure of arrays, component-major, n trajectories):
// the library keeps each trajectory in the rotated coordinates
//     u = x + y,  v = x - y,  z,   q_u = p_x + p_y,  q_v = p_x - p_y,  p_z,
// in which the potential of Eq. 2 is a sum of its resonance modes,
//     cos x cos y (1 + cos 2z) = (cos u + cos v) cos^2 z,
// so a kick needs no products of sines of different angles.  u, v, z are
// reduced into [0, 2pi) with integer lap counters; x = (u + v)/2 and
// y = (u - v)/2 are recovered exactly modulo 2pi from the parity of the
// total laps of u and v.  Conversions to the paper's (X, P) happen only at
// set_state and when indicators are read.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/arnold.h"

namespace arnold {

constexpr double kTwoPi = 6.283185307179586476925286766559;
constexpr double kPi = 3.14159265358979323846264338328;
// Bit pattern of the double closest to 2 pi (positive doubles order like int64).
constexpr long long kTwoPiBits = 0x401921FB54442D18LL;

// Table-driven sincos (Tang's table-lookup method): theta_j = j * D with
// D ~= 2 pi / N rounded to a double whose low 14 mantissa bits are zero, so
// every theta_j (j <= N) is an exact double; the table holds
// (sin theta_j, cos theta_j) rounded from long-double libm values, and theta_j.
constexpr int kTabN = 4096;
constexpr int kTabEntries = kTabN + 1;
constexpr size_t kTabSmemBytes = kTabEntries * (sizeof(double2) + sizeof(double));

// Composite-step coefficients of one scheme, scaled for one launch:
// drifts sig[0..m] (merged half-substeps times h) and kicks
// k2 = 2 tau eps, k4 = 4 tau eps with tau = w_k h.
struct StepCoef {
  int m;             // kicks per step
  double sig[10];
  double k2[9];
  double k4[9];
  float sig_hi[10], sig_lo[10];   // FP32C: sigma as a float pair
  float k2f[9], k4f[9];
};

// Device-side error flags (bits of one int, set with atomicOr, read by the host).
enum : int { kFlagNonFinite = 1, kFlagTimeout = 2, kFlagBadIndex = 4, kFlagRange = 8 };

struct Fp64State {
  double* st;      // [6][n] u, v, z, q_u, q_v, p_z (null for FP32C contexts)
  double* tg;      // [6][n] du, dv, dz, dq_u, dq_v, dp_z (null when tangent off or FP32C)
  int* lap;        // [3][n] total laps of u, v, z
  int* lapref;     // [3][n] laps at the window start
  double* ref;     // [3][n] reduced u, v, z at the window start
  double* logsum;  // [n]
  double* demax;   // [n]
  double* e0;      // [n] H at t = 0
  double* V;       // [3][n] V (x, y, z components) of the last closed window
  double* p0;      // [3][n] momenta p_x, p_y, p_z at t = 0 (for |V - P(0)|)
  unsigned char* left;  // [n] area tracking: 1 once the momentum direction left the patch (null = off)
  double patch[4];      // cos_lo, cos_hi, phi_lo, phi_hi of the tracked patch
  double* megno;        // [2][n] MEGNO sums S = sum_j j l_j and Ysum = sum_j Y_j (null = off)
  double* snap;         // [snap_k][3][n] V of window w in slot w - 1 (caller-owned device memory; null = off)
  long long snap_k;     // slots in snap
};

// Snapshot of the V of window w (w = 1, 2, ... from the clock reset) into slot
// w - 1 of the caller's [snap_k][3][n] array, if there is one and it has room.
__device__ __forceinline__ void snapshot_v(const Fp64State& s, long long n, long long i, long long w, double vx,
                                           double vy, double vz) {
  if (s.snap && w >= 1 && w <= s.snap_k) {
    double* o = s.snap + (w - 1) * 3 * n;
    o[i] = vx;
    o[n + i] = vy;
    o[2 * n + i] = vz;
  }
}

// MEGNO (Cincotta & Simo 2000) sampled at the renormalisation points: at the
// j-th renormalisation (j counted from the start of the run) with log growth
// l over the interval, S += j l and Ysum += Y_j = 2 S / j.  Read-modify-write
// in HBM once per renormalisation interval, so nothing stays live in the step.
__device__ __forceinline__ void megno_update(double* mg, long long n, long long i, long long j, double l) {
  const double jd = (double)j;
  const double S = mg[i] + jd * l;
  mg[i] = S;
  mg[n + i] += 2.0 * S / jd;
}

// Area tracking (Sec. IV, zooms of Fig. 3): is the momentum direction inside
// [cos_lo, cos_hi] x [phi_lo, phi_hi] (phi = atan2(p_y, p_x) in [0, 2pi))?
__device__ __forceinline__ bool inside_patch(double px, double py, double pz, const double* patch) {
  const double m = sqrt(px * px + py * py + pz * pz);
  const double c = pz / m;
  double phi = atan2(py, px);
  if (phi < 0.0) phi += kTwoPi;
  return c >= patch[0] && c <= patch[1] && phi >= patch[2] && phi <= patch[3];
}

struct Fp32cState {
  float* hi;       // [6][n] u, v, z, q_u, q_v, p_z (leading parts)
  float* lo;       // [6][n] trailing parts (value = hi + lo)
  float* tg;       // [6][n] tangent in FP32 (DF64: the leading words)
  float* tg_lo;    // [6][n] DF64 only: trailing words of the double-float tangent (null otherwise)
};

struct IterArgs {
  Fp64State s;
  Fp32cState f;
  const double2* sc;   // FP64 sincos table
  const double* th;
  const float2* scf;   // FP32 sincos table
  const float4* scd;   // DF64 sincos table (sin hi, sin lo, cos hi, cos lo)
  long long n;
  long long step0;     // steps taken before this launch
  int nsteps;          // steps in this launch
  int R;               // renormalisation / energy-sampling interval
  long long W;         // window (0 = none)
  double h, eps;
  StepCoef cf;
  int* flags;
};

// Host helpers implemented in the .cu files.
cudaError_t launch_iterate_fp64(const IterArgs& a, int scheme, bool tangent, int block, int grid,
                                cudaStream_t st);
cudaError_t launch_iterate_fp32c(const IterArgs& a, int scheme, bool tangent, int block, int grid,
                                 cudaStream_t st);
cudaError_t launch_iterate_df64(const IterArgs& a, int scheme, bool tangent, bool fast, int block, int grid,
                                cudaStream_t st);
int fp64_blocks_per_sm(int scheme, bool tangent, int block);
int df64_blocks_per_sm(int scheme, bool tangent, bool fast, int block);
int fp32c_blocks_per_sm(int scheme, bool tangent, int block);

}  // namespace arnold
