// FP64 composite-step building blocks (drift, kick with tangent, energy) in
// the rotated coordinates u = x + y, v = x - y; shared by the iterate and
// adjoint kernels so that recomputed forward states are bit-identical.
#pragma once
#include "devmath.cuh"

namespace arnold {

struct Traj64 {
  double u, v, z, qu, qv, pz;
  double du, dv, dz, dqu, dqv, dpz;
  int lu, lv, lz;
};

template <bool TAN>
__device__ __forceinline__ void drift64(Traj64& t, double s) {
  t.u = fma(s, t.qu, t.u);
  t.v = fma(s, t.qv, t.v);
  t.z = fma(s, t.pz, t.z);
  wrap_angle(t.u, t.lu);
  wrap_angle(t.v, t.lv);
  wrap_angle(t.z, t.lz);
  if (TAN) {
    t.du = fma(s, t.dqu, t.du);
    t.dv = fma(s, t.dqv, t.dv);
    t.dz = fma(s, t.dpz, t.dz);
  }
}

// k2 = 2 tau eps; the Hessian term 4 tau eps c_z^2 - 2 tau eps is formed as
// 2G - k2 with G = k2 c_z^2 (2G exact).  26 FP64 instructions with tangent.
template <bool TAN>
__device__ __forceinline__ void kick64(Traj64& t, double k2, const double2* sc, const double* th) {
  double su, cu, sv, cv, sz, cz;
  sincos_tab64(t.u, sc, th, su, cu);
  sincos_tab64(t.v, sc, th, sv, cv);
  sincos_tab64(t.z, sc, th, sz, cz);
  const double kc = k2 * cz;
  const double G = kc * cz;    // k2 c_z^2
  const double Sp = kc * sz;   // k2 s_z c_z
  const double A = cu + cv;
  t.qu = fma(G, su, t.qu);
  t.qv = fma(G, sv, t.qv);
  t.pz = fma(Sp, A, t.pz);
  if (TAN) {
    const double Gu = G * cu, Gv = G * cv;
    const double Yu = Sp * su, Yv = Sp * sv;
    const double Z = A * (times2(G) - k2);
    const double m2dz = neg_times2(t.dz);
    t.dqu = fma(Gu, t.du, t.dqu);
    t.dqu = fma(Yu, m2dz, t.dqu);
    t.dqv = fma(Gv, t.dv, t.dqv);
    t.dqv = fma(Yv, m2dz, t.dqv);
    t.dpz = fma(Z, t.dz, t.dpz);
    t.dpz = fma(-Yu, t.du, t.dpz);
    t.dpz = fma(-Yv, t.dv, t.dpz);
  }
}

// H = (q_u^2 + q_v^2)/4 + p_z^2/2 + eps (c_u + c_v) c_z^2   (Eq. 1 in rotated coordinates)
__device__ __forceinline__ double energy64(const Traj64& t, double eps, const double2* sc, const double* th) {
  double su, cu, sv, cv, sz, cz;
  sincos_tab64(t.u, sc, th, su, cu);
  sincos_tab64(t.v, sc, th, sv, cv);
  sincos_tab64(t.z, sc, th, sz, cz);
  const double kin = 0.25 * (t.qu * t.qu + t.qv * t.qv) + 0.5 * (t.pz * t.pz);
  return kin + eps * ((cu + cv) * (cz * cz));
}

}  // namespace arnold
