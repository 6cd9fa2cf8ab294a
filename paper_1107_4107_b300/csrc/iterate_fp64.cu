// FP64 ensemble propagator: one thread per trajectory, state and tangent in
// registers for a whole launch, FP64 sincos tables in shared memory.  The
// FP64 pipe (1/74 of the FP32 one on this part) is the binding unit, so FP64
// instructions are spent only where FP64 accuracy needs them: 230 per
// composite step (sincos corrections, reductions, wraps and exponent scalings
// run on the integer and FP32 pipes; see devmath.cuh and step64.cuh).
//
// Per composite step (paper Sec. III: sixth-order symplectic integrator,
// read as a symmetric composition of drift-kick-drift leapfrogs with
// adjacent half-drifts merged): drift(sig_0), then for each substep k
// kick(tau_k) and drift(sig_{k+1}).
//   drift(s):  u += s q_u, v += s q_v, z += s p_z (wrapped, laps counted);
//              tangent du += s dq_u, ...
//   kick:      with (s_u, c_u), (s_v, c_v), (s_z, c_z) and g = c_z^2, sh = s_z c_z,
//              G = 2 tau eps g, Sp = 2 tau eps sh, A = c_u + c_v:
//              q_u += G s_u, q_v += G s_v, p_z += Sp A            (= -tau eps grad Hp)
//              dq_u += G c_u du - 2 Sp s_u dz
//              dq_v += G c_v dv - 2 Sp s_v dz
//              dp_z += A (4 tau eps g - 2 tau eps) dz - Sp (s_u du + s_v dv)
//              (the Hessian of Eq. 2 in rotated coordinates applied to the tangent)
// Every R steps: tangent renormalised (log of its norm accumulated, and the
// MEGNO sums when enabled) and the energy error sampled; every W steps: the
// window velocity V (Sec. IV) closed.
#include "step64.cuh"

namespace arnold {

namespace {

template <int M, bool TAN>
__global__ void __launch_bounds__(256) k_iterate_fp64(IterArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  double2* ssc = reinterpret_cast<double2*>(smem);
  double* sth = reinterpret_cast<double*>(smem + kTabEntries * sizeof(double2));
  // step coefficients in shared memory: the substep loop below is not unrolled
  __shared__ double s_sig[10], s_k2[9];
  if (threadIdx.x < 10) s_sig[threadIdx.x] = a.cf.sig[threadIdx.x];
  if (threadIdx.x < 9) s_k2[threadIdx.x] = a.cf.k2[threadIdx.x];
  load_tab64(a.sc, a.th, ssc, sth);   // ends with a block barrier

  const long long n = a.n;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    Traj64 t;
    t.u = a.s.st[i];
    t.v = a.s.st[n + i];
    t.z = a.s.st[2 * n + i];
    t.qu = a.s.st[3 * n + i];
    t.qv = a.s.st[4 * n + i];
    t.pz = a.s.st[5 * n + i];
    if (TAN) {
      t.du = a.s.tg[i];
      t.dv = a.s.tg[n + i];
      t.dz = a.s.tg[2 * n + i];
      t.dqu = a.s.tg[3 * n + i];
      t.dqv = a.s.tg[4 * n + i];
      t.dpz = a.s.tg[5 * n + i];
    }
    t.lu = a.s.lap[i];
    t.lv = a.s.lap[n + i];
    t.lz = a.s.lap[2 * n + i];
    double logsum = TAN ? a.s.logsum[i] : 0.0;
    double demax = a.s.demax[i];
    const double e0 = a.s.e0[i];
    int to_renorm = a.R - (int)(a.step0 % a.R);
    long long to_window = a.W > 0 ? a.W - a.step0 % a.W : 0;
    int bad = 0;

#pragma unroll 1
    for (int s = 0; s < a.nsteps; ++s) {
      drift64<TAN>(t, s_sig[0]);
      // Not unrolled: seven inlined kicks with their double-float sincos
      // overflow the instruction cache (ncu: fetch stalls).
#pragma unroll 1
      for (int k = 0; k < M; ++k) {
        kick64<TAN>(t, s_k2[k], ssc, sth);
        drift64<TAN>(t, s_sig[k + 1]);
      }
      if (--to_renorm == 0) {
        to_renorm = a.R;
        if (TAN) {
          const double n2 = 0.5 * (t.du * t.du + t.dv * t.dv) + t.dz * t.dz +
                            0.5 * (t.dqu * t.dqu + t.dqv * t.dqv) + t.dpz * t.dpz;
          const double l = 0.5 * log(n2);
          logsum += l;
          if (a.s.megno) megno_update(a.s.megno, n, i, (a.step0 + s + 1) / a.R, l);
          const double inv = rsqrt(n2);
          t.du *= inv; t.dv *= inv; t.dz *= inv;
          t.dqu *= inv; t.dqv *= inv; t.dpz *= inv;
          if (!isfinite(logsum)) bad = 1;
        }
        const double dE = fabs(energy64(t, a.eps, ssc, sth) - e0);
        demax = fmax(demax, dE);
        if (!isfinite(dE)) bad = 1;
        if (a.s.left && !inside_patch(0.5 * (t.qu + t.qv), 0.5 * (t.qu - t.qv), t.pz, a.s.patch)) a.s.left[i] = 1;
      }
      if (a.W > 0 && --to_window == 0) {
        to_window = a.W;
        const double inv_dt = 1.0 / ((double)a.W * a.h);
        const double dU = (t.u - a.s.ref[i]) + kTwoPi * (double)(t.lu - a.s.lapref[i]);
        const double dV = (t.v - a.s.ref[n + i]) + kTwoPi * (double)(t.lv - a.s.lapref[n + i]);
        const double dZ = (t.z - a.s.ref[2 * n + i]) + kTwoPi * (double)(t.lz - a.s.lapref[2 * n + i]);
        const double vx = 0.5 * (dU + dV) * inv_dt, vy = 0.5 * (dU - dV) * inv_dt, vz = dZ * inv_dt;
        a.s.V[i] = vx;
        a.s.V[n + i] = vy;
        a.s.V[2 * n + i] = vz;
        snapshot_v(a.s, n, i, (a.step0 + s + 1) / a.W, vx, vy, vz);
        a.s.ref[i] = t.u; a.s.ref[n + i] = t.v; a.s.ref[2 * n + i] = t.z;
        a.s.lapref[i] = t.lu; a.s.lapref[n + i] = t.lv; a.s.lapref[2 * n + i] = t.lz;
      }
    }

    a.s.st[i] = t.u;
    a.s.st[n + i] = t.v;
    a.s.st[2 * n + i] = t.z;
    a.s.st[3 * n + i] = t.qu;
    a.s.st[4 * n + i] = t.qv;
    a.s.st[5 * n + i] = t.pz;
    if (TAN) {
      a.s.tg[i] = t.du;
      a.s.tg[n + i] = t.dv;
      a.s.tg[2 * n + i] = t.dz;
      a.s.tg[3 * n + i] = t.dqu;
      a.s.tg[4 * n + i] = t.dqv;
      a.s.tg[5 * n + i] = t.dpz;
      a.s.logsum[i] = logsum;
    }
    a.s.lap[i] = t.lu;
    a.s.lap[n + i] = t.lv;
    a.s.lap[2 * n + i] = t.lz;
    a.s.demax[i] = demax;
    if (bad) atomicOr(a.flags, kFlagNonFinite);
  }
}

template <int M, bool TAN>
cudaError_t launch_one(const IterArgs& a, int block, int grid, cudaStream_t st) {
  auto k = k_iterate_fp64<M, TAN>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTabSmemBytes);
  if (e != cudaSuccess) return e;
  k<<<grid, block, kTabSmemBytes, st>>>(a);
  return cudaGetLastError();
}

template <int M, bool TAN>
int occupancy_one(int block) {
  auto k = k_iterate_fp64<M, TAN>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTabSmemBytes) != cudaSuccess)
    return 1;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, block, kTabSmemBytes) != cudaSuccess) return 1;
  return nb > 0 ? nb : 1;
}

}  // namespace

cudaError_t launch_iterate_fp64(const IterArgs& a, int scheme, bool tangent, int block, int grid, cudaStream_t st) {
  switch (scheme) {
    case ARNOLD_SCHEME_YOSHIDA6A:
      return tangent ? launch_one<7, true>(a, block, grid, st) : launch_one<7, false>(a, block, grid, st);
    case ARNOLD_SCHEME_TRIPLEJUMP6:
      return tangent ? launch_one<9, true>(a, block, grid, st) : launch_one<9, false>(a, block, grid, st);
    case ARNOLD_SCHEME_LEAPFROG2:
      return tangent ? launch_one<1, true>(a, block, grid, st) : launch_one<1, false>(a, block, grid, st);
  }
  return cudaErrorInvalidValue;
}

int fp64_blocks_per_sm(int scheme, bool tangent, int block) {
  switch (scheme) {
    case ARNOLD_SCHEME_YOSHIDA6A: return tangent ? occupancy_one<7, true>(block) : occupancy_one<7, false>(block);
    case ARNOLD_SCHEME_TRIPLEJUMP6: return tangent ? occupancy_one<9, true>(block) : occupancy_one<9, false>(block);
    case ARNOLD_SCHEME_LEAPFROG2: return tangent ? occupancy_one<1, true>(block) : occupancy_one<1, false>(block);
  }
  return 1;
}

}  // namespace arnold
