// Adjoint (reverse-mode) of the N-step map, for gradients of a loss of the
// final state with respect to the initial state and to (h, eps).
//
// The forward map is the composite step of Sec. III (see step64.cuh) in the
// rotated coordinates; one step is D(s_0) K(tau_0) D(s_1) ... K(tau_{m-1}) D(s_m).
// Given lambda = dL/d(state) after an operation, the reverse sweep applies:
//   drift D(s = c h):  lambda_q += s lambda_X;          dL/dh += c (lambda_X . q)
//   kick at X_k:       lambda_X += J_k^T lambda_q,       J_k = d(kick increment)/dX
//                      (the transpose of the tangent update: Hessian of Eq. 2)
//                      F = lambda_q . (kick increment) / (2 tau eps);
//                      dL/dh += 2 d_k eps F;  dL/deps += 2 d_k h F
// States are recomputed from checkpoints: the forward run stores the state
// every C steps (C ~ sqrt(N)); for each segment, in reverse, the kernel
// re-runs the segment (same device functions as the forward kernels, so bit
// for bit) storing the state after every step in a scratch buffer; then, step
// by step in reverse, it runs each step backwards from its stored end state
// (reverse drift X -= s q, reverse kick q -= increment(X), sharing the kick's
// sincos with the adjoint), so the positions and momenta inside a step are
// regained to rounding without storing them.
#include "kernels.cuh"
#include "step32.cuh"
#include "step64.cuh"

namespace arnold {

namespace {

// Adjoint of kick k at X (sincos shared): lambda_X += J^T lambda_q and the
// parameter terms; then the kick is undone, q -= increment(X).
__device__ __forceinline__ void adj_kick64(double& lu, double& lv, double& lz, double lqu, double lqv, double lpz,
                                           Traj64& t, double k2, double k4, double ch, double ce, double& gh,
                                           double& ge, const double2* sc, const double* th) {
  double su, cu, sv, cv, sz, cz;
  sincos_tab64(t.u, sc, th, su, cu);
  sincos_tab64(t.v, sc, th, sv, cv);
  sincos_tab64(t.z, sc, th, sz, cz);
  const double g = cz * cz, sh = sz * cz;
  const double kc = k2 * cz;
  const double G = kc * cz, Sp = kc * sz, A = cu + cv;   // as the forward kick forms them
  const double sl = fma(su, lqu, sv * lqv);             // s_u lq_u + s_v lq_v, used twice
  const double F = fma(g, sl, (sh * A) * lpz);
  gh = fma(ch, F, gh);
  ge = fma(ce, F, ge);
  const double Z = A * fma(k4, g, -k2);
  lu = fma(G * cu, lqu, fma(-Sp * su, lpz, lu));
  lv = fma(G * cv, lqv, fma(-Sp * sv, lpz, lv));
  lz = fma(neg_times2(Sp), sl, fma(Z, lpz, lz));
  t.qu = fma(-G, su, t.qu);
  t.qv = fma(-G, sv, t.qv);
  t.pz = fma(-Sp, A, t.pz);
}

// Step coefficients of the FP64 adjoint, staged in shared memory (the
// substep loops are not unrolled: the inlined kicks would overflow the
// instruction cache).
struct AdjCoef64 {
  double sig[10], k2[9], k4[9], ch[9], ce[9], cd[10];
};

// Reverse sweep of one step: from the step's end state, undo drift m, kick
// m-1, ..., drift 0 (positions and momenta within the step are regained by
// running the step backwards; they match the forward ones to rounding),
// applying the adjoint of each operation on the way.
template <int M>
__device__ __forceinline__ void reverse_step64(Traj64& t, double& lu, double& lv, double& lz, double& lqu,
                                               double& lqv, double& lpz, double& gh, double& ge, const AdjCoef64& a,
                                               const double2* sc, const double* th) {
#pragma unroll 1
  for (int k = M; k >= 0; --k) {
    const double sg = a.sig[k];
    gh = fma(a.cd[k], fma(lu, t.qu, fma(lv, t.qv, lz * t.pz)), gh);
    lqu = fma(sg, lu, lqu);
    lqv = fma(sg, lv, lqv);
    lpz = fma(sg, lz, lpz);
    t.u = fma(-sg, t.qu, t.u);
    t.v = fma(-sg, t.qv, t.v);
    t.z = fma(-sg, t.pz, t.z);
    wrap_angle(t.u, t.lu);
    wrap_angle(t.v, t.lv);
    wrap_angle(t.z, t.lz);
    if (k > 0) adj_kick64(lu, lv, lz, lqu, lqv, lpz, t, a.k2[k - 1], a.k4[k - 1], a.ch[k - 1], a.ce[k - 1], gh, ge, sc, th);
  }
}

template <int M>
__global__ void __launch_bounds__(256) k_adjoint_fp64(AdjArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  double2* ssc = reinterpret_cast<double2*>(smem);
  double* sth = reinterpret_cast<double*>(smem + kTabEntries * sizeof(double2));
  __shared__ AdjCoef64 cf;
  if (threadIdx.x < 10) {
    cf.sig[threadIdx.x] = a.cf.sig[threadIdx.x];
    cf.cd[threadIdx.x] = a.cd[threadIdx.x];
  }
  if (threadIdx.x < 9) {
    cf.k2[threadIdx.x] = a.cf.k2[threadIdx.x];
    cf.k4[threadIdx.x] = a.cf.k4[threadIdx.x];
    cf.ch[threadIdx.x] = a.ch[threadIdx.x];
    cf.ce[threadIdx.x] = a.ce[threadIdx.x];
  }
  load_tab64(a.sc, a.th, ssc, sth);   // ends with a block barrier
  const long long n = a.n;
  const double* ck = a.ck64 + (long long)a.k * 6 * n;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    Traj64 t;
    t.u = ck[i]; t.v = ck[n + i]; t.z = ck[2 * n + i];
    t.qu = ck[3 * n + i]; t.qv = ck[4 * n + i]; t.pz = ck[5 * n + i];
    t.lu = t.lv = t.lz = 0;
    // pass 1: the state after every step of the segment (slot s = end of step s)
#pragma unroll 1
    for (int s = 0; s < a.steps; ++s) {
      drift64<false>(t, cf.sig[0]);
#pragma unroll 1
      for (int k = 0; k < M; ++k) {
        kick64<false>(t, cf.k2[k], ssc, sth);
        drift64<false>(t, cf.sig[k + 1]);
      }
      double* sg = a.seg64 + (long long)s * 6 * n;
      sg[i] = t.u; sg[n + i] = t.v; sg[2 * n + i] = t.z;
      sg[3 * n + i] = t.qu; sg[4 * n + i] = t.qv; sg[5 * n + i] = t.pz;
    }
    // pass 2: reverse sweep, each step run backwards from its stored end state
    double lu = a.lam[i], lv = a.lam[n + i], lz = a.lam[2 * n + i];
    double lqu = a.lam[3 * n + i], lqv = a.lam[4 * n + i], lpz = a.lam[5 * n + i];
    double gh = a.gh[i], ge = a.ge[i];
#pragma unroll 1
    for (int s = a.steps - 1; s >= 0; --s) {
      const double* sg = a.seg64 + (long long)s * 6 * n;
      t.u = sg[i]; t.v = sg[n + i]; t.z = sg[2 * n + i];
      t.qu = sg[3 * n + i]; t.qv = sg[4 * n + i]; t.pz = sg[5 * n + i];
      reverse_step64<M>(t, lu, lv, lz, lqu, lqv, lpz, gh, ge, cf, ssc, sth);
    }
    a.lam[i] = lu; a.lam[n + i] = lv; a.lam[2 * n + i] = lz;
    a.lam[3 * n + i] = lqu; a.lam[4 * n + i] = lqv; a.lam[5 * n + i] = lpz;
    a.gh[i] = gh;
    a.ge[i] = ge;
  }
}

// ------------------------------------------------------------------ FP32C ---
// Float-pair accumulator for the parameter gradients.
__device__ __forceinline__ void acc_pair(Pair& acc, float x) { add_comp(acc, x); }

__device__ __forceinline__ void adj_kick32(float& lu, float& lv, float& lz, float lqu, float lqv, float lpz,
                                           Traj32& t, float k2, float k4, float ch, float ce, Pair& gh, Pair& ge,
                                           const float2* sc, const Tab32& tb) {
  float su, cu, sv, cv, sz, cz;
  sincos_tab32(t.u, sc, tb, su, cu);
  sincos_tab32(t.v, sc, tb, sv, cv);
  sincos_tab32(t.z, sc, tb, sz, cz);
  const float g = cz * cz, sh = sz * cz;
  const float kc = k2 * cz;
  const float G = kc * cz, Sp = kc * sz, A = cu + cv;   // as the forward kick forms them
  const float F = fmaf(lqu * su, g, fmaf(lqv * sv, g, lpz * (sh * A)));
  acc_pair(gh, ch * F);
  acc_pair(ge, ce * F);
  const float Z = A * fmaf(k4, g, -k2);
  lu = fmaf(G * cu, lqu, fmaf(-Sp * su, lpz, lu));
  lv = fmaf(G * cv, lqv, fmaf(-Sp * sv, lpz, lv));
  lz = fmaf(-2.0f * Sp, fmaf(su, lqu, sv * lqv), fmaf(Z, lpz, lz));
  add_comp(t.qu, -(G * su));
  add_comp(t.qv, -(G * sv));
  add_comp(t.pz, -(Sp * A));
}

template <int M>
__global__ void __launch_bounds__(256) k_adjoint_fp32c(AdjArgs a, Tab32 tb) {
  extern __shared__ __align__(16) unsigned char smem[];
  float2* ssc = reinterpret_cast<float2*>(smem);
  for (int k = threadIdx.x; k <= tb.jmax; k += blockDim.x) ssc[k] = a.scf[k];
  __syncthreads();
  const long long n = a.n;
  const float* ck = a.ck32 + (long long)a.k * 12 * n;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    Traj32 t;
    t.u = {ck[i], ck[6 * n + i]};
    t.v = {ck[n + i], ck[7 * n + i]};
    t.z = {ck[2 * n + i], ck[8 * n + i]};
    t.qu = {ck[3 * n + i], ck[9 * n + i]};
    t.qv = {ck[4 * n + i], ck[10 * n + i]};
    t.pz = {ck[5 * n + i], ck[11 * n + i]};
    t.lu = t.lv = t.lz = 0;
    // pass 1: the state after every step of the segment
#pragma unroll 1
    for (int s = 0; s < a.steps; ++s) {
      drift32<false, true>(t, a.cf.sig_hi[0], a.cf.sig_lo[0]);
#pragma unroll
      for (int k = 0; k < M; ++k) {
        kick32<false>(t, a.cf.k2f[k], ssc, tb);
        drift32<false, true>(t, a.cf.sig_hi[k + 1], a.cf.sig_lo[k + 1]);
      }
      end_step32<false>(t, tb);
      float* sg = a.seg32 + (long long)s * 12 * n;
      sg[i] = t.u.hi; sg[n + i] = t.v.hi; sg[2 * n + i] = t.z.hi;
      sg[3 * n + i] = t.qu.hi; sg[4 * n + i] = t.qv.hi; sg[5 * n + i] = t.pz.hi;
      sg[6 * n + i] = t.u.lo; sg[7 * n + i] = t.v.lo; sg[8 * n + i] = t.z.lo;
      sg[9 * n + i] = t.qu.lo; sg[10 * n + i] = t.qv.lo; sg[11 * n + i] = t.pz.lo;
    }
    float lu = a.lamf[i], lv = a.lamf[n + i], lz = a.lamf[2 * n + i];
    float lqu = a.lamf[3 * n + i], lqv = a.lamf[4 * n + i], lpz = a.lamf[5 * n + i];
    Pair gh = {0.0f, 0.0f}, ge = {0.0f, 0.0f};
#pragma unroll 1
    for (int s = a.steps - 1; s >= 0; --s) {
      const float* sg = a.seg32 + (long long)s * 12 * n;
      t.u = {sg[i], sg[6 * n + i]};
      t.v = {sg[n + i], sg[7 * n + i]};
      t.z = {sg[2 * n + i], sg[8 * n + i]};
      t.qu = {sg[3 * n + i], sg[9 * n + i]};
      t.qv = {sg[4 * n + i], sg[10 * n + i]};
      t.pz = {sg[5 * n + i], sg[11 * n + i]};
#pragma unroll
      for (int k = M; k >= 0; --k) {
        acc_pair(gh, a.cdf[k] * fmaf(lu, t.qu.hi, fmaf(lv, t.qv.hi, lz * t.pz.hi)));
        lqu = fmaf(a.cf.sig_hi[k], lu, lqu);
        lqv = fmaf(a.cf.sig_hi[k], lv, lqv);
        lpz = fmaf(a.cf.sig_hi[k], lz, lpz);
        drift32<false, true>(t, -a.cf.sig_hi[k], -a.cf.sig_lo[k]);
        if (k > 0)
          adj_kick32(lu, lv, lz, lqu, lqv, lpz, t, a.cf.k2f[k - 1], a.cf.k4f[k - 1], a.chf[k - 1], a.cef[k - 1], gh,
                     ge, ssc, tb);
      }
    }
    a.lamf[i] = lu; a.lamf[n + i] = lv; a.lamf[2 * n + i] = lz;
    a.lamf[3 * n + i] = lqu; a.lamf[4 * n + i] = lqv; a.lamf[5 * n + i] = lpz;
    a.gh[i] += (double)gh.hi + (double)gh.lo;
    a.ge[i] += (double)ge.hi + (double)ge.lo;
  }
}

// Upstream dL/d(x, y, z, px, py, pz) -> rotated-coordinate adjoint; zero the
// parameter accumulators.  (u = x + y, v = x - y: dL/du = (dL/dx + dL/dy)/2.)
__global__ void k_adj_init(long long n, const double* dx, const double* dp, double* lam, float* lamf, double* gh,
                           double* ge) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const double ax = dx ? dx[i] : 0.0, ay = dx ? dx[n + i] : 0.0, az = dx ? dx[2 * n + i] : 0.0;
    const double bx = dp ? dp[i] : 0.0, by = dp ? dp[n + i] : 0.0, bz = dp ? dp[2 * n + i] : 0.0;
    const double l6[6] = {0.5 * (ax + ay), 0.5 * (ax - ay), az, 0.5 * (bx + by), 0.5 * (bx - by), bz};
    for (int c = 0; c < 6; ++c) {
      if (lam) lam[c * n + i] = l6[c];
      if (lamf) lamf[c * n + i] = (float)l6[c];
    }
    gh[i] = 0.0;
    ge[i] = 0.0;
  }
}

// Rotated-coordinate adjoint -> dL/d(x0, y0, z0) and dL/d(px0, py0, pz0).
__global__ void k_adj_finish(long long n, const double* lam, const float* lamf, double* gx, double* gp) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double l[6];
    for (int c = 0; c < 6; ++c) l[c] = lam ? lam[c * n + i] : (double)lamf[c * n + i];
    gx[i] = l[0] + l[1];
    gx[n + i] = l[0] - l[1];
    gx[2 * n + i] = l[2];
    gp[i] = l[3] + l[4];
    gp[n + i] = l[3] - l[4];
    gp[2 * n + i] = l[5];
  }
}

// Deterministic sum of two arrays: per-block fixed-tree partial sums, then one
// block sums the partials in order.
__global__ void k_sum2_partial(long long n, const double* a, const double* b, double* part) {
  __shared__ double sa[256], sb[256];
  double x = 0.0, y = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    x += a[i];
    y += b[i];
  }
  sa[threadIdx.x] = x;
  sb[threadIdx.x] = y;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sa[threadIdx.x] += sa[threadIdx.x + s];
      sb[threadIdx.x] += sb[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = sa[0];
    part[2 * blockIdx.x + 1] = sb[0];
  }
}

__global__ void k_sum2_final(int np, const double* part, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double x = 0.0, y = 0.0;
    for (int b = 0; b < np; ++b) {
      x += part[2 * b];
      y += part[2 * b + 1];
    }
    out[0] = x;
    out[1] = y;
  }
}

template <int M>
cudaError_t launch64(const AdjArgs& a, int grid, cudaStream_t st) {
  auto k = k_adjoint_fp64<M>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTabSmemBytes);
  if (e != cudaSuccess) return e;
  k<<<grid, 256, kTabSmemBytes, st>>>(a);
  return cudaGetLastError();
}

template <int M>
int occ64() {
  auto k = k_adjoint_fp64<M>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTabSmemBytes) != cudaSuccess) return 1;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, 256, kTabSmemBytes) != cudaSuccess) return 1;
  return nb > 0 ? nb : 1;
}

template <int M>
cudaError_t launch32(const AdjArgs& a, const Tab32& tb, int grid, cudaStream_t st) {
  k_adjoint_fp32c<M><<<grid, 256, (size_t)(tb.jmax + 1) * sizeof(float2), st>>>(a, tb);
  return cudaGetLastError();
}

template <int M>
int occ32(size_t smem) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_adjoint_fp32c<M>, 256, smem) != cudaSuccess) return 1;
  return nb > 0 ? nb : 1;
}

}  // namespace

void fp32_tab(Tab32* tb);

cudaError_t launch_adjoint_segment(const AdjArgs& a, int scheme, bool fp32c, int grid, cudaStream_t st) {
  if (fp32c) {
    Tab32 tb;
    fp32_tab(&tb);
    switch (scheme) {
      case ARNOLD_SCHEME_YOSHIDA6A: return launch32<7>(a, tb, grid, st);
      case ARNOLD_SCHEME_TRIPLEJUMP6: return launch32<9>(a, tb, grid, st);
      case ARNOLD_SCHEME_LEAPFROG2: return launch32<1>(a, tb, grid, st);
    }
  } else {
    switch (scheme) {
      case ARNOLD_SCHEME_YOSHIDA6A: return launch64<7>(a, grid, st);
      case ARNOLD_SCHEME_TRIPLEJUMP6: return launch64<9>(a, grid, st);
      case ARNOLD_SCHEME_LEAPFROG2: return launch64<1>(a, grid, st);
    }
  }
  return cudaErrorInvalidValue;
}

int adjoint_blocks_per_sm(int scheme, bool fp32c) {
  if (fp32c) {
    Tab32 tb;
    fp32_tab(&tb);
    const size_t smem = (size_t)(tb.jmax + 1) * sizeof(float2);
    return scheme == ARNOLD_SCHEME_YOSHIDA6A ? occ32<7>(smem)
                                             : (scheme == ARNOLD_SCHEME_TRIPLEJUMP6 ? occ32<9>(smem) : occ32<1>(smem));
  }
  return scheme == ARNOLD_SCHEME_YOSHIDA6A ? occ64<7>() : (scheme == ARNOLD_SCHEME_TRIPLEJUMP6 ? occ64<9>() : occ64<1>());
}

cudaError_t launch_adj_init(long long n, const double* dx, const double* dp, double* lam, float* lamf, double* gh,
                            double* ge, int grid, cudaStream_t st) {
  k_adj_init<<<grid, 256, 0, st>>>(n, dx, dp, lam, lamf, gh, ge);
  return cudaGetLastError();
}

cudaError_t launch_adj_finish(long long n, const double* lam, const float* lamf, double* gx, double* gp, int grid,
                              cudaStream_t st) {
  k_adj_finish<<<grid, 256, 0, st>>>(n, lam, lamf, gx, gp);
  return cudaGetLastError();
}

cudaError_t launch_sum2(long long n, const double* a, const double* b, double* part, int grid, double* out,
                        cudaStream_t st) {
  k_sum2_partial<<<grid, 256, 0, st>>>(n, a, b, part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sum2_final<<<1, 32, 0, st>>>(grid, part, out);
  return cudaGetLastError();
}

}  // namespace arnold
