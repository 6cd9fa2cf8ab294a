// Argument blocks and launchers of the set-up, read-out and statistics kernels.
#pragma once
#include "arnold_internal.cuh"
#include "step32.cuh"

namespace arnold {

struct InitArgs {
  Fp64State s;          // st / tg may be null (FP32C context: f used instead)
  Fp32cState f;         // hi/lo/tg null for FP64 contexts
  const double* x_in;   // [3][n] (set_state)
  const double* p_in;   // [3][n]
  const double* w_in;   // [6][n] or null
  double* raw_out;      // [6][n] or null: generated x, y, z, p_x, p_y, p_z (init_grid)
  const double2* sc;
  const double* th;
  long long n;
  long long G, row0;    // init_grid
  double E, eps, half_width;
  unsigned long long seed;
  int tangent;
  int shell_mode;       // set_state: 0 P given, 1 P = |P| p (unit direction), 2 p_z from the energy
  int window_turns;     // FP32C: whole turns added to each angle pair (into its window), laps debited
  Tab32 tab32;          // FP32C: the 2 pi split used for those turns
  int* flags;
};

struct ReadArgs {
  Fp64State s;
  Fp32cState f;
  const double2* sc;
  const double* th;
  long long n;
  long long W;
  int kind;
  int fp32c;
  double t;             // steps * h
  double eps;
  double threshold;     // chaos threshold kappa ln(max(t, e)) / t
  long long m;          // renormalisations so far (steps / R): the MEGNO sample index
  void* out;
};

struct StatsPartial {   // one per block, merged in block order
  unsigned long long hist[ARNOLD_HIST_BINS];
  unsigned long long under, over, chaotic, n;
  double dE_max;
  double mean[3], m2[3];
};

// One segment of the reverse sweep (adjoint.cu).
struct AdjArgs {
  const double* ck64;   // [K][6][n] FP64 checkpoints (rotated coordinates)
  double* seg64;        // [C][6][n] step-start states of the current segment
  const float* ck32;    // [K][12][n] FP32C checkpoints (6 hi, then 6 lo)
  float* seg32;         // [C][12][n]
  double* lam;          // [6][n] adjoint (FP64 path)
  float* lamf;          // [6][n] adjoint (FP32C path)
  double* gh;           // [n] per-trajectory dL/dh
  double* ge;           // [n] per-trajectory dL/deps
  const double2* sc;
  const double* th;
  const float2* scf;
  long long n;
  int k;                // segment index
  int steps;            // steps in the segment
  StepCoef cf;
  double ch[9], ce[9];  // per kick: 2 w_k eps, 2 w_k h
  double cd[10];        // per drift: sigma_k / h
  float chf[9], cef[9], cdf[10];
};

cudaError_t launch_adjoint_segment(const AdjArgs& a, int scheme, bool fp32c, int grid, cudaStream_t st);
int adjoint_blocks_per_sm(int scheme, bool fp32c);   // with 256-thread blocks
cudaError_t launch_adj_init(long long n, const double* dx, const double* dp, double* lam, float* lamf, double* gh,
                            double* ge, int grid, cudaStream_t st);
cudaError_t launch_adj_finish(long long n, const double* lam, const float* lamf, double* gx, double* gp, int grid,
                              cudaStream_t st);
cudaError_t launch_sum2(long long n, const double* a, const double* b, double* part, int grid, double* out,
                        cudaStream_t st);

cudaError_t launch_set_state(const InitArgs& a, int grid, int block, cudaStream_t st);
cudaError_t launch_vhist(long long n, const double* V, const unsigned char* left, int filtered, const double* patch4,
                         int n_cos, int n_phi, unsigned long long* counts, int grid, cudaStream_t st);
cudaError_t launch_init_grid(const InitArgs& a, int grid, int block, cudaStream_t st);
cudaError_t launch_init_sphere(const InitArgs& a, unsigned long long offset, const double* patch4, int grid,
                               cudaStream_t st);
// One chunk of 256 * nb Gaussian candidates from t0: count, prefix, place.
cudaError_t launch_gauss_chunk(const InitArgs& a, unsigned long long t0, int nb, double cx, double cy, double sigma,
                               int* counts, long long* offs, long long* have, unsigned long long* drawn,
                               cudaStream_t st);
cudaError_t launch_indicator(const ReadArgs& a, int grid, int block, cudaStream_t st);
cudaError_t launch_debug_sincos64(const double* x, double* s, double* c, long long n, const double2* sc,
                                  const double* th, cudaStream_t st);
cudaError_t launch_debug_sincos_df(const double* x, double* s, double* c, long long n, const float4* scd, bool fast,
                                   cudaStream_t st);
cudaError_t launch_debug_sincos32(const double* x, double* s, double* c, long long n, const float2* scf,
                                  cudaStream_t st);
cudaError_t launch_stats(long long n, const double* chi, const double* dE, const double* p, double threshold,
                         StatsPartial* partials, int grid, StatsPartial* out, cudaStream_t st);
cudaError_t launch_probe(int kind, int grid, int block, int iters, double* sink, cudaStream_t st);

}  // namespace arnold
