// Argument blocks and launchers of the set-up, read-out and statistics kernels.
#pragma once
#include "arnold_internal.cuh"

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
  void* out;
};

struct StatsPartial {   // one per block, merged in block order
  unsigned long long hist[ARNOLD_HIST_BINS];
  unsigned long long under, over, chaotic, n;
  double dE_max;
  double mean[3], m2[3];
};

cudaError_t launch_set_state(const InitArgs& a, int grid, int block, cudaStream_t st);
cudaError_t launch_init_grid(const InitArgs& a, int grid, int block, cudaStream_t st);
cudaError_t launch_indicator(const ReadArgs& a, int grid, int block, cudaStream_t st);
cudaError_t launch_debug_sincos64(const double* x, double* s, double* c, long long n, const double2* sc,
                                  const double* th, cudaStream_t st);
cudaError_t launch_debug_sincos32(const double* x, double* s, double* c, long long n, const float2* scf,
                                  cudaStream_t st);
cudaError_t launch_stats(long long n, const double* chi, const double* dE, const double* p, double threshold,
                         StatsPartial* partials, int grid, StatsPartial* out, cudaStream_t st);
cudaError_t launch_probe(int kind, int grid, int block, int iters, double* sink, cudaStream_t st);

}  // namespace arnold
