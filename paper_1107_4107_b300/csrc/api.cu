// C-ABI layer of libarnold (declared in include/arnold.h): contexts, device
// memory, sincos tables, launch planning, read-out and host fault injection.
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include "kernels.cuh"
#include "run32.cuh"
#include "step_df.cuh"

namespace arnold {
cudaError_t launch_iterate_fp32c_v(const IterArgs& a, int scheme, bool tangent, bool reduce64, int block, int grid,
                                   cudaStream_t st);

// x rounded to `bits` significant bits.
static long double round_bits(long double x, int bits) {
  int e;
  const long double m = frexpl(x, &e);
  return ldexpl(roundl(ldexpl(m, bits)), e - bits);
}

// FP32 table geometry (see Tab32 in step32.cuh): D = 2 pi / 2048 split into
// d1 (4 significant bits, so j d1 is exact for j < 2^20: angles below 3217
// rad) + d2 + d3; 2 pi split into c1 (14 bits) + c2 (16 bits) + c3, so k c1
// and k c2 are exact for |k| < 256 turns.
// DF64 table geometry (TabDF in step_df.cuh): D = 2 pi / 2048 split d1 (11
// significant bits) + d2 + d3; 2 pi split into c1 and c2 of 18 significant
// bits each + c3, so k c1 and k c2 are exact for |k| < 64 turns.
void df_tab(TabDF* tb) {
  const long double two_pi = 6.283185307179586476925286766559005768L;
  const long double D = two_pi / 2048.0L;
  const long double d1 = round_bits(D, 11);
  const float d2 = (float)(D - d1);
  const float d3 = (float)(D - d1 - (long double)d2);
  tb->inv_d = (float)(1.0L / D);
  tb->d1 = (float)d1;
  tb->d2 = d2;
  tb->d3 = d3;
  tb->mask = 2047;
  tb->inv2pi = (float)(1.0L / two_pi);
  const long double c1 = round_bits(two_pi, 18);
  const long double c2 = round_bits(two_pi - c1, 18);
  tb->c1 = (float)c1;
  tb->c2 = (float)c2;
  tb->c3 = (float)(two_pi - c1 - c2);
}

void fp32_tab(Tab32* tb) {
  const long double two_pi = 6.283185307179586476925286766559005768L;
  const long double D = two_pi / 2048.0L;
  const long double d1 = round_bits(D, 4);
  const float d2 = (float)(D - d1);
  const float d3 = (float)(D - d1 - (long double)d2);
  tb->inv_d = (float)(1.0L / D);
  tb->d1 = (float)d1;
  tb->d2 = d2;
  tb->d3 = d3;
  tb->jmax = 2047;
  tb->inv2pi = (float)(1.0L / two_pi);
  const long double c1 = round_bits(two_pi, 14);
  const long double c2 = round_bits(two_pi - c1, 16);
  tb->c1 = (float)c1;
  tb->c2 = (float)c2;
  tb->c3 = (float)(two_pi - c1 - c2);
}
}  // namespace arnold

using namespace arnold;

struct arnold_ctx {
  arnold_params prm;
  long long n = 0;
  int device = 0;
  cudaStream_t stream = nullptr;
  long long steps = 0;
  int sms = 148;
  long long launches = 0;
  Fp64State s{};
  Fp32cState f{};
  double2* sc = nullptr;   // FP64 sincos table
  double* th = nullptr;
  float2* scf = nullptr;   // FP32 sincos table
  float4* scd = nullptr;   // DF64 sincos table
  int* flags = nullptr;    // device error flags
  StatsPartial* partials = nullptr;
  StatsPartial* stats_out = nullptr;
  int stats_grid = 0;
  double* scratch = nullptr;   // [6][n] f64 read-out scratch (lazy)
  double* scratch2 = nullptr;  // [5][n] f64 statistics inputs (lazy)
  int reduce64 = 0;            // FP32C variant: FP64 mod-2pi reduction
  // adjoint (forward_ckpt / grad)
  void* ck = nullptr;          // [K][6][n] f64 or [K][12][n] f32
  void* seg = nullptr;         // [C][...][n]
  size_t ck_bytes = 0, seg_bytes = 0;
  double* lam = nullptr;       // [6][n]
  float* lamf = nullptr;       // [6][n]
  double* gh = nullptr;        // [n]
  double* ge = nullptr;        // [n]
  double* sum_part = nullptr;  // [2 * stats_grid + 2]
  int adj_valid = 0;
  long long adj_N = 0, adj_C = 0, adj_K = 0;
  unsigned long long* vhist = nullptr;   // device counts for host-side histograms
  size_t vhist_cells = 0;
  void* draw = nullptr;                  // Gaussian redraw scratch: block counts, offsets, kept, drawn (lazy)
};

namespace {

int fault_is(const char* what) {
  const char* f = getenv("ARNOLD_FAULT");
  return f && strcmp(f, what) == 0;
}

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return ARNOLD_OK;
  if (e == cudaErrorMemoryAllocation) return ARNOLD_ENOMEM;
  if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return ARNOLD_EUNSUPPORTED;
  return ARNOLD_ECUDA;
}

#define ACHECK(expr)                                   \
  do {                                                 \
    cudaError_t _e = (expr);                           \
    if (_e != cudaSuccess) return cuda_status(_e);     \
  } while (0)

static_assert(sizeof(arnold_params) == 64, "arnold_params layout is part of the ABI");

int params_ok(const arnold_params* p) {
  if (!p) return 0;
  if (!(p->h != 0.0) || !isfinite(p->h) || !isfinite(p->eps)) return 0;
  if (p->scheme < 0 || p->scheme > 2) return 0;
  if (p->precision < ARNOLD_FP64 || p->precision > ARNOLD_DF64F) return 0;
  if (p->tangent != 0 && p->tangent != 1) return 0;
  if (p->renorm_every < 1 || p->window < 0) return 0;
  if (!(p->chaos_kappa > 0.0)) return 0;
  if (p->block_size != 0 && (p->block_size < 32 || p->block_size > 256 || p->block_size % 32)) return 0;
  if (p->launch_steps < 0) return 0;
  if (p->megno != 0 && p->megno != 1) return 0;
  if (p->megno && !p->tangent) return 0;
  if (p->reserved != 0) return 0;
  return 1;
}

// Leapfrog weights of one composite step (Sec. III reading).
int scheme_weights(int scheme, double* w) {
  if (scheme == ARNOLD_SCHEME_YOSHIDA6A) {
    // Yoshida, Phys. Lett. A 150 (1990) 262, solution A.
    const double w1 = -1.17767998417887, w2 = 0.235573213359357, w3 = 0.784513610477560;
    const double w0 = 1.0 - 2.0 * (w1 + w2 + w3);
    const double seq[7] = {w3, w2, w1, w0, w1, w2, w3};
    for (int k = 0; k < 7; ++k) w[k] = seq[k];
    return 7;
  }
  if (scheme == ARNOLD_SCHEME_TRIPLEJUMP6) {
    const double g1 = 1.0 / (2.0 - cbrt(2.0)), g0 = 1.0 - 2.0 * g1;
    const double d1 = 1.0 / (2.0 - pow(2.0, 0.2)), d0 = 1.0 - 2.0 * d1;
    const double outer[3] = {d1, d0, d1}, inner[3] = {g1, g0, g1};
    int k = 0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) w[k++] = outer[a] * inner[b];
    return 9;
  }
  w[0] = 1.0;
  return 1;
}

StepCoef make_coef(const arnold_params& p) {
  StepCoef c;
  memset(&c, 0, sizeof c);
  double w[9];
  const int m = scheme_weights(p.scheme, w);
  c.m = m;
  for (int k = 0; k <= m; ++k) {
    const double left = k > 0 ? w[k - 1] : 0.0, right = k < m ? w[k] : 0.0;
    c.sig[k] = 0.5 * (left + right) * p.h;
    c.sig_hi[k] = (float)c.sig[k];
    c.sig_lo[k] = (float)(c.sig[k] - (double)c.sig_hi[k]);
  }
  for (int k = 0; k < m; ++k) {
    const double tau = w[k] * p.h;
    c.k2[k] = 2.0 * tau * p.eps;
    c.k4[k] = 4.0 * tau * p.eps;
    c.k2f[k] = (float)c.k2[k];
    c.k4f[k] = (float)c.k4[k];
  }
  return c;
}

int build_tables(arnold_ctx* c) {
  // FP64: theta_j = j D, D = 2pi/4096 with the low 14 mantissa bits cleared.
  const double D0 = kTwoPi / (double)kTabN;
  unsigned long long bits;
  memcpy(&bits, &D0, 8);
  bits &= ~((1ULL << 14) - 1ULL);
  double D;
  memcpy(&D, &bits, 8);
  double2* hsc = (double2*)malloc(sizeof(double2) * kTabEntries);
  double* hth = (double*)malloc(sizeof(double) * kTabEntries);
  if (!hsc || !hth) { free(hsc); free(hth); return ARNOLD_ENOMEM; }
  for (int j = 0; j < kTabEntries; ++j) {
    const double t = (double)j * D;   // exact
    hth[j] = t;
    hsc[j].x = (double)sinl((long double)t);
    hsc[j].y = (double)cosl((long double)t);
  }
  cudaError_t e = cudaMalloc(&c->sc, sizeof(double2) * kTabEntries);
  if (e == cudaSuccess) e = cudaMalloc(&c->th, sizeof(double) * kTabEntries);
  if (e == cudaSuccess) e = cudaMemcpy(c->sc, hsc, sizeof(double2) * kTabEntries, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(c->th, hth, sizeof(double) * kTabEntries, cudaMemcpyHostToDevice);
  free(hsc);
  free(hth);
  if (e != cudaSuccess) return cuda_status(e);
  // FP32 table: exactly periodic, (sin, cos)(2 pi j / 2048)
  Tab32 tb;
  fp32_tab(&tb);
  const int jmax = tb.jmax;
  float2* hf = (float2*)malloc(sizeof(float2) * (jmax + 1));
  if (!hf) return ARNOLD_ENOMEM;
  for (int j = 0; j <= jmax; ++j) {
    const long double t = (long double)j * (6.283185307179586476925286766559005768L / 2048.0L);
    hf[j].x = (float)sinl(t);
    hf[j].y = (float)cosl(t);
  }
  e = cudaMalloc(&c->scf, sizeof(float2) * (jmax + 1));
  if (e == cudaSuccess) e = cudaMemcpy(c->scf, hf, sizeof(float2) * (jmax + 1), cudaMemcpyHostToDevice);
  free(hf);
  if (e != cudaSuccess) return cuda_status(e);
  // DF64 table: (sin, cos)(2 pi j / 2048) as float pairs
  float4* hd = (float4*)malloc(sizeof(float4) * 2048);
  if (!hd) return ARNOLD_ENOMEM;
  for (int j = 0; j < 2048; ++j) {
    const long double t = (long double)j * (6.283185307179586476925286766559005768L / 2048.0L);
    const long double sv = sinl(t), cv = cosl(t);
    hd[j].x = (float)sv;
    hd[j].y = (float)(sv - (long double)hd[j].x);
    hd[j].z = (float)cv;
    hd[j].w = (float)(cv - (long double)hd[j].z);
  }
  e = cudaMalloc(&c->scd, sizeof(float4) * 2048);
  if (e == cudaSuccess) e = cudaMemcpy(c->scd, hd, sizeof(float4) * 2048, cudaMemcpyHostToDevice);
  free(hd);
  return cuda_status(e);
}

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, sizeof(T) * (count ? count : 1));
}

void free_all(arnold_ctx* c) {
  void* ptrs[] = {c->s.st, c->s.tg, c->s.lap, c->s.lapref, c->s.ref, c->s.logsum, c->s.demax, c->s.e0, c->s.V,
                  c->f.hi, c->f.lo, c->f.tg, c->sc, c->th, c->scf, c->scd, c->flags, c->partials, c->stats_out,
                  c->scratch, c->scratch2, c->ck, c->seg, c->lam, c->lamf, c->gh, c->ge, c->sum_part, c->s.left,
                  c->vhist, c->s.megno, c->f.tg_lo, c->draw, c->s.p0};
  for (void* p : ptrs)
    if (p) cudaFree(p);
}

int grid_for(const arnold_ctx* c, int block) {
  long long g = (c->n + block - 1) / block;
  long long cap = (long long)c->sms * 8;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

int check_flags(arnold_ctx* c) {
  int h = 0;
  ACHECK(cudaMemcpyAsync(&h, c->flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  ACHECK(cudaStreamSynchronize(c->stream));
  if (h & kFlagTimeout) return ARNOLD_ETIMEOUT;
  if (h & kFlagRange) return ARNOLD_ERANGE;
  if (h & kFlagNonFinite) return ARNOLD_ENONFINITE;
  return ARNOLD_OK;
}

InitArgs init_args(arnold_ctx* c) {
  InitArgs a;
  memset(&a, 0, sizeof a);
  a.s = c->s;
  a.f = c->f;
  a.sc = c->sc;
  a.th = c->th;
  a.n = c->n;
  a.eps = c->prm.eps;
  a.tangent = c->prm.tangent;
  a.flags = c->flags;
  if (c->prm.precision == ARNOLD_FP32C) {   // angles held in [kWinLo, kWinHi): 244 turns = 1533.1 rad
    a.window_turns = 244;
    fp32_tab(&a.tab32);
  }
  return a;
}

int device_scratch(arnold_ctx* c) {
  if (!c->scratch) ACHECK(dalloc(&c->scratch, 6 * (size_t)c->n));
  return ARNOLD_OK;
}

int read_indicator(arnold_ctx* c, int kind, void* dst) {
  ReadArgs r;
  memset(&r, 0, sizeof r);
  r.s = c->s;
  r.f = c->f;
  r.sc = c->sc;
  r.th = c->th;
  r.n = c->n;
  r.W = c->prm.window;
  r.kind = kind;
  r.fp32c = c->prm.precision != ARNOLD_FP64;   // pair state
  r.t = (double)c->steps * c->prm.h;
  r.eps = c->prm.eps;
  const double tt = fabs(r.t);
  r.threshold = c->prm.chaos_kappa * log(tt > M_E ? tt : M_E) / tt;
  r.m = c->steps / c->prm.renorm_every;
  r.out = dst;
  ACHECK(launch_indicator(r, grid_for(c, 256), 256, c->stream));
  c->launches++;
  return ARNOLD_OK;
}

size_t indicator_bytes(int kind, long long n) {
  switch (kind) {
    case ARNOLD_IND_CHI: case ARNOLD_IND_DE: case ARNOLD_IND_DE_MAX: case ARNOLD_IND_LOGSUM:
    case ARNOLD_IND_MEGNO: case ARNOLD_IND_MEGNO_Y: case ARNOLD_IND_VDEV: return 8 * (size_t)n;
    case ARNOLD_IND_CLASS: case ARNOLD_IND_LEFT: return (size_t)n;
    case ARNOLD_IND_V: case ARNOLD_IND_X: case ARNOLD_IND_P: case ARNOLD_IND_DX: return 24 * (size_t)n;
    case ARNOLD_IND_TANGENT: return 48 * (size_t)n;
  }
  return 0;
}

}  // namespace

namespace arnold {
// Accessors used by the batched launch (batch.cu).
int ctx_run_args(arnold_ctx* c, RunArgs32* ra, StepCoef* sc, const float2** scf, const float4** scd) {
  if (c->prm.precision == ARNOLD_FP64) return ARNOLD_EUNSUPPORTED;
  ra->s = c->s;
  ra->f = c->f;
  ra->n = c->n;
  ra->R = c->prm.renorm_every;
  ra->W = c->prm.window;
  ra->h = c->prm.h;
  ra->eps = c->prm.eps;
  ra->flags = c->flags;
  *sc = make_coef(c->prm);
  *scf = c->scf;
  *scd = c->scd;
  return ARNOLD_OK;
}
void ctx_add_steps(arnold_ctx* c, long long s) {
  c->steps += s;
  c->adj_valid = 0;
}
long long ctx_steps(arnold_ctx* c) { return c->steps; }
}  // namespace arnold

extern "C" {

void arnold_params_default(arnold_params* p) {
  if (!p) return;
  memset(p, 0, sizeof *p);
  p->eps = 1.0;
  p->h = 0.02 * 3.14159265358979323846;
  p->scheme = ARNOLD_SCHEME_YOSHIDA6A;
  p->precision = ARNOLD_FP64;
  p->tangent = 1;
  p->renorm_every = 100;
  p->window = 0;
  p->chaos_kappa = 10.0;
}

const char* arnold_strerror(int s) {
  switch (s) {
    case ARNOLD_OK: return "ok";
    case ARNOLD_EINVAL: return "invalid argument";
    case ARNOLD_ENOMEM: return "out of memory";
    case ARNOLD_ECUDA: return "CUDA error";
    case ARNOLD_ETIMEOUT: return "device wait timed out";
    case ARNOLD_ENONFINITE: return "non-finite state";
    case ARNOLD_EUNSUPPORTED: return "unsupported (no CUDA device or combination not built)";
    case ARNOLD_ESTATE: return "call out of order";
    case ARNOLD_ERANGE: return "parameters outside the range of the precision mode";
  }
  return "unknown status";
}

int arnold_create(const arnold_params* prm, int64_t n_traj, int device, void* cuda_stream, arnold_ctx** out) {
  if (out) *out = nullptr;
  if (!out || !params_ok(prm) || n_traj <= 0 || n_traj > (1LL << 40)) return ARNOLD_EINVAL;
  if (fault_is("alloc")) return ARNOLD_ENOMEM;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) return ARNOLD_EUNSUPPORTED;
  if (device < 0 || device >= ndev) return ARNOLD_EINVAL;
  ACHECK(cudaSetDevice(device));
  arnold_ctx* c = new (std::nothrow) arnold_ctx();
  if (!c) return ARNOLD_ENOMEM;
  c->prm = *prm;
  c->n = n_traj;
  c->device = device;
  c->stream = (cudaStream_t)cuda_stream;
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
  const size_t n = (size_t)n_traj;
  const int tan = prm->tangent;
  cudaError_t e = cudaSuccess;
  if (prm->precision == ARNOLD_FP64) {   // FP32C and DF64 keep float pairs
    e = dalloc(&c->s.st, 6 * n);
    if (e == cudaSuccess && tan) e = dalloc(&c->s.tg, 6 * n);
  } else {
    e = dalloc(&c->f.hi, 6 * n);
    if (e == cudaSuccess) e = dalloc(&c->f.lo, 6 * n);
    if (e == cudaSuccess && tan) e = dalloc(&c->f.tg, 6 * n);
    if (e == cudaSuccess && tan && (prm->precision == ARNOLD_DF64 || prm->precision == ARNOLD_DF64F))
      e = dalloc(&c->f.tg_lo, 6 * n);
  }
  if (e == cudaSuccess) e = dalloc(&c->s.lap, 3 * n);
  if (e == cudaSuccess) e = dalloc(&c->s.lapref, 3 * n);
  if (e == cudaSuccess) e = dalloc(&c->s.ref, 3 * n);
  if (e == cudaSuccess && tan) e = dalloc(&c->s.logsum, n);
  if (e == cudaSuccess && prm->megno) e = dalloc(&c->s.megno, 2 * n);
  if (e == cudaSuccess) e = dalloc(&c->s.demax, n);
  if (e == cudaSuccess) e = dalloc(&c->s.e0, n);
  if (e == cudaSuccess) e = dalloc(&c->s.V, 3 * n);
  if (e == cudaSuccess) e = dalloc(&c->s.p0, 3 * n);
  if (e == cudaSuccess) e = dalloc(&c->flags, 1);
  if (e == cudaSuccess) e = cudaMemset(c->flags, 0, sizeof(int));
  c->stats_grid = c->sms * 4;
  if (e == cudaSuccess) e = dalloc(&c->partials, (size_t)c->stats_grid);
  if (e == cudaSuccess) e = dalloc(&c->stats_out, 1);
  int st = cuda_status(e);
  if (st == ARNOLD_OK) st = build_tables(c);
  if (st != ARNOLD_OK) {
    free_all(c);
    delete c;
    cudaGetLastError();
    return st;
  }
  const char* r64 = getenv("ARNOLD_FP32C_REDUCE64");
  c->reduce64 = r64 && r64[0] == '1';
  *out = c;
  return ARNOLD_OK;
}

void arnold_destroy(arnold_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  free_all(c);
  delete c;
}

static int set_state_mode(arnold_ctx* c, const double* x, const double* p, const double* w, int ptr_kind, int mode,
                          double E) {
  if (!c || !x || !p || (ptr_kind != ARNOLD_HOST && ptr_kind != ARNOLD_DEVICE)) return ARNOLD_EINVAL;
  ACHECK(cudaSetDevice(c->device));
  InitArgs a = init_args(c);
  a.shell_mode = mode;
  a.E = E;
  const size_t n = (size_t)c->n;
  if (ptr_kind == ARNOLD_HOST) {
    int st = device_scratch(c);
    if (st) return st;
    double* d = c->scratch;    // x [3][n], p [3][n]
    ACHECK(cudaMemcpyAsync(d, x, 24 * n, cudaMemcpyHostToDevice, c->stream));
    ACHECK(cudaMemcpyAsync(d + 3 * n, p, 24 * n, cudaMemcpyHostToDevice, c->stream));
    a.x_in = d;
    a.p_in = d + 3 * n;
    double* dw = nullptr;
    if (w && c->prm.tangent) {
      if (!c->scratch2) ACHECK(dalloc(&c->scratch2, 6 * n));
      dw = c->scratch2;
      ACHECK(cudaMemcpyAsync(dw, w, 48 * n, cudaMemcpyHostToDevice, c->stream));
    }
    a.w_in = dw;
  } else {
    a.x_in = x;
    a.p_in = p;
    a.w_in = c->prm.tangent ? w : nullptr;
  }
  ACHECK(cudaMemsetAsync(c->flags, 0, sizeof(int), c->stream));
  c->adj_valid = 0;
  ACHECK(launch_set_state(a, grid_for(c, 256), 256, c->stream));
  c->launches++;
  c->steps = 0;
  if (ptr_kind == ARNOLD_HOST) ACHECK(cudaStreamSynchronize(c->stream));   // host buffers may be freed on return
  return ARNOLD_OK;
}

int arnold_set_state(arnold_ctx* c, const double* x, const double* p, const double* w, int ptr_kind) {
  return set_state_mode(c, x, p, w, ptr_kind, 0, 0.0);
}

int arnold_set_state_shell(arnold_ctx* c, const double* x, const double* p, int mode, double E, int ptr_kind) {
  if (mode != ARNOLD_SHELL_DIRECTION && mode != ARNOLD_SHELL_PZ) return ARNOLD_EINVAL;
  if (!isfinite(E)) return ARNOLD_EINVAL;
  return set_state_mode(c, x, p, nullptr, ptr_kind, mode, E);
}

int arnold_track_patch(arnold_ctx* c, double cos_lo, double cos_hi, double phi_lo, double phi_hi) {
  if (!c || !(cos_lo <= cos_hi) || !(phi_lo <= phi_hi) || !isfinite(cos_lo + cos_hi + phi_lo + phi_hi))
    return ARNOLD_EINVAL;
  ACHECK(cudaSetDevice(c->device));
  if (!c->s.left) ACHECK(dalloc(&c->s.left, (size_t)c->n));
  ACHECK(cudaMemsetAsync(c->s.left, 0, (size_t)c->n, c->stream));
  c->s.patch[0] = cos_lo;
  c->s.patch[1] = cos_hi;
  c->s.patch[2] = phi_lo;
  c->s.patch[3] = phi_hi;
  return ARNOLD_OK;
}

int arnold_velocity_histogram(arnold_ctx* c, int n_cos, int n_phi, double cos_lo, double cos_hi, double phi_lo,
                              double phi_hi, int filtered, uint64_t* counts, int ptr_kind, int accumulate) {
  if (!c || !counts || n_cos <= 0 || n_phi <= 0 || (long long)n_cos * n_phi > (1LL << 28) || !(cos_lo < cos_hi) ||
      !(phi_lo < phi_hi) || (ptr_kind != ARNOLD_HOST && ptr_kind != ARNOLD_DEVICE) || c->steps == 0)
    return ARNOLD_EINVAL;
  ACHECK(cudaSetDevice(c->device));
  const size_t cells = (size_t)n_cos * n_phi;
  int st = device_scratch(c);
  if (st) return st;
  st = read_indicator(c, ARNOLD_IND_V, c->scratch);
  if (st) return st;
  unsigned long long* d = (unsigned long long*)counts;
  if (ptr_kind == ARNOLD_HOST) {
    if (c->vhist_cells < cells) {
      if (c->vhist) cudaFree(c->vhist);
      c->vhist = nullptr;
      c->vhist_cells = 0;
      ACHECK(dalloc(&c->vhist, cells));
      c->vhist_cells = cells;
    }
    d = c->vhist;
    if (accumulate) ACHECK(cudaMemcpyAsync(d, counts, cells * 8, cudaMemcpyHostToDevice, c->stream));
  }
  if (!accumulate) ACHECK(cudaMemsetAsync(d, 0, cells * 8, c->stream));
  const double p4[4] = {cos_lo, cos_hi, phi_lo, phi_hi};
  ACHECK(launch_vhist(c->n, c->scratch, c->s.left, filtered, p4, n_cos, n_phi, d, grid_for(c, 256), c->stream));
  c->launches++;
  if (ptr_kind == ARNOLD_HOST) {
    ACHECK(cudaMemcpyAsync(counts, d, cells * 8, cudaMemcpyDeviceToHost, c->stream));
    return check_flags(c);
  }
  return ARNOLD_OK;
}

int arnold_init_grid(arnold_ctx* c, int64_t G, int64_t row0, double E, uint64_t seed, double* raw_out) {
  if (!c || G <= 0 || row0 < 0 || c->n % G != 0) return ARNOLD_EINVAL;
  const int64_t rows = c->n / G;
  if (rows < 1 || row0 + rows > G) return ARNOLD_EINVAL;
  if (!(E > 2.0 * fabs(c->prm.eps))) return ARNOLD_EINVAL;
  ACHECK(cudaSetDevice(c->device));
  InitArgs a = init_args(c);
  a.G = G;
  a.row0 = row0;
  a.E = E;
  a.seed = seed;
  a.half_width = 0.9 * sqrt(E - 2.0 * fabs(c->prm.eps));
  a.raw_out = raw_out;
  ACHECK(cudaMemsetAsync(c->flags, 0, sizeof(int), c->stream));
  c->adj_valid = 0;
  ACHECK(launch_init_grid(a, grid_for(c, 256), 256, c->stream));
  c->launches++;
  c->steps = 0;
  return ARNOLD_OK;
}

int arnold_init_sphere(arnold_ctx* c, double E, uint64_t seed, int64_t offset, double cos_lo, double cos_hi,
                       double phi_lo, double phi_hi) {
  if (!c || offset < 0 || !isfinite(E) || !(E > 2.0 * fabs(c->prm.eps))) return ARNOLD_EINVAL;
  if (!(cos_lo >= -1.0 && cos_lo <= cos_hi && cos_hi <= 1.0) || !(phi_lo <= phi_hi) || !isfinite(phi_lo + phi_hi))
    return ARNOLD_EINVAL;
  ACHECK(cudaSetDevice(c->device));
  InitArgs a = init_args(c);
  a.E = E;
  a.seed = seed;
  a.shell_mode = 1;
  ACHECK(cudaMemsetAsync(c->flags, 0, sizeof(int), c->stream));
  c->adj_valid = 0;
  const double p4[4] = {cos_lo, cos_hi, phi_lo, phi_hi};
  ACHECK(launch_init_sphere(a, (unsigned long long)offset, p4, grid_for(c, 256), c->stream));
  c->launches++;
  c->steps = 0;
  return ARNOLD_OK;
}

int arnold_init_gaussian(arnold_ctx* c, double E, double px0, double py0, double sigma, uint64_t seed,
                         int64_t offset, int64_t* n_drawn) {
  if (!c || offset < 0 || !isfinite(E) || !isfinite(px0) || !isfinite(py0) || !(sigma >= 0.0) || !isfinite(sigma))
    return ARNOLD_EINVAL;
  ACHECK(cudaSetDevice(c->device));
  const int kMaxBlocks = 65536;   // candidates per chunk: 256 per block
  const size_t bytes = (size_t)kMaxBlocks * (sizeof(int) + sizeof(long long)) + 2 * sizeof(long long);
  if (!c->draw) ACHECK(cudaMalloc(&c->draw, bytes));
  int* counts = (int*)c->draw;
  long long* offs = (long long*)(counts + kMaxBlocks);
  long long* have_d = offs + kMaxBlocks;
  unsigned long long* drawn_d = (unsigned long long*)(have_d + 1);
  ACHECK(cudaMemsetAsync(have_d, 0, 2 * sizeof(long long), c->stream));
  ACHECK(cudaMemsetAsync(c->flags, 0, sizeof(int), c->stream));
  c->adj_valid = 0;
  InitArgs a = init_args(c);
  a.E = E;
  a.seed = seed;
  a.shell_mode = 2;
  unsigned long long t0 = (unsigned long long)offset;
  long long kept = 0;
  // give up when almost no draw has a real p_z (the cloud lies outside the shell)
  const unsigned long long limit = 64ULL * (unsigned long long)c->n + (1ULL << 24);
  long long nb = 0;
  while (kept < c->n) {
    if (t0 - (unsigned long long)offset > limit) return ARNOLD_ERANGE;
    // twice the candidates still needed, and at least twice the last chunk (few
    // real p_z: the chunks grow geometrically to the 2^24-candidate cap)
    const long long need = (2 * (c->n - kept) + 255) / 256;
    nb = need > 2 * nb ? need : 2 * nb;
    nb = nb < 4 ? 4 : (nb > kMaxBlocks ? kMaxBlocks : nb);
    ACHECK(launch_gauss_chunk(a, t0, (int)nb, px0, py0, sigma, counts, offs, have_d, drawn_d, c->stream));
    c->launches += 3;
    ACHECK(cudaMemcpyAsync(&kept, have_d, sizeof kept, cudaMemcpyDeviceToHost, c->stream));
    ACHECK(cudaStreamSynchronize(c->stream));
    t0 += (unsigned long long)nb * 256ULL;
  }
  unsigned long long drawn = 0;
  ACHECK(cudaMemcpyAsync(&drawn, drawn_d, sizeof drawn, cudaMemcpyDeviceToHost, c->stream));
  ACHECK(cudaStreamSynchronize(c->stream));
  if (n_drawn) *n_drawn = (int64_t)(drawn - (unsigned long long)offset);
  c->steps = 0;
  return ARNOLD_OK;
}

int arnold_iterate(arnold_ctx* c, int64_t n_steps) {
  if (!c || n_steps < 0) return ARNOLD_EINVAL;
  c->adj_valid = 0;
  if (fault_is("launch")) return ARNOLD_ECUDA;
  if (n_steps == 0) return ARNOLD_OK;
  ACHECK(cudaSetDevice(c->device));
  const arnold_params& p = c->prm;
  const bool fp32c = p.precision == ARNOLD_FP32C;
  const bool df64 = p.precision == ARNOLD_DF64 || p.precision == ARNOLD_DF64F;
  const bool fast = p.precision == ARNOLD_DF64F;
  int block = p.block_size;
  if (block == 0) {
    block = 256;
    const long long per_sm = (c->n + c->sms - 1) / c->sms;
    if (per_sm < 256) block = (int)((per_sm + 31) / 32 * 32);
    if (block < 32) block = 32;
  }
  const int bps = fp32c  ? fp32c_blocks_per_sm(p.scheme, p.tangent, block)
                  : df64 ? df64_blocks_per_sm(p.scheme, p.tangent, fast, block)
                         : fp64_blocks_per_sm(p.scheme, p.tangent, block);
  long long grid = (c->n + block - 1) / block;
  const long long cap = (long long)c->sms * bps;
  if (grid > cap) grid = cap;
  long long chunk = p.launch_steps;
  if (chunk == 0) {
    // aim at ~0.2 s per launch from the measured rates (map-steps/s, 7 kicks)
    const double rate = (fp32c ? 3.0e10 : (fast ? 1.2e10 : (df64 ? 8.0e9 : 1.0e9))) * 7.0 / (double)make_coef(p).m;
    chunk = (long long)(0.2 * rate / (double)c->n);
    if (chunk < 1) chunk = 1;
    if (chunk > (1 << 20)) chunk = 1 << 20;
  }
  IterArgs a;
  memset(&a, 0, sizeof a);
  a.s = c->s;
  a.f = c->f;
  a.sc = c->sc;
  a.th = c->th;
  a.scf = c->scf;
  a.scd = c->scd;
  a.n = c->n;
  a.R = p.renorm_every;
  a.W = p.window;
  a.h = p.h;
  a.eps = p.eps;
  a.cf = make_coef(p);
  a.flags = c->flags;
  long long left = n_steps;
  while (left > 0) {
    const long long s = left < chunk ? left : chunk;
    a.step0 = c->steps;
    a.nsteps = (int)s;
    cudaError_t e = fp32c  ? launch_iterate_fp32c_v(a, p.scheme, p.tangent, c->reduce64, block, (int)grid, c->stream)
                    : df64 ? launch_iterate_df64(a, p.scheme, p.tangent, fast, block, (int)grid, c->stream)
                           : launch_iterate_fp64(a, p.scheme, p.tangent, block, (int)grid, c->stream);
    if (e != cudaSuccess) return cuda_status(e);
    c->launches++;
    c->steps += s;
    left -= s;
  }
  return ARNOLD_OK;
}

int64_t arnold_steps_done(const arnold_ctx* c) { return c ? c->steps : -1; }

int arnold_set_snapshots(arnold_ctx* c, double* v_snap, int64_t k_max) {
  if (!c) return ARNOLD_EINVAL;
  if (!v_snap) {
    c->s.snap = nullptr;
    c->s.snap_k = 0;
    return ARNOLD_OK;
  }
  if (c->prm.window <= 0 || k_max < 1 || ((uintptr_t)v_snap & 7)) return ARNOLD_EINVAL;
  c->s.snap = v_snap;
  c->s.snap_k = k_max;
  return ARNOLD_OK;
}

int64_t arnold_launch_count(const arnold_ctx* c) { return c ? c->launches : -1; }

int arnold_indicator(arnold_ctx* c, int kind, void* out, int ptr_kind) {
  if (!c || !out || (ptr_kind != ARNOLD_HOST && ptr_kind != ARNOLD_DEVICE)) return ARNOLD_EINVAL;
  const size_t bytes = indicator_bytes(kind, c->n);
  if (!bytes) return ARNOLD_EINVAL;
  const bool needs_tan = kind == ARNOLD_IND_CHI || kind == ARNOLD_IND_CLASS || kind == ARNOLD_IND_LOGSUM ||
                         kind == ARNOLD_IND_TANGENT;
  if (needs_tan && !c->prm.tangent) return ARNOLD_EINVAL;
  if ((kind == ARNOLD_IND_MEGNO || kind == ARNOLD_IND_MEGNO_Y) && !c->s.megno) return ARNOLD_EINVAL;
  if (fault_is("nan")) return ARNOLD_ENONFINITE;
  ACHECK(cudaSetDevice(c->device));
  if (ptr_kind == ARNOLD_DEVICE) return read_indicator(c, kind, out);
  int st = device_scratch(c);
  if (st) return st;
  st = read_indicator(c, kind, c->scratch);
  if (st) return st;
  ACHECK(cudaMemcpyAsync(out, c->scratch, bytes, cudaMemcpyDeviceToHost, c->stream));
  return check_flags(c);
}

int arnold_stats_arrays(arnold_ctx* c, int64_t n, const double* chi, const double* dE, const double* p, double t,
                        double kappa, arnold_stats* out) {
  if (!c || !out || !chi || !p || n <= 0 || !(kappa > 0.0) || t == 0.0) return ARNOLD_EINVAL;
  ACHECK(cudaSetDevice(c->device));
  long long g = (n + 255) / 256;
  const int grid = (int)(g < c->stats_grid ? g : c->stats_grid);
  const double tt = fabs(t);
  const double thr = kappa * log(tt > M_E ? tt : M_E) / tt;
  ACHECK(launch_stats(n, chi, dE, p, thr, c->partials, grid, c->stats_out, c->stream));
  c->launches += 2;
  StatsPartial h;
  ACHECK(cudaMemcpyAsync(&h, c->stats_out, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  ACHECK(cudaStreamSynchronize(c->stream));
  memcpy(out->hist, h.hist, sizeof out->hist);
  out->under = h.under;
  out->over = h.over;
  out->chaotic = h.chaotic;
  out->n = h.n;
  out->dE_max = h.dE_max;
  for (int k = 0; k < 3; ++k) {
    out->p_mean[k] = h.mean[k];
    out->p_var[k] = h.n ? h.m2[k] / (double)h.n : 0.0;
  }
  out->t = t;
  return ARNOLD_OK;
}

int arnold_stats_compute(arnold_ctx* c, arnold_stats* out) {
  if (!c || !out || !c->prm.tangent) return ARNOLD_EINVAL;
  if (c->steps == 0) return ARNOLD_ESTATE;
  ACHECK(cudaSetDevice(c->device));
  const size_t n = (size_t)c->n;
  if (!c->scratch2) ACHECK(dalloc(&c->scratch2, 6 * n));
  double* chi = c->scratch2;
  double* de = c->scratch2 + n;
  double* pp = c->scratch2 + 2 * n;
  int st = read_indicator(c, ARNOLD_IND_CHI, chi);
  if (!st) st = read_indicator(c, ARNOLD_IND_DE_MAX, de);
  if (!st) st = read_indicator(c, ARNOLD_IND_P, pp);
  if (st) return st;
  st = arnold_stats_arrays(c, c->n, chi, de, pp, (double)c->steps * c->prm.h, c->prm.chaos_kappa, out);
  if (st) return st;
  return check_flags(c);
}

static int ensure_bytes(void** p, size_t* have, size_t need) {
  if (*have >= need && *p) return ARNOLD_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  ACHECK(cudaMalloc(p, need));
  *have = need;
  return ARNOLD_OK;
}

int arnold_forward_ckpt(arnold_ctx* c, int64_t n_steps, int64_t ckpt_every) {
  if (!c || n_steps < 1 || ckpt_every < 0) return ARNOLD_EINVAL;
  if ((c->prm.precision == ARNOLD_FP32C && c->reduce64) || c->prm.precision == ARNOLD_DF64 ||
      c->prm.precision == ARNOLD_DF64F)
    return ARNOLD_EUNSUPPORTED;
  ACHECK(cudaSetDevice(c->device));
  long long C = ckpt_every > 0 ? ckpt_every : (long long)ceil(sqrt((double)n_steps));
  if (C > n_steps) C = n_steps;
  const long long K = (n_steps + C - 1) / C;
  const bool f32 = c->prm.precision == ARNOLD_FP32C;
  const size_t n = (size_t)c->n;
  const size_t per = f32 ? 12 * sizeof(float) * n : 6 * sizeof(double) * n;
  int st = ensure_bytes(&c->ck, &c->ck_bytes, per * (size_t)K);
  if (!st) st = ensure_bytes(&c->seg, &c->seg_bytes, per * (size_t)C);
  if (st) return st;
  if (!c->gh) ACHECK(dalloc(&c->gh, n));
  if (!c->ge) ACHECK(dalloc(&c->ge, n));
  if (!c->sum_part) ACHECK(dalloc(&c->sum_part, 2 * (size_t)c->stats_grid + 2));
  if (f32) {
    if (!c->lamf) ACHECK(dalloc(&c->lamf, 6 * n));
  } else {
    if (!c->lam) ACHECK(dalloc(&c->lam, 6 * n));
  }
  long long left = n_steps;
  for (long long k = 0; k < K; ++k) {
    char* dst = (char*)c->ck + per * (size_t)k;
    if (f32) {
      ACHECK(cudaMemcpyAsync(dst, c->f.hi, 6 * sizeof(float) * n, cudaMemcpyDeviceToDevice, c->stream));
      ACHECK(cudaMemcpyAsync(dst + 6 * sizeof(float) * n, c->f.lo, 6 * sizeof(float) * n, cudaMemcpyDeviceToDevice,
                             c->stream));
    } else {
      ACHECK(cudaMemcpyAsync(dst, c->s.st, per, cudaMemcpyDeviceToDevice, c->stream));
    }
    const long long s = left < C ? left : C;
    st = arnold_iterate(c, s);
    if (st) return st;
    left -= s;
  }
  c->adj_valid = 1;
  c->adj_N = n_steps;
  c->adj_C = C;
  c->adj_K = K;
  return ARNOLD_OK;
}

int arnold_grad(arnold_ctx* c, const double* dL_dx, const double* dL_dp, double* g_x0, double* g_p0,
                double* g_params, int ptr_kind) {
  if (!c || !g_x0 || !g_p0 || !g_params || (ptr_kind != ARNOLD_HOST && ptr_kind != ARNOLD_DEVICE))
    return ARNOLD_EINVAL;
  if (!c->adj_valid) return ARNOLD_ESTATE;
  ACHECK(cudaSetDevice(c->device));
  const bool f32 = c->prm.precision == ARNOLD_FP32C;
  const size_t n = (size_t)c->n;
  int st = device_scratch(c);
  if (st) return st;
  const double* dx = dL_dx;
  const double* dp = dL_dp;
  double* gx = g_x0;
  double* gp = g_p0;
  if (ptr_kind == ARNOLD_HOST) {   // stage through the [6][n] scratch
    double* d = c->scratch;
    if (dL_dx) ACHECK(cudaMemcpyAsync(d, dL_dx, 24 * n, cudaMemcpyHostToDevice, c->stream));
    if (dL_dp) ACHECK(cudaMemcpyAsync(d + 3 * n, dL_dp, 24 * n, cudaMemcpyHostToDevice, c->stream));
    dx = dL_dx ? d : nullptr;
    dp = dL_dp ? d + 3 * n : nullptr;
    gx = d;
    gp = d + 3 * n;
  }
  const int g256 = grid_for(c, 256);
  ACHECK(launch_adj_init(c->n, dx, dp, f32 ? nullptr : c->lam, f32 ? c->lamf : nullptr, c->gh, c->ge, g256,
                         c->stream));
  c->launches++;
  AdjArgs a;
  memset(&a, 0, sizeof a);
  a.ck64 = f32 ? nullptr : (const double*)c->ck;
  a.seg64 = f32 ? nullptr : (double*)c->seg;
  a.ck32 = f32 ? (const float*)c->ck : nullptr;
  a.seg32 = f32 ? (float*)c->seg : nullptr;
  a.lam = c->lam;
  a.lamf = c->lamf;
  a.gh = c->gh;
  a.ge = c->ge;
  a.sc = c->sc;
  a.th = c->th;
  a.scf = c->scf;
  a.n = c->n;
  a.cf = make_coef(c->prm);
  double w[9];
  const int m = scheme_weights(c->prm.scheme, w);
  for (int k = 0; k < m; ++k) {
    a.ch[k] = 2.0 * w[k] * c->prm.eps;
    a.ce[k] = 2.0 * w[k] * c->prm.h;
    a.chf[k] = (float)a.ch[k];
    a.cef[k] = (float)a.ce[k];
  }
  for (int k = 0; k <= m; ++k) {
    const double left = k > 0 ? w[k - 1] : 0.0, right = k < m ? w[k] : 0.0;
    a.cd[k] = 0.5 * (left + right);
    a.cdf[k] = (float)a.cd[k];
  }
  long long g = (c->n + 255) / 256;
  const long long cap = (long long)c->sms * adjoint_blocks_per_sm(c->prm.scheme, f32);
  if (g > cap) g = cap;
  for (long long k = c->adj_K - 1; k >= 0; --k) {
    a.k = (int)k;
    const long long s0 = k * c->adj_C;
    a.steps = (int)((c->adj_N - s0) < c->adj_C ? (c->adj_N - s0) : c->adj_C);
    ACHECK(launch_adjoint_segment(a, c->prm.scheme, f32, (int)g, c->stream));
    c->launches++;
  }
  ACHECK(launch_adj_finish(c->n, f32 ? nullptr : c->lam, f32 ? c->lamf : nullptr, gx, gp, g256, c->stream));
  long long gs = (c->n + 255) / 256;
  const int sg = (int)(gs < c->stats_grid ? gs : c->stats_grid);
  double* out2 = c->sum_part + 2 * c->stats_grid;
  ACHECK(launch_sum2(c->n, c->gh, c->ge, c->sum_part, sg, out2, c->stream));
  c->launches += 3;
  if (ptr_kind == ARNOLD_HOST) {
    ACHECK(cudaMemcpyAsync(g_x0, gx, 24 * n, cudaMemcpyDeviceToHost, c->stream));
    ACHECK(cudaMemcpyAsync(g_p0, gp, 24 * n, cudaMemcpyDeviceToHost, c->stream));
    ACHECK(cudaMemcpyAsync(g_params, out2, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    ACHECK(cudaStreamSynchronize(c->stream));
  } else {
    ACHECK(cudaMemcpyAsync(g_params, out2, 2 * sizeof(double), cudaMemcpyDeviceToDevice, c->stream));
  }
  return ARNOLD_OK;
}

struct CkptHeader {
  char magic[8];
  int32_t precision, tangent;
  int64_t n, steps;
  int32_t scheme, megno;
  double eps, h;
  int32_t tracking, reserved0;   // area tracking on (1) / off (0)
  double patch[4];               // the tracked patch (cos_lo, cos_hi, phi_lo, phi_hi) when on
  int64_t reserved[4];
};
static_assert(sizeof(CkptHeader) == 128, "checkpoint header is 128 bytes");

// (device pointer, bytes) of every array that makes up the state, the
// area-tracking flags included when tracking is on.
static int ckpt_arrays(const arnold_ctx* c, void** ptrs, size_t* sizes) {
  const size_t n = (size_t)c->n;
  int k = 0;
  auto add = [&](void* p, size_t b) {
    if (p) { ptrs[k] = p; sizes[k] = b; ++k; }
  };
  add(c->s.st, 48 * n);
  add(c->s.tg, 48 * n);
  add(c->f.hi, 24 * n);
  add(c->f.lo, 24 * n);
  add(c->f.tg, 24 * n);
  add(c->f.tg_lo, 24 * n);
  add(c->s.lap, 12 * n);
  add(c->s.lapref, 12 * n);
  add(c->s.ref, 24 * n);
  add(c->s.logsum, 8 * n);
  add(c->s.demax, 8 * n);
  add(c->s.e0, 8 * n);
  add(c->s.V, 24 * n);
  add(c->s.p0, 24 * n);
  add(c->s.megno, 16 * n);
  add(c->s.left, n);
  return k;
}

int arnold_checkpoint_size(const arnold_ctx* c, size_t* bytes) {
  if (!c || !bytes) return ARNOLD_EINVAL;
  void* p[16];
  size_t sz[16];
  const int k = ckpt_arrays(c, p, sz);
  size_t total = sizeof(CkptHeader);
  for (int i = 0; i < k; ++i) total += sz[i];
  *bytes = total;
  return ARNOLD_OK;
}

int arnold_checkpoint_save(arnold_ctx* c, void* buf, size_t bytes) {
  size_t need = 0;
  if (!c || !buf || arnold_checkpoint_size(c, &need) || bytes < need) return ARNOLD_EINVAL;
  ACHECK(cudaSetDevice(c->device));
  CkptHeader hd;
  memset(&hd, 0, sizeof hd);
  memcpy(hd.magic, "ARNOLDC2", 8);
  hd.precision = c->prm.precision;
  hd.tangent = c->prm.tangent;
  hd.n = c->n;
  hd.steps = c->steps;
  hd.scheme = c->prm.scheme;
  hd.megno = c->prm.megno;
  hd.eps = c->prm.eps;
  hd.h = c->prm.h;
  hd.tracking = c->s.left != nullptr;
  if (hd.tracking) memcpy(hd.patch, c->s.patch, sizeof hd.patch);
  memcpy(buf, &hd, sizeof hd);
  void* p[16];
  size_t sz[16];
  const int k = ckpt_arrays(c, p, sz);
  char* dst = (char*)buf + sizeof hd;
  for (int i = 0; i < k; ++i) {
    ACHECK(cudaMemcpyAsync(dst, p[i], sz[i], cudaMemcpyDeviceToHost, c->stream));
    dst += sz[i];
  }
  ACHECK(cudaStreamSynchronize(c->stream));
  return ARNOLD_OK;
}

int arnold_checkpoint_load(arnold_ctx* c, const void* buf, size_t bytes) {
  if (!c || !buf || bytes < sizeof(CkptHeader)) return ARNOLD_EINVAL;
  CkptHeader hd;
  memcpy(&hd, buf, sizeof hd);
  if (memcmp(hd.magic, "ARNOLDC2", 8) || hd.precision != c->prm.precision || hd.tangent != c->prm.tangent ||
      hd.n != c->n || hd.scheme != c->prm.scheme || hd.megno != c->prm.megno || hd.eps != c->prm.eps ||
      hd.h != c->prm.h || hd.steps < 0)
    return ARNOLD_EINVAL;
  // area tracking must match: on with the same patch (arnold_track_patch first), or off
  const int tracking = c->s.left != nullptr;
  if (hd.tracking != tracking || (tracking && memcmp(hd.patch, c->s.patch, sizeof hd.patch)))
    return ARNOLD_EINVAL;
  size_t need = 0;
  if (arnold_checkpoint_size(c, &need) || bytes < need) return ARNOLD_EINVAL;
  ACHECK(cudaSetDevice(c->device));
  void* p[16];
  size_t sz[16];
  const int k = ckpt_arrays(c, p, sz);
  const char* src = (const char*)buf + sizeof hd;
  for (int i = 0; i < k; ++i) {
    ACHECK(cudaMemcpyAsync(p[i], src, sz[i], cudaMemcpyHostToDevice, c->stream));
    src += sz[i];
  }
  ACHECK(cudaMemsetAsync(c->flags, 0, sizeof(int), c->stream));
  ACHECK(cudaStreamSynchronize(c->stream));
  c->steps = hd.steps;
  c->adj_valid = 0;
  return ARNOLD_OK;
}

int arnold_sync(arnold_ctx* c) {
  if (!c) return ARNOLD_EINVAL;
  if (fault_is("timeout")) return ARNOLD_ETIMEOUT;
  ACHECK(cudaSetDevice(c->device));
  ACHECK(cudaStreamSynchronize(c->stream));
  ACHECK(cudaGetLastError());
  return check_flags(c);
}

int arnold_debug_sincos(arnold_ctx* c, int precision, int64_t n, const double* x, double* s, double* co) {
  if (!c || !x || !s || !co || n <= 0) return ARNOLD_EINVAL;
  ACHECK(cudaSetDevice(c->device));
  cudaError_t e = precision == ARNOLD_FP32C  ? launch_debug_sincos32(x, s, co, n, c->scf, c->stream)
                 : precision == ARNOLD_DF64 ? launch_debug_sincos_df(x, s, co, n, c->scd, false, c->stream)
                 : precision == ARNOLD_DF64F ? launch_debug_sincos_df(x, s, co, n, c->scd, true, c->stream)
                                            : launch_debug_sincos64(x, s, co, n, c->sc, c->th, c->stream);
  ACHECK(e);
  c->launches++;
  ACHECK(cudaStreamSynchronize(c->stream));
  return ARNOLD_OK;
}

int arnold_probe_peak(int device, int kind, double* ops) {
  if (!ops || kind < 0 || kind > 2) return ARNOLD_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= 0) return ARNOLD_EUNSUPPORTED;
  if (device < 0 || device >= ndev) return ARNOLD_EINVAL;
  ACHECK(cudaSetDevice(device));
  int sms = 0;
  ACHECK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  // full occupancy (8 x 256 threads per SM), 8 independent chains per thread
  const int block = 256, grid = sms * 8;
  double* sink = nullptr;
  ACHECK(cudaMalloc(&sink, sizeof(double) * (size_t)grid * block));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  // size one launch to ~100 ms from a short one, run ~300 ms to bring the clocks
  // up, then keep the best of 6 timed launches (~0.6 s)
  int iters = kind == 0 ? 256 : (kind == 1 ? 8192 : 2048);
  float ms = 0.f, best = 1e30f;
  cudaError_t err = cudaEventRecord(e0, 0);
  if (err == cudaSuccess) err = launch_probe(kind, grid, block, iters, sink, 0);
  if (err == cudaSuccess) err = cudaEventRecord(e1, 0);
  if (err == cudaSuccess) err = cudaEventSynchronize(e1);
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  if (err == cudaSuccess && ms > 0.f) {
    const double scale = 100.0 / ms;
    iters = (int)fmin(fmax(iters * scale, 16.0), 1.0e8);
  }
  for (int r = 0; r < 9 && err == cudaSuccess; ++r) {
    err = cudaEventRecord(e0, 0);
    if (err == cudaSuccess) err = launch_probe(kind, grid, block, iters, sink, 0);
    if (err == cudaSuccess) err = cudaEventRecord(e1, 0);
    if (err == cudaSuccess) err = cudaEventSynchronize(e1);
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    if (err == cudaSuccess && r >= 3 && ms > 0.f && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (err != cudaSuccess) return cuda_status(err);
  *ops = (double)grid * block * (double)iters * 8.0 / (best * 1e-3);
  return ARNOLD_OK;
}

}  // extern "C"
