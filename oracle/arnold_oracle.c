/*
 * Oracle for the Arnold-web ensemble propagator -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded FP64 CPU implementation of what the GPU hot
 * path computes, written for a reader checking it against the paper by eye.
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
 * leg may load it.  It shares no code, header, table or constant generator
 * with the CUDA path (paper_1107_4107_b300/csrc), and neither side includes
 * the other.  Build: gcc -O2 -ffp-contract=off -fPIC -shared -lm (no FMA
 * contraction, no fast-math).
 *
 * Model (paper Sec. II, Eqs. 1-2):
 *   H(P, X) = |P|^2 / 2 + eps * Hp(X),   Hp(x, y, z) = cos x cos y (1 + cos 2z),
 *   X on the torus [0, 2pi)^3.  Equations of motion dX/dt = P, dP/dt = -eps grad Hp.
 *
 * Integrator (paper Sec. III: "sixth-order symplectic integrator", h = 1e-2 T,
 * T = 2 pi).  The cited reference for the scheme is missing from the paper;
 * the reading adopted is a symmetric composition of drift-kick-drift leapfrog
 * substeps  L(tau) = D(tau/2) K(tau) D(tau/2)  with
 *   scheme 0: Yoshida (1990) 6th order, "solution A" weights (7 substeps),
 *   scheme 1: 6th-order recursive triple jump (9 substeps),
 *   scheme 2: plain leapfrog, 2nd order (1 substep).
 *   D(s): X += s P, then each angle brought back into [0, 2pi) one lap of the
 *         FP64 constant 2pi at a time, counting laps (+1 / -1).
 *   K(t): P -= t eps grad Hp(X).
 *
 * Tangent map (chaos indicator; the paper contrasts its method with finite-time
 * Lyapunov exponents, Sec. V): the same composition applied to w = (dX, dP):
 *   D(s): dX += s dP;   K(t): dP -= t eps Hess Hp(X) dX  (Hessian at the kick's X).
 *   Every R steps (global step index multiple of R): l = |w|, logsum += ln l, w /= l.
 *
 * MEGNO (the mean exponential growth factor of nearby orbits; Cincotta and
 * Simo, Astron. Astrophys. Suppl. 147 (2000) 205; for maps Cincotta, Giordano
 * and Simo, Physica D 182 (2003) 151) -- not in the paper, an alternative
 * tangent-based indicator.  Its continuous definitions are
 *   Y(t) = (2/t) int_0^t s d ln|w(s)|,   <Y>(t) = (1/t) int_0^t Y(s) ds.
 * Sampled at the renormalisation points t_j = j R h (j = 1, 2, ... counted from
 * the start of the run) with the increment over (t_{j-1}, t_j] taken at its
 * right end, as the map form does: with l_j = ln of the norm growth over
 * interval j,  Y_m = (2/m) sum_{j<=m} j l_j  and  <Y>_m = (1/m) sum_{k<=m} Y_k.
 * Accumulated per trajectory: S_m = sum_{j<=m} j l_j and Ysum_m = sum_{k<=m} Y_k.
 *
 * Parity: pinned (see tests/test_oracle_pins.py) by the free-rotation closed
 * form at eps = 0, the Chirikov standard map on an invariant subspace, the
 * pendulum period on that subspace, invariant subspaces, sixth-order
 * convergence, symplecticity of the tangent map, reversibility, and central
 * finite differences; MEGNO (tests/test_oracle_megno.py) by the free-flow
 * closed form of the tangent norm, its limits 0 (stable equilibrium), 2
 * (linear growth) and lambda t / 2 (chaos), and the summation-by-parts
 * identity against the log-sum history.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_TWO_PI 6.283185307179586476925286766559

typedef struct {
  double eps;           /* epsilon of Eq. 1 (the paper sets it to 1, Eq. 3)        */
  double h;             /* time step of one composite step (paper: 0.01 * 2 pi)   */
  int32_t scheme;       /* 0 Yoshida-6A, 1 triple-jump-6, 2 leapfrog-2           */
  int32_t renorm_every; /* R: tangent renormalisation interval in steps (>= 1)   */
  int64_t window;       /* W: steps per averaging window of V (0 = whole run)     */
} oracle_params;

/* ---------------------------------------------------------------- scheme --- */
/* Leapfrog weights w_k of one composite step; returns the count m.
 * Yoshida, Phys. Lett. A 150 (1990) 262, Table 1, solution A:
 *   w1 = -1.17767998417887, w2 = 0.235573213359357, w3 = 0.784513610477560,
 *   w0 = 1 - 2 (w1 + w2 + w3); order of application w3 w2 w1 w0 w1 w2 w3.
 * Triple jump (Creutz-Gocksch 1989, Suzuki 1990, Yoshida 1990):
 *   S4(h) = S2(g1 h) S2(g0 h) S2(g1 h), g1 = 1/(2 - 2^(1/3)), g0 = 1 - 2 g1,
 *   S6(h) = S4(d1 h) S4(d0 h) S4(d1 h), d1 = 1/(2 - 2^(1/5)), d0 = 1 - 2 d1. */
int oracle_scheme_weights(int scheme, double* w) {
  if (scheme == 0) {
    double w1 = -1.17767998417887, w2 = 0.235573213359357, w3 = 0.784513610477560;
    double w0 = 1.0 - 2.0 * (w1 + w2 + w3);
    w[0] = w3; w[1] = w2; w[2] = w1; w[3] = w0; w[4] = w1; w[5] = w2; w[6] = w3;
    return 7;
  }
  if (scheme == 1) {
    double g1 = 1.0 / (2.0 - pow(2.0, 1.0 / 3.0)), g0 = 1.0 - 2.0 * g1;
    double d1 = 1.0 / (2.0 - pow(2.0, 1.0 / 5.0)), d0 = 1.0 - 2.0 * d1;
    double outer[3] = {d1, d0, d1}, inner[3] = {g1, g0, g1};
    int k = 0;
    for (int a = 0; a < 3; a++)
      for (int b = 0; b < 3; b++) w[k++] = outer[a] * inner[b];
    return 9;
  }
  if (scheme == 2) { w[0] = 1.0; return 1; }
  return -1;
}

/* ------------------------------------------------------------- potential --- */
/* Eq. 2: Hp = cos x cos y (1 + cos 2z). */
double oracle_hp(double x, double y, double z) {
  return cos(x) * cos(y) * (1.0 + cos(2.0 * z));
}

/* Gradient of Eq. 2, differentiated term by term. */
static void grad_hp(const double X[3], double g[3]) {
  double x = X[0], y = X[1], z = X[2];
  g[0] = -sin(x) * cos(y) * (1.0 + cos(2.0 * z));
  g[1] = -cos(x) * sin(y) * (1.0 + cos(2.0 * z));
  g[2] = -2.0 * cos(x) * cos(y) * sin(2.0 * z);
}

/* Hessian of Eq. 2 (symmetric 3x3). */
static void hess_hp(const double X[3], double H[3][3]) {
  double x = X[0], y = X[1], z = X[2];
  H[0][0] = -cos(x) * cos(y) * (1.0 + cos(2.0 * z));
  H[1][1] = -cos(x) * cos(y) * (1.0 + cos(2.0 * z));
  H[2][2] = -4.0 * cos(x) * cos(y) * cos(2.0 * z);
  H[0][1] = H[1][0] = sin(x) * sin(y) * (1.0 + cos(2.0 * z));
  H[0][2] = H[2][0] = 2.0 * sin(x) * cos(y) * sin(2.0 * z);
  H[1][2] = H[2][1] = 2.0 * cos(x) * sin(y) * sin(2.0 * z);
}

void oracle_grad_hp(const double* X, double* g) { grad_hp(X, g); }
void oracle_hess_hp(const double* X, double* H9) {
  double H[3][3];
  hess_hp(X, H);
  for (int a = 0; a < 3; a++)
    for (int b = 0; b < 3; b++) H9[3 * a + b] = H[a][b];
}

/* Eq. 1 for one phase-space point. */
double oracle_energy1(double eps, const double X[3], const double P[3]) {
  return 0.5 * (P[0] * P[0] + P[1] * P[1] + P[2] * P[2]) + eps * oracle_hp(X[0], X[1], X[2]);
}

/* ------------------------------------------------------ one trajectory --- */
typedef struct {
  double X[3], P[3];
  double w[6];          /* tangent (dX, dP) */
  int64_t lap[3];       /* laps since the window started */
  double logsum;
  double mg_s;          /* MEGNO: sum over renormalisations j of j * ln(growth) */
  double mg_y;          /* MEGNO: sum over renormalisations of Y_j              */
  double dE_max;
  double e0;
  double xref[3];       /* reduced angle at the window start */
  double V[3];          /* finite-time averaged velocity of the last closed window */
} traj;

/* Bring one angle into [0, 2pi), one lap of 2pi at a time. */
static void wrap_angle(double* x, int64_t* lap) {
  for (;;) {
    if (*x >= ORACLE_TWO_PI) { *x -= ORACLE_TWO_PI; (*lap)++; }
    else if (*x < 0.0) { *x += ORACLE_TWO_PI; (*lap)--; }
    else break;
  }
}

static void drift(traj* t, double s, int tangent) {
  for (int a = 0; a < 3; a++) {
    t->X[a] += s * t->P[a];
    wrap_angle(&t->X[a], &t->lap[a]);
    if (tangent) t->w[a] += s * t->w[3 + a];
  }
}

static void kick(traj* t, double tau, double eps, int tangent) {
  double g[3];
  grad_hp(t->X, g);
  for (int a = 0; a < 3; a++) t->P[a] -= tau * eps * g[a];
  if (tangent) {
    double H[3][3];
    hess_hp(t->X, H);
    double dX[3] = {t->w[0], t->w[1], t->w[2]};
    for (int a = 0; a < 3; a++) {
      double hv = H[a][0] * dX[0] + H[a][1] * dX[1] + H[a][2] * dX[2];
      t->w[3 + a] -= tau * eps * hv;
    }
  }
}

/* One composite step: L(w_0 h) ... L(w_{m-1} h), L(tau) = D(tau/2) K(tau) D(tau/2). */
static void composite_step(traj* t, const oracle_params* prm, const double* wts, int m, int tangent) {
  for (int k = 0; k < m; k++) {
    double tau = wts[k] * prm->h;
    drift(t, 0.5 * tau, tangent);
    kick(t, tau, prm->eps, tangent);
    drift(t, 0.5 * tau, tangent);
  }
}

static double norm6(const double* w) {
  double s = 0.0;
  for (int k = 0; k < 6; k++) s += w[k] * w[k];
  return sqrt(s);
}

/* Bookkeeping at the end of global step `step` (1-based count of steps taken). */
static void end_of_step(traj* t, const oracle_params* prm, int64_t step, int tangent) {
  if (step % prm->renorm_every == 0) {
    if (tangent) {
      double l = norm6(t->w);
      t->logsum += log(l);
      for (int k = 0; k < 6; k++) t->w[k] /= l;
      double j = (double)(step / prm->renorm_every);   /* index of this renormalisation */
      t->mg_s += j * log(l);
      t->mg_y += 2.0 * t->mg_s / j;
    }
    double dE = fabs(oracle_energy1(prm->eps, t->X, t->P) - t->e0);
    if (dE > t->dE_max) t->dE_max = dE;
  }
  if (prm->window > 0 && step % prm->window == 0) {
    double dt = (double)prm->window * prm->h;
    for (int a = 0; a < 3; a++) {
      t->V[a] = (t->X[a] - t->xref[a] + ORACLE_TWO_PI * (double)t->lap[a]) / dt;
      t->xref[a] = t->X[a];
      t->lap[a] = 0;
    }
  }
}

/*
 * Propagate n trajectories for n_steps composite steps starting at global step
 * step0 (the number of steps already taken).  All arrays are structure-of-
 * arrays [component][n], updated in place:
 *   X[3][n], P[3][n]     state (X reduced into [0, 2pi))
 *   W[6][n] or NULL      tangent (dX, dP); NULL = no tangent
 *   lap[3][n]            laps since the current window started
 *   xref[3][n]           reduced angle at the window start
 *   logsum[n], dE_max[n], e0[n]  (logsum may be NULL when W is NULL)
 *   V[3][n] or NULL      V of the last closed window (written when a window closes)
 *   megno[2][n] or NULL  MEGNO sums (S, Ysum) over the renormalisations so far
 * Returns 0, or -1 on a bad argument.
 */
int oracle_run(const oracle_params* prm, int64_t n, int64_t step0, int64_t n_steps,
               double* X, double* P, double* W, int64_t* lap, double* xref,
               double* logsum, double* dE_max, const double* e0, double* V, double* megno) {
  double wts[9];
  int m = oracle_scheme_weights(prm->scheme, wts);
  if (m < 0 || n < 0 || n_steps < 0 || prm->renorm_every < 1 || prm->window < 0) return -1;
  int tangent = (W != NULL);
  for (int64_t i = 0; i < n; i++) {
    traj t;
    memset(&t, 0, sizeof t);
    for (int a = 0; a < 3; a++) {
      t.X[a] = X[a * n + i];
      t.P[a] = P[a * n + i];
      t.lap[a] = lap[a * n + i];
      t.xref[a] = xref[a * n + i];
      t.V[a] = V ? V[a * n + i] : 0.0;
    }
    if (tangent)
      for (int k = 0; k < 6; k++) t.w[k] = W[k * n + i];
    t.logsum = logsum ? logsum[i] : 0.0;
    t.mg_s = megno ? megno[i] : 0.0;
    t.mg_y = megno ? megno[n + i] : 0.0;
    t.dE_max = dE_max[i];
    t.e0 = e0[i];
    for (int64_t s = 0; s < n_steps; s++) {
      composite_step(&t, prm, wts, m, tangent);
      end_of_step(&t, prm, step0 + s + 1, tangent);
    }
    for (int a = 0; a < 3; a++) {
      X[a * n + i] = t.X[a];
      P[a * n + i] = t.P[a];
      lap[a * n + i] = t.lap[a];
      xref[a * n + i] = t.xref[a];
      if (V) V[a * n + i] = t.V[a];
    }
    if (tangent)
      for (int k = 0; k < 6; k++) W[k * n + i] = t.w[k];
    if (logsum) logsum[i] = t.logsum;
    if (megno) {
      megno[i] = t.mg_s;
      megno[n + i] = t.mg_y;
    }
    dE_max[i] = t.dE_max;
  }
  return 0;
}

/*
 * Momenta on the energy shell along given unit directions (the ensembles of
 * Sec. IV, uniform over the sphere S): |P| = sqrt(2 (E - eps Hp(X))),
 * P = |P| nhat.  Returns the number of points with a negative radicand (P = NaN).
 */
int64_t oracle_momenta_on_shell(double E, double eps, int64_t n, const double* X, const double* nhat, double* P) {
  int64_t bad = 0;
  for (int64_t i = 0; i < n; i++) {
    double r = 2.0 * (E - eps * oracle_hp(X[i], X[n + i], X[2 * n + i]));
    double m = r >= 0.0 ? sqrt(r) : NAN;
    if (!(r >= 0.0)) bad++;
    for (int a = 0; a < 3; a++) P[a * n + i] = m * nhat[a * n + i];
  }
  return bad;
}

/*
 * Area tracking (Sec. IV, Fig. 3 zooms: only trajectories that stay within the
 * scanned area for the whole observation time are kept).  Sampled every R
 * steps: the momentum direction (cos theta = p_z / |P|, phi = atan2(p_y, p_x)
 * in [0, 2pi)) must stay inside [cos_lo, cos_hi] x [phi_lo, phi_hi];
 * left[i] becomes 1 the first time it does not.
 */
static int inside_patch(const double P[3], const double* patch) {
  double m = sqrt(P[0] * P[0] + P[1] * P[1] + P[2] * P[2]);
  double c = P[2] / m;
  double phi = atan2(P[1], P[0]);
  if (phi < 0.0) phi += ORACLE_TWO_PI;
  return c >= patch[0] && c <= patch[1] && phi >= patch[2] && phi <= patch[3];
}

int oracle_track(const oracle_params* prm, int64_t n, int64_t step0, int64_t n_steps, double* X, double* P,
                 const double* patch, uint8_t* left) {
  double wts[9];
  int m = oracle_scheme_weights(prm->scheme, wts);
  if (m < 0 || prm->renorm_every < 1) return -1;
  for (int64_t i = 0; i < n; i++) {
    traj t;
    memset(&t, 0, sizeof t);
    for (int a = 0; a < 3; a++) { t.X[a] = X[a * n + i]; t.P[a] = P[a * n + i]; }
    for (int64_t s = 0; s < n_steps; s++) {
      composite_step(&t, prm, wts, m, 0);
      if ((step0 + s + 1) % prm->renorm_every == 0 && !inside_patch(t.P, patch)) left[i] = 1;
    }
    for (int a = 0; a < 3; a++) { X[a * n + i] = t.X[a]; P[a * n + i] = t.P[a]; }
  }
  return 0;
}

/* Energy (Eq. 1) of n SoA points. */
void oracle_energy(double eps, int64_t n, const double* X, const double* P, double* E) {
  for (int64_t i = 0; i < n; i++) {
    double x[3] = {X[i], X[n + i], X[2 * n + i]};
    double p[3] = {P[i], P[n + i], P[2 * n + i]};
    E[i] = oracle_energy1(eps, x, p);
  }
}

/*
 * Initial p_z from the fixed-energy condition (paper Sec. IV, Fig. 4 caption:
 * v_z "calculated from the fixed energy condition"):
 *   p_z = + sqrt( 2 (E - eps Hp(X)) - p_x^2 - p_y^2 ).
 * P[2][n] is overwritten; returns the number of points with a negative
 * radicand (their p_z is set to NaN).
 */
int64_t oracle_pz_from_energy(double E, double eps, int64_t n, const double* X, double* P) {
  int64_t bad = 0;
  for (int64_t i = 0; i < n; i++) {
    double px = P[i], py = P[n + i];
    double r = 2.0 * (E - eps * oracle_hp(X[i], X[n + i], X[2 * n + i])) - px * px - py * py;
    if (r < 0.0) { P[2 * n + i] = NAN; bad++; }
    else P[2 * n + i] = sqrt(r);
  }
  return bad;
}

/*
 * Forward-mode derivatives of the N-step map z_N = Phi(z_0; h, eps), z = (X, P),
 * for the gradient check of the adjoint.  Propagates, per trajectory, the 6x6
 * Jacobian J = dz_N/dz_0 and the parameter derivatives dz_N/dh, dz_N/deps
 * through every drift and kick:
 *   D(s = c h):  X' = X + c h P       ->  dX' = dX + c h dP (+ c P dh)
 *   K(t = d h):  P' = P - d h eps g(X) ->  dP' = dP - d h eps Hess dX
 *                                            (- d eps g dh - d h g deps)
 * Angle wrapping adds constants and does not change derivatives.
 * Outputs (row-major per trajectory): J[n][6][6], dzdh[n][6], dzdeps[n][6];
 * X, P are advanced in place.
 */
int oracle_jacobian(const oracle_params* prm, int64_t n, int64_t n_steps, double* X, double* P,
                    double* J, double* dzdh, double* dzdeps) {
  double wts[9];
  int m = oracle_scheme_weights(prm->scheme, wts);
  if (m < 0) return -1;
  double h = prm->h, eps = prm->eps;
  for (int64_t i = 0; i < n; i++) {
    double x[3], p[3];
    int64_t lap[3] = {0, 0, 0};
    /* columns 0..5: d/dz0_k ; column 6: d/dh ; column 7: d/deps.  D[row][col]. */
    double D[6][8];
    memset(D, 0, sizeof D);
    for (int k = 0; k < 6; k++) D[k][k] = 1.0;
    for (int a = 0; a < 3; a++) { x[a] = X[a * n + i]; p[a] = P[a * n + i]; }
    for (int64_t s = 0; s < n_steps; s++) {
      for (int k = 0; k < m; k++) {
        double c = 0.5 * wts[k], d = wts[k];
        for (int half = 0; half < 2; half++) {
          if (half == 1) {
            /* kick at the midpoint of the substep */
            double g[3], Hm[3][3];
            grad_hp(x, g);
            hess_hp(x, Hm);
            for (int col = 0; col < 8; col++) {
              double dx[3] = {D[0][col], D[1][col], D[2][col]};
              for (int a = 0; a < 3; a++) {
                double hv = Hm[a][0] * dx[0] + Hm[a][1] * dx[1] + Hm[a][2] * dx[2];
                D[3 + a][col] -= d * h * eps * hv;
                if (col == 6) D[3 + a][col] -= d * eps * g[a];
                if (col == 7) D[3 + a][col] -= d * h * g[a];
              }
            }
            for (int a = 0; a < 3; a++) p[a] -= d * h * eps * g[a];
          }
          /* drift by c h */
          for (int col = 0; col < 8; col++)
            for (int a = 0; a < 3; a++) {
              D[a][col] += c * h * D[3 + a][col];
              if (col == 6) D[a][col] += c * p[a];
            }
          for (int a = 0; a < 3; a++) {
            x[a] += c * h * p[a];
            wrap_angle(&x[a], &lap[a]);
          }
        }
      }
    }
    for (int a = 0; a < 3; a++) { X[a * n + i] = x[a]; P[a * n + i] = p[a]; }
    for (int r = 0; r < 6; r++) {
      for (int col = 0; col < 6; col++) J[i * 36 + r * 6 + col] = D[r][col];
      dzdh[i * 6 + r] = D[r][6];
      dzdeps[i * 6 + r] = D[r][7];
    }
  }
  return 0;
}
