/*
 * EM-PP oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 statement on the CPU of one EM-PP step of arXiv 2605.05543:
 *
 *   Sec. 2.2  for every target i and source j != i, bracket the retarded time in j's stored
 *             trajectory history (near-field shortcut, bisection, out-of-history case), then
 *             rebuild the retarded position, velocity and acceleration by the linear
 *             reconstruction (eq:dt, eq:linear) or the extrapolation of eq:linear2;
 *   Sec. 2.1  form the Lienard-Wiechert fields eq:LW_E and eq:LW_B and superpose them over
 *             j != i, adding the prescribed background field B_geo;
 *   Sec. 2.6  the centred-dipole background field (and a uniform field);
 *   Sec. 2.3  advance every particle with the Higuera-Cary pusher.
 *
 * Only the test suite, the package's smoke check and the benchmark's CPU-baseline leg load this
 * file. It shares no code, header, constant or helper with the CUDA library. It is compiled with
 * -ffp-contract=off so that no a*b+c is ever fused, and every per-target sum runs over j in
 * increasing order with Neumaier compensation (the sum is the plain definition; compensation only
 * makes the FP64 value closer to it). OpenMP, where enabled, splits the targets between threads;
 * it does not change any per-target arithmetic.
 *
 * Readings of the paper that this file fixes (each is listed with its reason in the design notes):
 *   - P(k) = [c (t - t_k)]^2 <= |r - w_k|^2 is the bisection test of Sec. 2.2, written without a
 *     square root and evaluated at the node itself at every iteration; "<=" sends ties to the
 *     older half as the paper's inequality does.
 *   - history depth D counts the present slot: usable slots are k0..n with k0 = max(0, n-D+1).
 *   - order of the three cases: P(k0) -> out-of-history case (eq:linear2, t_r < t_0);
 *     else not P(n-1) -> near-field shortcut [t-dt, t]; else bisection on slot indices
 *     starting from [t_0, t].
 *   - the root of the quadratic eq:dt is the smaller (minus-sign) root, formed without cancellation
 *     as q / C2 or C0 / q with q = -(C1 + sgn(C1) sqrt(C1^2 - 4 C2 C0)) / 2.
 *   - the retarded position is w1 + v1 dt (first form of eq:linear); the velocity is
 *     v1 (1 - df) + v2 df and the acceleration (v2 - v1) / (t2 - t1).
 *   - self fields are evaluated at the present positions x^n and time t_n; the background field
 *     at the half-step position x^{n+1/2}; the push is drift (dt/2) - HC kick - drift (dt/2).
 *   - charge of particle j is -e w_j and its mass m_e w_j.
 *   - adaptive time step (Sec. 2.4): eta_min and v_max come from the retarded solve of step n, with
 *     v_i(t) the target's stored velocity at slot n; the resulting dt is the one the push from n to
 *     n+1 uses; with no qualifying pair, or v_max = 0, dt = dt_max.
 *   - variants kept as accuracy comparisons (not the method): the midpoint reconstruction eq:mid of
 *     the authors' earlier scheme applies to bracketed pairs only (t_r, w, v the bracket's midpoint
 *     values, a the finite difference); out-of-history pairs keep eq:linear2, which eq:mid does not
 *     cover. The half-step field point evaluates the self fields at (x^{n+1/2}, t_n + dt/2), the point
 *     the pusher's kick uses: the history gains a provisional slot n+1 holding (t_n + dt/2, x^{n+1/2},
 *     v^n), formed with the push's own half drift, and counted in the depth D; the push then replaces
 *     it with slot n+1.
 *   - stage switch (Sec. 2.7): E_i is the kinetic energy (gamma_i - 1) m_e c^2 per represented
 *     electron, so the weighted mean is the mean energy per electron; dE/dt at step n is the backward
 *     difference (E_n - E_{n-1}) / (t_n - t_{n-1}); the criterion arms once |dE/dt| >= eps_E (the rate
 *     "falls below" the threshold, so a bunch at rest does not switch at once); the switch step is the
 *     first n at which |dE/dt| < eps_E has held, after arming, for `hold` consecutive steps, n being the
 *     last of them.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* CODATA 2018 (SI): speed of light, elementary charge, electron mass, vacuum permittivity and
   permeability. */
static const double C_LIGHT = 299792458.0;
static const double Q_E = 1.602176634e-19;
static const double M_ELEC = 9.1093837015e-31;
static const double EPS0 = 8.8541878128e-12;
static const double MU0 = 1.25663706212e-6;
static const double PI = 3.14159265358979323846;

/* status codes returned by the entry points below */
enum { ORC_OK = 0, ORC_ERR_ARG = 1, ORC_ERR_NUMERIC = 2 };

/* branches of the retarded-time search */
enum { BR_OUT_OF_HISTORY = 0, BR_SHORTCUT = 1, BR_BISECTION = 2 };

/* step variants (bit mask): the midpoint reconstruction eq:mid, the half-step field point */
enum { VAR_MIDPOINT = 1, VAR_HALF_STEP = 2 };

/* ------------------------------------------------------------------------------------------ */
/* small vector helpers                                                                         */
/* ------------------------------------------------------------------------------------------ */
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void cross3(const double a[3], const double b[3], double out[3]) {
  out[0] = a[1] * b[2] - a[2] * b[1];
  out[1] = a[2] * b[0] - a[0] * b[2];
  out[2] = a[0] * b[1] - a[1] * b[0];
}

/* Neumaier-compensated running sum */
typedef struct {
  double s, c;
} csum;

static void csum_add(csum* a, double x) {
  double t = a->s + x;
  if (fabs(a->s) >= fabs(x))
    a->c += (a->s - t) + x;
  else
    a->c += (x - t) + a->s;
  a->s = t;
}

static double csum_get(const csum* a) { return a->s + a->c; }

/* ------------------------------------------------------------------------------------------ */
/* Trajectory history (Sec. 2.2): slot k holds time T[k] and, for every particle j, the position  */
/* W[k][j][0..2] and velocity V[k][j][0..2]. The oracle keeps every slot 0..n; the depth D only   */
/* sets the earliest usable slot k0.                                                            */
/* ------------------------------------------------------------------------------------------ */
typedef struct {
  int64_t N;
  const double* T;
  const double* W;
  const double* V;
} history;

static const double* hist_w(const history* h, int64_t k, int64_t j) { return h->W + (k * h->N + j) * 3; }
static const double* hist_v(const history* h, int64_t k, int64_t j) { return h->V + (k * h->N + j) * 3; }

/* The bisection test of Sec. 2.2 at node k: true when c (t - t_k) <= |r - w_k|, i.e. when the
   retarded time lies at or before t_k. */
static int node_test(const double r[3], double t, double tk, const double wk[3]) {
  double ct = C_LIGHT * (t - tk);
  double lhs = ct * ct;
  double d0 = r[0] - wk[0], d1 = r[1] - wk[1], d2 = r[2] - wk[2];
  double rhs = d0 * d0 + d1 * d1 + d2 * d2;
  return lhs <= rhs;
}

/* Bracket of Sec. 2.2 for field point (r, t) and source j with usable slots k0..n.
   Returns the branch and sets *k1 (the older node) and *ntest (node tests evaluated). */
static int bracket(const history* h, int64_t j, const double r[3], double t, int64_t k0, int64_t n,
                   int64_t* k1, int* ntest) {
  *ntest = 1;
  if (node_test(r, t, h->T[k0], hist_w(h, k0, j))) {
    /* c (t - t_0) <= |r - w_0|: the retarded time is older than the stored history */
    *k1 = k0;
    return BR_OUT_OF_HISTORY;
  }
  *ntest = 2;
  if (!node_test(r, t, h->T[n - 1], hist_w(h, n - 1, j))) {
    /* |r - w(t - dt)| < c dt: the near-field shortcut [t - dt, t] */
    *k1 = n - 1;
    return BR_SHORTCUT;
  }
  /* bisection on [t_0, t]: the test is false at lo and true at hi */
  int64_t lo = k0, hi = n;
  while (hi - lo > 1) {
    int64_t m = (lo + hi) / 2;
    *ntest += 1;
    if (node_test(r, t, h->T[m], hist_w(h, m, j)))
      hi = m; /* retarded time in [t_lo, t_m] */
    else
      lo = m; /* retarded time in (t_m, t_hi] */
  }
  *k1 = lo;
  return BR_BISECTION;
}

/* Quadratic of eq:dt for delta t = t_r - t1 on the line w1 + v1 delta t, with T1 = t - t1 and
   d = r - w1: C2 x^2 + C1 x + C0 = 0. The physically relevant root is the one with the minus sign,
   i.e. the smaller root (the other lies on the future light cone, delta t > t - t1). Both roots are
   formed in the textbook cancellation-free way, q = -(C1 + sgn(C1) sqrt(disc)) / 2 with roots
   q / C2 and C0 / q, and the smaller one is returned. */
static int solve_dt(const double d[3], double T1, const double v1[3], double* dt_out) {
  double C2 = C_LIGHT * C_LIGHT - dot3(v1, v1);
  double C1 = 2.0 * (dot3(d, v1) - C_LIGHT * C_LIGHT * T1);
  double C0 = C_LIGHT * C_LIGHT * T1 * T1 - dot3(d, d);
  double disc = C1 * C1 - 4.0 * C2 * C0;
  if (!(C2 > 0.0) || !(disc >= 0.0)) return ORC_ERR_NUMERIC;
  double sq = sqrt(disc);
  double q = -0.5 * (C1 + (C1 >= 0.0 ? sq : -sq));
  if (!(q != 0.0)) return ORC_ERR_NUMERIC;
  double ra = q / C2, rb = C0 / q;
  *dt_out = ra < rb ? ra : rb;
  return ORC_OK;
}

/* Retarded position, velocity and acceleration of source j seen from (r, t) at step n
   (eq:linear for the shortcut and bisection branches, eq:linear2 out of history; with `midpoint`,
   eq:mid for the shortcut and bisection branches). */
static int retarded_state(const history* h, int64_t j, const double r[3], double t, int64_t k0, int64_t n,
                          int midpoint, double w[3], double v[3], double a[3], double* tr, int* branch,
                          int64_t* k1out, int* ntest) {
  int64_t k1;
  int br = bracket(h, j, r, t, k0, n, &k1, ntest);
  const double* w1 = hist_w(h, k1, j);
  const double* v1 = hist_v(h, k1, j);
  double t1 = h->T[k1];
  *branch = br;
  *k1out = k1;
  if (midpoint && br != BR_OUT_OF_HISTORY) {
    /* eq:mid: the midpoint of the bracket [t1, t2] stands for the retarded time */
    const double* w2 = hist_w(h, k1 + 1, j);
    const double* v2 = hist_v(h, k1 + 1, j);
    double t2 = h->T[k1 + 1];
    double span = t2 - t1;
    *tr = (t1 + t2) / 2.0;
    for (int c = 0; c < 3; c++) {
      w[c] = (w1[c] + w2[c]) / 2.0;
      v[c] = (v1[c] + v2[c]) / 2.0;
      a[c] = (v2[c] - v1[c]) / span;
    }
    return ORC_OK;
  }
  double d[3] = {r[0] - w1[0], r[1] - w1[1], r[2] - w1[2]};
  double dt;
  int st = solve_dt(d, t - t1, v1, &dt);
  if (st != ORC_OK) return st;
  *tr = t1 + dt;
  for (int c = 0; c < 3; c++) w[c] = w1[c] + v1[c] * dt;
  if (br == BR_OUT_OF_HISTORY) {
    for (int c = 0; c < 3; c++) {
      v[c] = v1[c];
      a[c] = 0.0;
    }
  } else {
    const double* v2 = hist_v(h, k1 + 1, j);
    double t2 = h->T[k1 + 1];
    double df = dt / (t2 - t1);
    for (int c = 0; c < 3; c++) {
      v[c] = v1[c] * (1.0 - df) + v2[c] * df;
      a[c] = (v2[c] - v1[c]) / (t2 - t1);
    }
  }
  return ORC_OK;
}

/* Lienard-Wiechert fields eq:LW_E and eq:LW_B of a charge q seen along eta = r - w(t_r), with
   retarded velocity v and acceleration a. */
static int lw_fields(const double eta[3], const double v[3], const double a[3], double q, double E[3],
                     double B[3]) {
  double R = sqrt(dot3(eta, eta));
  if (!(R > 0.0)) return ORC_ERR_NUMERIC;
  double nhat[3] = {eta[0] / R, eta[1] / R, eta[2] / R};
  double vp[3] = {C_LIGHT * nhat[0] - v[0], C_LIGHT * nhat[1] - v[1], C_LIGHT * nhat[2] - v[2]};
  double eta_vp = dot3(eta, vp);
  if (!(eta_vp > 0.0)) return ORC_ERR_NUMERIC;
  double vp_x_a[3], acc[3];
  cross3(vp, a, vp_x_a);
  cross3(eta, vp_x_a, acc);
  double c2mv2 = C_LIGHT * C_LIGHT - dot3(v, v);
  double pref = q * R / (4.0 * PI * EPS0 * eta_vp * eta_vp * eta_vp);
  for (int c = 0; c < 3; c++) E[c] = pref * (c2mv2 * vp[c] + acc[c]);
  double nxE[3];
  cross3(nhat, E, nxE);
  for (int c = 0; c < 3; c++) B[c] = nxE[c] / C_LIGHT;
  return ORC_OK;
}

/* Background magnetic field (Sec. 2.6): kind 0 none, 1 uniform b, 2 centred dipole with moment
   m0 along +z about `center`: B = mu0/(4 pi) [3 (M.rhat) rhat - M] / r^3. */
static void background_b(int kind, const double* par, const double x[3], double B[3]) {
  B[0] = B[1] = B[2] = 0.0;
  if (kind == 1) {
    B[0] = par[0];
    B[1] = par[1];
    B[2] = par[2];
  } else if (kind == 2) {
    double m0 = par[3];
    double rv[3] = {x[0] - par[4], x[1] - par[5], x[2] - par[6]};
    double r = sqrt(dot3(rv, rv));
    double rhat[3] = {rv[0] / r, rv[1] / r, rv[2] / r};
    double M[3] = {0.0, 0.0, m0};
    double Mr = dot3(M, rhat);
    double k = MU0 / (4.0 * PI) / (r * r * r);
    for (int c = 0; c < 3; c++) B[c] = k * (3.0 * Mr * rhat[c] - M[c]);
  }
}

/* Higuera-Cary velocity update of Sec. 2.3 (Ripperda form) with h = q dt / (2 m). */
static void hc_kick(const double u[3], const double E[3], const double B[3], double h, double unew[3]) {
  double um[3] = {u[0] + h * E[0], u[1] + h * E[1], u[2] + h * E[2]};
  double gm = sqrt(1.0 + dot3(um, um) / (C_LIGHT * C_LIGHT));
  double tau[3] = {h * B[0], h * B[1], h * B[2]};
  double tau2 = dot3(tau, tau);
  double ustar = dot3(um, tau) / C_LIGHT;
  double sigma = gm * gm - tau2;
  double gp = sqrt((sigma + sqrt(sigma * sigma + 4.0 * (tau2 + ustar * ustar))) / 2.0);
  double tv[3] = {tau[0] / gp, tau[1] / gp, tau[2] / gp};
  double s = 1.0 / (1.0 + dot3(tv, tv));
  double umt = dot3(um, tv);
  double um_x_t[3];
  cross3(um, tv, um_x_t);
  double up[3];
  for (int c = 0; c < 3; c++) up[c] = s * (um[c] + umt * tv[c] + um_x_t[c]);
  double up_x_t[3];
  cross3(up, tv, up_x_t);
  for (int c = 0; c < 3; c++) unew[c] = up[c] + h * E[c] + up_x_t[c];
}

static double gamma_of_u(const double u[3]) { return sqrt(1.0 + dot3(u, u) / (C_LIGHT * C_LIGHT)); }

/* ------------------------------------------------------------------------------------------ */
/* Entry points (called through ctypes by the tests)                                           */
/* ------------------------------------------------------------------------------------------ */

/* physical constants, for tests that need them: c, e, m_e, eps0, mu0 */
void orc_constants(double out[5]) {
  out[0] = C_LIGHT;
  out[1] = Q_E;
  out[2] = M_ELEC;
  out[3] = EPS0;
  out[4] = MU0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* eq:LW_E / eq:LW_B for given eta, v, a and charge q. */
int orc_lw_fields(const double* eta, const double* v, const double* a, double q, double* E, double* B) {
  return lw_fields(eta, v, a, q, E, B);
}

/* Background field at x. par = {bx, by, bz, m0, cx, cy, cz}. */
void orc_background_b(int kind, const double* par, const double* x, double* B) { background_b(kind, par, x, B); }

/* One Higuera-Cary velocity update with h = q dt / (2 m). */
void orc_hc_kick(const double* u, const double* E, const double* B, double h, double* unew) {
  hc_kick(u, E, B, h, unew);
}

/* Node test P(k) of source j, for tests of the bracket. */
int orc_node_test(int64_t N, const double* T, const double* W, int64_t j, const double* r, double t, int64_t k) {
  history h = {N, T, W, NULL};
  return node_test(r, t, T[k], hist_w(&h, k, j));
}

/* Retarded state of source j seen from (r, t = T[n]) with depth D; variant & VAR_MIDPOINT selects
   eq:mid. out9 = {w[3], v[3], a[3]}; info = {branch, k1, ntest}; *tr = t_r. */
int orc_retarded_ex(int64_t N, const double* T, const double* W, const double* V, int64_t n, int64_t D, int64_t j,
                    const double* r, int variant, double* out9, double* tr, int64_t* info) {
  if (N < 1 || n < 0 || D < 1 || j < 0 || j >= N) return ORC_ERR_ARG;
  history h = {N, T, W, V};
  int64_t k0 = n - D + 1 > 0 ? n - D + 1 : 0;
  int br, nt;
  int64_t k1;
  int st = retarded_state(&h, j, r, T[n], k0, n, variant & VAR_MIDPOINT, out9, out9 + 3, out9 + 6, tr, &br, &k1,
                          &nt);
  info[0] = br;
  info[1] = k1;
  info[2] = nt;
  return st;
}

/* Bracket of every ordered pair at step n with depth D (the search of Sec. 2.2 alone): for target i at
   (W[n][i], T[n]) and source j != i, out[i * N + j] = 4 (k1 - k0) + branch with k1 the older node of the
   bracket and k0 = max(0, n - D + 1); out[i * N + i] = -1. */
int orc_bracket_table(int64_t N, const double* T, const double* W, int64_t n, int64_t D, int32_t* out) {
  if (N < 1 || n < 0 || D < 1) return ORC_ERR_ARG;
  history h = {N, T, W, NULL};
  int64_t k0 = n - D + 1 > 0 ? n - D + 1 : 0;
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t i = 0; i < N; i++) {
    const double* r = hist_w(&h, n, i);
    for (int64_t j = 0; j < N; j++) {
      if (j == i) {
        out[i * N + j] = -1;
        continue;
      }
      int64_t k1;
      int nt;
      int br = bracket(&h, j, r, T[n], k0, n, &k1, &nt);
      out[i * N + j] = (int32_t)(4 * (k1 - k0) + br);
    }
  }
  return ORC_OK;
}

/* the same with the method's own reconstruction */
int orc_retarded(int64_t N, const double* T, const double* W, const double* V, int64_t n, int64_t D, int64_t j,
                 const double* r, double* out9, double* tr, int64_t* info) {
  return orc_retarded_ex(N, T, W, V, n, D, j, r, 0, out9, tr, info);
}

/* Self fields (Sec. 2.1 superposition over j != i) at the present positions W[n][i] and time
   T[n] for the targets listed in tgt (or all N if tgt is NULL, ntgt ignored), using history
   slots k0..n, k0 = max(0, n - D + 1). q[j] = -e w[j] (wts NULL: w = 1).
   E, B: [ntgt][3]. mags (may be NULL): [ntgt][2] = {sum_j |E_ij|, sum_j |B_ij|}, the scale against
   which a per-component error of the sum is measured. stats (may be NULL): {out-of-history,
   shortcut, bisection, node tests}. variant & VAR_MIDPOINT selects eq:mid. */
int orc_self_fields_ex(int64_t N, const double* T, const double* W, const double* V, int64_t n, int64_t D,
                       const double* wts, const int64_t* tgt, int64_t ntgt, int variant, double* E, double* B,
                       double* mags, int64_t* stats) {
  if (N < 1 || n < 0 || D < 1) return ORC_ERR_ARG;
  history h = {N, T, W, V};
  int64_t k0 = n - D + 1 > 0 ? n - D + 1 : 0;
  int64_t nt_all = tgt ? ntgt : N;
  double t = T[n];
  int64_t s_oh = 0, s_sc = 0, s_bi = 0, s_nt = 0;
  int err = ORC_OK;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : s_oh, s_sc, s_bi, s_nt) reduction(| : err)
  for (int64_t ii = 0; ii < nt_all; ii++) {
    int64_t i = tgt ? tgt[ii] : ii;
    const double* r = hist_w(&h, n, i);
    csum Es[3] = {{0, 0}, {0, 0}, {0, 0}}, Bs[3] = {{0, 0}, {0, 0}, {0, 0}};
    csum Em = {0, 0}, Bm = {0, 0};
    for (int64_t j = 0; j < N; j++) {
      if (j == i) continue;
      double w[3], v[3], a[3], tr, Ej[3], Bj[3];
      int br, nt;
      int64_t k1;
      int st = retarded_state(&h, j, r, t, k0, n, variant & VAR_MIDPOINT, w, v, a, &tr, &br, &k1, &nt);
      if (st == ORC_OK) {
        double eta[3] = {r[0] - w[0], r[1] - w[1], r[2] - w[2]};
        double q = -Q_E * (wts ? wts[j] : 1.0);
        st = lw_fields(eta, v, a, q, Ej, Bj);
      }
      if (st != ORC_OK) {
        err |= st;
        continue;
      }
      if (br == BR_OUT_OF_HISTORY) s_oh++;
      else if (br == BR_SHORTCUT) s_sc++;
      else s_bi++;
      s_nt += nt;
      for (int c = 0; c < 3; c++) {
        csum_add(&Es[c], Ej[c]);
        csum_add(&Bs[c], Bj[c]);
      }
      csum_add(&Em, sqrt(dot3(Ej, Ej)));
      csum_add(&Bm, sqrt(dot3(Bj, Bj)));
    }
    for (int c = 0; c < 3; c++) {
      E[ii * 3 + c] = csum_get(&Es[c]);
      B[ii * 3 + c] = csum_get(&Bs[c]);
    }
    if (mags) {
      mags[ii * 2] = csum_get(&Em);
      mags[ii * 2 + 1] = csum_get(&Bm);
    }
  }
  if (stats) {
    stats[0] = s_oh;
    stats[1] = s_sc;
    stats[2] = s_bi;
    stats[3] = s_nt;
  }
  return err;
}

/* the same with the method's own reconstruction */
int orc_self_fields(int64_t N, const double* T, const double* W, const double* V, int64_t n, int64_t D,
                    const double* wts, const int64_t* tgt, int64_t ntgt, double* E, double* B, double* mags,
                    int64_t* stats) {
  return orc_self_fields_ex(N, T, W, V, n, D, wts, tgt, ntgt, 0, E, B, mags, stats);
}

/* Push of Sec. 2.3 for all N particles with the given self fields: x^{n+1/2} = x^n + dt/2 v^n,
   B = Bself + B_geo(x^{n+1/2}), HC kick with h = -e dt / (2 m_e), x^{n+1} = x^{n+1/2} + dt/2 v^{n+1}.
   x, u are updated in place; v receives v^{n+1}; Btot (may be NULL) receives the B used. */
int orc_push(int64_t N, double dt, double* x, double* u, const double* Eself, const double* Bself, int bkind,
             const double* bpar, double* v, double* Btot) {
  if (N < 0) return ORC_ERR_ARG;
  double h = -Q_E * dt / (2.0 * M_ELEC);
  for (int64_t i = 0; i < N; i++) {
    double* xi = x + 3 * i;
    double* ui = u + 3 * i;
    double g0 = gamma_of_u(ui);
    double xh[3];
    for (int c = 0; c < 3; c++) xh[c] = xi[c] + 0.5 * dt * (ui[c] / g0);
    double Bg[3], Bt[3];
    background_b(bkind, bpar, xh, Bg);
    for (int c = 0; c < 3; c++) Bt[c] = Bself[3 * i + c] + Bg[c];
    double un[3];
    hc_kick(ui, Eself + 3 * i, Bt, h, un);
    double g1 = gamma_of_u(un);
    for (int c = 0; c < 3; c++) {
      ui[c] = un[c];
      v[3 * i + c] = un[c] / g1;
      xi[c] = xh[c] + 0.5 * dt * v[3 * i + c];
      if (Btot) Btot[3 * i + c] = Bt[c];
    }
  }
  return ORC_OK;
}

/* One full EM-PP step from step n to n+1 (Sec. 2.1-2.3) on a history with room for slot n+1:
   self fields at (W[n], T[n]) over slots k0..n, push with the background field, then append
   slot n+1: T[n+1] = T[n] + dt, W[n+1] = x^{n+1}, V[n+1] = v^{n+1}. u holds u^n on entry and
   u^{n+1} on return. self_on = 0 drops the pair fields (E = 0, B = B_geo).
   variant: VAR_MIDPOINT reconstructs bracketed pairs by eq:mid; VAR_HALF_STEP evaluates the self
   fields at (x^{n+1/2}, t_n + dt/2) from the history with the provisional slot n+1 = (t_n + dt/2,
   x^n + (dt/2) v^n, v^n), v^n = u^n / gamma^n formed as the push's half drift forms it, over slots
   max(0, n+2-D)..n+1; the push then overwrites slot n+1.
   E, B (may be NULL) receive the fields used (B including the background). */
int orc_step_ex(int64_t N, double* T, double* W, double* V, double* u, int64_t n, int64_t D, double dt,
                const double* wts, int bkind, const double* bpar, int self_on, int variant, double* E, double* B,
                int64_t* stats) {
  double* Es = (double*)calloc((size_t)N * 3, sizeof(double));
  double* Bs = (double*)calloc((size_t)N * 3, sizeof(double));
  double* x = (double*)malloc((size_t)N * 3 * sizeof(double));
  if (!Es || !Bs || !x) {
    free(Es);
    free(Bs);
    free(x);
    return ORC_ERR_ARG;
  }
  int st = ORC_OK;
  if (self_on && (variant & VAR_HALF_STEP)) {
    double* Wp = W + (n + 1) * N * 3;
    double* Vp = V + (n + 1) * N * 3;
    const double* Wn = W + n * N * 3;
    for (int64_t i = 0; i < N; i++) {
      double g0 = gamma_of_u(u + 3 * i);
      for (int c = 0; c < 3; c++) {
        Vp[3 * i + c] = u[3 * i + c] / g0;
        Wp[3 * i + c] = Wn[3 * i + c] + 0.5 * dt * (u[3 * i + c] / g0);
      }
    }
    T[n + 1] = T[n] + 0.5 * dt;
    st = orc_self_fields_ex(N, T, W, V, n + 1, D, wts, NULL, 0, variant, Es, Bs, NULL, stats);
  } else if (self_on) {
    st = orc_self_fields_ex(N, T, W, V, n, D, wts, NULL, 0, variant, Es, Bs, NULL, stats);
  }
  memcpy(x, W + n * N * 3, (size_t)N * 3 * sizeof(double));
  if (st == ORC_OK) {
    double* vnew = V + (n + 1) * N * 3;
    orc_push(N, dt, x, u, Es, Bs, bkind, bpar, vnew, B);
    memcpy(W + (n + 1) * N * 3, x, (size_t)N * 3 * sizeof(double));
    T[n + 1] = T[n] + dt;
    if (E) memcpy(E, Es, (size_t)N * 3 * sizeof(double));
  }
  free(Es);
  free(Bs);
  free(x);
  return st;
}

/* the method's own step: present field point, linear reconstruction */
int orc_step(int64_t N, double* T, double* W, double* V, double* u, int64_t n, int64_t D, double dt,
             const double* wts, int bkind, const double* bpar, int self_on, double* E, double* B,
             int64_t* stats) {
  return orc_step_ex(N, T, W, V, u, n, D, dt, wts, bkind, bpar, self_on, 0, E, B, stats);
}

/* Interaction scale of the adaptive time step (Sec. 2.4) at step n, from the same retarded solve as the
   fields: over ordered pairs i != j whose retarded separation |eta_ij| = |x_i^n - w_j(t_r)| is at least
   eta_allow, eta_min = min |eta_ij| and v_max = max |v_i(t_n) - v_j(t_r)|, with v_i(t_n) the target's
   stored velocity at slot n and v_j(t_r) the reconstructed retarded velocity (eq:linear, eq:linear2).
   out[0] = eta_min (+inf when no pair qualifies), out[1] = v_max (0 when none). */
int orc_interaction_scale(int64_t N, const double* T, const double* W, const double* V, int64_t n, int64_t D,
                          double eta_allow, double* out) {
  if (N < 1 || n < 0 || D < 1 || !out) return ORC_ERR_ARG;
  history h = {N, T, W, V};
  int64_t k0 = n - D + 1 > 0 ? n - D + 1 : 0;
  double t = T[n];
  double emin = INFINITY, vmax = 0.0;
  int err = ORC_OK;
#pragma omp parallel for schedule(dynamic, 4) reduction(min : emin) reduction(max : vmax) reduction(| : err)
  for (int64_t i = 0; i < N; i++) {
    const double* r = hist_w(&h, n, i);
    const double* vi = hist_v(&h, n, i);
    for (int64_t j = 0; j < N; j++) {
      if (j == i) continue;
      double w[3], v[3], a[3], tr;
      int br, nt;
      int64_t k1;
      int st = retarded_state(&h, j, r, t, k0, n, 0, w, v, a, &tr, &br, &k1, &nt);
      if (st != ORC_OK) {
        err |= st;
        continue;
      }
      double eta[3] = {r[0] - w[0], r[1] - w[1], r[2] - w[2]};
      double R = sqrt(dot3(eta, eta));
      if (R < eta_allow) continue;
      double dv[3] = {vi[0] - v[0], vi[1] - v[1], vi[2] - v[2]};
      double vr = sqrt(dot3(dv, dv));
      if (R < emin) emin = R;
      if (vr > vmax) vmax = vr;
    }
  }
  out[0] = emin;
  out[1] = vmax;
  return err;
}

/* Step size of Sec. 2.4: dt = c_dt eta_min / v_max, then dt <- min(dt_max, max(dt_min, dt)); when no pair
   qualifies or v_max = 0 the interaction time is unbounded and dt = dt_max. */
double orc_adaptive_dt(double eta_min, double v_max, double c_dt, double dt_min, double dt_max) {
  double dt = (v_max > 0.0 && isfinite(eta_min)) ? c_dt * eta_min / v_max : dt_max;
  return fmin(dt_max, fmax(dt_min, dt));
}

/* orc_step with the step size of the adaptive rule of Sec. 2.4, computed from the state at step n and
   used for the push from n to n+1: par = {c_dt, eta_allow, dt_min, dt_max}; info (may be NULL) receives
   {dt, eta_min, v_max}. */
int orc_step_adaptive(int64_t N, double* T, double* W, double* V, double* u, int64_t n, int64_t D,
                      const double* par, const double* wts, int bkind, const double* bpar, double* E, double* B,
                      int64_t* stats, double* info) {
  if (!par) return ORC_ERR_ARG;
  double sc[2];
  int st = orc_interaction_scale(N, T, W, V, n, D, par[1], sc);
  if (st != ORC_OK) return st;
  double dt = orc_adaptive_dt(sc[0], sc[1], par[0], par[2], par[3]);
  if (info) {
    info[0] = dt;
    info[1] = sc[0];
    info[2] = sc[1];
  }
  return orc_step(N, T, W, V, u, n, D, dt, wts, bkind, bpar, 1, E, B, stats);
}

/* Mean kinetic energy of Sec. 2.7: E = sum_i w_i E_i / sum_i w_i with E_i = (gamma_i - 1) m_e c^2 and
   gamma_i = sqrt(1 + u_i.u_i / c^2); w = NULL means unit weights. Returns J (per electron). gamma - 1 is
   written as (u.u / c^2) / (gamma + 1), the same quantity without the cancellation of 1 from gamma. */
double orc_mean_kinetic_energy(int64_t N, const double* u, const double* w) {
  csum num = {0.0, 0.0}, den = {0.0, 0.0};
  for (int64_t i = 0; i < N; i++) {
    double wi = w ? w[i] : 1.0;
    double uu = dot3(u + 3 * i, u + 3 * i) / (C_LIGHT * C_LIGHT);
    double Ei = uu / (gamma_of_u(u + 3 * i) + 1.0) * M_ELEC * C_LIGHT * C_LIGHT;
    csum_add(&num, wi * Ei);
    csum_add(&den, wi);
  }
  return csum_get(&num) / csum_get(&den);
}

/* Switching step of Sec. 2.7 from a record of the mean energy E[0..m-1] at times T[0..m-1], with the
   backward difference r_k = (E[k] - E[k-1]) / (T[k] - T[k-1]): the criterion arms at the first k with
   |r_k| >= eps; the switch step is the first n at which |r_k| < eps held for the `hold` steps
   k = n - hold + 1 .. n, all after arming. rate[k] (may be NULL) receives r_k (rate[0] = 0). Returns -1
   when no step qualifies. */
int64_t orc_energy_switch(int64_t m, const double* T, const double* E, double eps, int64_t hold, double* rate) {
  int64_t run = 0, found = -1;
  int armed = 0;
  if (rate && m > 0) rate[0] = 0.0;
  for (int64_t n = 1; n < m; n++) {
    double r = (E[n] - E[n - 1]) / (T[n] - T[n - 1]);
    if (rate) rate[n] = r;
    if (fabs(r) >= eps) armed = 1;
    run = (armed && fabs(r) < eps) ? run + 1 : 0;
    if (found < 0 && run >= hold) found = n;
  }
  return found;
}
