/*
 * gap_oracle.c -- plain FP64 CPU oracle for one time step of the 1D radiative
 * particle-in-cell model of a pulsar polar-cap pair discharge
 * (paper: "Pair Discharges and Radio Emission from Pulsar Magnetospheres").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * execute this file: only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline leg use it.  It shares no code, header, table or constant
 * generator with the CUDA library; the two agree only because both follow
 * the paper and the readings written down beside each function.
 *
 * Style: slow and literal.  One lepton at a time, in storage order; every
 * formula is written as the paper states it in the code units below.
 *
 * Code units (Sect. 2.2, eq. ngj): length c/omega_p,co, time 1/omega_p,co,
 * momentum u = gamma*beta (m_e c), density n_co, charge e n_co, current
 * e n_co c, field m_e c omega_p / e.  Then the 1D Gauss and Ampere laws of
 * Sect. 2.2 read  dE/dx = eta - eta_co  and  dE/dt = j_m - J,  with
 * eta_co = -1 (aligned rotator: electrons fill the gap) and j_m = alpha j_co
 * = -alpha.  Charges q/m = -1 (e-), +1 (e+).
 *
 * QED scales in code units: lambda_hat = (reduced Compton wavelength)/d_e,
 * rho_hat = R_curv/d_e, r_g = lambda_C/b (from B_Q = m^2 c^3/(hbar e)).
 *   lepton (Sect. 3.1, eq. chipm with sin(psi) -> gamma r_g/R_curv):
 *     chi = gamma^2 lambda_hat/rho_hat,
 *     d tau/dt = alpha_em gamma T_syn(chi)/rho_hat   (eq. tau_syn),
 *     spectrum scale x_c = (3/2) gamma chi            (eq. xcurv).
 *   photon (Sect. 3.2, eq. tau_bw; Sect. 6.1 for the accumulated angle):
 *     sin(psi) = |sin(l/rho_hat)|, chi_x = x b sin(psi),
 *     d tau/dt = (alpha_em/lambda_hat) b sin(psi) T_BW(chi_x).
 *
 * Parity status: every function below is pinned by tests/test_oracle_pins.py
 * (closed forms, published test vectors, brute force or library routines),
 * except the full discharge run as a whole, whose plotted curves are absent
 * from the paper: "parity unpinned" for the discharge statistics; only the
 * order-of-magnitude statements of Sect. 6.3 are checked there.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_ALPHA_EM 7.2973525693e-3 /* fine-structure constant (CODATA 2018) */

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11,  */
/* "Parallel random numbers: as easy as 1, 2, 3"), written from its           */
/* published definition: 10 rounds of a two-multiplier S-box with a Weyl key  */
/* schedule.                                                                  */
/* ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                       uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += W0; k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform deviate in (0,1] for the draw keyed by (seed; id, step, channel, k).
 * Counter = (id low word, id high word, step, channel<<16 | k); key = seed.
 * 53 bits are taken from the first two output words (27 + 26 bits), so the
 * value m in [0, 2^53) maps to (m + 1) 2^-53 and -ln(U) is always finite. */
double orc_uniform(uint64_t seed, uint64_t id, uint32_t step, uint32_t channel,
                   uint32_t k) {
  uint32_t ctr[4] = {(uint32_t)id, (uint32_t)(id >> 32), step,
                     (channel << 16) | (k & 0xFFFFu)};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t o[4];
  orc_philox4x32_10(ctr, key, o);
  uint64_t m = ((uint64_t)(o[0] >> 5) << 26) | (uint64_t)(o[1] >> 6);
  return ((double)m + 1.0) * 0x1.0p-53;
}

/* SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014): golden-ratio
 * increment followed by the two xor-shift-multiply rounds. */
uint64_t orc_mix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

#define ORC_PHOTON_BIT 0x8000000000000000ull
/* Identity of a particle created by `parent` at `step` through `channel`,
 * draw k: a pure function of its inputs, so it does not depend on the order
 * in which new particles are appended.  Photons carry the top bit. */
uint64_t orc_child_id(uint64_t parent, uint32_t step, uint32_t channel,
                      uint32_t k) {
  uint64_t salt = ((uint64_t)step << 32) | ((uint64_t)channel << 16) | (k & 0xFFFFu);
  return orc_mix64(parent ^ orc_mix64(salt));
}

/* Draw channels (shared interface with the library; values only). */
enum {
  CH_INIT_U = 1, CH_TAU0 = 3, CH_EMIT_X = 4, CH_EMIT_TAU = 5,
  CH_BW_TAU = 6, CH_INJECT = 7, CH_PAIR = 8, CH_PHOTON = 9, CH_MERGE = 10,
  CH_INJECT_U = 12, CH_PAIR_E = 13, CH_INJECT_P = 14
};

/* ------------------------------------------------------------------------- */
/* QED rate functions                                                         */
/* ------------------------------------------------------------------------- */
/* Sect. 3.1: fit of the synchrotron emission function,
 * T_syn(chi) = 5/(2 sqrt3) (1 + (16 sqrt3/5) chi + 1.1 chi^2)^(-1/6). */
double orc_tsyn(double chi) {
  const double a0 = 5.0 / (2.0 * sqrt(3.0));
  const double a1 = 16.0 * sqrt(3.0) / 5.0;
  return a0 * pow(1.0 + a1 * chi + 1.1 * chi * chi, -1.0 / 6.0);
}

/* Sect. 3.2: fit of the one-photon pair-creation function,
 * T_BW(chi) = 0.23 exp(-8/(3 chi)) (1 + 0.22 chi)^(-1/3). */
double orc_tbw(double chi) {
  if (!(chi > 0.0)) return 0.0;
  return 0.23 * exp(-8.0 / (3.0 * chi)) * pow(1.0 + 0.22 * chi, -1.0 / 3.0);
}

/* Classical curvature (synchrotron-shape) photon spectrum, the reading of
 * the unspecified S(gamma,x) of Sect. 3.1: dN/dxi proportional to F(xi)/xi with
 * F(xi) = xi int_xi^inf K_{5/3}(t) dt and xi = x/x_c.  Its survival function
 *   S(xi) = P(xi' > xi) = int_xi^inf int_s^inf K_{5/3} dt ds / (5 pi/3)
 * follows from K_nu(z) = int_0^inf exp(-z cosh t) cosh(nu t) dt by doing the
 * two outer integrals in closed form:
 *   S(xi) = 3/(5 pi) int_0^inf cosh(5t/3) exp(-xi cosh t) / cosh(t)^2 dt.
 * The integrand is analytic in the strip |Im t| < pi/2, so the trapezoid rule
 * with step h converges like exp(-pi^2/h); h = 1/8 gives exp(-79). */
double orc_spec_survival(double xi) {
  if (!(xi > 0.0)) return 1.0;
  const double h = 0.125;
  double sum = 0.0;
  for (int k = 0;; ++k) {
    double t = k * h;
    double ch = cosh(t);
    double arg = xi * ch;
    if (arg > 745.0 || t > 700.0) break;
    double f = cosh(5.0 * t / 3.0) * exp(-arg) / (ch * ch);
    sum += (k == 0 ? 0.5 : 1.0) * f;
  }
  return 3.0 / (5.0 * M_PI) * h * sum;
}

/* S(xi) and dS/dxi = -3/(5 pi) int_0^inf cosh(5t/3) exp(-xi cosh t)/cosh t dt
 * by the same trapezoid rule. */
static void spec_survival_deriv(double xi, double *S, double *dS) {
  const double h = 0.125;
  double s0 = 0.0, s1 = 0.0;
  for (int k = 0;; ++k) {
    double t = k * h;
    double ch = cosh(t);
    double arg = xi * ch;
    if (arg > 745.0 || t > 700.0) break;
    double f = cosh(5.0 * t / 3.0) * exp(-arg) / ch;
    double wk = k == 0 ? 0.5 : 1.0;
    s0 += wk * f / ch;
    s1 += wk * f;
  }
  *S = 3.0 / (5.0 * M_PI) * h * s0;
  *dS = -3.0 / (5.0 * M_PI) * h * s1;
}

/* Inverse of the survival function: the xi with S(xi) = U, U in (0,1].
 * Newton iteration in y = ln(xi), safeguarded by the bracket [ln 1e-60,
 * ln 800] on which S is strictly decreasing: a step that leaves the current
 * bracket is replaced by bisection. */
double orc_spec_inverse(double U) {
  double lo = log(1e-60), hi = log(800.0);
  if (orc_spec_survival(1e-60) <= U) return 1e-60;
  double y = -log(U);
  y = y > 1e-30 ? log(y) : lo;
  if (!(y > lo && y < hi)) y = 0.5 * (lo + hi);
  for (int it = 0; it < 200; ++it) {
    double xi = exp(y), S, dS;
    spec_survival_deriv(xi, &S, &dS);
    if (S > U) lo = y; else hi = y;
    double step = (S - U) / (xi * dS);
    double yn = y - step;
    if (!(yn > lo && yn < hi)) yn = 0.5 * (lo + hi);
    double d = fabs(yn - y);
    y = yn;
    if (d < 1e-14 || hi - lo < 1e-15) break;
  }
  return exp(y);
}

/* Quantum photon spectrum of a lepton with quantum parameter chi (an option;
 * Sect. 3.1 leaves the shape S(gamma, x) unspecified and the default is the
 * classical shape above).  Photon energy fraction xi = x/gamma in (0, 1);
 * the number per unit xi is proportional to (Baier & Katkov 1968)
 *   n(xi) = (1 - xi + 1/(1 - xi)) K_{2/3}(d) - int_d^inf K_{1/3}(s) ds,
 *   d = 2 xi / (3 chi (1 - xi)),
 * whose chi -> 0 limit is int_y^inf K_{5/3}, y = x/x_c, x_c = (3/2) gamma chi.
 * With K_nu(d) = int_0^inf exp(-d cosh t) cosh(nu t) dt and
 * int_d^inf K_nu = int_0^inf exp(-d cosh t) cosh(nu t) / cosh t dt, n is one
 * integral over t (trapezoid rule, h = 1/8, to exp(-745)).  In the variable
 * s = d^(1/3) both ends of the xi range are smooth: xi = 3 chi s^3 /
 * (2 + 3 chi s^3), dxi/ds = 18 chi s^2 / (2 + 3 chi s^3)^2. */
static double qspec_density_d(double d, double xi) {
  const double B = 1.0 - xi + 1.0 / (1.0 - xi);
  const double h = 0.125;
  double sum = 0.0;
  for (int k = 0;; ++k) {
    const double t = k * h, ch = cosh(t), arg = d * ch;
    if (arg > 745.0 || t > 700.0) break;
    const double f = exp(-arg) * (B * cosh(2.0 * t / 3.0) - cosh(t / 3.0) / ch);
    sum += (k == 0 ? 0.5 : 1.0) * f;
  }
  return h * sum;
}

double orc_qspec_density(double chi, double xi) {
  if (!(xi > 0.0 && xi < 1.0)) return 0.0;
  return qspec_density_d(2.0 * xi / (3.0 * chi * (1.0 - xi)), xi);
}

/* n(xi(s)) dxi/ds */
static double qspec_ds(double chi, double s) {
  const double d = s * s * s, w = 2.0 + 3.0 * chi * d;
  const double xi = 3.0 * chi * d / w;
  if (!(s > 0.0) || xi >= 1.0) return 0.0;
  return qspec_density_d(d, xi) * 18.0 * chi * s * s / (w * w);
}

/* 8-point Gauss-Legendre nodes and weights on [-1, 1], by Newton's method on
 * the Legendre polynomial P_8 (three-term recurrence). */
static void gauss_legendre8(double *x, double *w) {
  const int n = 8;
  for (int i = 0; i < n; ++i) {
    double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

/* S_q(xi) = int_xi^1 n: composite 8-point Gauss-Legendre in s over
 * [s(xi), (d(xi) + 60)^(1/3)] (the rest is below exp(-60) of the integrand
 * at the lower end), in 160 panels whose ends s0 + (s1 - s0)(j/160)^2 crowd
 * towards s0: at large chi the spectrum's scale in s, (2/(3 chi))^(1/3),
 * is a small part of the range. */
double orc_qspec_survival(double chi, double xi) {
  double gx[8], gw[8];
  gauss_legendre8(gx, gw);
  const double d0 = xi > 0.0 ? 2.0 * xi / (3.0 * chi * (1.0 - xi)) : 0.0;
  const double s0 = cbrt(d0), s1 = cbrt(d0 + 60.0);
  const int panels = 160;
  double sum = 0.0;
  for (int pnl = 0; pnl < panels; ++pnl) {
    const double fa = (double)pnl / panels, fb = (double)(pnl + 1) / panels;
    const double a = s0 + (s1 - s0) * fa * fa, hp = (s1 - s0) * (fb * fb - fa * fa);
    double part = 0.0;
    for (int i = 0; i < 8; ++i) part += gw[i] * qspec_ds(chi, a + 0.5 * hp * (gx[i] + 1.0));
    sum += 0.5 * hp * part;
  }
  return sum;
}

/* Inverse: the xi with S_q(xi) = U S_q(0), U in (0, 1].  Newton in s,
 * safeguarded by a bracket (bisection when a step leaves it). */
double orc_qspec_inverse(double chi, double U) {
  const double target = U * orc_qspec_survival(chi, 0.0);
  double lo = 0.0, hi = cbrt(800.0);
  double s = 1.0;
  for (int it = 0; it < 200; ++it) {
    const double d = s * s * s, w = 2.0 + 3.0 * chi * d;
    const double xi = 3.0 * chi * d / w;
    const double S = orc_qspec_survival(chi, xi);
    if (S > target) lo = s; else hi = s;
    const double dS = -qspec_ds(chi, s);
    double sn = dS < 0.0 ? s - (S - target) / dS : 0.5 * (lo + hi);
    if (!(sn > lo && sn < hi)) sn = 0.5 * (lo + hi);
    const double step = fabs(sn - s);
    s = sn;
    if (step < 1e-14 * (s > 1e-300 ? s : 1.0) || hi - lo < 1e-15) break;
  }
  const double d = s * s * s;
  return 3.0 * chi * d / (2.0 + 3.0 * chi * d);
}

/* Energy split of one-photon pair creation (with qed_quantum; the default
 * gives each lepton x/2).  The electron's fraction e of the photon energy
 * has density (Baier & Katkov 1968)
 *   p(e) = (e/(1 - e) + (1 - e)/e) K_{2/3}(y) + int_y^inf K_{1/3},
 *   y = 2 / (3 chi e (1 - e)),
 * symmetric about 1/2, with (1/(pi sqrt3 chi)) int_0^1 p de the T_BW of
 * eq. tau_bw (its asymptotes 0.23 e^(-8/(3 chi)) and 0.38 chi^(-1/3)).  The
 * Bessel integrals as for the photon spectrum (trapezoid in t, h = 1/8). */
static double bw_density_y(double y, double e) {
  const double A = e / (1.0 - e) + (1.0 - e) / e;
  const double h = 0.125;
  double sum = 0.0;
  for (int k = 0;; ++k) {
    const double t = k * h, ch = cosh(t), arg = y * ch;
    if (arg > 745.0 || t > 700.0) break;
    sum += (k == 0 ? 0.5 : 1.0) * exp(-arg) * (A * cosh(2.0 * t / 3.0) + cosh(t / 3.0) / ch);
  }
  return h * sum;
}

double orc_bw_density(double chi, double e) {
  if (!(e > 0.0 && e < 1.0) || !(chi > 0.0)) return 0.0;
  return bw_density_y(2.0 / (3.0 * chi * e * (1.0 - e)), e);
}

/* p e^(y0), y0 = 8/(3 chi) the smallest y (at e = 1/2): the same ratios
 * without underflow (p itself is below the smallest double for chi < 0.0036). */
static double bw_density_scaled(double chi, double e) {
  if (!(e > 0.0 && e < 1.0)) return 0.0;
  const double y = 2.0 / (3.0 * chi * e * (1.0 - e)), y0 = 8.0 / (3.0 * chi);
  const double A = e / (1.0 - e) + (1.0 - e) / e;
  const double h = 0.125;
  double sum = 0.0;
  for (int k = 0;; ++k) {
    const double t = k * h, ch = cosh(t), arg = y * ch - y0;
    if (arg > 745.0 || t > 700.0) break;
    sum += (k == 0 ? 0.5 : 1.0) * exp(-arg) * (A * cosh(2.0 * t / 3.0) + cosh(t / 3.0) / ch);
  }
  return h * sum;
}

/* int_0^e0 p de e^(y0), e0 <= 1/2: 800 Gauss-Legendre panels uniform in tau
 * of the map e = e0 (3 tau^2 - 2 tau^3), which crowds them towards both
 * ends (the structure near e ~ 1/chi of a large chi, the narrow peak at 1/2
 * of a small one); 200 panels left 7e-10 at chi = 5e3, 800 agree with an
 * independent tanh-sinh rule to 1e-15.  Integrating from e = 0 keeps the
 * far tail (a lepton with a small share) free of cancellation. */
static double bw_tail_scaled(double chi, double e0) {
  double gx[8], gw[8];
  gauss_legendre8(gx, gw);
  const int panels = 800;
  const double ht = 1.0 / panels;
  double sum = 0.0;
  for (int pnl = 0; pnl < panels; ++pnl) {
    double part = 0.0;
    for (int i = 0; i < 8; ++i) {
      const double tau = (pnl + 0.5 * (gx[i] + 1.0)) * ht;
      const double e = e0 * tau * tau * (3.0 - 2.0 * tau);
      part += gw[i] * bw_density_scaled(chi, e) * e0 * 6.0 * tau * (1.0 - tau);
    }
    sum += 0.5 * ht * part;
  }
  return sum;
}

/* int_0^e0 p de (unscaled; zero below chi ~ 0.0036 by underflow). */
double orc_bw_tail(double chi, double e0) { return bw_tail_scaled(chi, e0) * exp(-8.0 / (3.0 * chi)); }

/* The electron's fraction for a draw U in (0, 1]: F(e) = U, F the
 * distribution of p.  With u = min(U, 1 - U) the e <= 1/2 with
 * int_0^e p = 2 u int_0^(1/2) p is found by Newton steps in e, bracketed
 * (bisection when a step leaves the bracket); U > 1/2 takes 1 - e. */
double orc_bw_split(double chi, double U) {
  if (!(chi > 0.0)) return 0.5;
  const double u = U < 0.5 ? U : 1.0 - U;
  const double target = 2.0 * u * bw_tail_scaled(chi, 0.5);
  double lo = 0.0, hi = 0.5, e = 0.5 - 0.25 * sqrt(chi / (chi + 1.0));
  for (int it = 0; it < 200; ++it) {
    const double T = bw_tail_scaled(chi, e);
    if (T < target) lo = e; else hi = e;
    const double dT = bw_density_scaled(chi, e);
    double en = dT > 0.0 ? e - (T - target) / dT : 0.5 * (lo + hi);
    if (!(en > lo && en < hi)) en = 0.5 * (lo + hi);
    const double step = fabs(en - e);
    e = en;
    if (step < 1e-16 * (e > 1e-300 ? e : 1.0) || hi - lo < 1e-16 * hi) break;
  }
  return U < 0.5 ? e : 1.0 - e;
}

/* 1D Maxwell-Juttner deviate, f(u) proportional to exp(-(gamma-1)/theta), by
 * the ratio-of-uniforms method (Kinderman & Monahan 1977): (a, v) uniform on
 * (0,1] x [-bmax, bmax], u = v/a accepted when a^2 <= f(u).  bmax =
 * sup |u| sqrt(f(u)), attained at u^2 = 2 theta gamma, gamma = theta +
 * sqrt(theta^2+1).  Draws: (id, step, channel), k = 2r, 2r+1 for round r. */
double orc_mj_draw(uint64_t seed, uint64_t id, uint32_t step, uint32_t ch, double theta, int *ok) {
  double gs = theta + sqrt(theta * theta + 1.0);
  double us = sqrt(2.0 * theta * gs);
  double bmax = us * exp(-(gs - 1.0) / (2.0 * theta));
  for (uint32_t r = 0; r < 64; ++r) {
    double a = orc_uniform(seed, id, step, ch, 2 * r);
    double v = bmax * (2.0 * orc_uniform(seed, id, step, ch, 2 * r + 1) - 1.0);
    double u = v / a;
    double gm1 = u * u / (sqrt(1.0 + u * u) + 1.0);
    if (2.0 * log(a) <= -gm1 / theta) { *ok = 1; return u; }
  }
  *ok = 0;
  return 0.0;
}

/* The loader's draw: step 0, channel CH_INIT_U. */
double orc_mj_sample(uint64_t seed, uint64_t id, double theta, int *ok) {
  return orc_mj_draw(seed, id, 0, CH_INIT_U, theta, ok);
}

/* ------------------------------------------------------------------------- */
/* PIC model                                                                  */
/* ------------------------------------------------------------------------- */
enum { ORC_BC_SURFACE = 0, ORC_BC_PERIODIC = 1 };
enum { ORC_INIT_EMPTY = 0, ORC_INIT_COLD = 1, ORC_INIT_PAIR_THERMAL = 2, ORC_INIT_GAP_PROTONS = 3 };

typedef struct {
  double alpha;      /* j_m / j_co (Sect. 2.2) */
  double b;          /* B / B_Q (Sect. 2.1) */
  double lambda_hat; /* lambda_C / d_e */
  double rho_hat;    /* R_curv / d_e */
  double rate_mult;  /* multiplies both QED rates (macro-particle rescale, Sect. 6.1) */
  double gap_length; /* H_gap in d_e; QED inhibited above it (Sect. 6.1) */
  double density;    /* initial lepton density in n_co = |eta_co|/e */
  double dx, dt;     /* grid spacing (d_e) and time step (1/omega_p) */
  double theta;      /* temperature of the thermal loader (m_e c^2) */
  double seed_amp;   /* Langmuir seed: relative density perturbation */
  int64_t nx;        /* cells */
  int64_t ppc;       /* macro-particles per cell per species at load */
  int64_t cap;       /* macro-particle cap (leptons + photons); 0 = none */
  uint64_t seed;     /* Philox key */
  int32_t gap_index; /* enters the initial ids */
  int32_t qed;       /* 0/1 */
  int32_t boundary;  /* ORC_BC_* */
  int32_t init;      /* ORC_INIT_* */
  int32_t kmax_emit; /* emission events per lepton per step (sub-cycling cap) */
  int32_t kmax_inject; /* injected electrons per step cap */
  double inject_theta; /* temperature of the injected atmosphere (m_e c^2); 0 = cold */
  int32_t filter_passes; /* binomial smoothing passes of the current per step; 0 = none */
  int32_t qed_quantum;   /* 1: quantum photon spectrum (orc_qspec_*); 0: classical */
  int32_t protons;       /* 1: the surface also supplies protons (see the injection) */
  double m_ion;          /* proton mass in m_e (0 -> 1836) */
  int32_t em;            /* 1: transverse fields E_y, E_z, B_y, B_z (see em_advance) */
  int32_t pml_cells;     /* absorbing layer below the top of a surface gap; 0 = none */
  double beta_y, beta_z; /* velocity of the co-rotating frame (App. A), across h */
  double pml_sigma;      /* peak conductivity of the layer (omega_p); 0 -> a 1e-6 reflection */
  int32_t jperp;         /* 1 (with em): transverse particle current (see jperp_deposit) */
  int32_t pad_jperp;
} orc_params;

/* heavy = 1 marks a proton (charge +1, mass m_ion; u is its momentum per
 * m_ion c, so gamma = sqrt(1 + u^2) for every species). */
typedef struct { uint64_t id; double X, u, w, tau; int32_t q; int32_t alive; int32_t heavy, pad; } orc_lepton;
/* A photon moves at c along h from X_ref, where it was at the start of step
 * n_ref (its birth step n0 for photons born in the run); X is its current
 * position, kept for export. */
typedef struct { uint64_t id; double X, x, w, tau_star, tau_acc, X_ref; int32_t dir, n0, n_ref, alive; } orc_photon;

/* Event counters and the energy ledger.  Energies are total energies (rest
 * mass included: w gamma for leptons, w x for photons) per unit area in
 * n_co m_e c^2 d_e, so that emission (gamma -> gamma - x + x), pair creation
 * (x -> 2 (x/2)) and injection (rest energy w) are exact ledger moves. */
typedef struct {
  int64_t emit_events, photons, pairs, injected, absorbed, escaped,
      photons_escaped, emit_overflow, inject_overflow, load_overflow, merged, photons_merged;
  double e_radiated, e_absorbed, e_escaped, e_photon_escaped, e_injected, work_jm;
} orc_counters;

typedef struct {
  orc_params p;
  int64_t nnode;       /* nodes holding E: nx+1 (surface) or nx (periodic) */
  double *E, *D;       /* E on nodes; D = sum q w dF, the charge through each node */
  double *Ey, *Ez;     /* em: transverse E on cells (centres c + 1/2), at half steps */
  double *By, *Bz;     /* em: transverse B on nodes, at whole steps */
  double *Jv;          /* em: dt j_vir,h on nodes for this step's Ampere */
  double *Jy, *Jz;     /* em with jperp: transverse particle current of the step on cells */
  double eta_bg;       /* Gauss background: eta_co = -1 (surface), mean load charge (periodic) */
  double w0;           /* weight of a loaded / injected macro-particle */
  orc_lepton *lep; int64_t nlep, caplep;
  orc_photon *ph;  int64_t nph, capph;
  int64_t step;
  int32_t merge_level; /* consecutive over-cap steps (bin width 0.1 * 2^level) */
  double ret_hist[64]; /* return flux (Sect. 6.5, Fig. 7): weight of e+- absorbed at
                          h < 0 per bin of ln gamma, eight bins per decade from gamma = 1 */
  orc_counters cnt;
} orc_sim;

static double Fshape(double s) { /* fraction of the unit cloud right of a node */
  double v = s + 0.5;
  return v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
}
static int64_t imod(int64_t a, int64_t n) { int64_t r = a % n; return r < 0 ? r + n : r; }

static double ion_mass(const orc_params *p) { return p->m_ion > 0.0 ? p->m_ion : 1836.0; }
static double lepton_mass(const orc_params *p, const orc_lepton *L) { return L->heavy ? ion_mass(p) : 1.0; }

static void push_lepton(orc_sim *s, orc_lepton L) {
  if (s->nlep == s->caplep) {
    s->caplep = s->caplep ? 2 * s->caplep : 1024;
    s->lep = (orc_lepton *)realloc(s->lep, (size_t)s->caplep * sizeof(orc_lepton));
  }
  s->lep[s->nlep++] = L;
}
/* bin of the return-flux tally: eight per decade of gamma from gamma = 1 */
static int return_bin(double g) {
  double b = floor(log(g) / (log(10.0) / 8.0));
  if (!(b >= 0.0)) b = 0.0;
  if (b > 63.0) b = 63.0;
  return (int)b;
}
/* bin of a spectrum over [lo, hi) in nbins uniform bins, clamped */
static int spectrum_bin(double z, int32_t nbins, double lo, double hi) {
  double b = floor((z - lo) / (hi - lo) * (double)nbins);
  if (!(b >= 0.0)) b = 0.0;
  if (b > (double)(nbins - 1)) b = (double)(nbins - 1);
  return (int)b;
}

static void push_photon(orc_sim *s, orc_photon P) {
  if (s->nph == s->capph) {
    s->capph = s->capph ? 2 * s->capph : 1024;
    s->ph = (orc_photon *)realloc(s->ph, (size_t)s->capph * sizeof(orc_photon));
  }
  s->ph[s->nph++] = P;
}

/* Initial identity of loaded particle j of cell c of species sp. */
static uint64_t load_id(int32_t gap, int32_t sp, int64_t cell, int64_t ppc, int64_t j) {
  return ((uint64_t)gap << 40) | ((uint64_t)sp << 39) | (uint64_t)(cell * ppc + j);
}
static uint64_t inject_root(int32_t gap) { return ((uint64_t)gap << 40) | (1ull << 38); }

double orc_cell_charge(const orc_sim *s, int64_t c);

/* Binomial smoothing (Sect. 6.1: the current is smoothed by a 3-point
 * binomial filter, 8 passes per step): each pass replaces a[i] by
 * (a[i-1] + 2 a[i] + a[i+1]) / 4.  Values beyond the ends, re-derived before
 * every pass: a periodic gap wraps; on a surface gap a node array is
 * mirrored evenly about its end nodes (a[-1] = a[1], a[n] = a[n-2]) and a
 * cell array oddly about the same nodes (q[-1] = -q[0], q[n] = -q[n-1]).
 * Under that pair of rules smoothing commutes with the node-to-cell
 * difference (D_c - D_{c+1}), so Gauss's law holds for the smoothed charge
 * (image charges of opposite sign behind each end). */
enum { ORC_EXT_PERIODIC = 0, ORC_EXT_NODE_EVEN = 1, ORC_EXT_CELL_ODD = 2 };
static void binomial_smooth(double *a, int64_t n, int passes, int ext) {
  double *e = (double *)malloc((size_t)(n + 2) * sizeof(double));
  for (int pass = 0; pass < passes; ++pass) {
    for (int64_t i = 0; i < n; ++i) e[i + 1] = a[i];
    if (ext == ORC_EXT_PERIODIC) { e[0] = a[n - 1]; e[n + 1] = a[0]; }
    else if (ext == ORC_EXT_NODE_EVEN) { e[0] = a[1]; e[n + 1] = a[n - 2]; }
    else { e[0] = -a[0]; e[n + 1] = -a[n - 1]; }
    for (int64_t i = 0; i < n; ++i) a[i] = 0.25 * (e[i] + 2.0 * e[i + 1] + e[i + 2]);
  }
  free(e);
}

/* Gauss's law (Sect. 2.2) on the grid: E_{c+1} - E_c = Q_c - eta_bg dx, with
 * Q_c the cloud-in-cell charge of cell c (between nodes c and c+1).  Surface:
 * E_0 = 0 (conductor).  Periodic: zero-mean E. */
void orc_solve_gauss(orc_sim *s) {
  const orc_params *p = &s->p;
  double *Q = (double *)calloc((size_t)p->nx, sizeof(double));
  for (int64_t i = 0; i < s->nlep; ++i) {
    const orc_lepton *L = &s->lep[i];
    int64_t c0 = (int64_t)floor(L->X - 0.5);
    for (int64_t c = c0; c <= c0 + 1; ++c) {
      double fr = Fshape(L->X - c) - Fshape(L->X - c - 1);
      if (fr == 0.0) continue;
      int64_t cc = c;
      if (p->boundary == ORC_BC_PERIODIC) cc = imod(c, p->nx);
      else if (c < 0 || c >= p->nx) continue;
      Q[cc] += L->q * L->w * fr;
    }
  }
  s->E[0] = 0.0;
  int64_t last = p->boundary == ORC_BC_PERIODIC ? p->nx - 1 : p->nx;
  if (p->filter_passes > 0) { /* the field of the smoothed charge */
    for (int64_t c = 0; c < p->nx; ++c) Q[c] -= s->eta_bg * p->dx;
    binomial_smooth(Q, p->nx, p->filter_passes,
                    p->boundary == ORC_BC_PERIODIC ? ORC_EXT_PERIODIC : ORC_EXT_CELL_ODD);
    for (int64_t c = 0; c < last; ++c) s->E[c + 1] = s->E[c] + Q[c];
  } else {
    for (int64_t c = 0; c < last; ++c) s->E[c + 1] = s->E[c] + Q[c] - s->eta_bg * p->dx;
  }
  if (p->boundary == ORC_BC_PERIODIC) {
    double m = 0.0;
    for (int64_t i = 0; i < s->nnode; ++i) m += s->E[i];
    m /= (double)s->nnode;
    for (int64_t i = 0; i < s->nnode; ++i) s->E[i] -= m;
  }
  free(Q);
}

orc_sim *orc_create(const orc_params *pin) {
  orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
  s->p = *pin;
  const orc_params *p = &s->p;
  s->nnode = p->boundary == ORC_BC_PERIODIC ? p->nx : p->nx + 1;
  s->E = (double *)calloc((size_t)s->nnode, sizeof(double));
  s->D = (double *)calloc((size_t)s->nnode, sizeof(double));
  if (p->em) {
    s->Ey = (double *)calloc((size_t)p->nx, sizeof(double));
    s->Ez = (double *)calloc((size_t)p->nx, sizeof(double));
    s->By = (double *)calloc((size_t)s->nnode, sizeof(double));
    s->Bz = (double *)calloc((size_t)s->nnode, sizeof(double));
    s->Jv = (double *)calloc((size_t)s->nnode, sizeof(double));
    s->Jy = (double *)calloc((size_t)p->nx, sizeof(double));
    s->Jz = (double *)calloc((size_t)p->nx, sizeof(double));
  }
  s->w0 = p->ppc > 0 ? p->density * p->dx / (double)p->ppc : 0.0;
  s->eta_bg = -1.0;
  if (p->init == ORC_INIT_COLD) {
    /* Cold electrons at rest, quiet start: X = c + (j + 1/2)/ppc. */
    for (int64_t c = 0; c < p->nx; ++c)
      for (int64_t j = 0; j < p->ppc; ++j) {
        orc_lepton L = {0};
        L.id = load_id(p->gap_index, 0, c, p->ppc, j);
        L.X = (double)c + ((double)j + 0.5) / (double)p->ppc;
        L.u = 0.0; L.w = s->w0; L.q = -1; L.alive = 1;
        L.tau = -log(orc_uniform(p->seed, L.id, 0, CH_TAU0, 0));
        push_lepton(s, L);
      }
  } else if (p->init == ORC_INIT_GAP_PROTONS) {
    /* Sect. 6.1 start: electrons at n_co everywhere and protons at the same
     * positions below H_gap (eta = 0 there, eta_co above), all at rest; the
     * Gauss solve then gives the linear ramp of E up to H_gap. */
    const double Hc = p->gap_length / p->dx;
    for (int sp = 0; sp < 2; ++sp)
      for (int64_t c = 0; c < p->nx; ++c)
        for (int64_t j = 0; j < p->ppc; ++j) {
          const double X = (double)c + ((double)j + 0.5) / (double)p->ppc;
          if (sp == 1 && !(X < Hc)) continue;
          orc_lepton L = {0};
          L.id = load_id(p->gap_index, sp, c, p->ppc, j);
          L.X = X; L.u = 0.0; L.w = s->w0; L.q = sp == 0 ? -1 : +1; L.heavy = sp; L.alive = 1;
          L.tau = -log(orc_uniform(p->seed, L.id, 0, CH_TAU0, 0));
          push_lepton(s, L);
        }
  } else if (p->init == ORC_INIT_PAIR_THERMAL) {
    /* e- and e+ at density/2 each, 1D Maxwell-Juttner momenta; the electrons
     * are displaced by (A/k) sin(k X) with k = 2 pi / nx (cells): a Langmuir
     * seed of relative density amplitude A. */
    double w = 0.5 * p->density * p->dx / (double)p->ppc;
    double k1 = 2.0 * M_PI / (double)p->nx;
    for (int sp = 0; sp < 2; ++sp)
      for (int64_t c = 0; c < p->nx; ++c)
        for (int64_t j = 0; j < p->ppc; ++j) {
          orc_lepton L = {0};
          L.id = load_id(p->gap_index, sp, c, p->ppc, j);
          double X = (double)c + ((double)j + 0.5) / (double)p->ppc;
          if (sp == 0 && p->seed_amp != 0.0) {
            X += p->seed_amp / k1 * sin(k1 * X);
            X = fmod(X, (double)p->nx);
            if (X < 0.0) X += (double)p->nx;
          }
          int ok = 1;
          L.X = X;
          L.u = p->theta > 0.0 ? orc_mj_sample(p->seed, L.id, p->theta, &ok) : 0.0;
          if (!ok) s->cnt.load_overflow++;
          L.w = w; L.q = sp == 0 ? -1 : +1; L.alive = 1;
          L.tau = -log(orc_uniform(p->seed, L.id, 0, CH_TAU0, 0));
          push_lepton(s, L);
        }
    s->w0 = w;
  }
  if (p->boundary == ORC_BC_PERIODIC) {
    double qt = 0.0;
    for (int64_t i = 0; i < s->nlep; ++i) qt += s->lep[i].q * s->lep[i].w;
    s->eta_bg = qt / ((double)p->nx * p->dx);
  }
  orc_solve_gauss(s);
  return s;
}

void orc_destroy(orc_sim *s) {
  if (!s) return;
  free(s->Ey); free(s->Ez); free(s->By); free(s->Bz); free(s->Jv); free(s->Jy); free(s->Jz);
  free(s->E); free(s->D); free(s->lep); free(s->ph); free(s);
}

/* Append a test particle (tests build tiny hand-checkable states). */
void orc_add_lepton(orc_sim *s, uint64_t id, int32_t q, double X, double u,
                    double w, double tau) {
  orc_lepton L = {0};
  L.id = id; L.q = q; L.X = X; L.u = u; L.w = w; L.tau = tau; L.alive = 1;
  push_lepton(s, L);
}
void orc_add_proton(orc_sim *s, uint64_t id, double X, double u, double w) {
  orc_lepton L = {0};
  L.id = id; L.q = +1; L.heavy = 1; L.X = X; L.u = u; L.w = w; L.tau = 1e30; L.alive = 1;
  push_lepton(s, L);
}
void orc_add_photon(orc_sim *s, uint64_t id, double X, double x, double w,
                    int32_t dir, int32_t n0, double tau_star) {
  orc_photon P = {0};
  P.id = id | ORC_PHOTON_BIT; P.X = X; P.x = x; P.w = w; P.dir = dir; P.n0 = n0;
  P.tau_star = tau_star; P.tau_acc = 0.0; P.alive = 1;
  P.X_ref = X; P.n_ref = (int32_t)s->step;
  push_photon(s, P);
}
void orc_set_eta_bg(orc_sim *s, double eta) { s->eta_bg = eta; }
void orc_binomial_smooth(double *a, int64_t n, int32_t passes, int32_t ext) { binomial_smooth(a, n, passes, ext); }
void orc_set_E(orc_sim *s, const double *E) { memcpy(s->E, E, (size_t)s->nnode * sizeof(double)); }
/* transverse fields (em = 1): E_y, E_z have nx entries, B_y, B_z nnode */
void orc_set_em(orc_sim *s, const double *Ey, const double *Ez, const double *By, const double *Bz) {
  memcpy(s->Ey, Ey, (size_t)s->p.nx * sizeof(double));
  memcpy(s->Ez, Ez, (size_t)s->p.nx * sizeof(double));
  memcpy(s->By, By, (size_t)s->nnode * sizeof(double));
  memcpy(s->Bz, Bz, (size_t)s->nnode * sizeof(double));
}
void orc_get_em(const orc_sim *s, double *Ey, double *Ez, double *By, double *Bz) {
  memcpy(Ey, s->Ey, (size_t)s->p.nx * sizeof(double));
  memcpy(Ez, s->Ez, (size_t)s->p.nx * sizeof(double));
  memcpy(By, s->By, (size_t)s->nnode * sizeof(double));
  memcpy(Bz, s->Bz, (size_t)s->nnode * sizeof(double));
}
/* the transverse particle current of the last step (em with jperp), nx cells each */
void orc_get_jperp(const orc_sim *s, double *Jy, double *Jz) {
  memcpy(Jy, s->Jy, (size_t)s->p.nx * sizeof(double));
  memcpy(Jz, s->Jz, (size_t)s->p.nx * sizeof(double));
}

/* Deposit of one move X0 -> X1 (unwrapped): the charge through node i is
 * q w [F(X1 - i) - F(X0 - i)], the change of the cloud fraction right of i
 * (first-order shape; the ZigZag-type flux of Sect. 6.1 in 1D). */
static void deposit(orc_sim *s, double q, double w, double X0, double X1) {
  const orc_params *p = &s->p;
  if (!isfinite(X0) || !isfinite(X1) || fabs(X1 - X0) > 1.0) abort(); /* never reached */
  double lo = X0 < X1 ? X0 : X1, hi = X0 < X1 ? X1 : X0;
  int64_t i0 = (int64_t)floor(lo - 0.5), i1 = (int64_t)floor(hi + 0.5);
  for (int64_t i = i0; i <= i1; ++i) {
    double dF = Fshape(X1 - (double)i) - Fshape(X0 - (double)i);
    if (dF == 0.0) continue;
    int64_t node = i;
    if (p->boundary == ORC_BC_PERIODIC) node = imod(i, p->nx);
    else if (i < 0 || i > p->nx) continue;
    s->D[node] += q * w * dF;
  }
}

/* Linear ("first-order", Sect. 6.1) gather of node E at X. */
static double gather(const orc_sim *s, double X) {
  const orc_params *p = &s->p;
  double cf = floor(X);
  double o = X - cf;
  int64_t c = (int64_t)cf, c1 = c + 1;
  if (p->boundary == ORC_BC_PERIODIC) { c = imod(c, p->nx); c1 = imod(c1, p->nx); }
  return (1.0 - o) * s->E[c] + o * s->E[c1];
}

static int in_domain(const orc_params *p, double X) {
  return X >= 0.0 && X < (double)p->nx;
}
static double wrap(const orc_params *p, double X) {
  double L = (double)p->nx;
  X = fmod(X, L);
  if (X < 0.0) X += L;
  if (X >= L) X -= L;
  return X;
}

/* Position of a photon at the start of step m (Sect. 6.1: photons move at c
 * along the field line): X_ref + dir (m - n_ref) c dt/dx, the closed form of
 * the straight-line motion (one rounding of the product, one of the sum). */
static double photon_pos(const orc_params *p, const orc_photon *P, int64_t m, double cdx) {
  double X = P->X_ref + (double)P->dir * ((double)(m - (int64_t)P->n_ref) * cdx);
  if (p->boundary == ORC_BC_PERIODIC) X = wrap(p, X);
  return X;
}

/* Weight-conserving merge (the macro-particle cap of the workloads; the paper
 * gives no scheme).  When leptons + photons exceed the cap after a step, the
 * leptons of each (species, dual cell k = floor(X + 1/2), direction, bin of
 * ln(gamma) of width 0.1 * 2^level) group with at least three members are
 * replaced by two leptons of weights W/2 at the weight-averaged offset in the
 * dual cell, with momenta from two-body kinematics on S+ = sum w (gamma + u)
 * and S- = sum w (gamma - u): rapidity of the centre eta = 0.5 ln(S+/S-),
 * invariant mass M = sqrt(S+ S-) = sum w cosh(asinh(u) - eta), CM momentum
 * p* = sqrt(M^2 - W^2)/2; this conserves weight, energy and momentum.
 * Moving the charge inside the dual cell carries charge across node k, which
 * is applied to E_k as a deposit, so Gauss's law holds.  level grows by one
 * per consecutive over-cap step (up to 7) and returns to 0 when the gap is
 * under the cap. */
typedef struct { int32_t q, dir; int64_t k; int64_t bin; uint64_t id; int64_t idx; int32_t heavy, pad; } mkey;
static int mkey_cmp(const void *a, const void *b) {
  const mkey *x = (const mkey *)a, *y = (const mkey *)b;
  if (x->heavy != y->heavy) return x->heavy < y->heavy ? -1 : 1;
  if (x->q != y->q) return x->q < y->q ? -1 : 1;
  if (x->k != y->k) return x->k < y->k ? -1 : 1;
  if (x->dir != y->dir) return x->dir < y->dir ? -1 : 1;
  if (x->bin != y->bin) return x->bin < y->bin ? -1 : 1;
  if (x->id != y->id) return x->id < y->id ? -1 : 1;
  return 0;
}
/* Photons under the cap (N -> 1, conserving w and w x), merged
 * at birth: while the gap is over its cap, the photons born in this step's
 * push (n0 = n + 1) of each (cell floor(X), direction, bin of ln x of the
 * leptons' width) group with at least two members become one photon of
 * weight W = sum w and energy x = sum w x / W at the weighted mean position
 * sum w X / W, so that the number of real photons, their energy and their
 * momentum are kept.  Members share their birth step, hence their angle to
 * the field at every later step (R10), and none has accumulated any depth
 * yet, so the new photon is a newborn photon in every respect: it draws its
 * threshold depth like one (channel BW_TAU at step n + 1) and starts its
 * accumulation at step n + 1.  Its id is the child (channel MERGE) of the
 * group's smallest id.  Older photons are left alone. */
typedef struct { int64_t k; int32_t dir, pad; int64_t bin; uint64_t id; int64_t idx; } pkey;
static int pkey_cmp(const void *a, const void *b) {
  const pkey *x = (const pkey *)a, *y = (const pkey *)b;
  if (x->k != y->k) return x->k < y->k ? -1 : 1;
  if (x->dir != y->dir) return x->dir < y->dir ? -1 : 1;
  if (x->bin != y->bin) return x->bin < y->bin ? -1 : 1;
  if (x->id != y->id) return x->id < y->id ? -1 : 1;
  return 0;
}
static void merge_photons(orc_sim *s, uint32_t n, double width) {
  const orc_params *p = &s->p;
  const int64_t np = s->nph;
  pkey *key = (pkey *)malloc((size_t)(np > 0 ? np : 1) * sizeof(pkey));
  int64_t nk = 0;
  for (int64_t i = 0; i < np; ++i) {
    const orc_photon *P = &s->ph[i];
    if (P->n0 != (int32_t)n + 1) continue;
    int64_t b = (int64_t)floor(log(P->x) / width);
    if (b < 0) b = 0;
    if (b > 255) b = 255;
    int64_t k = (int64_t)floor(P->X);
    if (p->boundary == ORC_BC_PERIODIC) k = imod(k, p->nx);
    key[nk].k = k; key[nk].dir = P->dir; key[nk].pad = 0; key[nk].bin = b; key[nk].id = P->id; key[nk].idx = i;
    ++nk;
  }
  qsort(key, (size_t)nk, sizeof(pkey), pkey_cmp);
  int64_t a = 0;
  while (a < nk) {
    int64_t e = a + 1;
    while (e < nk && key[e].k == key[a].k && key[e].dir == key[a].dir && key[e].bin == key[a].bin) ++e;
    if (e - a >= 2) {
      double W = 0.0, Wx = 0.0, WX = 0.0;
      for (int64_t j = a; j < e; ++j) {
        orc_photon *P = &s->ph[key[j].idx];
        W += P->w; Wx += P->w * P->x; WX += P->w * P->X;
        P->alive = 0;
      }
      orc_photon Q = {0};
      Q.id = orc_child_id(key[a].id, n, CH_MERGE, 0) | ORC_PHOTON_BIT;
      Q.X = WX / W; Q.X_ref = Q.X; Q.n_ref = (int32_t)n + 1;
      Q.x = Wx / W; Q.w = W; Q.dir = key[a].dir; Q.n0 = (int32_t)n + 1;
      Q.tau_star = -log(orc_uniform(p->seed, Q.id, n + 1, CH_BW_TAU, 0));
      Q.tau_acc = 0.0; Q.alive = 1;
      push_photon(s, Q);
      s->cnt.photons_merged += (e - a) - 1;
    }
    a = e;
  }
  free(key);
  int64_t m = 0;
  for (int64_t i = 0; i < s->nph; ++i) if (s->ph[i].alive) s->ph[m++] = s->ph[i];
  s->nph = m;
}

static void merge(orc_sim *s, uint32_t n) {
  const orc_params *p = &s->p;
  /* the cap bounds the pair cascade: e+- and photons count, and only e+-
   * merge; protons, which no process multiplies, are left alone */
  int64_t n_pairs = 0;
  for (int64_t i = 0; i < s->nlep; ++i) n_pairs += !s->lep[i].heavy;
  if (p->cap <= 0 || n_pairs + s->nph <= p->cap) { s->merge_level = 0; return; }
  const double width = 0.1 * (double)(1 << s->merge_level);
  if (s->merge_level < 7) s->merge_level++;
  int64_t nl = 0;
  mkey *key = (mkey *)malloc((size_t)(s->nlep > 0 ? s->nlep : 1) * sizeof(mkey));
  for (int64_t i = 0; i < s->nlep; ++i) {
    const orc_lepton *L = &s->lep[i];
    if (L->heavy) continue;
    double g = sqrt(1.0 + L->u * L->u);
    int64_t b = (int64_t)floor(log(g) / width);
    if (b < 0) b = 0;
    if (b > 255) b = 255;
    int64_t k = (int64_t)floor(L->X + 0.5);
    if (p->boundary == ORC_BC_PERIODIC) k = imod(k, p->nx);
    key[nl].q = L->q; key[nl].dir = L->u >= 0.0 ? 1 : 0; key[nl].k = k; key[nl].bin = b;
    key[nl].id = L->id; key[nl].idx = i; key[nl].heavy = L->heavy;
    ++nl;
  }
  qsort(key, (size_t)nl, sizeof(mkey), mkey_cmp);
  /* with smoothing, the re-centring flux is gathered per node, smoothed like
   * the current and then applied (Gauss's law for the smoothed charge) */
  double *mflux = p->filter_passes > 0 ? (double *)calloc((size_t)s->nnode, sizeof(double)) : NULL;
  int64_t a = 0;
  while (a < nl) {
    int64_t e = a + 1;
    while (e < nl && key[e].heavy == key[a].heavy && key[e].q == key[a].q && key[e].k == key[a].k &&
           key[e].dir == key[a].dir && key[e].bin == key[a].bin)
      ++e;
    if (e - a >= 3) {
      double W = 0.0, Sp = 0.0, Sm = 0.0, Sphi = 0.0;
      const int64_t k = key[a].k;
      for (int64_t j = a; j < e; ++j) {
        orc_lepton *L = &s->lep[key[j].idx];
        double g = sqrt(1.0 + L->u * L->u);
        double big = g + fabs(L->u);
        double gp = L->u >= 0.0 ? big : 1.0 / big, gm = L->u >= 0.0 ? 1.0 / big : big;
        double X = L->X;
        if (p->boundary == ORC_BC_PERIODIC && X + 0.5 - (double)k >= (double)p->nx) X -= (double)p->nx;
        double phi = X + 0.5 - (double)k; /* [0, 1): fraction right of node k */
        W += L->w; Sp += L->w * gp; Sm += L->w * gm; Sphi += L->w * phi;
        L->alive = 0;
      }
      const double phim = Sphi / W;
      /* charge moved across node k by re-centring: q (W phim - sum w phi) */
      const double flux = (double)key[a].q * (W * phim - Sphi);
      int64_t node = k;
      if (mflux) { if (p->boundary == ORC_BC_PERIODIC || node <= p->nx) mflux[node] += flux; }
      else if (p->boundary == ORC_BC_PERIODIC || (node > 0 && node <= p->nx)) s->E[node] -= flux;
      /* centre rapidity; the invariant mass as M = sum w cosh(a - eta) with
       * a = asinh(u) the rapidity of each member, written as W + D with
       * D = sum w 2 sinh^2((a - eta)/2) >= 0, so that M^2 - W^2 = D (2W + D)
       * carries no cancellation for nearly cold groups (sqrt(S+ S-) - W
       * would lose all digits of a small momentum spread). */
      const double eta = 0.5 * log(Sp / Sm);
      double D = 0.0;
      for (int64_t j = a; j < e; ++j) {
        const orc_lepton *L = &s->lep[key[j].idx];
        const double h = sinh(0.5 * (asinh(L->u) - eta));
        D += L->w * 2.0 * h * h;
      }
      const double M = W + D;
      const double wa = 0.5 * W, wb = W - wa;
      double q2 = D * (2.0 * W + D) * (M * M - (wa - wb) * (wa - wb));
      const double ps = q2 > 0.0 ? sqrt(q2) / (2.0 * M) : 0.0;
      const double ua = sinh(eta + asinh(ps / wa)), ub = sinh(eta - asinh(ps / wb));
      double X = (double)k + phim - 0.5;
      if (p->boundary == ORC_BC_PERIODIC && X < 0.0) X += (double)p->nx;
      for (int c = 0; c < 2; ++c) {
        orc_lepton L = {0};
        L.id = orc_child_id(key[a].id, n, CH_MERGE, (uint32_t)c) & ~ORC_PHOTON_BIT;
        L.q = key[a].q; L.heavy = key[a].heavy; L.X = X; L.u = c == 0 ? ua : ub; L.w = c == 0 ? wa : wb;
        L.alive = 1;
        L.tau = -log(orc_uniform(p->seed, L.id, n + 1, CH_TAU0, 0));
        push_lepton(s, L);
      }
      s->cnt.merged += (e - a) - 2;
    }
    a = e;
  }
  free(key);
  if (mflux) {
    binomial_smooth(mflux, s->nnode, p->filter_passes,
                    p->boundary == ORC_BC_PERIODIC ? ORC_EXT_PERIODIC : ORC_EXT_NODE_EVEN);
    for (int64_t i = p->boundary == ORC_BC_PERIODIC ? 0 : 1; i < s->nnode; ++i) s->E[i] -= mflux[i];
    free(mflux);
  }
  int64_t m = 0;
  for (int64_t i = 0; i < s->nlep; ++i) if (s->lep[i].alive) s->lep[m++] = s->lep[i];
  s->nlep = m;
  merge_photons(s, n, width);
}

/* ------------------------------------------------------------------------- */
/* Transverse fields in the co-rotating frame (App. A), in the 1D reduction:  */
/* every quantity depends on h alone, B = B_* h-hat + B_perp, and the frame   */
/* moves at beta = (0, beta_y, beta_z) across h.  In code units (c = 1, 4 pi  */
/* absorbed) App. A's Maxwell equations give, with d = d/dh,                  */
/*   dB_y/dt =  d E_z,            dB_z/dt = -d E_y,                           */
/*   dE_y/dt = -d B_z + jv_y,     dE_z/dt =  d B_y + jv_z,                    */
/*   dE_h/dt = (Ampere of Sect. 2.2) + jv_h,                                  */
/* and the virtual current jv = -{curl(beta x E) + beta x curl E              */
/*   - curl[beta x (beta x B)]} at r = R reads, with P = beta (beta.B)        */
/*   - beta^2 B_perp,                                                         */
/*   jv_h = -(beta_y d E_y + beta_z d E_z),                                   */
/*   jv_y = -beta_y d E_h - d P_z,  jv_z = -beta_z d E_h + d P_y.             */
/* The virtual charge eta_vir = eta_co + beta . curl B = eta_co               */
/*   - beta_y d B_z + beta_z d B_y enters Gauss's law (see the residual).     */
/* Particles move along B_* (the strong-field limit); with jperp they also    */
/* carry the guiding-centre transverse current of jperp_deposit, which joins  */
/* the cells' update as dE_perp/dt = ... - j_perp.                           */
/*                                                                           */
/* Grid (Yee, second order): E_y, E_z at cell centres and half steps, B_y,    */
/* B_z at nodes and whole steps; d E_h lives on cells, d E_perp on nodes.     */
/* Called after the particle push, before Ampere: E_h is still E^n, the cells */
/* go from n - 1/2 to n + 1/2 with B^n and E_h^n, then the nodes from n to    */
/* n + 1 with E_perp^{n+1/2}, and Jv = dt jv_h^{n+1/2} is left for Ampere.    */
/* Surface gap: the star (node 0) is a conductor, E_perp = 0 there (cell -1   */
/* mirrors cell 0 with a sign change); so is the top (node nx), behind an     */
/* absorbing layer of pml_cells cells (Sect. 6.1: escaping fields are damped  */
/* to vacuum).  The layer is a matched electric and magnetic conductivity     */
/* sigma(X) = sigma_max ((X - X_p)/pml_cells)^3 above X_p = nx - pml_cells    */
/* (Berenger's layer in 1D, where matching needs no field splitting), each    */
/* field advanced by the lossy-medium update F <- a F + b (rhs) with          */
/* a = (1 - sigma dt/2)/(1 + sigma dt/2), b = dt/(1 + sigma dt/2); the        */
/* default sigma_max = 4 ln(1e6)/(2 pml_cells dx) gives a continuum normal-   */
/* incidence reflection of 1e-6.  Periodic gap: both grids wrap.              */
/* ------------------------------------------------------------------------- */
static double pml_sigma_max(const orc_params *p) {
  if (p->pml_sigma > 0.0) return p->pml_sigma;
  return 4.0 * log(1e6) / (2.0 * (double)p->pml_cells * p->dx);
}
static double pml_sigma_at(const orc_params *p, double X) {
  if (p->boundary == ORC_BC_PERIODIC || p->pml_cells <= 0) return 0.0;
  const double Xp = (double)(p->nx - p->pml_cells);
  if (!(X > Xp)) return 0.0;
  const double f = (X - Xp) / (double)p->pml_cells;
  return pml_sigma_max(p) * f * f * f;
}
/* transverse E of cell c, with the conductor images of a surface gap */
static double cell_field(const orc_sim *s, const double *F, int64_t c) {
  const int64_t nx = s->p.nx;
  if (s->p.boundary == ORC_BC_PERIODIC) return F[imod(c, nx)];
  if (c < 0) return -F[-1 - c];
  if (c >= nx) return -F[2 * nx - 1 - c];
  return F[c];
}
/* Transverse particle current (App. A; Sect. 6.6, Fig. 8), in the guiding-   */
/* centre limit of the strong field: with B = B_* h-hat + B_perp, B_* =       */
/* b / lambda_hat in code units (omega_B / omega_p), a particle slides along  */
/* its field line at beta_h and drifts at E x B / B^2, which to first order   */
/* in B_perp / B_* and E_perp / B_* gives, for any mass,                      */
/*   v_y = (beta_h B_y + E_z) / B_*,   v_z = (beta_h B_z - E_y) / B_*.        */
/* The current of step n, which advances E_perp from n - 1/2 to n + 1/2, is   */
/* deposited from the start-of-step position X^n with the step's velocity     */
/* beta_h = u / gamma after the kick and emissions, E_perp^{n-1/2} taken      */
/* linearly between cell centres (conductor images at a surface gap's ends)   */
/* and B_perp^n linearly between nodes, both at X^n: j_perp(c) += q w v_perp  */
/* S_c / dx, S_c the overlap of the unit top-hat cloud [X - 1/2, X + 1/2]     */
/* with cell c.  A cloud's part outside a surface gap (below the star, above  */
/* the top conductor) carries no current.  The particle state keeps u_h only: */
/* the drift's energy, O((E_perp / B_*)^2), is not tracked.                   */
static void jperp_deposit(orc_sim *s, double q, double w, double X, double u) {
  const orc_params *p = &s->p;
  const int64_t nx = p->nx;
  const double Bs = p->b / p->lambda_hat;
  const double bh = u / sqrt(1.0 + u * u);
  /* cell centres c + 1/2: the cloud covers c0 = floor(X - 1/2) and c0 + 1 */
  const double sc = X - 0.5;
  const int64_t c0 = (int64_t)floor(sc);
  const double tc = sc - (double)c0;
  const double Ey = (1.0 - tc) * cell_field(s, s->Ey, c0) + tc * cell_field(s, s->Ey, c0 + 1);
  const double Ez = (1.0 - tc) * cell_field(s, s->Ez, c0) + tc * cell_field(s, s->Ez, c0 + 1);
  /* nodes i0 = floor(X) and i0 + 1 */
  int64_t i0 = (int64_t)floor(X), i1 = i0 + 1;
  const double tn = X - (double)i0;
  if (p->boundary == ORC_BC_PERIODIC) { i0 = imod(i0, nx); i1 = imod(i1, nx); }
  const double By = (1.0 - tn) * s->By[i0] + tn * s->By[i1];
  const double Bz = (1.0 - tn) * s->Bz[i0] + tn * s->Bz[i1];
  const double vy = (bh * By + Ez) / Bs, vz = (bh * Bz - Ey) / Bs;
  const double S[2] = {1.0 - tc, tc};
  for (int j = 0; j < 2; ++j) {
    int64_t c = c0 + j;
    if (p->boundary == ORC_BC_PERIODIC) c = imod(c, nx);
    else if (c < 0 || c >= nx) continue;
    s->Jy[c] += q * w * vy * S[j] / p->dx;
    s->Jz[c] += q * w * vz * S[j] / p->dx;
  }
}

static void em_advance(orc_sim *s) {
  const orc_params *p = &s->p;
  const double dt = p->dt, dx = p->dx, by = p->beta_y, bz = p->beta_z;
  const double b2 = by * by + bz * bz;
  const int64_t nx = p->nx;
  for (int64_t c = 0; c < nx; ++c) {
    const int64_t i0 = c, i1 = p->boundary == ORC_BC_PERIODIC ? imod(c + 1, nx) : c + 1;
    const double dEh = (s->E[i1] - s->E[i0]) / dx;
    const double bB0 = by * s->By[i0] + bz * s->Bz[i0], bB1 = by * s->By[i1] + bz * s->Bz[i1];
    const double Py0 = by * bB0 - b2 * s->By[i0], Py1 = by * bB1 - b2 * s->By[i1];
    const double Pz0 = bz * bB0 - b2 * s->Bz[i0], Pz1 = bz * bB1 - b2 * s->Bz[i1];
    const double jvy = -by * dEh - (Pz1 - Pz0) / dx;
    const double jvz = -bz * dEh + (Py1 - Py0) / dx;
    double ry = -(s->Bz[i1] - s->Bz[i0]) / dx + jvy;
    double rz = (s->By[i1] - s->By[i0]) / dx + jvz;
    if (p->jperp) {
      ry -= s->Jy[c];
      rz -= s->Jz[c];
    }
    const double sg = pml_sigma_at(p, (double)c + 0.5);
    const double a = (1.0 - 0.5 * sg * dt) / (1.0 + 0.5 * sg * dt), b = dt / (1.0 + 0.5 * sg * dt);
    s->Ey[c] = a * s->Ey[c] + b * ry;
    s->Ez[c] = a * s->Ez[c] + b * rz;
  }
  for (int64_t i = 0; i < s->nnode; ++i) {
    const double dEy = (cell_field(s, s->Ey, i) - cell_field(s, s->Ey, i - 1)) / dx;
    const double dEz = (cell_field(s, s->Ez, i) - cell_field(s, s->Ez, i - 1)) / dx;
    const double sg = pml_sigma_at(p, (double)i);
    const double a = (1.0 - 0.5 * sg * dt) / (1.0 + 0.5 * sg * dt), b = dt / (1.0 + 0.5 * sg * dt);
    s->Bz[i] = a * s->Bz[i] - b * dEy;
    s->By[i] = a * s->By[i] + b * dEz;
    s->Jv[i] = -dt * (by * dEy + bz * dEz);
  }
}

/* One time step n -> n+1.  Order (Sect. 6.1 PIC cycle, reduced to 1D along B):
 *  1. every lepton: gather E^n, kick (Sect. 4: du/dt = (q/m) E), curvature
 *     emission by optical-depth sub-cycling (eq. tau_syn, Sect. 6.1 MC
 *     sub-cycling), drift, charge-conserving deposit, boundaries;
 *  2. every photon alive at step start: propagate at c, accumulate the
 *     Breit-Wheeler optical depth (eq. tau_bw) at the accumulated angle of
 *     Sect. 6.1, convert into an e-e+ pair when it reaches its threshold;
 *  3. with em, the transverse fields (em_advance); Ampere (Sect. 2.2):
 *     E_i += dt j_m - D_i (+ dt jv_h with em), E_0 = 0 at the surface (D
 *     smoothed by filter_passes binomial passes first, when asked);
 *  4. surface injection of electrons, and with protons of protons
 *     (Sect. 2.3 / 6.1 atmosphere);
 *  5. merge when leptons + photons exceed the cap (see merge()). */
void orc_step(orc_sim *s) {
  const orc_params *p = &s->p;
  const double dt = p->dt, dx = p->dx, cdx = dt / dx;
  const double Hc = p->gap_length / dx;   /* gap height in cells */
  const double jm = -p->alpha;            /* j_m = alpha j_co, j_co = -1 */
  const uint32_t n = (uint32_t)s->step;
  memset(s->D, 0, (size_t)s->nnode * sizeof(double));
  if (p->em) {
    memset(s->Jy, 0, (size_t)p->nx * sizeof(double));
    memset(s->Jz, 0, (size_t)p->nx * sizeof(double));
  }
  int64_t nph_old = s->nph;

  for (int64_t ip = 0; ip < s->nlep; ++ip) {
    orc_lepton *L = &s->lep[ip];
    double X0 = L->X, u = L->u;
    /* a1-a2: gather and kick */
    if (L->heavy) u += (double)L->q * gather(s, X0) * dt / ion_mass(p);
    else u += (double)L->q * gather(s, X0) * dt;
    /* a3: emission sub-cycling within this step */
    orc_photon born[64];
    int nborn = 0;
    if (p->qed && X0 < Hc && !L->heavy) {
      double trem = dt, tau = L->tau;
      int k = 0;
      for (;;) {
        double g = sqrt(1.0 + u * u);
        double chi = g * g * p->lambda_hat / p->rho_hat;
        double r = p->rate_mult * ORC_ALPHA_EM * g * orc_tsyn(chi) / p->rho_hat;
        if (!(r > 0.0)) break;
        if (tau > r * trem) { tau -= r * trem; break; }
        trem -= tau / r;
        double U = orc_uniform(p->seed, L->id, n, CH_EMIT_X, (uint32_t)k);
        /* photon energy: classical shape (x = xi x_c), or with qed_quantum the
         * quantum shape (x = xi gamma, xi the energy fraction) */
        double x = p->qed_quantum ? orc_qspec_inverse(chi, U) * g : orc_spec_inverse(U) * 1.5 * g * chi;
        double gm1 = u * u / (g + 1.0);
        double dir = u >= 0.0 ? 1.0 : -1.0;
        if (x >= gm1) {
          /* the photon takes the whole kinetic energy: the lepton is at rest
           * (gamma - x would otherwise carry only rounding noise) */
          x = gm1;
          u = 0.0;
        } else {
          double g2 = g - x;
          double pp = (g2 - 1.0) * (g2 + 1.0);
          u = pp > 0.0 ? dir * sqrt(pp) : 0.0;
        }
        s->cnt.emit_events++;
        if (x >= 2.0) {
          orc_photon P = {0};
          P.id = orc_child_id(L->id, n, CH_PHOTON, (uint32_t)k) | ORC_PHOTON_BIT;
          P.x = x; P.w = L->w; P.dir = (int32_t)dir; P.n0 = (int32_t)n + 1;
          P.tau_star = -log(orc_uniform(p->seed, P.id, n + 1, CH_BW_TAU, 0));
          P.tau_acc = 0.0; P.alive = 1;
          born[nborn++] = P;
        } else {
          s->cnt.e_radiated += L->w * x;
        }
        tau = -log(orc_uniform(p->seed, L->id, n, CH_EMIT_TAU, (uint32_t)k));
        if (++k >= p->kmax_emit) { s->cnt.emit_overflow++; break; }
      }
      L->tau = tau;
    }
    /* with em and jperp: the transverse current of the step at X^n */
    if (p->em && p->jperp) jperp_deposit(s, (double)L->q, L->w, X0, u);
    /* a4: drift; a8: deposit of the move */
    double g = sqrt(1.0 + u * u);
    double X1 = X0 + u / g * cdx;
    deposit(s, (double)L->q, L->w, X0, X1);
    L->u = u;
    /* a7: boundaries */
    if (p->boundary == ORC_BC_PERIODIC) {
      X1 = wrap(p, X1);
    } else if (X1 < 0.0) {
      L->alive = 0; s->cnt.absorbed++; s->cnt.e_absorbed += L->w * g * lepton_mass(p, L);
      if (!L->heavy) s->ret_hist[return_bin(g)] += L->w;
    } else if (X1 >= (double)p->nx) {
      L->alive = 0; s->cnt.escaped++; s->cnt.e_escaped += L->w * g * lepton_mass(p, L);
    }
    L->X = X1;
    for (int b = 0; b < nborn; ++b) {
      born[b].X = X1;
      born[b].X_ref = X1;
      born[b].n_ref = born[b].n0;
      if (p->boundary != ORC_BC_PERIODIC && !in_domain(p, X1)) {
        s->cnt.photons_escaped++; s->cnt.e_photon_escaped += born[b].w * born[b].x;
        continue;
      }
      s->cnt.photons++;
      push_photon(s, born[b]);
    }
  }

  /* a5: photons alive at the start of the step */
  for (int64_t ip = 0; ip < nph_old; ++ip) {
    orc_photon *P = &s->ph[ip];
    if (!P->alive) continue;
    if (photon_pos(p, P, n, cdx) < Hc) {
      double lmid = ((double)n - (double)P->n0 + 0.5) * dt;
      double sp = fabs(sin(lmid / p->rho_hat));
      double chi = P->x * p->b * sp;
      P->tau_acc += dt * p->rate_mult * ORC_ALPHA_EM / p->lambda_hat * p->b * sp * orc_tbw(chi);
    }
    double X1 = photon_pos(p, P, n + 1, cdx);
    P->X = X1;
    if (p->boundary != ORC_BC_PERIODIC && !in_domain(p, X1)) {
      P->alive = 0; s->cnt.photons_escaped++; s->cnt.e_photon_escaped += P->w * P->x;
      continue;
    }
    if (P->tau_acc >= P->tau_star) {
      P->alive = 0;
      /* energies: x/2 each, or with qed_quantum the electron takes e x with e
       * from the differential rate at this step's chi (both at least 1) */
      double ge = 0.5 * P->x;
      if (p->qed_quantum) {
        const double lmid = ((double)n - (double)P->n0 + 0.5) * dt;
        const double chi = P->x * p->b * fabs(sin(lmid / p->rho_hat));
        double e = orc_bw_split(chi, orc_uniform(p->seed, P->id, n, CH_PAIR_E, 0));
        /* a share below one rest mass is raised to it, on the energies
         * themselves: (1/x) x can round to just below 1 */
        ge = e * P->x;
        if (ge < 1.0) ge = 1.0;
        if (P->x - ge < 1.0) ge = P->x - 1.0;
      }
      for (int k = 0; k < 2; ++k) {
        const double gk = k == 0 ? ge : P->x - ge;
        const double pk = (gk - 1.0) * (gk + 1.0);
        const double up = (double)P->dir * sqrt(pk > 0.0 ? pk : 0.0);
        orc_lepton L = {0};
        L.id = orc_child_id(P->id, n, CH_PAIR, (uint32_t)k) & ~ORC_PHOTON_BIT;
        L.q = k == 0 ? -1 : +1;
        L.X = X1; L.u = up; L.w = P->w; L.alive = 1;
        L.tau = -log(orc_uniform(p->seed, L.id, n + 1, CH_TAU0, 0));
        push_lepton(s, L);
      }
      s->cnt.pairs++;
    }
  }

  /* compaction (storage order of the survivors is kept) */
  int64_t m = 0;
  for (int64_t i = 0; i < s->nlep; ++i) if (s->lep[i].alive) s->lep[m++] = s->lep[i];
  s->nlep = m;
  m = 0;
  for (int64_t i = 0; i < s->nph; ++i) if (s->ph[i].alive) s->ph[m++] = s->ph[i];
  s->nph = m;

  /* a9: Ampere, with the work of the imposed current on the field; the
   * current is smoothed first when filter_passes > 0 */
  if (p->filter_passes > 0)
    binomial_smooth(s->D, s->nnode, p->filter_passes,
                    p->boundary == ORC_BC_PERIODIC ? ORC_EXT_PERIODIC : ORC_EXT_NODE_EVEN);
  if (p->em) em_advance(s);
  int64_t i0 = p->boundary == ORC_BC_PERIODIC ? 0 : 1;
  double work = 0.0;
  for (int64_t i = i0; i < s->nnode; ++i) {
    double En = s->E[i];
    s->E[i] = En + (dt * jm - s->D[i]);
    if (p->em) s->E[i] += s->Jv[i];
    work += 0.5 * (En + s->E[i]);
  }
  if (p->boundary != ORC_BC_PERIODIC) s->E[0] = 0.0;
  s->cnt.work_jm += dt * dx * jm * work;

  /* a7: surface injection.  Cell 0 must hold the co-rotation charge
   * eta_co dx = -dx; while its deficit exceeds half a macro-particle charge,
   * add an electron at X = U/2 in (0, 1/2] (cloud inside cell 0 and the
   * conductor only, so no other cell's Gauss balance changes).  The
   * atmosphere has a temperature (Sect. 6.1): with inject_theta > 0 the
   * electron's momentum is |u| of a 1D Maxwell-Juttner draw at that
   * temperature, pointing into the gap (the half of the distribution that
   * leaves the surface); otherwise it starts at rest. */
  if (p->boundary == ORC_BC_SURFACE && s->w0 > 0.0) {
    double Q0 = orc_cell_charge(s, 0);
    double deficit = Q0 - (-1.0) * dx;
    int j = 0;
    while (deficit > 0.5 * s->w0) {
      if (j >= p->kmax_inject) { s->cnt.inject_overflow++; break; }
      orc_lepton L = {0};
      L.id = orc_child_id(inject_root(p->gap_index), n, CH_INJECT, (uint32_t)j) & ~ORC_PHOTON_BIT;
      double o = 0.5 * orc_uniform(p->seed, L.id, n + 1, CH_INJECT, 0);
      L.q = -1; L.X = o; L.u = 0.0; L.w = s->w0; L.alive = 1;
      if (p->inject_theta > 0.0) {
        int ok = 1;
        L.u = fabs(orc_mj_draw(p->seed, L.id, (uint32_t)(n + 1), CH_INJECT_U, p->inject_theta, &ok));
        if (!ok) s->cnt.load_overflow++;
      }
      L.tau = -log(orc_uniform(p->seed, L.id, n + 1, CH_TAU0, 0));
      push_lepton(s, L);
      deficit -= s->w0 * (o + 0.5);
      s->cnt.injected++;
      s->cnt.e_injected += s->w0 * sqrt(1.0 + L.u * L.u); /* total energy w gamma */
      ++j;
    }
    /* with protons, an excess of negative charge is screened the other way:
     * while it exceeds half a macro-particle charge a proton is added (its
     * own channel; the temperature in its rest-mass units is theta/m_ion) */
    for (int jp = 0; p->protons && deficit < -0.5 * s->w0; ++jp) {
      if (jp >= p->kmax_inject) { s->cnt.inject_overflow++; break; }
      orc_lepton L = {0};
      L.id = orc_child_id(inject_root(p->gap_index), n, CH_INJECT_P, (uint32_t)jp) & ~ORC_PHOTON_BIT;
      double o = 0.5 * orc_uniform(p->seed, L.id, n + 1, CH_INJECT_P, 0);
      L.q = +1; L.heavy = 1; L.X = o; L.u = 0.0; L.w = s->w0; L.tau = 1e30; L.alive = 1;
      if (p->inject_theta > 0.0) {
        int ok = 1;
        L.u = fabs(orc_mj_draw(p->seed, L.id, (uint32_t)(n + 1), CH_INJECT_U, p->inject_theta / ion_mass(p), &ok));
        if (!ok) s->cnt.load_overflow++;
      }
      push_lepton(s, L);
      deficit += s->w0 * (o + 0.5);
      s->cnt.injected++;
      s->cnt.e_injected += s->w0 * ion_mass(p) * sqrt(1.0 + L.u * L.u);
    }
  }
  merge(s, n);
  s->step++;
}

void orc_run(orc_sim *s, int64_t nsteps) { for (int64_t i = 0; i < nsteps; ++i) orc_step(s); }

/* Cloud-in-cell charge of cell c (between nodes c and c+1). */
double orc_cell_charge(const orc_sim *s, int64_t c) {
  double Q = 0.0;
  for (int64_t i = 0; i < s->nlep; ++i) {
    const orc_lepton *L = &s->lep[i];
    double X = L->X;
    if (s->p.boundary == ORC_BC_PERIODIC) {
      /* nearest periodic image of the cell */
      double L0 = (double)s->p.nx;
      double d = X - (double)c;
      d -= L0 * floor(d / L0 + 0.5);
      X = (double)c + d;
    }
    double fr = Fshape(X - (double)c) - Fshape(X - (double)c - 1.0);
    Q += L->q * L->w * fr;
  }
  return Q;
}

/* Largest |Gauss residual| (E_{c+1} - E_c) - (Q_c - eta_bg dx) over the cells
 * that touch no boundary (surface: 1..nx-2; periodic: all).  With smoothing
 * the charge term is smoothed like the current, and on a surface gap the
 * cells within filter_passes of a boundary cell are left out too (charge
 * that enters or leaves through an end without a flux spreads that far). */
double orc_gauss_residual(const orc_sim *s, double *max_abs_E) {
  const orc_params *p = &s->p;
  double *Q = (double *)calloc((size_t)p->nx, sizeof(double));
  for (int64_t i = 0; i < s->nlep; ++i) {
    const orc_lepton *L = &s->lep[i];
    int64_t c0 = (int64_t)floor(L->X - 0.5);
    for (int64_t c = c0; c <= c0 + 1; ++c) {
      double fr = Fshape(L->X - c) - Fshape(L->X - c - 1);
      if (fr == 0.0) continue;
      int64_t cc = c;
      if (p->boundary == ORC_BC_PERIODIC) cc = imod(c, p->nx);
      else if (c < 0 || c >= p->nx) continue;
      Q[cc] += L->q * L->w * fr;
    }
  }
  double r = 0.0, em = 0.0;
  const int P = p->filter_passes;
  for (int64_t c = 0; c < p->nx; ++c) Q[c] -= s->eta_bg * p->dx;
  if (P > 0) binomial_smooth(Q, p->nx, P, p->boundary == ORC_BC_PERIODIC ? ORC_EXT_PERIODIC : ORC_EXT_CELL_ODD);
  int64_t c_lo = p->boundary == ORC_BC_PERIODIC ? 0 : 1 + P;
  int64_t c_hi = p->boundary == ORC_BC_PERIODIC ? p->nx - 1 : p->nx - 2 - P;
  /* with transverse fields: the virtual charge -beta_y dB_z + beta_z dB_y
   * joins eta_co; the layer's damping of B breaks that balance inside it */
  if (p->em && p->boundary != ORC_BC_PERIODIC && p->pml_cells > 0 && c_hi > p->nx - p->pml_cells - 1)
    c_hi = p->nx - p->pml_cells - 1;
  for (int64_t c = c_lo; c <= c_hi; ++c) {
    int64_t c1 = p->boundary == ORC_BC_PERIODIC ? imod(c + 1, p->nx) : c + 1;
    double res = (s->E[c1] - s->E[c]) - Q[c];
    if (p->em) res -= p->beta_y * (s->Bz[c1] - s->Bz[c]) - p->beta_z * (s->By[c1] - s->By[c]);
    if (fabs(res) > r) r = fabs(res);
  }
  for (int64_t i = 0; i < s->nnode; ++i) if (fabs(s->E[i]) > em) em = fabs(s->E[i]);
  if (max_abs_E) *max_abs_E = em;
  free(Q);
  return r;
}

/* Per-cell moments for the diagnostics of Sect. 6.2 (Fig. 5): cloud-in-cell
 * density of each species split by direction (u >= 0 up, u < 0 down), the
 * weighted sums of gamma^-3 and of the weight (for <gamma^-3>), and the
 * charge.  Arrays have nx entries; dens is [2 species][2 dirs][nx]. */
/* Return flux (Sect. 6.5): the e+- absorbed at h < 0 since the start, as
 * weight per bin of ln gamma: bin i holds 10^(i/8) <= gamma < 10^((i+1)/8),
 * the last bin everything above. */
void orc_return_spectrum(const orc_sim *s, double *out) {
  for (int i = 0; i < 64; ++i) out[i] = s->ret_hist[i];
}

/* Spectra of the gap (Sect. 6.4, Fig. 6: the pair plasma's momentum
 * distribution over h in [0, H_gap] and the photon energy spectrum): the
 * weight of the electrons (lep[0..nbins)), the positrons (lep[nbins..2 nbins))
 * and the photons (ph) in the gap, per bin of ln p (p = |u| = gamma beta) or
 * ln x, nbins uniform bins over [lo, hi); values below lo (p = 0 included)
 * count in the first bin, values at or above hi in the last. */
void orc_spectra(const orc_sim *s, int32_t nbins, double lo, double hi, double *lep, double *ph) {
  const orc_params *p = &s->p;
  const double Hc = p->gap_length / p->dx;
  for (int i = 0; i < 2 * nbins; ++i) lep[i] = 0.0;
  for (int i = 0; i < nbins; ++i) ph[i] = 0.0;
  for (int64_t i = 0; i < s->nlep; ++i) {
    const orc_lepton *L = &s->lep[i];
    if (L->heavy || !(L->X < Hc)) continue;
    const int sp = L->q < 0 ? 0 : 1;
    lep[sp * nbins + spectrum_bin(log(fabs(L->u)), nbins, lo, hi)] += L->w;
  }
  for (int64_t i = 0; i < s->nph; ++i) {
    const orc_photon *P = &s->ph[i];
    if (!(P->X < Hc)) continue;
    ph[spectrum_bin(log(P->x), nbins, lo, hi)] += P->w;
  }
}

void orc_moments(const orc_sim *s, double *dens, double *g3w, double *wsum, double *charge) {
  const orc_params *p = &s->p;
  int64_t nx = p->nx;
  memset(dens, 0, (size_t)(4 * nx) * sizeof(double));
  memset(g3w, 0, (size_t)nx * sizeof(double));
  memset(wsum, 0, (size_t)nx * sizeof(double));
  memset(charge, 0, (size_t)nx * sizeof(double));
  for (int64_t i = 0; i < s->nlep; ++i) {
    const orc_lepton *L = &s->lep[i];
    if (L->heavy) continue;  /* the pair plasma's moments: protons are left out */
    double g = sqrt(1.0 + L->u * L->u);
    int sp = L->q < 0 ? 0 : 1, dr = L->u >= 0.0 ? 0 : 1;
    int64_t c0 = (int64_t)floor(L->X - 0.5);
    for (int64_t c = c0; c <= c0 + 1; ++c) {
      double fr = Fshape(L->X - c) - Fshape(L->X - c - 1);
      if (fr == 0.0) continue;
      int64_t cc = c;
      if (p->boundary == ORC_BC_PERIODIC) cc = imod(c, nx);
      else if (c < 0 || c >= nx) continue;
      dens[(sp * 2 + dr) * nx + cc] += L->w * fr / p->dx;
      g3w[cc] += L->w * fr / (g * g * g);
      wsum[cc] += L->w * fr;
      charge[cc] += L->q * L->w * fr;
    }
  }
}

/* Accessors used by the Python wrapper. */
int64_t orc_nlep(const orc_sim *s) { return s->nlep; }
int64_t orc_nph(const orc_sim *s) { return s->nph; }
int64_t orc_nnode(const orc_sim *s) { return s->nnode; }
int64_t orc_stepno(const orc_sim *s) { return s->step; }
double orc_w0(const orc_sim *s) { return s->w0; }
double orc_eta_bg(const orc_sim *s) { return s->eta_bg; }
void orc_get_E(const orc_sim *s, double *E) { memcpy(E, s->E, (size_t)s->nnode * sizeof(double)); }
void orc_get_counters(const orc_sim *s, orc_counters *c) { *c = s->cnt; }
void orc_get_leptons(const orc_sim *s, uint64_t *id, int32_t *q, double *X, double *u,
                     double *w, double *tau) {
  for (int64_t i = 0; i < s->nlep; ++i) {
    id[i] = s->lep[i].id; q[i] = s->lep[i].q; X[i] = s->lep[i].X; u[i] = s->lep[i].u;
    w[i] = s->lep[i].w; tau[i] = s->lep[i].tau;
  }
}
void orc_get_lepton_heavy(const orc_sim *s, int32_t *heavy) {
  for (int64_t i = 0; i < s->nlep; ++i) heavy[i] = s->lep[i].heavy;
}
void orc_get_photons(const orc_sim *s, uint64_t *id, double *X, double *x, double *w,
                     double *tau_star, double *tau_acc, int32_t *dir, int32_t *n0) {
  for (int64_t i = 0; i < s->nph; ++i) {
    id[i] = s->ph[i].id; X[i] = s->ph[i].X; x[i] = s->ph[i].x; w[i] = s->ph[i].w;
    tau_star[i] = s->ph[i].tau_star; tau_acc[i] = s->ph[i].tau_acc;
    dir[i] = s->ph[i].dir; n0[i] = s->ph[i].n0;
  }
}
