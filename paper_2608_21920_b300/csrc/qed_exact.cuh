// qed_exact.cuh -- exact FP64 evaluation of the quantum photon spectrum's
// survival function and of the pair split's distribution (qed_quantum), with
// which the FP64 state refines the table inverses by Newton steps: its photon
// energies and pair shares are those of the definitions (R26, R27), not of
// the tables, to ~1e-14.  The FP32 state keeps the tables.
//
// Photon spectrum (Baier & Katkov; Sect. 3.1 leaves the shape open): with
// d = 2 xi / (3 chi (1 - xi)),
//   n(xi) = (1 - xi + 1/(1 - xi)) K_2/3(d) - int_d^inf K_1/3,
//   K_nu(d) = int_0^inf exp(-d cosh t) cosh(nu t) dt,
//   int_d^inf K_nu = int_0^inf exp(-d cosh t) cosh(nu t) / cosh t dt,
// and the survival S(xi) = int_xi^1 n.  Writing xi through w = 2 + 3 chi d
// (1 - xi = 2/w, dxi = 6 chi dd / w^2, 1 - xi + 1/(1 - xi) = 2/w + w/2), the
// integral over xi of each t-term is an exponential integral,
//   int_d0^inf exp(-c d) w^-m dd = exp(-c d0) w0^(1-m) Ehat_m(c w0/(3 chi)) / (3 chi),
// with c = cosh t, w0 = 2 + 3 chi d0 and Ehat_m(x) = e^x E_m(x), so that
//   S(xi) = 2 int_0^inf exp(-c d0) [cosh(2t/3) (2 Ehat_3/w0^2 + Ehat_1/2)
//                                   - cosh(t/3) Ehat_2 / (c w0)] dt,
// one integral over t (trapezoid rule, h = 1/8, analytic integrand).
//
// Pair split: the electron's fraction e has density
//   p(e) = (e/(1-e) + (1-e)/e) K_2/3(y) + int_y^inf K_1/3,  y = 2/(3 chi e(1-e)),
// handled as p e^(y0), y0 = 8/(3 chi) (its value at e = 1/2) against
// underflow; its integral from 0 to e0 <= 1/2 by the tanh-sinh rule in e
// (the essential singularity exp(-2/(3 chi e)) at e = 0 is harmless to it).
#pragma once

namespace gapk {

// Ehat_n(x) = e^x E_n(x), n = 1, 2, 3: the power series of E_1 (Abramowitz &
// Stegun 5.1.11) and the upward recurrence E_(m+1) = (e^-x - x E_m)/m for
// x <= 1; the continued fraction of E_n (A&S 5.1.22, even form, modified
// Lentz) for x > 1, where the recurrence would cancel.
__device__ __forceinline__ double scaled_expint(int n, double x) {
  if (x <= 1.0) {
    double s = 0.0, term = 1.0;
    for (int k = 1; k < 64; ++k) {
      term *= -x / (double)k;
      const double add = term / (double)k;
      s += add;
      if (fabs(add) < 1e-17 * fabs(s)) break;
    }
    double e = exp(x) * (-0.57721566490153286061 - log(x) - s);
    for (int m = 1; m < n; ++m) e = (1.0 - x * e) / (double)m;
    return e;
  }
  const double tiny = 1e-300;
  double f = tiny, C = f, D = 0.0;
  for (int i = 0; i < 400; ++i) {
    const double b = x + (double)n + 2.0 * i;
    const double a = i == 0 ? 1.0 : -(double)i * (double)(n - 1 + i);
    D = b + a * D;
    C = b + a / C;
    D = 1.0 / D;
    const double dl = C * D;
    f *= dl;
    if (fabs(dl - 1.0) < 1e-16) break;
  }
  return f;
}

// S(xi) of the quantum photon spectrum (not normalised).
__device__ __noinline__ static double qs_survival_exact(double chi, double xi) {
  const double d0 = xi > 0.0 ? 2.0 * xi / (3.0 * chi * (1.0 - xi)) : 0.0;
  const double w0 = 2.0 + 3.0 * chi * d0, i3chi = 1.0 / (3.0 * chi);
  const double h = 0.125;
  double s = 0.0;
  for (int k = 0; k < 6000; ++k) {
    const double t = k * h, c = cosh(t);
    if (c * d0 > 745.0) break;
    const double x = c * w0 * i3chi;
    const double f = exp(-c * d0) * (cosh(2.0 * t / 3.0) * (2.0 * scaled_expint(3, x) / (w0 * w0) +
                                                           0.5 * scaled_expint(1, x)) -
                                     cosh(t / 3.0) / c * scaled_expint(2, x) / w0);
    s += (k == 0 ? 0.5 : 1.0) * f;
    if (k > 8 && fabs(f) <= 1e-18 * fabs(s)) break;
  }
  return 2.0 * h * s;
}

// n(xi) of the quantum photon spectrum.
__device__ __noinline__ static double qs_density_exact(double chi, double xi) {
  if (!(xi > 0.0 && xi < 1.0)) return 0.0;
  const double d = 2.0 * xi / (3.0 * chi * (1.0 - xi));
  const double B = 1.0 - xi + 1.0 / (1.0 - xi);
  const double h = 0.125;
  double s = 0.0;
  for (int k = 0; k < 6000; ++k) {
    const double t = k * h, c = cosh(t);
    if (c * d > 745.0) break;
    s += (k == 0 ? 0.5 : 1.0) * exp(-c * d) * (B * cosh(2.0 * t / 3.0) - cosh(t / 3.0) / c);
  }
  return h * s;
}

// The xi with S(xi) = U S(0), from an estimate xi0 (the table's) by Newton
// steps dxi = (S(xi) - U S(0)) / n(xi); a step that would leave (0, 1) is
// halved towards the side it aims at.
__device__ __noinline__ static double qs_refine(double chi, double U, double xi0) {
  if (!(U < 1.0) || !(xi0 > 0.0)) return xi0;
  const double target = U * qs_survival_exact(chi, 0.0);
  double xi = xi0 < 1.0 ? xi0 : 1.0 - 1e-16;
  for (int it = 0; it < 6; ++it) {
    const double nd = qs_density_exact(chi, xi);
    if (!(nd > 0.0)) break;
    const double step = (qs_survival_exact(chi, xi) - target) / nd;
    double xn = xi + step;
    if (!(xn > 0.0)) xn = 0.5 * xi;
    if (!(xn < 1.0)) xn = 0.5 * (xi + 1.0);
    const double dx = fabs(xn - xi);
    xi = xn;
    if (dx <= 1e-15 * xi) break;
  }
  return xi;
}

// p(e) e^(y0) of the pair split.
__device__ __noinline__ static double bw_density_scaled_exact(double chi, double e) {
  if (!(e > 0.0 && e < 1.0)) return 0.0;
  const double q = e * (1.0 - e);
  const double y = 2.0 / (3.0 * chi * q), y0 = 8.0 / (3.0 * chi);
  const double A = (1.0 - 2.0 * q) / q;  // e/(1-e) + (1-e)/e
  const double h = 0.125;
  double s = 0.0;
  for (int k = 0; k < 6000; ++k) {
    const double t = k * h, c = cosh(t), arg = y * c - y0;
    if (arg > 745.0) break;
    s += (k == 0 ? 0.5 : 1.0) * exp(-arg) * (A * cosh(2.0 * t / 3.0) + cosh(t / 3.0) / c);
  }
  return h * s;
}

// int_0^e0 p de e^(y0), e0 <= 1/2, by the tanh-sinh rule: e = e0 (1 +
// tanh(pi/2 sinh tau))/2, step 1/64 over |tau| <= 3.6 (the weights beyond are
// below 1e-30 of the largest).
__device__ __noinline__ static double bw_tail_scaled_exact(double chi, double e0) {
  const double h = 1.0 / 64.0, hp = 1.5707963267948966;
  double s = 0.0;
  for (int i = -230; i <= 230; ++i) {
    const double tau = i * h;
    const double u = hp * sinh(tau);
    const double e = e0 / (1.0 + exp(-2.0 * u));  // e0 (1 + tanh u)/2 without cancellation
    const double cu = cosh(u);
    const double w = 0.5 * e0 * hp * cosh(tau) / (cu * cu);
    if (e > 0.0) s += w * bw_density_scaled_exact(chi, e);
  }
  return h * s;
}

// The smaller share e <= 1/2 with int_0^e p = 2 u int_0^(1/2) p (u =
// min(U, 1 - U)), from an estimate e_est by Newton steps; a step that would
// leave (0, 1/2] is halved towards the side it aims at.
__device__ __noinline__ static double bw_refine(double chi, double u, double e_est) {
  if (!(chi > 0.0)) return e_est;
  const double target = 2.0 * u * bw_tail_scaled_exact(chi, 0.5);
  double e = e_est > 0.0 ? (e_est < 0.5 ? e_est : 0.5) : 1e-300;
  for (int it = 0; it < 6; ++it) {
    const double dp = bw_density_scaled_exact(chi, e);
    if (!(dp > 0.0)) break;
    const double step = (bw_tail_scaled_exact(chi, e) - target) / dp;
    double en = e - step;
    if (!(en > 0.0)) en = 0.5 * e;
    if (en > 0.5) en = 0.5 * (e + 0.5);
    const double de = fabs(en - e);
    e = en;
    if (de <= 1e-15 * e) break;
  }
  return e;
}

}  // namespace gapk
