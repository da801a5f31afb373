// api.cu -- the C ABI (include/gap.h): workspace layout, initialisation,
// stepping, diagnostics and particle export/import.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "gap_internal.cuh"
#include "kernels.h"

using namespace gapk;

struct gap_handle {
  View v{};
  int32_t n_gaps = 0, precision = 0, threads = 256;
  double slack = 0.125;
  std::vector<gap_params> params;
  std::vector<GapDev> gaps_h;
  std::vector<TileDev> tiles_h;
  std::vector<LoadSpec> loads;
  std::vector<int32_t> proton_loads;  // gaps that start with protons below H_gap
  int64_t total_nodes = 0, steps_done = 0;
  char *ws = nullptr;
  size_t ws_bytes = 0;
  size_t ws_need = 0;  // bytes of the workspace the layout uses
  char *buf_base[2] = {nullptr, nullptr};
  size_t buf_bytes = 0;
  unsigned long long *export_count = nullptr;
  cudaGraphExec_t graph = nullptr;
  int32_t graph_chunk = 0;
  cudaStream_t graph_stream = nullptr;
  int status = GAP_OK;
  std::string err;
  // live timing of the step phases (gap_profile, gap_profile_phases)
  bool profiling = false;
  std::vector<cudaEvent_t> ev;  // kProfEvents per profiled step
  size_t ev_used = 0;
  double phase_ms[GAP_NPHASES] = {0, 0, 0, 0, 0};
  int64_t phase_steps = 0;
  // gap_get_field_async: after the enqueued steps; after the staging copy
  cudaEvent_t fa_after_steps = nullptr, fa_after_stage = nullptr;
};

static constexpr size_t kProfEvents = 6;

namespace {

struct Carver {
  char *base;
  size_t off = 0;
  explicit Carver(char *b) : base(b) {}
  template <class T>
  T *take(size_t n) {
    off = (off + 255) & ~(size_t)255;
    T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += n * sizeof(T);
    return p;
  }
};

int fail(gap_handle *h, int code, const std::string &msg) {
  if (h && h->status == GAP_OK) {
    h->status = code;
    h->err = msg;
  }
  return code;
}

int cuda_check(gap_handle *h, cudaError_t e, const char *what) {
  if (e == cudaSuccess) return GAP_OK;
  return fail(h, GAP_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

gap_config default_config(const gap_config *c) {
  gap_config d{};
  if (c) d = *c;
  if (d.tile <= 0) d.tile = 256;
  if (d.threads <= 0) d.threads = 256;
  if (d.rebin_every <= 0) d.rebin_every = 64;
  if (!(d.slack > 0.0)) d.slack = 0.125;
  return d;
}

int validate(const gap_params *p, int32_t n, const gap_config &cfg, std::string &msg) {
  if (!p || n <= 0) { msg = "no gaps"; return GAP_EINVAL; }
  if (cfg.precision != GAP_FP64_PLAIN && cfg.precision != GAP_FP32_STATE) { msg = "precision"; return GAP_EINVAL; }
  if (cfg.tile < 8 || cfg.tile > 4096) { msg = "tile must be in [8, 4096]"; return GAP_EINVAL; }
  if (cfg.threads < 32 || cfg.threads > 256 || cfg.threads % 32) { msg = "threads must be a multiple of 32 in [32, 256]"; return GAP_EINVAL; }
  if (cfg.variant < 0 || cfg.variant > 5) { msg = "variant must be in [0, 5]"; return GAP_EINVAL; }
  if (cfg.variant >= 4 && cfg.tile > 512) { msg = "TMA variants need tile <= 512 (48 KB shared memory)"; return GAP_EINVAL; }
  for (int i = 0; i < n; ++i) {
    const gap_params &q = p[i];
    if (q.nx < 8 || q.nx > (1ll << 28)) { msg = "nx out of range"; return GAP_EINVAL; }
    if (!(q.dx > 0) || !(q.dt > 0) || q.dt / q.dx >= 0.5) { msg = "need dx, dt > 0 and c dt/dx < 1/2"; return GAP_EINVAL; }
    if (q.boundary != GAP_BC_SURFACE && q.boundary != GAP_BC_PERIODIC) { msg = "boundary"; return GAP_EINVAL; }
    if (q.init < GAP_INIT_EMPTY || q.init > GAP_INIT_GAP_PROTONS) { msg = "init"; return GAP_EINVAL; }
    if (q.init != GAP_INIT_EMPTY && q.ppc <= 0) { msg = "ppc must be > 0 for a load"; return GAP_EINVAL; }
    if (q.kmax_emit < 0 || q.kmax_emit > kMaxEmit) { msg = "kmax_emit must be <= 16"; return GAP_EINVAL; }
    if (q.qed && (!(q.lambda_hat > 0) || !(q.rho_hat > 0) || q.rate_mult < 0)) { msg = "QED scales"; return GAP_EINVAL; }
    if (q.init == GAP_INIT_PAIR_THERMAL && q.boundary != GAP_BC_PERIODIC) { msg = "thermal pair load needs a periodic gap"; return GAP_EINVAL; }
    if (!(q.inject_theta >= 0.0) || q.inject_theta > 1e3) { msg = "inject_theta must be in [0, 1e3]"; return GAP_EINVAL; }
    if (q.filter_passes < 0 || q.filter_passes > 16) { msg = "filter_passes must be in [0, 16]"; return GAP_EINVAL; }
    if (q.filter_passes > 0 && q.nx < 2 * (int64_t)q.filter_passes + 2) { msg = "filter_passes needs nx >= 2 passes + 2"; return GAP_EINVAL; }
    if (q.qed_quantum != 0 && q.qed_quantum != 1) { msg = "qed_quantum must be 0 or 1"; return GAP_EINVAL; }
    if (q.protons != 0 && q.protons != 1) { msg = "protons must be 0 or 1"; return GAP_EINVAL; }
    if (q.init == GAP_INIT_GAP_PROTONS && (!q.protons || q.boundary != GAP_BC_SURFACE))
      { msg = "the proton start needs protons and a surface gap"; return GAP_EINVAL; }
    if (q.m_ion < 0.0) { msg = "m_ion must be >= 0"; return GAP_EINVAL; }
    if (q.em != 0 && q.em != 1) { msg = "em must be 0 or 1"; return GAP_EINVAL; }
    if (!std::isfinite(q.beta_y) || !std::isfinite(q.beta_z) || !(q.beta_y * q.beta_y + q.beta_z * q.beta_z < 1.0))
      { msg = "beta must be finite with |beta| < 1"; return GAP_EINVAL; }
    if (!q.em && (q.beta_y != 0.0 || q.beta_z != 0.0 || q.pml_cells != 0))
      { msg = "beta and pml_cells need em = 1"; return GAP_EINVAL; }
    if (q.pml_cells < 0 || (q.pml_cells > 0 && (q.boundary != GAP_BC_SURFACE || 2 * (int64_t)q.pml_cells > q.nx)))
      { msg = "pml_cells must be in [0, nx/2], on a surface gap"; return GAP_EINVAL; }
    if (!(q.pml_sigma >= 0.0) || !std::isfinite(q.pml_sigma)) { msg = "pml_sigma must be >= 0"; return GAP_EINVAL; }
    if (q.jperp != 0 && q.jperp != 1) { msg = "jperp must be 0 or 1"; return GAP_EINVAL; }
    if (q.jperp && (!q.em || !(q.b > 0.0) || !(q.lambda_hat > 0.0)))
      { msg = "jperp needs em = 1, b > 0 and lambda_hat > 0"; return GAP_EINVAL; }
    if (q.pad0 != 0) { msg = "pad0 must be zero"; return GAP_EINVAL; }
  }
  return GAP_OK;
}

// Host quadrature of the survival function S(xi) of the classical curvature
// spectrum and of dS/dxi (trapezoid in t with the integral representation
// S = 3/(5 pi) int cosh(5t/3) e^{-xi cosh t} / cosh^2 t dt), used to build the
// tables that the kernels read.
struct SpecQuad {
  double h;
  std::vector<double> c, a;
  explicit SpecQuad(double hh, double tmax) : h(hh) {
    for (int k = 0; k * h <= tmax; ++k) {
      double t = k * h;
      c.push_back(std::cosh(t));
      a.push_back(std::cosh(5.0 * t / 3.0) / std::cosh(t));
    }
  }
  void eval(double xi, double &S, double &dS) const {
    double s0 = 0, s1 = 0;
    for (size_t k = 0; k < c.size(); ++k) {
      if (xi * (c[k] - 1.0) - (double)k * h > 40.0) break;
      double f = a[k] * std::exp(-xi * c[k]);
      double wk = k == 0 ? 0.5 : 1.0;
      s0 += wk * f / c[k];
      s1 += wk * f;
    }
    const double norm = 3.0 / (5.0 * M_PI) * h;
    S = norm * s0;
    dS = -norm * s1;
  }
  // xi with S(xi) = exp(-v): bracketed Newton on ln xi.
  double inverse_of_v(double v) const {
    const double U = std::exp(-v);
    double lo = std::log(1e-45), hi = std::log(80.0);
    double y = v > 1.0 ? std::log(v) : 3.0 * std::log(v) + 0.5;
    if (!(y > lo && y < hi)) y = 0.5 * (lo + hi);
    for (int it = 0; it < 300; ++it) {
      double xi = std::exp(y), S, dS;
      eval(xi, S, dS);
      // compare in terms of -ln S to keep relative accuracy at both ends
      double g = -std::log(S) - v;  // increasing in y
      if (g < 0) lo = y; else hi = y;
      double dg = -xi * dS / S;
      double yn = y - g / dg;
      if (!(yn > lo && yn < hi)) yn = 0.5 * (lo + hi);
      if (std::fabs(yn - y) < 1e-13) { y = yn; break; }
      y = yn;
    }
    (void)U;
    return std::exp(y);
  }
};

}  // namespace

// Quantum photon spectrum (gaps with qed_quantum), built on the host.  The
// photon number per unit energy fraction xi is proportional to
//   n(xi) = (1 - xi + 1/(1 - xi)) K_2/3(d) - int_d^inf K_1/3,
//   d = 2 xi / (3 chi (1 - xi))   (Baier & Katkov 1968),
// with K_nu(d) = int_0^inf e^{-d cosh t} cosh(nu t) dt and
// int_d^inf K_nu = int_0^inf e^{-d cosh t} cosh(nu t) / cosh t dt (trapezoid
// in t, h = 1/8).  In s = d^(1/3), xi = 3 chi s^3 / (2 + 3 chi s^3) and the
// survival S(s) = int_s^inf n dxi/ds' ds' is smooth at both ends; each panel
// between nodes s_k = qs_node(k) is one 8-point Gauss-Legendre rule.  Row r holds chi =
// exp(kQsLchi0 + r kQsDlchi); node k holds (S(s_k)/S(0), dS/ds(s_k)/S(0)).
struct QSpecHost {
  static constexpr double kH = 0.125;
  double gx[8], gw[8];
  std::vector<double> c, c2, c1;  // cosh t, cosh(2t/3), cosh(t/3)/cosh t at t = k h
  QSpecHost() {
    for (int i = 0; i < 8; ++i) {  // Gauss-Legendre nodes: Newton on P_8 (three-term recurrence)
      double z = std::cos(M_PI * (i + 0.75) / 8.5), dp = 1.0;
      for (int it = 0; it < 100; ++it) {
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= 8; ++k) {
          const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        dp = 8.0 * (z * p1 - p0) / (z * z - 1.0);
        const double dz = p1 / dp;
        z -= dz;
        if (std::fabs(dz) < 1e-16) break;
      }
      gx[i] = z;
      gw[i] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
    for (int k = 0; k * kH <= 120.0; ++k) {
      const double t = k * kH;
      c.push_back(std::cosh(t));
      c2.push_back(std::cosh(2.0 * t / 3.0));
      c1.push_back(std::cosh(t / 3.0) / std::cosh(t));
    }
  }
  // n(d, xi); the t-sum stops once a term is below e^-40 of the first
  // (d (cosh t - 1) - 2t/3 > 40: the node weights grow at most like e^(2t/3))
  double density(double d, double xi) const {
    const double B = 1.0 - xi + 1.0 / (1.0 - xi);
    double sum = 0.0;
    for (size_t k = 0; k < c.size(); ++k) {
      const double arg = d * c[k];
      if (arg > 745.0 || d * (c[k] - 1.0) - (2.0 / 3.0) * k * kH > 40.0) break;
      sum += (k == 0 ? 0.5 : 1.0) * std::exp(-arg) * (B * c2[k] - c1[k]);
    }
    return kH * sum;
  }
  double per_s(double chi, double s) const {  // n(xi(s)) dxi/ds
    const double d = s * s * s, w = 2.0 + 3.0 * chi * d, xi = 3.0 * chi * d / w;
    if (!(s > 0.0) || xi >= 1.0) return 0.0;
    return density(d, xi) * 18.0 * chi * s * s / (w * w);
  }
  void row(double chi, double2 *out) const {
    std::vector<double> S(kQsNodes, 0.0);
    double acc = 0.0;  // the rest beyond the last node (below e^-60 of the total)
    {
      const double a = qs_node(kQsNodes - 1);
      for (int i = 0; i < 8; ++i) acc += 0.5 * gw[i] * per_s(chi, a + 0.5 * (gx[i] + 1.0));
    }
    S[kQsNodes - 1] = acc;
    for (int k = kQsNodes - 2; k >= 0; --k) {
      const double a = qs_node(k), hp = qs_node(k + 1) - a;
      double p = 0.0;
      for (int i = 0; i < 8; ++i) p += gw[i] * per_s(chi, a + 0.5 * hp * (gx[i] + 1.0));
      acc += 0.5 * hp * p;
      S[k] = acc;
    }
    const double S0 = S[0];
    for (int k = 0; k < kQsNodes; ++k) {
      // dS/ds has a finite limit at s = 0 (n ~ d^(-2/3), dxi/ds ~ s^2)
      const double sk = k > 0 ? qs_node(k) : 1e-12;
      out[k].x = S[k] / S0;
      out[k].y = -per_s(chi, sk) / S0;
    }
    out[0].x = 1.0;
  }
};

// Pair energy split (qed_quantum), built on the host: the electron's
// fraction e of the photon energy has density
//   p(e) = (e/(1 - e) + (1 - e)/e) K_2/3(y) + int_y^inf K_1/3,
//   y = 2 / (3 chi e (1 - e))   (Baier & Katkov 1968),
// symmetric about 1/2 (Bessel integrals as for the photon spectrum), taken
// times e^(y0), y0 = 8/(3 chi), so that small chi do not underflow.  Row r
// holds chi = exp(kBwLchi0 + r ln10/8); node k holds G = F(1/2 - eta_k) / F(1/2)
// (F(e) = int_0^e p, summed from the e = 0 end, free of cancellation in the
// far tail) and dG/deta, eta_k = bw_node(k), one 8-point Gauss-Legendre rule
// per panel.
struct BwHost {
  const QSpecHost &q;  // Gauss-Legendre nodes and the t-node values
  explicit BwHost(const QSpecHost &qq) : q(qq) {}
  double density_scaled(double chi, double e) const {
    if (!(e > 0.0 && e < 1.0)) return 0.0;
    const double y = 2.0 / (3.0 * chi * e * (1.0 - e)), y0 = 8.0 / (3.0 * chi);
    const double A = e / (1.0 - e) + (1.0 - e) / e;
    double sum = 0.0;
    for (size_t k = 0; k < q.c.size(); ++k) {
      const double arg = y * q.c[k] - y0;
      if (arg > 745.0 || y * (q.c[k] - 1.0) - (2.0 / 3.0) * k * QSpecHost::kH > 40.0) break;
      sum += (k == 0 ? 0.5 : 1.0) * std::exp(-arg) * (A * q.c2[k] + q.c1[k]);
    }
    return QSpecHost::kH * sum;
  }
  void row(double chi, double2 *out) const {
    std::vector<double> T(kQsNodes, 0.0);  // int over [eta_k, 1/2] of p(1/2 - eta)
    for (int k = kQsNodes - 2; k >= 0; --k) {
      const double a = bw_node(k), hp = bw_node(k + 1) - a;
      double p = 0.0;
      for (int i = 0; i < 8; ++i) p += q.gw[i] * density_scaled(chi, 0.5 - (a + 0.5 * hp * (q.gx[i] + 1.0)));
      T[k] = T[k + 1] + 0.5 * hp * p;
    }
    const double Ht = T[0];
    for (int k = 0; k < kQsNodes; ++k) {
      out[k].x = T[k] / Ht;
      out[k].y = -density_scaled(chi, 0.5 - bw_node(k)) / Ht;
    }
    out[0].x = 1.0;
    out[kQsNodes - 1].x = 0.0;
  }
};

static int64_t next_pow2(int64_t n) {
  int64_t p = 1;
  while (p < n) p <<= 1;
  return p;
}

// Lay out (or, with base == nullptr, only measure) one handle.
static int build_layout(const gap_params *p, int32_t n, const gap_config &cfg, char *base,
                        gap_handle *h, size_t *bytes_out) {
  const bool fp32 = cfg.precision == GAP_FP32_STATE;
  const size_t rs = fp32 ? 4 : 8, wsz = fp32 ? 4 : 8;
  const int T = cfg.tile;
  std::vector<GapDev> gaps(n);
  std::vector<TileDev> tiles;
  std::vector<LoadSpec> loads;
  std::vector<int64_t> cap0[2];
  int64_t total_nodes = 0, max_nx = 0, max_P = 2, lep_need[2] = {0, 0}, ph_need = 0;
  bool qed_any = false, surface_any = false, merge_any = false, filter_any = false, qs_any = false, pr_any = false;
  bool em_any = false, jperp_any = false;
  int64_t pr_need = 0;
  for (int i = 0; i < n; ++i) {
    const gap_params &q = p[i];
    GapDev &g = gaps[i];
    std::memset(&g, 0, sizeof(g));
    g.nx = q.nx;
    g.periodic = q.boundary == GAP_BC_PERIODIC;
    g.nnode = g.periodic ? q.nx : q.nx + 1;
    g.node_off = total_nodes;
    total_nodes += g.nnode;
    max_nx = std::max<int64_t>(max_nx, g.nnode);
    g.qed = q.qed ? 1 : 0;
    g.kmax_emit = q.kmax_emit > 0 ? q.kmax_emit : 16;
    g.kmax_inject = q.kmax_inject > 0 ? q.kmax_inject : 64;
    g.gap_index = q.gap_index;
    g.dx = q.dx;
    g.dt = q.dt;
    g.cdx = q.dt / q.dx;
    g.jm = -q.alpha;
    const double H = q.gap_length > 0 ? q.gap_length : 0.8 * (double)q.nx * q.dx;
    g.Hc = H / q.dx;
    g.lambda_hat = q.qed ? q.lambda_hat : 1.0;
    g.rho_hat = q.qed ? q.rho_hat : 1.0;
    g.rate_mult = q.rate_mult;
    g.b = q.b;
    g.eta_bg = -1.0;
    const double frac = q.init == GAP_INIT_PAIR_THERMAL ? 0.5 : 1.0;
    g.w0 = q.ppc > 0 ? frac * q.density * q.dx / (double)q.ppc : 0.0;
    g.w_unit = (g.w0 > 0 ? g.w0 : q.dx) / (double)(1 << kWeightShift);
    g.f_dt = (float)g.dt;
    g.f_cdx = (float)g.cdx;
    g.f_Hc = (float)g.Hc;
    g.f_lam = (float)g.lambda_hat;
    g.f_rho = (float)g.rho_hat;
    g.f_rate = (float)g.rate_mult;
    g.f_b = (float)q.b;
    g.inv_cdx = 1.0 / g.cdx;
    g.seed = q.seed;
    g.cap = q.cap > 0 ? q.cap : 0;
    g.inject_theta = q.inject_theta;
    g.filter_passes = q.filter_passes;
    g.protons = q.protons;
    g.m_ion = q.m_ion > 0.0 ? q.m_ion : 1836.0;
    g.em = q.em;
    g.pml_cells = q.em ? q.pml_cells : 0;
    g.beta_y = q.beta_y;
    g.beta_z = q.beta_z;
    g.pml_smax = g.pml_cells <= 0 ? 0.0
                 : (q.pml_sigma > 0.0 ? q.pml_sigma : 4.0 * std::log(1e6) / (2.0 * (double)g.pml_cells * q.dx));
    g.jperp = q.em ? q.jperp : 0;
    g.bstar_inv = g.jperp ? q.lambda_hat / q.b : 0.0;
    em_any |= q.em != 0;
    jperp_any |= g.jperp != 0;
    g.defer = q.filter_passes > 0 || q.protons || q.em ? 1 : 0;
    filter_any |= g.defer != 0;
    pr_any |= q.protons != 0;
    if (q.protons) pr_need += 2 * q.nx * std::max<int64_t>(q.ppc, 1) + 65536;
    g.qed_quantum = q.qed && q.qed_quantum ? 1 : 0;
    qs_any |= g.qed_quantum != 0;
    merge_any |= q.cap > 0;
    g.inj_root = ((uint64_t)(uint32_t)q.gap_index << 40) | (1ull << 38);
    qed_any |= g.qed != 0;
    surface_any |= !g.periodic;
    max_P = std::max<int64_t>(max_P, next_pow2(std::min<int64_t>((int64_t)std::floor(g.Hc) + 1, g.nnode)));
    // tiles of T dual cells; a remainder below 4 joins the previous tile
    int64_t nt = (g.nnode + T - 1) / T;
    int64_t rem = g.nnode - (nt - 1) * T;
    if (rem < 4 && nt > 1) nt -= 1;
    g.tile_begin = (int32_t)tiles.size();
    g.n_tiles = (int32_t)nt;
    const int64_t species =
        q.init == GAP_INIT_PAIR_THERMAL ? 2 : (q.init == GAP_INIT_COLD || q.init == GAP_INIT_GAP_PROTONS ? 1 : 0);
    for (int64_t t = 0; t < nt; ++t) {
      TileDev td{};
      td.gap = i;
      td.k0 = (int32_t)(t * T);
      td.nk = (int32_t)(t == nt - 1 ? g.nnode - t * T : T);
      tiles.push_back(td);
      for (int s = 0; s < 2; ++s) {
        int64_t cnt = (s < species) ? (int64_t)td.nk * q.ppc : 0;
        int64_t c = (int64_t)(cnt * (1.0 + cfg.slack)) + 64;
        c = (c + 31) & ~31ll;
        cap0[s].push_back(c);
      }
    }
    const int64_t load = q.nx * (q.init != GAP_INIT_EMPTY ? q.ppc : 0);
    for (int s = 0; s < 2; ++s) {
      const int64_t ls = s < species ? load : 0;
      int64_t need = (int64_t)(1.3 * (double)ls) + 160 * nt;
      if (q.qed) {
        int64_t grow = q.cap > 0 ? q.cap : 16 * std::max<int64_t>(load, 1024);
        need = std::max<int64_t>(need, grow + 160 * nt);
      }
      lep_need[s] += need;
    }
    // photons: the cap bounds the pair cascade only on average (photons merge
    // at birth, older ones wait to convert or escape), so a capped gap keeps
    // at least the uncapped default
    if (q.qed) ph_need += std::max<int64_t>(q.cap, 16 * std::max<int64_t>(load, 1024));
    if (q.init != GAP_INIT_EMPTY) {
      LoadSpec ls{};
      ls.gap = i;
      ls.init = q.init == GAP_INIT_GAP_PROTONS ? GAP_INIT_COLD : q.init;  // the electrons of that start
      ls.species_count = (int32_t)species;
      ls.ppc = q.ppc;
      ls.n_per_species = load;
      ls.density = q.density;
      ls.theta = q.theta;
      ls.seed_amp = q.seed_amp;
      loads.push_back(ls);
    }
  }
  const int NT = (int)tiles.size();
  int64_t lep_cap = cfg.lepton_capacity > 0 ? cfg.lepton_capacity : std::max(lep_need[0], lep_need[1]);
  int64_t cap_sum0 = 0, cap_sum1 = 0;
  for (int t = 0; t < NT; ++t) { cap_sum0 += cap0[0][t]; cap_sum1 += cap0[1][t]; }
  lep_cap = std::max<int64_t>(lep_cap, std::max(cap_sum0, cap_sum1));
  const int64_t ph_cap = cfg.photon_capacity > 0 ? cfg.photon_capacity : std::max<int64_t>(ph_need, 1024);
  const int64_t spill_cap = std::max<int64_t>(65536, lep_cap / 32);
  const int64_t dchg = std::max(total_nodes, max_nx);

  Carver C(base);
  // the two-pass FP32 QED push leaves Ampere to k_filter_apply for every gap
  // (its second pass deposits after the first has finished its tiles)
  const bool two_pass = fp32 && qed_any && (cfg.variant == 0 || cfg.variant == 1);
  for (auto &g : gaps) {
    g.ampere_late = g.defer || two_pass ? 1 : 0;
    filter_any |= g.ampere_late != 0;
  }
  View v{};
  v.n_gaps = n;
  v.n_tiles = NT;
  v.tile = T;
  v.precision = cfg.precision;
  v.qed_any = qed_any;
  v.surface_any = surface_any;
  v.has_w = (qed_any || merge_any) ? 1 : 0;  // merging makes weights unequal
  v.merge_any = merge_any ? 1 : 0;
  v.filter_any = filter_any ? 1 : 0;
  {
    bool da = false;
    for (const auto &g : gaps) da |= g.defer != 0;
    v.defer_any = da ? 1 : 0;
  }
  v.pr_any = pr_any ? 1 : 0;
  v.em_any = em_any ? 1 : 0;
  v.jperp_any = jperp_any ? 1 : 0;
  v.rebin_every = cfg.rebin_every;
  v.variant = cfg.variant;
  v.gaps = C.take<GapDev>(n);
  v.tiles = C.take<TileDev>(NT);
  v.ctl = C.take<Ctl>(1);
  v.E[0] = C.take<double>(total_nodes);
  v.E[1] = C.take<double>(total_nodes);
  v.Dg = C.take<unsigned long long>(total_nodes);
  v.arrive = C.take<int32_t>(total_nodes);
  v.expect = C.take<int8_t>(total_nodes);
  for (int s = 0; s < 2; ++s) {
    v.seg_start[s] = C.take<int64_t>(NT);
    v.seg_cap[s] = C.take<int32_t>(NT);
    v.seg_used[s] = C.take<int32_t>(NT);
    v.seg_append[s] = C.take<int32_t>(NT);
    v.seg_alive[s] = C.take<int32_t>(NT);
    v.spill_cnt[s] = C.take<int32_t>(NT);
    v.new_start[s] = C.take<int64_t>(NT);
    v.new_cap[s] = C.take<int32_t>(NT);
    v.new_fill[s] = C.take<int32_t>(NT);
    v.last_cnt[s] = C.take<int32_t>(NT);
    v.gross[s] = C.take<int32_t>(NT);
  }
  v.item_start = C.take<int32_t>((size_t)NT + 1);
  // items per tile: max(1, chunks of each species), each species' chunks at
  // most used / kPushChunkMin + 1, and the used slots of all tiles at most the
  // store's capacity
  const int64_t item_cap = 2 * (lep_cap / kPushChunkMin) + 2 * (int64_t)NT + 2;
  v.item_tile = C.take<int32_t>((size_t)item_cap);
  {  // the two-pass FP32 QED push (variants 0 and 1): its deferred list, an
     // eighth of the lepton slots, half for the tile movers and half for the
     // emitters (each a few per cent of a step's leptons; the rest, if ever,
     // are found in the store)
    const int64_t dcap = two_pass ? std::max<int64_t>(1 << 21, lep_cap / 8) : 0;
    v.defer_slot = C.take<int64_t>((size_t)dcap);
    v.defer_ts = C.take<uint32_t>((size_t)dcap);
    v.defer_cap = dcap;
    v.defer_use = dcap;
  }
  v.item_cap = (int32_t)std::min<int64_t>(item_cap, INT32_MAX);
  v.tile_done = C.take<int32_t>(NT);
  v.counters = C.take<unsigned long long>((size_t)n * C_NCNT);
  v.ledger = C.take<double>((size_t)n * L_NLED);
  v.q0 = C.take<unsigned long long>(n);
  v.merge_state = C.take<int32_t>(4 * (size_t)n);
  v.merge_width = C.take<double>(n);
  {
    const size_t nseg = merge_any ? 2 * (size_t)NT : 0;
    v.mlist = C.take<int32_t>(nseg);
    v.mout = C.take<int32_t>(nseg);
    v.mrun = C.take<int32_t>(nseg * (size_t)(cfg.tile + 4));
  }
  v.ph_gap = C.take<int32_t>(n);
  {  // photon merge table: twice the photon store (newborns are at most all of it), 2^10 .. 2^22 entries
    int64_t H = 0;
    if (merge_any && qed_any) {
      H = 1024;
      while (H < 2 * ph_cap && H < (int64_t(1) << 22)) H <<= 1;
    }
    v.phm_size = H;
    v.phm_key = C.take<unsigned long long>((size_t)H);
    v.phm_nid = C.take<unsigned long long>((size_t)H);
    v.phm_W = C.take<double>((size_t)H);
    v.phm_Wx = C.take<double>((size_t)H);
    v.phm_WX = C.take<double>((size_t)H);
    v.phm_cnt = C.take<unsigned>((size_t)H);
  }
  const int spec_n = 1024;
  v.spec_n = spec_n;
  v.spec_tab = C.take<float2>(spec_n);
  const double quad_h = 0.1, quad_tmax = 96.0;  // trapezoid error ~ exp(xi - pi^2/h) < 1e-27 for xi < 35
  v.quad_h = quad_h;
  v.quad_n = (int32_t)(quad_tmax / quad_h) + 1;
  v.quad_c = C.take<double>(v.quad_n);
  v.quad_a = C.take<double>(v.quad_n);
  v.qs_any = qs_any ? 1 : 0;
  v.qs_rows = kQsRows;
  v.qs_tab_d = C.take<double2>(qs_any ? (size_t)kQsRows * kQsNodes : 0);
  v.qs_tab_f = C.take<float2>(qs_any ? (size_t)kQsRows * kQsNodes : 0);
  v.bw_tab = C.take<float2>(qs_any ? (size_t)kBwRows * kQsNodes : 0);
  v.max_nx = max_nx;
  v.max_P = max_P;
  v.dmom = C.take<double>(8 * (size_t)max_nx);
  v.fstage = C.take<double>((size_t)max_nx);
  v.dcharge = C.take<unsigned long long>(dchg);
  v.dcharge_len = dchg;
  v.Dflt = C.take<double>(filter_any ? 2 * (size_t)dchg : 0);
  {  // transverse fields: zero at start (part of the cleared metadata)
    const size_t ne = em_any ? (size_t)total_nodes : 0;
    v.em_Ey = C.take<double>(ne);
    v.em_Ez = C.take<double>(ne);
    v.em_By = C.take<double>(ne);
    v.em_Bz = C.take<double>(ne);
    v.em_Jv = C.take<double>(ne);
    v.em_jy = C.take<double>(jperp_any ? ne : 0);
    v.em_jz = C.take<double>(jperp_any ? ne : 0);
  }
  v.fft[0] = C.take<double>(2 * (size_t)max_P);
  v.fft[1] = C.take<double>(2 * (size_t)max_P);
  v.dred = C.take<double>(32);
  v.ret_hist = C.take<double>((size_t)n * kRetBins);
  v.spec_buf = C.take<double>(3 * (size_t)kSpecMaxBins);
  unsigned long long *export_count = C.take<unsigned long long>(4);
  size_t meta_end = C.off;
  for (int s = 0; s < 2; ++s) {
    v.sk[s] = C.take<int32_t>(spill_cap);
    v.stile[s] = C.take<int32_t>(spill_cap);
    v.sphi[s] = C.take<double>(spill_cap);
    v.su[s] = C.take<double>(spill_cap);
    v.sw[s] = C.take<double>(spill_cap);
    v.stau[s] = C.take<double>(spill_cap);
    v.sid[s] = C.take<uint64_t>(spill_cap);
  }
  v.spill_capacity = spill_cap;
  for (int b = 0; b < 2; ++b) {
    v.pXr[b] = C.take<double>(ph_cap);
    v.px[b] = C.take<double>(ph_cap);
    v.pw[b] = C.take<double>(ph_cap);
    v.pts[b] = C.take<double>(ph_cap);
    v.pta[b] = C.take<double>(ph_cap);
    v.pid[b] = C.take<uint64_t>(ph_cap);
    v.pn0[b] = C.take<int32_t>(ph_cap);
    v.pnr[b] = C.take<int32_t>(ph_cap);
    v.pdir[b] = C.take<int32_t>(ph_cap);
    v.pgap[b] = C.take<int32_t>(ph_cap);
    v.pm[b] = C.take<int32_t>(ph_cap);
    v.pev[b] = C.take<int32_t>(ph_cap);
    v.pkind[b] = C.take<int32_t>(ph_cap);
    v.pmn[b] = C.take<int32_t>(ph_cap);
    v.ptan[b] = C.take<double>(ph_cap);
  }
  v.ph_work = C.take<int64_t>(ph_cap);
  v.pr_cap = pr_need;
  v.pr_X = C.take<double>(pr_need);
  v.pr_u = C.take<double>(pr_need);
  v.pr_w = C.take<double>(pr_need);
  v.pr_id = C.take<uint64_t>(pr_need);
  v.pr_gap = C.take<int32_t>(pr_need);
  v.pr_alive = C.take<int32_t>(pr_need);
  v.ph_capacity = ph_cap;
  char *bb[2];
  size_t bbytes = 0;
  for (int b = 0; b < 2; ++b) {
    C.off = (C.off + 255) & ~(size_t)255;
    size_t b0 = C.off;
    bb[b] = base ? base + b0 : nullptr;
    for (int s = 0; s < 2; ++s) {
      v.lk[b][s] = C.take<int32_t>(lep_cap);
      v.lphi[b][s] = C.take<char>(rs * lep_cap);
      v.lu[b][s] = C.take<char>(rs * lep_cap);
      v.lw[b][s] = C.take<char>(wsz * lep_cap);
      v.ltau[b][s] = C.take<char>(rs * lep_cap);
      v.lid[b][s] = C.take<uint64_t>(lep_cap);
    }
    bbytes = C.off - b0;
  }
  v.lep_capacity = lep_cap;
  *bytes_out = C.off + 256;
  if (!base) return GAP_OK;

  h->v = v;
  h->n_gaps = n;
  h->precision = cfg.precision;
  h->threads = cfg.threads;
  h->slack = cfg.slack;
  h->params.assign(p, p + n);
  h->gaps_h = gaps;
  h->tiles_h = tiles;
  h->loads = loads;
  h->proton_loads.clear();
  for (int i = 0; i < n; ++i)
    if (p[i].init == GAP_INIT_GAP_PROTONS) h->proton_loads.push_back(i);
  h->total_nodes = total_nodes;
  h->buf_base[0] = bb[0];
  h->buf_base[1] = bb[1];
  h->buf_bytes = bbytes;
  h->export_count = export_count;
  // expected contributors of every tile-edge node
  std::vector<int8_t> expect(total_nodes, 0);
  for (const TileDev &td : tiles) {
    const GapDev &g = gaps[td.gap];
    const int locals[4] = {0, 1, td.nk, td.nk + 1};
    for (int L : locals) {
      int64_t node = (int64_t)td.k0 - 1 + L;
      if (g.periodic) node = (node + g.nx) % g.nx;
      else if (node < 0 || node > g.nx) continue;
      expect[g.node_off + node] += 1;
    }
  }
  // initial segment layout
  std::vector<int64_t> start[2];
  std::vector<int32_t> capv[2];
  for (int s = 0; s < 2; ++s) {
    int64_t acc = 0;
    for (int t = 0; t < NT; ++t) {
      start[s].push_back(acc);
      capv[s].push_back((int32_t)cap0[s][t]);
      acc += cap0[s][t];
    }
  }
  cudaStream_t st = nullptr;
  cudaError_t e = cudaMemsetAsync(base, 0, meta_end, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(v.gaps, gaps.data(), sizeof(GapDev) * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(v.tiles, tiles.data(), sizeof(TileDev) * NT, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(v.expect, expect.data(), total_nodes, cudaMemcpyHostToDevice, st);
  for (int s = 0; s < 2 && e == cudaSuccess; ++s) {
    e = cudaMemcpyAsync(v.seg_start[s], start[s].data(), sizeof(int64_t) * NT, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(v.seg_cap[s], capv[s].data(), sizeof(int32_t) * NT, cudaMemcpyHostToDevice, st);
  }
  // spectrum tables
  SpecQuad sq(quad_h, quad_tmax);
  std::vector<double> qc(v.quad_n), qa(v.quad_n);
  for (int k = 0; k < v.quad_n; ++k) {
    const double t = k * quad_h;
    qc[k] = std::cosh(t);
    qa[k] = std::cosh(5.0 * t / 3.0) / std::cosh(t);
  }
  const double z0 = std::log(1e-7), z1 = std::log(40.0);
  const double dz = (z1 - z0) / (spec_n - 1);
  std::vector<float2> tab(spec_n);
  for (int i = 0; i < spec_n; ++i) {
    const double z = z0 + i * dz, vv = std::exp(z);
    const double xi = sq.inverse_of_v(vv);
    double S, dS;
    sq.eval(xi, S, dS);
    tab[i].x = (float)std::log(xi);
    tab[i].y = (float)(-vv * S / (xi * dS));
  }
  h->v.spec_z0 = (float)z0;
  h->v.spec_dz = (float)dz;
  if (e == cudaSuccess) e = cudaMemcpyAsync(v.spec_tab, tab.data(), sizeof(float2) * spec_n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(v.quad_c, qc.data(), sizeof(double) * v.quad_n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(v.quad_a, qa.data(), sizeof(double) * v.quad_n, cudaMemcpyHostToDevice, st);
  std::vector<double2> qtab_d, bwtab;
  std::vector<float2> qtab_f, bwtab_f;
  if (qs_any) {  // the quantum spectrum table, only when a gap asks for it
    qtab_d.resize((size_t)kQsRows * kQsNodes);
    qtab_f.resize(qtab_d.size());
    const QSpecHost qh;  // about 0.05 s for all rows
    for (int r = 0; r < kQsRows; ++r) qh.row(std::exp(kQsLchi0 + r * kQsDlchi), &qtab_d[(size_t)r * kQsNodes]);
    for (size_t i = 0; i < qtab_d.size(); ++i) qtab_f[i] = make_float2((float)qtab_d[i].x, (float)qtab_d[i].y);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(v.qs_tab_d, qtab_d.data(), sizeof(double2) * qtab_d.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(v.qs_tab_f, qtab_f.data(), sizeof(float2) * qtab_f.size(), cudaMemcpyHostToDevice, st);
    bwtab.resize((size_t)kBwRows * kQsNodes);
    const BwHost bh(qh);
    for (int r = 0; r < kBwRows; ++r) bh.row(std::exp(kBwLchi0 + r * kQsDlchi), &bwtab[(size_t)r * kQsNodes]);
    bwtab_f.resize(bwtab.size());  // (G, dG/d(1/2 - eta)) in float
    for (size_t i = 0; i < bwtab.size(); ++i) bwtab_f[i] = make_float2((float)bwtab[i].x, (float)(-bwtab[i].y));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(v.bw_tab, bwtab_f.data(), sizeof(float2) * bwtab_f.size(), cudaMemcpyHostToDevice, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return cuda_check(h, e, "layout upload");
}

static int read_ctl(gap_handle *h, Ctl *c, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(c, h->v.ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_check(h, e, "control block");
  if (c->error & 8) return fail(h, GAP_ECHECK, "store compaction overflowed a segment");
  if (c->error & 16) return fail(h, GAP_ETIMEOUT, "a bulk-copy stage of the push kernel never completed");
  if (c->error & 32) return fail(h, GAP_ECHECK, "a lepton outside its tile's nodes reached the merge");
  if (c->error & 64) return fail(h, GAP_ECHECK, "a photon event was not taken at its step");
  if (c->error & 128) return fail(h, GAP_ECAP, "proton storage exhausted");
  if (c->error & 256) return fail(h, GAP_ECHECK, "more push work items than the item table holds");
  if (c->error & 7)
    return fail(h, GAP_ECAP, c->error & 1 ? "lepton spill list exhausted"
                             : (c->error & 2 ? "photon storage exhausted" : "lepton storage exhausted"));
  return GAP_OK;
}

extern "C" {

int gap_workspace_bytes(const gap_params *params, int32_t n_gaps, const gap_config *cfg, size_t *bytes) {
  if (!bytes) return GAP_EINVAL;
  gap_config c = default_config(cfg);
  std::string msg;
  int r = validate(params, n_gaps, c, msg);
  if (r) return r;
  return build_layout(params, n_gaps, c, nullptr, nullptr, bytes);
}

int gap_init(const gap_params *params, int32_t n_gaps, const gap_config *cfg, void *dev_workspace,
             size_t bytes, void *stream, gap_handle **out) {
  if (!out) return GAP_EINVAL;
  *out = nullptr;
  gap_config c = default_config(cfg);
  std::string msg;
  int r = validate(params, n_gaps, c, msg);
  if (r) return r;
  size_t need = 0;
  build_layout(params, n_gaps, c, nullptr, nullptr, &need);
  if (!dev_workspace || bytes < need) return GAP_ENOSPACE;
  if (((uintptr_t)dev_workspace) & 255) return GAP_EINVAL;
  gap_handle *h = new gap_handle();
  h->ws = (char *)dev_workspace;
  h->ws_bytes = bytes;
  h->ws_need = need;
  r = build_layout(params, n_gaps, c, (char *)dev_workspace, h, &need);
  if (r) { *out = h; return r; }
  cudaStream_t st = (cudaStream_t)stream;
  launch_load(h->v, h->loads.data(), (int)h->loads.size(), 0, st);
  for (int32_t gi : h->proton_loads) launch_load_protons(h->v, gi, h->gaps_h[gi].nx * h->params[gi].ppc, st);
  launch_sync_used(h->v, st);
  launch_force_rebin(h->v, st);
  launch_rebin(h->v, h->slack, st);
  launch_gauss(h->v, 1, st);
  r = cuda_check(h, cudaGetLastError(), "init kernels");
  Ctl cc;
  if (!r) r = read_ctl(h, &cc, st);
  *out = h;
  return r;
}

int gap_step(gap_handle *h, int64_t nsteps, void *stream) {
  if (!h || nsteps < 0) return GAP_EINVAL;
  if (h->status) return h->status;
  cudaStream_t st = (cudaStream_t)stream;
  for (int64_t i = 0; i < nsteps; ++i) {
    if (h->profiling) {
      // six events per step, in order: before the push, after its
      // streaming kernel, after its tail, after the photon / injection /
      // bookkeeping launches, after the re-bin, after the merge
      if (h->ev_used + kProfEvents > h->ev.size()) {
        for (int k = 0; k < 16 * kProfEvents; ++k) {
          cudaEvent_t e;
          if (cudaEventCreate(&e) != cudaSuccess) return fail(h, GAP_ECUDA, "event create");
          h->ev.push_back(e);
        }
      }
      cudaEvent_t *ev = &h->ev[h->ev_used];
      cudaEventRecord(ev[0], st);
      launch_push(h->v, h->threads, st);
      cudaEventRecord(ev[1], st);
      launch_push_tail(h->v, st);
      cudaEventRecord(ev[2], st);
      launch_after_push(h->v, st);
      cudaEventRecord(ev[3], st);
      launch_rebin(h->v, h->slack, st);
      cudaEventRecord(ev[4], st);
      if (h->v.merge_any) launch_merge(h->v, st);
      cudaEventRecord(ev[5], st);
      h->ev_used += kProfEvents;
      continue;
    }
    launch_step(h->v, h->threads, st);
    launch_rebin(h->v, h->slack, st);
    if (h->v.merge_any) launch_merge(h->v, st);  // after the re-bin: no spilled leptons left
  }
  h->steps_done += nsteps;
  return cuda_check(h, cudaGetLastError(), "step launch");
}

int gap_step_graph(gap_handle *h, int64_t nsteps, int32_t chunk, void *stream) {
  if (!h || nsteps < 0 || chunk <= 0) return GAP_EINVAL;
  if (h->status) return h->status;
  cudaStream_t st = (cudaStream_t)stream;
  if (!st) return gap_step(h, nsteps, stream);
  if (!h->graph || h->graph_chunk != chunk) {
    if (h->graph) { cudaGraphExecDestroy(h->graph); h->graph = nullptr; }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_check(h, e, "begin capture");
    for (int i = 0; i < chunk; ++i) {
      launch_step(h->v, h->threads, st);
      launch_rebin(h->v, h->slack, st);
      if (h->v.merge_any) launch_merge(h->v, st);
    }
    e = cudaStreamEndCapture(st, &g);
    if (e != cudaSuccess) return cuda_check(h, e, "end capture");
    e = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_check(h, e, "instantiate");
    h->graph_chunk = chunk;
  }
  int64_t full = nsteps / chunk, rest = nsteps % chunk;
  for (int64_t i = 0; i < full; ++i) {
    cudaError_t e = cudaGraphLaunch(h->graph, st);
    if (e != cudaSuccess) return cuda_check(h, e, "graph launch");
  }
  h->steps_done += full * chunk;
  return gap_step(h, rest, stream);
}

int gap_get_field(gap_handle *h, int32_t gap, double *host_E, int64_t n, void *stream) {
  if (!h || gap < 0 || gap >= h->n_gaps || !host_E) return GAP_EINVAL;
  const GapDev &g = h->gaps_h[gap];
  if (n < g.nnode) return GAP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  Ctl c;
  int r = read_ctl(h, &c, st);
  if (r) return r;
  cudaError_t e = cudaMemcpyAsync(host_E, h->v.E[c.e_cur] + g.node_off, sizeof(double) * g.nnode,
                                  cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return cuda_check(h, e, "get field");
}

int gap_get_field_async(gap_handle *h, int32_t gap, double *host_E, int64_t n, void *stream, void *copy_stream) {
  if (!h || gap < 0 || gap >= h->n_gaps || !host_E) return GAP_EINVAL;
  if (h->status) return h->status;
  const GapDev &g = h->gaps_h[gap];
  if (n < g.nnode) return GAP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream, cs = (cudaStream_t)copy_stream;
  cudaError_t e = cudaSuccess;
  if (!h->fa_after_steps) e = cudaEventCreateWithFlags(&h->fa_after_steps, cudaEventDisableTiming);
  if (e == cudaSuccess && !h->fa_after_stage) e = cudaEventCreateWithFlags(&h->fa_after_stage, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventRecord(h->fa_after_steps, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, h->fa_after_steps, 0);
  if (e == cudaSuccess) {
    launch_copy_field(h->v, gap, cs);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(h->fa_after_stage, cs);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, h->fa_after_stage, 0);  // later steps wait for the staging only
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(host_E, h->v.fstage, sizeof(double) * g.nnode, cudaMemcpyDeviceToHost, cs);
  return cuda_check(h, e, "get field async");
}

int gap_set_field(gap_handle *h, int32_t gap, const double *host_E, int64_t n, void *stream) {
  if (!h || gap < 0 || gap >= h->n_gaps || !host_E) return GAP_EINVAL;
  const GapDev &g = h->gaps_h[gap];
  if (n < g.nnode) return GAP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  for (int b = 0; b < 2 && e == cudaSuccess; ++b)
    e = cudaMemcpyAsync(h->v.E[b] + g.node_off, host_E, sizeof(double) * g.nnode, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return cuda_check(h, e, "set field");
}

static int em_component(gap_handle *h, int32_t gap, int32_t component, int64_t n, double **dev, int64_t *len) {
  if (!h || gap < 0 || gap >= h->n_gaps || component < GAP_EM_EY || component > GAP_EM_BZ) return GAP_EINVAL;
  const GapDev &g = h->gaps_h[gap];
  if (!g.em) return GAP_EINVAL;
  *len = component <= GAP_EM_EZ ? g.nx : g.nnode;
  if (n < *len) return GAP_EINVAL;
  double *base[4] = {h->v.em_Ey, h->v.em_Ez, h->v.em_By, h->v.em_Bz};
  *dev = base[component] + g.node_off;
  return GAP_OK;
}

int gap_get_em(gap_handle *h, int32_t gap, int32_t component, double *host_dst, int64_t n, void *stream) {
  double *dev = nullptr;
  int64_t len = 0;
  if (!host_dst) return GAP_EINVAL;
  int r = em_component(h, gap, component, n, &dev, &len);
  if (r) return r;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(host_dst, dev, sizeof(double) * (size_t)len, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return cuda_check(h, e, "get em");
}

int gap_set_em(gap_handle *h, int32_t gap, int32_t component, const double *host_src, int64_t n, void *stream) {
  double *dev = nullptr;
  int64_t len = 0;
  if (!host_src) return GAP_EINVAL;
  int r = em_component(h, gap, component, n, &dev, &len);
  if (r) return r;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(dev, host_src, sizeof(double) * (size_t)len, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return cuda_check(h, e, "set em");
}

int gap_solve_gauss(gap_handle *h, int32_t set_background, void *stream) {
  if (!h) return GAP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  launch_gauss(h->v, set_background, st);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && set_background) {
    std::vector<GapDev> gd(h->n_gaps);
    e = cudaMemcpy(gd.data(), h->v.gaps, sizeof(GapDev) * h->n_gaps, cudaMemcpyDeviceToHost);
    for (int i = 0; i < h->n_gaps && e == cudaSuccess; ++i) h->gaps_h[i].eta_bg = gd[i].eta_bg;
  }
  return cuda_check(h, e, "gauss");
}

int gap_set_background(gap_handle *h, int32_t gap, double eta_bg) {
  if (!h || gap < 0 || gap >= h->n_gaps) return GAP_EINVAL;
  h->gaps_h[gap].eta_bg = eta_bg;
  cudaError_t e = cudaMemcpy(&h->v.gaps[gap].eta_bg, &eta_bg, sizeof(double), cudaMemcpyHostToDevice);
  return cuda_check(h, e, "set background");
}

// Shared by gap_get_particles (stride 1), gap_sample_particles and
// gap_tile_particles (tiles [tile_lo, tile_hi) of the gap; -1: all).
static int export_particles(gap_handle *h, int32_t gap, int32_t kind, int64_t stride, int64_t cap,
                            uint64_t *host_id, double *host_X, double *host_u, double *host_w,
                            double *host_tau, double *host_aux, int64_t *host_aux2, int64_t *n_out,
                            void *stream, int32_t tile_lo = -1, int32_t tile_hi = -1);

int gap_return_spectrum(gap_handle *h, int32_t gap, double *host_out, void *stream) {
  if (!h || gap < 0 || gap >= h->n_gaps || !host_out) return GAP_EINVAL;
  if (h->status) return h->status;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(host_out, h->v.ret_hist + (size_t)gap * kRetBins, sizeof(double) * kRetBins,
                                  cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return cuda_check(h, e, "return spectrum");
}

int gap_spectra(gap_handle *h, int32_t gap, int32_t nbins, double lo, double hi, double *host_leptons,
                double *host_photons, void *stream) {
  if (!h || gap < 0 || gap >= h->n_gaps || nbins < 1 || nbins > kSpecMaxBins || !(hi > lo)) return GAP_EINVAL;
  if (h->status) return h->status;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemsetAsync(h->v.spec_buf, 0, sizeof(double) * 3 * kSpecMaxBins, st);
  if (e == cudaSuccess) {
    launch_spectra(h->v, gap, h->gaps_h[gap].n_tiles, nbins, lo, hi, st);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && host_leptons) {
    e = cudaMemcpyAsync(host_leptons, h->v.spec_buf, sizeof(double) * nbins, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(host_leptons + nbins, h->v.spec_buf + kSpecMaxBins, sizeof(double) * nbins,
                          cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess && host_photons)
    e = cudaMemcpyAsync(host_photons, h->v.spec_buf + 2 * kSpecMaxBins, sizeof(double) * nbins,
                        cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return cuda_check(h, e, "spectra");
}

int gap_tile_particles(gap_handle *h, int32_t gap, int32_t kind, int32_t tile_lo, int32_t tile_hi, int64_t cap,
                       uint64_t *host_id, double *host_X, double *host_u, double *host_w, double *host_tau,
                       int64_t *n_out, void *stream) {
  if (!h || gap < 0 || gap >= h->n_gaps || kind == GAP_PHOTON || kind == GAP_PROTON) return GAP_EINVAL;
  if (tile_lo < 0 || tile_hi <= tile_lo || tile_hi > h->gaps_h[gap].n_tiles) return GAP_EINVAL;
  return export_particles(h, gap, kind, 1, cap, host_id, host_X, host_u, host_w, host_tau, nullptr, nullptr, n_out,
                          stream, tile_lo, tile_hi);
}

int gap_get_particles(gap_handle *h, int32_t gap, int32_t kind, int64_t cap, uint64_t *host_id,
                      double *host_X, double *host_u, double *host_w, double *host_tau, double *host_aux,
                      int64_t *host_aux2, int64_t *n_out, void *stream) {
  return export_particles(h, gap, kind, 1, cap, host_id, host_X, host_u, host_w, host_tau, host_aux,
                          host_aux2, n_out, stream);
}

int gap_sample_particles(gap_handle *h, int32_t gap, int32_t kind, int64_t stride, int64_t cap,
                         uint64_t *host_id, double *host_X, double *host_u, double *host_w, double *host_tau,
                         int64_t *n_out, void *stream) {
  if (kind == GAP_PHOTON || stride < 1) return GAP_EINVAL;
  return export_particles(h, gap, kind, stride, cap, host_id, host_X, host_u, host_w, host_tau, nullptr,
                          nullptr, n_out, stream);
}

static int export_particles(gap_handle *h, int32_t gap, int32_t kind, int64_t stride, int64_t cap,
                            uint64_t *host_id, double *host_X, double *host_u, double *host_w,
                            double *host_tau, double *host_aux, int64_t *host_aux2, int64_t *n_out,
                            void *stream, int32_t tile_lo, int32_t tile_hi) {
  if (!h || gap < 0 || gap >= h->n_gaps || kind < 0 || kind > GAP_PROTON || !n_out) return GAP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  Ctl c;
  int r = read_ctl(h, &c, st);
  if (r) return r;
  const int64_t scap = (int64_t)(h->buf_bytes / (8 * 7));
  double *stage = reinterpret_cast<double *>(h->buf_base[c.lep_cur ^ 1]);
  cudaError_t e = cudaMemsetAsync(h->export_count, 0, sizeof(unsigned long long), st);
  if (kind == GAP_PROTON)
    launch_export_protons(h->v, gap, stage, scap, h->export_count, stride, st);
  else
    launch_export_impl(h->v, gap, kind, stage, scap, h->export_count,
                       tile_lo >= 0 ? tile_hi - tile_lo : h->gaps_h[gap].n_tiles, st, stride,
                       tile_lo >= 0 ? tile_lo : 0);
  if (e == cudaSuccess) e = cudaGetLastError();
  unsigned long long cnt = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&cnt, h->export_count, sizeof(cnt), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_check(h, e, "export");
  *n_out = (int64_t)cnt;
  if ((int64_t)cnt > cap || (int64_t)cnt > scap) return GAP_ECAP;
  const size_t nb = sizeof(double) * cnt;
  struct { void *dst; int idx; } cp[7] = {{host_id, 0}, {host_X, 1}, {host_u, 2}, {host_w, 3},
                                          {nullptr, 4}, {nullptr, 5}, {nullptr, 6}};
  if (kind == GAP_PHOTON) {
    cp[4].dst = host_tau;   // tau_acc
    cp[5].dst = host_aux;   // tau_star
    cp[6].dst = host_aux2;  // (n0 << 1) | dir
  } else {
    cp[4].dst = host_tau;
  }
  for (auto &x : cp) {
    if (!x.dst || cnt == 0) continue;
    e = cudaMemcpyAsync(x.dst, stage + (size_t)x.idx * scap, nb, cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) break;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return cuda_check(h, e, "export copy");
}

int gap_add_particles(gap_handle *h, int32_t gap, int32_t kind, int64_t n, const uint64_t *host_id,
                      const double *host_X, const double *host_u, const double *host_w,
                      const double *host_tau, const int64_t *host_aux2, void *stream) {
  if (!h || gap < 0 || gap >= h->n_gaps || kind < 0 || kind > 2 || n < 0) return GAP_EINVAL;
  if (n == 0) return GAP_OK;
  if (!host_id || !host_X || !host_u || !host_w || !host_tau) return GAP_EINVAL;
  if (kind == GAP_PHOTON && !host_aux2) return GAP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  Ctl c;
  int r = read_ctl(h, &c, st);
  if (r) return r;
  const int64_t per = kind == GAP_PHOTON ? 7 : 5;
  if ((size_t)(n * per * 8) > h->buf_bytes) return GAP_ECAP;
  double *stage = reinterpret_cast<double *>(h->buf_base[c.lep_cur ^ 1]);
  const size_t nb = sizeof(double) * n;
  cudaError_t e = cudaMemcpyAsync(stage, host_id, nb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(stage + n, host_X, nb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(stage + 2 * n, host_u, nb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(stage + 3 * n, host_w, nb, cudaMemcpyHostToDevice, st);
  if (kind == GAP_PHOTON) {
    // photons: x in host_u, tau_star in host_tau (stage slot 5), tau_acc = 0
    if (e == cudaSuccess) e = cudaMemsetAsync(stage + 4 * n, 0, nb, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(stage + 5 * n, host_tau, nb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(stage + 6 * n, host_aux2, nb, cudaMemcpyHostToDevice, st);
  } else {
    if (e == cudaSuccess) e = cudaMemcpyAsync(stage + 4 * n, host_tau, nb, cudaMemcpyHostToDevice, st);
  }
  if (e != cudaSuccess) return cuda_check(h, e, "import copy");
  launch_import(h->v, gap, kind, n, stage, st);
  if (kind != GAP_PHOTON) {
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_check(h, e, "import");
    // fold the appended particles into the layout (the stage is the inactive
    // buffer, so the compaction runs after the import has finished)
    launch_sync_used(h->v, st);
    launch_force_rebin(h->v, st);
    launch_rebin(h->v, h->slack, st);
  }
  e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(h, e, "import");
  return read_ctl(h, &c, st);
}

int gap_diag(gap_handle *h, int32_t gap, gap_diag_out *out, double *host_spectrum, int64_t spectrum_cap,
             double *host_moments, void *stream) {
  if (!h || gap < 0 || gap >= h->n_gaps || !out) return GAP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  Ctl c;
  int r = read_ctl(h, &c, st);
  if (r) return r;
  const GapDev &g = h->gaps_h[gap];
  const int64_t ng = std::min<int64_t>((int64_t)std::floor(g.Hc) + 1, g.nnode);
  const int64_t P = next_pow2(ng);
  launch_diag(h->v, gap, g.nx, P, st);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_check(h, e, "diag launch");
  double red[32];
  e = cudaMemcpyAsync(red, h->v.dred, sizeof(red), cudaMemcpyDeviceToHost, st);
  std::vector<int32_t> alive[2];
  for (int s = 0; s < 2 && e == cudaSuccess; ++s) {
    alive[s].resize(g.n_tiles);
    e = cudaMemcpyAsync(alive[s].data(), h->v.seg_alive[s] + g.tile_begin, sizeof(int32_t) * g.n_tiles,
                        cudaMemcpyDeviceToHost, st);
  }
  unsigned long long cnt[C_NCNT];
  double led[L_NLED];
  if (e == cudaSuccess) e = cudaMemcpyAsync(cnt, h->v.counters + (size_t)gap * C_NCNT, sizeof(cnt), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(led, h->v.ledger + (size_t)gap * L_NLED, sizeof(led), cudaMemcpyDeviceToHost, st);
  if (host_spectrum && e == cudaSuccess) {
    const int64_t ns = std::min<int64_t>(spectrum_cap, P / 2 + 1);
    e = cudaMemcpyAsync(host_spectrum, h->v.fft[1], sizeof(double) * ns, cudaMemcpyDeviceToHost, st);
  }
  std::vector<unsigned long long> qbits;
  if (host_moments && e == cudaSuccess) {
    e = cudaMemcpyAsync(host_moments, h->v.dmom, sizeof(double) * 8 * g.nx, cudaMemcpyDeviceToHost, st);
    qbits.resize(g.nx);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(qbits.data(), h->v.dcharge, sizeof(unsigned long long) * g.nx, cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_check(h, e, "diag");
  if (host_moments) {
    for (int64_t i = 0; i < g.nx; ++i) {
      double q;
      if (h->precision == GAP_FP32_STATE) q = (double)(long long)qbits[i] * g.w_unit * kPhiUnit;
      else std::memcpy(&q, &qbits[i], sizeof(double));
      host_moments[6 * g.nx + i] = q;
    }
  }
  std::memset(out, 0, sizeof(*out));
  out->step = c.step;
  int64_t ne = 0, np = 0;
  for (int t = 0; t < g.n_tiles; ++t) { ne += alive[0][t]; np += alive[1][t]; }
  out->n_electrons = ne;
  out->n_positrons = np;
  unsigned long long phc;
  std::memcpy(&phc, &red[20], sizeof(phc));
  out->n_photons = (int64_t)phc;
  out->M_peak = red[0];
  out->M_avg = red[1];
  out->peak_cell = (int64_t)red[2];
  out->g3_peak = red[3];
  for (int q = 0; q < 4; ++q) out->M_split[q] = red[4 + q];
  out->E_min = red[8];
  out->E_max = red[9];
  out->gauss_residual = red[10];
  out->E_abs_max = red[11];
  out->field_energy = red[12];
  out->lepton_energy = red[16];
  out->photon_energy = red[17];
  out->spectrum_len = P / 2 + 1;
  int64_t *ci = &out->counters.emit_events;
  for (int q = 0; q < 16; ++q) ci[q] = (int64_t)cnt[q];
  double *cd = &out->counters.e_radiated;
  for (int q = 0; q < 8; ++q) cd[q] = led[q];
  return GAP_OK;
}

int gap_spectrum_inverse(gap_handle *h, const double *dev_U, double *dev_xi, int64_t n, int32_t precision,
                         void *stream) {
  if (!h || n < 0 || (n > 0 && (!dev_U || !dev_xi))) return GAP_EINVAL;
  if (precision != GAP_FP64_PLAIN && precision != GAP_FP32_STATE) return GAP_EINVAL;
  launch_spec_inverse(h->v, dev_U, dev_xi, n, precision == GAP_FP32_STATE, (cudaStream_t)stream);
  return cuda_check(h, cudaGetLastError(), "spectrum inverse");
}

int gap_qspectrum_inverse(gap_handle *h, const double *dev_chi, const double *dev_U, double *dev_xi, int64_t n,
                          int32_t precision, void *stream) {
  if (!h || n < 0 || (n > 0 && (!dev_chi || !dev_U || !dev_xi))) return GAP_EINVAL;
  if (precision != GAP_FP64_PLAIN && precision != GAP_FP32_STATE) return GAP_EINVAL;
  if (!h->v.qs_any) return fail(h, GAP_EINVAL, "no gap of this handle has qed_quantum");
  launch_qspec_inverse(h->v, dev_chi, dev_U, dev_xi, n, precision == GAP_FP32_STATE, (cudaStream_t)stream);
  return cuda_check(h, cudaGetLastError(), "quantum spectrum inverse");
}

int gap_pair_split(gap_handle *h, const double *dev_chi, const double *dev_U, double *dev_e, int64_t n,
                   void *stream) {
  if (!h || n < 0 || (n > 0 && (!dev_chi || !dev_U || !dev_e))) return GAP_EINVAL;
  if (!h->v.qs_any) return fail(h, GAP_EINVAL, "no gap of this handle has qed_quantum");
  launch_pair_split(h->v, dev_chi, dev_U, dev_e, n, (cudaStream_t)stream);
  return cuda_check(h, cudaGetLastError(), "pair split");
}

int64_t gap_steps_done(const gap_handle *h) { return h ? h->steps_done : 0; }

size_t gap_state_bytes(const gap_handle *h) { return h ? h->ws_need : 0; }

int gap_save(gap_handle *h, void *host_dst, size_t bytes, void *stream) {
  if (!h || !host_dst) return GAP_EINVAL;
  if (h->status) return h->status;
  if (bytes < h->ws_need) return GAP_ENOSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(host_dst, h->ws, h->ws_need, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return cuda_check(h, e, "save");
}

int gap_load(gap_handle *h, const void *host_src, size_t bytes, void *stream) {
  if (!h || !host_src || bytes != h->ws_need) return GAP_EINVAL;
  // the gap and tile tables follow from the parameters and the configuration;
  // a state from another layout is refused before anything is copied (only
  // the mutable background density of a gap may differ)
  const char *src = static_cast<const char *>(host_src);
  const size_t og = (size_t)(reinterpret_cast<char *>(h->v.gaps) - h->ws);
  const size_t ot = (size_t)(reinterpret_cast<char *>(h->v.tiles) - h->ws);
  std::vector<GapDev> gs((size_t)h->n_gaps);
  std::memcpy(gs.data(), src + og, sizeof(GapDev) * gs.size());
  for (size_t i = 0; i < gs.size(); ++i) {
    GapDev a = gs[i], b = h->gaps_h[i];
    a.eta_bg = b.eta_bg = 0.0;
    if (std::memcmp(&a, &b, sizeof(GapDev)) != 0) return GAP_EINVAL;
  }
  if (std::memcmp(src + ot, h->tiles_h.data(), sizeof(TileDev) * h->tiles_h.size()) != 0) return GAP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaMemcpyAsync(h->ws, host_src, h->ws_need, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_check(h, e, "load");
  for (size_t i = 0; i < gs.size(); ++i) h->gaps_h[i].eta_bg = gs[i].eta_bg;
  h->status = GAP_OK;
  h->err.clear();
  Ctl c;
  const int r = read_ctl(h, &c, st);
  if (r) return r;
  h->steps_done = c.step;
  return GAP_OK;
}

// Sum the event intervals recorded since the last read into phase_ms.
static int collect_phases(gap_handle *h) {
  if (!h->ev_used) return GAP_OK;
  cudaError_t e = cudaEventSynchronize(h->ev[h->ev_used - 1]);
  if (e != cudaSuccess) return cuda_check(h, e, "profile sync");
  // the phase of each interval between consecutive events
  static const int phase_of[GAP_NPHASES] = {GAP_PHASE_PUSH, GAP_PHASE_PUSH_TAIL, GAP_PHASE_AFTER, GAP_PHASE_REBIN,
                                            GAP_PHASE_MERGE};
  for (size_t i = 0; i + kProfEvents <= h->ev_used; i += kProfEvents) {
    for (int k = 0; k < GAP_NPHASES; ++k) {
      const int ph = phase_of[k];
      float ms = 0.f;
      e = cudaEventElapsedTime(&ms, h->ev[i + k], h->ev[i + k + 1]);
      if (e != cudaSuccess) return cuda_check(h, e, "profile read");
      h->phase_ms[ph] += ms;
    }
    ++h->phase_steps;
  }
  h->ev_used = 0;
  return GAP_OK;
}

int gap_profile(gap_handle *h, int32_t on, double *push_ms_total, int64_t *push_launches,
                int64_t *launches_per_step) {
  if (!h) return GAP_EINVAL;
  if (launches_per_step) *launches_per_step = ::gapk::launches_per_step(h->v);
  const int r = collect_phases(h);
  if (r) return r;
  const double tot = h->phase_ms[GAP_PHASE_PUSH];
  const int64_t n = h->phase_steps;
  for (int ph = 0; ph < GAP_NPHASES; ++ph) h->phase_ms[ph] = 0.0;
  h->phase_steps = 0;
  if (push_ms_total) *push_ms_total = tot;
  if (push_launches) *push_launches = n;
  h->profiling = on != 0;
  return GAP_OK;
}

int gap_defer_limit(gap_handle *h, int64_t n) {
  if (!h || n < 0) return GAP_EINVAL;
  h->v.defer_use = std::min<int64_t>(n, h->v.defer_cap);
  return GAP_OK;
}

int gap_hold_copies(gap_handle *h, int32_t on) {
  if (!h) return GAP_EINVAL;
  const int32_t flag = on != 0;
  return cuda_check(h, cudaMemcpy(&h->v.ctl->hold_copies, &flag, sizeof(flag), cudaMemcpyHostToDevice),
                    "hold copies");
}

int gap_profile_phases(gap_handle *h, double *ms_out, int64_t *steps_out) {
  if (!h || !ms_out) return GAP_EINVAL;
  const int r = collect_phases(h);
  if (r) return r;
  for (int ph = 0; ph < GAP_NPHASES; ++ph) ms_out[ph] = h->phase_ms[ph];
  if (steps_out) *steps_out = h->phase_steps;
  return GAP_OK;
}

void gap_free(gap_handle *h) {
  if (!h) return;
  if (h->graph) cudaGraphExecDestroy(h->graph);
  for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
  if (h->fa_after_steps) cudaEventDestroy(h->fa_after_steps);
  if (h->fa_after_stage) cudaEventDestroy(h->fa_after_stage);
  delete h;
}

const char *gap_last_error(const gap_handle *h) { return h ? h->err.c_str() : "null handle"; }

const char *gap_status_string(int s) {
  switch (s) {
    case GAP_OK: return "ok";
    case GAP_EINVAL: return "invalid argument";
    case GAP_ENOSPACE: return "workspace too small";
    case GAP_ECAP: return "particle storage exhausted";
    case GAP_ETIMEOUT: return "device wait timed out";
    case GAP_ECUDA: return "CUDA error";
    case GAP_ECHECK: return "device consistency check failed";
    case GAP_ETOOBIG: return "input larger than the fixed internal buffer (spectrum: n <= 32768)";
    default: return "unknown status";
  }
}

}  // extern "C"
