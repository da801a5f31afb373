// ode.cu -- batched RK4 integrator of the discharge concurrency model
// (Sect. 5.2, eq. dis1-dis4, units t_esc = 1) and its discrete adjoint.
//
//   dm/dt   = 2 m_x/t_pm - m
//   dm_x/dt = -m_x/t_pm + H(|eps| - 1) m/t_x - m_x
//   deps/dt = alpha - j
//   dj/dt   = -j + m eps g3/t_acc
//
// and, as an option, the extended model with the inertia density
// G = m <gamma^-3> as a fifth state (a moment of the 1D Vlasov equation with
// a cold-beam closure, pair birth at gamma_min and curvature losses):
//
//   dj/dt   = -j + eps G/t_acc
//   dG/dt   = 2 gamma_min^-3 m_x/t_pm - G - 3 eps j (G/m)^(4/3)/t_acc
//             + 3 m/(gamma_rad^4 t_acc)
//
// One thread integrates one parameter set.  The adjoint is the exact
// reverse-mode derivative of the RK4 map (not of the continuous ODE), so it
// agrees with finite differences of the forward kernel to rounding.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/gap.h"

namespace {

template <class R>
struct Model {
  static constexpr int NY = 4, NP = 5;
  R alpha, tx, tpm, tacc, g3, delta;
  // reciprocals and the ratio g3/t_acc, formed once per set: the right-hand
  // side then has no division (FP64 division is a long dependent sequence)
  R itx, itpm, itacc, gt, idelta;
  __device__ __forceinline__ R gate(R z) const {
    if (delta == (R)0) return z > (R)0 ? (R)1 : (R)0;
    return (R)0.5 * ((R)1 + tanh(z * idelta));
  }
  __device__ __forceinline__ R dgate(R z) const {
    if (delta == (R)0) return (R)0;
    const R th = tanh(z * idelta);
    return ((R)1 - th * th) * ((R)0.5 * idelta);
  }
  __device__ __forceinline__ void f(const R y[4], R k[4]) const {
    const R H = gate(fabs(y[2]) - (R)1);
    k[0] = (R)2 * y[1] * itpm - y[0];
    k[1] = -y[1] * itpm + H * y[0] * itx - y[1];
    k[2] = alpha - y[3];
    k[3] = -y[3] + y[0] * y[2] * gt;
  }
  // lam_y += J(y)^T a ; lam_p += Jp(y)^T a
  __device__ __forceinline__ void vjp(const R y[4], const R a[4], R ly[4], R lp[5]) const {
    const R z = fabs(y[2]) - (R)1;
    const R H = gate(z);
    const R sg = y[2] > (R)0 ? (R)1 : (y[2] < (R)0 ? (R)-1 : (R)0);
    const R dH = dgate(z) * sg;
    ly[0] += -a[0] + a[1] * H * itx + a[3] * y[2] * gt;
    ly[1] += a[0] * (R)2 * itpm + a[1] * (-itpm - (R)1);
    ly[2] += a[1] * dH * y[0] * itx + a[3] * y[0] * gt;
    ly[3] += -a[2] - a[3];
    lp[0] += a[2];
    lp[1] += -a[1] * H * y[0] * (itx * itx);
    lp[2] += (-a[0] * (R)2 * y[1] + a[1] * y[1]) * (itpm * itpm);
    lp[3] += -a[3] * y[0] * y[2] * gt * itacc;
    lp[4] += a[3] * y[0] * y[2] * itacc;
  }
  static __device__ __forceinline__ Model load(const R *p, int b, double delta) {
    Model m;
    m.alpha = p[5 * b + 0];
    m.tx = p[5 * b + 1];
    m.tpm = p[5 * b + 2];
    m.tacc = p[5 * b + 3];
    m.g3 = p[5 * b + 4];
    m.delta = (R)delta;
    m.itx = (R)1 / m.tx;
    m.itpm = (R)1 / m.tpm;
    m.itacc = (R)1 / m.tacc;
    m.gt = m.g3 / m.tacc;
    m.idelta = m.delta != (R)0 ? (R)1 / m.delta : (R)0;
    return m;
  }
};

// The extended model: state (m, m_x, eps, j, G), parameters (alpha, t_x,
// t_pm, t_acc, gamma_min, gamma_rad).  (G/m)^(4/3) is taken of max(G, 0).
template <class R>
struct ModelExt {
  static constexpr int NY = 5, NP = 6;
  R alpha, tx, tpm, tacc, gmin, grad, delta;
  // reciprocals, the pair-birth source 2 gamma_min^-3 / t_pm and the
  // radiative rate 3 / (gamma_rad^4 t_acc) of <gamma^-3>, formed once per set
  R itx, itpm, itacc, idelta, src, rad;
  __device__ __forceinline__ R gate(R z) const {
    if (delta == (R)0) return z > (R)0 ? (R)1 : (R)0;
    return (R)0.5 * ((R)1 + tanh(z * idelta));
  }
  __device__ __forceinline__ R dgate(R z) const {
    if (delta == (R)0) return (R)0;
    const R th = tanh(z * idelta);
    return ((R)1 - th * th) * ((R)0.5 * idelta);
  }
  // (G/m)^(1/3) of the non-negative part of G
  __device__ __forceinline__ R cube_root_g3(R G, R m) const { return G > (R)0 ? cbrt(G / m) : (R)0; }
  __device__ __forceinline__ void f(const R y[5], R k[5]) const {
    const R H = gate(fabs(y[2]) - (R)1);
    const R c = cube_root_g3(y[4], y[0]), c4 = (c * c) * (c * c);
    k[0] = (R)2 * y[1] * itpm - y[0];
    k[1] = -y[1] * itpm + H * y[0] * itx - y[1];
    k[2] = alpha - y[3];
    k[3] = -y[3] + y[2] * y[4] * itacc;
    k[4] = src * y[1] - y[4] - (R)3 * y[2] * y[3] * c4 * itacc + rad * y[0];
  }
  __device__ __forceinline__ void vjp(const R y[5], const R a[5], R ly[5], R lp[6]) const {
    const R z = fabs(y[2]) - (R)1;
    const R H = gate(z);
    const R sg = y[2] > (R)0 ? (R)1 : (y[2] < (R)0 ? (R)-1 : (R)0);
    const R dH = dgate(z) * sg;
    const R c = cube_root_g3(y[4], y[0]), c4 = (c * c) * (c * c);
    const R im = (R)1 / y[0];
    const R dc4_dG = (R)4 / (R)3 * c * im;        // d (G/m)^(4/3) / dG
    const R dc4_dm = -(R)4 / (R)3 * c4 * im;      // d (G/m)^(4/3) / dm
    const R acc = (R)3 * y[2] * y[3] * itacc;      // the acceleration term is acc (G/m)^(4/3)
    ly[0] += -a[0] + a[1] * H * itx + a[4] * (rad - acc * dc4_dm);
    ly[1] += a[0] * (R)2 * itpm + a[1] * (-itpm - (R)1) + a[4] * src;
    ly[2] += a[1] * dH * y[0] * itx + a[3] * y[4] * itacc - a[4] * (R)3 * y[3] * c4 * itacc;
    ly[3] += -a[2] - a[3] - a[4] * (R)3 * y[2] * c4 * itacc;
    ly[4] += a[3] * y[2] * itacc + a[4] * (-(R)1 - acc * dc4_dG);
    lp[0] += a[2];
    lp[1] += -a[1] * H * y[0] * (itx * itx);
    lp[2] += (-a[0] * (R)2 * y[1] + a[1] * y[1]) * (itpm * itpm) - a[4] * src * y[1] * itpm;
    lp[3] += (-a[3] * y[2] * y[4] * itacc + a[4] * (acc * c4 - rad * y[0])) * itacc;
    lp[4] += -a[4] * (R)3 * src * y[1] / gmin;
    lp[5] += -a[4] * (R)4 * rad * y[0] / grad;
  }
  static __device__ __forceinline__ ModelExt load(const R *p, int b, double delta) {
    ModelExt m;
    m.alpha = p[6 * b + 0];
    m.tx = p[6 * b + 1];
    m.tpm = p[6 * b + 2];
    m.tacc = p[6 * b + 3];
    m.gmin = p[6 * b + 4];
    m.grad = p[6 * b + 5];
    m.delta = (R)delta;
    m.itx = (R)1 / m.tx;
    m.itpm = (R)1 / m.tpm;
    m.itacc = (R)1 / m.tacc;
    m.idelta = m.delta != (R)0 ? (R)1 / m.delta : (R)0;
    m.src = (R)2 / (m.gmin * m.gmin * m.gmin) * m.itpm;
    const R g2 = m.grad * m.grad;
    m.rad = (R)3 / (g2 * g2) * m.itacc;
    return m;
  }
};

// One classical RK4 step of model M, and its reverse-mode adjoint: given lam
// (the adjoint of y_{n+1}) and y = y_n, lam becomes the adjoint of y_n and lp
// accumulates dL/dp.
template <class M, class R>
__device__ __forceinline__ void rk4_step(const M &m, R y[M::NY], R h) {
  constexpr int N = M::NY;
  R k1[N], k2[N], k3[N], k4[N], t[N];
  m.f(y, k1);
  for (int i = 0; i < N; ++i) t[i] = y[i] + (R)0.5 * h * k1[i];
  m.f(t, k2);
  for (int i = 0; i < N; ++i) t[i] = y[i] + (R)0.5 * h * k2[i];
  m.f(t, k3);
  for (int i = 0; i < N; ++i) t[i] = y[i] + h * k3[i];
  m.f(t, k4);
  for (int i = 0; i < N; ++i) y[i] += h / (R)6 * (k1[i] + (R)2 * k2[i] + (R)2 * k3[i] + k4[i]);
}

template <class M, class R>
__device__ __forceinline__ void rk4_step_adjoint(const M &m, const R y[M::NY], R h, R lam[M::NY], R lp[M::NP]) {
  constexpr int N = M::NY;
  R k1[N], k2[N], k3[N], y2[N], y3[N], y4[N];
  m.f(y, k1);
  for (int i = 0; i < N; ++i) y2[i] = y[i] + (R)0.5 * h * k1[i];
  m.f(y2, k2);
  for (int i = 0; i < N; ++i) y3[i] = y[i] + (R)0.5 * h * k2[i];
  m.f(y3, k3);
  for (int i = 0; i < N; ++i) y4[i] = y[i] + h * k3[i];
  R a1[N], a2[N], a3[N], a4[N], ly[N], t[N];
  for (int i = 0; i < N; ++i) {
    a1[i] = h / (R)6 * lam[i];
    a2[i] = h / (R)3 * lam[i];
    a3[i] = h / (R)3 * lam[i];
    a4[i] = h / (R)6 * lam[i];
    ly[i] = lam[i];
  }
  for (int i = 0; i < N; ++i) t[i] = 0;
  m.vjp(y4, a4, t, lp);  // t = J(y4)^T a4
  for (int i = 0; i < N; ++i) { ly[i] += t[i]; a3[i] += h * t[i]; t[i] = 0; }
  m.vjp(y3, a3, t, lp);
  for (int i = 0; i < N; ++i) { ly[i] += t[i]; a2[i] += (R)0.5 * h * t[i]; t[i] = 0; }
  m.vjp(y2, a2, t, lp);
  for (int i = 0; i < N; ++i) { ly[i] += t[i]; a1[i] += (R)0.5 * h * t[i]; t[i] = 0; }
  m.vjp(y, a1, t, lp);
  for (int i = 0; i < N; ++i) lam[i] = ly[i] + t[i];
}


template <class M, class R>
__global__ void k_ode_forward(const R *p, const R *y0, const R *dt, int B, int nsteps, int every,
                              int ckpt_every, double delta, R *out, R *ckpt) {
  constexpr int N = M::NY;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const M m = M::load(p, b, delta);
  const R h = dt[b];
  R y[N];
  for (int i = 0; i < N; ++i) {
    y[i] = y0[N * b + i];
    out[N * b + i] = y[i];
    if (ckpt) ckpt[N * b + i] = y[i];
  }
  for (int n = 0; n < nsteps; ++n) {
    rk4_step(m, y, h);
    if ((n + 1) % every == 0) {
      const int64_t o = ((int64_t)((n + 1) / every) * B + b) * N;
      for (int i = 0; i < N; ++i) out[o + i] = y[i];
    }
    if (ckpt && (n + 1) % ckpt_every == 0) {
      const int64_t o = ((int64_t)((n + 1) / ckpt_every) * B + b) * N;
      for (int i = 0; i < N; ++i) ckpt[o + i] = y[i];
    }
  }
}

template <class M, class R>
__global__ void k_ode_adjoint(const R *p, const R *dt, const R *ckpt, const R *gout, int B, int nsteps,
                              int every, int ckpt_every, double delta, R *gp, R *gy0, R *scratch) {
  constexpr int N = M::NY, NP = M::NP;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const M m = M::load(p, b, delta);
  const R h = dt[b];
  R lam[N], lp[NP];
  for (int i = 0; i < N; ++i) lam[i] = 0;
  for (int i = 0; i < NP; ++i) lp[i] = 0;
  const int nseg = (nsteps + ckpt_every - 1) / ckpt_every;
  for (int seg = nseg - 1; seg >= 0; --seg) {
    const int n0 = seg * ckpt_every;
    const int n1 = n0 + ckpt_every < nsteps ? n0 + ckpt_every : nsteps;
    // recompute y_n for n in [n0, n1) into scratch[(n - n0)][b]
    R y[N];
    for (int i = 0; i < N; ++i) y[i] = ckpt[((int64_t)seg * B + b) * N + i];
    for (int n = n0; n < n1; ++n) {
      const int64_t o = ((int64_t)(n - n0) * B + b) * N;
      for (int i = 0; i < N; ++i) scratch[o + i] = y[i];
      rk4_step(m, y, h);
    }
    for (int n = n1 - 1; n >= n0; --n) {
      if ((n + 1) % every == 0) {
        const int64_t o = ((int64_t)((n + 1) / every) * B + b) * N;
        for (int i = 0; i < N; ++i) lam[i] += gout[o + i];
      }
      const int64_t o = ((int64_t)(n - n0) * B + b) * N;
      for (int i = 0; i < N; ++i) y[i] = scratch[o + i];
      rk4_step_adjoint(m, y, h, lam, lp);
    }
  }
  for (int i = 0; i < N; ++i) gy0[N * b + i] = lam[i] + gout[N * b + i];
  for (int i = 0; i < NP; ++i) gp[NP * b + i] = lp[i];
}

template <template <class> class M>
int launch_forward(const void *dev_p, const void *dev_y0, const void *dev_dt, int32_t B, int32_t nsteps,
                   int32_t every, int32_t ckpt_every, double delta, int32_t dtype, void *dev_out, void *dev_ckpt,
                   void *stream) {
  if (!dev_p || !dev_y0 || !dev_dt || !dev_out || B <= 0 || nsteps < 0 || every <= 0 ||
      (dev_ckpt && ckpt_every <= 0) || delta < 0)
    return GAP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  // one thread per parameter set; small batches spread over more SMs
  const int threads = B >= 148 * 64 ? 64 : 32, blocks = (B + threads - 1) / threads;
  if (dtype == 0)
    k_ode_forward<M<double>, double><<<blocks, threads, 0, st>>>(
        (const double *)dev_p, (const double *)dev_y0, (const double *)dev_dt, B, nsteps, every, ckpt_every, delta,
        (double *)dev_out, (double *)dev_ckpt);
  else if (dtype == 1)
    k_ode_forward<M<float>, float><<<blocks, threads, 0, st>>>(
        (const float *)dev_p, (const float *)dev_y0, (const float *)dev_dt, B, nsteps, every, ckpt_every, delta,
        (float *)dev_out, (float *)dev_ckpt);
  else
    return GAP_EINVAL;
  return cudaGetLastError() == cudaSuccess ? GAP_OK : GAP_ECUDA;
}

template <template <class> class M>
int launch_adjoint(const void *dev_p, const void *dev_dt, const void *dev_ckpt, const void *dev_gout, int32_t B,
                   int32_t nsteps, int32_t every, int32_t ckpt_every, double delta, int32_t dtype, void *dev_gp,
                   void *dev_gy0, void *dev_scratch, void *stream) {
  if (!dev_p || !dev_dt || !dev_ckpt || !dev_gout || !dev_gp || !dev_gy0 || !dev_scratch || B <= 0 ||
      nsteps < 0 || every <= 0 || ckpt_every <= 0 || delta < 0)
    return GAP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const int threads = B >= 148 * 64 ? 64 : 32, blocks = (B + threads - 1) / threads;
  if (dtype == 0)
    k_ode_adjoint<M<double>, double><<<blocks, threads, 0, st>>>(
        (const double *)dev_p, (const double *)dev_dt, (const double *)dev_ckpt, (const double *)dev_gout, B,
        nsteps, every, ckpt_every, delta, (double *)dev_gp, (double *)dev_gy0, (double *)dev_scratch);
  else if (dtype == 1)
    k_ode_adjoint<M<float>, float><<<blocks, threads, 0, st>>>(
        (const float *)dev_p, (const float *)dev_dt, (const float *)dev_ckpt, (const float *)dev_gout, B,
        nsteps, every, ckpt_every, delta, (float *)dev_gp, (float *)dev_gy0, (float *)dev_scratch);
  else
    return GAP_EINVAL;
  return cudaGetLastError() == cudaSuccess ? GAP_OK : GAP_ECUDA;
}

}  // namespace

extern "C" int ode_forward(const void *dev_p, const void *dev_y0, const void *dev_dt, int32_t B,
                           int32_t nsteps, int32_t every, int32_t ckpt_every, double delta, int32_t dtype,
                           void *dev_out, void *dev_ckpt, void *stream) {
  return launch_forward<Model>(dev_p, dev_y0, dev_dt, B, nsteps, every, ckpt_every, delta, dtype, dev_out, dev_ckpt,
                               stream);
}

extern "C" int ode_adjoint(const void *dev_p, const void *dev_dt, const void *dev_ckpt, const void *dev_gout,
                           int32_t B, int32_t nsteps, int32_t every, int32_t ckpt_every, double delta,
                           int32_t dtype, void *dev_gp, void *dev_gy0, void *dev_scratch, void *stream) {
  return launch_adjoint<Model>(dev_p, dev_dt, dev_ckpt, dev_gout, B, nsteps, every, ckpt_every, delta, dtype, dev_gp,
                               dev_gy0, dev_scratch, stream);
}

extern "C" int ode_ext_forward(const void *dev_p, const void *dev_y0, const void *dev_dt, int32_t B,
                               int32_t nsteps, int32_t every, int32_t ckpt_every, double delta, int32_t dtype,
                               void *dev_out, void *dev_ckpt, void *stream) {
  return launch_forward<ModelExt>(dev_p, dev_y0, dev_dt, B, nsteps, every, ckpt_every, delta, dtype, dev_out,
                                  dev_ckpt, stream);
}

extern "C" int ode_ext_adjoint(const void *dev_p, const void *dev_dt, const void *dev_ckpt, const void *dev_gout,
                               int32_t B, int32_t nsteps, int32_t every, int32_t ckpt_every, double delta,
                               int32_t dtype, void *dev_gp, void *dev_gy0, void *dev_scratch, void *stream) {
  return launch_adjoint<ModelExt>(dev_p, dev_dt, dev_ckpt, dev_gout, B, nsteps, every, ckpt_every, delta, dtype,
                                  dev_gp, dev_gy0, dev_scratch, stream);
}
