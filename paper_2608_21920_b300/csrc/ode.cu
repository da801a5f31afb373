// ode.cu -- batched RK4 integrator of the discharge concurrency model
// (Sect. 5.2, eq. dis1-dis4, units t_esc = 1) and its discrete adjoint.
//
//   dm/dt   = 2 m_x/t_pm - m
//   dm_x/dt = -m_x/t_pm + H(|eps| - 1) m/t_x - m_x
//   deps/dt = alpha - j
//   dj/dt   = -j + m eps g3/t_acc
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
  __device__ __forceinline__ void step(R y[4], R h) const {
    R k1[4], k2[4], k3[4], k4[4], t[4];
    f(y, k1);
    for (int i = 0; i < 4; ++i) t[i] = y[i] + (R)0.5 * h * k1[i];
    f(t, k2);
    for (int i = 0; i < 4; ++i) t[i] = y[i] + (R)0.5 * h * k2[i];
    f(t, k3);
    for (int i = 0; i < 4; ++i) t[i] = y[i] + h * k3[i];
    f(t, k4);
    for (int i = 0; i < 4; ++i) y[i] += h / (R)6 * (k1[i] + (R)2 * k2[i] + (R)2 * k3[i] + k4[i]);
  }
  // Given lam (adjoint of y_{n+1}) and y = y_n: lam <- adjoint of y_n; lp += dL/dp.
  __device__ __forceinline__ void step_adjoint(const R y[4], R h, R lam[4], R lp[5]) const {
    R k1[4], k2[4], k3[4], y2[4], y3[4], y4[4];
    f(y, k1);
    for (int i = 0; i < 4; ++i) y2[i] = y[i] + (R)0.5 * h * k1[i];
    f(y2, k2);
    for (int i = 0; i < 4; ++i) y3[i] = y[i] + (R)0.5 * h * k2[i];
    f(y3, k3);
    for (int i = 0; i < 4; ++i) y4[i] = y[i] + h * k3[i];
    R a1[4], a2[4], a3[4], a4[4], ly[4], t[4];
    for (int i = 0; i < 4; ++i) {
      a1[i] = h / (R)6 * lam[i];
      a2[i] = h / (R)3 * lam[i];
      a3[i] = h / (R)3 * lam[i];
      a4[i] = h / (R)6 * lam[i];
      ly[i] = lam[i];
    }
    for (int i = 0; i < 4; ++i) t[i] = 0;
    vjp(y4, a4, t, lp);  // t = J(y4)^T a4
    for (int i = 0; i < 4; ++i) { ly[i] += t[i]; a3[i] += h * t[i]; t[i] = 0; }
    vjp(y3, a3, t, lp);
    for (int i = 0; i < 4; ++i) { ly[i] += t[i]; a2[i] += (R)0.5 * h * t[i]; t[i] = 0; }
    vjp(y2, a2, t, lp);
    for (int i = 0; i < 4; ++i) { ly[i] += t[i]; a1[i] += (R)0.5 * h * t[i]; t[i] = 0; }
    vjp(y, a1, t, lp);
    for (int i = 0; i < 4; ++i) lam[i] = ly[i] + t[i];
  }
};

template <class R>
__device__ __forceinline__ Model<R> load_model(const R *p, int b, double delta) {
  Model<R> m;
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

template <class R>
__global__ void k_ode_forward(const R *p, const R *y0, const R *dt, int B, int nsteps, int every,
                              int ckpt_every, double delta, R *out, R *ckpt) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const Model<R> m = load_model(p, b, delta);
  const R h = dt[b];
  R y[4];
  for (int i = 0; i < 4; ++i) {
    y[i] = y0[4 * b + i];
    out[4 * b + i] = y[i];
    if (ckpt) ckpt[4 * b + i] = y[i];
  }
  for (int n = 0; n < nsteps; ++n) {
    m.step(y, h);
    if ((n + 1) % every == 0) {
      const int64_t o = ((int64_t)((n + 1) / every) * B + b) * 4;
      for (int i = 0; i < 4; ++i) out[o + i] = y[i];
    }
    if (ckpt && (n + 1) % ckpt_every == 0) {
      const int64_t o = ((int64_t)((n + 1) / ckpt_every) * B + b) * 4;
      for (int i = 0; i < 4; ++i) ckpt[o + i] = y[i];
    }
  }
}

template <class R>
__global__ void k_ode_adjoint(const R *p, const R *dt, const R *ckpt, const R *gout, int B, int nsteps,
                              int every, int ckpt_every, double delta, R *gp, R *gy0, R *scratch) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const Model<R> m = load_model(p, b, delta);
  const R h = dt[b];
  R lam[4] = {0, 0, 0, 0}, lp[5] = {0, 0, 0, 0, 0};
  const int nseg = (nsteps + ckpt_every - 1) / ckpt_every;
  for (int seg = nseg - 1; seg >= 0; --seg) {
    const int n0 = seg * ckpt_every;
    const int n1 = n0 + ckpt_every < nsteps ? n0 + ckpt_every : nsteps;
    // recompute y_n for n in [n0, n1) into scratch[(n - n0)][b]
    R y[4];
    for (int i = 0; i < 4; ++i) y[i] = ckpt[((int64_t)seg * B + b) * 4 + i];
    for (int n = n0; n < n1; ++n) {
      const int64_t o = ((int64_t)(n - n0) * B + b) * 4;
      for (int i = 0; i < 4; ++i) scratch[o + i] = y[i];
      m.step(y, h);
    }
    for (int n = n1 - 1; n >= n0; --n) {
      if ((n + 1) % every == 0) {
        const int64_t o = ((int64_t)((n + 1) / every) * B + b) * 4;
        for (int i = 0; i < 4; ++i) lam[i] += gout[o + i];
      }
      const int64_t o = ((int64_t)(n - n0) * B + b) * 4;
      for (int i = 0; i < 4; ++i) y[i] = scratch[o + i];
      m.step_adjoint(y, h, lam, lp);
    }
  }
  for (int i = 0; i < 4; ++i) gy0[4 * b + i] = lam[i] + gout[4 * b + i];
  for (int i = 0; i < 5; ++i) gp[5 * b + i] = lp[i];
}

}  // namespace

extern "C" int ode_forward(const void *dev_p, const void *dev_y0, const void *dev_dt, int32_t B,
                           int32_t nsteps, int32_t every, int32_t ckpt_every, double delta, int32_t dtype,
                           void *dev_out, void *dev_ckpt, void *stream) {
  if (!dev_p || !dev_y0 || !dev_dt || !dev_out || B <= 0 || nsteps < 0 || every <= 0 ||
      (dev_ckpt && ckpt_every <= 0) || delta < 0)
    return GAP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  // one thread per parameter set; small batches spread over more SMs
  const int threads = B >= 148 * 64 ? 64 : 32, blocks = (B + threads - 1) / threads;
  if (dtype == 0)
    k_ode_forward<double><<<blocks, threads, 0, st>>>((const double *)dev_p, (const double *)dev_y0,
                                                      (const double *)dev_dt, B, nsteps, every,
                                                      ckpt_every, delta, (double *)dev_out, (double *)dev_ckpt);
  else if (dtype == 1)
    k_ode_forward<float><<<blocks, threads, 0, st>>>((const float *)dev_p, (const float *)dev_y0,
                                                     (const float *)dev_dt, B, nsteps, every, ckpt_every,
                                                     delta, (float *)dev_out, (float *)dev_ckpt);
  else
    return GAP_EINVAL;
  return cudaGetLastError() == cudaSuccess ? GAP_OK : GAP_ECUDA;
}

extern "C" int ode_adjoint(const void *dev_p, const void *dev_dt, const void *dev_ckpt, const void *dev_gout,
                           int32_t B, int32_t nsteps, int32_t every, int32_t ckpt_every, double delta,
                           int32_t dtype, void *dev_gp, void *dev_gy0, void *dev_scratch, void *stream) {
  if (!dev_p || !dev_dt || !dev_ckpt || !dev_gout || !dev_gp || !dev_gy0 || !dev_scratch || B <= 0 ||
      nsteps < 0 || every <= 0 || ckpt_every <= 0 || delta < 0)
    return GAP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  // one thread per parameter set; small batches spread over more SMs
  const int threads = B >= 148 * 64 ? 64 : 32, blocks = (B + threads - 1) / threads;
  if (dtype == 0)
    k_ode_adjoint<double><<<blocks, threads, 0, st>>>(
        (const double *)dev_p, (const double *)dev_dt, (const double *)dev_ckpt, (const double *)dev_gout, B,
        nsteps, every, ckpt_every, delta, (double *)dev_gp, (double *)dev_gy0, (double *)dev_scratch);
  else if (dtype == 1)
    k_ode_adjoint<float><<<blocks, threads, 0, st>>>(
        (const float *)dev_p, (const float *)dev_dt, (const float *)dev_ckpt, (const float *)dev_gout, B,
        nsteps, every, ckpt_every, delta, (float *)dev_gp, (float *)dev_gy0, (float *)dev_scratch);
  else
    return GAP_EINVAL;
  return cudaGetLastError() == cudaSuccess ? GAP_OK : GAP_ECUDA;
}
