// step.cu -- kernels of one time step of the 1D radiative PIC model
// (paper Sect. 6.1 cycle reduced to the field-aligned direction):
//   k_push      gather, kick, curvature emission, drift, deposit, boundaries,
//               Ampere update of E (one block per tile, fused)
//   k_photons   photon propagation, Breit-Wheeler optical depth, pair creation
//   k_inject    cold-electron surface injection (atmosphere, Sect. 2.3 / 6.1)
//   k_house     per-step bookkeeping of the tile segments and buffers
//   k_rebin_*   compaction of the particle store into the other buffer
#include "gap_internal.cuh"
#include "kernels.h"

namespace gapk {

// ---------------------------------------------------------------------------
// k_push: one block per tile.  Shared memory holds E^n on the tile's nodes
// k0-1 .. k0+nk (in the precision of the state) and the charge through the
// same nodes.  Interior nodes are complete when the block finishes and get
// E^{n+1} = E^n + (dt j_m - D) at once; the four edge nodes shared with the
// neighbouring tiles are finished by whichever of the two blocks arrives
// second (atomic arrival count, no waiting).
template <class R, bool QED, bool HAS_W>
__global__ void __launch_bounds__(256) k_push(View v) {
  using W = typename Prec<R>::W;
  using Acc = typename Prec<R>::Acc;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ Acc sQ0;
  __shared__ unsigned long long sCnt[8];
  __shared__ double sLed[4];
  __shared__ int sDead[2];

  const int t = blockIdx.x;
  const TileDev ti = v.tiles[t];
  const GapDev &g = v.gaps[ti.gap];
  const int nk = ti.nk, k0 = ti.k0;
  const int64_t nx = g.nx;
  const bool periodic = g.periodic != 0;
  Acc *sD = reinterpret_cast<Acc *>(smem);
  R *sE = reinterpret_cast<R *>(smem + sizeof(Acc) * (nk + 2));

  const Ctl *ctl = v.ctl;
  const int ecur = ctl->e_cur;
  const double *Eo = v.E[ecur] + g.node_off;
  double *En = v.E[ecur ^ 1] + g.node_off;
  const int64_t step = ctl->step;
  const int cur = ctl->lep_cur;
  const int phbuf = ctl->ph_cur;

  for (int i = threadIdx.x; i < nk + 2; i += blockDim.x) {
    int64_t node = (int64_t)k0 - 1 + i;
    R e = (R)0;
    if (periodic) {
      node = (node + nx) % nx;
      e = (R)Eo[node];
    } else if (node >= 0 && node <= nx) {
      e = (R)Eo[node];
    }
    sE[i] = e;
    sD[i] = (Acc)0;
  }
  if (threadIdx.x < 8) sCnt[threadIdx.x] = 0ull;
  if (threadIdx.x < 4) sLed[threadIdx.x] = 0.0;
  if (threadIdx.x < 2) sDead[threadIdx.x] = 0;
  if (threadIdx.x == 0) sQ0 = (Acc)0;
  __syncthreads();

  const R dt = (R)g.dt;
  const R cdx = (R)g.cdx;
  const R Hc15 = (R)(g.Hc + 1.5);
  const bool q0_tile = !periodic && k0 == 0;
  const W w_def = HAS_W ? (W)0 : (sizeof(R) == 4 ? (W)(1u << kWeightShift) : (W)g.w0);

  constexpr int VEC = 16 / (int)sizeof(R);  // particles per 16-byte vector load
  for (int s = 0; s < 2; ++s) {
    const int q = s == 0 ? -1 : 1;
    const int64_t start = v.seg_start[s][t];  // multiple of 32 slots: 16-byte aligned
    const int used = v.seg_used[s][t];
    int32_t *Kp = v.lk[cur][s];
    R *Pp = as<R>(v.lphi[cur][s]);
    R *Up = as<R>(v.lu[cur][s]);
    W *Wp = as<W>(v.lw[cur][s]);
    R *Tp = as<R>(v.ltau[cur][s]);
    uint64_t *Ip = v.lid[cur][s];
    int dead = 0;

    // One lepton: gather, kick, emission, drift, deposit, boundaries.  k is
    // set to -1 when the lepton leaves the tile (migrated or removed).
    auto push_one = [&](int32_t &k, R &phi, R &u, const W w, R &tau, const int64_t slot) {
      const int lk = k - (k0 - 1);
      // a1-a2: linear gather of node E at X = k + phi - 3/2, kick
      const R sph = phi - (R)1.5;
      const int j = sph >= (R)0 ? lk : lk - 1;
      const R tt = sph >= (R)0 ? sph : sph + (R)1;
      const R Ep = sE[j] + tt * (sE[j + 1] - sE[j]);
      u += (R)q * Ep * dt;
      // a3: curvature emission by optical-depth sub-cycling (eq. tau_syn)
      R ph_x[QED ? kMaxEmit : 1];
      int ph_k[QED ? kMaxEmit : 1];
      int nph = 0;
      bool have_id = false;
      uint64_t id = 0;
      if (QED && g.qed && phi < Hc15 - (R)k) {
        R trem = dt;
        int kk = 0;
        for (;;) {
          R gm = sqrt((R)1 + u * u);
          R chi = gm * gm * (R)g.lambda_hat / (R)g.rho_hat;
          R ts = sizeof(R) == 4 ? (R)tsyn_f((float)chi) : (R)tsyn_d((double)chi);
          R r = (R)g.rate_mult * (R)kAlphaEm * gm * ts / (R)g.rho_hat;
          if (!(r > (R)0)) break;
          if (tau > r * trem) {
            tau -= r * trem;
            break;
          }
          trem -= tau / r;
          if (!have_id) {
            id = Ip[slot];
            have_id = true;
          }
          double U = uniform53(g.seed, id, (uint32_t)step, CH_EMIT_X, (uint32_t)kk);
          R xi = sizeof(R) == 4 ? (R)spec_inverse_f(v, (float)U) : (R)spec_inverse_d(v, U);
          R x = xi * (R)1.5 * gm * chi;
          R gm1 = u * u / (gm + (R)1);
          R dir = u >= (R)0 ? (R)1 : (R)-1;
          if (x >= gm1) {  // the photon takes the whole kinetic energy: lepton at rest
            x = gm1;
            u = (R)0;
          } else {
            R g2 = gm - x;
            R pp = (g2 - (R)1) * (g2 + (R)1);
            u = pp > (R)0 ? dir * sqrt(pp) : (R)0;
          }
          atomicAdd(&sCnt[0], 1ull);
          if (x >= (R)2) {
            ph_x[nph] = dir * x;  // the sign carries the direction
            ph_k[nph] = kk;
            ++nph;
          } else {
            atomicAdd(&sLed[0], (double)w * (sizeof(R) == 4 ? g.w_unit : 1.0) * (double)x);
          }
          double U2 = uniform53(g.seed, id, (uint32_t)step, CH_EMIT_TAU, (uint32_t)kk);
          tau = (R)(-log(U2));
          if (++kk >= g.kmax_emit) {
            atomicAdd(&sCnt[1], 1ull);
            break;
          }
        }
      }
      // a4: drift
      R dX;
      if (sizeof(R) == 4) {
        dX = u * (R)rsqrtf((float)((R)1 + u * u)) * cdx;
      } else {
        dX = u / sqrt((R)1 + u * u) * cdx;
      }
      R pn = phi + dX;
      int32_t kn = k;
      if (pn >= (R)2) {
        pn -= (R)1;
        kn += 1;
      } else if (pn < (R)1) {
        pn += (R)1;
        kn -= 1;
        if (pn >= (R)2) {
          pn -= (R)1;
          kn += 1;
        }
      }
      // a8: charge through nodes k and kn (<= 2 nodes since |dX| < 1/2)
      const int dk = kn - k;
      if (sizeof(R) == 4) {
        const int Fo = __float2int_rn(((float)phi - 1.0f) * 8388608.0f);
        const int Fn = __float2int_rn(((float)pn - 1.0f) * 8388608.0f);
        const int f0 = dk == 0 ? Fn - Fo : (dk > 0 ? (1 << kPhiBits) - Fo : -Fo);
        const long long qw = (long long)q * (long long)w;
        acc_add(reinterpret_cast<long long *>(&sD[lk]), qw * (long long)f0);
        if (dk != 0) {
          const int f1 = dk > 0 ? Fn : Fn - (1 << kPhiBits);
          acc_add(reinterpret_cast<long long *>(&sD[lk + dk]), qw * (long long)f1);
        }
      } else {
        const double f0 = dk == 0 ? (double)pn - (double)phi
                                  : (dk > 0 ? 2.0 - (double)phi : 1.0 - (double)phi);
        const double qw = (double)q * (double)w;
        acc_add(reinterpret_cast<double *>(&sD[lk]), qw * f0);
        if (dk != 0) {
          const double f1 = dk > 0 ? (double)pn - 1.0 : (double)pn - 2.0;
          acc_add(reinterpret_cast<double *>(&sD[lk + dk]), qw * f1);
        }
      }
      // a7: boundaries
      bool gone = false;
      const double wd = (double)w * (sizeof(R) == 4 ? g.w_unit : 1.0);
      if (!periodic) {
        if (kn < 0 || (kn == 0 && pn < (R)1.5)) {
          gone = true;
          atomicAdd(&sCnt[2], 1ull);
          atomicAdd(&sLed[1], wd * (double)sqrt((R)1 + u * u));
        } else if ((int64_t)kn > nx || ((int64_t)kn == nx && pn >= (R)1.5)) {
          gone = true;
          atomicAdd(&sCnt[3], 1ull);
          atomicAdd(&sLed[2], wd * (double)sqrt((R)1 + u * u));
        }
      } else {
        if (kn < 0) kn += (int32_t)nx;
        else if ((int64_t)kn >= nx) kn -= (int32_t)nx;
      }
      // photons born this step sit at the lepton's new position
      if (QED && nph > 0) {
        double Xn = (double)kn + ((double)pn - 1.5);
        if (periodic && Xn < 0.0) Xn += (double)nx;
        const bool inside = periodic || (Xn >= 0.0 && Xn < (double)nx);
        for (int b = 0; b < nph; ++b) {
          double xb = (double)ph_x[b];
          int32_t dirb = xb >= 0.0 ? 1 : -1;
          xb = fabs(xb);
          if (!inside) {
            atomicAdd(&sCnt[4], 1ull);
            atomicAdd(&sLed[3], wd * xb);
            continue;
          }
          uint64_t pid = child_id(id, (uint32_t)step, CH_PHOTON, (uint32_t)ph_k[b]) | kPhotonBit;
          double tsb = -log(uniform53(g.seed, pid, (uint32_t)(step + 1), CH_BW_TAU, 0));
          photon_append(v, phbuf, ti.gap, Xn, xb, wd, tsb, 0.0, pid, (int32_t)(step + 1), dirb);
          atomicAdd(&sCnt[6], 1ull);
        }
      }
      if (gone) {
        k = -1;
        ++dead;
        return;
      }
      if (q0_tile && kn <= 1) {
        if (sizeof(R) == 4) {
          const int Fn = __float2int_rn(((float)pn - 1.0f) * 8388608.0f);
          const long long frac = kn == 0 ? Fn : (1 << kPhiBits) - Fn;
          acc_add(reinterpret_cast<long long *>(&sQ0), (long long)q * (long long)w * frac);
        } else {
          const double frac = kn == 0 ? (double)pn - 1.0 : 2.0 - (double)pn;
          acc_add(reinterpret_cast<double *>(&sQ0), (double)q * (double)w * frac);
        }
      }
      if (kn >= k0 && kn < k0 + nk) {
        k = kn;
        phi = pn;
      } else {
        if (!have_id) id = Ip[slot];
        const int tn = tile_of(v, g, kn);
        append_lepton<R>(v, s, tn, kn, pn, u, w, tau, id);
        k = -1;
        ++dead;
      }
    };

    const int ngroups = (used + VEC - 1) / VEC;
    for (int gi = threadIdx.x; gi < ngroups; gi += blockDim.x) {
      const int base = gi * VEC;
      const int64_t slot0 = start + base;
      // all loads of the group first (memory-level parallelism)
      Vec<int32_t, VEC> kv = *reinterpret_cast<const Vec<int32_t, VEC> *>(Kp + slot0);
      Vec<R, VEC> pv = *reinterpret_cast<const Vec<R, VEC> *>(Pp + slot0);
      Vec<R, VEC> uv = *reinterpret_cast<const Vec<R, VEC> *>(Up + slot0);
      Vec<W, VEC> wv;
      Vec<R, VEC> tv;
      if (HAS_W) wv = *reinterpret_cast<const Vec<W, VEC> *>(Wp + slot0);
      if (QED) tv = *reinterpret_cast<const Vec<R, VEC> *>(Tp + slot0);
      const int nvalid = used - base < VEC ? used - base : VEC;
#pragma unroll
      for (int jj = 0; jj < VEC; ++jj) {
        if (jj < nvalid && kv.a[jj] >= 0)
          push_one(kv.a[jj], pv.a[jj], uv.a[jj], HAS_W ? wv.a[jj] : w_def, tv.a[jj], slot0 + jj);
      }
      if (nvalid == VEC) {
        *reinterpret_cast<Vec<int32_t, VEC> *>(Kp + slot0) = kv;
        *reinterpret_cast<Vec<R, VEC> *>(Pp + slot0) = pv;
        *reinterpret_cast<Vec<R, VEC> *>(Up + slot0) = uv;
        if (QED) *reinterpret_cast<Vec<R, VEC> *>(Tp + slot0) = tv;
      } else {
        // the last group may share a vector with slots appended this step
        for (int jj = 0; jj < nvalid; ++jj) {
          Kp[slot0 + jj] = kv.a[jj];
          Pp[slot0 + jj] = pv.a[jj];
          Up[slot0 + jj] = uv.a[jj];
          if (QED) Tp[slot0 + jj] = tv.a[jj];
        }
      }
    }
    // one atomic per warp for the dead / migrated count
    for (int o = 16; o > 0; o >>= 1) dead += __shfl_down_sync(0xffffffffu, dead, o);
    if ((threadIdx.x & 31) == 0 && dead) atomicAdd(&sDead[s], dead);
  }
  __syncthreads();

  // a9: Ampere on the tile's nodes
  const double scale = sizeof(R) == 4 ? g.w_unit * kPhiUnit : 1.0;
  const double djm = g.dt * g.jm;
  double work = 0.0;
  for (int i = 2 + threadIdx.x; i <= nk - 1; i += blockDim.x) {
    const int64_t node = (int64_t)k0 - 1 + i;
    const double eo = Eo[node];
    const double en = eo + (djm - (double)sD[i] * scale);
    En[node] = en;
    work += eo + en;
  }
  if (threadIdx.x < 4) {
    const int local = threadIdx.x == 0 ? 0 : (threadIdx.x == 1 ? 1 : (threadIdx.x == 2 ? nk : nk + 1));
    int64_t node = (int64_t)k0 - 1 + local;
    bool valid = true;
    if (periodic) node = (node + nx) % nx;
    else valid = node >= 0 && node <= nx;
    if (valid) {
      const int64_t gn = g.node_off + node;
      acc_add_global(&v.Dg[gn], sD[local]);
      __threadfence();
      const int old = atomicAdd(&v.arrive[gn], 1);
      if (old == (int)v.expect[gn] - 1) {
        __threadfence();
        const double D = acc_take(&v.Dg[gn], (Acc *)nullptr) * scale;
        const double eo = Eo[node];
        const double en = (!periodic && node == 0) ? 0.0 : eo + (djm - D);
        En[node] = en;
        v.arrive[gn] = 0;
        work += eo + en;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) work += __shfl_down_sync(0xffffffffu, work, o);
  if ((threadIdx.x & 31) == 0 && work != 0.0)
    atomicAdd(&v.ledger[ti.gap * L_NLED + L_WORK], 0.5 * work * g.dt * g.dx * g.jm);
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long *C = v.counters + ti.gap * C_NCNT;
    double *Lg = v.ledger + ti.gap * L_NLED;
    if (sCnt[0]) atomicAdd(&C[C_EMIT], sCnt[0]);
    if (sCnt[1]) atomicAdd(&C[C_EMIT_OVF], sCnt[1]);
    if (sCnt[2]) atomicAdd(&C[C_ABSORBED], sCnt[2]);
    if (sCnt[3]) atomicAdd(&C[C_ESCAPED], sCnt[3]);
    if (sCnt[4]) atomicAdd(&C[C_PH_ESCAPED], sCnt[4]);
    if (sCnt[5]) atomicAdd(&C[C_PH_OVF], sCnt[5]);
    if (sCnt[6]) atomicAdd(&C[C_PHOTONS], sCnt[6]);
    if (sLed[0] != 0.0) atomicAdd(&Lg[L_RAD], sLed[0]);
    if (sLed[1] != 0.0) atomicAdd(&Lg[L_ABS], sLed[1]);
    if (sLed[2] != 0.0) atomicAdd(&Lg[L_ESC], sLed[2]);
    if (sLed[3] != 0.0) atomicAdd(&Lg[L_PH_ESC], sLed[3]);
    for (int s = 0; s < 2; ++s)
      if (sDead[s]) atomicAdd(&v.seg_alive[s][t], -sDead[s]);
    if (q0_tile) acc_add_global(&v.q0[ti.gap], sQ0);
  }
}

// ---------------------------------------------------------------------------
// k_push_lean: the push kernel specialised to FP32 state, uniform weights and
// no QED (the thermal and cold plasmas without emission).  Same arithmetic as
// k_push, arranged for memory-level parallelism and few shared-memory
// wavefronts: each thread loads VEC leptons with 16-byte vector loads, then
// gathers E for all of them (one 8-byte (E_i, E_{i+1}) pair each), then does
// the arithmetic, then deposits with 32-bit reductions that return nothing.
// The deposit accumulates c = q (F_new - F_old) in units of 2^-23 (|c| < 2^22)
// exactly in two 32-bit counters per node, hi = c >> 12 and lo = c & 4095,
// neither of which can overflow below 2^20 contributions; the node total is
// hi 2^12 + lo, and the uniform weight multiplies it once, when it leaves
// shared memory.
__device__ __forceinline__ void red_shared_add_u32(unsigned *p, unsigned v) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void red_shared_add_s32(int *p, int v) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void deposit_split(unsigned *lo, int *hi, int c) {
  red_shared_add_u32(lo, (unsigned)(c & 4095));
  red_shared_add_s32(hi, c >> 12);
}

template <int VEC, int MINB>
__global__ void __launch_bounds__(256, MINB) k_push_lean(View v) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long sQ0;
  __shared__ unsigned long long sCnt[4];
  __shared__ double sLed[4];
  __shared__ int sDead[2];

  const int t = blockIdx.x;
  const TileDev ti = v.tiles[t];
  const GapDev &g = v.gaps[ti.gap];
  const int nk = ti.nk, k0 = ti.k0;
  const int64_t nx = g.nx;
  const bool periodic = g.periodic != 0;
  unsigned *sLo = reinterpret_cast<unsigned *>(smem);
  int *sHi = reinterpret_cast<int *>(smem + sizeof(unsigned) * (nk + 2));
  float2 *sE2 = reinterpret_cast<float2 *>(smem + 2 * sizeof(unsigned) * (nk + 2) + 8);

  const Ctl *ctl = v.ctl;
  const int ecur = ctl->e_cur;
  const double *Eo = v.E[ecur] + g.node_off;
  double *En = v.E[ecur ^ 1] + g.node_off;
  const int cur = ctl->lep_cur;

  auto e_at = [&](int64_t node) -> float {
    if (periodic) return (float)Eo[(node + nx) % nx];
    return (node >= 0 && node <= nx) ? (float)Eo[node] : 0.0f;
  };
  for (int i = threadIdx.x; i < nk + 2; i += blockDim.x) {
    const int64_t node = (int64_t)k0 - 1 + i;
    sE2[i] = make_float2(e_at(node), e_at(node + 1));
    sLo[i] = 0u;
    sHi[i] = 0;
  }
  if (threadIdx.x < 4) {
    sCnt[threadIdx.x] = 0ull;
    sLed[threadIdx.x] = 0.0;
  }
  if (threadIdx.x < 2) sDead[threadIdx.x] = 0;
  if (threadIdx.x == 0) sQ0 = 0;
  __syncthreads();

  const float dt = (float)g.dt, cdx = (float)g.cdx;
  const bool q0_tile = !periodic && k0 == 0;
  const unsigned m0 = 1u << kWeightShift;

  for (int s = 0; s < 2; ++s) {
    const int q = s == 0 ? -1 : 1;
    const float qdt = (float)q * dt;
    const int64_t start = v.seg_start[s][t];
    const int used = v.seg_used[s][t];
    int32_t *Kp = v.lk[cur][s];
    float *Pp = as<float>(v.lphi[cur][s]);
    float *Up = as<float>(v.lu[cur][s]);
    int dead = 0;
    const int ngroups = (used + VEC - 1) / VEC;
    for (int gi = threadIdx.x; gi < ngroups; gi += blockDim.x) {
      const int base = gi * VEC;
      const int64_t slot0 = start + base;
      Vec<int32_t, VEC> kv = *reinterpret_cast<const Vec<int32_t, VEC> *>(Kp + slot0);
      Vec<float, VEC> pv = *reinterpret_cast<const Vec<float, VEC> *>(Pp + slot0);
      Vec<float, VEC> uv = *reinterpret_cast<const Vec<float, VEC> *>(Up + slot0);
      const int nvalid = used - base < VEC ? used - base : VEC;
      bool live[VEC];
      int jx[VEC];
      float tt[VEC];
      float2 e2[VEC];
#pragma unroll
      for (int j = 0; j < VEC; ++j) {
        live[j] = j < nvalid && kv.a[j] >= 0;
        const int lk = live[j] ? kv.a[j] - (k0 - 1) : 1;
        const float sph = pv.a[j] - 1.5f;
        jx[j] = sph >= 0.0f ? lk : lk - 1;
        tt[j] = sph >= 0.0f ? sph : sph + 1.0f;
      }
#pragma unroll
      for (int j = 0; j < VEC; ++j) e2[j] = sE2[jx[j]];
      int32_t kn[VEC];
      float pn[VEC];
      int f0[VEC], f1[VEC];
#pragma unroll
      for (int j = 0; j < VEC; ++j) {
        // a1-a2: gather and kick; a4: drift
        float u = uv.a[j] + qdt * (e2[j].x + tt[j] * (e2[j].y - e2[j].x));
        const float dX = u * rsqrtf(1.0f + u * u) * cdx;
        float p = pv.a[j] + dX;
        int32_t k = kv.a[j];
        if (p >= 2.0f) {
          p -= 1.0f;
          k += 1;
        } else if (p < 1.0f) {
          p += 1.0f;
          k -= 1;
          if (p >= 2.0f) {
            p -= 1.0f;
            k += 1;
          }
        }
        // a8: exact charge through nodes k_old and k_new, units 2^-23
        const int Fo = __float2int_rn((pv.a[j] - 1.0f) * 8388608.0f);
        const int Fn = __float2int_rn((p - 1.0f) * 8388608.0f);
        const int dk = k - kv.a[j];
        f0[j] = dk == 0 ? Fn - Fo : (dk > 0 ? (1 << kPhiBits) - Fo : -Fo);
        f1[j] = dk == 0 ? 0 : (dk > 0 ? Fn : Fn - (1 << kPhiBits));
        if (live[j]) uv.a[j] = u;
        kn[j] = k;
        pn[j] = p;
      }
#pragma unroll
      for (int j = 0; j < VEC; ++j) {
        if (!live[j]) continue;
        const int lk = kv.a[j] - (k0 - 1);
        deposit_split(&sLo[lk], &sHi[lk], q * f0[j]);
        if (kn[j] != kv.a[j]) {
          const int l1 = lk + kn[j] - kv.a[j];
          deposit_split(&sLo[l1], &sHi[l1], q * f1[j]);
        }
      }
#pragma unroll
      for (int j = 0; j < VEC; ++j) {
        if (!live[j]) continue;
        int32_t k = kn[j];
        const float p = pn[j];
        // a7: boundaries
        if (!periodic) {
          const bool below = k < 0 || (k == 0 && p < 1.5f);
          const bool above = (int64_t)k > nx || ((int64_t)k == nx && p >= 1.5f);
          if (below || above) {
            const float gm = sqrtf(1.0f + uv.a[j] * uv.a[j]);
            atomicAdd(&sCnt[below ? 0 : 1], 1ull);
            atomicAdd(&sLed[below ? 0 : 1], g.w0 * (double)gm);
            kv.a[j] = -1;
            ++dead;
            continue;
          }
        } else {
          if (k < 0) k += (int32_t)nx;
          else if ((int64_t)k >= nx) k -= (int32_t)nx;
        }
        if (q0_tile && k <= 1) {
          const int Fn = __float2int_rn((p - 1.0f) * 8388608.0f);
          const long long frac = k == 0 ? Fn : (1 << kPhiBits) - Fn;
          atomicAdd(reinterpret_cast<unsigned long long *>(&sQ0), (unsigned long long)((long long)q * m0 * frac));
        }
        if (k >= k0 && k < k0 + nk) {
          kv.a[j] = k;
          pv.a[j] = p;
        } else {
          const uint64_t id = v.lid[cur][s][slot0 + j];
          const float tau = as<float>(v.ltau[cur][s])[slot0 + j];
          append_lepton<float>(v, s, tile_of(v, g, k), k, p, uv.a[j], (uint32_t)m0, tau, id);
          kv.a[j] = -1;
          ++dead;
        }
      }
      if (nvalid == VEC) {
        *reinterpret_cast<Vec<int32_t, VEC> *>(Kp + slot0) = kv;
        *reinterpret_cast<Vec<float, VEC> *>(Pp + slot0) = pv;
        *reinterpret_cast<Vec<float, VEC> *>(Up + slot0) = uv;
      } else {
        for (int j = 0; j < nvalid; ++j) {
          Kp[slot0 + j] = kv.a[j];
          Pp[slot0 + j] = pv.a[j];
          Up[slot0 + j] = uv.a[j];
        }
      }
    }
    for (int o = 16; o > 0; o >>= 1) dead += __shfl_down_sync(0xffffffffu, dead, o);
    if ((threadIdx.x & 31) == 0 && dead) atomicAdd(&sDead[s], dead);
  }
  __syncthreads();

  // a9: Ampere on the tile's nodes (node sums carry the weight m0)
  const double scale = g.w_unit * (double)m0 * kPhiUnit;
  const double djm = g.dt * g.jm;
  double work = 0.0;
  auto node_sum = [&](int i) -> long long { return (long long)sHi[i] * 4096 + (long long)sLo[i]; };
  for (int i = 2 + threadIdx.x; i <= nk - 1; i += blockDim.x) {
    const int64_t node = (int64_t)k0 - 1 + i;
    const double eo = Eo[node];
    const double en = eo + (djm - (double)node_sum(i) * scale);
    En[node] = en;
    work += eo + en;
  }
  if (threadIdx.x < 4) {
    const int local = threadIdx.x == 0 ? 0 : (threadIdx.x == 1 ? 1 : (threadIdx.x == 2 ? nk : nk + 1));
    int64_t node = (int64_t)k0 - 1 + local;
    bool valid = true;
    if (periodic) node = (node + nx) % nx;
    else valid = node >= 0 && node <= nx;
    if (valid) {
      const int64_t gn = g.node_off + node;
      // global edge sums are in the units of k_push: weight units x 2^-23
      atomicAdd(&v.Dg[gn], (unsigned long long)(node_sum(local) * (long long)m0));
      __threadfence();
      const int old = atomicAdd(&v.arrive[gn], 1);
      if (old == (int)v.expect[gn] - 1) {
        __threadfence();
        const double D = (double)(long long)atomicExch(&v.Dg[gn], 0ull) * g.w_unit * kPhiUnit;
        const double eo = Eo[node];
        const double en = (!periodic && node == 0) ? 0.0 : eo + (djm - D);
        En[node] = en;
        v.arrive[gn] = 0;
        work += eo + en;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) work += __shfl_down_sync(0xffffffffu, work, o);
  if ((threadIdx.x & 31) == 0 && work != 0.0)
    atomicAdd(&v.ledger[ti.gap * L_NLED + L_WORK], 0.5 * work * g.dt * g.dx * g.jm);
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long *C = v.counters + ti.gap * C_NCNT;
    double *Lg = v.ledger + ti.gap * L_NLED;
    if (sCnt[0]) atomicAdd(&C[C_ABSORBED], sCnt[0]);
    if (sCnt[1]) atomicAdd(&C[C_ESCAPED], sCnt[1]);
    if (sLed[0] != 0.0) atomicAdd(&Lg[L_ABS], sLed[0]);
    if (sLed[1] != 0.0) atomicAdd(&Lg[L_ESC], sLed[1]);
    for (int s = 0; s < 2; ++s)
      if (sDead[s]) atomicAdd(&v.seg_alive[s][t], -sDead[s]);
    if (q0_tile) atomicAdd(&v.q0[ti.gap], (unsigned long long)sQ0);
  }
}

// ---------------------------------------------------------------------------
// TMA (bulk-copy) helpers: 1D cp.async.bulk into shared memory, completion
// tracked by an mbarrier transaction count.
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(mbar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(mbar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after 2^24 polls (each try_wait may itself suspend
// for a while), returning false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *mbar, uint32_t parity) {
  for (uint32_t it = 0; it < (1u << 24); ++it)
    if (mbar_try_wait(mbar, parity)) return true;
  return false;
}

// k_push_tma: k_push_lean with the particle arrays of the tile streamed
// through a ring of shared-memory stages by the TMA unit.  Thread 0 issues
// one bulk copy per array and chunk (CH leptons: k, phi', u); every thread
// waits on the stage's mbarrier, pushes its VEC leptons from shared memory
// and stores them straight back to global memory; after a block-wide barrier
// the stage is refilled with the chunk STAGES ahead.  Up to STAGES chunks per
// block are in flight, decoupling HBM latency from the arithmetic.
template <int STAGES>
__global__ void __launch_bounds__(256, 4) k_push_tma(View v) {
  constexpr int VEC = 4;
  constexpr int CH = 1024;  // leptons per chunk (4 per thread at 256 threads)
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t mbar[STAGES];
  __shared__ long long sQ0;
  __shared__ unsigned long long sCnt[4];
  __shared__ double sLed[4];
  __shared__ int sDead[2];
  __shared__ int sAbort;

  const int t = blockIdx.x;
  const TileDev ti = v.tiles[t];
  const GapDev &g = v.gaps[ti.gap];
  const int nk = ti.nk, k0 = ti.k0;
  const int64_t nx = g.nx;
  const bool periodic = g.periodic != 0;
  unsigned char *stage_base = smem;  // STAGES x (3 arrays x CH x 4 bytes)
  constexpr int STAGE_BYTES = 3 * CH * 4;
  unsigned *sLo = reinterpret_cast<unsigned *>(smem + STAGES * STAGE_BYTES);
  int *sHi = reinterpret_cast<int *>(smem + STAGES * STAGE_BYTES + sizeof(unsigned) * (nk + 2));
  float2 *sE2 = reinterpret_cast<float2 *>(smem + STAGES * STAGE_BYTES + 2 * sizeof(unsigned) * (nk + 2) + 8);

  const Ctl *ctl = v.ctl;
  const int ecur = ctl->e_cur;
  const double *Eo = v.E[ecur] + g.node_off;
  double *En = v.E[ecur ^ 1] + g.node_off;
  const int cur = ctl->lep_cur;

  // chunk list over both species
  const int used0 = v.seg_used[0][t], used1 = v.seg_used[1][t];
  const int n0 = (used0 + CH - 1) / CH, n1 = (used1 + CH - 1) / CH;
  const int nch = n0 + n1;
  auto chunk_info = [&](int gidx, int &s, int &c, int &cnt, int64_t &slot) {
    s = gidx < n0 ? 0 : 1;
    c = gidx < n0 ? gidx : gidx - n0;
    const int used = s == 0 ? used0 : used1;
    cnt = used - c * CH < CH ? used - c * CH : CH;
    slot = v.seg_start[s][t] + (int64_t)c * CH;
  };
  auto issue = [&](int gidx) {
    int s, c, cnt;
    int64_t slot;
    chunk_info(gidx, s, c, cnt, slot);
    const uint32_t bytes = (uint32_t)(((cnt + 3) & ~3) * 4);  // multiple of 16 inside the segment
    unsigned char *st = stage_base + (gidx % STAGES) * STAGE_BYTES;
    uint64_t *mb = &mbar[gidx % STAGES];
    mbar_expect_tx(mb, 3 * bytes);
    bulk_copy_g2s(st, v.lk[cur][s] + slot, bytes, mb);
    bulk_copy_g2s(st + CH * 4, as<float>(v.lphi[cur][s]) + slot, bytes, mb);
    bulk_copy_g2s(st + 2 * CH * 4, as<float>(v.lu[cur][s]) + slot, bytes, mb);
  };

  if (threadIdx.x == 0) {
    for (int i = 0; i < STAGES; ++i) mbar_init(&mbar[i], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    sAbort = 0;
  }
  auto e_at = [&](int64_t node) -> float {
    if (periodic) return (float)Eo[(node + nx) % nx];
    return (node >= 0 && node <= nx) ? (float)Eo[node] : 0.0f;
  };
  for (int i = threadIdx.x; i < nk + 2; i += blockDim.x) {
    const int64_t node = (int64_t)k0 - 1 + i;
    sE2[i] = make_float2(e_at(node), e_at(node + 1));
    sLo[i] = 0u;
    sHi[i] = 0;
  }
  if (threadIdx.x < 4) {
    sCnt[threadIdx.x] = 0ull;
    sLed[threadIdx.x] = 0.0;
  }
  if (threadIdx.x < 2) sDead[threadIdx.x] = 0;
  if (threadIdx.x == 0) sQ0 = 0;
  __syncthreads();
  if (threadIdx.x == 0)
    for (int i = 0; i < STAGES && i < nch; ++i) issue(i);

  const float dt = (float)g.dt, cdx = (float)g.cdx;
  const bool q0_tile = !periodic && k0 == 0;
  const unsigned m0 = 1u << kWeightShift;
  int dead0 = 0, dead1 = 0;
  int consumed = 0;

  for (int gidx = 0; gidx < nch; ++gidx) {
    int s, c, cnt;
    int64_t slot_c;
    chunk_info(gidx, s, c, cnt, slot_c);
    const bool ok = mbar_wait_bounded(&mbar[gidx % STAGES], (uint32_t)((gidx / STAGES) & 1));
    if (!ok) atomicExch(&sAbort, 1);
    __syncthreads();
    if (sAbort) break;
    consumed = gidx + 1;
    const int q = s == 0 ? -1 : 1;
    const float qdt = (float)q * dt;
    const unsigned char *st = stage_base + (gidx % STAGES) * STAGE_BYTES;
    const int base = threadIdx.x * VEC;
    if (base < cnt) {
      Vec<int32_t, VEC> kv = *reinterpret_cast<const Vec<int32_t, VEC> *>(st + base * 4);
      Vec<float, VEC> pv = *reinterpret_cast<const Vec<float, VEC> *>(st + CH * 4 + base * 4);
      Vec<float, VEC> uv = *reinterpret_cast<const Vec<float, VEC> *>(st + 2 * CH * 4 + base * 4);
      const int nvalid = cnt - base < VEC ? cnt - base : VEC;
      const int64_t slot0 = slot_c + base;
      bool live[VEC];
      int jx[VEC];
      float tt[VEC];
      float2 e2[VEC];
#pragma unroll
      for (int j = 0; j < VEC; ++j) {
        live[j] = j < nvalid && kv.a[j] >= 0;
        const int lk = live[j] ? kv.a[j] - (k0 - 1) : 1;
        const float sph = pv.a[j] - 1.5f;
        jx[j] = sph >= 0.0f ? lk : lk - 1;
        tt[j] = sph >= 0.0f ? sph : sph + 1.0f;
      }
#pragma unroll
      for (int j = 0; j < VEC; ++j) e2[j] = sE2[jx[j]];
      int32_t kn[VEC];
      float pn[VEC];
      int f0[VEC], f1[VEC];
#pragma unroll
      for (int j = 0; j < VEC; ++j) {
        float u = uv.a[j] + qdt * (e2[j].x + tt[j] * (e2[j].y - e2[j].x));
        const float dX = u * rsqrtf(1.0f + u * u) * cdx;
        float p = pv.a[j] + dX;
        int32_t k = kv.a[j];
        if (p >= 2.0f) {
          p -= 1.0f;
          k += 1;
        } else if (p < 1.0f) {
          p += 1.0f;
          k -= 1;
          if (p >= 2.0f) {
            p -= 1.0f;
            k += 1;
          }
        }
        const int Fo = __float2int_rn((pv.a[j] - 1.0f) * 8388608.0f);
        const int Fn = __float2int_rn((p - 1.0f) * 8388608.0f);
        const int dk = k - kv.a[j];
        f0[j] = dk == 0 ? Fn - Fo : (dk > 0 ? (1 << kPhiBits) - Fo : -Fo);
        f1[j] = dk == 0 ? 0 : (dk > 0 ? Fn : Fn - (1 << kPhiBits));
        if (live[j]) uv.a[j] = u;
        kn[j] = k;
        pn[j] = p;
      }
#pragma unroll
      for (int j = 0; j < VEC; ++j) {
        if (!live[j]) continue;
        const int lk = kv.a[j] - (k0 - 1);
        deposit_split(&sLo[lk], &sHi[lk], q * f0[j]);
        if (kn[j] != kv.a[j]) {
          const int l1 = lk + kn[j] - kv.a[j];
          deposit_split(&sLo[l1], &sHi[l1], q * f1[j]);
        }
      }
      int dead = 0;
#pragma unroll
      for (int j = 0; j < VEC; ++j) {
        if (!live[j]) continue;
        int32_t k = kn[j];
        const float p = pn[j];
        if (!periodic) {
          const bool below = k < 0 || (k == 0 && p < 1.5f);
          const bool above = (int64_t)k > nx || ((int64_t)k == nx && p >= 1.5f);
          if (below || above) {
            const float gm = sqrtf(1.0f + uv.a[j] * uv.a[j]);
            atomicAdd(&sCnt[below ? 0 : 1], 1ull);
            atomicAdd(&sLed[below ? 0 : 1], g.w0 * (double)gm);
            kv.a[j] = -1;
            ++dead;
            continue;
          }
        } else {
          if (k < 0) k += (int32_t)nx;
          else if ((int64_t)k >= nx) k -= (int32_t)nx;
        }
        if (q0_tile && k <= 1) {
          const int Fn = __float2int_rn((p - 1.0f) * 8388608.0f);
          const long long frac = k == 0 ? Fn : (1 << kPhiBits) - Fn;
          atomicAdd(reinterpret_cast<unsigned long long *>(&sQ0), (unsigned long long)((long long)q * m0 * frac));
        }
        if (k >= k0 && k < k0 + nk) {
          kv.a[j] = k;
          pv.a[j] = p;
        } else {
          const uint64_t id = v.lid[cur][s][slot0 + j];
          const float tau = as<float>(v.ltau[cur][s])[slot0 + j];
          append_lepton<float>(v, s, tile_of(v, g, k), k, p, uv.a[j], (uint32_t)m0, tau, id);
          kv.a[j] = -1;
          ++dead;
        }
      }
      if (s == 0) dead0 += dead;
      else dead1 += dead;
      int32_t *Kp = v.lk[cur][s];
      float *Pp = as<float>(v.lphi[cur][s]);
      float *Up = as<float>(v.lu[cur][s]);
      if (nvalid == VEC) {
        *reinterpret_cast<Vec<int32_t, VEC> *>(Kp + slot0) = kv;
        *reinterpret_cast<Vec<float, VEC> *>(Pp + slot0) = pv;
        *reinterpret_cast<Vec<float, VEC> *>(Up + slot0) = uv;
      } else {
        for (int j = 0; j < nvalid; ++j) {
          Kp[slot0 + j] = kv.a[j];
          Pp[slot0 + j] = pv.a[j];
          Up[slot0 + j] = uv.a[j];
        }
      }
    }
    __syncthreads();  // every thread is done with this stage
    if (threadIdx.x == 0 && gidx + STAGES < nch) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(gidx + STAGES);
    }
  }
  if (sAbort) {
    // a stage never completed: record it, then let the copies still in
    // flight land (bounded) before the block's shared memory is released
    if (threadIdx.x == 0) {
      atomicOr(&v.ctl->error, 16);
      const int issued = nch < consumed + STAGES ? nch : consumed + STAGES;
      for (int gi = consumed; gi < issued; ++gi)
        (void)mbar_wait_bounded(&mbar[gi % STAGES], (uint32_t)((gi / STAGES) & 1));
    }
    return;
  }
  for (int o = 16; o > 0; o >>= 1) {
    dead0 += __shfl_down_sync(0xffffffffu, dead0, o);
    dead1 += __shfl_down_sync(0xffffffffu, dead1, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (dead0) atomicAdd(&sDead[0], dead0);
    if (dead1) atomicAdd(&sDead[1], dead1);
  }
  __syncthreads();

  const double scale = g.w_unit * (double)m0 * kPhiUnit;
  const double djm = g.dt * g.jm;
  double work = 0.0;
  auto node_sum = [&](int i) -> long long { return (long long)sHi[i] * 4096 + (long long)sLo[i]; };
  for (int i = 2 + threadIdx.x; i <= nk - 1; i += blockDim.x) {
    const int64_t node = (int64_t)k0 - 1 + i;
    const double eo = Eo[node];
    const double en = eo + (djm - (double)node_sum(i) * scale);
    En[node] = en;
    work += eo + en;
  }
  if (threadIdx.x < 4) {
    const int local = threadIdx.x == 0 ? 0 : (threadIdx.x == 1 ? 1 : (threadIdx.x == 2 ? nk : nk + 1));
    int64_t node = (int64_t)k0 - 1 + local;
    bool valid = true;
    if (periodic) node = (node + nx) % nx;
    else valid = node >= 0 && node <= nx;
    if (valid) {
      const int64_t gn = g.node_off + node;
      atomicAdd(&v.Dg[gn], (unsigned long long)(node_sum(local) * (long long)m0));
      __threadfence();
      const int old = atomicAdd(&v.arrive[gn], 1);
      if (old == (int)v.expect[gn] - 1) {
        __threadfence();
        const double D = (double)(long long)atomicExch(&v.Dg[gn], 0ull) * g.w_unit * kPhiUnit;
        const double eo = Eo[node];
        const double en = (!periodic && node == 0) ? 0.0 : eo + (djm - D);
        En[node] = en;
        v.arrive[gn] = 0;
        work += eo + en;
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) work += __shfl_down_sync(0xffffffffu, work, o);
  if ((threadIdx.x & 31) == 0 && work != 0.0)
    atomicAdd(&v.ledger[ti.gap * L_NLED + L_WORK], 0.5 * work * g.dt * g.dx * g.jm);
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long *C = v.counters + ti.gap * C_NCNT;
    double *Lg = v.ledger + ti.gap * L_NLED;
    if (sCnt[0]) atomicAdd(&C[C_ABSORBED], sCnt[0]);
    if (sCnt[1]) atomicAdd(&C[C_ESCAPED], sCnt[1]);
    if (sLed[0] != 0.0) atomicAdd(&Lg[L_ABS], sLed[0]);
    if (sLed[1] != 0.0) atomicAdd(&Lg[L_ESC], sLed[1]);
    for (int s = 0; s < 2; ++s)
      if (sDead[s]) atomicAdd(&v.seg_alive[s][t], -sDead[s]);
    if (q0_tile) atomicAdd(&v.q0[ti.gap], (unsigned long long)sQ0);
  }
}

// ---------------------------------------------------------------------------
// k_photons: every photon alive at step start moves by c dt, accumulates the
// Breit-Wheeler optical depth at the mid-step angle sin(psi) = |sin(l/R_curv)|
// (eq. tau_bw, Sect. 6.1) inside the gap, and converts into an e-e+ pair with
// gamma = x/2 each once the depth reaches its threshold.  Survivors and the
// photons born during this step are copied into the other buffer.
template <class R>
__global__ void k_photons(View v) {
  using W = typename Prec<R>::W;
  const int cur = v.ctl->ph_cur, nxt = cur ^ 1;
  const int64_t n = v.ctl->ph_count[cur];
  const int64_t step = v.ctl->step;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int gap = v.pgap[cur][i];
    const GapDev &g = v.gaps[gap];
    double X = v.pX[cur][i];
    const double x = v.px[cur][i];
    const double w = v.pw[cur][i];
    const double ts = v.pts[cur][i];
    double ta = v.pta[cur][i];
    const uint64_t id = v.pid[cur][i];
    const int32_t n0 = v.pn0[cur][i];
    const int32_t dir = v.pdir[cur][i];
    if ((int64_t)n0 > step) {  // born during this step: untouched
      if (photon_append(v, nxt, gap, X, x, w, ts, ta, id, n0, dir)) atomicAdd(&v.ph_gap[nxt][gap], 1);
      continue;
    }
    if (X < g.Hc) {
      const double lmid = ((double)step - (double)n0 + 0.5) * g.dt;
      const double sp = fabs(sin(lmid / g.rho_hat));
      const double chi = x * g.b * sp;
      ta += g.dt * g.rate_mult * kAlphaEm / g.lambda_hat * g.b * sp * tbw_d(chi);
    }
    X += (double)dir * g.cdx;
    if (g.periodic) {
      const double L = (double)g.nx;
      X = fmod(X, L);
      if (X < 0.0) X += L;
      if (X >= L) X -= L;
    } else if (X < 0.0 || X >= (double)g.nx) {
      atomicAdd(&v.counters[gap * C_NCNT + C_PH_ESCAPED], 1ull);
      atomicAdd(&v.ledger[gap * L_NLED + L_PH_ESC], w * x);
      continue;
    }
    if (ta >= ts) {
      const double gp = 0.5 * x;
      const double up = (double)dir * sqrt((gp - 1.0) * (gp + 1.0));
      int32_t k;
      R phi;
      split_position<R>(X, g.nx, g.periodic != 0, k, phi);
      const int tn = tile_of(v, g, k);
      W wq;
      if (sizeof(R) == 4) wq = (W)llrint(w / g.w_unit);
      else wq = (W)w;
      for (int s = 0; s < 2; ++s) {
        const uint64_t lid = child_id(id, (uint32_t)step, CH_PAIR, (uint32_t)s) & ~kPhotonBit;
        const R tau = (R)(-log(uniform53(g.seed, lid, (uint32_t)(step + 1), CH_TAU0, 0)));
        append_lepton<R>(v, s, tn, k, phi, (R)up, wq, tau, lid);
      }
      atomicAdd(&v.counters[gap * C_NCNT + C_PAIRS], 1ull);
      continue;
    }
    if (photon_append(v, nxt, gap, X, x, w, ts, ta, id, n0, dir)) atomicAdd(&v.ph_gap[nxt][gap], 1);
  }
}

// Per-gap photon counts of the buffer k_photons fills (the photons emitted in
// the push and the survivors of the step) start at 0.
__global__ void k_photon_count_reset(View v) {
  const int nxt = v.ctl->ph_cur ^ 1;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < v.n_gaps; i += gridDim.x * blockDim.x)
    v.ph_gap[nxt][i] = 0;
}

// ---------------------------------------------------------------------------
// k_inject: one thread per gap with a surface.  Cell 0 must hold the
// co-rotation charge eta_co dx = -dx; while its deficit exceeds half a
// macro-particle charge a cold electron is added at X = U/2 in (0, 1/2].
template <class R>
__global__ void k_inject(View v) {
  using W = typename Prec<R>::W;
  const int gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi >= v.n_gaps) return;
  const GapDev &g = v.gaps[gi];
  if (g.periodic) return;
  const int64_t step = v.ctl->step;
  double Q0;
  if (sizeof(R) == 4) Q0 = (double)(long long)atomicExch(&v.q0[gi], 0ull) * g.w_unit * kPhiUnit;
  else Q0 = __longlong_as_double((long long)atomicExch(&v.q0[gi], 0ull));
  if (!(g.w0 > 0.0)) return;
  double deficit = Q0 + g.dx;
  int j = 0;
  unsigned long long *C = v.counters + gi * C_NCNT;
  while (deficit > 0.5 * g.w0) {
    if (j >= g.kmax_inject) {
      atomicAdd(&C[C_INJ_OVF], 1ull);
      break;
    }
    const uint64_t id = child_id(g.inj_root, (uint32_t)step, CH_INJECT, (uint32_t)j) & ~kPhotonBit;
    const double o = 0.5 * uniform53(g.seed, id, (uint32_t)(step + 1), CH_INJECT, 0);
    int32_t k;
    R phi;
    split_position<R>(o, g.nx, false, k, phi);
    const R tau = (R)(-log(uniform53(g.seed, id, (uint32_t)(step + 1), CH_TAU0, 0)));
    W w;
    if (sizeof(R) == 4) w = (W)(1u << kWeightShift);
    else w = (W)g.w0;
    append_lepton<R>(v, 0, tile_of(v, g, k), k, phi, (R)0, w, tau, id);
    deficit -= g.w0 * (o + 0.5);
    atomicAdd(&C[C_INJECTED], 1ull);
    atomicAdd(&v.ledger[gi * L_NLED + L_INJ], g.w0);
    ++j;
  }
}

// k_house: the appends of this step become part of the next step's work;
// buffers of E and photons flip; the step counter advances.
__global__ void k_house(View v) {
  const int n = 2 * v.n_tiles;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int s = i / v.n_tiles, t = i % v.n_tiles;
    const int a = v.seg_append[s][t], c = v.seg_cap[s][t];
    v.seg_used[s][t] = a < c ? a : c;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    Ctl *c = v.ctl;
    c->step += 1;
    c->e_cur ^= 1;
    if (v.qed_any) {
      const int old = c->ph_cur;
      c->ph_cur = old ^ 1;
      c->ph_count[old] = 0;
    }
    if (c->spill_n[0] > 0 || c->spill_n[1] > 0 || (v.rebin_every > 0 && c->step % v.rebin_every == 0))
      c->need_rebin = 1;
  }
}

// k_sync_used: appends made outside a step (initial load, import) become
// visible to the next compaction and push.
__global__ void k_sync_used(View v) {
  const int n = 2 * v.n_tiles;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int s = i / v.n_tiles, t = i % v.n_tiles;
    const int a = v.seg_append[s][t], c = v.seg_cap[s][t];
    v.seg_used[s][t] = a < c ? a : c;
  }
}

// ---------------------------------------------------------------------------
// Store compaction (the amortised re-bin of the particle store).
// r1: new segment capacities and starts from the alive counts (one block).
__global__ void __launch_bounds__(1024) k_rebin_layout(View v, double slack) {
  if (!v.ctl->need_rebin) return;
  __shared__ long long warp_sums[32];
  __shared__ long long carry;
  const int n = v.n_tiles;
  for (int s = 0; s < 2; ++s) {
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < n; base += blockDim.x) {
      const int t = base + threadIdx.x;
      long long cap = 0;
      if (t < n) {
        long long cnt = (long long)v.seg_alive[s][t] + (long long)v.spill_cnt[s][t];
        if (cnt < 0) cnt = 0;
        long long head = (long long)(cnt * slack);
        if (head < 64) head = 64;
        cap = (cnt + head + 31) & ~31ll;
        v.new_cap[s][t] = (int32_t)cap;
      }
      // block exclusive scan of cap
      long long x = cap;
      const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
      for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) warp_sums[wid] = x;
      __syncthreads();
      if (wid == 0) {
        long long ws = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
          long long y = __shfl_up_sync(0xffffffffu, ws, o);
          if (lane >= o) ws += y;
        }
        warp_sums[lane] = ws;
      }
      __syncthreads();
      const long long before = (wid > 0 ? warp_sums[wid - 1] : 0) + x - cap;
      if (t < n) v.new_start[s][t] = carry + before;
      __syncthreads();
      if (threadIdx.x == blockDim.x - 1) carry += before + cap;
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      v.ctl->new_total[s] = carry;
      if (carry > v.lep_capacity) atomicOr(&v.ctl->error, 4);
    }
    __syncthreads();
  }
}

// r2: one block per (species, tile): ordered compaction of the alive slots
// into the other buffer (the order within the tile is kept: the push kernel
// measured fastest on the interleaved order of the initial load, slower on
// random order and slowest on fully node-sorted order).  Without QED and with
// uniform weights the optical depth and the weight are not part of the state
// and are not copied.
template <class R>
__global__ void k_rebin_compact(View v) {
  using W = typename Prec<R>::W;
  if (!v.ctl->need_rebin || (v.ctl->error & 4)) return;
  __shared__ int warp_cnt[32];
  __shared__ int carry;
  const int s = blockIdx.x / v.n_tiles, t = blockIdx.x % v.n_tiles;
  const int cur = v.ctl->lep_cur, nxt = cur ^ 1;
  const int64_t src0 = v.seg_start[s][t];
  const int used = v.seg_used[s][t];
  const int64_t dst0 = v.new_start[s][t];
  const bool full_state = v.qed_any || v.has_w;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < used; base += blockDim.x) {
    const int i = base + threadIdx.x;
    int32_t k = -1;
    if (i < used) k = v.lk[cur][s][src0 + i];
    const bool alive = k >= 0;
    const unsigned bal = __ballot_sync(0xffffffffu, alive);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) warp_cnt[wid] = __popc(bal);
    __syncthreads();
    if (threadIdx.x == 0) {
      int acc = 0;
      for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) {
        int c = warp_cnt[wv];
        warp_cnt[wv] = acc;
        acc += c;
      }
      warp_cnt[31] = acc;  // block total (blockDim <= 992 threads keeps slot 31 free)
    }
    __syncthreads();
    const int pos = carry + warp_cnt[wid] + __popc(bal & ((1u << lane) - 1u));
    if (alive && pos >= v.new_cap[s][t]) atomicOr(&v.ctl->error, 8);  // never: cap >= alive count
    if (alive && pos < v.new_cap[s][t]) {
      const int64_t d = dst0 + pos, sidx = src0 + i;
      v.lk[nxt][s][d] = k;
      as<R>(v.lphi[nxt][s])[d] = as<R>(v.lphi[cur][s])[sidx];
      as<R>(v.lu[nxt][s])[d] = as<R>(v.lu[cur][s])[sidx];
      v.lid[nxt][s][d] = v.lid[cur][s][sidx];
      if (full_state) {
        as<W>(v.lw[nxt][s])[d] = as<W>(v.lw[cur][s])[sidx];
        as<R>(v.ltau[nxt][s])[d] = as<R>(v.ltau[cur][s])[sidx];
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_cnt[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) v.new_fill[s][t] = carry;
}

// r2b: spilled particles go after the compacted ones of their tile.
template <class R>
__global__ void k_rebin_spill(View v) {
  using W = typename Prec<R>::W;
  if (!v.ctl->need_rebin || (v.ctl->error & 4)) return;
  const int nxt = v.ctl->lep_cur ^ 1;
  for (int s = 0; s < 2; ++s) {
    long long n = v.ctl->spill_n[s];
    if (n > v.spill_capacity) n = v.spill_capacity;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
      const int t = v.stile[s][i];
      const int pos = atomicAdd(&v.new_fill[s][t], 1);
      if (pos >= v.new_cap[s][t]) {  // never: the capacity counted the spills
        atomicOr(&v.ctl->error, 8);
        continue;
      }
      const int64_t d = v.new_start[s][t] + pos;
      v.lk[nxt][s][d] = v.sk[s][i];
      as<R>(v.lphi[nxt][s])[d] = (R)v.sphi[s][i];
      as<R>(v.lu[nxt][s])[d] = (R)v.su[s][i];
      if (sizeof(R) == 4) as<W>(v.lw[nxt][s])[d] = (W)llrint(v.sw[s][i]);
      else as<W>(v.lw[nxt][s])[d] = (W)v.sw[s][i];
      as<R>(v.ltau[nxt][s])[d] = (R)v.stau[s][i];
      v.lid[nxt][s][d] = v.sid[s][i];
    }
  }
}

// r3: adopt the new layout.
__global__ void k_rebin_adopt(View v) {
  if (!v.ctl->need_rebin || (v.ctl->error & 4)) return;
  const int n = 2 * v.n_tiles;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int s = i / v.n_tiles, t = i % v.n_tiles;
    const int f = v.new_fill[s][t];
    v.seg_start[s][t] = v.new_start[s][t];
    v.seg_cap[s][t] = v.new_cap[s][t];
    v.seg_used[s][t] = f;
    v.seg_append[s][t] = f;
    v.seg_alive[s][t] = f;
    v.spill_cnt[s][t] = 0;
  }
}

// r4: flip the buffer; clear the spill lists.
__global__ void k_rebin_finish(View v) {
  Ctl *c = v.ctl;
  if (!c->need_rebin) return;
  if (!(c->error & 4)) {
    c->lep_cur ^= 1;
    c->spill_n[0] = 0;
    c->spill_n[1] = 0;
  }
  c->need_rebin = 0;
}

// ---------------------------------------------------------------------------
template <class R>
static void launch_push_impl(const View &v, int threads, cudaStream_t st) {
  if (sizeof(R) == 4 && !v.qed_any && !v.has_w) {
    const size_t smem_lean = (size_t)(v.tile + 8) * (2 * sizeof(unsigned) + sizeof(float2)) + 64;
    switch (v.variant) {
      case 1: k_push_lean<4, 6><<<v.n_tiles, threads, smem_lean, st>>>(v); break;
      case 2: k_push_lean<2, 8><<<v.n_tiles, threads, smem_lean, st>>>(v); break;
      case 3: k_push_lean<4, 8><<<v.n_tiles, threads, smem_lean, st>>>(v); break;
      case 4:
      case 5: {
        // TMA pipeline: 256 threads, 3 or 2 stages of 12 KB
        const int stages = v.variant == 4 ? 3 : 2;
        const size_t smem_tma = (size_t)stages * 3 * 1024 * 4 + (size_t)(v.tile + 8) * 16 + 64;
        if (stages == 3) k_push_tma<3><<<v.n_tiles, 256, smem_tma, st>>>(v);
        else k_push_tma<2><<<v.n_tiles, 256, smem_tma, st>>>(v);
        break;
      }
      default: k_push_lean<4, 4><<<v.n_tiles, threads, smem_lean, st>>>(v); break;
    }
    return;
  }
  const size_t smem = (size_t)(v.tile + 8) * (sizeof(typename Prec<R>::Acc) + sizeof(R)) + 64;
  if (v.qed_any) {
    if (v.has_w)
      k_push<R, true, true><<<v.n_tiles, threads, smem, st>>>(v);
    else
      k_push<R, true, false><<<v.n_tiles, threads, smem, st>>>(v);
  } else {
    if (v.has_w)
      k_push<R, false, true><<<v.n_tiles, threads, smem, st>>>(v);
    else
      k_push<R, false, false><<<v.n_tiles, threads, smem, st>>>(v);
  }
}

template <class R>
static void launch_after_push_impl(const View &v, cudaStream_t st) {
  if (v.qed_any) {
    k_photon_count_reset<<<(v.n_gaps + 255) / 256, 256, 0, st>>>(v);
    k_photons<R><<<4 * 148, 256, 0, st>>>(v);
  }
  if (v.surface_any) k_inject<R><<<(v.n_gaps + 127) / 128, 128, 0, st>>>(v);
  k_house<<<(2 * v.n_tiles + 255) / 256, 256, 0, st>>>(v);
}

template <class R>
static void launch_rebin_impl(const View &v, double slack, cudaStream_t st) {
  k_rebin_layout<<<1, 1024, 0, st>>>(v, slack);
  k_rebin_compact<R><<<2 * v.n_tiles, 256, 0, st>>>(v);
  k_rebin_spill<R><<<64, 256, 0, st>>>(v);
  k_rebin_adopt<<<(2 * v.n_tiles + 255) / 256, 256, 0, st>>>(v);
  k_rebin_finish<<<1, 1, 0, st>>>(v);
}

void launch_push(const View &v, int threads, cudaStream_t st) {
  if (v.precision == GAP_FP32_STATE) launch_push_impl<float>(v, threads, st);
  else launch_push_impl<double>(v, threads, st);
}

void launch_after_push(const View &v, cudaStream_t st) {
  if (v.precision == GAP_FP32_STATE) launch_after_push_impl<float>(v, st);
  else launch_after_push_impl<double>(v, st);
}

void launch_step(const View &v, int threads, cudaStream_t st) {
  launch_push(v, threads, st);
  launch_after_push(v, st);
}

int launches_per_step(const View &v) {
  return 1 + (v.qed_any ? 2 : 0) + (v.surface_any ? 1 : 0) + 1 + (v.merge_any ? 3 : 0) + 5;
}

void launch_sync_used(const View &v, cudaStream_t st) {
  k_sync_used<<<(2 * v.n_tiles + 255) / 256, 256, 0, st>>>(v);
}

void launch_rebin(const View &v, double slack, cudaStream_t st) {
  if (v.precision == GAP_FP32_STATE) launch_rebin_impl<float>(v, slack, st);
  else launch_rebin_impl<double>(v, slack, st);
}

}  // namespace gapk
