// photons.cu -- photon propagation and one-photon pair creation (eq. tau_bw,
// Sect. 6.1), with each photon's fate scheduled ahead of time.
//
// A photon's optical depth depends only on its energy, its direction and the
// time since its birth (the angle to B grows with the path length), and its
// position is a closed form of the step; so the step at which it converts,
// or leaves the domain, follows from its birth record.  The photon pass
// therefore reads one int32 (the event step) per stored photon and step; a
// photon is touched only when it is scheduled (at birth, after an import, or
// every kSchedIters accumulated steps) and at its event.  The accumulation is
// the same sequence of per-step depths that a step-by-step integration adds,
// in the same order, so the event step is the same.  Two shortcuts keep the
// scheduling cheap, both exact: steps where the photon is above the gap
// (QED inhibited, h > H_gap) add nothing and are skipped in closed form, and a
// photon whose remaining depth cannot reach its threshold -- the per-step
// depth is at most dt rate_mult alpha_em / lambda_hat b T_BW(x b), because
// chi T_BW(chi) increases with chi -- goes straight to its escape step.
#include "gap_internal.cuh"
#include "kernels.h"

namespace gapk {

constexpr int kSchedIters = 64;  // accumulated steps per photon per scheduling pass (a multiple of 4)

// Smallest step j >= j0 with pos(j) >= T (dir > 0) or pos(j) < T (dir < 0),
// for a non-periodic gap, where pos is monotone in j.
__device__ int64_t first_step(const GapDev &g, double Xr, int32_t nr, int32_t dir, int64_t j0, double T) {
  auto hit = [&](int64_t j) {
    const double X = photon_pos(g, Xr, nr, dir, j);
    return dir > 0 ? X >= T : X < T;
  };
  if (hit(j0)) return j0;
  // an estimate (the walk below finds the exact step): a product, not a
  // division, which is long on the FP64 units
  const double d = (dir > 0 ? T - Xr : Xr - T) * g.inv_cdx;
  // the exact motion puts the answer within rounding of the estimate: walk
  // the last steps; a long walk falls back to bisection
  {
    int64_t j = (int64_t)nr + (int64_t)ceil(d > 0.0 ? d : 0.0);
    if (j <= j0) j = j0 + 1;
    int guard = 0;
    while (j > j0 + 1 && guard < 8 && hit(j - 1)) {
      --j;
      ++guard;
    }
    while (guard < 16 && !hit(j)) {
      ++j;
      ++guard;
    }
    if (hit(j) && (j == j0 + 1 || !hit(j - 1))) return j;
  }
  int64_t lo = j0;  // !hit(lo)
  int64_t hi = (int64_t)nr + (int64_t)ceil(d > 0.0 ? d : 0.0) + 2;
  if (hi <= lo) hi = lo + 1;
  for (int guard = 0; guard < 62 && !hit(hi); ++guard) hi = lo + 2 * (hi - lo);
  while (hi - lo > 1) {
    const int64_t mid = lo + (hi - lo) / 2;
    if (hit(mid)) hi = mid;
    else lo = mid;
  }
  return hi;
}

template <class R>
struct BwDepth;
template <>
struct BwDepth<double> {
  static __device__ double step(const GapDev &g, double x, int32_t n0, int64_t m) {
    return bw_step_depth(g, x, n0, m);
  }
  static __device__ double bound(const GapDev &g, double x) {
    return g.dt * g.rate_mult * kAlphaEm / g.lambda_hat * g.b * tbw_d(x * g.b);
  }
  static __device__ double add(double a, double b) { return __dadd_rn(a, b); }
  static constexpr double margin = 1e-9;
};
template <>
struct BwDepth<float> {
  static __device__ float step(const GapDev &g, float x, int32_t n0, int64_t m) {
    return bw_step_depth_f(g, x, n0, m);
  }
  static __device__ float bound(const GapDev &g, double x) {
    return g.f_dt * g.f_rate * (float)kAlphaEm / g.f_lam * g.f_b * tbw_f((float)(x * g.b));
  }
  static __device__ float add(float a, float b) { return __fadd_rn(a, b); }
  static constexpr float margin = 2e-2f;  // covers FP32 rounding of sums of up to ~1e5 terms
};

// Optical depth accumulated over the steps [m, n) (active steps only), from
// tau at the start of step m: the same sequence the scheduler adds.
template <class R>
__device__ R photon_depth_at(const GapDev &g, double Xr, int32_t nr, int32_t dir, double x, int32_t n0,
                             int32_t m, R tau, int64_t n) {
  for (int64_t j = m; j < n; ++j)
    if (photon_pos(g, Xr, nr, dir, j) < g.Hc) tau = BwDepth<R>::add(tau, BwDepth<R>::step(g, (R)x, n0, j));
  return tau;
}

// Schedule photon i of buffer b from its checkpoint (tau_acc before step pm).
template <class R>
__device__ void schedule_photon(const View &v, int b, int64_t i) {
  const int gap = v.pgap[b][i];
  const GapDev &g = v.gaps[gap];
  const double Xr = v.pXr[b][i], x = v.px[b][i];
  const R xs = (R)x;  // the energy in the state's precision, converted once
  const int32_t nr = v.pnr[b][i], dir = v.pdir[b][i], n0 = v.pn0[b][i];
  if (v.pkind[b][i] == PH_RESCHEDULE) {  // the walk so far becomes the checkpoint
    v.pm[b][i] = v.pmn[b][i];
    v.pta[b][i] = v.ptan[b][i];
  }
  const int64_t m = v.pm[b][i];
  const R ts = (R)v.pts[b][i];
  R tau = (R)v.pta[b][i];
  int32_t kind, ev;
  if (g.periodic) {
    if (tau >= ts) {
      kind = PH_CONVERT;
      ev = (int32_t)m;
    } else if (BwDepth<R>::bound(g, x) == (R)0) {
      kind = PH_INERT;
      ev = kPhNever;
    } else {
      int64_t j = m;
      kind = 0;
      for (int it = 0; it < kSchedIters; ++it, ++j) {
        if (photon_pos(g, Xr, nr, dir, j) < g.Hc) tau = BwDepth<R>::add(tau, BwDepth<R>::step(g, xs, n0, j));
        if (tau >= ts) {
          kind = PH_CONVERT;
          break;
        }
      }
      if (kind == PH_CONVERT) {
        ev = (int32_t)j;
      } else {
        kind = PH_RESCHEDULE;
        ev = (int32_t)(j - 1);
        v.pmn[b][i] = (int32_t)j;
        v.ptan[b][i] = (double)tau;
      }
    }
  } else {
    // escape step: the first step whose move ends outside [0, nx)
    const int64_t jx = first_step(g, Xr, nr, dir, m + 1, dir > 0 ? (double)g.nx : 0.0) - 1;
    // steps of the life with QED active (start-of-step position below H_gap)
    int64_t lo, hi;
    if (dir > 0) {
      lo = m;
      hi = first_step(g, Xr, nr, dir, m, g.Hc);
    } else {
      lo = first_step(g, Xr, nr, dir, m, g.Hc);
      hi = jx;
    }
    if (hi > jx) hi = jx;
    if (tau >= ts) {
      kind = m == jx ? PH_ESCAPE : PH_CONVERT;
      ev = (int32_t)m;
    } else {
      const R rmax = BwDepth<R>::bound(g, x) * ((R)1 + BwDepth<R>::margin);
      int64_t j = lo > m ? lo : m;
      kind = PH_ESCAPE;
      ev = (int32_t)jx;
      for (int it = 0; j < hi;) {
        if ((it & 63) == 0 && tau + (R)(hi - j) * rmax < ts) break;  // cannot reach its threshold
        if (it == kSchedIters) {
          kind = PH_RESCHEDULE;
          ev = (int32_t)(j - 1);
          v.pmn[b][i] = (int32_t)j;
          v.ptan[b][i] = (double)tau;
          break;
        }
        // four steps' depths at once (independent), added in step order
        const int nb = hi - j < 4 ? (int)(hi - j) : 4;
        R r[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) r[q] = q < nb ? BwDepth<R>::step(g, xs, n0, j + q) : (R)0;
        bool conv = false;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (q >= nb || conv) continue;
          tau = BwDepth<R>::add(tau, r[q]);
          if (tau >= ts) {
            kind = PH_CONVERT;
            ev = (int32_t)(j + q);
            conv = true;
          }
        }
        if (conv) break;
        j += nb;
        it += nb;
      }
    }
  }
  v.pkind[b][i] = kind;
  v.pev[b][i] = ev;
}

// The event of photon i at step `step`: conversion into an e-e+ pair at the
// photon's new position (gamma = x/2 each, or with qed_quantum the electron
// e x with e from the differential rate at this step's chi, both at least 1),
// or escape through a boundary.
template <class R>
__device__ void photon_event(const View &v, int b, int64_t i, int64_t step) {
  using W = typename Prec<R>::W;
  const int kind = v.pkind[b][i];
  const int gap = v.pgap[b][i];
  const GapDev &g = v.gaps[gap];
  const double x = v.px[b][i], w = v.pw[b][i];
  if (kind == PH_ESCAPE) {
    atomicAdd(&v.counters[gap * C_NCNT + C_PH_ESCAPED], 1ull);
    atomicAdd(&v.ledger[gap * L_NLED + L_PH_ESC], w * x);
  } else if (kind == PH_CONVERT) {
    const int32_t dir = v.pdir[b][i];
    const double X1 = photon_pos(g, v.pXr[b][i], v.pnr[b][i], dir, step + 1);
    const uint64_t id = v.pid[b][i];
    double ge = 0.5 * x;
    if (g.qed_quantum) {
      const double lmid = ((double)step - (double)v.pn0[b][i] + 0.5) * g.dt;
      const double chi = x * g.b * fabs(sin(lmid / g.rho_hat));
      const double e = bw_split(v, chi, uniform53(g.seed, id, (uint32_t)step, CH_PAIR_E, 0), sizeof(R) == 8);
      // each share at least one rest mass, clamped on the energies (a
      // clamp on e would leave (1/x) x just below 1 for some x)
      ge = e * x;
      if (ge < 1.0) ge = 1.0;
      if (x - ge < 1.0) ge = x - 1.0;
    }
    int32_t k;
    R phi;
    split_position<R>(X1, g.nx, g.periodic != 0, k, phi);
    const int tn = tile_of(v, g, k);
    W wq;
    if (sizeof(R) == 4) wq = (W)llrint(w / g.w_unit);
    else wq = (W)w;
    for (int s = 0; s < 2; ++s) {
      const double gs = s == 0 ? ge : x - ge;
      const double ps = (gs - 1.0) * (gs + 1.0);
      const double up = (double)dir * sqrt(ps > 0.0 ? ps : 0.0);
      const uint64_t lid = child_id(id, (uint32_t)step, CH_PAIR, (uint32_t)s) & ~kPhotonBit;
      const R tau = (R)(-log(uniform53(g.seed, lid, (uint32_t)(step + 1), CH_TAU0, 0)));
      append_lepton<R>(v, s, tn, k, phi, (R)up, wq, tau, lid);
    }
    atomicAdd(&v.counters[gap * C_NCNT + C_PAIRS], 1ull);
  } else {
    return;
  }
  v.pev[b][i] = kPhDead;
  atomicSub(&v.ph_gap[gap], 1);
  const unsigned mask = __activemask();  // one count per warp of the dead since the last compaction
  if ((threadIdx.x & 31) == __ffs(mask) - 1)
    atomicAdd(reinterpret_cast<unsigned long long *>(&v.ctl->ph_dead), (unsigned long long)__popc(mask));
}

// Photon pass of step n, part 1: a scan of the event steps.  Every photon
// with something to do this step (new or imported and not yet scheduled, at
// its re-schedule step, or at its event) goes to a dense work list, so that
// the scan streams the event steps and the work runs in full warps.  Each
// warp gathers its photons in shared memory and reserves their slots of the
// list with one atomic per ~256 (one counter serves the whole GPU: reserving
// a few at a time had the scan wait on it).
constexpr int kScanBuf = 256;  // photons a warp gathers before it reserves

__global__ void __launch_bounds__(256, 5) k_photon_scan(View v) {
  __shared__ long long sbuf[8][kScanBuf + 128];  // <= 8 warps; a warp adds at most 128 at a time
  const int b = v.ctl->ph_cur;
  const int64_t n = photon_fill(v, b);
  const int64_t step = v.ctl->step;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  long long *wb = sbuf[wid];
  int wn = 0;  // warp-uniform
  auto flush = [&]() {
    unsigned long long base = 0ull;
    if (lane == 0) base = atomicAdd(reinterpret_cast<unsigned long long *>(&v.ctl->ph_work_n), (unsigned long long)wn);
    base = __shfl_sync(0xffffffffu, base, 0);
    for (int j = lane; j < wn; j += 32) v.ph_work[base + j] = wb[j];
    __syncwarp();
    wn = 0;
  };
  auto due = [&](int32_t ev) { return ev == kPhPending || ev == step; };
  const int32_t *ev1 = v.pev[b];
  const int4 *ev4 = reinterpret_cast<const int4 *>(ev1);
  const int64_t n4 = (n + 3) / 4;  // four event steps per 16-byte load; a ragged last vector as scalars
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // warp-uniform trip count (lanes past the end hold dead photons)
  for (int64_t q0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); q0 < n4; q0 += stride) {
    const int64_t q = q0 + lane;
    int32_t e[4] = {kPhDead, kPhDead, kPhDead, kPhDead};
    if (4 * q + 3 < n) {
      const int4 x = ev4[q];
      e[0] = x.x;
      e[1] = x.y;
      e[2] = x.z;
      e[3] = x.w;
    } else if (q < n4) {
      for (int j = 0; 4 * q + j < n; ++j) e[j] = ev1[4 * q + j];
    }
    unsigned mine = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (due(e[j])) mine |= 1u << j;
      else if (e[j] != kPhDead && e[j] < step) atomicOr(&v.ctl->error, 64);  // never: events are taken at their step
    }
    // a lane's photons go after those of the lanes below it
    const unsigned below = (1u << lane) - 1u;
    int before = 0, total = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const unsigned bj = __ballot_sync(0xffffffffu, (mine >> j) & 1u);
      before += __popc(bj & below);
      total += __popc(bj);
    }
    if (total == 0) continue;  // warp-uniform
    if (wn + total > kScanBuf) flush();
    int pos = wn + before;
    for (unsigned m = mine; m; m &= m - 1u) wb[pos++] = 4 * q + (__ffs(m) - 1);
    wn += total;
    __syncwarp();
  }
  if (wn > 0) flush();
}

// Part 2 (four blocks of 256 threads per SM, at most 64 registers: the
// kernel is latency-bound and needs the warps, and at five blocks, 51
// registers, it measured 2 % slower): the work list, one photon per thread:
// a photon to be scheduled (new, imported, or at its re-schedule step) is
// scheduled, and may have its event in this very step; a photon at its
// event converts or escapes.
template <class R>
__global__ void __launch_bounds__(256, 4) k_photon_schedule(View v) {
  const int b = v.ctl->ph_cur;
  const int64_t n = v.ctl->ph_work_n;
  const int64_t step = v.ctl->step;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = v.ph_work[t];
    if (v.pev[b][i] == kPhPending || v.pkind[b][i] == PH_RESCHEDULE) schedule_photon<R>(v, b, i);
    if (v.pev[b][i] == step) photon_event<R>(v, b, i, step);
  }
}

__global__ void k_photon_work_reset(View v) { v.ctl->ph_work_n = 0; }

// Compaction of the photon store into the other buffer (once a quarter of
// the store is dead, or it is half full): the survivors keep their records;
// the order is not kept.  A block takes kPhCompactPer photons per thread in a
// round and reserves its survivors' slots with one atomic (one counter
// serves the whole GPU: an atomic per warp had the copy wait on it).
constexpr int kPhCompactPer = 4;
__global__ void __launch_bounds__(256) k_photon_compact(View v) {
  if (!v.ctl->need_ph_compact) return;
  __shared__ int wcnt[8];  // <= 8 warps
  __shared__ long long sbase;
  const int b = v.ctl->ph_cur, o = b ^ 1;
  const int64_t n = photon_fill(v, b);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int64_t per_round = (int64_t)blockDim.x * kPhCompactPer;
  for (int64_t r0 = (int64_t)blockIdx.x * per_round; r0 < n; r0 += (int64_t)gridDim.x * per_round) {
    // photon r0 + j blockDim + thread: the j-th vector of the warp's lanes;
    // survivors of vector j go after those of vectors < j, in lane order
    unsigned bal[kPhCompactPer];
    int total = 0;
#pragma unroll
    for (int j = 0; j < kPhCompactPer; ++j) {
      const int64_t i = r0 + (int64_t)j * blockDim.x + threadIdx.x;
      bal[j] = __ballot_sync(0xffffffffu, i < n && v.pev[b][i] != kPhDead);
      total += __popc(bal[j]);
    }
    if (lane == 0) wcnt[wid] = total;
    __syncthreads();
    if (threadIdx.x == 0) {
      int acc = 0;
      for (int w = 0; w < nw; ++w) {
        const int c = wcnt[w];
        wcnt[w] = acc;
        acc += c;
      }
      sbase = acc > 0 ? (long long)atomicAdd(reinterpret_cast<unsigned long long *>(&v.ctl->ph_count[o]),
                                             (unsigned long long)acc)
                      : 0ll;
    }
    __syncthreads();
    long long d0 = sbase + wcnt[wid];
    const unsigned below = (1u << lane) - 1u;
#pragma unroll
    for (int j = 0; j < kPhCompactPer; ++j) {
      const long long d = d0 + __popc(bal[j] & below);
      d0 += __popc(bal[j]);
      if (!((bal[j] >> lane) & 1u)) continue;
      const int64_t i = r0 + (int64_t)j * blockDim.x + threadIdx.x;
      v.pXr[o][d] = v.pXr[b][i];
      v.px[o][d] = v.px[b][i];
      v.pw[o][d] = v.pw[b][i];
      v.pts[o][d] = v.pts[b][i];
      v.pta[o][d] = v.pta[b][i];
      v.pid[o][d] = v.pid[b][i];
      v.pn0[o][d] = v.pn0[b][i];
      v.pnr[o][d] = v.pnr[b][i];
      v.pdir[o][d] = v.pdir[b][i];
      v.pgap[o][d] = v.pgap[b][i];
      v.pm[o][d] = v.pm[b][i];
      v.pmn[o][d] = v.pmn[b][i];
      v.ptan[o][d] = v.ptan[b][i];
      v.pkind[o][d] = v.pkind[b][i];
      v.pev[o][d] = v.pev[b][i];
    }
    __syncthreads();  // wcnt and sbase are rewritten by the next round
  }
}

__global__ void k_photon_flip(View v) {
  Ctl *c = v.ctl;
  if (!c->need_ph_compact) return;
  const int b = c->ph_cur;
  c->ph_count[b] = 0;
  c->ph_cur = b ^ 1;
  c->ph_dead = 0;
  c->need_ph_compact = 0;
  c->ph_nb_start = 0;  // survivors in any order: the photon merge scans them all
}

void launch_photon_step(const View &v, cudaStream_t st) {
  k_photon_work_reset<<<1, 1, 0, st>>>(v);
  if (v.precision == GAP_FP32_STATE) {
    k_photon_scan<<<16 * 148, 256, 0, st>>>(v);  // many loads in flight
    k_photon_schedule<float><<<4 * 148, 256, 0, st>>>(v);
  } else {
    k_photon_scan<<<16 * 148, 256, 0, st>>>(v);
    k_photon_schedule<double><<<4 * 148, 256, 0, st>>>(v);
  }
}

void launch_photon_compact(const View &v, cudaStream_t st) {
  k_photon_compact<<<4 * 148, 256, 0, st>>>(v);
  k_photon_flip<<<1, 1, 0, st>>>(v);
}

// Photon state at the start of the current step for export: position and
// optical depth replayed from the checkpoint.
template <class R>
__global__ void k_export_photons_t(View v, int gap, double *stage, int64_t cap, unsigned long long *count) {
  const int b = v.ctl->ph_cur;
  const int64_t n = photon_fill(v, b);
  const int64_t step = v.ctl->step;
  const GapDev &g = v.gaps[gap];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (v.pgap[b][i] != gap || v.pev[b][i] == kPhDead) continue;
    const unsigned long long o = atomicAdd(count, 1ull);
    if ((int64_t)o >= cap) continue;
    const double Xr = v.pXr[b][i], x = v.px[b][i];
    const int32_t nr = v.pnr[b][i], dir = v.pdir[b][i], n0 = v.pn0[b][i];
    const int64_t m = v.pm[b][i];
    const double ta = (double)photon_depth_at<R>(g, Xr, nr, dir, x, n0, (int32_t)m, (R)v.pta[b][i],
                                                 m < step ? step : m);
    reinterpret_cast<uint64_t *>(stage)[o] = v.pid[b][i];
    stage[cap + o] = photon_pos(g, Xr, nr, dir, step);
    stage[2 * cap + o] = x;
    stage[3 * cap + o] = v.pw[b][i];
    stage[4 * cap + o] = ta;
    stage[5 * cap + o] = v.pts[b][i];
    reinterpret_cast<int64_t *>(stage)[6 * cap + o] = ((int64_t)n0 << 1) | (dir > 0 ? 1 : 0);
  }
}

void launch_export_photons(const View &v, int gap, double *stage, int64_t cap, unsigned long long *count,
                           cudaStream_t st) {
  if (v.precision == GAP_FP32_STATE) k_export_photons_t<float><<<148, 256, 0, st>>>(v, gap, stage, cap, count);
  else k_export_photons_t<double><<<148, 256, 0, st>>>(v, gap, stage, cap, count);
}

__global__ void k_import_photons(View v, int gap, int64_t n, const double *stage) {
  const int b = v.ctl->ph_cur;
  const int32_t step = (int32_t)v.ctl->step;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t id = reinterpret_cast<const uint64_t *>(stage)[i] | kPhotonBit;
    const int64_t aux = reinterpret_cast<const int64_t *>(stage)[6 * n + i];
    if (photon_append(v, b, gap, stage[n + i], step, stage[2 * n + i], stage[3 * n + i], stage[5 * n + i],
                      stage[4 * n + i], id, (int32_t)(aux >> 1), (aux & 1) ? 1 : -1, step))
      atomicAdd(&v.ph_gap[gap], 1);
  }
}

void launch_import_photons(const View &v, int gap, int64_t n, const double *stage, cudaStream_t st) {
  const int blocks = (int)((n + 255) / 256 < 1184 ? (n + 255) / 256 : 1184);
  if (n > 0) k_import_photons<<<blocks, 256, 0, st>>>(v, gap, n, stage);
}

// Photon moments of one gap at the start of the current step: density per
// cell (dmom row 7), energy sum w x (dred[17]) and count (dred[20]).
__global__ void k_photon_moments(View v, int gap) {
  const int b = v.ctl->ph_cur;
  const int64_t n = photon_fill(v, b);
  const int64_t step = v.ctl->step;
  const GapDev &g = v.gaps[gap];
  double en = 0.0;
  unsigned long long cnt = 0;  // summed per warp: one global atomic per warp, not per photon
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (v.pgap[b][i] != gap || v.pev[b][i] == kPhDead) continue;
    const double X = photon_pos(g, v.pXr[b][i], v.pnr[b][i], v.pdir[b][i], step);
    int64_t c = (int64_t)floor(X);
    if (c < 0) c = 0;
    if (c >= g.nx) c = g.nx - 1;
    atomicAdd(&v.dmom[7 * g.nx + c], v.pw[b][i] / g.dx);
    en += v.pw[b][i] * v.px[b][i];
    ++cnt;
  }
  for (int o = 16; o > 0; o >>= 1) {
    en += __shfl_down_sync(0xffffffffu, en, o);
    cnt += __shfl_down_sync(0xffffffffu, cnt, o);
  }
  if ((threadIdx.x & 31) == 0 && cnt) {
    atomicAdd(&v.dred[17], en);
    atomicAdd(reinterpret_cast<unsigned long long *>(&v.dred[20]), cnt);
  }
}

void launch_photon_moments(const View &v, int gap, cudaStream_t st) {
  k_photon_moments<<<4 * 148, 256, 0, st>>>(v, gap);
}

}  // namespace gapk
