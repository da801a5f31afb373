// init.cu -- initial loads, Gauss solve, diagnostics (moments, reductions,
// FFT of E) and particle export/import.
#include "gap_internal.cuh"
#include "kernels.h"

namespace gapk {

// ---------------------------------------------------------------------------
// Loader: quiet start X = cell + (j + 1/2)/ppc; for the thermal pair load the
// electrons are displaced by (A/k1) sin(k1 X), k1 = 2 pi/nx (a Langmuir seed
// of relative density amplitude A) and momenta are 1D Maxwell-Juttner by the
// mj_draw_b (step 0, channel CH_INIT_U, the bound formed once).
template <class R>
__global__ void k_load(View v, LoadSpec sp) {
  using W = typename Prec<R>::W;
  const GapDev &g = v.gaps[sp.gap];
  const int64_t total = sp.n_per_species * sp.species_count;
  const double w = (sp.init == GAP_INIT_PAIR_THERMAL ? 0.5 : 1.0) * sp.density * g.dx / (double)sp.ppc;
  const double k1 = 2.0 * 3.141592653589793 / (double)g.nx;
  const double bmax = sp.theta > 0.0 ? mj_bmax(sp.theta) : 0.0;
  const bool full_state = v.qed_any || v.has_w;  // the lean store keeps no optical depth
  // warp-uniform grid-stride loop (the append is a warp collective); lanes
  // past the end take part without appending
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; p0 < total; p0 += stride) {
    const int64_t p = p0 + lane;
    const bool valid = p < total;
    int s = 0, t = 0;
    int32_t k = 0;
    R phi = (R)1;
    double u = 0.0, tau = 0.0;
    uint64_t id = 0;
    if (valid) {
      s = (int)(p / sp.n_per_species);
      const int64_t idx = p % sp.n_per_species;
      const int64_t cell = idx / sp.ppc, j = idx % sp.ppc;
      id = ((uint64_t)g.gap_index << 40) | ((uint64_t)s << 39) | (uint64_t)(cell * sp.ppc + j);
      double X = (double)cell + ((double)j + 0.5) / (double)sp.ppc;
      if (sp.init == GAP_INIT_PAIR_THERMAL) {
        if (s == 0 && sp.seed_amp != 0.0) {
          X += sp.seed_amp / k1 * sin(k1 * X);
          // X mod nx: within (-nx, 2 nx) one exact subtraction or addition
          // gives fmod's result (fmod is a long FP64 sequence)
          const double L = (double)g.nx;
          if (X >= L && X < 2.0 * L) X -= L;
          else if (!(X >= 0.0 && X < L)) X = fmod(X, L);
          if (X < 0.0) X += L;
        }
        if (sp.theta > 0.0) {
          bool ok = true;
          u = mj_draw_b(g.seed, id, 0, CH_INIT_U, sp.theta, bmax, ok);
          if (!ok) atomicAdd(&v.counters[sp.gap * C_NCNT + C_LOAD_OVF], 1ull);
        }
      }
      if (full_state) tau = -log(uniform53(g.seed, id, 0, CH_TAU0, 0));
      split_position<R>(X, g.nx, g.periodic != 0, k, phi);
      t = tile_of(v, g, k);
    }
    W wq;
    if (sizeof(R) == 4) wq = (W)(1u << kWeightShift);
    else wq = (W)w;
    append_lepton_warp<R>(v, valid, s, t, k, phi, (R)u, wq, (R)tau, id);
  }
}

// Protons of the Sect. 6.1 start: the quiet-start positions of the electrons
// below H_gap, at rest, weight w0 (FP64 state), ids with species bit 1.
__global__ void k_load_protons(View v, int gap, int64_t n) {
  const GapDev &g = v.gaps[gap];
  const int64_t ppc = n / g.nx;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = p / ppc, j = p % ppc;
    const double X = (double)cell + ((double)j + 0.5) / (double)ppc;
    if (!(X < g.Hc)) continue;
    const long long i = (long long)atomicAdd(reinterpret_cast<unsigned long long *>(&v.ctl->pr_count), 1ull);
    if (i >= v.pr_cap) {
      atomicOr(&v.ctl->error, 128);  // proton storage exhausted
      continue;
    }
    v.pr_X[i] = v.precision == GAP_FP32_STATE ? grid_position(X) : X;
    v.pr_u[i] = 0.0;
    v.pr_w[i] = g.w0;
    v.pr_id[i] = ((uint64_t)g.gap_index << 40) | (1ull << 39) | (uint64_t)(cell * ppc + j);
    v.pr_gap[i] = gap;
    v.pr_alive[i] = 1;
  }
}

void launch_load_protons(const View &v, int gap, int64_t n, cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 148 * 8);
  if (n > 0) k_load_protons<<<blocks, 256, 0, st>>>(v, gap, n);
}

// Charge of the protons per cell (cloud in cell) into Q: all gaps at their
// node offsets (gap < 0, the Gauss solve), or one gap from 0 (the diagnostics).
__global__ void k_proton_charge(View v, int gap, unsigned long long *Q) {
  const int64_t n = v.ctl->pr_count < v.pr_cap ? v.ctl->pr_count : v.pr_cap;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (!v.pr_alive[i]) continue;
    const int gi = v.pr_gap[i];
    if (gap >= 0 && gi != gap) continue;
    const GapDev &g = v.gaps[gi];
    const int64_t off = gap >= 0 ? 0 : g.node_off;
    const double X = v.pr_X[i];
    const int64_t c0 = (int64_t)floor(X - 0.5);
    for (int64_t c = c0; c <= c0 + 1; ++c) {
      const double a = X - (double)c, b = X - (double)c - 1.0;
      const double fa = a + 0.5 < 0.0 ? 0.0 : (a + 0.5 > 1.0 ? 1.0 : a + 0.5);
      const double fb = b + 0.5 < 0.0 ? 0.0 : (b + 0.5 > 1.0 ? 1.0 : b + 0.5);
      const double fr = fa - fb;
      if (fr == 0.0) continue;
      int64_t cc = c;
      if (g.periodic) cc = (c % g.nx + g.nx) % g.nx;
      else if (c < 0 || c >= g.nx) continue;
      if (v.precision == GAP_FP32_STATE)  // whole charge units (positions on the offset grid)
        atomicAdd(&Q[off + cc], (unsigned long long)(grid_units(fr) * (1ll << kWeightShift)));
      else
        atomicAdd(reinterpret_cast<double *>(&Q[off + cc]), v.pr_w[i] * fr);
    }
  }
}

// Export of one gap's live protons (every stride-th by id), lepton layout.
__global__ void k_export_protons(View v, int gap, double *stage, int64_t cap, unsigned long long *count,
                                 int64_t stride) {
  const int64_t n = v.ctl->pr_count < v.pr_cap ? v.ctl->pr_count : v.pr_cap;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (!v.pr_alive[i] || v.pr_gap[i] != gap) continue;
    if (stride > 1 && (v.pr_id[i] % (uint64_t)stride) != 0) continue;
    const unsigned long long o = atomicAdd(count, 1ull);
    if ((int64_t)o >= cap) continue;
    reinterpret_cast<uint64_t *>(stage)[o] = v.pr_id[i];
    stage[cap + o] = v.pr_X[i];
    stage[2 * cap + o] = v.pr_u[i];
    stage[3 * cap + o] = v.pr_w[i];
    stage[4 * cap + o] = 1e30;  // no optical depth: protons do not radiate
  }
}

void launch_export_protons(const View &v, int gap, double *stage, int64_t cap, unsigned long long *count,
                           int64_t stride, cudaStream_t st) {
  k_export_protons<<<148, 256, 0, st>>>(v, gap, stage, cap, count, stride);
}

void launch_load(const View &v, const LoadSpec *spec, int n_specs, int64_t max_n, cudaStream_t st) {
  (void)max_n;
  for (int i = 0; i < n_specs; ++i) {
    const LoadSpec &sp = spec[i];
    const int64_t total = sp.n_per_species * sp.species_count;
    if (total <= 0) continue;
    int blocks = (int)((total + 255) / 256);
    if (blocks > 148 * 32) blocks = 148 * 32;
    if (v.precision == GAP_FP32_STATE) k_load<float><<<blocks, 256, 0, st>>>(v, sp);
    else k_load<double><<<blocks, 256, 0, st>>>(v, sp);
  }
}

__global__ void k_set_rebin(View v) { v.ctl->need_rebin = 1; }
void launch_force_rebin(const View &v, cudaStream_t st) { k_set_rebin<<<1, 1, 0, st>>>(v); }

// ---------------------------------------------------------------------------
// Cell charges of every gap (cloud in cell: a lepton at dual cell k with
// offset phi' puts 2 - phi' of its charge in cell k-1 and phi' - 1 in cell
// k), exact in the FP32 state (integer units w_unit 2^-23).
template <class R>
__device__ __forceinline__ void cell_fracs(R phi, long long &fl, long long &fr, double &dl, double &dr) {
  if (sizeof(R) == 4) {
    const int F = __float2int_rn(((float)phi - 1.0f) * 8388608.0f);
    fr = F;
    fl = (1 << kPhiBits) - F;
  } else {
    dr = (double)phi - 1.0;
    dl = 2.0 - (double)phi;
  }
}

template <class R>
__global__ void k_cell_charge(View v, int only_gap, unsigned long long *Q) {
  using W = typename Prec<R>::W;
  const int t = blockIdx.x;
  const TileDev ti = v.tiles[t];
  if (only_gap >= 0 && ti.gap != only_gap) return;
  const GapDev &g = v.gaps[ti.gap];
  const int cur = v.ctl->lep_cur;
  const int64_t off = only_gap >= 0 ? 0 : g.node_off;
  for (int s = 0; s < 2; ++s) {
    const int q = s == 0 ? -1 : 1;
    const int64_t start = v.seg_start[s][t];
    const int used = v.seg_used[s][t];
    for (int i = threadIdx.x; i < used; i += blockDim.x) {
      const int64_t slot = start + i;
      const int32_t k = v.lk[cur][s][slot];
      if (k < 0) continue;
      const R phi = as<R>(v.lphi[cur][s])[slot];
      const W w = lepton_weight<R>(v, g, cur, s, slot);
      long long fl = 0, fr = 0;
      double dl = 0, dr = 0;
      cell_fracs<R>(phi, fl, fr, dl, dr);
      for (int side = 0; side < 2; ++side) {
        int64_t c = side == 0 ? (int64_t)k - 1 : (int64_t)k;
        if (g.periodic) c = (c + g.nx) % g.nx;
        else if (c < 0 || c >= g.nx) continue;
        if (sizeof(R) == 4) {
          const long long val = (long long)q * (long long)w * (side == 0 ? fl : fr);
          atomicAdd(&Q[off + c], (unsigned long long)val);
        } else {
          const double val = (double)q * (double)w * (side == 0 ? dl : dr);
          atomicAdd(reinterpret_cast<double *>(&Q[off + c]), val);
        }
      }
    }
  }
}

__device__ __forceinline__ double charge_value(const View &v, const GapDev &g, unsigned long long bits) {
  if (v.precision == GAP_FP32_STATE) return (double)(long long)bits * g.w_unit * kPhiUnit;
  return __longlong_as_double((long long)bits);
}

// Block-wide exclusive scan of one double per thread; returns the prefix.
__device__ double block_exclusive_scan(double x, double *total) {
  __shared__ double ws[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double y = x;
  for (int o = 1; o < 32; o <<= 1) {
    double z = __shfl_up_sync(0xffffffffu, y, o);
    if (lane >= o) y += z;
  }
  if (lane == 31) ws[wid] = y;
  __syncthreads();
  if (wid == 0) {
    double a = lane < (int)(blockDim.x >> 5) ? ws[lane] : 0.0;
    for (int o = 1; o < 32; o <<= 1) {
      double z = __shfl_up_sync(0xffffffffu, a, o);
      if (lane >= o) a += z;
    }
    ws[lane] = a;
  }
  __syncthreads();
  const double before = (wid > 0 ? ws[wid - 1] : 0.0) + y - x;
  if (total) *total = ws[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before;
}

// P binomial passes over the cell array a[0..n) of one gap, run by one block
// (a periodic gap wraps; a surface gap mirrors the charge oddly about its end
// nodes: a[-1] = -a[0], a[n] = -a[n-1]), ping-ponging between a and b in
// global memory.  Returns the buffer that holds the result.
__device__ double *filter_cells_block(double *a, double *b, int64_t n, int P, bool periodic) {
  for (int p = 0; p < P; ++p) {
    __syncthreads();
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
      const double l = i > 0 ? a[i - 1] : (periodic ? a[n - 1] : -a[0]);
      const double r = i < n - 1 ? a[i + 1] : (periodic ? a[0] : -a[n - 1]);
      b[i] = 0.25 * (l + 2.0 * a[i] + r);
    }
    double *t = a;
    a = b;
    b = t;
  }
  __syncthreads();
  return a;
}

// Gauss's law (Sect. 2.2) per gap, one block each: E_0 = 0 and
// E_{c+1} = E_c + Q_c - eta_bg dx; periodic gaps take zero-mean E.  A gap
// with a current filter takes the field of the smoothed Q_c - eta_bg dx.
__global__ void __launch_bounds__(1024) k_gauss_scan(View v, int set_background) {
  const int gi = blockIdx.x;
  GapDev &g = v.gaps[gi];
  const int64_t nx = g.nx;
  double *E = v.E[v.ctl->e_cur] + g.node_off;
  const unsigned long long *Q = v.dcharge + g.node_off;
  const int T = blockDim.x;
  const int64_t chunk = (nx + T - 1) / T;
  const int64_t c0 = threadIdx.x * chunk;
  const int64_t c1 = c0 + chunk < nx ? c0 + chunk : nx;
  double local = 0.0;
  for (int64_t c = c0; c < c1; ++c) local += charge_value(v, g, Q[c]);
  double total = 0.0;
  (void)block_exclusive_scan(local, &total);
  __shared__ double eta;
  if (threadIdx.x == 0) {
    if (set_background && g.periodic) g.eta_bg = total / ((double)nx * g.dx);
    eta = g.eta_bg;
  }
  __syncthreads();
  const double bg = eta * g.dx;
  const double *Qs = nullptr;  // smoothed Q_c - bg of a filter gap
  if (g.filter_passes > 0) {
    double *A = v.Dflt + g.node_off, *B = v.Dflt + v.dcharge_len + g.node_off;
    for (int64_t c = threadIdx.x; c < nx; c += T) A[c] = charge_value(v, g, Q[c]) - bg;
    Qs = filter_cells_block(A, B, nx, g.filter_passes, g.periodic != 0);
  }
  auto qv = [&](int64_t c) { return Qs ? Qs[c] : charge_value(v, g, Q[c]) - bg; };
  // prefix of (Q_c - bg) over the cells of the preceding threads
  double mine = 0.0;
  for (int64_t c = c0; c < c1; ++c) mine += qv(c);
  double run = block_exclusive_scan(mine, nullptr);
  const int64_t last = g.periodic ? nx - 1 : nx;  // E has nodes 0..last
  if (threadIdx.x == 0) E[0] = 0.0;
  for (int64_t c = c0; c < c1; ++c) {
    run += qv(c);
    if (c + 1 <= last) E[c + 1] = run;
  }
  if (g.periodic) {
    __syncthreads();
    double part = 0.0;
    for (int64_t i = threadIdx.x; i < nx; i += T) part += E[i];
    double tot = 0.0;
    (void)block_exclusive_scan(part, &tot);
    const double mean = tot / (double)nx;
    __syncthreads();
    for (int64_t i = threadIdx.x; i < nx; i += T) E[i] -= mean;
  }
  // both E buffers start equal
  __syncthreads();
  double *E2 = v.E[v.ctl->e_cur ^ 1] + g.node_off;
  for (int64_t i = threadIdx.x; i < g.nnode; i += T) E2[i] = E[i];
}

void launch_gauss(const View &v, int set_background, cudaStream_t st) {
  // dcharge covers every node of every gap (>= every cell)
  cudaMemsetAsync(v.dcharge, 0, sizeof(unsigned long long) * (size_t)v.dcharge_len, st);
  if (v.precision == GAP_FP32_STATE) k_cell_charge<float><<<v.n_tiles, 256, 0, st>>>(v, -1, v.dcharge);
  else k_cell_charge<double><<<v.n_tiles, 256, 0, st>>>(v, -1, v.dcharge);
  if (v.pr_any) k_proton_charge<<<148 * 4, 256, 0, st>>>(v, -1, v.dcharge);
  k_gauss_scan<<<v.n_gaps, 1024, 0, st>>>(v, set_background);
}

// ---------------------------------------------------------------------------
// Diagnostics of one gap (Sect. 6.2 Fig. 5, Sect. 6.6 Fig. 8).
// dmom layout: [0..3] density of (species, direction) per cell, [4] sum w
// gamma^-3, [5] sum w, [6] charge (double copy), [7] photon density.
// One block per tile.  With priv, the tile's cells k0-1 .. k0+nk-1 are summed
// in shared memory and added to the gap's arrays once per cell (the leptons
// of a tile crowd few cells, and their global atomics had contended).
template <class R>
__global__ void __launch_bounds__(256) k_moments(View v, int gap, int priv) {
  using W = typename Prec<R>::W;
  const GapDev &g = v.gaps[gap];
  const int t = g.tile_begin + blockIdx.x;
  const TileDev ti = v.tiles[t];
  const int cur = v.ctl->lep_cur;
  const int64_t nx = g.nx;
  double *M = v.dmom;
  const int ncell = ti.nk + 1;
  extern __shared__ __align__(16) unsigned char msh[];
  double *sM = reinterpret_cast<double *>(msh);                                  // [6][ncell]
  unsigned long long *sQ = reinterpret_cast<unsigned long long *>(sM + 6 * ncell);  // [ncell]
  if (priv) {
    for (int i = threadIdx.x; i < 6 * ncell; i += blockDim.x) sM[i] = 0.0;
    for (int i = threadIdx.x; i < ncell; i += blockDim.x) sQ[i] = 0ull;
    __syncthreads();
  }
  double en = 0.0;
  for (int s = 0; s < 2; ++s) {
    const int q = s == 0 ? -1 : 1;
    const int64_t start = v.seg_start[s][t];
    const int used = v.seg_used[s][t];
    for (int i = threadIdx.x; i < used; i += blockDim.x) {
      const int64_t slot = start + i;
      const int32_t k = v.lk[cur][s][slot];
      if (k < 0) continue;
      const R phi = as<R>(v.lphi[cur][s])[slot];
      const double u = (double)as<R>(v.lu[cur][s])[slot];
      const W wq = lepton_weight<R>(v, g, cur, s, slot);
      const double w = sizeof(R) == 4 ? (double)wq * g.w_unit : (double)wq;
      const double gm = sqrt(1.0 + u * u);
      en += w * gm;
      const int dir = u >= 0.0 ? 0 : 1;
      long long fl = 0, fr = 0;
      double dl = 0, dr = 0;
      cell_fracs<R>(phi, fl, fr, dl, dr);
      if (sizeof(R) == 4) {
        dl = (double)fl * kPhiUnit;
        dr = (double)fr * kPhiUnit;
      }
      for (int side = 0; side < 2; ++side) {
        const double fr_ = side == 0 ? dl : dr;
        if (fr_ == 0.0) continue;
        const int64_t cu = side == 0 ? (int64_t)k - 1 : (int64_t)k;  // before the wrap
        const int64_t lc = cu - (ti.k0 - 1);
        const long long qv = sizeof(R) == 4 ? (long long)q * (long long)wq * (side == 0 ? fl : fr) : 0ll;
        if (priv && lc >= 0 && lc < ncell) {
          atomicAdd(&sM[(s * 2 + dir) * ncell + lc], w * fr_ / g.dx);
          atomicAdd(&sM[4 * ncell + lc], w * fr_ / (gm * gm * gm));
          atomicAdd(&sM[5 * ncell + lc], w * fr_);
          if (sizeof(R) == 4) atomicAdd(&sQ[lc], (unsigned long long)qv);
          else atomicAdd(reinterpret_cast<double *>(&sQ[lc]), (double)q * w * fr_);
          continue;
        }
        int64_t c = cu;
        if (g.periodic) c = (c + nx) % nx;
        else if (c < 0 || c >= nx) continue;
        atomicAdd(&M[(s * 2 + dir) * nx + c], w * fr_ / g.dx);
        atomicAdd(&M[4 * nx + c], w * fr_ / (gm * gm * gm));
        atomicAdd(&M[5 * nx + c], w * fr_);
        if (sizeof(R) == 4) atomicAdd(&v.dcharge[c], (unsigned long long)qv);
        else atomicAdd(reinterpret_cast<double *>(&v.dcharge[c]), (double)q * w * fr_);
      }
    }
  }
  if (priv) {
    __syncthreads();
    for (int lc = threadIdx.x; lc < ncell; lc += blockDim.x) {
      int64_t c = (int64_t)ti.k0 - 1 + lc;
      if (g.periodic) c = (c + nx) % nx;
      else if (c < 0 || c >= nx) continue;
      for (int row = 0; row < 6; ++row) {
        const double x = sM[row * ncell + lc];
        if (x != 0.0) atomicAdd(&M[row * nx + c], x);
      }
      if (sQ[lc] != 0ull) {
        if (sizeof(R) == 4) atomicAdd(&v.dcharge[c], sQ[lc]);
        else atomicAdd(reinterpret_cast<double *>(&v.dcharge[c]), __longlong_as_double((long long)sQ[lc]));
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) en += __shfl_down_sync(0xffffffffu, en, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(&v.dred[16], en);
}

// One block: peak and mean multiplicity over the gap cells, <gamma^-3> at
// the peak, E extrema, Gauss residual, field energy.  dred layout:
// 0 M_peak, 1 M_avg, 2 peak cell, 3 g3_peak, 4-7 split, 8 E_min, 9 E_max,
// 10 gauss residual, 11 |E| max, 12 field energy, 16 lepton energy,
// 17 photon energy, 20 photon count (integer bits).
__global__ void __launch_bounds__(1024) k_reduce(View v, int gap) {
  const GapDev &g = v.gaps[gap];
  const int64_t nx = g.nx;
  const double *M = v.dmom;
  const double *E = v.E[v.ctl->e_cur] + g.node_off;
  __shared__ double sv[1024];
  __shared__ long long si[1024];
  double best = -1.0, sum = 0.0;
  long long bi = 0;
  long long ncell = 0;
  for (int64_t c = threadIdx.x; c < nx; c += blockDim.x) {
    if (!((double)c + 0.5 < g.Hc)) continue;
    const double m = M[c] + M[nx + c] + M[2 * nx + c] + M[3 * nx + c];
    sum += m;
    ++ncell;
    if (m > best) {
      best = m;
      bi = c;
    }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      const double b2 = sv[threadIdx.x + o];
      const long long i2 = si[threadIdx.x + o];
      if (b2 > sv[threadIdx.x] || (b2 == sv[threadIdx.x] && i2 < si[threadIdx.x])) {
        sv[threadIdx.x] = b2;
        si[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  const double Mpk = sv[0];
  const long long ipk = si[0];
  __syncthreads();
  // sums
  double tot = 0.0;
  (void)block_exclusive_scan(sum, &tot);
  double tcell = 0.0;
  (void)block_exclusive_scan((double)ncell, &tcell);
  // E extrema over gap nodes, |E| max and field energy over all nodes
  double emin = 1e300, emax = -1e300, eabs = 0.0, fe = 0.0;
  for (int64_t i = threadIdx.x; i < g.nnode; i += blockDim.x) {
    const double e = E[i];
    if ((double)i <= g.Hc) {
      emin = fmin(emin, e);
      emax = fmax(emax, e);
    }
    eabs = fmax(eabs, fabs(e));
    fe += 0.5 * g.dx * e * e;
  }
  // Gauss residual over cells touching no boundary; with a current filter,
  // against the smoothed charge and P cells further from each end
  const int P = g.filter_passes;
  const double *Qs = nullptr;
  if (P > 0) {
    double *A = v.Dflt, *B = v.Dflt + v.dcharge_len;
    for (int64_t c = threadIdx.x; c < nx; c += blockDim.x)
      A[c] = charge_value(v, g, v.dcharge[c]) - g.eta_bg * g.dx;
    Qs = filter_cells_block(A, B, nx, P, g.periodic != 0);
  }
  double gr = 0.0;
  int64_t clo = g.periodic ? 0 : 1 + P, chi = g.periodic ? nx - 1 : nx - 2 - P;
  // transverse fields: the virtual charge -beta_y dB_z + beta_z dB_y joins
  // eta_co; the absorbing layer's damping of B breaks that balance inside it
  if (g.em && !g.periodic && g.pml_cells > 0 && chi > nx - g.pml_cells - 1) chi = nx - g.pml_cells - 1;
  const double *By = v.em_By + g.node_off, *Bz = v.em_Bz + g.node_off;
  for (int64_t c = clo + threadIdx.x; c <= chi; c += blockDim.x) {
    const int64_t c1 = g.periodic ? (c + 1) % nx : c + 1;
    const double q = Qs ? Qs[c] : charge_value(v, g, v.dcharge[c]) - g.eta_bg * g.dx;
    double r = (E[c1] - E[c]) - q;
    if (g.em) r -= g.beta_y * (Bz[c1] - Bz[c]) - g.beta_z * (By[c1] - By[c]);
    gr = fmax(gr, fabs(r));
  }
  sv[threadIdx.x] = emin;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sv[threadIdx.x] = fmin(sv[threadIdx.x], sv[threadIdx.x + o]);
    __syncthreads();
  }
  const double Emin = sv[0];
  __syncthreads();
  sv[threadIdx.x] = emax;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sv[threadIdx.x] = fmax(sv[threadIdx.x], sv[threadIdx.x + o]);
    __syncthreads();
  }
  const double Emax = sv[0];
  __syncthreads();
  sv[threadIdx.x] = eabs;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sv[threadIdx.x] = fmax(sv[threadIdx.x], sv[threadIdx.x + o]);
    __syncthreads();
  }
  const double Eabs = sv[0];
  __syncthreads();
  sv[threadIdx.x] = gr;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sv[threadIdx.x] = fmax(sv[threadIdx.x], sv[threadIdx.x + o]);
    __syncthreads();
  }
  const double Gr = sv[0];
  __syncthreads();
  double fet = 0.0;
  (void)block_exclusive_scan(fe, &fet);
  if (threadIdx.x == 0) {
    double *o = v.dred;
    o[0] = Mpk < 0 ? 0.0 : Mpk;
    o[1] = tcell > 0 ? tot / tcell : 0.0;
    o[2] = (double)ipk;
    const double ws = M[5 * nx + ipk];
    o[3] = ws > 0 ? M[4 * nx + ipk] / ws : 0.0;
    for (int q = 0; q < 4; ++q) o[4 + q] = M[q * nx + ipk];
    o[8] = Emin;
    o[9] = Emax;
    o[10] = Gr;
    o[11] = Eabs;
    o[12] = fet;
  }
}

// Radix-2 Stockham FFT stage (self-sorting, out of place): with n the current
// sub-transform length and s the stride, for p < n/2, q < s:
//   a = x[q + s p], b = x[q + s (p + n/2)], w = exp(-2 pi i p / n),
//   y[q + s 2p] = a + b, y[q + s (2p + 1)] = (a - b) w.
__global__ void k_fft_stage(const double2 *x, double2 *y, int64_t n, int64_t s, int64_t P) {
  const int64_t half = P / 2;
  const int64_t m = n / 2;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < half;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = idx / s, q = idx % s;
    const double2 a = x[q + s * p];
    const double2 b = x[q + s * (p + m)];
    double sn, cs;
    sincospi(-2.0 * (double)p / (double)n, &sn, &cs);
    const double2 d = make_double2(a.x - b.x, a.y - b.y);
    y[q + s * (2 * p)] = make_double2(a.x + b.x, a.y + b.y);
    y[q + s * (2 * p + 1)] = make_double2(d.x * cs - d.y * sn, d.x * sn + d.y * cs);
  }
}

__global__ void k_fft_fill(View v, int gap, double2 *buf, int64_t P) {
  const GapDev &g = v.gaps[gap];
  const double *E = v.E[v.ctl->e_cur] + g.node_off;
  int64_t ng = (int64_t)floor(g.Hc) + 1;
  if (ng > g.nnode) ng = g.nnode;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P;
       i += (int64_t)gridDim.x * blockDim.x)
    buf[i] = make_double2(i < ng ? E[i] : 0.0, 0.0);
}

__global__ void k_fft_power(const double2 *X, double *out, int64_t P) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= P / 2;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (X[i].x * X[i].x + X[i].y * X[i].y) / (double)P;
}

void launch_diag(const View &v, int gap, int64_t nx, int64_t P, cudaStream_t st) {
  cudaMemsetAsync(v.dmom, 0, sizeof(double) * 8 * (size_t)nx, st);
  cudaMemsetAsync(v.dcharge, 0, sizeof(unsigned long long) * (size_t)nx, st);
  cudaMemsetAsync(v.dred, 0, sizeof(double) * 32, st);
  GapDev gh;
  cudaMemcpyAsync(&gh, &v.gaps[gap], sizeof(GapDev), cudaMemcpyDeviceToHost, st);
  cudaStreamSynchronize(st);
  // a tile's cells summed in shared memory while they fit without opting
  // into more than 48 KB (7 sums of 8 bytes per cell)
  const size_t msm = (size_t)(v.tile + 4) * 7 * sizeof(double);
  const int priv = msm <= 48 * 1024 ? 1 : 0;
  if (v.precision == GAP_FP32_STATE) k_moments<float><<<gh.n_tiles, 256, priv ? msm : 0, st>>>(v, gap, priv);
  else k_moments<double><<<gh.n_tiles, 256, priv ? msm : 0, st>>>(v, gap, priv);
  launch_photon_moments(v, gap, st);
  if (v.pr_any) k_proton_charge<<<148 * 4, 256, 0, st>>>(v, gap, v.dcharge);  // for the Gauss residual
  k_reduce<<<1, 1024, 0, st>>>(v, gap);
  if (P >= 2) {
    double2 *a = reinterpret_cast<double2 *>(v.fft[0]);
    double2 *b = reinterpret_cast<double2 *>(v.fft[1]);
    const int blocks = (int)((P / 2 + 255) / 256 < 1184 ? (P / 2 + 255) / 256 : 1184);
    k_fft_fill<<<blocks, 256, 0, st>>>(v, gap, a, P);
    int64_t s = 1;
    for (int64_t n = P; n > 1; n /= 2) {
      k_fft_stage<<<blocks, 256, 0, st>>>(a, b, n, s, P);
      double2 *tmp = a;
      a = b;
      b = tmp;
      s *= 2;
    }
    // result in `a`; power spectrum into the other buffer (real part reused)
    k_fft_power<<<blocks, 256, 0, st>>>(a, reinterpret_cast<double *>(b), P);
    if (b != reinterpret_cast<double2 *>(v.fft[1])) {
      cudaMemcpyAsync(v.fft[1], b, sizeof(double) * (size_t)(P / 2 + 1), cudaMemcpyDeviceToDevice, st);
    }
  }
}

// ---------------------------------------------------------------------------
// Export / import through a staging area (the inactive particle buffers).
// Lepton stage: id | X | u | w | tau, each an array of `cap` doubles.
// Photon stage: id | X | x | w | tau_acc | tau_star | aux2.
template <class R>
__global__ void k_export_leptons(View v, int gap, int s, double *stage, int64_t cap,
                                 unsigned long long *count, int64_t stride, int tile_first) {
  using W = typename Prec<R>::W;
  const GapDev &g = v.gaps[gap];
  const int t = g.tile_begin + tile_first + blockIdx.x;
  const int cur = v.ctl->lep_cur;
  const int64_t start = v.seg_start[s][t];
  const int used = v.seg_used[s][t];
  for (int i = threadIdx.x; i < used; i += blockDim.x) {
    const int64_t slot = start + i;
    const int32_t k = v.lk[cur][s][slot];
    if (k < 0) continue;
    if (stride > 1 && v.lid[cur][s][slot] % (uint64_t)stride != 0) continue;  // a sample by id
    const unsigned long long o = atomicAdd(count, 1ull);
    if ((int64_t)o >= cap) continue;
    const R phi = as<R>(v.lphi[cur][s])[slot];
    reinterpret_cast<uint64_t *>(stage)[o] = v.lid[cur][s][slot];
    stage[cap + o] = (double)k + ((double)phi - 1.5);
    stage[2 * cap + o] = (double)as<R>(v.lu[cur][s])[slot];
    // without QED or variable weights every lepton carries w0 and no optical depth
    const bool full_state = v.qed_any || v.has_w;
    const W wq = as<W>(v.lw[cur][s])[slot];
    stage[3 * cap + o] = !full_state ? g.w0 : (sizeof(R) == 4 ? (double)wq * g.w_unit : (double)wq);
    stage[4 * cap + o] = full_state ? (double)as<R>(v.ltau[cur][s])[slot] : 0.0;
  }
}

template <class R>
__global__ void k_import_leptons(View v, int gap, int s, int64_t n, const double *stage) {
  using W = typename Prec<R>::W;
  const GapDev &g = v.gaps[gap];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint64_t id = reinterpret_cast<const uint64_t *>(stage)[i];
    const double X = stage[n + i];
    const double u = stage[2 * n + i];
    const double w = stage[3 * n + i];
    const double tau = stage[4 * n + i];
    int32_t k;
    R phi;
    split_position<R>(X, g.nx, g.periodic != 0, k, phi);
    W wq;
    if (sizeof(R) == 4) wq = (W)llrint(w / g.w_unit);
    else wq = (W)w;
    append_lepton<R>(v, s, tile_of(v, g, k), k, phi, (R)u, wq, (R)tau, id);
  }
}

// Inverse CDF of the classical curvature spectrum as the emission kernels
// evaluate it (FP64: table + Newton on the quadrature; FP32: table).
__global__ void k_spec_inverse(View v, const double *U, double *xi, int64_t n, int fp32) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    xi[i] = fp32 ? (double)spec_inverse_f(v, (float)U[i]) : spec_inverse_d(v, U[i]);
}

__global__ void k_qspec_inverse(View v, const double *chi, const double *U, double *xi, int64_t n, int fp32) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    xi[i] = fp32 ? (double)qspec_inverse<float>(v, (float)chi[i], (float)U[i]) : qspec_inverse<double>(v, chi[i], U[i]);
}

void launch_qspec_inverse(const View &v, const double *chi, const double *U, double *xi, int64_t n, int fp32,
                          cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 148 * 8);
  if (n > 0) k_qspec_inverse<<<blocks, 256, 0, st>>>(v, chi, U, xi, n, fp32);
}

__global__ void k_pair_split(View v, const double *chi, const double *U, double *e, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    e[i] = bw_split(v, chi[i], U[i], true);
}

void launch_pair_split(const View &v, const double *chi, const double *U, double *e, int64_t n, cudaStream_t st) {
  const int blocks = (int)std::min<int64_t>((n + 255) / 256, 148 * 8);
  if (n > 0) k_pair_split<<<blocks, 256, 0, st>>>(v, chi, U, e, n);
}

void launch_spec_inverse(const View &v, const double *U, double *xi, int64_t n, int fp32, cudaStream_t st) {
  int blocks = (int)((n + 255) / 256);
  if (blocks > 1184) blocks = 1184;
  if (n > 0) k_spec_inverse<<<blocks, 256, 0, st>>>(v, U, xi, n, fp32);
}

void launch_import(const View &v, int gap, int kind, int64_t n, const double *stage, cudaStream_t st) {
  if (n <= 0) return;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 1184) blocks = 1184;
  if (kind == GAP_PHOTON) {
    launch_import_photons(v, gap, n, stage, st);
  } else if (v.precision == GAP_FP32_STATE) {
    k_import_leptons<float><<<blocks, 256, 0, st>>>(v, gap, kind, n, stage);
  } else {
    k_import_leptons<double><<<blocks, 256, 0, st>>>(v, gap, kind, n, stage);
  }
}

void launch_export_impl(const View &v, int gap, int kind, double *stage, int64_t cap,
                        unsigned long long *count, int n_tiles_gap, cudaStream_t st, int64_t stride,
                        int tile_first) {
  if (kind == GAP_PHOTON) {
    launch_export_photons(v, gap, stage, cap, count, st);
  } else if (v.precision == GAP_FP32_STATE) {
    k_export_leptons<float><<<n_tiles_gap, 256, 0, st>>>(v, gap, kind, stage, cap, count, stride, tile_first);
  } else {
    k_export_leptons<double><<<n_tiles_gap, 256, 0, st>>>(v, gap, kind, stage, cap, count, stride, tile_first);
  }
}

// ---------------------------------------------------------------------------
// Spectra of one gap (Sect. 6.4, Fig. 6): the weight of the e- and e+ in the
// gap (X < H_gap) per bin of ln p, p = |u| = gamma beta, and of its photons
// per bin of ln x, nbins uniform bins over [lo, hi) clamped at both ends, into
// v.spec_buf [e- | e+ | photons], kSpecMaxBins each (cleared by the caller).
__device__ __forceinline__ int spectrum_bin(double z, int nbins, double lo, double hi) {
  double b = floor((z - lo) / (hi - lo) * (double)nbins);
  if (!(b >= 0.0)) b = 0.0;
  if (b > (double)(nbins - 1)) b = (double)(nbins - 1);
  return (int)b;
}

template <class R>
__global__ void k_spectra_leptons(View v, int gap, int nbins, double lo, double hi) {
  using W = typename Prec<R>::W;
  extern __shared__ double sh[];  // [2][nbins]
  for (int i = threadIdx.x; i < 2 * nbins; i += blockDim.x) sh[i] = 0.0;
  __syncthreads();
  const GapDev &g = v.gaps[gap];
  const int t = g.tile_begin + blockIdx.x;
  const int cur = v.ctl->lep_cur;
  for (int s = 0; s < 2; ++s) {
    const int64_t start = v.seg_start[s][t];
    const int used = v.seg_used[s][t];
    for (int i = threadIdx.x; i < used; i += blockDim.x) {
      const int64_t slot = start + i;
      const int32_t k = v.lk[cur][s][slot];
      if (k < 0) continue;
      const double X = (double)k + ((double)as<R>(v.lphi[cur][s])[slot] - 1.5);
      if (!(X < g.Hc)) continue;
      const double u = (double)as<R>(v.lu[cur][s])[slot];
      const double w = v.has_w ? (sizeof(R) == 4 ? (double)as<W>(v.lw[cur][s])[slot] * g.w_unit
                                                 : (double)as<W>(v.lw[cur][s])[slot])
                               : g.w0;
      atomicAdd(&sh[s * nbins + spectrum_bin(log(fabs(u)), nbins, lo, hi)], w);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * nbins; i += blockDim.x)  // species s at spec_buf[s kSpecMaxBins + bin]
    if (sh[i] != 0.0) atomicAdd(&v.spec_buf[(i / nbins) * kSpecMaxBins + i % nbins], sh[i]);
}

__global__ void k_spectra_photons(View v, int gap, int nbins, double lo, double hi) {
  const int b = v.ctl->ph_cur;
  const int64_t n = photon_fill(v, b);
  const int64_t step = v.ctl->step;
  const GapDev &g = v.gaps[gap];
  double *out = v.spec_buf + 2 * kSpecMaxBins;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (v.pev[b][i] == kPhDead || v.pgap[b][i] != gap) continue;
    const double X = photon_pos(g, v.pXr[b][i], v.pnr[b][i], v.pdir[b][i], step);
    if (!(X < g.Hc)) continue;
    atomicAdd(&out[spectrum_bin(log(v.px[b][i]), nbins, lo, hi)], v.pw[b][i]);
  }
}

void launch_spectra(const View &v, int gap, int n_tiles_gap, int nbins, double lo, double hi, cudaStream_t st) {
  const size_t smem = 2 * (size_t)nbins * sizeof(double);
  static bool attr = false;
  if (!attr) {  // up to 2 x 1024 doubles of shared memory
    cudaFuncSetAttribute(k_spectra_leptons<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * kSpecMaxBins * 8);
    cudaFuncSetAttribute(k_spectra_leptons<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * kSpecMaxBins * 8);
    attr = true;
  }
  if (v.precision == GAP_FP32_STATE) k_spectra_leptons<float><<<n_tiles_gap, 256, smem, st>>>(v, gap, nbins, lo, hi);
  else k_spectra_leptons<double><<<n_tiles_gap, 256, smem, st>>>(v, gap, nbins, lo, hi);
  if (v.qed_any) k_spectra_photons<<<148, 256, 0, st>>>(v, gap, nbins, lo, hi);
}

// E of one gap (the buffer of the current step) into the staging buffer of
// gap_get_field_async: the host does not read the control block to choose it.
__global__ void k_copy_field(View v, int gap) {
  const GapDev &g = v.gaps[gap];
  const double *E = v.E[v.ctl->e_cur] + g.node_off;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < g.nnode; i += (int64_t)gridDim.x * blockDim.x)
    v.fstage[i] = E[i];
}

void launch_copy_field(const View &v, int gap, cudaStream_t st) { k_copy_field<<<2 * 148, 256, 0, st>>>(v, gap); }

}  // namespace gapk
