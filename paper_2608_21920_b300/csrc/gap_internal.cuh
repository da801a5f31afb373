// gap_internal.cuh -- device-side data layout and helpers of the B300 PIC library.
//
// Particle positions are node-centred: a lepton is a dual-cell index k (the
// grid node nearest to it) plus an offset phi' in [1, 2), so that its
// first-order cloud [X - 1/2, X + 1/2] (X = k + phi' - 3/2 in cell units)
// covers node k and the fraction right of node k is phi = phi' - 1.  Storing
// the offset biased into [1, 2) puts every representable value on a uniform
// grid (2^-23 in FP32, 2^-52 in FP64), so the charge flux through a node,
// a difference of two such offsets, is exact; in FP32 it is accumulated as an
// integer number of 2^-23 units and the deposit conserves charge exactly.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/gap.h"
#include "qed_exact.cuh"

namespace gapk {

constexpr double kAlphaEm = 7.2973525693e-3;  // fine-structure constant
constexpr uint64_t kPhotonBit = 0x8000000000000000ull;
constexpr int kPhiBits = 23;                   // FP32 offset grid 2^-23
constexpr double kPhiUnit = 1.0 / 8388608.0;   // 2^-23
constexpr int kWeightShift = 8;                // FP32 weight unit = w0 / 2^8

// Protons with the FP32 state keep FP64 positions on the leptons' offset
// grid: X + 1/2 a multiple of 2^-23 (exact in double up to 2^29 cells), so
// that every cloud fraction and flux of a proton is a whole number of the
// state's charge units (grid_units times 2^kWeightShift for weight w0).
__device__ __forceinline__ double grid_position(double X) { return rint((X + 0.5) * 8388608.0) * kPhiUnit - 0.5; }
__device__ __forceinline__ long long grid_units(double f) { return llrint(f * 8388608.0); }
constexpr int kMaxEmit = 16;                   // emission events per lepton-step (upper bound)
// Return-flux tally (Sect. 6.5): eight bins per decade of gamma from gamma = 1
constexpr int kRetBins = 64;
constexpr double kRetDln = 0.28782313662425574;  // ln 10 / 8
constexpr int kSpecMaxBins = 1024;              // gap_spectra: bins per histogram at most
// Leptons per push work item: a power of two from kPushChunkMin to kPushChunk,
// chosen each step so that a large store is cut into at least ~2048 items
// (long items cost less at their ends; enough of them keep every SM busy).
constexpr int kPushChunk = 32768;  // the largest (multiple of 32; the limb bound below)
constexpr int kPushChunkMin = 8192;
constexpr int kPushGrid = 148 * 4;  // blocks of the persistent push grid (4 per SM)
static_assert(kPushChunk <= 32768, "the 17-bit charge limbs hold at most 32768 contributions per node");

// Quantum photon spectrum table: rows of ln chi from ln 1e-6 in steps of
// ln 10 / 8 (89 rows to chi = 1e5); nodes s_k = 4 (k/256)^2, k < kQsNodes
// (s <= 4, d <= 64: the survival there is below e^-60), crowded towards
// s = 0, where the spectrum of a large chi lies (s ~ (2/(3 chi))^(1/3)).
constexpr int kQsNodes = 257;
constexpr int kQsRows = 89;
constexpr double kQsLchi0 = -13.815510557964274;  // ln 1e-6
constexpr double kQsDlchi = 0.28782313662425574;  // ln 10 / 8
template <class R = double>
__host__ __device__ __forceinline__ R qs_node(int k) {  // in the precision of the caller
  const R f = (R)k / (R)(kQsNodes - 1);
  return (R)4 * f * f;
}
// Pair energy split table (qed_quantum): rows of ln chi from ln 1e-3 in steps
// of ln 10 / 8 (57 rows to chi = 1e4); nodes eta_k = |e - 1/2| on a quintic
// smootherstep of [0, 1/2] (cubic crowding towards both ends: the narrow
// peak of a small chi at e = 1/2, the structure near e ~ 1/chi of a large one).
constexpr int kBwRows = 57;
constexpr double kBwLchi0 = -6.907755278982137;  // ln 1e-3
template <class R = double>
__host__ __device__ __forceinline__ R bw_node(int k) {
  const R f = (R)k / (R)(kQsNodes - 1);
  return (R)0.5 * f * f * f * (f * ((R)6 * f - (R)15) + (R)10);
}
// The same nodes as the smaller share 1/2 - eta_k, without cancellation.
template <class R = double>
__host__ __device__ __forceinline__ R bw_node_small(int k) {
  const R g = (R)(kQsNodes - 1 - k) / (R)(kQsNodes - 1);
  return (R)0.5 * g * g * g * (g * ((R)6 * g - (R)15) + (R)10);
}

// Draw channels of the counter-based generator (interface values).
enum Channel : uint32_t {
  CH_INIT_U = 1, CH_TAU0 = 3, CH_EMIT_X = 4, CH_EMIT_TAU = 5,
  CH_BW_TAU = 6, CH_INJECT = 7, CH_PAIR = 8, CH_PHOTON = 9, CH_INJECT_U = 12, CH_PAIR_E = 13,
  CH_INJECT_P = 14
};

enum Counter {
  C_EMIT = 0, C_PHOTONS, C_PAIRS, C_INJECTED, C_ABSORBED, C_ESCAPED, C_PH_ESCAPED,
  C_EMIT_OVF, C_INJ_OVF, C_LOAD_OVF, C_SPILL, C_PH_OVF, C_MERGED, C_PH_MERGED, C_R1, C_R2, C_NCNT
};
enum Ledger { L_RAD = 0, L_ABS, L_ESC, L_PH_ESC, L_INJ, L_WORK, L_R3, L_R4, L_NLED };

struct GapDev {
  int64_t nx, nnode, node_off;
  int32_t periodic, qed, kmax_emit, kmax_inject;
  int32_t tile_begin, n_tiles, gap_index, pad;
  double dx, dt, cdx, jm, Hc, lambda_hat, rho_hat, rate_mult, b, eta_bg, w0, w_unit;
  float f_dt, f_cdx, f_Hc, f_lam, f_rho, f_rate;
  float f_b, f_pad;  // (float)b: FP64 -> FP32 conversions run on the FP64 units
  double inv_cdx;     // 1 / cdx
  uint64_t seed, inj_root;
  int64_t cap;  // macro-particle cap (leptons + photons); 0 = none
  double inject_theta;  // temperature of the injected atmosphere (m_e c^2); 0 = cold
  int32_t filter_passes;  // binomial current-smoothing passes per step; 0 = none
  int32_t qed_quantum;    // 1: quantum photon spectrum (table below); 0: classical
  int32_t protons;        // 1: a proton store and proton supply (FP64 state)
  int32_t defer;          // Ampere left to filter.cu (a current filter, or protons)
  double m_ion;           // proton mass in m_e
  int32_t em;             // 1: transverse fields of the co-rotating frame (em.cu)
  int32_t pml_cells;      // absorbing layer below the top of a surface gap; 0 = none
  double beta_y, beta_z;  // velocity of the co-rotating frame across h
  double pml_smax;        // peak conductivity of the layer (omega_p)
  int32_t jperp;          // 1: the particles' transverse current (guiding centres)
  int32_t ampere_late;    // Ampere after the push kernels (filter.cu): defer, or the two-pass QED push
  double bstar_inv;       // 1 / B_* = lambda_hat / b (code units)
};

struct TileDev {
  int32_t gap, k0, nk, pad;
};

// Device control block (all mutable scalars of a handle live here so that a
// captured CUDA graph replays correctly).
struct Ctl {
  int64_t step;
  int32_t lep_cur, ph_cur, e_cur, need_rebin;
  int32_t error, flags;
  int64_t ph_count[2];
  int64_t ph_work_n;  // photons on the scheduling work list this step
  int64_t last_rebin_step;
  int64_t ph_dead;  // photons dead since the last photon compaction
  int64_t pr_count;  // protons stored (alive or not)
  int32_t need_ph_compact;
  int32_t hold_copies;  // test hook: bulk-copy pushes leave their first stage unissued
  int32_t push_items, push_next;  // the push work list of this step and its counter
  int32_t push_chunk, push_pad;   // leptons per item this step (kPushChunkMin .. kPushChunk)
  unsigned long long defer_n;     // movers on the deferred list this step (may exceed its half)
  unsigned long long defer_ne;    // emitters on the deferred list this step (may exceed its half)
  int32_t defer_over, defer_pad;  // some deferred lepton did not fit on the list this step
  int64_t spill_n[2];
  int64_t new_total[2];
  int64_t ph_nb_start;  // photon store fill before this step's push (0 after a photon compaction)
  int64_t phm_end;      // photon store fill when the photon merge began
  int32_t mlist_n, mlist_pad;  // (species, tile) segments of merging gaps listed this step
};

// Everything a kernel needs, passed by value.
struct View {
  GapDev *gaps;
  TileDev *tiles;
  int32_t n_gaps, n_tiles, tile, precision;
  int32_t qed_any, surface_any, has_w, rebin_every;
  int32_t variant, merge_any;
  int32_t filter_any, pr_any;  // some gap's Ampere runs in k_filter_apply; some gap has protons
  int32_t defer_any, defer_pad;  // some gap defers Ampere for a filter, protons or transverse fields
  int64_t pr_cap;             // proton store (unsorted, FP64): position, momentum per m_ion c, weight
  double *pr_X, *pr_u, *pr_w;
  uint64_t *pr_id;
  int32_t *pr_gap, *pr_alive;
  // transverse fields (some gap with em), indexed like the nodes (node_off):
  // E_y, E_z on cells c < nx, B_y, B_z on nodes; Jv = dt jv_h of this step
  int32_t em_any, jperp_any;
  double *em_Ey, *em_Ez, *em_By, *em_Bz, *em_Jv;
  double *em_jy, *em_jz;      // jperp: the particles' transverse current of the step (cells)
  double *Dflt;               // [2 x dcharge_len] smoothing scratch (node flux; two cell buffers)
  // quantum photon spectrum (some gap with qed_quantum): per row of ln chi,
  // the normalised survival S(s)/S(0) and its s-derivative on kQsNodes nodes
  // of s = d^(1/3), d = 2 xi / (3 chi (1 - xi)); FP64 and FP32 copies
  int32_t qs_any, qs_rows;
  double2 *qs_tab_d;
  float2 *qs_tab_f;
  float2 *bw_tab;  // pair energy split: per row of ln chi, (G, dG/d(1/2 - eta)) on kQsNodes nodes
  int32_t *merge_state;  // [gap][4]: merge flag, level
  double *merge_width;   // [gap]
  // the merge's segments: [2 n_tiles] list of s n_tiles + t, output cursors;
  // [2 n_tiles][tile + 4] end of each node's run after the sort by node
  int32_t *mlist, *mout, *mrun;
  // photon merge at birth: open-addressing table of phm_size (a power of
  // two) keys with the sums of each group; zero between merges
  int64_t phm_size;
  unsigned long long *phm_key, *phm_nid;  // key (0 = empty); max of ~id over the group
  double *phm_W, *phm_Wx, *phm_WX;        // sum w, sum w x, sum w X
  unsigned *phm_cnt;
  int32_t *ph_gap;       // photons alive per gap
  Ctl *ctl;
  double *E[2];
  unsigned long long *Dg;  // int64 (FP32) or double (FP64) bit patterns
  int32_t *arrive;
  int8_t *expect;
  // segments [species][tile]
  int64_t *seg_start[2];
  int32_t *seg_cap[2], *seg_used[2], *seg_append[2], *seg_alive[2], *spill_cnt[2];
  int64_t *new_start[2];
  int32_t *new_cap[2], *new_fill[2];
  int32_t *last_cnt[2];  // per tile: alive count after the last re-bin
  int32_t *gross[2];     // per tile: appends since the last re-bin
  int32_t *item_start;   // [n_tiles + 1] first push item of each tile
  int32_t *item_tile;    // [item_cap] tile of each push item
  // leptons the FP32 QED push defers to k_push_deferred (emitters, and
  // leptons that moved into another tile): store slot, and tile | species
  // << 30 | mover << 31
  int64_t *defer_slot;
  uint32_t *defer_ts;
  int64_t defer_cap;
  int64_t defer_use;     // its usable length: defer_cap (smaller in a test of the overflow)
  int32_t item_cap;      // bound on the push items of a step
  int32_t *tile_done;    // [n_tiles] items of the tile finished this step
  // lepton stores [buffer][species]
  int32_t *lk[2][2];
  void *lphi[2][2], *lu[2][2], *lw[2][2], *ltau[2][2];
  uint64_t *lid[2][2];
  int64_t lep_capacity;
  // spill buffers [species]
  int32_t *sk[2], *stile[2];
  double *sphi[2], *su[2], *sw[2], *stau[2];
  uint64_t *sid[2];
  int64_t spill_capacity;
  // photon stores [buffer]: the current buffer is append-only between
  // compactions.  A photon moves from X_ref (its position at the start of
  // step n_ref); its optical depth tau_acc holds the steps before pm; pev is
  // the step of its next event (conversion, escape or re-schedule: pkind),
  // kPhPending before it is scheduled, kPhDead after its event.
  double *pXr[2], *px[2], *pw[2], *pts[2], *pta[2];
  uint64_t *pid[2];
  int32_t *pn0[2], *pnr[2], *pdir[2], *pgap[2], *pm[2], *pev[2], *pkind[2];
  int32_t *pmn[2];   // checkpoint a pending re-schedule starts from (step, tau
  double *ptan[2];   // before it), adopted when the re-schedule is taken
  int64_t *ph_work;  // photon indices to schedule this step
  int64_t ph_capacity;
  // per-gap accumulators
  unsigned long long *counters;  // [gap][C_NCNT]
  double *ledger;                // [gap][L_NLED]
  unsigned long long *q0;        // [gap] cell-0 charge (int64 or double bits)
  // emission-spectrum tables (built by the library at init)
  float2 *spec_tab;  // (ln xi, d ln xi / d ln v) on a uniform grid of z = ln v, v = -ln U
  int32_t spec_n;
  float spec_z0, spec_dz;
  double *quad_c, *quad_a;  // cosh t_k and cosh(5 t_k/3)/cosh t_k (trapezoid nodes)
  int32_t quad_n;
  double quad_h;
  // diagnostics scratch
  double *fstage;         // [max_nx] staging of gap_get_field_async
  double *dmom;                 // [8][max_nx]
  unsigned long long *dcharge;  // [max_nx] exact charge (int64 or double bits)
  double *fft[2];               // complex scratch [2][2*max_P]
  int64_t max_nx, max_P, dcharge_len;
  double *dred;                 // reduction outputs
  double *ret_hist;             // [gap][kRetBins] return flux: weight of e+- absorbed at h < 0 per ln gamma bin
  double *spec_buf;             // [3][kSpecMaxBins] scratch of gap_spectra
  // export / import staging (the inactive buffers are used as scratch)
};

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), device implementation.
__device__ __forceinline__ void philox10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t lo0 = 0xD2511F53u * c[0];
    uint32_t hi0 = __umulhi(0xD2511F53u, c[0]);
    uint32_t lo1 = 0xCD9E8D57u * c[2];
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]);
    uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
}

// Uniform in (0, 1] keyed by (seed; id, step, channel, k): 53 bits from the
// first two output words.
__device__ __forceinline__ double uniform53(uint64_t seed, uint64_t id, uint32_t step,
                                            uint32_t channel, uint32_t k) {
  uint32_t c[4] = {(uint32_t)id, (uint32_t)(id >> 32), step, (channel << 16) | (k & 0xFFFFu)};
  philox10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  uint64_t m = ((uint64_t)(c[0] >> 5) << 26) | (uint64_t)(c[1] >> 6);
  return ((double)m + 1.0) * 1.1102230246251565e-16;  // 2^-53
}

// 24-bit uniform in (0, 1) from the same counter (the FP32 state's draws).
__device__ __forceinline__ float uniform24(uint64_t seed, uint64_t id, uint32_t step, uint32_t channel,
                                           uint32_t k) {
  uint32_t c[4] = {(uint32_t)id, (uint32_t)(id >> 32), step, (channel << 16) | (k & 0xFFFFu)};
  philox10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
  return ((float)(c[0] >> 8) + 0.5f) * 5.9604644775390625e-8f;  // 2^-24
}

// SplitMix64 output function (Steele, Lea, Flood 2014).
// 1D Maxwell-Juttner deviate, f(u) ~ exp(-(gamma - 1)/theta), by the
// ratio-of-uniforms method (Kinderman & Monahan 1977): (a, v) uniform on
// (0,1] x [-bmax, bmax] with bmax = sup |u| sqrt(f(u)) (at u^2 = 2 theta
// gamma, gamma = theta + sqrt(theta^2 + 1)); u = v/a is accepted when
// 2 ln a <= -(gamma - 1)/theta.  Round r draws k = 2r, 2r+1 of (id, step,
// channel); after 64 rejected rounds ok is false and u = 0.
__device__ __forceinline__ double mj_bmax(double theta) {
  const double gs = theta + sqrt(theta * theta + 1.0);
  const double us = sqrt(2.0 * theta * gs);
  return us * exp(-(gs - 1.0) / (2.0 * theta));
}

// The draw with bmax given (a loader forms it once).  Each round's test
// 2 ln a <= -(gamma - 1)/theta is first evaluated in float (u = v/a,
// gamma - 1 = u^2/(sqrt(1 + u^2) + 1), logf): it decides only when its two
// sides differ by more than 4e-6 (|lhs| + |rhs|) + 1e-6, about four times
// their float rounding (a few ulp each, the ulp of logf and the rounding of
// a to float included), so every decision it takes is the FP64 one; it
// settles all but about 1e-5 of the rounds, and FP64 is left with the
// accepted round's u = v/a.  The rest go to the FP64 test: the bounds
// 1 - 1/a <= ln a <= a - 1, and ln a itself only where a bound lies within
// a relative 1e-12 of the threshold, so every decision is the one the
// logarithm gives.
__device__ __noinline__ static double mj_draw_b(uint64_t seed, uint64_t id, uint32_t step, uint32_t channel,
                                                double theta, double bmax, bool &ok) {
  const float inv_theta_f = 1.0f / (float)theta;
  for (uint32_t r = 0; r < 64; ++r) {
    const double a = uniform53(seed, id, step, channel, 2 * r);
    const double vv = bmax * (2.0 * uniform53(seed, id, step, channel, 2 * r + 1) - 1.0);
    {
      const float af = (float)a, uf = (float)vv / af;
      const float u2 = uf * uf;
      const float rf = -(u2 / (sqrtf(1.0f + u2) + 1.0f)) * inv_theta_f;
      const float lf = 2.0f * logf(af);
      const float m = 4e-6f * (fabsf(rf) + fabsf(lf)) + 1e-6f;
      if (lf <= rf - m) {
        ok = true;
        return vv / a;
      }
      if (lf > rf + m) continue;
    }
    const double u = vv / a;
    const double gm1 = u * u / (sqrt(1.0 + u * u) + 1.0);
    const double rhs = -gm1 / theta;
    const double up = 2.0 * (a - 1.0);  // >= 2 ln a
    bool accept;
    if (up <= rhs - 1e-12 * (fabs(rhs) + fabs(up))) {
      accept = true;
    } else if (up - rhs * a > 1e-12 * (fabs(rhs) * a + fabs(up))) {  // 2 (1 - 1/a) > rhs, times a > 0
      accept = false;
    } else {
      accept = 2.0 * log(a) <= rhs;
    }
    if (accept) {
      ok = true;
      return u;
    }
  }
  ok = false;
  return 0.0;
}

__device__ __forceinline__ double mj_draw(uint64_t seed, uint64_t id, uint32_t step, uint32_t channel,
                                          double theta, bool &ok) {
  return mj_draw_b(seed, id, step, channel, theta, mj_bmax(theta), ok);
}

__device__ __host__ __forceinline__ uint64_t mix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __host__ __forceinline__ uint64_t child_id(uint64_t parent, uint32_t step,
                                                      uint32_t channel, uint32_t k) {
  uint64_t salt = ((uint64_t)step << 32) | ((uint64_t)channel << 16) | (k & 0xFFFFu);
  return mix64(parent ^ mix64(salt));
}

// ---------------------------------------------------------------------------
// QED rate functions: Sect. 3.1 fit of T_syn and Sect. 3.2 fit of T_BW.
__device__ __forceinline__ double tsyn_d(double chi) {
  const double a0 = 1.4433756729740644;  // 5/(2 sqrt 3)
  const double a1 = 5.542562584220407;   // 16 sqrt3 / 5
  return a0 * pow(1.0 + a1 * chi + 1.1 * chi * chi, -1.0 / 6.0);
}
// (FP32: the fast base-2 logarithm, relative error ~2^-22, well inside the
// fit's own accuracy)
__device__ __forceinline__ float tsyn_f(float chi) {
  const float a0 = 1.4433757f, a1 = 5.5425626f;
  return a0 * exp2f(-__log2f(1.0f + a1 * chi + 1.1f * chi * chi) * (1.0f / 6.0f));
}
__device__ __forceinline__ double tbw_d(double chi) {
  if (!(chi > 0.0)) return 0.0;
  return 0.23 * exp(-8.0 / (3.0 * chi)) * pow(1.0 + 0.22 * chi, -1.0 / 3.0);
}

// ---------------------------------------------------------------------------
// Classical curvature spectrum: xi with S(xi) = U, S the survival function
//   S(xi) = 3/(5 pi) int_0^inf cosh(5t/3) exp(-xi cosh t)/cosh^2 t dt.
// Table: Hermite interpolation of y = ln xi in z = ln v, v = -ln U, on a
// uniform grid; linear extrapolation with the end slopes (the small-v end is
// the xi^(1/3) asymptote of the spectrum, slope 3).
template <class R>
__device__ __forceinline__ R spec_y_table(const View &v, R z) {
  R s = (z - (R)v.spec_z0) / (R)v.spec_dz;
  int n = v.spec_n;
  if (s <= (R)0) {
    float2 a = v.spec_tab[0];
    return (R)a.x + (R)a.y * (z - (R)v.spec_z0);
  }
  if (s >= (R)(n - 1)) {
    float2 a = v.spec_tab[n - 1];
    return (R)a.x + (R)a.y * (z - ((R)v.spec_z0 + (R)(n - 1) * (R)v.spec_dz));
  }
  int i = (int)s;
  R t = s - (R)i;
  float2 a = v.spec_tab[i], b = v.spec_tab[i + 1];
  R h = (R)v.spec_dz;
  R t2 = t * t, t3 = t2 * t;
  return ((R)2 * t3 - (R)3 * t2 + (R)1) * (R)a.x + (t3 - (R)2 * t2 + t) * h * (R)a.y +
         ((R)-2 * t3 + (R)3 * t2) * (R)b.x + (t3 - t2) * h * (R)b.y;
}

// FP32 path: table only.
__device__ __forceinline__ float spec_inverse_f(const View &v, float U) {
  if (!(U < 1.0f)) return 0.0f;
  float lv = -logf(U);
  return expf(spec_y_table<float>(v, logf(lv)));
}

// FP64 path: the table value refined by Newton steps in ln xi on the
// trapezoid quadrature of S and dS/dxi (nodes t_k = k h).  The sum stops once
// a term is below e^-40 of the first: xi (cosh t - 1) - t > 40, since the
// node weight cosh(5t/3)/cosh t is at most e^(2t/3).
__device__ __forceinline__ void spec_S_dS(const View &v, double xi, double &S, double &dS) {
  double s0 = 0.0, s1 = 0.0;
  for (int k = 0; k < v.quad_n; ++k) {
    double c = v.quad_c[k];
    if (xi * (c - 1.0) - k * v.quad_h > 40.0) break;
    double f = v.quad_a[k] * exp(-xi * c);
    double wk = k == 0 ? 0.5 : 1.0;
    s0 += wk * f / c;
    s1 += wk * f;
  }
  const double norm = 3.0 / (5.0 * 3.141592653589793) * v.quad_h;
  S = norm * s0;
  dS = -norm * s1;
}
__device__ __forceinline__ double spec_inverse_d(const View &v, double U) {
  if (U >= 1.0 - 1e-13) return 0.0;  // xi < 1e-36: no energy at double precision
  double lv = -log1p(U - 1.0);
  double y = spec_y_table<double>(v, log(lv));
  for (int it = 0; it < 12; ++it) {
    double xi = exp(y), S, dS;
    spec_S_dS(v, xi, S, dS);
    double step = (S - U) / (xi * dS);
    if (step > 1.0) step = 1.0;
    if (step < -1.0) step = -1.0;
    y -= step;
    if (fabs(step) < 1e-14) break;
  }
  return exp(y);
}

// Quantum photon spectrum: the photon energy fraction xi of an emission at
// chi for a draw U.  In each of four table rows the node with
// S_k >= U > S_{k+1} is found by bisection and the cubic Hermite
// interpolant of S(s) on that panel (nodes s_k = qs_node(k)) is solved by
// Newton steps; ln s is blended over four rows of ln chi
// (Catmull-Rom).  Below chi = 1e-6 the classical inverse gives d (the
// quantum correction is O(chi)); above 1e5 the last row is used.
// Inversion of a decreasing tabulated function G (G(node 0) = 1) for the
// target U in four rows at once: each bisection level issues four
// independent loads (the emissions of a discharge are frequent: a serial
// chain of dependent loads would dominate the push); then the cubic Hermite
// interpolant of the panel found is solved by Newton steps.  T2 holds
// (G, dG/dnode); Node gives the node positions.
template <class R, class T2, class Node>
__device__ void rows_invert(const T2 *tab, const int r[4], R U, R s[4]) {
  int lo[4], hi[4];
  bool live[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    lo[j] = 0;
    hi[j] = kQsNodes - 1;
    live[j] = U > (R)tab[r[j] * kQsNodes + kQsNodes - 1].x;
    if (!live[j]) s[j] = Node::template at<R>(kQsNodes - 1);
  }
  for (int level = 0; level < 8; ++level) {  // 2^8 panels
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (!live[j] || hi[j] - lo[j] <= 1) continue;
      const int mid = (lo[j] + hi[j]) >> 1;
      if ((R)tab[r[j] * kQsNodes + mid].x >= U) lo[j] = mid;
      else hi[j] = mid;
    }
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (!live[j]) continue;
    const T2 a = tab[r[j] * kQsNodes + lo[j]], b = tab[r[j] * kQsNodes + hi[j]];
    const R ax = (R)a.x, ay = (R)a.y, bx = (R)b.x, by = (R)b.y;
    const R s_lo = Node::template at<R>(lo[j]), h = Node::template at<R>(hi[j]) - s_lo;
    R t = (ax - U) / (ax - bx);  // linear start, in [0, 1]
    for (int it = 0; it < 4; ++it) {
      const R t2 = t * t, t3 = t2 * t;
      const R H = ((R)2 * t3 - (R)3 * t2 + (R)1) * ax + (t3 - (R)2 * t2 + t) * h * ay +
                  ((R)-2 * t3 + (R)3 * t2) * bx + (t3 - t2) * h * by;
      const R dH = ((R)6 * t2 - (R)6 * t) * ax + ((R)3 * t2 - (R)4 * t + (R)1) * h * ay +
                   ((R)-6 * t2 + (R)6 * t) * bx + ((R)3 * t2 - (R)2 * t) * h * by;
      if (!(dH < (R)0)) break;
      R tn = t - (H - U) / dH;
      tn = tn < (R)0 ? (R)0 : (tn > (R)1 ? (R)1 : tn);
      if (tn == t) break;
      t = tn;
    }
    s[j] = s_lo + t * h;
  }
}
struct QsNode {
  template <class R>
  __device__ static R at(int k) { return qs_node<R>(k); }
};
struct BwNodeSmall {
  template <class R>
  __device__ static R at(int k) { return bw_node_small<R>(k); }
};

// Catmull-Rom blend of four row values over ln chi (t in [0, 1] between the
// middle two)
template <class R>
__device__ __forceinline__ R catmull_rom(const R p[4], R t) {
  return (R)0.5 * ((R)2 * p[1] + (-p[0] + p[2]) * t + ((R)2 * p[0] - (R)5 * p[1] + (R)4 * p[2] - p[3]) * t * t +
                   (-p[0] + (R)3 * p[1] - (R)3 * p[2] + p[3]) * t * t * t);
}

template <class R>
__device__ __noinline__ R qspec_inverse(const View &v, R chi, R U) {
  if (!(U < (R)1)) return (R)0;
  R d;
  if (chi < (R)1e-6) {
    d = sizeof(R) == 4 ? (R)spec_inverse_f(v, (float)U) : (R)spec_inverse_d(v, (double)U);
  } else {
    R rr = (log(chi) - (R)kQsLchi0) / (R)kQsDlchi;
    if (rr > (R)(v.qs_rows - 1)) rr = (R)(v.qs_rows - 1);
    int i = (int)rr;
    if (i > v.qs_rows - 2) i = v.qs_rows - 2;
    const R t = rr - (R)i;
    int rows[4];
    R p[4];
    for (int j = 0; j < 4; ++j) {
      const int r = i - 1 + j;
      rows[j] = r < 0 ? 0 : (r > v.qs_rows - 1 ? v.qs_rows - 1 : r);
    }
    if (sizeof(R) == 4) rows_invert<R, float2, QsNode>(v.qs_tab_f, rows, U, p);
    else rows_invert<R, double2, QsNode>(v.qs_tab_d, rows, U, p);
    for (int j = 0; j < 4; ++j) p[j] = p[j] > (R)0 ? log(p[j]) : (R)-700;
    d = exp((R)3 * catmull_rom<R>(p, t));
  }
  const R w = (R)3 * chi * d;
  const R xi = w / ((R)2 + w);
  // FP64: Newton steps on the exact survival from the table's estimate
  if (sizeof(R) == 8) return (R)qs_refine((double)chi, (double)U, (double)xi);
  return xi;
}

// Pair energy split (qed_quantum): the electron's fraction e of the photon
// energy for a conversion at chi and a draw U (with `exact`, the FP64 state's
// case, refined on the exact distribution: qed_exact.cuh): the smaller share
// e_s = 1/2 - eta with G = 2 min(U, 1 - U), inverted in float in four rows
// of the table (the table's precision; float keeps the FP64 units free for
// the conversions of a discharge) and its logarithm blended over ln chi in
// double; e = e_s for U < 1/2, else 1 - e_s.  Below chi = 1e-3 the Gaussian
// limit (variance 3 chi / 64) applies; above 1e4 the last row.
__device__ __noinline__ static double bw_split(const View &v, double chi, double U, bool exact) {
  const double u = U < 0.5 ? U : 1.0 - U;
  double eta;
  if (!(chi > 0.0)) {
    eta = 0.0;
  } else if (chi < 1e-3) {
    eta = sqrt(3.0 * chi / 64.0) * 1.4142135623730951 * erfinv(1.0 - 2.0 * u);
    if (exact) {  // FP64: Newton steps on the exact distribution from the Gaussian estimate
      const double small = bw_refine(chi, u, 0.5 - eta);
      return U < 0.5 ? small : 1.0 - small;
    }
  } else {
    double rr = (log(chi) - kBwLchi0) / kQsDlchi;
    if (rr > (double)(kBwRows - 1)) rr = (double)(kBwRows - 1);
    int i = (int)rr;
    if (i > kBwRows - 2) i = kBwRows - 2;
    const double t = rr - (double)i;
    int rows[4];
    float ps[4];
    double p[4];
    for (int j = 0; j < 4; ++j) {
      const int r = i - 1 + j;
      rows[j] = r < 0 ? 0 : (r > kBwRows - 1 ? kBwRows - 1 : r);
    }
    rows_invert<float, float2, BwNodeSmall>(v.bw_tab, rows, (float)(2.0 * u), ps);
    for (int j = 0; j < 4; ++j) p[j] = ps[j] > 0.0f ? log((double)ps[j]) : -700.0;
    double small = exp(catmull_rom<double>(p, t));
    if (small > 0.5) small = 0.5;
    if (exact) small = bw_refine(chi, u, small);  // FP64: the exact distribution
    return U < 0.5 ? small : 1.0 - small;
  }
  return U < 0.5 ? 0.5 - eta : 0.5 + eta;
}

// ---------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ T *as(void *p) { return reinterpret_cast<T *>(p); }

// N values of T moved by one vector load or store.
template <class T, int N>
struct alignas(sizeof(T) * N) Vec {
  T a[N];
};

__device__ __forceinline__ int tile_of(const View &v, const GapDev &g, int64_t k) {
  int64_t lt = k / v.tile;
  if (lt >= g.n_tiles) lt = g.n_tiles - 1;
  if (lt < 0) lt = 0;
  return g.tile_begin + (int)lt;
}

// Warp-aggregated atomic increment of a 64-bit counter; returns this lane's slot.
__device__ __forceinline__ long long warp_reserve(unsigned long long *ctr) {
  unsigned mask = __activemask();
  int leader = __ffs(mask) - 1;
  int lane = threadIdx.x & 31;
  int rank = __popc(mask & ((1u << lane) - 1u));
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(ctr, (unsigned long long)__popc(mask));
  base = __shfl_sync(mask, base, leader);
  return (long long)(base + rank);
}

// ---------------------------------------------------------------------------
template <class R> struct Prec;
template <> struct Prec<float> {
  using W = uint32_t;   // weight in units of w_unit = w0 / 2^8
  using Acc = long long;  // charge in units of w_unit * 2^-23
};
template <> struct Prec<double> {
  using W = double;
  using Acc = double;
};

__device__ __forceinline__ void acc_add(long long *p, long long v) {
  atomicAdd(reinterpret_cast<unsigned long long *>(p), (unsigned long long)v);
}
__device__ __forceinline__ void acc_add(double *p, double v) { atomicAdd(p, v); }
__device__ __forceinline__ void red_shared_add_u32(unsigned *p, unsigned v) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void red_shared_add_s32(int *p, int v) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

// Exact 64-bit charge sums from 32-bit shared reductions: a contribution
// c = q w F (|c| < 2^55: weight units w < 2^32, offset flux |F| <= 2^23) is
// split as c = c2 2^34 + c1 2^17 + c0 with c0, c1 in [0, 2^17) and c2 =
// floor(c / 2^34), each added to its own 32-bit counter.  A node receives at
// most one contribution per lepton of a push item (a move crosses a node at
// most once), at most kPushChunk <= 32768, so the two unsigned limbs stay
// below 32768 (2^17 - 1) < 2^32 and are exact.  The signed limb may wrap: the
// node's sum c2sum 2^34 + c1sum 2^17 + c0sum is formed modulo 2^64, where
// c2sum enters only through its value modulo 2^30, so the sum is exact
// whenever it fits in 64 bits (the bound of the global accumulators too).
__device__ __forceinline__ void limb_add(unsigned *L0, unsigned *L1, int *L2, int i, long long c) {
  const unsigned long long u = (unsigned long long)c;
  red_shared_add_u32(&L0[i], (unsigned)(u & 0x1FFFFull));
  red_shared_add_u32(&L1[i], (unsigned)((u >> 17) & 0x1FFFFull));
  red_shared_add_s32(&L2[i], (int)(c >> 34));
}
__device__ __forceinline__ long long limb_value(unsigned l0, unsigned l1, int l2) {
  return (long long)(((unsigned long long)(long long)l2 << 34) + ((unsigned long long)l1 << 17) +
                     (unsigned long long)l0);
}

__device__ __forceinline__ void acc_add_global(unsigned long long *p, long long v) {
  atomicAdd(p, (unsigned long long)v);
}
__device__ __forceinline__ void acc_add_global(unsigned long long *p, double v) {
  atomicAdd(reinterpret_cast<double *>(p), v);
}
__device__ __forceinline__ double acc_take(unsigned long long *p, long long *) {
  return (double)(long long)atomicExch(p, 0ull);
}
__device__ __forceinline__ double acc_take(unsigned long long *p, double *) {
  return __longlong_as_double((long long)atomicExch(p, 0ull));
}

// Append one lepton to tile t of species s (current buffer); spills to the
// overflow list when the segment is full.
template <class R>
__device__ __noinline__ void append_lepton(const View &v, int s, int t, int32_t k, R phi, R u,
                              typename Prec<R>::W w, R tau, uint64_t id) {
  const int cur = v.ctl->lep_cur;
  int pos = atomicAdd(&v.seg_append[s][t], 1);
  if (pos < v.seg_cap[s][t]) {
    int64_t slot = v.seg_start[s][t] + pos;
    as<R>(v.lphi[cur][s])[slot] = phi;
    as<R>(v.lu[cur][s])[slot] = u;
    as<typename Prec<R>::W>(v.lw[cur][s])[slot] = w;
    as<R>(v.ltau[cur][s])[slot] = tau;
    v.lid[cur][s][slot] = id;
    __threadfence_block();
    v.lk[cur][s][slot] = k;
    atomicAdd(&v.seg_alive[s][t], 1);
  } else {
    long long i = (long long)atomicAdd(reinterpret_cast<unsigned long long *>(&v.ctl->spill_n[s]), 1ull);
    if (i < v.spill_capacity) {
      v.sk[s][i] = k;
      v.stile[s][i] = t;
      v.sphi[s][i] = (double)phi;
      v.su[s][i] = (double)u;
      v.sw[s][i] = (double)w;
      v.stau[s][i] = (double)tau;
      v.sid[s][i] = id;
      atomicAdd(&v.spill_cnt[s][t], 1);
    } else {
      atomicOr(&v.ctl->error, 1);  // storage exhausted
    }
    v.ctl->need_rebin = 1;
    atomicAdd(&v.counters[v.tiles[t].gap * C_NCNT + C_SPILL], 1ull);
  }
}

// append_lepton for a loader, where whole warps append to few tiles: the
// lanes that append to the same (species, tile) reserve their slots with one
// atomic (slots in lane order) and count the stored ones with one more.  The
// whole warp calls it together; lanes with valid == false append nothing.
template <class R>
__device__ __forceinline__ void append_lepton_warp(const View &v, bool valid, int s, int t, int32_t k, R phi,
                                                   R u, typename Prec<R>::W w, R tau, uint64_t id) {
  __syncwarp();
  const int lane = threadIdx.x & 31;
  const unsigned peers = __match_any_sync(0xffffffffu, valid ? s * v.n_tiles + t : -1);
  if (!valid) return;  // the invalid lanes form their own group
  const int leader = __ffs(peers) - 1;
  const int rank = __popc(peers & ((1u << lane) - 1u));
  int base = 0;
  if (lane == leader) base = atomicAdd(&v.seg_append[s][t], __popc(peers));
  base = __shfl_sync(peers, base, leader);
  const int pos = base + rank;
  const bool fits = pos < v.seg_cap[s][t];
  const unsigned stored = __ballot_sync(peers, fits) & peers;
  if (fits) {
    const int cur = v.ctl->lep_cur;
    const int64_t slot = v.seg_start[s][t] + pos;
    as<R>(v.lphi[cur][s])[slot] = phi;
    as<R>(v.lu[cur][s])[slot] = u;
    as<typename Prec<R>::W>(v.lw[cur][s])[slot] = w;
    as<R>(v.ltau[cur][s])[slot] = tau;
    v.lid[cur][s][slot] = id;
    __threadfence_block();
    v.lk[cur][s][slot] = k;
  }
  if (lane == leader && stored) atomicAdd(&v.seg_alive[s][t], __popc(stored));
  if (!fits) {  // the segment is full: the single-lepton path spills (its reservation fails too)
    long long i = (long long)atomicAdd(reinterpret_cast<unsigned long long *>(&v.ctl->spill_n[s]), 1ull);
    if (i < v.spill_capacity) {
      v.sk[s][i] = k;
      v.stile[s][i] = t;
      v.sphi[s][i] = (double)phi;
      v.su[s][i] = (double)u;
      v.sw[s][i] = (double)w;
      v.stau[s][i] = (double)tau;
      v.sid[s][i] = id;
      atomicAdd(&v.spill_cnt[s][t], 1);
    } else {
      atomicOr(&v.ctl->error, 1);  // storage exhausted
    }
    v.ctl->need_rebin = 1;
    atomicAdd(&v.counters[v.tiles[t].gap * C_NCNT + C_SPILL], 1ull);
  }
}

// Weight of a stored lepton in the units of its precision: without QED and
// variable weights the state carries no weights and every lepton has w0
// (FP32: 2^kWeightShift weight units).
template <class R>
__device__ __forceinline__ typename Prec<R>::W lepton_weight(const View &v, const GapDev &g, int buf, int s,
                                                            int64_t slot) {
  using W = typename Prec<R>::W;
  if (v.qed_any || v.has_w) return as<W>(v.lw[buf][s])[slot];
  if (sizeof(R) == 4) return (W)(1u << kWeightShift);
  return (W)g.w0;
}

// Lepton position from an absolute X (cells): node-centred (k, phi').
template <class R>
__device__ __forceinline__ void split_position(double X, int64_t nx, bool periodic, int32_t &k,
                                               R &phi) {
  double a = X + 0.5;
  double kf = floor(a);
  double f = a - kf;  // [0, 1)
  int64_t kk = (int64_t)kf;
  R p = (R)(1.0 + f);
  if (p >= (R)2) {
    p -= (R)1;
    kk += 1;
  }
  if (periodic) {
    kk %= nx;
    if (kk < 0) kk += nx;
  }
  k = (int32_t)kk;
  phi = p;
}

// Photon event kinds and markers of pev.
enum PhotonEvent : int32_t { PH_CONVERT = 1, PH_ESCAPE = 2, PH_RESCHEDULE = 3, PH_INERT = 4 };
constexpr int32_t kPhPending = -2, kPhDead = -1, kPhNever = 0x7fffffff;

// Append a photon, unscheduled: it sits at X_ref at the start of step n_ref,
// has accumulated tau_acc before step m, and will be scheduled by the next
// photon pass.
static __device__ __noinline__ bool photon_append(const View &v, int buf, int gap, double X_ref, int32_t n_ref,
                                              double x, double w, double tau_star, double tau_acc,
                                              uint64_t id, int32_t n0, int32_t dir, int32_t m) {
  long long slot = warp_reserve(reinterpret_cast<unsigned long long *>(&v.ctl->ph_count[buf]));
  if (slot < v.ph_capacity) {
    v.pXr[buf][slot] = X_ref;
    v.px[buf][slot] = x;
    v.pw[buf][slot] = w;
    v.pts[buf][slot] = tau_star;
    v.pta[buf][slot] = tau_acc;
    v.pid[buf][slot] = id;
    v.pn0[buf][slot] = n0;
    v.pnr[buf][slot] = n_ref;
    v.pdir[buf][slot] = dir;
    v.pgap[buf][slot] = gap;
    v.pm[buf][slot] = m;
    v.pkind[buf][slot] = 0;
    v.pev[buf][slot] = kPhPending;
    return true;
  }
  atomicAdd(&v.counters[gap * C_NCNT + C_PH_OVF], 1ull);
  atomicOr(&v.ctl->error, 2);
  return false;
}

// Photons stored in buffer b.  The fill counter keeps counting appends that
// found the store full (they are refused and flagged), so readers clamp it.
__device__ __forceinline__ int64_t photon_fill(const View &v, int b) {
  const int64_t n = v.ctl->ph_count[b];
  return n < v.ph_capacity ? n : v.ph_capacity;
}

// Position of a photon at the start of step m: photons move at c along h
// (Sect. 6.1), X = X_ref + dir (m - n_ref) c dt/dx, rounded once in the
// product and once in the sum (never fused), wrapped into the box when
// periodic.
__device__ __forceinline__ double photon_pos(const GapDev &g, double Xr, int32_t nr, int32_t dir, int64_t m) {
  const double t = __dmul_rn((double)(m - (int64_t)nr), g.cdx);
  double X = __dadd_rn(Xr, dir > 0 ? t : -t);
  if (g.periodic) {
    const double L = (double)g.nx;
    X = fmod(X, L);
    if (X < 0.0) X += L;
    if (X >= L) X -= L;
  }
  return X;
}

// Breit-Wheeler optical depth gained in step m (eq. tau_bw) at the mid-step
// angle sin(psi) = |sin(l / R_curv)|, l = c (m - n0 + 1/2) dt (Sect. 6.1
// virtual B_y), chi_x = x b sin(psi).  FP64: evaluated left to right as
// dt rate_mult alpha_em / lambda_hat b sin(psi) T_BW(chi_x).
__device__ __forceinline__ double bw_step_depth(const GapDev &g, double x, int32_t n0, int64_t m) {
  const double lmid = ((double)m - (double)n0 + 0.5) * g.dt;
  const double sp = fabs(sin(lmid / g.rho_hat));
  const double chi = x * g.b * sp;
  return g.dt * g.rate_mult * kAlphaEm / g.lambda_hat * g.b * sp * tbw_d(chi);
}
__device__ __forceinline__ float tbw_f(float chi) {
  if (!(chi > 0.0f)) return 0.0f;
  return 0.23f * expf(-8.0f / (3.0f * chi)) * exp2f(-log2f(1.0f + 0.22f * chi) * (1.0f / 3.0f));
}
__device__ __forceinline__ float bw_step_depth_f(const GapDev &g, float x, int32_t n0, int64_t m) {
  // the step count since birth fits 32 bits: converted from int32 (64-bit
  // type conversions run at the low FP64 rate here)
  const float lmid = ((float)(int32_t)(m - (int64_t)n0) + 0.5f) * g.f_dt;
  const float sp = fabsf(sinf(lmid / g.f_rho));
  const float chi = x * g.f_b * sp;
  return g.f_dt * g.f_rate * (float)kAlphaEm / g.f_lam * g.f_b * sp * tbw_f(chi);
}

// Tally one e+- absorbed at h < 0 (the return flux of Sect. 6.5) with weight
// w in the bin of ln gamma, gamma from its momentum in double precision.
// Cell c of a transverse E array, with the conductor images of a surface gap
// (c in [-1, nx] here).
__device__ __forceinline__ double cell_at(const double *F, int64_t c, const GapDev &g) {
  if (g.periodic) return F[c < 0 ? c + g.nx : (c >= g.nx ? c - g.nx : c)];
  if (c < 0) return -F[-1 - c];
  if (c >= g.nx) return -F[2 * g.nx - 1 - c];
  return F[c];
}

__device__ __forceinline__ void tally_return(const View &v, int gap, double u, double w) {
  double b = floor(log(sqrt(1.0 + u * u)) / kRetDln);
  if (!(b >= 0.0)) b = 0.0;
  if (b > (double)(kRetBins - 1)) b = (double)(kRetBins - 1);
  atomicAdd(&v.ret_hist[gap * kRetBins + (int)b], w);
}

}  // namespace gapk
