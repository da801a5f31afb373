// merge.cu -- weight-conserving merge of leptons under the macro-particle cap,
// and of the photons born in a step (at the end of the file).
//
// When a gap holds more leptons + photons than its cap after a step, the
// leptons of every (species, dual cell k, direction, bin of ln gamma of width
// 0.1 * 2^level) group with at least three members become two leptons at the
// weight-averaged offset of the dual cell.  Their momenta follow from
// two-body kinematics on S+ = sum w (gamma + u) and S- = sum w (gamma - u):
// the centre moves with rapidity eta = 0.5 ln(S+/S-), the invariant mass is
// M = sqrt(S+ S-) = W + D with D = sum w 2 sinh^2((asinh u - eta)/2) (a
// second pass, free of the cancellation in S+ S- - W^2), and in the centre
// frame the two move apart with momentum
// p* = sqrt((M^2 - W^2)(M^2 - (w_a - w_b)^2)) / (2M); weight, momentum and
// energy are conserved.  Re-centring moves charge across node k; that charge
// is applied to E_k like a deposit, so Gauss's law holds (exactly, in the
// integer charge units of the FP32 state).  level counts the consecutive
// over-cap steps of the gap (at most 7) and resets when the gap is under cap.
#include "gap_internal.cuh"
#include "kernels.h"

namespace gapk {

constexpr int kMergeBins = 256;
constexpr int kMergeKeys = 2 * kMergeBins;  // direction x bin
constexpr int kMergeCache = 256;  // leptons of a node whose gamma + |u| and its inverse a warp keeps
// one warp's key table, touched list and the cache of its node's leptons
constexpr int kMergeWarpBytes = 46 * kMergeKeys + 16 * kMergeCache;
constexpr uint32_t CH_MERGE = 10;

// One thread per gap: decide whether the gap merges this step.
__global__ void k_merge_check(View v) {
  const int gi = blockIdx.x * blockDim.x + threadIdx.x;
  if (gi == 0) v.ctl->mlist_n = 0;  // the merging segments of this step are listed afresh
  if (gi >= v.n_gaps) return;
  const GapDev &g = v.gaps[gi];
  int32_t *st = v.merge_state + 4 * gi;  // [flag, level, -, -]
  double *width = v.merge_width + gi;
  if (g.cap <= 0) {
    st[0] = 0;
    return;
  }
  int64_t total = v.ph_gap[gi];
  for (int t = g.tile_begin; t < g.tile_begin + g.n_tiles; ++t)
    total += (int64_t)v.seg_alive[0][t] + (int64_t)v.seg_alive[1][t];
  if (total > g.cap) {
    const int level = st[1];
    *width = 0.1 * (double)(1 << level);
    st[1] = level < 7 ? level + 1 : 7;
    st[0] = 1;
    atomicOr(&v.ctl->flags, 1);
  } else {
    st[0] = 0;
    st[1] = 0;
  }
}

template <class R>
struct MergeAcc;
template <>
struct MergeAcc<double> {  // FP64 state: FP64 sums of w and w phi
  using T = double;
};
template <>
struct MergeAcc<float> {  // FP32 state: exact integer sums of m and m Phi (2^-23 units)
  using T = unsigned long long;
};

constexpr int kMergeWarps = 4;  // warps per merge block, each with its own key table
// nodes of a tile: tile, or up to 3 more for the last tile of a gap (a
// remainder below 4 joins the previous tile); mrun rows have this length
__device__ __forceinline__ int merge_row(const View &v) { return v.tile + 4; }

// An output slot for each lane of a warp that asks for one.
__device__ __forceinline__ int warp_slot(int *cursor) {
  const unsigned mask = __activemask();
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(cursor, __popc(mask));
  base = __shfl_sync(mask, base, leader);
  return base + __popc(mask & ((1u << lane) - 1u));
}

// Part 1, per (species, tile) segment of a merging gap: a counting sort of
// the segment by node into the other buffer; the end of each node's run
// (from the segment's start) goes to mrun, and the segment is listed.
template <class R>
__global__ void __launch_bounds__(256) k_merge_sort(View v) {
  using W = typename Prec<R>::W;
  if (!(v.ctl->flags & 1)) return;
  const int s = blockIdx.x / v.n_tiles, t = blockIdx.x % v.n_tiles;
  const TileDev ti = v.tiles[t];
  if (!v.merge_state[4 * ti.gap]) return;
  const GapDev &g = v.gaps[ti.gap];
  const int nk = ti.nk, k0 = ti.k0;
  const int cur = v.ctl->lep_cur, nxt = cur ^ 1;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  extern __shared__ int hist[];  // [nk + 1]
  __shared__ int wsum[8];        // <= 8 warps
  __shared__ int carry;
  const int64_t seg0 = v.seg_start[s][t];
  const int used = v.seg_used[s][t];
  for (int i = threadIdx.x; i <= nk; i += blockDim.x) hist[i] = 0;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < used; i += blockDim.x) {
    const int32_t k = v.lk[cur][s][seg0 + i];
    if (k < 0) continue;
    if (k < k0 || k >= k0 + nk) {  // never: a tile holds only its own nodes
      atomicOr(&v.ctl->error, 32);
      continue;
    }
    atomicAdd(&hist[k - k0], 1);
  }
  __syncthreads();
  for (int base = 0; base < nk; base += blockDim.x) {  // exclusive scan in place
    const int i = base + threadIdx.x;
    const int x = i < nk ? hist[i] : 0;
    int y = x;
    for (int o = 1; o < 32; o <<= 1) {
      const int z = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) y += z;
    }
    if (lane == 31) wsum[wid] = y;
    __syncthreads();
    int before = carry;
    for (int w = 0; w < wid; ++w) before += wsum[w];
    if (i < nk) hist[i] = before + y - x;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = before + y;
    __syncthreads();
  }
  // scatter: hist[i] is the next free slot of node i's run
  for (int i = threadIdx.x; i < used; i += blockDim.x) {
    const int64_t src = seg0 + i;
    const int32_t k = v.lk[cur][s][src];
    if (k < k0 || k >= k0 + nk) continue;
    const int pos = atomicAdd(&hist[k - k0], 1);
    const int64_t d = seg0 + pos;
    v.lk[nxt][s][d] = k;
    as<R>(v.lphi[nxt][s])[d] = as<R>(v.lphi[cur][s])[src];
    as<R>(v.lu[nxt][s])[d] = as<R>(v.lu[cur][s])[src];
    as<W>(v.lw[nxt][s])[d] = lepton_weight<R>(v, g, cur, s, src);
    as<R>(v.ltau[nxt][s])[d] = as<R>(v.ltau[cur][s])[src];
    v.lid[nxt][s][d] = v.lid[cur][s][src];
  }
  __syncthreads();
  // after the scatter hist[i] holds the end of node i's run
  const int seg = s * v.n_tiles + t;
  for (int i = threadIdx.x; i < nk; i += blockDim.x) v.mrun[(int64_t)seg * merge_row(v) + i] = hist[i];
  if (threadIdx.x == 0) {
    v.mout[seg] = 0;
    v.mlist[atomicAdd(&v.ctl->mlist_n, 1)] = seg;
  }
}

// Part 2: the nodes of the listed segments, one warp per node, spread over
// every warp of the GPU (a tile's nodes in one block made the densest tiles
// a long serial chain that the rest of the GPU waited on): group, merge,
// write back into the current buffer at the segment's output cursor.
template <class R>
__global__ void __launch_bounds__(32 * kMergeWarps) k_merge_nodes(View v) {
  using W = typename Prec<R>::W;
  using A = typename MergeAcc<R>::T;
  if (!(v.ctl->flags & 1)) return;
  const int cur = v.ctl->lep_cur, nxt = cur ^ 1;
  const int64_t step = v.ctl->step;  // the step just completed is step - 1
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;

  // per warp: a direct-mapped table over the 512 (direction, bin) keys, the
  // list of keys the current node touched (only those are reset), and the
  // cache of the node's gamma + |u|
  extern __shared__ __align__(16) unsigned char msm[];
  unsigned char *wb = msm + (size_t)wid * kMergeWarpBytes;
  int *cnt = reinterpret_cast<int *>(wb);
  unsigned long long *minid = reinterpret_cast<unsigned long long *>(wb + 4 * kMergeKeys);
  A *sw = reinterpret_cast<A *>(wb + 12 * kMergeKeys);                                // sum w
  A *sphi = reinterpret_cast<A *>(wb + 20 * kMergeKeys);                              // sum w phi
  double *sp = reinterpret_cast<double *>(wb + 28 * kMergeKeys);                      // sum w (g+u), then E = exp(eta)
  double *sm = reinterpret_cast<double *>(wb + 36 * kMergeKeys);                      // sum w (g-u), then D
  short *touched = reinterpret_cast<short *>(wb + 44 * kMergeKeys);                   // [kMergeKeys]
  double *cbig = reinterpret_cast<double *>(wb + 46 * kMergeKeys);                    // [kMergeCache]
  double *crb = cbig + kMergeCache;                                                   // [kMergeCache]
  __shared__ int ntouched[kMergeWarps];
  for (int i = lane; i < kMergeKeys; i += 32) {
    cnt[i] = 0;
    minid[i] = ~0ull;
    sw[i] = (A)0;
    sphi[i] = (A)0;
    sp[i] = 0.0;
    sm[i] = 0.0;
  }
  if (lane == 0) ntouched[wid] = 0;
  __syncwarp();

  const int row = merge_row(v);
  const int64_t ntask = (int64_t)v.ctl->mlist_n * row;
  const int64_t nwarps = (int64_t)gridDim.x * kMergeWarps;
  for (int64_t task = (int64_t)blockIdx.x * kMergeWarps + wid; task < ntask; task += nwarps) {
    const int seg = v.mlist[task / row], node = (int)(task % row);
    const int s = seg / v.n_tiles, t = seg % v.n_tiles;
    const TileDev ti = v.tiles[t];
    if (node >= ti.nk) continue;
    const GapDev &g = v.gaps[ti.gap];
    const double width = v.merge_width[ti.gap];
    const int q = s == 0 ? -1 : 1;
    const int64_t seg0 = v.seg_start[s][t];
    int *out_cursor = &v.mout[seg];
    const int32_t *run = v.mrun + (int64_t)seg * row;
    const int r0 = node == 0 ? 0 : run[node - 1], r1 = run[node];

    auto copy_out = [&](int64_t src) {
      const int64_t d = seg0 + warp_slot(out_cursor);
      v.lk[cur][s][d] = v.lk[nxt][s][src];
      as<R>(v.lphi[cur][s])[d] = as<R>(v.lphi[nxt][s])[src];
      as<R>(v.lu[cur][s])[d] = as<R>(v.lu[nxt][s])[src];
      as<W>(v.lw[cur][s])[d] = as<W>(v.lw[nxt][s])[src];
      as<R>(v.ltau[cur][s])[d] = as<R>(v.ltau[nxt][s])[src];
      v.lid[cur][s][d] = v.lid[nxt][s][src];
    };
    if (r1 - r0 < 3) {  // nothing to merge: copy through
      for (int i = r0 + lane; i < r1; i += 32) copy_out(seg0 + i);
      continue;
    }
    // the bin floor(ln gamma / width) of the FP64 evaluation (FP64 runs at a
    // small fraction of the FP32 rate here): taken from an FP32 evaluation t
    // where that lies more than 1e-3 of a bin from a bin edge, else evaluated
    // in FP64.  The FP32 t is within 1e-4 of a bin of the FP64 one: the
    // rounding of u, 1 + u^2 and the square root moves ln gamma by ~2e-7,
    // logf's ulp at ln gamma <= 21 is <= 2e-6, times 1/width <= 10, and the
    // rounding of t <= 256 and of 1/width adds ~2e-5.
    const float winv_f = (float)(1.0 / width);
    auto key_of = [&](int64_t src) -> int {
      const R ur = as<R>(v.lu[nxt][s])[src];
      const float uf = (float)ur;  // FP32 state: the stored value, no 64-bit type conversion (FP64 rate)
      const float tf = logf(sqrtf(1.0f + uf * uf)) * winv_f;
      const float bf = floorf(tf);
      int b;
      if (tf - bf > 1e-3f && bf + 1.0f - tf > 1e-3f && tf < (float)(kMergeBins - 1)) {
        b = (int)bf;
      } else {
        const double u = (double)ur;
        const double tt = floor(log(sqrt(1.0 + u * u)) / width);
        b = tt < 0.0 ? 0 : (tt > (double)(kMergeBins - 1) ? kMergeBins - 1 : (int)tt);
      }
      return (ur >= (R)0 ? 1 : 0) * kMergeBins + b;
    };
    // a group merges when it has three or more members; in the FP32 state
    // its children carry 32-bit weights, so a group whose summed weight would
    // not split into two of them is left unmerged
    auto merges = [&](int key) -> bool {
      if (cnt[key] < 3) return false;
      if (sizeof(R) == 4 && (unsigned long long)sw[key] > 2ull * 0xffffffffull) return false;
      return true;
    };
    // weights in the state's units (FP32 state: integer multiples of w_unit);
    // S+, S- and D are summed in these units and D converted per group
    auto weight_of = [&](int64_t src) -> double { return (double)as<W>(v.lw[nxt][s])[src]; };
    const double wscale = sizeof(R) == 4 ? g.w_unit : 1.0;

    for (int i = r0 + lane; i < r1; i += 32) {
      const int64_t src = seg0 + i;
      const int key = key_of(src);
      const double u = (double)as<R>(v.lu[nxt][s])[src];
      const double w = weight_of(src);
      const double big = sqrt(1.0 + u * u) + fabs(u), rb = 1.0 / big;  // gamma + |u| and its inverse
      if (i - r0 < kMergeCache) {  // kept for the D pass (a square root and a division in FP64)
        cbig[i - r0] = big;
        crb[i - r0] = rb;
      }
      const double gp = u >= 0.0 ? big : rb, gmn = u >= 0.0 ? rb : big;
      const R phi = as<R>(v.lphi[nxt][s])[src];
      if (atomicAdd(&cnt[key], 1) == 0) touched[atomicAdd(&ntouched[wid], 1)] = (short)key;
      atomicMin(&minid[key], (unsigned long long)v.lid[nxt][s][src]);
      atomicAdd(&sp[key], w * gp);
      atomicAdd(&sm[key], w * gmn);
      if (sizeof(R) == 4) {
        const W wq = as<W>(v.lw[nxt][s])[src];
        const long long F = __float2int_rn(((float)phi - 1.0f) * 8388608.0f);
        atomicAdd(reinterpret_cast<unsigned long long *>(&sw[key]), (unsigned long long)wq);
        atomicAdd(reinterpret_cast<unsigned long long *>(&sphi[key]), (unsigned long long)((long long)wq * F));
      } else {
        atomicAdd(reinterpret_cast<double *>(&sw[key]), w);
        atomicAdd(reinterpret_cast<double *>(&sphi[key]), w * ((double)phi - 1.0));
      }
    }
    __syncwarp();
    const int nt = ntouched[wid];
    // E = exp(eta) = sqrt(S+/S-), the centre's rapidity factor, into sp[];
    // sm[] then accumulates D = sum w 2 sinh^2((asinh u - eta)/2), so that
    // M = W + D and M^2 - W^2 = D (2W + D) carry no cancellation for nearly
    // cold groups
    for (int j = lane; j < nt; j += 32) {
      const int key = touched[j];
      if (!merges(key)) continue;
      sp[key] = sqrt(sp[key] / sm[key]);
      sm[key] = 0.0;
    }
    __syncwarp();
    // With e = exp(asinh u) = gamma + u and x = e/E = exp(asinh u - eta),
    // 2 sinh^2((asinh u - eta)/2) = (x + 1/x - 2)/2 = (e - E)^2/(2 e E):
    // for u >= 0, e = gamma + |u|; for u < 0, e = 1/(gamma + |u|) and the
    // term is (1 - E (gamma + |u|))^2/(2 E (gamma + |u|)).  The difference
    // carries the rounding of e and E alone (a few 1e-16 relative), as
    // asinh u - eta does, without the FP64 asinh and sinh (FP64 runs at a
    // small fraction of the FP32 rate); sm[] sums w d^2/(gamma + |u|) and
    // the group's 1/(2E) is applied once.
    for (int i = r0 + lane; i < r1; i += 32) {
      const int64_t src = seg0 + i;
      const int key = key_of(src);
      if (!merges(key)) continue;
      const R ur = as<R>(v.lu[nxt][s])[src];
      double big, rb;
      if (i - r0 < kMergeCache) {
        big = cbig[i - r0];
        rb = crb[i - r0];
      } else {
        const double u = (double)ur;
        big = sqrt(1.0 + u * u) + fabs(u);
        rb = 1.0 / big;
      }
      const double E = sp[key];
      const double d = ur >= (R)0 ? big - E : fma(-E, big, 1.0);
      atomicAdd(&sm[key], weight_of(src) * (d * d) * rb);
    }
    __syncwarp();
    // leptons of groups that do not merge are copied through
    for (int i = r0 + lane; i < r1; i += 32) {
      const int64_t src = seg0 + i;
      if (!merges(key_of(src))) copy_out(src);
    }
    // groups of three or more become two
    const int32_t kn = ti.k0 + node;
    unsigned long long merged = 0;
    for (int j = lane; j < nt; j += 32) {
      const int key = touched[j];
      const int n = cnt[key];
      if (!merges(key)) continue;
      double Wt, flux;
      long long flux_units = 0;  // FP32 state: the moved charge in integer units
      W wa, wb;
      R phi_store;
      if (sizeof(R) == 4) {
        const long long Wi = (long long)sw[key], Si = (long long)sphi[key];
        const long long Fm = (2 * Si + Wi) / (2 * Wi);  // round(S/W) for S >= 0
        flux_units = (long long)q * (Wi * Fm - Si);
        flux = (double)flux_units * g.w_unit * kPhiUnit;
        phi_store = (R)(1.0f + (float)Fm * (float)kPhiUnit);
        wa = (W)(Wi / 2);
        wb = (W)(Wi - Wi / 2);
        Wt = (double)Wi * g.w_unit;
      } else {
        const double Wd = (double)sw[key], Sd = (double)sphi[key];
        const double phim = Sd / Wd;
        flux = (double)q * (Wd * phim - Sd);
        phi_store = (R)(1.0 + phim);
        if (phi_store >= (R)2) phi_store = (R)2 - (R)2.220446049250313e-16;
        wa = (W)(0.5 * Wd);
        wb = (W)(Wd - 0.5 * Wd);
        Wt = Wd;
      }
      const double wad = sizeof(R) == 4 ? (double)wa * g.w_unit : (double)wa;
      const double wbd = sizeof(R) == 4 ? (double)wb * g.w_unit : (double)wb;
      const double E = sp[key], eta = log(E), D = sm[key] * wscale / (2.0 * E), M = Wt + D;
      const double q2 = D * (2.0 * Wt + D) * (M * M - (wad - wbd) * (wad - wbd));
      const double ps = q2 > 0.0 ? sqrt(q2) / (2.0 * M) : 0.0;
      const double ua = sinh(eta + asinh(ps / wad)), ub = sinh(eta - asinh(ps / wbd));
      // the charge moved across node kn by re-centring; a gap with a current
      // filter collects it for smoothing (k_filter_apply, mode 1)
      int64_t node_g = kn;
      if (g.periodic) node_g %= g.nx;
      if (flux != 0.0 && g.defer) {
        if (sizeof(R) == 4) acc_add_global(&v.Dg[g.node_off + node_g], flux_units);
        else acc_add_global(&v.Dg[g.node_off + node_g], flux);
      } else if (flux != 0.0 && (g.periodic || node_g > 0)) {
        atomicAdd(&v.E[v.ctl->e_cur][g.node_off + node_g], -flux);
      }
      const int o = atomicAdd(out_cursor, 2);
      for (int c = 0; c < 2; ++c) {
        const int64_t d = seg0 + o + c;
        const uint64_t id = child_id(minid[key], (uint32_t)(step - 1), CH_MERGE, (uint32_t)c) & ~kPhotonBit;
        v.lk[cur][s][d] = kn;
        as<R>(v.lphi[cur][s])[d] = phi_store;
        as<R>(v.lu[cur][s])[d] = (R)(c == 0 ? ua : ub);
        as<W>(v.lw[cur][s])[d] = c == 0 ? wa : wb;
        as<R>(v.ltau[cur][s])[d] = (R)(-log(uniform53(g.seed, id, (uint32_t)step, CH_TAU0, 0)));
        v.lid[cur][s][d] = id;
      }
      merged += (unsigned long long)(n - 2);
    }
    for (int o = 16; o > 0; o >>= 1) merged += __shfl_down_sync(0xffffffffu, merged, o);
    if (lane == 0 && merged) atomicAdd(&v.counters[ti.gap * C_NCNT + C_MERGED], merged);
    __syncwarp();
    // reset the touched keys for the warp's next node
    for (int j = lane; j < nt; j += 32) {
      const int key = touched[j];
      cnt[key] = 0;
      minid[key] = ~0ull;
      sw[key] = (A)0;
      sphi[key] = (A)0;
      sp[key] = 0.0;
      sm[key] = 0.0;
    }
    __syncwarp();
    if (lane == 0) ntouched[wid] = 0;
    __syncwarp();
  }
}

// Part 3: the listed segments take their output cursors as their fill.
__global__ void k_merge_fin(View v) {
  if (!(v.ctl->flags & 1)) return;
  const int n = v.ctl->mlist_n;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
    const int seg = v.mlist[j];
    const int s = seg / v.n_tiles, t = seg % v.n_tiles;
    const int o = v.mout[seg];
    v.seg_used[s][t] = o;
    v.seg_append[s][t] = o;
    v.seg_alive[s][t] = o;
  }
}

// ---------------------------------------------------------------------------
// Photons merged at birth.  While a gap is over its cap, the photons born in
// this step's push (n0 = the step now beginning) of each (cell, direction,
// bin of ln x of the leptons' width) group with at least two members become
// one photon: weight W = sum w, energy sum w x / W, position sum w X / W,
// the group's birth step, a fresh threshold depth (channel BW_TAU) and no
// accumulated depth, scheduled by the next photon pass; its id is the child
// (channel MERGE) of the group's smallest id.  Groups are gathered in an
// open-addressing table keyed by (gap + 1, cell, direction, bin): one pass
// adds every newborn photon's weight and moments to its key's entry, a
// second retires the members of groups of two or more and lets the member
// with the smallest id append the merged photon, a third clears the table.
// A photon whose key finds no free entry within kPhmProbe probes (the table
// holds twice the photon store, so only a store larger than 2^21 photons can
// fill it that far) stays unmerged.
constexpr int kPhmProbe = 64;

__device__ __forceinline__ uint64_t phm_photon_key(const View &v, int b, int64_t i, int64_t step, double &X) {
  if (v.pev[b][i] == kPhDead || v.pn0[b][i] != (int32_t)step) return 0ull;
  const int gap = v.pgap[b][i];
  if (!v.merge_state[4 * gap]) return 0ull;
  const GapDev &g = v.gaps[gap];
  const int32_t dir = v.pdir[b][i];
  X = photon_pos(g, v.pXr[b][i], v.pnr[b][i], dir, step);
  int64_t cell = (int64_t)floor(X);
  if (g.periodic) {
    cell %= g.nx;
    if (cell < 0) cell += g.nx;
  }
  int64_t bin = (int64_t)floor(log(v.px[b][i]) / v.merge_width[gap]);
  if (bin < 0) bin = 0;
  if (bin > kMergeBins - 1) bin = kMergeBins - 1;
  return ((uint64_t)(gap + 1) << 40) | ((uint64_t)cell << 9) | ((uint64_t)(dir > 0) << 8) | (uint64_t)bin;
}

// Entry of `key`: inserted when `insert`, else looked up; -1 if not found.
__device__ __forceinline__ int64_t phm_slot(const View &v, uint64_t key, bool insert) {
  const uint64_t mask = (uint64_t)v.phm_size - 1;
  uint64_t h = mix64(key) & mask;
  for (int p = 0; p < kPhmProbe; ++p, h = (h + 1) & mask) {
    if (insert) {
      const unsigned long long old = atomicCAS(&v.phm_key[h], 0ull, (unsigned long long)key);
      if (old == 0ull || old == key) return (int64_t)h;
    } else {
      const unsigned long long k = v.phm_key[h];
      if (k == key) return (int64_t)h;
      if (k == 0ull) return -1;
    }
  }
  return -1;
}

__global__ void k_phm_insert(View v) {
  if (!(v.ctl->flags & 1)) return;
  const int b = v.ctl->ph_cur;
  const int64_t step = v.ctl->step;
  const int64_t n = photon_fill(v, b);
  const int64_t i0 = v.ctl->ph_nb_start < n ? v.ctl->ph_nb_start : n;
  if (blockIdx.x == 0 && threadIdx.x == 0) v.ctl->phm_end = n;  // appends of the next pass lie beyond
  for (int64_t i = i0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double X = 0.0;
    const uint64_t key = phm_photon_key(v, b, i, step, X);
    if (!key) continue;
    const int64_t h = phm_slot(v, key, true);
    if (h < 0) continue;
    const double w = v.pw[b][i], x = v.px[b][i];
    atomicAdd(&v.phm_cnt[h], 1u);
    atomicAdd(&v.phm_W[h], w);
    atomicAdd(&v.phm_Wx[h], w * x);
    atomicAdd(&v.phm_WX[h], w * X);
    atomicMax(&v.phm_nid[h], ~(unsigned long long)v.pid[b][i]);
  }
}

__global__ void k_phm_emit(View v) {
  if (!(v.ctl->flags & 1)) return;
  const int b = v.ctl->ph_cur;
  const int64_t step = v.ctl->step;
  const int64_t n = v.ctl->phm_end;
  const int64_t i0 = v.ctl->ph_nb_start < n ? v.ctl->ph_nb_start : n;
  unsigned long long killed = 0;
  for (int64_t i = i0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double X = 0.0;
    const uint64_t key = phm_photon_key(v, b, i, step, X);
    if (!key) continue;
    const int64_t h = phm_slot(v, key, false);
    if (h < 0) continue;
    const unsigned c = v.phm_cnt[h];
    if (c < 2) continue;
    const int gap = v.pgap[b][i];
    const uint64_t id = v.pid[b][i];
    v.pev[b][i] = kPhDead;
    atomicSub(&v.ph_gap[gap], 1);
    ++killed;
    if (~id == v.phm_nid[h]) {  // the group's smallest id appends the merged photon
      const GapDev &g = v.gaps[gap];
      const double W = v.phm_W[h];
      const uint64_t nid = child_id(id, (uint32_t)(step - 1), CH_MERGE, 0u) | kPhotonBit;
      const double ts = -log(uniform53(g.seed, nid, (uint32_t)step, CH_BW_TAU, 0));
      if (photon_append(v, b, gap, v.phm_WX[h] / W, (int32_t)step, v.phm_Wx[h] / W, W, ts, 0.0, nid, (int32_t)step,
                        v.pdir[b][i], (int32_t)step))
        atomicAdd(&v.ph_gap[gap], 1);
      atomicAdd(&v.counters[gap * C_NCNT + C_PH_MERGED], (unsigned long long)(c - 1));
    }
  }
  if (killed) atomicAdd(reinterpret_cast<unsigned long long *>(&v.ctl->ph_dead), killed);
}

__global__ void k_phm_clear(View v) {
  if (!(v.ctl->flags & 1)) return;
  for (int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; h < v.phm_size; h += (int64_t)gridDim.x * blockDim.x) {
    if (v.phm_key[h] == 0ull) continue;
    v.phm_key[h] = 0ull;
    v.phm_nid[h] = 0ull;
    v.phm_W[h] = 0.0;
    v.phm_Wx[h] = 0.0;
    v.phm_WX[h] = 0.0;
    v.phm_cnt[h] = 0u;
  }
}

__global__ void k_merge_done(View v) { v.ctl->flags &= ~1; }

void launch_merge(const View &v, cudaStream_t st) {
  k_merge_check<<<(v.n_gaps + 127) / 128, 128, 0, st>>>(v);
  const size_t hist = (size_t)(v.tile + 8) * sizeof(int);
  const int smem = kMergeWarps * kMergeWarpBytes;  // above 48 KB: opted into once
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_merge_nodes<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    cudaFuncSetAttribute(k_merge_nodes<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    attr_set = true;
  }
  // the node kernel runs two blocks per SM (its tables), each warp taking nodes in turn
  if (v.precision == GAP_FP32_STATE) {
    k_merge_sort<float><<<2 * v.n_tiles, 256, hist, st>>>(v);
    k_merge_nodes<float><<<2 * 148, 32 * kMergeWarps, smem, st>>>(v);
  } else {
    k_merge_sort<double><<<2 * v.n_tiles, 256, hist, st>>>(v);
    k_merge_nodes<double><<<2 * 148, 32 * kMergeWarps, smem, st>>>(v);
  }
  k_merge_fin<<<(2 * v.n_tiles + 255) / 256, 256, 0, st>>>(v);
  if (v.phm_size > 0) {
    k_phm_insert<<<2 * 148, 256, 0, st>>>(v);
    k_phm_emit<<<2 * 148, 256, 0, st>>>(v);
    k_phm_clear<<<2 * 148, 256, 0, st>>>(v);
  }
  k_merge_done<<<1, 1, 0, st>>>(v);
  if (v.defer_any) launch_filter(v, 1, st);  // smoothed re-centring correction of filter gaps
}

}  // namespace gapk
