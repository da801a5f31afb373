// filter.cu -- the binomial current filter (Sect. 6.1: the current is
// smoothed by a 3-point binomial filter, 8 passes per step).
//
//   k_flux_take     the node flux a step (or a merge) left in the global
//                   accumulators -> scratch; the accumulators are zeroed
//   k_filter_apply  P passes of (1/4, 1/2, 1/4), as the equal binomial
//                   convolution, over chunks of each tile's nodes held in
//                   shared memory with P-node halos (exact integers for the
//                   FP32 state's integer flux, doubles otherwise), then Ampere
//                   E^{n+1} = E^n + (dt j_m - S D) (mode 0) or the merge's
//                   re-centring correction E -= S F (mode 1)
//
// Values beyond the ends of a node array: a periodic gap wraps; a surface gap
// mirrors evenly about nodes 0 and nx.  The cell charge of the Gauss solve
// and residual is mirrored oddly about the same nodes (init.cu), the pairing
// under which smoothing commutes with the node-to-cell difference, so Gauss's
// law holds for the smoothed charge.  Both kernels touch only gaps that defer
// Ampere (filter_passes > 0, or protons or transverse fields: zero passes,
// the update alone, plus dt jv_h of the transverse fields; and every gap
// under the two-pass FP32 QED push, zero passes, for the update), the merge's
// correction (mode 1) only those with a filter or protons or fields, and
// the tiles of a gap cover its nodes k0 .. k0 + nk - 1 without overlap.
#include <algorithm>

#include "gap_internal.cuh"
#include "kernels.h"

namespace gapk {

constexpr int kFilterChunk = 1024;  // nodes smoothed per shared-memory round
constexpr int kMaxPasses = 16;      // upper bound of filter_passes (checked at init)
static_assert(kMaxPasses <= 16, "the integer smoothing of the FP32 flux holds 16 passes");

// Source index of position j of a node array of n values extended beyond its
// ends (|j| and j - n stay below n: the init check nx >= 2 P + 2 keeps every
// halo within one mirror image).
__device__ __forceinline__ int64_t node_source(int64_t j, int64_t n, bool periodic) {
  if (periodic) {
    j %= n;
    return j < 0 ? j + n : j;
  }
  if (j < 0) return -j;
  if (j > n - 1) return 2 * (n - 1) - j;
  return j;
}

// The push has finished: every node has one owner here, so plain loads and
// stores take and clear the accumulators.  FP32 state: the exact integer
// flux is kept as is (the smoothing runs in integers); FP64 state: doubles.
template <class R>
__global__ void k_flux_take(View v, int mode) {
  const TileDev ti = v.tiles[blockIdx.x];
  const GapDev &g = v.gaps[ti.gap];
  if (!(mode == 0 ? g.ampere_late : g.defer)) return;
  unsigned long long *out = reinterpret_cast<unsigned long long *>(v.Dflt);
  for (int i = threadIdx.x; i < ti.nk; i += blockDim.x) {
    const int64_t gn = g.node_off + ti.k0 + i;
    out[gn] = v.Dg[gn];
    v.Dg[gn] = 0ull;
  }
}

// Block-wide sum of one double per thread, added to *dst by thread 0.
__device__ void block_add(double x, double *dst) {
  __shared__ double part[32];
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  __syncthreads();  // part[] is free
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += part[w];
    if (t != 0.0) atomicAdd(dst, t);
  }
}

// P passes of (a + 2 b + c) / 4 equal one convolution with the binomial
// weights C(2P, k) / 4^P, k = 0..2P, so each output is formed directly from
// the chunk in shared memory (one barrier per chunk instead of one per
// pass).  coef[k] = C(2P, k) < 2^30 for P <= 16.
//
// FP64 state: doubles, weights C(2P, k) 2^-2P (exact dyadic numbers).
struct SmoothF64 {
  double a[kFilterChunk + 2 * kMaxPasses];
  __device__ void load(int i, unsigned long long bits) { a[i] = __longlong_as_double((long long)bits); }
  __device__ double value(int i, int P, const int *coef, double) const {
    const double inv = ldexp(1.0, -2 * P);
    double s = 0.0;
    for (int k = 0; k <= 2 * P; ++k) s += ((double)coef[k] * inv) * a[i - P + k];
    return s;
  }
};

// FP32 state: the flux is an exact integer, split into a signed high and an
// unsigned low 32-bit word; each is convolved in 64-bit integers (32 x 32 ->
// 64-bit products).  The weights sum to 4^P <= 2^32, so the high sum stays
// within int64 and the low sum within uint64, and the result
// (hi 2^32 + lo) / 4^P is exact until its conversion to double.  (Double
// arithmetic here would run on the FP64 units, a small fraction of the
// integer rate.)
struct SmoothI64 {
  int hi[kFilterChunk + 2 * kMaxPasses];
  unsigned lo[kFilterChunk + 2 * kMaxPasses];
  __device__ void load(int i, unsigned long long bits) {
    hi[i] = (int)((long long)bits >> 32);
    lo[i] = (unsigned)bits;
  }
  __device__ double value(int i, int P, const int *coef, double scale) const {
    long long sh = 0;
    unsigned long long sl = 0;
    for (int k = 0; k <= 2 * P; ++k) {
      sh += (long long)coef[k] * (long long)hi[i - P + k];
      sl += (unsigned long long)(unsigned)coef[k] * (unsigned long long)lo[i - P + k];
    }
    return ((double)sh * 4294967296.0 + (double)sl) * (scale * ldexp(1.0, -2 * P));
  }
};

template <class R>
struct Smoother;
template <>
struct Smoother<double> { using T = SmoothF64; };
template <>
struct Smoother<float> { using T = SmoothI64; };

// A persistent grid: block b smooths the contiguous tiles [t0, t1), so a gap's
// work of j_m reaches the ledger once per block (one address per gap takes
// the atomics of every block on it).
template <class R>
__global__ void __launch_bounds__(256) k_filter_apply(View v, int mode) {
  using S = typename Smoother<R>::T;
  __shared__ S sm;
  __shared__ int coef[2 * kMaxPasses + 1];
  int coef_P = -1;  // passes the weights in coef[] belong to
  const unsigned long long *D0 = reinterpret_cast<const unsigned long long *>(v.Dflt);
  const int t0 = (int)((int64_t)blockIdx.x * v.n_tiles / gridDim.x);
  const int t1 = (int)((int64_t)(blockIdx.x + 1) * v.n_tiles / gridDim.x);
  double work = 0.0;
  int work_gap = -1;
  for (int t = t0; t < t1; ++t) {
    const TileDev ti = v.tiles[t];
    const GapDev &g = v.gaps[ti.gap];
    if (!(mode == 0 ? g.ampere_late : g.defer)) continue;
    const int P = g.filter_passes;  // 0: Ampere alone (a gap with protons)
    if (mode == 0 && ti.gap != work_gap) {  // block-uniform
      if (work_gap >= 0) {
        const GapDev &gw = v.gaps[work_gap];
        block_add(0.5 * work * gw.dt * gw.dx * gw.jm, &v.ledger[work_gap * L_NLED + L_WORK]);
      }
      work = 0.0;
      work_gap = ti.gap;
    }
    const bool periodic = g.periodic != 0;
    const int64_t n = g.nnode;
    const unsigned long long *D = D0 + g.node_off;
    const int ecur = v.ctl->e_cur;
    const double *Eo = v.E[ecur] + g.node_off;
    double *En = v.E[mode == 0 ? ecur ^ 1 : ecur] + g.node_off;
    const double djm = g.dt * g.jm;
    const double scale = sizeof(R) == 4 ? g.w_unit * kPhiUnit : 1.0;
    for (int c0 = 0; c0 < ti.nk; c0 += kFilterChunk) {
      const int len = min(kFilterChunk, ti.nk - c0);
      const int64_t first = (int64_t)ti.k0 + c0 - P;  // node held by position 0
      const int w = len + 2 * P;
      __syncthreads();  // the previous chunk is done with the shared buffers
      if (P != coef_P && threadIdx.x == 0) {  // C(2P, k) by the exact recurrence
        long long c = 1;
        for (int k = 0; k <= 2 * P; ++k) {
          coef[k] = (int)c;
          c = c * (2 * P - k) / (k + 1);
        }
      }
      coef_P = P;
      for (int i = threadIdx.x; i < w; i += blockDim.x) sm.load(i, D[node_source(first + i, n, periodic)]);
      __syncthreads();
      for (int i = threadIdx.x; i < len; i += blockDim.x) {
        const int64_t node = (int64_t)ti.k0 + c0 + i;
        const double sd = sm.value(P + i, P, coef, scale);
        if (mode == 0) {
          const double eo = Eo[node];
          double en = (!periodic && node == 0) ? 0.0 : eo + (djm - sd);
          if (g.em && (periodic || node > 0)) en += v.em_Jv[g.node_off + node];  // dt jv_h (em.cu)
          En[node] = en;
          work += eo + en;
        } else if (periodic || node > 0) {
          En[node] -= sd;
        }
      }
    }
  }
  if (mode == 0 && work_gap >= 0) {
    const GapDev &gw = v.gaps[work_gap];
    block_add(0.5 * work * gw.dt * gw.dx * gw.jm, &v.ledger[work_gap * L_NLED + L_WORK]);
  }
}

void launch_filter(const View &v, int mode, cudaStream_t st) {
  if (!v.filter_any) return;
  const int grid = std::min(v.n_tiles, 148 * 8);
  if (v.precision == GAP_FP32_STATE) {
    k_flux_take<float><<<v.n_tiles, 256, 0, st>>>(v, mode);
    k_filter_apply<float><<<grid, 256, 0, st>>>(v, mode);
  } else {
    k_flux_take<double><<<v.n_tiles, 256, 0, st>>>(v, mode);
    k_filter_apply<double><<<grid, 256, 0, st>>>(v, mode);
  }
}

}  // namespace gapk
