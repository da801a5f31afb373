// filter.cu -- the binomial current filter (Sect. 6.1: the current is
// smoothed by a 3-point binomial filter, 8 passes per step).
//
//   k_flux_take     the node flux a step (or a merge) left in the global
//                   accumulators -> doubles; the accumulators are zeroed
//   k_filter_apply  P passes of (1/4, 1/2, 1/4) in shared memory over chunks
//                   of a tile's nodes with P-node halos, then Ampere
//                   E^{n+1} = E^n + (dt j_m - S D) (mode 0) or the merge's
//                   re-centring correction E -= S F (mode 1)
//
// Values beyond the ends of a node array: a periodic gap wraps; a surface gap
// mirrors evenly about nodes 0 and nx.  The cell charge of the Gauss solve
// and residual is mirrored oddly about the same nodes (init.cu), the pairing
// under which smoothing commutes with the node-to-cell difference, so Gauss's
// law holds for the smoothed charge.  Both kernels touch only gaps with
// filter_passes > 0; one block per tile, and the tiles of a gap cover its
// nodes k0 .. k0 + nk - 1 without overlap.
#include "gap_internal.cuh"
#include "kernels.h"

namespace gapk {

constexpr int kFilterChunk = 1024;  // nodes smoothed per shared-memory round
constexpr int kMaxPasses = 16;      // upper bound of filter_passes (checked at init)

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

template <class R>
__global__ void k_flux_take(View v) {
  using Acc = typename Prec<R>::Acc;
  const TileDev ti = v.tiles[blockIdx.x];
  const GapDev &g = v.gaps[ti.gap];
  if (g.filter_passes <= 0) return;
  const double scale = sizeof(R) == 4 ? g.w_unit * kPhiUnit : 1.0;
  for (int i = threadIdx.x; i < ti.nk; i += blockDim.x) {
    const int64_t gn = g.node_off + ti.k0 + i;
    v.Dflt[gn] = acc_take(&v.Dg[gn], (Acc *)nullptr) * scale;
  }
}

__global__ void __launch_bounds__(256) k_filter_apply(View v, int mode) {
  __shared__ double sa[kFilterChunk + 2 * kMaxPasses], sb[kFilterChunk + 2 * kMaxPasses];
  const TileDev ti = v.tiles[blockIdx.x];
  const GapDev &g = v.gaps[ti.gap];
  const int P = g.filter_passes;
  if (P <= 0) return;
  const bool periodic = g.periodic != 0;
  const int64_t n = g.nnode;
  const double *D = v.Dflt + g.node_off;
  const int ecur = v.ctl->e_cur;
  const double *Eo = v.E[ecur] + g.node_off;
  double *En = v.E[mode == 0 ? ecur ^ 1 : ecur] + g.node_off;
  const double djm = g.dt * g.jm;
  double work = 0.0;
  for (int c0 = 0; c0 < ti.nk; c0 += kFilterChunk) {
    const int len = min(kFilterChunk, ti.nk - c0);
    const int64_t first = (int64_t)ti.k0 + c0 - P;  // node held by sa[0]
    const int w = len + 2 * P;
    __syncthreads();  // the previous chunk is done with sa / sb
    for (int i = threadIdx.x; i < w; i += blockDim.x) sa[i] = D[node_source(first + i, n, periodic)];
    __syncthreads();
    double *a = sa, *b = sb;
    for (int p = 1; p <= P; ++p) {  // pass p is valid on [p, w - p)
      for (int i = p + threadIdx.x; i < w - p; i += blockDim.x) b[i] = 0.25 * (a[i - 1] + 2.0 * a[i] + a[i + 1]);
      __syncthreads();
      double *t = a;
      a = b;
      b = t;
    }
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
      const int64_t node = (int64_t)ti.k0 + c0 + i;
      const double sd = a[P + i];
      if (mode == 0) {
        const double eo = Eo[node];
        const double en = (!periodic && node == 0) ? 0.0 : eo + (djm - sd);
        En[node] = en;
        work += eo + en;
      } else if (periodic || node > 0) {
        En[node] -= sd;
      }
    }
  }
  if (mode == 0) {
    for (int o = 16; o > 0; o >>= 1) work += __shfl_down_sync(0xffffffffu, work, o);
    if ((threadIdx.x & 31) == 0 && work != 0.0)
      atomicAdd(&v.ledger[ti.gap * L_NLED + L_WORK], 0.5 * work * g.dt * g.dx * g.jm);
  }
}

void launch_filter(const View &v, int mode, cudaStream_t st) {
  if (!v.filter_any) return;
  if (v.precision == GAP_FP32_STATE) k_flux_take<float><<<v.n_tiles, 256, 0, st>>>(v);
  else k_flux_take<double><<<v.n_tiles, 256, 0, st>>>(v);
  k_filter_apply<<<v.n_tiles, 256, 0, st>>>(v, mode);
}

}  // namespace gapk
