// spectrum_noalloc.cu -- power spectrum |E_k|^2 / P of a field with no device
// allocation at all, for callers that cannot allocate device memory.
//
// Some callers have no way to obtain device memory: code running inside a
// fixed memory budget handed out once at start-up, plugins hosted by another
// runtime that owns the allocator, or callers that must not introduce an
// allocation (and its implicit synchronisation) between two launches.  This
// entry point needs only the caller's input and output buffers; its working
// storage is the file-scope array below, which every GPU that loads the
// library holds until the process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "../../include/gap.h"

namespace {

constexpr int64_t kMaxLen = 1 << 15;  // largest transform length P (power of two)
constexpr int kMaxDevices = 64;

// Two ping-pong buffers of kMaxLen complex doubles: 1 MiB per device.
static __device__ __align__(256) double2 g_noalloc_scratch[2 * kMaxLen];

// Host-side copy of the array's device address, obtained once per device
// with that device current (the array's name in host code is only a
// host-side stand-in for the symbol, not a device address).
double2 *g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

int scratch_for_current_device(double2 **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GAP_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return GAP_EINVAL;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return GAP_ECUDA;
    g_scratch_addr[dev] = static_cast<double2 *>(p);
  }
  *out = g_scratch_addr[dev];
  return GAP_OK;
}

// Copy E (n values) into the first buffer, zero-padded to P: every entry the
// transform reads is written here, so nothing left by a previous call leaks in.
__global__ void k_noalloc_fill(const double *E, int64_t n, double2 *buf, int64_t P) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P;
       i += (int64_t)gridDim.x * blockDim.x)
    buf[i] = make_double2(i < n ? E[i] : 0.0, 0.0);
}

// Radix-2 self-sorting (Stockham) stage: for p < n/2, q < s,
// y[q + s 2p] = a + b, y[q + s (2p + 1)] = (a - b) exp(-2 pi i p / n),
// with a = x[q + s p], b = x[q + s (p + n/2)].
__global__ void k_noalloc_stage(const double2 *x, double2 *y, int64_t n, int64_t s, int64_t P) {
  const int64_t m = n / 2;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < P / 2;
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

__global__ void k_noalloc_power(const double2 *X, double *out, int64_t P) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i <= P / 2;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (X[i].x * X[i].x + X[i].y * X[i].y) / (double)P;
}

}  // namespace

extern "C" int gap_power_spectrum_noalloc(const double *dev_E, int64_t n, double *dev_power, void *stream) {
  if (!dev_E || !dev_power || n < 1) return GAP_EINVAL;
  int64_t P = 1;
  while (P < n) P <<= 1;
  if (P > kMaxLen) return GAP_ETOOBIG;
  double2 *a = nullptr;
  const int r = scratch_for_current_device(&a);
  if (r != GAP_OK) return r;
  double2 *b = a + kMaxLen;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t work = P / 2 + 1;
  const int blocks = (int)((work + 255) / 256);
  k_noalloc_fill<<<blocks, 256, 0, st>>>(dev_E, n, a, P);
  int64_t s = 1;
  for (int64_t len = P; len > 1; len /= 2) {
    k_noalloc_stage<<<blocks, 256, 0, st>>>(a, b, len, s, P);
    double2 *t = a;
    a = b;
    b = t;
    s *= 2;
  }
  k_noalloc_power<<<blocks, 256, 0, st>>>(a, dev_power, P);
  return cudaGetLastError() == cudaSuccess ? GAP_OK : GAP_ECUDA;
}
