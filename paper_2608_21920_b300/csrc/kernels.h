// kernels.h -- launchers of the device kernels (host-callable, internal).
#pragma once
#include <cuda_runtime.h>

#include "gap_internal.cuh"

namespace gapk {

struct LoadSpec {  // initial load of one gap
  int32_t gap, init, species_count;
  int64_t ppc, n_per_species;
  double density, theta, seed_amp;
};

void launch_step(const View &v, int threads, cudaStream_t st);
void launch_push(const View &v, int threads, cudaStream_t st);
void launch_push_tail(const View &v, cudaStream_t st);
void launch_copy_field(const View &v, int gap, cudaStream_t st);
void launch_after_push(const View &v, cudaStream_t st);
int launches_per_step(const View &v);
void launch_rebin(const View &v, double slack, cudaStream_t st);
void launch_merge(const View &v, cudaStream_t st);
void launch_filter(const View &v, int mode, cudaStream_t st);
void launch_em(const View &v, cudaStream_t st);
void launch_load_protons(const View &v, int gap, int64_t n, cudaStream_t st);
void launch_export_protons(const View &v, int gap, double *stage, int64_t cap, unsigned long long *count,
                           int64_t stride, cudaStream_t st);
void launch_photon_step(const View &v, cudaStream_t st);
void launch_photon_compact(const View &v, cudaStream_t st);
void launch_export_photons(const View &v, int gap, double *stage, int64_t cap, unsigned long long *count,
                           cudaStream_t st);
void launch_import_photons(const View &v, int gap, int64_t n, const double *stage, cudaStream_t st);
void launch_photon_moments(const View &v, int gap, cudaStream_t st);
void launch_force_rebin(const View &v, cudaStream_t st);
void launch_sync_used(const View &v, cudaStream_t st);

void launch_load(const View &v, const LoadSpec *specs_dev, int n_specs, int64_t max_n,
                 cudaStream_t st);
void launch_gauss(const View &v, int set_background, cudaStream_t st);
void launch_spec_inverse(const View &v, const double *U, double *xi, int64_t n, int fp32, cudaStream_t st);
void launch_pair_split(const View &v, const double *chi, const double *U, double *e, int64_t n, cudaStream_t st);
void launch_qspec_inverse(const View &v, const double *chi, const double *U, double *xi, int64_t n, int fp32,
                          cudaStream_t st);
void launch_diag(const View &v, int gap, int64_t nx, int64_t P, cudaStream_t st);
void launch_export_impl(const View &v, int gap, int kind, double *stage, int64_t cap,
                        unsigned long long *count, int n_tiles_gap, cudaStream_t st, int64_t stride = 1,
                        int tile_first = 0);
void launch_import(const View &v, int gap, int kind, int64_t n, const double *stage,
                   cudaStream_t st);
void launch_spectra(const View &v, int gap, int n_tiles_gap, int nbins, double lo, double hi, cudaStream_t st);

}  // namespace gapk
