/*
 * gap.h -- C ABI of the B300 library for the time step of the 1D radiative
 * particle-in-cell model of a pulsar polar-cap pair discharge, and of the
 * batched integrator of the discharge concurrency model with its adjoint.
 *
 * Paper: "Pair Discharges and Radio Emission from Pulsar Magnetospheres".
 *
 * Conventions for every entry point
 *  - Status: 0 (GAP_OK) or a negative GAP_E* code.  The first error is sticky
 *    on a handle; gap_last_error() returns a one-line description.
 *  - Device memory is owned by the caller.  gap_workspace_bytes() says how
 *    much one handle needs; the caller allocates it (for example a torch
 *    uint8 CUDA tensor) and passes the pointer to gap_init().  The library
 *    never calls cudaMalloc/cudaFree.  Host memory of the handle itself is
 *    owned by the library and released by gap_free().
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Calls that return host data synchronise that stream; the
 *    others only enqueue work.
 *  - Pointers named host_* are host memory; pointers named dev_* are device
 *    memory on the current device.
 *
 * Code units (Sect. 2.2): length c/omega_p,co, time 1/omega_p,co, momentum
 * u = gamma beta, density n_co = |eta_co|/e, field m_e c omega_p/e.  In them
 * Gauss reads dE/dx = eta - eta_co and Ampere dE/dt = j_m - J, with
 * eta_co = -1 and j_m = alpha j_co = -alpha (aligned rotator).
 */
#ifndef GAP_H
#define GAP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define GAP_OK 0
#define GAP_EINVAL (-1)   /* bad argument or parameter */
#define GAP_ENOSPACE (-2) /* workspace smaller than gap_workspace_bytes() */
#define GAP_ECAP (-3)     /* particle storage exhausted (cap / capacity) */
#define GAP_ETIMEOUT (-4) /* a bounded device wait gave up */
#define GAP_ECUDA (-5)    /* a CUDA runtime call failed */
#define GAP_ECHECK (-6)   /* a device-side consistency check failed */
#define GAP_ETOOBIG (-7)  /* input larger than a fixed-size internal buffer */

/* precision of the particle state (Sect. 6.1 pushes) */
#define GAP_FP64_PLAIN 0 /* FP64 offsets, momenta, weights; FP64 charge deposit */
#define GAP_FP32_STATE 1 /* FP32 offsets and momenta; exact integer charge deposit; FP64 field */

/* boundaries (Sect. 6.1: star + atmosphere at h = 0, free outflow at the top) */
#define GAP_BC_SURFACE 0
#define GAP_BC_PERIODIC 1

/* initial loads */
#define GAP_INIT_EMPTY 0        /* no particles (use gap_add_particles) */
#define GAP_INIT_COLD 1         /* cold electrons at rest, `density`, ppc per cell */
#define GAP_INIT_PAIR_THERMAL 2 /* e- and e+ at density/2 each, 1D Maxwell-Juttner(theta),
                                   electrons displaced by a Langmuir seed of amplitude seed_amp */
#define GAP_INIT_GAP_PROTONS 3  /* Sect. 6.1 start: cold electrons at `density` everywhere and
                                   protons at the same positions below H_gap (eta = 0 there,
                                   eta_co above): E rises linearly to H_gap.  Needs protons = 1
                                   and a surface gap */

/* particle kinds for gap_get_particles / gap_add_particles */
#define GAP_ELECTRON 0
#define GAP_POSITRON 1
#define GAP_PHOTON 2
#define GAP_PROTON 3 /* export only (gap_get_particles / gap_sample_particles) */

/* Parameters of one gap.  The problem statement of the paper (Sect. 2.2 and
 * 6.1): twist alpha = j_m/j_co, field b = B/B_Q, field-line curvature radius
 * R_curv (as rho_hat = R_curv/d_e), gap height H_gap and density in units of
 * |eta_co|/e.  QED rates follow Sect. 3 (eq. tau_syn, eq. tau_bw) with the
 * Compton wavelength lambda_hat = lambda_C/d_e; rate_mult multiplies both
 * rates (the macro-particle rescaling of Sect. 6.1). */
typedef struct gap_params {
  double alpha;      /* j_m / j_co */
  double b;          /* B / B_Q */
  double lambda_hat; /* reduced Compton wavelength / skin depth */
  double rho_hat;    /* field-line curvature radius / skin depth.  The caller converts
                        the paper's rho_c (cm) to it: rho_c / d_e with the skin depth
                        d_e of Sect. 2.2, or, for boxes too small for the physical
                        value to give pairs, a rescaled value in the spirit of Sect.
                        6.1's rescaling of the QED scales (the workload recipes use
                        rho_hat = 20 rho_c / 1e7 cm) */
  double rate_mult;  /* multiplier of both QED rates (>= 0) */
  double gap_length; /* H_gap in skin depths; QED inhibited above it.  0 -> 0.8 nx dx */
  double density;    /* initial lepton density, units of n_co */
  double dx;         /* cell size (skin depths) */
  double dt;         /* time step (1/omega_p); c dt/dx must be < 0.5 */
  double theta;      /* temperature of GAP_INIT_PAIR_THERMAL (m_e c^2) */
  double seed_amp;   /* Langmuir seed relative density amplitude */
  int64_t nx;        /* cells (>= 8) */
  int64_t ppc;       /* macro-particles per cell per species at load */
  int64_t cap;       /* macro-particle cap (leptons + photons) of this gap; 0 -> none.
                        Over the cap after a step, leptons of the same species,
                        dual cell, direction and ln(gamma) bin (width
                        0.1 * 2^level, level = consecutive over-cap steps, at
                        most 7) are merged in groups of >= 3 into two, keeping
                        weight, momentum, energy and Gauss's law (with the
                        FP32 state a group whose weight exceeds 2^33 - 2
                        units of w0/256 stays unmerged: its children would
                        overflow their 32-bit weights).  The photons born in
                        an over-cap step merge too: those of the same cell,
                        direction and ln(x) bin (the leptons' width) become
                        one photon of the group's weight, energy sum w x and
                        mean position, with a fresh threshold depth.  The
                        paper describes no merging scheme; this one is the
                        library's own. */
  uint64_t seed;     /* Philox4x32-10 key of this gap */
  int32_t qed;       /* 0/1: curvature emission and one-photon pair creation */
  int32_t boundary;  /* GAP_BC_* */
  int32_t init;      /* GAP_INIT_* */
  int32_t kmax_emit; /* emission events per lepton per step (0 -> 16) */
  int32_t kmax_inject; /* injected electrons per step (0 -> 64) */
  int32_t gap_index; /* enters the ids of loaded and injected particles */
  double inject_theta; /* temperature of the surface atmosphere (m_e c^2, Sect. 6.1):
                          injected electrons get |u| of a 1D Maxwell-Juttner draw
                          at this temperature, moving into the gap; 0 -> at rest.
                          In [0, 1e3], else GAP_EINVAL */
  int32_t filter_passes; /* passes of the binomial (1/4, 1/2, 1/4) current filter per
                            step (Sect. 6.1 uses 8); 0 -> none.  Ends of a surface
                            gap: node arrays mirror evenly about the end nodes,
                            cell charge oddly, so Gauss's law holds for the
                            smoothed charge (the Gauss solve and residual use it).
                            In [0, 16] with nx >= 2 passes + 2, else GAP_EINVAL */
  int32_t qed_quantum;   /* 1: the photon energy of an emission follows the quantum
                            spectrum n(xi) ~ (1 - xi + 1/(1 - xi)) K_2/3(d)
                            - int_d^inf K_1/3, d = 2 xi / (3 chi (1 - xi)),
                            xi = x/gamma (Baier & Katkov; Sect. 3.1 leaves the
                            shape open), read from a table of the inverse
                            distribution built at init (relative error of xi
                            about 1e-5; chi above 1e5 uses the chi = 1e5 row);
                            and a converting photon gives the electron e x of
                            its energy x, e from the differential one-photon
                            pair rate (e/(1-e) + (1-e)/e) K_2/3(y)
                            + int_y^inf K_1/3, y = 2 / (3 chi e (1 - e)), at
                            the conversion step's chi (table, Gaussian limit
                            below chi = 1e-3), the positron the rest;
                            0: the classical shape and x/2 each.  0 or 1,
                            else GAP_EINVAL */
  int32_t protons;       /* 1: protons (charge +1, mass m_ion, u their momentum per
                            m_ion c; no QED): the GAP_INIT_GAP_PROTONS start, and
                            the surface also draws protons while cell 0 holds more
                            negative charge than eta_co dx by over half a macro-
                            particle charge (thermal at inject_theta / m_ion).  The
                            gap's Ampere step runs after the push (as with a current
                            filter).  Protons are neither merged nor counted toward
                            the cap.  With the FP32 state the protons keep FP64
                            positions on the state's offset grid (X + 1/2 a multiple
                            of 2^-23), so their charge is exact too */
  double m_ion;          /* proton mass in m_e (0 -> 1836) */
  int32_t em;            /* 1: transverse fields E_y, E_z (cells, half steps) and B_y,
                            B_z (nodes, whole steps) of App. A's co-rotating frame in
                            the 1D reduction: a Yee leapfrog driven by the virtual
                            current jv = -{curl(beta x E) + beta x curl E
                            - curl[beta x (beta x B)]} (particles move along B_*; with
                            jperp they also carry the transverse current of their
                            guiding centres); jv_h joins the Ampere step
                            of E_h and the virtual charge -beta_y dB_z/dh +
                            beta_z dB_y/dh joins Gauss's law.  The star is a
                            conductor.  The gap's Ampere step runs after the push.
                            0 or 1, else GAP_EINVAL */
  int32_t pml_cells;     /* em on a surface gap: an absorbing layer of this many cells
                            below the top (a conductor behind it): matched electric
                            and magnetic conductivity sigma_max ((X - X_p)/pml_cells)^3
                            above X_p = nx - pml_cells (Sect. 6.1: escaping fields are
                            damped).  0 = none (the top is a bare conductor);
                            0 <= pml_cells <= nx/2, else GAP_EINVAL */
  double beta_y, beta_z; /* velocity of the co-rotating frame across h (App. A; the
                            paper's 3e-6); |beta| < 1, zero unless em */
  double pml_sigma;      /* sigma_max in omega_p; 0 -> 4 ln(1e6) / (2 pml_cells dx), a
                            continuum reflection of 1e-6 */
  int32_t jperp;         /* em: 1 adds the particles' transverse current in the
                            guiding-centre limit of the strong field (App. A; Sect.
                            6.6, Fig. 8).  With B_* = b / lambda_hat (omega_B /
                            omega_p in code units) a particle slides along its field
                            line at beta_h and drifts at E x B / B^2: v_y = (beta_h
                            B_y + E_z) / B_*, v_z = (beta_h B_z - E_y) / B_*, with
                            beta_h = u / gamma after the step's kick and emissions
                            and E_perp^{n-1/2}, B_perp^n taken linearly at the start-
                            of-step position, whose unit cloud deposits j_perp =
                            q w v_perp / dx on the cells it covers (inside the gap);
                            dE_perp/dt gains -j_perp.  The particle state keeps u_h
                            alone.  Needs em, b > 0 and lambda_hat > 0; 0 or 1,
                            else GAP_EINVAL */
  int32_t pad0;          /* zero */
} gap_params;

/* Options shared by all gaps of one handle. */
typedef struct gap_config {
  int32_t precision;       /* GAP_FP64_PLAIN or GAP_FP32_STATE */
  int32_t tile;            /* dual cells per tile (>= 8; 0 -> 256) */
  int32_t threads;         /* threads per block of the push kernel (0 -> 256) */
  int32_t rebin_every;     /* steps between store compactions (0 -> 64) */
  int32_t variant;         /* push-kernel variant of the FP32 path without QED:
                              0: 4 leptons/thread, >= 4 blocks/SM; 1: 4, >= 6;
                              2: 2, >= 8; 3: 4, >= 8; 4, 5: TMA bulk-copy
                              pipeline with 3 or 2 stages (the autotuner picks).
                              FP32 path with QED: 0: two passes, the quiet
                              leptons streamed at >= 5 blocks/SM and the
                              leptons that emit within the step or move into
                              another tile pushed by a second kernel from a
                              list (Ampere then follows for every gap); 1: the
                              same at >= 4 blocks/SM; 2-5: every lepton pushed
                              in place.  All variants give the same results */
  int32_t reserved;
  double slack;            /* headroom of each tile segment (0 -> 0.125) */
  int64_t lepton_capacity; /* slots per species over all gaps (0 -> derived) */
  int64_t photon_capacity; /* photon slots (0 -> derived) */
} gap_config;

typedef struct gap_handle gap_handle;

/* Event counters and energy ledger of one gap (cumulative since init).
 * Energies are total energies (rest mass included) per unit area in units of
 * n_co m_e c^2 d_e. */
typedef struct gap_counters {
  int64_t emit_events, photons, pairs, injected, absorbed, escaped, photons_escaped,
      emit_overflow, inject_overflow, load_overflow, spilled, photon_overflow, merged,
      photons_merged, reserved1, reserved2;
  double e_radiated, e_absorbed, e_escaped, e_photon_escaped, e_injected, work_jm,
      reserved3, reserved4;
} gap_counters;

/* Diagnostics of one gap (Sect. 6.2, Fig. 5; Sect. 6.6, Fig. 8). */
typedef struct gap_diag_out {
  int64_t step;
  int64_t n_electrons, n_positrons, n_photons;
  double M_peak;      /* max over gap cells of (n_e- + n_e+)/n_co */
  double M_avg;       /* mean over gap cells */
  int64_t peak_cell;
  double g3_peak;     /* <gamma^-3> at the peak cell */
  double M_split[4];  /* at the peak cell: e- up, e- down, e+ up, e+ down */
  double E_min, E_max;/* over gap nodes */
  double gauss_residual; /* max |(E_{c+1}-E_c) - (Q_c - eta_bg dx)| over interior cells;
                            Q smoothed like the current with a filter, the virtual
                            charge included with em, cells in the absorbing layer left
                            out */
  double E_abs_max;
  double field_energy, lepton_energy, photon_energy;
  int64_t spectrum_len; /* P/2 + 1 entries written to host_spectrum when given */
  gap_counters counters;
} gap_diag_out;

/* Workspace size for n_gaps gaps (params[0..n_gaps-1]) and options cfg
 * (NULL -> defaults).  Returns GAP_EINVAL for inconsistent parameters. */
int gap_workspace_bytes(const gap_params *params, int32_t n_gaps, const gap_config *cfg,
                        size_t *bytes);

/* Lay out the handle in dev_workspace (>= gap_workspace_bytes, 256-byte
 * aligned), load the initial particles, solve Gauss's law for the initial E
 * and build the emission-spectrum tables.  Synchronises `stream`. */
int gap_init(const gap_params *params, int32_t n_gaps, const gap_config *cfg,
             void *dev_workspace, size_t bytes, void *stream, gap_handle **out);

/* Advance every gap by nsteps time steps (Sect. 6.1 cycle: gather, kick,
 * emission, drift, deposit, photon propagation and pair creation, Ampere,
 * surface injection; compaction of the particle store when due).  Enqueues
 * work only; no host synchronisation. */
int gap_step(gap_handle *h, int64_t nsteps, void *stream);

/* Same as gap_step, but replays a CUDA graph of `chunk` steps (captured on
 * first use) for the whole multiples of chunk and launches the remainder
 * directly. */
int gap_step_graph(gap_handle *h, int64_t nsteps, int32_t chunk, void *stream);

/* Diagnostics of gap `gap`.  host_spectrum (may be NULL) receives |E_k|^2/P
 * of E over the gap nodes zero-padded to P = next power of two, P/2+1
 * values; host_moments (may be NULL) receives 8 arrays of nx doubles:
 * density e-up, e-down, e+up, e+down, sum w gamma^-3, sum w, charge, photon
 * density.  Synchronises `stream`. */
int gap_diag(gap_handle *h, int32_t gap, gap_diag_out *out, double *host_spectrum,
             int64_t spectrum_cap, double *host_moments, void *stream);

/* Copy E of gap `gap` (nnode = nx+1 surface, nx periodic values). */
int gap_get_field(gap_handle *h, int32_t gap, double *host_E, int64_t n, void *stream);
int gap_set_field(gap_handle *h, int32_t gap, const double *host_E, int64_t n, void *stream);

/* E of gap `gap` after the steps enqueued on `stream`, copied to host_E
 * (pinned host memory, n >= the gap's node count) on `copy_stream` without a
 * host synchronisation, so that the transfer overlaps the later steps: a
 * kernel on copy_stream, after the work enqueued on `stream`, copies E to a
 * staging buffer of the workspace; `stream` waits for that copy only, not
 * for the transfer; the transfer to host_E then runs on copy_stream.  host_E
 * is complete when copy_stream has passed the call (synchronise it, or an
 * event recorded on it).  A later call reuses the staging buffer after the
 * earlier transfer (both on copy_stream).  The two streams must differ.
 * GAP_EINVAL for a bad gap, buffer or n; device errors surface at the next
 * call that reads the control block (gap_diag, gap_get_field). */
int gap_get_field_async(gap_handle *h, int32_t gap, double *host_E, int64_t n, void *stream, void *copy_stream);

/* Transverse fields of a gap with em = 1 (App. A): component GAP_EM_EY or
   GAP_EM_EZ (nx cell values, at step - 1/2 after `step` steps), GAP_EM_BY or
   GAP_EM_BZ (nnode node values, at the step).  `n` must be at least the
   component's length; a gap without em, a bad component or a short buffer
   returns GAP_EINVAL.  Synchronises the stream.  Setting writes the values the
   next step starts from. */
#define GAP_EM_EY 0
#define GAP_EM_EZ 1
#define GAP_EM_BY 2
#define GAP_EM_BZ 3
int gap_get_em(gap_handle *h, int32_t gap, int32_t component, double *host_dst, int64_t n, void *stream);
int gap_set_em(gap_handle *h, int32_t gap, int32_t component, const double *host_src, int64_t n, void *stream);

/* Export the particles of one kind of one gap, in arbitrary order, as FP64:
 * X is the absolute position in cells, u = gamma beta (photons: x, the
 * energy in m_e c^2, in host_u), w the weight, tau the remaining optical
 * depth (photons: tau_acc in host_tau and tau_star in host_aux).  host_aux
 * may be NULL for leptons; for photons host_aux2 receives dir and birth
 * step packed as (n0 << 1) | (dir > 0).  *n_out = count; GAP_ECAP if cap is
 * too small.  Synchronises `stream`. */
int gap_get_particles(gap_handle *h, int32_t gap, int32_t kind, int64_t cap, uint64_t *host_id,
                      double *host_X, double *host_u, double *host_w, double *host_tau,
                      double *host_aux, int64_t *host_aux2, int64_t *n_out, void *stream);

/* Export the leptons of one species (kind 0 electrons, 1 positrons) of one
 * gap whose id is a multiple of `stride` (>= 1), as gap_get_particles does:
 * a fixed sample of a large gap that stays the same from step to step (ids
 * do not change when leptons move between tiles or the store is compacted).
 * GAP_EINVAL for photons or stride < 1.  Synchronises `stream`. */
int gap_sample_particles(gap_handle *h, int32_t gap, int32_t kind, int64_t stride, int64_t cap,
                         uint64_t *host_id, double *host_X, double *host_u, double *host_w, double *host_tau,
                         int64_t *n_out, void *stream);

/* Spectra of gap `gap` (Sect. 6.4, Fig. 6: the momentum distribution of the
 * pair plasma over h in [0, H_gap] and the photon energy spectrum): the total
 * weight (real particles per unit area, n_co d_e units) of the electrons
 * (host_leptons[0 .. nbins)), the positrons (host_leptons[nbins .. 2 nbins))
 * and the photons (host_photons[0 .. nbins)) with position below H_gap, per
 * bin of ln p (p = |u| = gamma beta) or ln x (photons): nbins uniform bins
 * over [lo, hi), values below lo (p = 0 included) counted in the first bin,
 * values at or above hi in the last.  Leptons spilled since the last
 * compaction (counter `spilled`) are left out.  1 <= nbins <= 1024 and
 * hi > lo, else GAP_EINVAL.  Either output may be NULL.  Synchronises
 * `stream`. */
int gap_spectra(gap_handle *h, int32_t gap, int32_t nbins, double lo, double hi, double *host_leptons,
                double *host_photons, void *stream);

/* Return flux of gap `gap` (Sect. 6.5, Fig. 7: the pairs that fall back onto
 * the star and heat its atmosphere): the total weight of the electrons and
 * positrons absorbed at h < 0 since gap_init, per bin of ln gamma at
 * absorption: host_out[i] holds 10^(i/8) <= gamma < 10^((i+1)/8) for
 * i < GAP_RETURN_BINS - 1, the last bin every gamma above.  Protons are not
 * tallied.  Synchronises `stream`. */
#define GAP_RETURN_BINS 64
int gap_return_spectrum(gap_handle *h, int32_t gap, double *host_out, void *stream);

/* Export the leptons of one species (kind 0 electrons, 1 positrons) stored
 * in tiles [tile_lo, tile_hi) of gap `gap` (tile i holds the leptons whose
 * dual cell k = floor(X + 1/2) lies in [i tile, (i + 1) tile), tile the
 * configuration's tile size), as gap_get_particles does: a window of a large
 * gap, complete, with which the charge-conserving deposit and the Ampere
 * step of Sect. 6.1 (Sect. 2.2, dE/dt = j_m - J) can be recomputed on the
 * window's nodes.  Leptons spilled since the last compaction (counter
 * `spilled`) are not in their tiles' segments and are left out.
 * GAP_EINVAL for photons, protons or an empty or out-of-range tile range;
 * GAP_ECAP if cap is too small (*n_out is the count).  Synchronises `stream`. */
int gap_tile_particles(gap_handle *h, int32_t gap, int32_t kind, int32_t tile_lo, int32_t tile_hi, int64_t cap,
                       uint64_t *host_id, double *host_X, double *host_u, double *host_w, double *host_tau,
                       int64_t *n_out, void *stream);

/* Append n particles of one kind to gap `gap` (tests build hand-checkable
 * states).  Photons: host_u is x, host_tau is tau_star, host_aux2 packs
 * (n0 << 1) | (dir > 0).  In a handle without QED and without a cap
 * every lepton carries the uniform weight w0 = density dx / ppc (host_w is
 * not used) and no optical depth; otherwise weights are stored (FP32 state:
 * rounded to multiples of w0 / 256).  Synchronises `stream`. */
int gap_add_particles(gap_handle *h, int32_t gap, int32_t kind, int64_t n, const uint64_t *host_id,
                      const double *host_X, const double *host_u, const double *host_w,
                      const double *host_tau, const int64_t *host_aux2, void *stream);

/* Recompute E of every gap from Gauss's law (Sect. 2.2): E_0 = 0 at the
 * surface, zero mean for periodic gaps; the periodic background eta_bg is
 * set to the mean charge density when set_background is nonzero.  The
 * virtual charge of a gap with em (its B_y, B_z term) is not included: it is
 * zero while the transverse B is, as at the start. */
int gap_solve_gauss(gap_handle *h, int32_t set_background, void *stream);

/* Override the Gauss background eta_bg of a gap (default: -1 at a surface). */
int gap_set_background(gap_handle *h, int32_t gap, double eta_bg);

/* The inverse CDF of the classical curvature-photon spectrum used by the
 * emission sampler (reading of the unspecified S(gamma, x) of Sect. 3.1:
 * dN/dxi proportional to F(xi)/xi, F(xi) = xi int_xi^inf K_5/3): for each
 * uniform U in (0,1] of dev_U, dev_xi receives the xi with P(xi' > xi) = U,
 * as the FP64 path (precision GAP_FP64_PLAIN: table and Newton steps on the
 * quadrature) or the FP32 path (GAP_FP32_STATE: table only) evaluates it.
 * n doubles each, device memory; enqueues work only. */
int gap_spectrum_inverse(gap_handle *h, const double *dev_U, double *dev_xi, int64_t n, int32_t precision,
                         void *stream);

/* Power spectrum of a field without allocating anything.  (The paper has no
 * counterpart: this is a library facility.)  For callers that cannot
 * allocate device memory -- a fixed budget handed out at start-up, a host
 * runtime that owns the allocator, or code that must not add an allocation
 * and its implicit synchronisation between launches -- this computes the
 * same |E_k|^2/P as gap_diag's spectrum (E zero-padded to P = the next power
 * of two >= n, P/2+1 values written to dev_power) using only the caller's
 * buffers and a fixed working array inside the library.
 *  - n <= 32768 (P <= 2^15); larger n returns GAP_ETOOBIG.
 *  - dev_E: n doubles, dev_power: P/2+1 doubles, both device memory of the
 *    current device; the call enqueues work on `stream` and returns.
 *  - The working array (1 MiB) is a file-scope device array that every GPU
 *    loading the library holds until the process exits.  The first call on a
 *    device looks its address up (cudaGetSymbolAddress) with that device
 *    current; make that first call before any stream capture.  The address
 *    is kept for the life of the process: after cudaDeviceReset (or anything
 *    else that destroys the device's context) the module may load elsewhere,
 *    so do not call this entry point on that device again in the same
 *    process.
 *  - All calls share the array: calls that overlap on the GPU (for example on
 *    two streams) race; serialise them.  Each call rewrites every entry it
 *    reads, so no state carries over between calls.
 *  - Calls no cudaMalloc, cudaFree or allocating library routine. */
int gap_power_spectrum_noalloc(const double *dev_E, int64_t n, double *dev_power, void *stream);

/* Steps taken so far (host mirror). */
int64_t gap_steps_done(const gap_handle *h);

/* Live timing of the push kernel (the dominant kernel of a step).  With
 * on != 0, later gap_step calls bracket each phase of the step (the push
 * launch among them) with CUDA events on the launching stream.  Every call first returns, through the non-NULL
 * outputs, the summed push duration (ms) and the number of push launches
 * timed since the previous call (synchronising on the last event), and the
 * number of kernel launches one step makes; then it resets the sums and sets
 * the mode.  Graph replays are not timed. */
int gap_profile(gap_handle *h, int32_t on, double *push_ms_total, int64_t *push_launches,
                int64_t *launches_per_step);

/* Phases of a profiled step (gap_profile_phases). */
#define GAP_PHASE_PUSH 0   /* the streaming push kernel (with its item list): gather, kick,
                              emission, drift, deposit, and Ampere where it is fused */
#define GAP_PHASE_AFTER 1  /* photon propagation and conversion, injection, bookkeeping */
#define GAP_PHASE_REBIN 2  /* store compaction (a no-op launch sequence between re-bins) */
#define GAP_PHASE_MERGE 3  /* the over-cap check and merge */
#define GAP_PHASE_PUSH_TAIL 4 /* after the streaming push: the second pass of the two-pass
                              QED push, protons, transverse fields, Ampere of the gaps
                              that leave it to a separate kernel */
#define GAP_NPHASES 5

/* Durations (ms) of each phase summed over the steps profiled since the last
 * gap_profile call (which clears them), without clearing; ms_out holds
 * GAP_NPHASES values, *steps_out the number of profiled steps.  Synchronises
 * on the last recorded event.  The mode is switched by gap_profile. */
int gap_profile_phases(gap_handle *h, double *ms_out, int64_t *steps_out);

/* Test hook for the timeout path of the bulk-copy push variants (config
 * variant 4 or 5): with on != 0, later push launches leave the first copy
 * stage of every tile unissued and poll its barrier only 2^14 times, so the
 * wait runs out; the kernel records the failure and returns, the next call
 * that reads the control block returns GAP_ETIMEOUT, and the GPU context
 * stays usable.  The handle's state is then invalid and the handle is to be
 * freed.  For tests of error handling only; other variants ignore it. */
int gap_hold_copies(gap_handle *h, int32_t on);

/* Test hook for the overflow path of the two-pass FP32 QED push (variants 0
 * and 1): the push's list of deferred leptons (leptons that moved into
 * another tile in its first half, emitters in its second; sized for an
 * eighth of the lepton slots) is used up to n entries (n/2 per half) in the
 * later steps; the leptons that do not fit are found in the store by a third
 * kernel, with the same results.  n is clamped to the list's size;
 * GAP_EINVAL for n < 0.  The value is a launch parameter: steps replayed
 * from CUDA graphs captured earlier keep the old one. */
int gap_defer_limit(gap_handle *h, int64_t n);

/* Checkpoint and resume.  A handle's whole state (particles, photons and
 * their schedules, E, counters, ledgers, step number) lives in its
 * workspace and holds no device addresses, so gap_save copies the
 * gap_state_bytes(h) bytes in use to host memory and gap_load copies such a
 * state into a handle made with the same parameters and configuration (any
 * workspace address): stepping on continues exactly as the saved handle
 * would (the random draws are keyed by particle id and step, with no
 * generator state).  gap_load returns GAP_EINVAL, copying nothing, for a
 * state of another layout or size; it clears an error status of the handle
 * and returns that of the loaded state.  Both synchronise `stream`. */
size_t gap_state_bytes(const gap_handle *h);
int gap_save(gap_handle *h, void *host_dst, size_t bytes, void *stream);
int gap_load(gap_handle *h, const void *host_src, size_t bytes, void *stream);

/* Release host state.  The caller frees the workspace afterwards. */
void gap_free(gap_handle *h);

const char *gap_last_error(const gap_handle *h);
const char *gap_status_string(int status);

/* The photon energy fraction xi in (0, 1) of the quantum spectrum for
 * emission parameter chi and draw U in (0, 1] (n values, device arrays; the
 * inverse the emissions of qed_quantum gaps use), in the FP64 (precision =
 * GAP_FP64_PLAIN) or the FP32 (GAP_FP32_STATE) evaluation.  GAP_EINVAL when
 * no gap of the handle has qed_quantum.  Enqueued on `stream`. */
int gap_qspectrum_inverse(gap_handle *h, const double *dev_chi, const double *dev_U, double *dev_xi, int64_t n,
                          int32_t precision, void *stream);

/* The electron's fraction e of a converting photon's energy for
 * conversion parameter chi and draw U in (0, 1] (n values, device arrays;
 * the split of qed_quantum gaps, FP64).  GAP_EINVAL when no gap of the
 * handle has qed_quantum.  Enqueued on `stream`. */
int gap_pair_split(gap_handle *h, const double *dev_chi, const double *dev_U, double *dev_e, int64_t n,
                   void *stream);

/* ------------------------------------------------------------------------
 * Concurrency model (Sect. 5.2, eq. dis1-dis4) -- batched RK4 integrator
 * with a hand-written discrete adjoint.
 *
 * State y = (m_pm, m_x, eps, j), parameters p = (alpha, t_x, t_pm, t_acc, g3)
 * in units of t_esc = 1.  The gate H(|eps| - 1) is the Heaviside step when
 * delta == 0 and the smoothed (1 + tanh(z/delta))/2 otherwise.
 * Layouts (row-major, device memory):
 *   dev_p   [B][5], dev_y0 [B][4], dev_dt [B] (per-set step size),
 *   dev_out [T][B][4] states at steps 0, every, 2*every, ... (T = nsteps/every + 1),
 *   dev_ckpt [nsteps/ckpt_every + 1][B][4] checkpoints kept for the adjoint.
 * Precision: dtype 0 = FP64, 1 = FP32 (all arrays of that type).
 * ------------------------------------------------------------------------ */
int ode_forward(const void *dev_p, const void *dev_y0, const void *dev_dt, int32_t B, int32_t nsteps,
                int32_t every, int32_t ckpt_every, double delta, int32_t dtype, void *dev_out,
                void *dev_ckpt, void *stream);

/* Given dL/d(out) in dev_gout [T][B][4], accumulate dL/dp into dev_gp [B][5]
 * and dL/dy0 into dev_gy0 [B][4] (both overwritten) by the discrete adjoint
 * of the same RK4 steps, recomputing each checkpoint segment forward.
 * dev_scratch holds ckpt_every+1 states per set: (ckpt_every+1)*B*4 values. */
int ode_adjoint(const void *dev_p, const void *dev_dt, const void *dev_ckpt, const void *dev_gout,
                int32_t B, int32_t nsteps, int32_t every, int32_t ckpt_every, double delta,
                int32_t dtype, void *dev_gp, void *dev_gy0, void *dev_scratch, void *stream);

/* ------------------------------------------------------------------------
 * Extended concurrency model: the plasma-inertia measure <gamma^-3> as a
 * state (Sect. 5.2 says the paper solved such a moment expansion of the 1D
 * Vlasov equation without giving it; this one is the library's reading, in
 * the paper's approximations).  State y = (m_pm, m_x, eps, j, G) with
 * G = m_pm <gamma^-3>; parameters p = (alpha, t_x, t_pm, t_acc, gamma_min,
 * gamma_rad), units t_esc = 1:
 *   dm_pm/dt, dm_x/dt, deps/dt as in eq. dis1-dis3,
 *   dj/dt = -j + eps G / t_acc                                  (eq. dis4)
 *   dG/dt = 2 gamma_min^-3 m_x / t_pm                  (pairs born at gamma_min,
 *                                                      eq. gam_inj)
 *         - G                                          (escape)
 *         - 3 eps j (G/m_pm)^(4/3) / t_acc             (field work on cold
 *                                                      streams: <gamma^-4 q beta>
 *                                                      = <gamma^-3>^(4/3) j/m_pm)
 *         + 3 m_pm / (gamma_rad^4 t_acc)               (curvature losses,
 *                                                      eq. dgamma_curv, balanced
 *                                                      at gamma_rad, eq. gam_rad)
 * (G/m)^(4/3) of max(G, 0).  Layouts as for ode_forward / ode_adjoint with
 * 5 state and 6 parameter entries per set: dev_p [B][6], dev_y0 [B][5],
 * dev_out [T][B][5], dev_ckpt [nsteps/ckpt_every + 1][B][5], dev_gp [B][6],
 * dev_gy0 [B][5], dev_scratch (ckpt_every+1)*B*5 values.  The term in
 * (G/m)^(4/3) makes the system stiff where t_acc is small: the step must
 * resolve 3 eps (j/m) (G/m)^(1/3) / t_acc.
 * ------------------------------------------------------------------------ */
int ode_ext_forward(const void *dev_p, const void *dev_y0, const void *dev_dt, int32_t B, int32_t nsteps,
                    int32_t every, int32_t ckpt_every, double delta, int32_t dtype, void *dev_out,
                    void *dev_ckpt, void *stream);
int ode_ext_adjoint(const void *dev_p, const void *dev_dt, const void *dev_ckpt, const void *dev_gout,
                    int32_t B, int32_t nsteps, int32_t every, int32_t ckpt_every, double delta,
                    int32_t dtype, void *dev_gp, void *dev_gy0, void *dev_scratch, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* GAP_H */
