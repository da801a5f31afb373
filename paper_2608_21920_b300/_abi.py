"""ctypes declarations of include/gap.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
SO_PATH = os.path.join(HERE, "libgap.so")

GAP_OK, GAP_EINVAL, GAP_ENOSPACE, GAP_ECAP, GAP_ETIMEOUT, GAP_ECUDA, GAP_ECHECK, GAP_ETOOBIG = 0, -1, -2, -3, -4, -5, -6, -7
GAP_FP64_PLAIN, GAP_FP32_STATE = 0, 1
GAP_BC_SURFACE, GAP_BC_PERIODIC = 0, 1
GAP_INIT_EMPTY, GAP_INIT_COLD, GAP_INIT_PAIR_THERMAL, GAP_INIT_GAP_PROTONS = 0, 1, 2, 3
GAP_ELECTRON, GAP_POSITRON, GAP_PHOTON, GAP_PROTON = 0, 1, 2, 3
GAP_EM_EY, GAP_EM_EZ, GAP_EM_BY, GAP_EM_BZ = 0, 1, 2, 3
GAP_RETURN_BINS = 64


class GapParams(C.Structure):
    _fields_ = [
        ("alpha", C.c_double), ("b", C.c_double), ("lambda_hat", C.c_double),
        ("rho_hat", C.c_double), ("rate_mult", C.c_double), ("gap_length", C.c_double),
        ("density", C.c_double), ("dx", C.c_double), ("dt", C.c_double),
        ("theta", C.c_double), ("seed_amp", C.c_double),
        ("nx", C.c_int64), ("ppc", C.c_int64), ("cap", C.c_int64), ("seed", C.c_uint64),
        ("qed", C.c_int32), ("boundary", C.c_int32), ("init", C.c_int32),
        ("kmax_emit", C.c_int32), ("kmax_inject", C.c_int32), ("gap_index", C.c_int32),
        ("inject_theta", C.c_double), ("filter_passes", C.c_int32), ("qed_quantum", C.c_int32),
        ("protons", C.c_int32), ("m_ion", C.c_double),
        ("em", C.c_int32), ("pml_cells", C.c_int32), ("beta_y", C.c_double), ("beta_z", C.c_double),
        ("pml_sigma", C.c_double), ("jperp", C.c_int32), ("pad0", C.c_int32),
    ]


class GapConfig(C.Structure):
    _fields_ = [
        ("precision", C.c_int32), ("tile", C.c_int32), ("threads", C.c_int32),
        ("rebin_every", C.c_int32), ("variant", C.c_int32), ("reserved", C.c_int32),
        ("slack", C.c_double),
        ("lepton_capacity", C.c_int64), ("photon_capacity", C.c_int64),
    ]


class GapCounters(C.Structure):
    _fields_ = [(n, C.c_int64) for n in (
        "emit_events", "photons", "pairs", "injected", "absorbed", "escaped", "photons_escaped",
        "emit_overflow", "inject_overflow", "load_overflow", "spilled", "photon_overflow", "merged",
        "photons_merged", "reserved1", "reserved2")] + [(n, C.c_double) for n in (
            "e_radiated", "e_absorbed", "e_escaped", "e_photon_escaped", "e_injected", "work_jm",
            "reserved3", "reserved4")]


class GapDiagOut(C.Structure):
    _fields_ = [
        ("step", C.c_int64), ("n_electrons", C.c_int64), ("n_positrons", C.c_int64),
        ("n_photons", C.c_int64), ("M_peak", C.c_double), ("M_avg", C.c_double),
        ("peak_cell", C.c_int64), ("g3_peak", C.c_double), ("M_split", C.c_double * 4),
        ("E_min", C.c_double), ("E_max", C.c_double), ("gauss_residual", C.c_double),
        ("E_abs_max", C.c_double), ("field_energy", C.c_double), ("lepton_energy", C.c_double),
        ("photon_energy", C.c_double), ("spectrum_len", C.c_int64), ("counters", GapCounters),
    ]


_lib = None


def lib():
    """Load libgap.so.  Raises if the CUDA library has not been built: there is
    no CPU fallback."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(SO_PATH):
        raise RuntimeError(f"CUDA library missing: {SO_PATH} (run paper_2608_21920_b300/build.py)")
    L = C.CDLL(SO_PATH)
    vp, i32, i64, d, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_size_t
    PP, PC = C.POINTER(GapParams), C.POINTER(GapConfig)
    L.gap_workspace_bytes.argtypes = [PP, i32, PC, C.POINTER(sz)]
    L.gap_init.argtypes = [PP, i32, PC, vp, sz, vp, C.POINTER(vp)]
    L.gap_step.argtypes = [vp, i64, vp]
    L.gap_step_graph.argtypes = [vp, i64, i32, vp]
    L.gap_diag.argtypes = [vp, i32, C.POINTER(GapDiagOut), vp, i64, vp, vp]
    L.gap_get_field.argtypes = [vp, i32, vp, i64, vp]
    L.gap_set_field.argtypes = [vp, i32, vp, i64, vp]
    L.gap_get_em.argtypes = [vp, i32, i32, vp, i64, vp]
    L.gap_set_em.argtypes = [vp, i32, i32, vp, i64, vp]
    L.gap_get_particles.argtypes = [vp, i32, i32, i64, vp, vp, vp, vp, vp, vp, vp, C.POINTER(i64), vp]
    L.gap_sample_particles.argtypes = [vp, i32, i32, i64, i64, vp, vp, vp, vp, vp, C.POINTER(i64), vp]
    L.gap_tile_particles.argtypes = [vp, i32, i32, i32, i32, i64, vp, vp, vp, vp, vp, C.POINTER(i64), vp]
    L.gap_spectra.argtypes = [vp, i32, i32, d, d, vp, vp, vp]
    L.gap_return_spectrum.argtypes = [vp, i32, vp, vp]
    L.gap_add_particles.argtypes = [vp, i32, i32, i64, vp, vp, vp, vp, vp, vp, vp]
    L.gap_solve_gauss.argtypes = [vp, i32, vp]
    L.gap_set_background.argtypes = [vp, i32, d]
    L.gap_steps_done.argtypes = [vp]
    L.gap_steps_done.restype = i64
    L.gap_spectrum_inverse.argtypes = [vp, vp, vp, i64, i32, vp]
    L.gap_qspectrum_inverse.argtypes = [vp, vp, vp, vp, i64, i32, vp]
    L.gap_pair_split.argtypes = [vp, vp, vp, vp, i64, vp]
    L.gap_power_spectrum_noalloc.argtypes = [vp, i64, vp, vp]
    L.gap_profile.argtypes = [vp, i32, C.POINTER(d), C.POINTER(i64), C.POINTER(i64)]
    L.gap_profile_phases.argtypes = [vp, C.POINTER(d), C.POINTER(i64)]
    L.gap_hold_copies.argtypes = [vp, i32]
    L.gap_defer_limit.argtypes = [vp, i64]
    L.gap_get_field_async.argtypes = [vp, i32, vp, i64, vp, vp]
    L.gap_state_bytes.argtypes = [vp]
    L.gap_state_bytes.restype = sz
    L.gap_save.argtypes = [vp, vp, sz, vp]
    L.gap_load.argtypes = [vp, vp, sz, vp]
    L.gap_free.argtypes = [vp]
    L.gap_free.restype = None
    L.gap_last_error.argtypes = [vp]
    L.gap_last_error.restype = C.c_char_p
    L.gap_status_string.argtypes = [C.c_int]
    L.gap_status_string.restype = C.c_char_p
    L.ode_forward.argtypes = [vp, vp, vp, i32, i32, i32, i32, d, i32, vp, vp, vp]
    L.ode_adjoint.argtypes = [vp, vp, vp, vp, i32, i32, i32, i32, d, i32, vp, vp, vp, vp]
    L.ode_ext_forward.argtypes = [vp, vp, vp, i32, i32, i32, i32, d, i32, vp, vp, vp]
    L.ode_ext_adjoint.argtypes = [vp, vp, vp, vp, i32, i32, i32, i32, d, i32, vp, vp, vp, vp]
    _lib = L
    return L


EXPORTED = ["gap_workspace_bytes", "gap_init", "gap_step", "gap_step_graph", "gap_diag",
            "gap_get_field", "gap_set_field", "gap_get_em", "gap_set_em", "gap_get_particles", "gap_sample_particles", "gap_tile_particles", "gap_spectra", "gap_return_spectrum", "gap_add_particles",
            "gap_solve_gauss", "gap_set_background", "gap_steps_done", "gap_profile", "gap_profile_phases", "gap_hold_copies", "gap_defer_limit", "gap_get_field_async", "gap_state_bytes", "gap_save", "gap_load", "gap_spectrum_inverse", "gap_qspectrum_inverse", "gap_pair_split", "gap_power_spectrum_noalloc", "gap_free",
            "gap_last_error", "gap_status_string", "ode_forward", "ode_adjoint", "ode_ext_forward", "ode_ext_adjoint"]


class GapError(RuntimeError):
    pass


def check(status, handle=None, what=""):
    if status == GAP_OK:
        return
    L = lib()
    msg = L.gap_status_string(status).decode()
    if handle:
        detail = L.gap_last_error(handle).decode()
        if detail:
            msg += f" ({detail})"
    raise GapError(f"{what}: {msg}")
