"""FP64 CPU oracle of the 1D radiative PIC discharge step, plus the FP64
reference integrator of the concurrency model (Sect. 5.2, eq. dis1-dis4).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product library never calls it and shares no code with it.

The PIC oracle is plain C (``gap_oracle.c``), built by :func:`build` into
``liboracle.so`` next to this file and loaded through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_SRC = os.path.join(_HERE, "gap_oracle.c")

BC_SURFACE, BC_PERIODIC = 0, 1
INIT_EMPTY, INIT_COLD, INIT_PAIR_THERMAL, INIT_GAP_PROTONS = 0, 1, 2, 3
ALPHA_EM = 7.2973525693e-3
PHOTON_BIT = 1 << 63
CH_INIT_U, CH_TAU0, CH_EMIT_X, CH_EMIT_TAU, CH_BW_TAU, CH_INJECT, CH_PAIR, CH_PHOTON, CH_MERGE = (
    1, 3, 4, 5, 6, 7, 8, 9, 10)


def build(force: bool = False) -> str:
    """Compile the C oracle (plain FP64, no fast-math) into liboracle.so."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fPIC", "-shared",
               "-std=c11", "-D_DEFAULT_SOURCE", "-o", _SO, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _SO


class Params(C.Structure):
    _fields_ = [
        ("alpha", C.c_double), ("b", C.c_double), ("lambda_hat", C.c_double),
        ("rho_hat", C.c_double), ("rate_mult", C.c_double), ("gap_length", C.c_double),
        ("density", C.c_double), ("dx", C.c_double), ("dt", C.c_double),
        ("theta", C.c_double), ("seed_amp", C.c_double),
        ("nx", C.c_int64), ("ppc", C.c_int64), ("cap", C.c_int64), ("seed", C.c_uint64),
        ("gap_index", C.c_int32), ("qed", C.c_int32), ("boundary", C.c_int32),
        ("init", C.c_int32), ("kmax_emit", C.c_int32), ("kmax_inject", C.c_int32),
        ("inject_theta", C.c_double), ("filter_passes", C.c_int32), ("qed_quantum", C.c_int32),
        ("protons", C.c_int32), ("m_ion", C.c_double),
        ("em", C.c_int32), ("pml_cells", C.c_int32), ("beta_y", C.c_double), ("beta_z", C.c_double),
        ("pml_sigma", C.c_double), ("jperp", C.c_int32), ("pad_jperp", C.c_int32),
    ]


class Counters(C.Structure):
    _fields_ = [(n, C.c_int64) for n in (
        "emit_events", "photons", "pairs", "injected", "absorbed", "escaped",
        "photons_escaped", "emit_overflow", "inject_overflow", "load_overflow", "merged",
        "photons_merged")] + [
        (n, C.c_double) for n in (
            "e_radiated", "e_absorbed", "e_escaped", "e_photon_escaped", "e_injected",
            "work_jm")]

    def as_dict(self):
        return {n: getattr(self, n) for n, _ in self._fields_}


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_SO)
        d, i64, u64, u32, i32, vp = C.c_double, C.c_int64, C.c_uint64, C.c_uint32, C.c_int32, C.c_void_p
        pd = C.POINTER(C.c_double)
        L.orc_philox4x32_10.argtypes = [C.POINTER(u32), C.POINTER(u32), C.POINTER(u32)]
        L.orc_uniform.argtypes = [u64, u64, u32, u32, u32]; L.orc_uniform.restype = d
        L.orc_mix64.argtypes = [u64]; L.orc_mix64.restype = u64
        L.orc_child_id.argtypes = [u64, u32, u32, u32]; L.orc_child_id.restype = u64
        for f in ("orc_tsyn", "orc_tbw", "orc_spec_survival", "orc_spec_inverse"):
            getattr(L, f).argtypes = [d]; getattr(L, f).restype = d
        L.orc_mj_sample.argtypes = [u64, u64, d, C.POINTER(C.c_int)]; L.orc_mj_sample.restype = d
        for f in ("orc_qspec_density", "orc_qspec_survival", "orc_qspec_inverse", "orc_bw_density",
                  "orc_bw_tail", "orc_bw_split"):
            getattr(L, f).argtypes = [d, d]; getattr(L, f).restype = d
        L.orc_binomial_smooth.argtypes = [C.POINTER(d), i64, C.c_int32, C.c_int32]
        L.orc_mj_draw.argtypes = [u64, u64, u32, u32, d, C.POINTER(C.c_int)]; L.orc_mj_draw.restype = d
        L.orc_create.argtypes = [C.POINTER(Params)]; L.orc_create.restype = vp
        L.orc_destroy.argtypes = [vp]
        L.orc_step.argtypes = [vp]
        L.orc_run.argtypes = [vp, i64]
        L.orc_solve_gauss.argtypes = [vp]
        L.orc_add_lepton.argtypes = [vp, u64, i32, d, d, d, d]
        L.orc_add_photon.argtypes = [vp, u64, d, d, d, i32, i32, d]
        L.orc_set_eta_bg.argtypes = [vp, d]
        L.orc_set_E.argtypes = [vp, pd]
        L.orc_cell_charge.argtypes = [vp, i64]; L.orc_cell_charge.restype = d
        L.orc_gauss_residual.argtypes = [vp, pd]; L.orc_gauss_residual.restype = d
        L.orc_moments.argtypes = [vp, pd, pd, pd, pd]
        L.orc_return_spectrum.argtypes = [vp, pd]
        L.orc_spectra.argtypes = [vp, i32, d, d, pd, pd]
        for f in ("orc_nlep", "orc_nph", "orc_nnode", "orc_stepno"):
            getattr(L, f).argtypes = [vp]; getattr(L, f).restype = i64
        for f in ("orc_w0", "orc_eta_bg"):
            getattr(L, f).argtypes = [vp]; getattr(L, f).restype = d
        L.orc_get_E.argtypes = [vp, pd]
        L.orc_get_counters.argtypes = [vp, C.POINTER(Counters)]
        L.orc_get_leptons.argtypes = [vp] + [vp] * 6
        L.orc_get_photons.argtypes = [vp] + [vp] * 8
        L.orc_get_lepton_heavy.argtypes = [vp, vp]
        L.orc_add_proton.argtypes = [vp, u64, d, d, d]
        L.orc_set_em.argtypes = [vp, pd, pd, pd, pd]
        L.orc_get_em.argtypes = [vp, pd, pd, pd, pd]
        L.orc_get_jperp.argtypes = [vp, pd, pd]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _pd(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


# ---------------------------------------------------------------- primitives
def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def uniform(seed, pid, step, channel, k):
    return lib().orc_uniform(seed, pid, step, channel, k)


def mix64(x):
    return lib().orc_mix64(x)


def child_id(parent, step, channel, k):
    return lib().orc_child_id(parent, step, channel, k)


def tsyn(chi):
    return lib().orc_tsyn(float(chi))


def tbw(chi):
    return lib().orc_tbw(float(chi))


def spec_survival(xi):
    return lib().orc_spec_survival(float(xi))


def spec_inverse(U):
    return lib().orc_spec_inverse(float(U))


def qspec_density(chi, xi):
    return lib().orc_qspec_density(float(chi), float(xi))


def qspec_survival(chi, xi):
    return lib().orc_qspec_survival(float(chi), float(xi))


def qspec_inverse(chi, U):
    return lib().orc_qspec_inverse(float(chi), float(U))


def bw_density(chi, e):
    return lib().orc_bw_density(float(chi), float(e))


def bw_tail(chi, e0):
    return lib().orc_bw_tail(float(chi), float(e0))


def bw_split(chi, U):
    return lib().orc_bw_split(float(chi), float(U))


EXT_PERIODIC, EXT_NODE_EVEN, EXT_CELL_ODD = 0, 1, 2


def binomial_smooth(a, passes, ext):
    """The oracle's binomial current/charge smoother on a copy of a."""
    b = np.ascontiguousarray(a, dtype=np.float64).copy()
    lib().orc_binomial_smooth(b.ctypes.data_as(C.POINTER(C.c_double)), b.size, passes, ext)
    return b


def mj_draw(seed, pid, step, channel, theta):
    ok = C.c_int(0)
    u = lib().orc_mj_draw(seed, pid, step, channel, float(theta), C.byref(ok))
    return u, bool(ok.value)


def mj_sample(seed, pid, theta):
    ok = C.c_int(0)
    u = lib().orc_mj_sample(seed, pid, float(theta), C.byref(ok))
    return u, bool(ok.value)


# ---------------------------------------------------------------- PIC model
DEFAULTS = dict(alpha=0.0, b=0.1, lambda_hat=1e-5, rho_hat=100.0, rate_mult=1.0,
                gap_length=0.0, density=1.0, dx=0.1, dt=0.045, theta=0.0, seed_amp=0.0,
                nx=64, ppc=0, cap=0, seed=0, gap_index=0, qed=0, boundary=BC_SURFACE,
                init=INIT_EMPTY, kmax_emit=16, kmax_inject=64, inject_theta=0.0,
                filter_passes=0, qed_quantum=0, protons=0, m_ion=1836.0,
                em=0, pml_cells=0, beta_y=0.0, beta_z=0.0, pml_sigma=0.0, jperp=0)


class Sim:
    """One gap of the oracle PIC model (FP64, single-threaded)."""

    def __init__(self, **kw):
        cfg = dict(DEFAULTS)
        cfg.update(kw)
        if cfg["gap_length"] == 0.0:
            cfg["gap_length"] = 0.8 * cfg["nx"] * cfg["dx"]
        self.cfg = cfg
        self.params = Params(**cfg)
        self.h = lib().orc_create(C.byref(self.params))

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_destroy(self.h)
            self.h = None

    # state ---------------------------------------------------------------
    def add_lepton(self, pid, q, X, u, w, tau=1e30):
        lib().orc_add_lepton(self.h, pid, q, X, u, w, tau)

    def add_proton(self, pid, X, u, w):
        lib().orc_add_proton(self.h, pid, X, u, w)

    def add_photon(self, pid, X, x, w, direction, n0, tau_star):
        lib().orc_add_photon(self.h, pid, X, x, w, direction, n0, tau_star)

    def set_eta_bg(self, eta):
        lib().orc_set_eta_bg(self.h, float(eta))

    def set_E(self, E):
        E = np.ascontiguousarray(E, dtype=np.float64)
        assert E.size == self.nnode
        lib().orc_set_E(self.h, _pd(E))

    def solve_gauss(self):
        lib().orc_solve_gauss(self.h)

    def set_em(self, Ey, Ez, By, Bz):
        """Transverse fields (em = 1): E_y, E_z on the nx cells (half steps),
        B_y, B_z on the nodes."""
        nx = self.cfg["nx"]
        a = [np.ascontiguousarray(f, dtype=np.float64) for f in (Ey, Ez, By, Bz)]
        assert a[0].size == a[1].size == nx and a[2].size == a[3].size == self.nnode
        lib().orc_set_em(self.h, *[_pd(f) for f in a])

    def em(self):
        """(E_y, E_z, B_y, B_z) of an em = 1 gap."""
        nx = self.cfg["nx"]
        out = [np.empty(nx), np.empty(nx), np.empty(self.nnode), np.empty(self.nnode)]
        lib().orc_get_em(self.h, *[_pd(f) for f in out])
        return tuple(out)

    def jperp(self):
        """(j_y, j_z) on the nx cells: the transverse particle current of the
        last step (em = 1 with jperp = 1)."""
        nx = self.cfg["nx"]
        out = [np.empty(nx), np.empty(nx)]
        lib().orc_get_jperp(self.h, *[_pd(f) for f in out])
        return tuple(out)

    def step(self, n=1):
        lib().orc_run(self.h, int(n))

    @property
    def nnode(self):
        return lib().orc_nnode(self.h)

    @property
    def stepno(self):
        return lib().orc_stepno(self.h)

    @property
    def w0(self):
        return lib().orc_w0(self.h)

    @property
    def eta_bg(self):
        return lib().orc_eta_bg(self.h)

    def E(self):
        out = np.empty(self.nnode)
        lib().orc_get_E(self.h, _pd(out))
        return out

    def counters(self):
        c = Counters()
        lib().orc_get_counters(self.h, C.byref(c))
        return c.as_dict()

    def leptons(self):
        n = lib().orc_nlep(self.h)
        out = dict(id=np.empty(n, np.uint64), q=np.empty(n, np.int32), X=np.empty(n),
                   u=np.empty(n), w=np.empty(n), tau=np.empty(n))
        lib().orc_get_leptons(self.h, *(_p(out[k]) for k in ("id", "q", "X", "u", "w", "tau")))
        out["heavy"] = np.empty(n, np.int32)
        lib().orc_get_lepton_heavy(self.h, _p(out["heavy"]))
        return out

    def photons(self):
        n = lib().orc_nph(self.h)
        out = dict(id=np.empty(n, np.uint64), X=np.empty(n), x=np.empty(n), w=np.empty(n),
                   tau_star=np.empty(n), tau_acc=np.empty(n), dir=np.empty(n, np.int32),
                   n0=np.empty(n, np.int32))
        lib().orc_get_photons(self.h, *(_p(out[k]) for k in (
            "id", "X", "x", "w", "tau_star", "tau_acc", "dir", "n0")))
        return out

    def cell_charge(self, c):
        return lib().orc_cell_charge(self.h, int(c))

    def gauss_residual(self):
        em = C.c_double(0.0)
        r = lib().orc_gauss_residual(self.h, C.byref(em))
        return r, em.value

    def moments(self):
        nx = self.cfg["nx"]
        dens = np.empty(4 * nx)
        g3w, wsum, charge = np.empty(nx), np.empty(nx), np.empty(nx)
        lib().orc_moments(self.h, _pd(dens), _pd(g3w), _pd(wsum), _pd(charge))
        return dict(dens=dens.reshape(2, 2, nx), g3w=g3w, wsum=wsum, charge=charge)

    def return_spectrum(self):
        """Weight of the e+- absorbed at h < 0 so far per bin of ln gamma
        (bin i: 10^(i/8) <= gamma < 10^((i+1)/8), the last open)."""
        out = np.empty(64)
        lib().orc_return_spectrum(self.h, _pd(out))
        return out

    def spectra(self, nbins, lo, hi):
        """Weight per bin of ln p (electrons, positrons) and ln x (photons) in
        the gap, nbins uniform bins over [lo, hi), clamped at both ends."""
        lep, ph = np.empty(2 * nbins), np.empty(nbins)
        lib().orc_spectra(self.h, int(nbins), float(lo), float(hi), _pd(lep), _pd(ph))
        return lep.reshape(2, nbins), ph

    def diag(self):
        """Gap diagnostics of Sect. 6.2 / Fig. 5 from the per-cell moments."""
        return diag_from_state(self.cfg, self.moments(), self.E())


def diag_from_state(cfg, mom, E):
    nx, dx = cfg["nx"], cfg["dx"]
    Hc = cfg["gap_length"] / dx
    cells = np.arange(nx)
    gap_cells = cells[(cells + 0.5) < Hc]
    dens = mom["dens"]
    m_tot = dens.sum(axis=(0, 1))
    mg = m_tot[gap_cells]
    ipk = int(gap_cells[np.argmax(mg)]) if mg.size else 0
    g3 = mom["g3w"][ipk] / mom["wsum"][ipk] if mom["wsum"][ipk] > 0 else 0.0
    nodes = np.arange(E.size)
    gap_nodes = nodes[nodes <= Hc]
    Eg = E[gap_nodes]
    P = 1
    while P < Eg.size:
        P *= 2
    spec = np.abs(np.fft.rfft(np.concatenate([Eg, np.zeros(P - Eg.size)]))) ** 2 / P
    return dict(M_peak=float(mg.max()) if mg.size else 0.0,
                M_avg=float(mg.mean()) if mg.size else 0.0,
                peak_cell=ipk, g3_peak=float(g3),
                M_split=dens[:, :, ipk].copy(),
                E_min=float(Eg.min()), E_max=float(Eg.max()), spectrum=spec)
