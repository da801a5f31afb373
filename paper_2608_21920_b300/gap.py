"""Python binding of the PIC library: argument marshalling only.

Device memory comes from torch (one uint8 CUDA tensor per handle is the
library workspace) and work is enqueued on torch's current stream; every
step of the method runs in the CUDA kernels of libgap.so.
"""
from __future__ import annotations

import ctypes as C
from typing import Iterable

import numpy as np
import torch

from . import _abi as A

PARAM_DEFAULTS = dict(
    alpha=0.0, b=0.1, lambda_hat=1e-5, rho_hat=100.0, rate_mult=1.0, gap_length=0.0,
    density=1.0, dx=0.1, dt=0.045, theta=0.0, seed_amp=0.0, nx=64, ppc=0, cap=0, seed=0,
    qed=0, boundary=A.GAP_BC_SURFACE, init=A.GAP_INIT_EMPTY, kmax_emit=16, kmax_inject=64,
    gap_index=0, inject_theta=0.0, filter_passes=0, qed_quantum=0, protons=0, m_ion=1836.0,
    em=0, pml_cells=0, beta_y=0.0, beta_z=0.0, pml_sigma=0.0, jperp=0)

PRECISION = {"fp64": A.GAP_FP64_PLAIN, "fp32": A.GAP_FP32_STATE}


def make_params(**kw) -> A.GapParams:
    cfg = dict(PARAM_DEFAULTS)
    unknown = set(kw) - set(cfg)
    if unknown:
        raise KeyError(f"unknown gap parameters: {sorted(unknown)}")
    cfg.update(kw)
    return A.GapParams(**cfg)


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, torch.Tensor):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


class Gap:
    """A batch of independent gaps advanced together by one launch per step."""

    def __init__(self, params: dict | Iterable[dict], precision: str = "fp32", tile: int = 0,
                 threads: int = 0, rebin_every: int = 0, slack: float = 0.0, variant: int = 0,
                 lepton_capacity: int = 0, photon_capacity: int = 0, device: str = "cuda:0"):
        if isinstance(params, dict):
            params = [params]
        plist = [dict(p) for p in params]
        self.param_dicts = []
        for i, p in enumerate(plist):
            p.setdefault("gap_index", i)
            merged = dict(PARAM_DEFAULTS)
            merged.update(p)
            if merged["gap_length"] == 0.0:
                merged["gap_length"] = 0.8 * merged["nx"] * merged["dx"]
            self.param_dicts.append(merged)
        n = len(plist)
        self._params = (A.GapParams * n)(*[make_params(**p) for p in self.param_dicts])
        self._cfg = A.GapConfig(precision=PRECISION[precision], tile=tile, threads=threads,
                                rebin_every=rebin_every, variant=variant, slack=slack,
                                lepton_capacity=lepton_capacity, photon_capacity=photon_capacity)
        self.precision = precision
        self.n_gaps = n
        self.device = torch.device(device)
        L = A.lib()
        nbytes = C.c_size_t(0)
        A.check(L.gap_workspace_bytes(self._params, n, C.byref(self._cfg), C.byref(nbytes)),
                None, "gap_workspace_bytes")
        self.workspace_bytes = nbytes.value
        self.workspace = torch.empty(self.workspace_bytes, dtype=torch.uint8, device=self.device)
        self._h = C.c_void_p()
        st = self.stream()
        A.check(L.gap_init(self._params, n, C.byref(self._cfg), C.c_void_p(self.workspace.data_ptr()),
                           self.workspace_bytes, st, C.byref(self._h)), self._h, "gap_init")

    # ------------------------------------------------------------------
    def stream(self):
        return C.c_void_p(torch.cuda.current_stream(self.device).cuda_stream)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            A.lib().gap_free(self._h)
            self._h = C.c_void_p()
        self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def nnode(self, gap=0):
        p = self.param_dicts[gap]
        return p["nx"] if p["boundary"] == A.GAP_BC_PERIODIC else p["nx"] + 1

    # ------------------------------------------------------------------
    def step(self, n: int = 1, graph_chunk: int = 0):
        L = A.lib()
        if graph_chunk > 0:
            A.check(L.gap_step_graph(self._h, int(n), int(graph_chunk), self.stream()), self._h, "gap_step_graph")
        else:
            A.check(L.gap_step(self._h, int(n), self.stream()), self._h, "gap_step")

    def profile(self, on: bool):
        """Switch live timing of the push kernel; returns (ms summed, launches
        timed, kernel launches per step) since the previous call."""
        ms, n, lps = C.c_double(0), C.c_int64(0), C.c_int64(0)
        A.check(A.lib().gap_profile(self._h, int(on), C.byref(ms), C.byref(n), C.byref(lps)), self._h,
                "gap_profile")
        return ms.value, n.value, lps.value

    PHASES = ("push", "photons+inject+house", "rebin", "merge", "push_tail")

    def profile_phases(self) -> tuple[dict, int]:
        """Per-phase durations (ms, summed) of the steps profiled since the
        last profile() call, and the number of those steps."""
        ms = (C.c_double * len(self.PHASES))()
        n = C.c_int64(0)
        A.check(A.lib().gap_profile_phases(self._h, ms, C.byref(n)), self._h, "gap_profile_phases")
        return {k: ms[i] for i, k in enumerate(self.PHASES)}, n.value

    def spectrum_inverse(self, U, precision: str | None = None):
        """xi with P(xi' > xi) = U for a CUDA tensor of uniforms (float64)."""
        U = U.to(device=self.device, dtype=torch.float64).contiguous()
        xi = torch.empty_like(U)
        prec = PRECISION[precision or self.precision]
        A.check(A.lib().gap_spectrum_inverse(self._h, _ptr(U), _ptr(xi), U.numel(), prec, self.stream()),
                self._h, "gap_spectrum_inverse")
        return xi

    def qspectrum_inverse(self, chi, U, precision: str | None = None):
        """Energy fraction xi of the quantum spectrum (qed_quantum gaps) for
        CUDA tensors of chi and uniforms U (float64)."""
        chi = chi.to(device=self.device, dtype=torch.float64).contiguous()
        U = U.to(device=self.device, dtype=torch.float64).contiguous()
        xi = torch.empty_like(U)
        prec = PRECISION[precision or self.precision]
        A.check(A.lib().gap_qspectrum_inverse(self._h, _ptr(chi), _ptr(U), _ptr(xi), U.numel(), prec,
                                              self.stream()), self._h, "gap_qspectrum_inverse")
        return xi

    def pair_split(self, chi, U):
        """Electron's energy fraction of a conversion (qed_quantum gaps) for
        CUDA tensors of chi and uniforms U (float64)."""
        chi = chi.to(device=self.device, dtype=torch.float64).contiguous()
        U = U.to(device=self.device, dtype=torch.float64).contiguous()
        e = torch.empty_like(U)
        A.check(A.lib().gap_pair_split(self._h, _ptr(chi), _ptr(U), _ptr(e), U.numel(), self.stream()),
                self._h, "gap_pair_split")
        return e

    @property
    def steps_done(self) -> int:
        return A.lib().gap_steps_done(self._h)

    def field(self, gap: int = 0) -> np.ndarray:
        out = np.empty(self.nnode(gap))
        A.check(A.lib().gap_get_field(self._h, gap, _ptr(out), out.size, self.stream()), self._h, "gap_get_field")
        return out

    def field_async(self, out, copy_stream, gap: int = 0):
        """E after the steps enqueued so far, copied into `out` (a pinned
        host float64 tensor of at least nnode(gap) values) on `copy_stream`
        (a torch.cuda.Stream other than the current one) without waiting:
        later steps overlap the transfer; `out` is complete once copy_stream
        has passed this call."""
        assert out.dtype == torch.float64 and out.is_pinned() and out.numel() >= self.nnode(gap)
        A.check(A.lib().gap_get_field_async(self._h, gap, C.c_void_p(out.data_ptr()), out.numel(), self.stream(),
                                            C.c_void_p(copy_stream.cuda_stream)), self._h, "gap_get_field_async")

    def set_field(self, E, gap: int = 0):
        E = np.ascontiguousarray(E, dtype=np.float64)
        A.check(A.lib().gap_set_field(self._h, gap, _ptr(E), E.size, self.stream()), self._h, "gap_set_field")

    def em(self, gap: int = 0):
        """Transverse fields of an em = 1 gap: (E_y, E_z) on the nx cells at
        the half step before the current one, (B_y, B_z) on the nodes."""
        nx = int(self.param_dicts[gap]["nx"])
        out = []
        for comp, n in ((A.GAP_EM_EY, nx), (A.GAP_EM_EZ, nx), (A.GAP_EM_BY, self.nnode(gap)),
                        (A.GAP_EM_BZ, self.nnode(gap))):
            a = np.empty(n)
            A.check(A.lib().gap_get_em(self._h, gap, comp, _ptr(a), n, self.stream()), self._h, "gap_get_em")
            out.append(a)
        return tuple(out)

    def set_em(self, Ey, Ez, By, Bz, gap: int = 0):
        for comp, f in ((A.GAP_EM_EY, Ey), (A.GAP_EM_EZ, Ez), (A.GAP_EM_BY, By), (A.GAP_EM_BZ, Bz)):
            f = np.ascontiguousarray(f, dtype=np.float64)
            A.check(A.lib().gap_set_em(self._h, gap, comp, _ptr(f), f.size, self.stream()), self._h, "gap_set_em")

    def solve_gauss(self, set_background: bool = True):
        A.check(A.lib().gap_solve_gauss(self._h, int(set_background), self.stream()), self._h, "gap_solve_gauss")

    def set_background(self, eta: float, gap: int = 0):
        A.check(A.lib().gap_set_background(self._h, gap, float(eta)), self._h, "gap_set_background")

    def particles(self, kind: int, gap: int = 0, cap: int | None = None) -> dict:
        L = A.lib()
        n = C.c_int64(0)
        if cap is None:
            A.lib().gap_get_particles(self._h, gap, kind, 0, None, None, None, None, None, None, None,
                                      C.byref(n), self.stream())
            cap = n.value
        out = dict(id=np.empty(cap, np.uint64), X=np.empty(cap), u=np.empty(cap), w=np.empty(cap),
                   tau=np.empty(cap))
        aux = np.empty(cap) if kind == A.GAP_PHOTON else None
        aux2 = np.empty(cap, np.int64) if kind == A.GAP_PHOTON else None
        A.check(L.gap_get_particles(self._h, gap, kind, cap, _ptr(out["id"]), _ptr(out["X"]), _ptr(out["u"]),
                                    _ptr(out["w"]), _ptr(out["tau"]), _ptr(aux), _ptr(aux2), C.byref(n),
                                    self.stream()), self._h, "gap_get_particles")
        m = n.value
        res = {k: v[:m] for k, v in out.items()}
        if kind == A.GAP_PHOTON:
            res = dict(id=res["id"], X=res["X"], x=res["u"], w=res["w"], tau_acc=res["tau"],
                       tau_star=aux[:m], n0=(aux2[:m] >> 1).astype(np.int64),
                       dir=np.where(aux2[:m] & 1, 1, -1).astype(np.int32))
        return res

    def save(self) -> np.ndarray:
        """The handle's whole state as host bytes (checkpoint)."""
        L = A.lib()
        n = L.gap_state_bytes(self._h)
        buf = np.empty(n, np.uint8)
        A.check(L.gap_save(self._h, _ptr(buf), n, self.stream()), self._h, "gap_save")
        return buf

    def load(self, state: np.ndarray):
        """Resume from a state saved by a handle with the same parameters and
        configuration."""
        buf = np.ascontiguousarray(state, dtype=np.uint8)
        A.check(A.lib().gap_load(self._h, _ptr(buf), buf.size, self.stream()), self._h, "gap_load")

    def sample_particles(self, kind: int, stride: int, gap: int = 0) -> dict:
        """Leptons of one species whose id is a multiple of `stride`: the same
        sample from step to step, for large gaps."""
        L = A.lib()
        n = C.c_int64(0)
        L.gap_sample_particles(self._h, gap, kind, int(stride), 0, None, None, None, None, None, C.byref(n),
                               self.stream())
        cap = n.value
        out = dict(id=np.empty(cap, np.uint64), X=np.empty(cap), u=np.empty(cap), w=np.empty(cap),
                   tau=np.empty(cap))
        A.check(L.gap_sample_particles(self._h, gap, kind, int(stride), cap, _ptr(out["id"]), _ptr(out["X"]),
                                       _ptr(out["u"]), _ptr(out["w"]), _ptr(out["tau"]), C.byref(n),
                                       self.stream()), self._h, "gap_sample_particles")
        return {k: v[:n.value] for k, v in out.items()}

    def spectra(self, nbins: int, lo: float, hi: float, gap: int = 0):
        """Weight per bin of ln p (electrons, positrons: [2, nbins]) and of ln x
        (photons: [nbins]) in the gap, nbins uniform bins over [lo, hi)."""
        lep, ph = np.empty(2 * nbins), np.empty(nbins)
        A.check(A.lib().gap_spectra(self._h, gap, int(nbins), float(lo), float(hi), _ptr(lep), _ptr(ph),
                                    self.stream()), self._h, "gap_spectra")
        return lep.reshape(2, nbins), ph

    def return_spectrum(self, gap: int = 0) -> np.ndarray:
        """Weight of the e+- absorbed at h < 0 per bin of ln gamma (eight per
        decade from gamma = 1; the last bin open)."""
        out = np.empty(A.GAP_RETURN_BINS)
        A.check(A.lib().gap_return_spectrum(self._h, gap, _ptr(out), self.stream()), self._h,
                "gap_return_spectrum")
        return out

    def tile_particles(self, kind: int, tile_lo: int, tile_hi: int, gap: int = 0) -> dict:
        """Leptons of one species stored in tiles [tile_lo, tile_hi) of a gap."""
        L = A.lib()
        n = C.c_int64(0)
        L.gap_tile_particles(self._h, gap, kind, int(tile_lo), int(tile_hi), 0, None, None, None, None, None,
                             C.byref(n), self.stream())
        cap = n.value
        out = dict(id=np.empty(cap, np.uint64), X=np.empty(cap), u=np.empty(cap), w=np.empty(cap),
                   tau=np.empty(cap))
        A.check(L.gap_tile_particles(self._h, gap, kind, int(tile_lo), int(tile_hi), cap, _ptr(out["id"]),
                                     _ptr(out["X"]), _ptr(out["u"]), _ptr(out["w"]), _ptr(out["tau"]),
                                     C.byref(n), self.stream()), self._h, "gap_tile_particles")
        return {k: v[:n.value] for k, v in out.items()}

    def add_particles(self, kind: int, id, X, u, w, tau, n0=None, direction=None, gap: int = 0):
        id = np.ascontiguousarray(id, dtype=np.uint64)
        X, u, w, tau = (np.ascontiguousarray(a, dtype=np.float64) for a in (X, u, w, tau))
        aux2 = None
        if kind == A.GAP_PHOTON:
            aux2 = (np.asarray(n0, np.int64) << 1) | (np.asarray(direction) > 0).astype(np.int64)
            aux2 = np.ascontiguousarray(aux2, dtype=np.int64)
        A.check(A.lib().gap_add_particles(self._h, gap, kind, id.size, _ptr(id), _ptr(X), _ptr(u), _ptr(w),
                                          _ptr(tau), _ptr(aux2), self.stream()), self._h, "gap_add_particles")

    def diag(self, gap: int = 0, spectrum: bool = True, moments: bool = False) -> dict:
        out = A.GapDiagOut()
        p = self.param_dicts[gap]
        P = 1
        ng = min(int(np.floor(p["gap_length"] / p["dx"])) + 1, self.nnode(gap))
        while P < ng:
            P *= 2
        spec = np.empty(P // 2 + 1) if spectrum else None
        mom = np.empty(8 * p["nx"]) if moments else None
        A.check(A.lib().gap_diag(self._h, gap, C.byref(out), _ptr(spec), 0 if spec is None else spec.size,
                                 _ptr(mom), self.stream()), self._h, "gap_diag")
        res = {n: getattr(out, n) for n, _ in A.GapDiagOut._fields_ if n not in ("M_split", "counters")}
        res["M_split"] = np.array(out.M_split[:]).reshape(2, 2)
        res["counters"] = {n: getattr(out.counters, n) for n, _ in A.GapCounters._fields_}
        if spec is not None:
            res["spectrum"] = spec
        if mom is not None:
            nx = p["nx"]
            m = mom.reshape(8, nx)
            res["moments"] = dict(dens=m[0:4].reshape(2, 2, nx).copy(), g3w=m[4].copy(), wsum=m[5].copy(),
                                  charge=m[6].copy(), photon_dens=m[7].copy())
        return res
