"""Batched integrator of the discharge concurrency model (Sect. 5.2,
eq. dis1-dis4, and the extended model with the <gamma^-3> moment equation)
behind torch.autograd.Function: the forward RK4 and the discrete adjoint both
run in the CUDA kernels of libgap.so."""
from __future__ import annotations

import ctypes as C

import torch

from . import _abi as A

_DT = {torch.float64: 0, torch.float32: 1}


def _vp(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _stream(dev):
    return C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


# (state entries, parameter entries, forward entry point, adjoint entry point)
_MODELS = {"base": (4, 5, "ode_forward", "ode_adjoint"), "ext": (5, 6, "ode_ext_forward", "ode_ext_adjoint")}


def forward(p, y0, dt, nsteps, every=1, ckpt_every=0, delta=0.0, model="base"):
    """Integrate B parameter sets.  Base model: p [B,5] = (alpha, t_x, t_pm,
    t_acc, g3), y0 [B,4] = (m_pm, m_x, eps, j); extended model ("ext"):
    p [B,6] = (alpha, t_x, t_pm, t_acc, gamma_min, gamma_rad), y0 [B,5] =
    (m_pm, m_x, eps, j, G = m_pm <gamma^-3>).  dt [B]; returns out [T,B,NY]
    and the checkpoints [nsteps/ckpt_every+1, B, NY] (None if ckpt_every == 0)."""
    ny, npar, fwd, _ = _MODELS[model]
    assert p.is_cuda and p.dtype in _DT and p.shape[1] == npar and y0.shape[1] == ny
    B = p.shape[0]
    T = nsteps // every + 1
    out = torch.empty(T, B, ny, dtype=p.dtype, device=p.device)
    ckpt = None
    if ckpt_every > 0:
        ckpt = torch.empty(nsteps // ckpt_every + 1, B, ny, dtype=p.dtype, device=p.device)
    A.check(getattr(A.lib(), fwd)(_vp(p), _vp(y0), _vp(dt), B, nsteps, every, max(ckpt_every, 1), float(delta),
                                  _DT[p.dtype], _vp(out), _vp(ckpt), _stream(p.device)), None, fwd)
    return out, ckpt


def adjoint(p, dt, ckpt, gout, nsteps, every, ckpt_every, delta=0.0, model="base"):
    ny, npar, _, adj = _MODELS[model]
    B = p.shape[0]
    gp = torch.empty_like(p)
    gy0 = torch.empty(B, ny, dtype=p.dtype, device=p.device)
    scratch = torch.empty(ckpt_every + 1, B, ny, dtype=p.dtype, device=p.device)
    A.check(getattr(A.lib(), adj)(_vp(p), _vp(dt), _vp(ckpt), _vp(gout), B, nsteps, every, ckpt_every,
                                  float(delta), _DT[p.dtype], _vp(gp), _vp(gy0), _vp(scratch),
                                  _stream(p.device)), None, adj)
    return gp, gy0


class ConcurrencyModel(torch.autograd.Function):
    """out = RK4(p, y0) sampled every `every` steps; backward by the
    hand-written discrete adjoint (exact derivative of the RK4 map)."""

    @staticmethod
    def forward(ctx, p, y0, dt, nsteps: int, every: int, ckpt_every: int, delta: float, model: str = "base"):
        p = p.contiguous()
        y0 = y0.contiguous()
        dt = dt.contiguous()
        out, ckpt = forward(p, y0, dt, nsteps, every, ckpt_every, delta, model)
        ctx.save_for_backward(p, dt, ckpt)
        ctx.cfg = (nsteps, every, ckpt_every, delta, model)
        return out

    @staticmethod
    def backward(ctx, gout):
        p, dt, ckpt = ctx.saved_tensors
        nsteps, every, ckpt_every, delta, model = ctx.cfg
        gp, gy0 = adjoint(p, dt, ckpt, gout.contiguous(), nsteps, every, ckpt_every, delta, model)
        return gp, gy0, None, None, None, None, None, None


def integrate(p, y0, dt, nsteps, every=1, ckpt_every=None, delta=0.0, model="base"):
    """out [T,B,NY] of the base model (eq. dis1-dis4) or, with model="ext",
    the extended model with G = m_pm <gamma^-3> as a fifth state."""
    if ckpt_every is None:
        ckpt_every = max(1, int(round(nsteps ** 0.5)))
    return ConcurrencyModel.apply(p, y0, dt, nsteps, every, ckpt_every, delta, model)
