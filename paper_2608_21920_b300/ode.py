"""Batched integrator of the discharge concurrency model (Sect. 5.2,
eq. dis1-dis4) behind torch.autograd.Function: the forward RK4 and the
discrete adjoint both run in the CUDA kernels of libgap.so."""
from __future__ import annotations

import ctypes as C

import torch

from . import _abi as A

_DT = {torch.float64: 0, torch.float32: 1}


def _vp(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _stream(dev):
    return C.c_void_p(torch.cuda.current_stream(dev).cuda_stream)


def forward(p, y0, dt, nsteps, every=1, ckpt_every=0, delta=0.0):
    """Integrate B parameter sets.  p [B,5] = (alpha, t_x, t_pm, t_acc, g3),
    y0 [B,4] = (m_pm, m_x, eps, j), dt [B]; returns out [T,B,4] and the
    checkpoints [nsteps/ckpt_every+1, B, 4] (None if ckpt_every == 0)."""
    assert p.is_cuda and p.dtype in _DT and p.shape[1] == 5 and y0.shape[1] == 4
    B = p.shape[0]
    T = nsteps // every + 1
    out = torch.empty(T, B, 4, dtype=p.dtype, device=p.device)
    ckpt = None
    if ckpt_every > 0:
        ckpt = torch.empty(nsteps // ckpt_every + 1, B, 4, dtype=p.dtype, device=p.device)
    A.check(A.lib().ode_forward(_vp(p), _vp(y0), _vp(dt), B, nsteps, every, max(ckpt_every, 1), float(delta),
                                _DT[p.dtype], _vp(out), _vp(ckpt), _stream(p.device)), None, "ode_forward")
    return out, ckpt


def adjoint(p, dt, ckpt, gout, nsteps, every, ckpt_every, delta=0.0):
    B = p.shape[0]
    gp = torch.empty_like(p)
    gy0 = torch.empty(B, 4, dtype=p.dtype, device=p.device)
    scratch = torch.empty(ckpt_every + 1, B, 4, dtype=p.dtype, device=p.device)
    A.check(A.lib().ode_adjoint(_vp(p), _vp(dt), _vp(ckpt), _vp(gout), B, nsteps, every, ckpt_every,
                                float(delta), _DT[p.dtype], _vp(gp), _vp(gy0), _vp(scratch),
                                _stream(p.device)), None, "ode_adjoint")
    return gp, gy0


class ConcurrencyModel(torch.autograd.Function):
    """out = RK4(p, y0) sampled every `every` steps; backward by the
    hand-written discrete adjoint (exact derivative of the RK4 map)."""

    @staticmethod
    def forward(ctx, p, y0, dt, nsteps: int, every: int, ckpt_every: int, delta: float):
        p = p.contiguous()
        y0 = y0.contiguous()
        dt = dt.contiguous()
        out, ckpt = forward(p, y0, dt, nsteps, every, ckpt_every, delta)
        ctx.save_for_backward(p, dt, ckpt)
        ctx.cfg = (nsteps, every, ckpt_every, delta)
        return out

    @staticmethod
    def backward(ctx, gout):
        p, dt, ckpt = ctx.saved_tensors
        nsteps, every, ckpt_every, delta = ctx.cfg
        gp, gy0 = adjoint(p, dt, ckpt, gout.contiguous(), nsteps, every, ckpt_every, delta)
        return gp, gy0, None, None, None, None, None


def integrate(p, y0, dt, nsteps, every=1, ckpt_every=None, delta=0.0):
    if ckpt_every is None:
        ckpt_every = max(1, int(round(nsteps ** 0.5)))
    return ConcurrencyModel.apply(p, y0, dt, nsteps, every, ckpt_every, delta)
