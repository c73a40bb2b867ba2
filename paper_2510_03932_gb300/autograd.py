"""Differentiation form: torch.autograd.Functions over the transcription evaluator.

  c = constraints(H, x, p)     c(x; p), the constraint vector, p the model's dynamics parameters
                               (Van der Pol mu; cart-pole m_c, m_p, l, g; Goddard Cd, beta,
                               Tmax, b; quadrotor g; none for the double integrator and heat)
  F = objective(H, x)          the trapezoidal objective

Every forward and backward step is one launch of the CUDA library; node states are
recomputed from x in each kernel, never stored.  Derivatives:
  constraints   forward:   c(x; p)                               ocp_eval_cons_params
                backward:  (J^T w, (dc/dp)^T w)                  ocp_vjp_params
                double backward (Van der Pol), for cotangents (gx, gmu) of that pair:
                  w-bar  = J gx + (dc/dmu) gmu                    ocp_jprod_param
                  x-bar  = (sum_r w_r Hess c_r) gx + gmu m(x, w)   ocp_hprod_param (sigma = 0)
                  mu-bar = m(x, w) . gx                            (same launch)
                where m(x, w) = sum_r w_r d2 c_r / dx dmu  (c is linear in mu: d2c/dmu2 = 0);
                the other models: w-bar = J gx and x-bar = (sum_r w_r Hess c_r) gx, the terms
                in x alone (second derivatives in their parameters are not provided)
  objective     backward:  s grad F(x)                             ocp_eval_grad_scaled
                double backward:  x-bar = s Hess F gx,  s-bar = grad F . gx   ocp_obj_hvp
The parameters and the upstream scalars stay on the device: the kernels read them through
pointers.
"""
from __future__ import annotations

import torch

from .ocp import OCP, _check, _raw_stream


def _zero_scalar(like):
    return torch.zeros(1, dtype=torch.float64, device=like.device)


class _ConsVJP(torch.autograd.Function):
    @staticmethod
    def forward(ctx, H: OCP, x, mu, w):
        ctx.H = H
        ctx.set_materialize_grads(False)
        ctx.save_for_backward(x, mu, w)
        w = w.contiguous()
        if H.nparams > 0:
            gx, gp = H.vjp_params(x, w, mu.reshape(-1))
            return gx, gp.reshape(mu.shape)
        return H.jtprod(x, w), torch.zeros_like(mu)

    @staticmethod
    def backward(ctx, ggx, ggmu):
        H = ctx.H
        x, mu, w = ctx.saved_tensors
        ggx = torch.zeros_like(x) if ggx is None else ggx.contiguous()
        if H.model == "vdp":
            s = _zero_scalar(x) if ggmu is None else ggmu.reshape(1).contiguous()
            dmu = torch.empty(1, dtype=torch.float64, device=x.device)
            with H.param0(mu.reshape(1)):
                dw = H.jprod_param(x, ggx, s)
                dx = H.hprod_param(x, w.contiguous(), 0.0, ggx, s, dmu=dmu)
            return None, dx, dmu.reshape(mu.shape), dw
        if H.nparams > 0 and (ggmu is not None or ctx.needs_input_grad[2]):
            raise NotImplementedError("second derivatives in the dynamics parameters are provided for the "
                                      "Van der Pol model; differentiate the %s model's J^T w in x only "
                                      "(parameters without requires_grad)" % H.model)
        if H.nparams > 0:
            with H.params_bound(mu.reshape(-1)):
                dw = H.jprod(x, ggx)
                dx = H.hprod(x, w.contiguous(), 0.0, ggx)
        else:
            dw = H.jprod(x, ggx)
            dx = H.hprod(x, w.contiguous(), 0.0, ggx)
        return None, dx, None, dw


def _cur_stream(t):
    """Handle of the current stream of t's device (the stream the autograd engine runs on)."""
    if _raw_stream is not None:
        return _raw_stream(t.get_device())
    return torch.cuda.current_stream(t.device).cuda_stream


class _Constraints(torch.autograd.Function):
    # The first-order path makes one C-ABI call each way with the arguments checked once in
    # constraints(): the step is host-bound at the sizes where autograd overhead matters.
    @staticmethod
    def forward(ctx, H: OCP, x, p):
        ctx.H = H
        ctx.save_for_backward(x, p)
        c = torch.empty(H.m, dtype=torch.float64, device=x.device)
        st = H._lib.ocp_eval_cons_params(H.h, x.data_ptr(), p.data_ptr() if H.nparams else None, c.data_ptr(),
                                         _cur_stream(x))
        if st:
            _check(st, H.h)
        return c

    @staticmethod
    def backward(ctx, gc):
        x, p = ctx.saved_tensors
        H = ctx.H
        if torch.is_grad_enabled():   # create_graph: the backward itself is differentiated
            return (None,) + _ConsVJP.apply(H, x, p, gc.contiguous())
        if not gc.is_contiguous():
            gc = gc.contiguous()
        gx = torch.empty_like(x)
        if H.nparams:   # one launch: J^T w at the parameters p and (dc/dp)^T w
            gp = torch.empty_like(p)
            st = H._lib.ocp_vjp_params(H.h, x.data_ptr(), gc.data_ptr(), p.data_ptr(), gx.data_ptr(), gp.data_ptr(),
                                       _cur_stream(x))
            if not ctx.needs_input_grad[2]:
                gp = None
        else:
            gp = None
            st = H._lib.jtprod(H.h, x.data_ptr(), gc.data_ptr(), gx.data_ptr(), _cur_stream(x))
        if st:
            _check(st, H.h)
        return None, gx, gp


class _ObjGrad(torch.autograd.Function):
    @staticmethod
    def forward(ctx, H: OCP, x, s):
        ctx.H = H
        ctx.save_for_backward(x, s)
        return H.eval_grad_scaled(x, s.reshape(1).contiguous())

    @staticmethod
    def backward(ctx, gg):
        x, s = ctx.saved_tensors
        dot = torch.empty(1, dtype=torch.float64, device=x.device)
        dx = ctx.H.obj_hvp(x, s.reshape(1).contiguous(), gg.contiguous(), dot=dot)
        return None, dx, dot.reshape(s.shape)


class _Objective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, H: OCP, x):
        ctx.H = H
        ctx.save_for_backward(x)
        return H.eval_obj(x).reshape(())

    @staticmethod
    def backward(ctx, gF):
        (x,) = ctx.saved_tensors
        return None, _ObjGrad.apply(ctx.H, x, gF.reshape(1))


def constraints(H: OCP, x: torch.Tensor, p: torch.Tensor) -> torch.Tensor:
    """c(x; p) with backward (J^T w, (dc/dp)^T w) and a double backward.  x: contiguous float64
    CUDA tensor of H.n entries; p: contiguous float64 CUDA tensor holding the model's H.nparams
    dynamics parameters (Van der Pol: mu alone; any shape); for models without parameters
    (double integrator, heat) p is not read and receives no gradient."""
    H._vec(x, H.n, "x")
    if H.nparams > 0:
        if p.dtype != torch.float64 or not p.is_cuda or not p.is_contiguous() or p.numel() != H.nparams:
            raise ValueError("p must be a contiguous float64 CUDA tensor of the %d dynamics parameters of the "
                             "%s model" % (H.nparams, H.model))
    return _Constraints.apply(H, x, p)


def objective(H: OCP, x: torch.Tensor) -> torch.Tensor:
    """F(x) with backward grad F and double backward Hess F v."""
    return _Objective.apply(H, x)
