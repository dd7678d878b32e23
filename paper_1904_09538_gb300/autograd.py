"""Differentiable residual of a performance model for PyTorch.

Residual.apply(p, model, X, t) -> r with r_k = 1 - g(p; X_k) / t_k, computed
by the library's residual kernel; its backward is the library's adjoint
(vector-Jacobian product) kernel, reverse-mode over the model program.  X
(l x n_features), t (l) and p are float64 CUDA tensors; the kernels evaluate
in float-float arithmetic on the FP32 pipes.

lm_fit() is the plain per-model calibration (Section "Computing Model
Parameters"): a host-driven Levenberg-Marquardt loop over one model at a
time.  Each iteration takes J^T r from autograd through Residual (the adjoint
kernel), J from the Jacobian kernel, and hands them to the library's step
(pm_lm_step: damped normal-equation solve) and update (pm_lm_update: SSR,
accept / reject, damping, stopping) calls; the loop reads one status word per
trial and does no arithmetic itself.  The batched persistent-kernel path
(FitPlan) computes the same fit in one launch for many models.
"""
import ctypes

import numpy as np
import torch

from ._lib import lib, check, pm_fit_opts, pm_fit_report

LM_STATE_BYTES = 4096
LM_RUNNING = 1


def _cs():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(x):
    return ctypes.c_void_p(x.data_ptr())


def _check_inputs(p, X, t):
    if not (p.is_cuda and p.dtype == torch.float64 and X.dtype == torch.float64 and t.dtype == torch.float64):
        raise TypeError("Residual: p, X and t float64 CUDA tensors")


class Residual(torch.autograd.Function):
    @staticmethod
    def forward(ctx, p, model, X, t):
        _check_inputs(p, X, t)
        p, X, t = p.contiguous(), X.contiguous(), t.contiguous()
        r = torch.empty(t.shape[0], dtype=torch.float64, device=t.device)
        check(lib().pm_residual(model.handle, _ptr(X), _ptr(t), t.shape[0], _ptr(p), _ptr(r), _cs()))
        ctx.save_for_backward(p, X, t)
        ctx.model = model
        return r

    @staticmethod
    def backward(ctx, rbar):
        p, X, t = ctx.saved_tensors
        rbar = rbar.contiguous().to(torch.float64)
        pbar = torch.empty_like(p)
        check(lib().pm_residual_vjp(ctx.model.handle, _ptr(X), _ptr(t), t.shape[0], _ptr(p), _ptr(rbar),
                                    _ptr(pbar), _cs()))
        return pbar, None, None, None


def residual(model, X, t, p):
    return Residual.apply(p, model, X, t)


def jacobian(model, X, t, p):
    """J[k, i] = dr_k/dp_i (FP32, l x m) from the Jacobian kernel."""
    _check_inputs(p, X, t)
    J = torch.empty((t.shape[0], len(model.params)), dtype=torch.float32, device=t.device)
    check(lib().pm_jacobian(model.handle, _ptr(X), _ptr(t), t.shape[0], _ptr(p), _ptr(J), _cs()))
    return J


def lm_fit(model, X, t, p0, max_iter=200, ftol=1e-15, xtol=1e-12):
    """Plain per-model Levenberg-Marquardt through the autograd.Function.

    X: (l, nf) float64 CUDA, t: (l,) float64 CUDA, p0: start point (m,).
    Same damping and stopping rules as the batched fit (include/pm.h,
    pm_fit_opts).  Returns (p as numpy, report dict)."""
    dev = t.device
    m = len(model.params)
    l = t.shape[0]
    L = lib()
    p0 = np.ascontiguousarray(p0, dtype=np.float64)
    state = torch.empty(LM_STATE_BYTES, dtype=torch.uint8, device=dev)
    p = torch.empty(m, dtype=torch.float64, device=dev)
    p_try = torch.empty_like(p)
    flags = torch.zeros(2, dtype=torch.int32, device=dev)
    opts = pm_fit_opts(max_iter, ftol, xtol, 1)
    check(L.pm_lm_init(model.handle, p0.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(opts),
                       _ptr(state), _ptr(p), _cs()))
    status = LM_RUNNING if max_iter > 0 else -4
    while status == LM_RUNNING:
        pg = p.clone().requires_grad_(True)
        r = Residual.apply(pg, model, X, t)
        (b,) = torch.autograd.grad(r, pg, grad_outputs=r)      # J^T r by the adjoint kernel
        J = jacobian(model, X, t, pg.detach())
        r = r.detach()
        while True:
            check(L.pm_lm_step(_ptr(state), _ptr(r), _ptr(b), _ptr(J), l, _ptr(p_try), _cs()))
            with torch.no_grad():
                r_try = Residual.apply(p_try, model, X, t)
            check(L.pm_lm_update(_ptr(state), _ptr(r_try), l, _ptr(p), _ptr(flags), _cs()))
            status, accepted = flags.tolist()
            if status != LM_RUNNING or accepted:
                break
    rep = pm_fit_report()
    check(L.pm_lm_report(_ptr(state), ctypes.byref(rep), _cs()))
    return p.cpu().numpy(), {"status": rep.status, "iterations": rep.iterations, "residual": rep.residual,
                             "lambda": rep.lambda_}
