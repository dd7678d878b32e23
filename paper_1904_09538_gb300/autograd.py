"""Differentiable residual of a performance model for PyTorch.

Residual.apply(p, model, X, t) -> r with r_k = 1 - g(p; X_k) / t_k, computed
by the library's residual kernel; its backward is the library's adjoint
(vector-Jacobian product) kernel, reverse-mode over the model program.

lm_fit() is the plain per-model calibration: a host-driven Levenberg-Marquardt
loop (one model at a time) whose J^T r comes from autograd through Residual
and whose J^T J comes from the adjoint kernel applied to J's columns
(Section "Computing Model Parameters").  The batched persistent-kernel path
(FitPlan) computes the same fit in one launch for many models.
"""
import ctypes

import numpy as np
import torch

from ._lib import lib, check


def _cs():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


class Residual(torch.autograd.Function):
    @staticmethod
    def forward(ctx, p, model, X, t):
        if not (p.is_cuda and p.dtype == torch.float64 and X.dtype == torch.float32 and t.dtype == torch.float32):
            raise TypeError("Residual: p float64, X and t float32, all CUDA")
        p, X, t = p.contiguous(), X.contiguous(), t.contiguous()
        r = torch.empty(t.shape[0], dtype=torch.float32, device=t.device)
        check(lib().pm_residual(model.handle, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                t.shape[0], ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(r.data_ptr()), _cs()))
        ctx.save_for_backward(p, X, t)
        ctx.model = model
        return r

    @staticmethod
    def backward(ctx, rbar):
        p, X, t = ctx.saved_tensors
        rbar = rbar.contiguous().to(torch.float32)
        pbar = torch.empty_like(p)
        check(lib().pm_residual_vjp(ctx.model.handle, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                    t.shape[0], ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(rbar.data_ptr()),
                                    ctypes.c_void_p(pbar.data_ptr()), _cs()))
        return pbar, None, None, None


def residual(model, X, t, p):
    return Residual.apply(p, model, X, t)


def jacobian(model, X, t, p):
    """J[k, i] = dr_k/dp_i (FP32, l x m) from the Jacobian kernel."""
    J = torch.empty((t.shape[0], len(model.params)), dtype=torch.float32, device=t.device)
    check(lib().pm_jacobian(model.handle, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(t.data_ptr()), t.shape[0],
                            ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(J.data_ptr()), _cs()))
    return J


def _jtv(model, X, t, p, v):
    pbar = torch.empty_like(p)
    v = v.contiguous().to(torch.float32)
    check(lib().pm_residual_vjp(model.handle, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                t.shape[0], ctypes.c_void_p(p.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                                ctypes.c_void_p(pbar.data_ptr()), _cs()))
    return pbar


def lm_fit(model, X, t, p0, max_iter=200, xtol=1e-12):
    """Plain per-model Levenberg-Marquardt through the autograd.Function.

    X: (l, nf) float32 CUDA, t: (l,) float32 CUDA, p0: start point (m,).
    Scaled coordinates q = p / |p0|, Marquardt damping diag(J^T J), lambda
    x10 on rejection, /10 on acceptance; steps whose predicted SSR decrease is
    below the FP32 noise floor are accepted and end the fit.  Returns
    (p as numpy, iterations)."""
    dev = t.device
    p0 = torch.as_tensor(np.asarray(p0, dtype=np.float64), device=dev)
    s = torch.where(p0 != 0, p0.abs(), torch.ones_like(p0))
    q = p0 / s
    lam = 1e-3
    l = t.shape[0]
    eps = 5.9604645e-8
    it = 0

    def ssr_b_A(q):
        p = (q * s).detach().requires_grad_(True)
        r = Residual.apply(p, model, X, t)
        (b,) = torch.autograd.grad(r, p, grad_outputs=r)          # J^T r via the adjoint kernel
        J = jacobian(model, X, t, p.detach())
        A = torch.stack([_jtv(model, X, t, p.detach(), J[:, i]) for i in range(J.shape[1])], dim=1)
        Sd = s
        return float((r.detach().double() ** 2).sum()), b * Sd, A * Sd[:, None] * Sd[None, :]

    ssr, b, A = ssr_b_A(q)
    for it in range(1, max_iter + 1):
        noise = 4 * eps * (l * ssr) ** 0.5 + l * eps * eps
        d = torch.diagonal(A).clamp_min(1e-300)
        accepted = False
        for _ in range(16):
            Ah = A / torch.sqrt(d[:, None] * d[None, :]) + lam * torch.eye(A.shape[0], dtype=A.dtype, device=dev)
            y = torch.linalg.solve(Ah, -b / torch.sqrt(d))
            dq = y / torch.sqrt(d)
            pred = float(-(2 * dq @ b + dq @ A @ dq))
            p_try = ((q + dq) * s)
            with torch.no_grad():
                r_try = Residual.apply(p_try, model, X, t)
            sn = float((r_try.double() ** 2).sum())
            if np.isfinite(sn) and (sn <= ssr or pred <= noise):
                accepted = True
                break
            lam *= 10
        if not accepted:
            break
        q = q + dq
        lam = max(lam * 0.1, 1e-12)
        ssr_old = ssr
        ssr, b, A = ssr_b_A(q)
        if float(dq.norm()) <= xtol * (float(q.norm()) + xtol) or pred <= noise or ssr_old - ssr <= 1e-15 * ssr_old:
            break
    return (q * s).cpu().numpy(), it
