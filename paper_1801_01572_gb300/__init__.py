"""GB300 (sm_103a) global point-cloud registration of LoopSmart (arXiv 1801.01572).

The registration path (Sec. IV, Algorithm 1, eq. (1), eq. (3)-(5)) runs in the
CUDA library ``_lib/liblsr.so`` behind the C ABI of ``include/lsr.h``; this
package only marshals arguments (``lsr.py``) and wraps the robust alignment
objective and its hand-written adjoint in a ``torch.autograd.Function``.
"""
from __future__ import annotations

from .lsr import (DESC_DIM, LSR_E_ARG, LSR_E_CUDA, LSR_E_OOM, LSR_E_STATE, LSR_E_TIMEOUT, LSR_E_TOO_LARGE,  # noqa: F401
                  LSR_OK,
                  MATCH_BF16, MATCH_BF16_PLAIN, MATCH_FP32, NN_EXACT, NN_SINGLE_CELL, NORMALS_INLIERS, NORMALS_SAMPLES, STATUS_ALIGNED, STATUS_NO_ALIGNMENT, ABI_FUNCTIONS, Context, LsrError,
                  Params, Registration, context, default_params, launch_count, lib, library_path, register_pair,
                  transfer_bytes, INJECT_ALLOC, INJECT_CHECK, INJECT_MATCH_STALL, INJECT_NONE, LSR_E_CHECK)


def _torch():
    import torch
    return torch


class RobustAlignBatch:
    """E_i(xi_i) = sum_j rho~(|T(xi_i) p_j - q_nn(j)|^2) for n pairs, differentiable in the
    points and the 6-vector poses xi = (alpha, beta, gamma, x, y, z), T(xi) = [Exp(w) | v] T0.

    ``apply(xis, T0s, eps, mu, ctx, P0, Q0, P1, Q1, ...)`` with P_i, Q_i CUDA float32 (N, 3)
    tensors, xis (n, 6) float64, T0s (n, 4, 4) float64; returns E (n,) float64.
    The backward recomputes the nearest neighbours on the device (nothing is stored).
    """

    _fn = None

    @classmethod
    def function(cls):
        if cls._fn is None:
            torch = _torch()

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(fctx, xis, T0s, eps, mu, lctx, *clouds):
                    Ps, Qs = list(clouds[0::2]), list(clouds[1::2])
                    E = lctx.objective_fwd(Ps, Qs, xis.detach().cpu().numpy(), T0s.detach().cpu().numpy(), eps, mu)
                    fctx.save_for_backward(xis, T0s, *clouds)
                    fctx.eps, fctx.mu, fctx.lctx = eps, mu, lctx
                    return torch.as_tensor(E, dtype=torch.float64, device=xis.device)

                @staticmethod
                def backward(fctx, gE):
                    xis, T0s, *clouds = fctx.saved_tensors
                    Ps, Qs = list(clouds[0::2]), list(clouds[1::2])
                    dPs = [torch.empty_like(p, dtype=torch.float32) for p in Ps]
                    dQs = [torch.empty_like(q, dtype=torch.float32) for q in Qs]
                    dxi = fctx.lctx.objective_bwd([p.contiguous() for p in Ps], [q.contiguous() for q in Qs],
                                                  xis.detach().cpu().numpy(), T0s.detach().cpu().numpy(),
                                                  gE.detach().cpu().numpy(), dPs, dQs, fctx.eps, fctx.mu)
                    grads = []
                    for dp, dq in zip(dPs, dQs):
                        grads += [dp, dq]
                    return (torch.as_tensor(dxi, dtype=xis.dtype, device=xis.device), None, None, None, None, *grads)

            cls._fn = _F
        return cls._fn

    @classmethod
    def apply(cls, xis, T0s, eps, mu, lctx, *clouds):
        return cls.function().apply(xis, T0s, eps, mu, lctx, *clouds)


class RefinedPose:
    """T* = the graduated robust refinement of T0 (lsr_stage_refine: the
    Geman-McClure IRLS of eq. (3)-(5)), differentiable in the points.

    ``apply(P, Q, T0, eps, mu_scale, levels, iters, lctx)`` with P, Q CUDA
    float32 (N, 3) tensors and T0 a (4, 4) float64 tensor; returns T* (4, 4)
    float64. The backward differentiates the optimality condition at T*
    (lsr_pose_implicit_grad, on the finest level's pairs, recomputed): the
    gradient reaches P and Q; T0 gets none (the optimum does not move with the
    start inside its basin)."""

    _fn = None

    @classmethod
    def function(cls):
        if cls._fn is None:
            torch = _torch()

            class _F(torch.autograd.Function):
                @staticmethod
                def forward(fctx, P, Q, T0, eps, mu_scale, levels, iters, lctx):
                    T, _ = lctx.stage_refine(P.detach(), Q.detach(), T0.detach().cpu().numpy(), eps, mu_scale,
                                             levels, iters)
                    Tt = torch.as_tensor(T, dtype=torch.float64, device=T0.device)
                    fctx.save_for_backward(P, Q, Tt)
                    fctx.eps, fctx.mu, fctx.lctx = eps, mu_scale * eps * eps, lctx
                    return Tt

                @staticmethod
                def backward(fctx, gT):
                    P, Q, Tt = fctx.saved_tensors
                    dP = torch.empty(P.shape, dtype=torch.float32, device=P.device)
                    dQ = torch.empty(Q.shape, dtype=torch.float32, device=Q.device)
                    fctx.lctx.pose_implicit_grad(P.detach().contiguous(), Q.detach().contiguous(),
                                                 Tt.detach().cpu().numpy(), gT.detach().cpu().numpy(), fctx.eps,
                                                 fctx.mu, dP, dQ)
                    return dP.to(P.dtype), dQ.to(Q.dtype), None, None, None, None, None, None

            cls._fn = _F
        return cls._fn

    @classmethod
    def apply(cls, P, Q, T0, eps=0.0375, mu_scale=1.0, levels=3, iters=50, lctx=None):
        lctx = lctx or context(P.device.index or 0)
        return cls.function().apply(P, Q, T0, eps, mu_scale, levels, iters, lctx)


def robust_align(P, Q, xi, T0, eps: float = 0.0375, mu: float | None = None, lctx: Context | None = None):
    """Single-pair objective E(xi) as a differentiable torch scalar (float64)."""
    torch = _torch()
    mu = eps * eps if mu is None else mu
    lctx = lctx or context(P.device.index or 0)
    T0 = torch.as_tensor(T0, dtype=torch.float64).reshape(1, 4, 4)
    return RobustAlignBatch.apply(xi.reshape(1, 6), T0, eps, mu, lctx, P, Q)[0]
