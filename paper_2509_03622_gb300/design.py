"""Inverse design on the library's kernels (Sec. 2.2: density-based
optimisation with filtering, projection and Adam; gradients from the adjoint
solve).  Marshalling only: the filter, projection, chain rule and Adam update
run in fdfd_design_eps / fdfd_design_grad / fdfd_adam_step.

    D = Design(solver, x0, y0, w, h, radius=3, beta=8)
    eps = density_to_eps(D, rho, eps_base)      # differentiable in rho
    E = fdfd_field(solver, eps, J, weights)     # autograd.py
    F = figure_of_merit(E); F.backward()        # rho.grad = dF/drho
    opt.step(rho, rho.grad, scale=1 / F0)       # Adam ascent on the GPU
"""
from __future__ import annotations

import ctypes as C

import torch

from . import fdfd as F


def _ptr(t: torch.Tensor):
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError("expected a contiguous float32 CUDA tensor")
    return C.c_void_p(t.data_ptr())


class Design:
    """Rectangle (x0, y0, w, h) of the grid and its filter / projection."""

    def __init__(self, solver: "F.Solver", x0: int, y0: int, w: int, h: int, radius: float = 3.0,
                 beta: float = 8.0, eta: float = 0.5, eps_lo: float = 2.1, eps_hi: float = 12.25):
        self.solver = solver
        self.d = F.DesignDesc(x0, y0, w, h, radius, beta, eta, eps_lo, eps_hi)
        self.shape = (h, w)
        self.rho_f = None

    def set_beta(self, beta: float):
        self.d.beta = beta

    def eps(self, rho: torch.Tensor, eps: torch.Tensor) -> torch.Tensor:
        """Writes the rectangle of eps (in place) from rho; keeps rho_f."""
        self.rho_f = torch.empty(self.shape, dtype=torch.float32, device=rho.device)
        F._check(F.lib.fdfd_design_eps(self.solver.h, C.byref(self.d), _ptr(rho), _ptr(self.rho_f), _ptr(eps)),
                 "fdfd_design_eps")
        return eps

    def grad(self, g_eps: torch.Tensor) -> torch.Tensor:
        """dF/drho from dF/deps over the grid (after eps() of the same rho)."""
        work = torch.empty(self.shape, dtype=torch.float32, device=g_eps.device)
        g_rho = torch.empty_like(work)
        F._check(F.lib.fdfd_design_grad(self.solver.h, C.byref(self.d), _ptr(self.rho_f), _ptr(g_eps),
                                        _ptr(work), _ptr(g_rho)), "fdfd_design_grad")
        return g_rho


class _DensityToEps(torch.autograd.Function):
    @staticmethod
    def forward(ctx, rho, eps_base, design):
        eps = eps_base.detach().clone().contiguous()
        design.eps(rho.detach().contiguous(), eps)
        ctx.design = design
        return eps

    @staticmethod
    def backward(ctx, g_eps):
        return ctx.design.grad(g_eps.contiguous().float()), None, None


def density_to_eps(design: Design, rho: torch.Tensor, eps_base: torch.Tensor) -> torch.Tensor:
    """Permittivity of the grid with the design rectangle set from rho
    (differentiable in rho; eps_base supplies everything else)."""
    return _DensityToEps.apply(rho, eps_base, design)


class Adam:
    """Adam ascent of a figure of merit on the GPU (moments kept here)."""

    def __init__(self, solver: "F.Solver", shape, lr: float = 0.01, beta1: float = 0.9, beta2: float = 0.999,
                 eps: float = 1e-8, device="cuda"):
        self.solver = solver
        self.a = F.AdamDesc(lr, beta1, beta2, eps)
        self.m = torch.zeros(shape, dtype=torch.float32, device=device)
        self.v = torch.zeros_like(self.m)
        self.t = 0

    def step(self, theta: torch.Tensor, g: torch.Tensor, scale: float = 1.0):
        """theta += Adam step along scale * g, in place, clipped to [0, 1]."""
        self.t += 1
        g = g.contiguous().float()
        F._check(F.lib.fdfd_adam_step(self.solver.h, C.byref(self.a), self.t, float(scale), _ptr(theta), _ptr(g),
                                      _ptr(self.m), _ptr(self.v), theta.numel()), "fdfd_adam_step")
        return theta
