"""Differentiable solve for inverse design (Sec. 2.2, adjoint variable method).

`fdfd_field(solver, eps, J, ...)` returns E = A~(eps)^-1 b~(J) from the
library's FGMRES solve and, on backward, runs the library's adjoint solve on
A~^T with the same preconditioner and its dF/deps kernel; nothing of the
solve is traced by autograd (implicit differentiation, as the paper does to
keep the graph small for large problems).

Gradient convention: for a real loss L of the complex field E, PyTorch hands
backward grad_E = 2 conj(dL/dE) (conjugate Wirtinger, doubled).  With
g = dL/dE = conj(grad_E)/2 and A~^T lam = g,
    dL/deps_p = 2 Re(g . dE/deps_p) = -2 Re(lam_p (k0 dx)^2 E_p),
which is exactly what fdfd_grad_eps computes.
"""
from __future__ import annotations

import warnings

import torch

from . import fdfd as F

# statistics of the most recent forward and adjoint solves (for inspection)
last_stats = {"forward": None, "adjoint": None}


def _setup(solver, eps, weights, opts):
    """Load eps into the handle and redo its Schwarz set-up; every set-up
    bumps the handle's version so that a pending backward can tell whether
    the handle still holds the operator and preconditioner of its forward."""
    solver.set_eps(eps)
    if opts.get("precond", F.PRECOND_SCHWARZ) == F.PRECOND_SCHWARZ:
        solver.schwarz_setup(weights, k_coarse=opts.get("k_coarse", 0), inner_iters=opts.get("inner", 0),
                             ritz_tol=opts.get("ritz_tol", 0.0))
    solver._setup_version = getattr(solver, "_setup_version", 0) + 1
    return solver._setup_version


class _FieldSolve(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps, J, solver, weights, opts):
        eps_saved = eps.detach().contiguous().clone()
        version = _setup(solver, eps_saved, weights, opts)
        E = torch.zeros(J.shape, dtype=torch.complex64, device=J.device)
        kw = {k: v for k, v in opts.items() if k in ("restart", "max_iters", "tol", "precond")}
        rc, st = solver.solve(J, E, **kw)
        last_stats["forward"] = st
        if rc != F.OK:
            warnings.warn(f"forward solve: {F.status_string(rc)} (relres {st['relres_true']:.2e})")
        ctx.solver, ctx.kw, ctx.stats = solver, kw, st
        ctx.weights, ctx.opts, ctx.version = weights, opts, version
        ctx.save_for_backward(E, eps_saved)
        return E

    @staticmethod
    def backward(ctx, grad_E):
        E, eps_saved = ctx.saved_tensors
        S = ctx.solver
        # The adjoint needs A~(eps) of this forward solve: if the handle was
        # set up again since (another fdfd_field call on it), restore it.
        if getattr(S, "_setup_version", None) != ctx.version:
            ctx.version = _setup(S, eps_saved, ctx.weights, ctx.opts)
        g = torch.empty_like(E)
        S.adjoint_rhs(grad_E.to(torch.complex64).contiguous(), g)  # g = dL/dE = conj(grad_E) / 2
        lam = torch.zeros_like(E)
        rc, st = S.solve_adjoint(g, lam, **ctx.kw)
        last_stats["adjoint"] = st
        if rc != F.OK:
            warnings.warn(f"adjoint solve: {F.status_string(rc)} (relres {st['relres_true']:.2e})")
        grad = torch.empty(E.shape, dtype=torch.float32, device=E.device)
        S.grad_eps(E, lam, grad)
        return grad, None, None, None, None


def fdfd_field(solver: "F.Solver", eps: torch.Tensor, J: torch.Tensor, weights=None, **opts) -> torch.Tensor:
    """Field of the current density J in the permittivity eps (float32 CUDA
    tensor, may require grad).  opts: restart, max_iters, tol, precond,
    k_coarse, inner, ritz_tol (Schwarz set-up is redone for every new eps)."""
    return _FieldSolve.apply(eps, J, solver, weights, opts)


class _Overlap(torch.autograd.Function):
    @staticmethod
    def forward(ctx, E, mode, port_x, y0, dx):
        c = torch.empty(2, dtype=torch.float64, device=E.device)
        F.mode_overlap(E.to(torch.complex64).contiguous(), mode.contiguous(), port_x, y0, dx, c)
        ctx.shape, ctx.args = E.shape, (port_x, y0, dx)
        ctx.save_for_backward(mode)
        return torch.view_as_complex(c)

    @staticmethod
    def backward(ctx, grad_c):
        (mode,) = ctx.saved_tensors
        port_x, y0, dx = ctx.args
        grad_E = torch.empty(ctx.shape, dtype=torch.complex64, device=mode.device)
        F.mode_overlap_grad(ctx.shape, mode.contiguous(), port_x, y0, dx, complex(grad_c.item()), grad_E)
        return grad_E, None, None, None, None


def mode_overlap(E: torch.Tensor, port_x: int, mode: torch.Tensor, y0: int, dx: float) -> torch.Tensor:
    """c = dx sum_port conj(m) E along the vertical line x = port_x, from the
    library's overlap kernel (complex128 scalar tensor, differentiable in E:
    its backward is the library's chain-rule kernel)."""
    return _Overlap.apply(E, mode.to(torch.complex64), int(port_x), int(y0), float(dx))


class FDFDSolve:
    """Fields of one current density at several wavelengths, differentiable
    in eps: one library handle per wavelength (created on the first call, on
    eps's device), each solved by fdfd_field with the same options.

        solve = FDFDSolve(dx, [1.50e-6, 1.55e-6, 1.60e-6], weights, tol=1e-6)
        E1, E2, E3 = solve(eps, J)
    """

    def __init__(self, dx: float, wavelengths, weights=None, npml=20, **opts):
        self.dx, self.wavelengths = dx, list(wavelengths)
        self.weights, self.npml, self.opts = weights, npml, opts
        self.solvers = None
        self._key = None

    def __call__(self, eps: torch.Tensor, J: torch.Tensor):
        if eps.dim() != 2 or J.shape != eps.shape:
            raise ValueError("eps must be 2D and J of the same shape")
        key = (tuple(eps.shape), eps.device)
        if self.solvers is not None and key != self._key:
            self.close()  # another grid or device: new handles
        if self.solvers is None:
            self.solvers = [F.Solver(eps.detach().contiguous(), self.dx, lam, npml=self.npml)
                            for lam in self.wavelengths]
            self._key = key
        return [fdfd_field(S, eps, J, self.weights, **self.opts) for S in self.solvers]

    def close(self):
        """Free the per-wavelength handles (they are recreated on the next call)."""
        for S in self.solvers or []:
            S.close()
        self.solvers, self._key = None, None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
