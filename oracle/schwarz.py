"""One two-level overlapping Schwarz sweep as the FGMRES preconditioner.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Reading of how Algorithm 3 enters the outer flexible GMRES: the
preconditioner M(v) is one sweep of Algorithm 3 applied to the residual
equation A~ e = v from e = 0 (so every window starts with zero Robin data):
    r_w = R_w v                                 (partition)
    e_w = M.solve(r_w, g = 0)                   (local solves)
    u   = sum_w R~_w^T e_w                      (assemble, restricted)
    e_bc = traces of u on every window's interface sides (minus g = 0)
    z   = coarse solve of e_bc (Galerkin form, or Eq. 8),
    u  += sum_w R~_w^T sum_m z Phi
Local solves are the neural operator (product semantics) or exact SuperLU
solves of the local Robin problem (the ideal-preconditioner diagnostic).

Parity: the neural-operator sweep is the parity target of the GPU
preconditioner; its own pins are those of the modules it composes
(partition, nno, coarse).  Iteration counts of the outer solve are parity
unpinned (many preconditioners give the same converged answer).
"""
from __future__ import annotations

import numpy as np

from . import fdfd, krylov, nno
from .partition import Windows, restrict, prolong, traces, local_operator, local_rhs, WIN
from .coarse import CoarseSpace


class Schwarz:
    def __init__(self, eps, dx, wavelength, npml, weights=None, k_coarse: int = 0,
                 local: str = "nno", inner: int = 0, ritz_tol: float = 0.0,
                 coarse_form: str = "galerkin"):
        """local = "nno": neural local solves -- one application of the
        network to (residual, Robin data) when inner = 0, else `inner` steps
        of NN-preconditioned FGMRES (Algorithm 1) on the window's Robin
        problem; local = "exact": SuperLU local solves."""
        self.inner = inner
        ny, nx = eps.shape
        self.eps = np.asarray(eps, dtype=np.float32)
        self.dx, self.wavelength = dx, wavelength
        self.win = Windows(nx, ny)
        self.A = fdfd.assemble_operator(self.eps, dx, wavelength, npml)
        sxn, _, syn, _ = fdfd.pml_factors(nx, ny, dx, wavelength, npml)
        self.inv_sx, self.inv_sy = 1.0 / sxn, 1.0 / syn
        self.k2 = fdfd.k0dx_of(dx, wavelength) ** 2
        self.weights = weights
        self.local = local
        self._lu = None
        if local == "exact" or inner > 0:
            self._ops = [local_operator(self.win, w, self.A, self.eps, dx, wavelength)
                         for w in range(self.win.n)]
        if local == "exact":
            import scipy.sparse.linalg as spla
            self._lu = [spla.splu(op.tocsc()) for op, _ in self._ops]
        self.coarse = None
        if k_coarse > 0:
            zero = np.zeros((self.win.n, WIN, WIN), dtype=np.complex128)
            self.coarse = CoarseSpace(self.win, self.eps, dx, wavelength, k_coarse,
                                      lambda g: self.local_solve(zero, g), ritz_tol=ritz_tol,
                                      form=coarse_form)

    def aux(self, w: int):
        x0, y0 = int(self.win.x0[w]), int(self.win.y0[w])
        return (self.k2 * self.eps[y0:y0 + WIN, x0:x0 + WIN].astype(np.float64),
                self.inv_sx[x0:x0 + WIN], self.inv_sy[y0:y0 + WIN])

    def local_solve(self, r_loc: np.ndarray, g_loc: np.ndarray) -> np.ndarray:
        out = np.zeros((self.win.n, WIN, WIN), dtype=np.complex128)
        for w in range(self.win.n):
            if self.local == "exact":
                rhs = local_rhs(r_loc[w], g_loc[w], self._ops[w][1])
                out[w] = self._lu[w].solve(rhs).reshape(WIN, WIN)
            elif self.inner > 0:
                Aw, bnd = self._ops[w]
                rhs = local_rhs(r_loc[w], g_loc[w], bnd)
                k2e, isx, isy = self.aux(w)
                zero_g = np.zeros((4, WIN))
                M = lambda v, k2e=k2e, isx=isx, isy=isy: nno.solve(
                    v.reshape(WIN, WIN), zero_g, k2e, isx, isy, self.weights).ravel()
                x, _ = krylov.fgmres(lambda u, Aw=Aw: Aw @ u, rhs, precond=M, restart=self.inner,
                                     tol=0.0, max_iters=self.inner)
                out[w] = x.reshape(WIN, WIN)
            else:
                k2e, isx, isy = self.aux(w)
                out[w] = nno.solve(r_loc[w], g_loc[w], k2e, isx, isy, self.weights)
        return out

    def one_level(self, v: np.ndarray) -> np.ndarray:
        v = np.asarray(v, dtype=np.complex128).reshape(self.eps.shape)
        r_loc = restrict(self.win, v)
        g_loc = np.zeros((self.win.n, 4, WIN), dtype=np.complex128)
        return prolong(self.win, self.local_solve(r_loc, g_loc))

    def apply(self, v: np.ndarray) -> np.ndarray:
        u = self.one_level(v)
        if self.coarse is not None:
            e_bc = traces(self.win, u, self.eps, self.dx, self.wavelength)
            z = self.coarse.solve(e_bc)
            u = u + self.coarse.correction(z)
        return u

    def __call__(self, v):
        return self.apply(v).ravel()


def stationary_solve(S: Schwarz, b: np.ndarray, tol: float = 1e-6, max_iters: int = 200,
                     momentum: float = 0.0):
    """The literal domain-decomposition loop of Algorithm 3: local solves
    with the current Robin data, new data from the assembled field, momentum
    blend bc = m bc + (1-m) bc_new, and (two-level) the coarse correction of
    the boundary mismatch.  With the correction the corrected field's traces
    become the next data (bc_new + BQ z).  Returns (u, iterations, relres)."""
    ny, nx = S.eps.shape
    b = np.asarray(b, dtype=np.complex128).reshape(ny, nx)
    r_loc = restrict(S.win, b)
    bc = np.zeros((S.win.n, 4, WIN), dtype=np.complex128)
    rr = np.inf
    u = np.zeros((ny, nx), dtype=np.complex128)
    for it in range(1, max_iters + 1):
        u = prolong(S.win, S.local_solve(r_loc, bc))
        bc_new = traces(S.win, u, S.eps, S.dx, S.wavelength)
        if S.coarse is not None:
            z = S.coarse.solve(bc_new - bc)
            u = u + S.coarse.correction(z)
            bc_new = traces(S.win, u, S.eps, S.dx, S.wavelength)
        bc = momentum * bc + (1.0 - momentum) * bc_new
        rr = fdfd.relres(S.A, u.ravel(), b.ravel())
        if rr <= tol:
            return u, it, rr
    return u, max_iters, rr
