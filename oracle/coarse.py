"""Coarse space of the two-level Schwarz method (Sec. 2.2, Methods,
Algorithm 3 set-up and correction, Eq. 7-8), FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Set-up, in the order of Algorithm 3:
1. pseudo-plane-wave trial Robin data: for k directions theta_m = 2 pi m / k
   walk the window perimeter counter-clockwise from its (x-, y-) corner and
   accumulate the phase phi += kd * (d . ds), kd = k0 dx sqrt(eps) averaged
   over the two cells of the step; the trial datum is exp(-j phi) on every
   interface slot (Methods: "compute the wave vector inside the medium ...
   accumulate the phase around the boundary");
2. Gram-Schmidt (modified, l2 over the slots) per window -> Q_w;
3. homogeneous local solves with Robin data q_{w,m}: Phi_{w,m} = M.solve;
4. traces of the restricted basis fields on the neighbours' boundaries
   (extract_neighboring_bc) -> the columns of B Q;
5. assemble and factor the coarse matrix (the Galerkin G, or the normal
   matrix of Eq. 8; see "Coarse equation" below).
The Rayleigh-Ritz step (eig of (x, y)) keeping all k Ritz vectors leaves
span(Q) and hence the correction unchanged, so by default it is omitted
(reading).  With ritz_tol > 0 the basis is truncated instead:
6. H_w = (x, y) over the trials of window w, where y = B x is the Robin
   data the window's basis field hands to each neighbour, read on that
   neighbour's side facing w and identified with w's own side
   (robin_to_robin).  With orthonormal trials H_w = Q_w^H B Q_w is the
   Rayleigh-Ritz matrix; its eigenpairs H_w u = eta u give the Ritz vectors
   Q_w u.  Q_w, Phi_w and the window's columns of C are combined by the
   eigenvectors with |eta| >= ritz_tol (the fields are combined linearly,
   not solved again) and the other directions are dropped (Sec. 2.2: the
   slowly decaying modes, those with the largest eta, above a threshold span
   the coarse space).

Coarse equation (reading of Eq. 7): after adding sum_m z_{w,m} Phi_{w,m} to
window w the boundary mismatch becomes e_bc + (BQ - Q) z with C = BQ - Q.
Two ways of choosing z from that mismatch are built:
* form = "galerkin" (default): the mismatch left after the correction is
  made orthogonal to the coarse trial space itself, Q^H (e_bc + C z) = 0,
  i.e. the square system  G z = -Q^H e_bc  with  G = Q^H C  -- the
  Rayleigh-Ritz (Galerkin) projection of the interface operator B - I onto
  span(Q), in the spirit of the Rayleigh-Ritz step of Algorithm 3.  G has a
  9-block stencil over the window grid (window w's test functions see the
  basis of w and of its 8 neighbours);
* form = "normal": the least-squares fit  min || C z + e_bc ||  through the
  normal equations of Eq. 8,  C^H C z = -C^H e_bc  (25-block stencil).
With exact local Robin solves the Galerkin form is the one that makes the
two-level preconditioner scale (FGMRES(30) to 1e-6 on the freeform 256^2
grid, k = 64: 11 iterations against 107 for the normal equations and 353
for one level; 512^2: 24 against 1219 one-level).

Trials that Gram-Schmidt finds exactly dependent are dropped (zero basis
vector, zero field); their coefficients are pinned to zero by a unit
diagonal in the normal matrix.

Parity: pinned in tests/test_oracle_coarse.py (normal-equation solve equals
numpy.linalg.lstsq; the Galerkin correction leaves a mismatch orthogonal
to every trial vector of every window; both forms remove a mismatch that
lies in the range of C exactly; the Galerkin two-level FGMRES iteration
count stays nearly flat from 4 x 4 to 8 x 8 windows while one level
grows; Gram-Schmidt orthonormality; exact plane-wave phase on a
homogeneous window; the Ritz step: keeping every direction leaves the
correction unchanged, truncation equals least squares over the kept
columns, |eta| <= 1 with a strongly transmitting interior window in a
lossless medium, and the truncated two-level loop still converges).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .partition import Windows, WIN, CORE, SIDES, traces, kd_map


def perimeter_walk(win: Windows, w: int):
    """Counter-clockwise list of (side, t, gx, gy) around window w."""
    x0, y0 = int(win.x0[w]), int(win.y0[w])
    walk = []
    for t in range(WIN):
        walk.append((2, t, x0 + t, y0))
    for t in range(WIN):
        walk.append((1, t, x0 + WIN - 1, y0 + t))
    for t in range(WIN - 1, -1, -1):
        walk.append((3, t, x0 + t, y0 + WIN - 1))
    for t in range(WIN - 1, -1, -1):
        walk.append((0, t, x0, y0 + t))
    return walk


def plane_wave_trials(win: Windows, eps, dx, wavelength, k: int) -> np.ndarray:
    """[n_win][k][4][80] trial Robin data (zero on grid-edge sides)."""
    kd = kd_map(eps, dx, wavelength)
    out = np.zeros((win.n, k, SIDES, WIN), dtype=np.complex128)
    for w in range(win.n):
        walk = perimeter_walk(win, w)
        for m in range(k):
            th = 2.0 * np.pi * m / k
            d = np.array([np.cos(th), np.sin(th)])
            phi = 0.0
            prev = None
            for (s, t, gx, gy) in walk:
                if prev is not None:
                    px, py = prev
                    step = np.array([gx - px, gy - py], dtype=np.float64)
                    kav = 0.5 * (kd[py, px] + kd[gy, gx])
                    phi += kav * float(d @ step)
                prev = (gx, gy)
                if win.interface[w, s]:
                    out[w, m, s, t] = np.exp(-1j * phi)
    return out


def gram_schmidt(X: np.ndarray, drop_tol: float = 1e-10) -> np.ndarray:
    """Modified Gram-Schmidt of the k rows of each window's [k][320] block."""
    nw, k = X.shape[:2]
    Q = X.reshape(nw, k, -1).astype(np.complex128).copy()
    for w in range(nw):
        for m in range(k):
            v = Q[w, m]
            n0 = np.linalg.norm(v)
            for i in range(m):
                v = v - np.vdot(Q[w, i], v) * Q[w, i]
            nv = np.linalg.norm(v)
            Q[w, m] = 0.0 if (n0 == 0 or nv <= drop_tol * n0) else v / nv
    return Q.reshape(X.shape)


class CoarseSpace:
    """Q, Phi, C = BQ - Q and the factored coarse matrix (G = Q^H C, or the
    normal matrix C^H C)."""

    def __init__(self, win: Windows, eps, dx, wavelength, k: int, local_solve, ritz_tol: float = 0.0,
                 form: str = "galerkin"):
        """local_solve(g [n_win][4][80]) -> fields [n_win][80][80]: the
        homogeneous (zero-source) local Robin solver of every window.
        ritz_tol > 0: keep per window the Ritz vectors of the Robin-to-Robin
        map whose eigenvalue has modulus >= ritz_tol (step 6 above).
        form: "galerkin" (G z = -Q^H e_bc) or "normal" (Eq. 8)."""
        if form not in ("galerkin", "normal"):
            raise ValueError(form)
        self.form = form
        self.win, self.k = win, k
        self.eps, self.dx, self.wavelength = eps, dx, wavelength
        X = plane_wave_trials(win, eps, dx, wavelength, k)
        self.Q = gram_schmidt(X)                       # [n][k][4][80]
        self.Phi = np.zeros((win.n, k, WIN, WIN), dtype=np.complex128)
        for m in range(k):
            self.Phi[:, m] = local_solve(self.Q[:, m])
        self.C = self.assemble_C()
        self.eta = None
        if ritz_tol > 0.0:
            self.truncate(ritz_tol)
        # Trial vectors removed by Gram-Schmidt (exactly dependent trials,
        # e.g. symmetric direction sets on a corner window's two sides) give
        # zero columns; their unknowns are pinned to z = 0 by a unit diagonal.
        self.dropped = ~np.any(self.Q.reshape(win.n * k, -1), axis=1)
        if form == "normal":
            self.N = self.C.conj().T @ self.C
            self.N[self.dropped, self.dropped] = 1.0
            self.L = np.linalg.cholesky(self.N)
        else:
            self.G = self.test_space().conj().T @ self.C
            self.G[self.dropped, self.dropped] = 1.0
            self.G_lu = sla.lu_factor(self.G)

    def test_space(self) -> np.ndarray:
        """The trial data as a [n_win*320][n_win*k] matrix: window w's basis
        vectors on w's own slots (the test functions of the Galerkin form)."""
        win, k = self.win, self.k
        T = np.zeros((win.n * SIDES * WIN, win.n * k), dtype=np.complex128)
        for w in range(win.n):
            T[w * SIDES * WIN:(w + 1) * SIDES * WIN, w * k:(w + 1) * k] = self.Q[w].reshape(k, -1).T
        return T

    def robin_to_robin(self, w: int) -> np.ndarray:
        """Y_w [k][4][80]: for each interface side s of window w, the trace
        that each basis field of w leaves on the neighbour across s, on that
        neighbour's side facing w (read from C, whose rows off window w hold
        the traces alone)."""
        win, k = self.win, self.k
        a, b = w % win.nwx, w // win.nwx
        across = {0: (a - 1, b, 1), 1: (a + 1, b, 0), 2: (a, b - 1, 3), 3: (a, b + 1, 2)}
        Y = np.zeros((k, SIDES, WIN), dtype=np.complex128)
        for s, (ai, bi, facing) in across.items():
            if not win.interface[w, s]:
                continue
            i = bi * win.nwx + ai
            r0 = (i * SIDES + facing) * WIN
            Y[:, s, :] = self.C[r0:r0 + WIN, w * k:(w + 1) * k].T
        return Y

    def ritz_matrix(self, w: int) -> np.ndarray:
        """H_w[p, q] = (q_p, y_q) = sum conj(Q_w[p]) Y_w[q] (k x k)."""
        k = self.k
        return self.Q[w].reshape(k, -1).conj() @ self.robin_to_robin(w).reshape(k, -1).T

    def truncate(self, ritz_tol: float) -> None:
        """Step 6: per window, the eigenpairs H u = eta u of the Ritz matrix;
        Q, Phi and the window's columns of C are combined by the eigenvectors
        with |eta| >= ritz_tol, the other directions become zero columns
        (their unknowns are then pinned like dropped trials)."""
        win, k = self.win, self.k
        H = [self.ritz_matrix(w) for w in range(win.n)]  # all from the untruncated C
        self.eta = np.zeros((win.n, k), dtype=np.complex128)
        for w in range(win.n):
            eta, U = np.linalg.eig(H[w])
            U = U * (np.abs(eta) >= ritz_tol)[None, :]
            self.eta[w] = eta
            self.Q[w] = np.einsum("mq,msl->qsl", U, self.Q[w])
            self.Phi[w] = np.einsum("mq,myx->qyx", U, self.Phi[w])
            cols = slice(w * k, (w + 1) * k)
            self.C[:, cols] = self.C[:, cols] @ U

    def restricted_field(self, w: int, f_loc: np.ndarray) -> np.ndarray:
        """R~_w^T f: window field placed on w's core only."""
        win = self.win
        u = np.zeros((win.ny, win.nx), dtype=np.complex128)
        cx, cy = win.core_offset(w)
        a, b = w % win.nwx, w // win.nwx
        u[CORE * b:CORE * b + CORE, CORE * a:CORE * a + CORE] = f_loc[cy:cy + CORE, cx:cx + CORE]
        return u

    def assemble_C(self) -> np.ndarray:
        win, k = self.win, self.k
        nrow = win.n * SIDES * WIN
        C = np.zeros((nrow, win.n * k), dtype=np.complex128)
        for w in range(win.n):
            for m in range(k):
                u = self.restricted_field(w, self.Phi[w, m])
                col = traces(win, u, self.eps, self.dx, self.wavelength).ravel()
                q = np.zeros((win.n, SIDES, WIN), dtype=np.complex128)
                q[w] = self.Q[w, m]
                C[:, w * k + m] = col - q.ravel()
        return C

    def solve(self, e_bc: np.ndarray) -> np.ndarray:
        """Galerkin: z = G^{-1} (-Q^H e_bc) (LU with partial pivoting).
        Normal: z = (C^H C)^{-1} (-C^H e_bc) via the Cholesky factor (Eq. 8)."""
        if self.form == "galerkin":
            rhs = -self.test_space().conj().T @ e_bc.ravel()
            rhs[self.dropped] = 0.0
            return sla.lu_solve(self.G_lu, rhs)
        rhs = -self.C.conj().T @ e_bc.ravel()
        rhs[self.dropped] = 0.0
        y = sla.solve_triangular(self.L, rhs, lower=True)
        return sla.solve_triangular(self.L.conj().T, y, lower=False)

    def correction(self, z: np.ndarray) -> np.ndarray:
        """sum_w R~_w^T sum_m z_{w,m} Phi_{w,m} as a global field."""
        win, k = self.win, self.k
        loc = np.einsum("wm,wmyx->wyx", z.reshape(win.n, k), self.Phi)
        u = np.zeros((win.ny, win.nx), dtype=np.complex128)
        for w in range(win.n):
            u += self.restricted_field(w, loc[w])
        return u
