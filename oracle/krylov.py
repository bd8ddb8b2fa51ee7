"""Flexible GMRES (Algorithm 1) in FP64, with restarts.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Algorithm 1 as printed: x0 = 0, r0 = b - A x0, beta = ||r0||, v1 = r0/beta;
for each j: z_j = M(v_j), w = A z_j, Gram-Schmidt of w against v_1..v_j
(h_ij = (w, v_i) = v_i^H w), h_{j+1,j} = ||w||, v_{j+1} = w / h_{j+1,j},
y_j = argmin ||beta e1 - H_j y||, x_j = x0 + Z_j y_j.  Two readings:
* the orthogonalisation line subtracts h_ij v_i (printed with v_j, a typo);
* the stop test uses the least-squares residual |g_{j+1}| (the printed
  test compares a vector with a scalar); converged solutions are confirmed
  with the true residual ||b - A x|| / ||b||, and the outer loop restarts
  every `restart` steps from the current x (restart 30 in the workloads).
The least-squares problem is solved with Givens rotations, the textbook way.

Parity: pinned in tests/test_oracle_krylov.py against the explicit minimal
residual over the Krylov space (dense least squares on tiny problems) and
against the direct solve.
"""
from __future__ import annotations

import numpy as np


def _givens(a: complex, b: complex):
    """Rotation [c s; -conj(s) c] with c real that zeroes b in (a, b)."""
    if b == 0:
        return 1.0, 0.0 + 0.0j
    if a == 0:
        return 0.0, np.conj(b) / abs(b)
    t = np.hypot(abs(a), abs(b))
    c = abs(a) / t
    s = (a / abs(a)) * np.conj(b) / t
    return c, s


def fgmres(matvec, b, precond=None, restart: int = 30, tol: float = 1e-6,
           max_iters: int = 1000, x0=None):
    """Returns (x, info) with info = dict(iters, restarts, history, relres).

    history[k] = least-squares residual estimate ||b - A x_k|| / ||b|| after
    k inner steps in total (k = 0 is the initial residual).  The true
    relative residual of the returned x is info['relres'].
    """
    b = np.asarray(b, dtype=np.complex128).ravel()
    n = b.size
    M = precond if precond is not None else (lambda v: v)
    x = np.zeros(n, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128).ravel()
    bnorm = np.linalg.norm(b)
    if bnorm == 0:
        return x, dict(iters=0, restarts=0, history=[0.0], relres=0.0, converged=True)
    r = b - matvec(x)
    beta = np.linalg.norm(r)
    history = [beta / bnorm]
    iters = 0
    restarts = 0
    while True:
        if beta / bnorm <= tol or iters >= max_iters:
            break
        m = restart
        V = np.zeros((m + 1, n), dtype=np.complex128)
        Z = np.zeros((m, n), dtype=np.complex128)
        H = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            Z[j] = M(V[j])
            w = matvec(Z[j])
            for i in range(j + 1):          # Gram-Schmidt against v_1..v_j
                H[i, j] = np.vdot(V[i], w)  # (w, v_i) = v_i^H w
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] != 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):              # apply earlier rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -np.conj(sn[i]) * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            cs[j], sn[j] = _givens(H[j, j], H[j + 1, j])
            H[j, j] = cs[j] * H[j, j] + sn[j] * H[j + 1, j]
            H[j + 1, j] = 0.0
            g[j + 1] = -np.conj(sn[j]) * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            iters += 1
            history.append(abs(g[j + 1]) / bnorm)
            if abs(g[j + 1]) / bnorm <= tol or iters >= max_iters:
                break
        # y = H_k^{-1} g_k (upper triangular after rotations)
        y = np.zeros(k, dtype=np.complex128)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - np.dot(H[i, i + 1:k], y[i + 1:k])) / H[i, i]
        x = x + Z[:k].T @ y
        r = b - matvec(x)
        beta = np.linalg.norm(r)
        restarts += 1
        if abs(g[k]) / bnorm <= tol and beta / bnorm > tol:
            history[-1] = beta / bnorm  # estimate fooled by rounding; keep going
    relres = beta / bnorm
    return x, dict(iters=iters, restarts=restarts, history=history, relres=relres,
                   converged=relres <= tol)
