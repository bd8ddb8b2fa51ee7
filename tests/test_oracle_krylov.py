"""Pins of the FGMRES oracle (Algorithm 1): minimal residual over the
Krylov space by explicit least squares, and convergence to the direct
solution with fixed and varying preconditioners."""
import numpy as np

from oracle import fdfd, krylov
from paper_2509_03622_gb300 import workloads as wl

LAM = 1.55e-6


def _problem(n=24, npml=4, seed=1):
    eps = wl.rectangles_eps(n, n, npml=npml, n_rect=4, seed=seed)
    A = fdfd.assemble_operator(eps, LAM / 25, LAM, npml=npml)
    b = fdfd.source_rhs(wl.random_field(n, n, seed + 1), LAM / 25, LAM)
    return A, b


def test_unpreconditioned_history_is_krylov_minimum():
    """history[k] = min_{x in K_k(A, b)} ||b - A x|| / ||b|| (brute force)."""
    A, b = _problem()
    _, info = krylov.fgmres(lambda v: A @ v, b, restart=30, tol=1e-14, max_iters=8)
    K = [b]
    for _ in range(7):
        K.append(A @ K[-1])
    K = np.array(K).T
    for k in range(1, 9):
        Q, _ = np.linalg.qr(K[:, :k])
        AQ = A @ Q
        y, *_ = np.linalg.lstsq(AQ, b, rcond=None)
        best = np.linalg.norm(b - AQ @ y) / np.linalg.norm(b)
        assert abs(info["history"][k] - best) < 1e-9 * max(best, 1e-3)


def test_restarted_reaches_direct_solution():
    """Restarted (restart 10) FGMRES with a complex-shifted-operator
    preconditioner (A - 0.3j I)^-1 reaches the direct solution."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    A, b = _problem(n=32, npml=6, seed=4)
    lu = spla.splu((A - 0.3j * sp.identity(A.shape[0])).tocsc())
    x, info = krylov.fgmres(lambda v: A @ v, b, precond=lu.solve,
                            restart=10, tol=1e-11, max_iters=3000)
    xs = fdfd.DirectSolver(A).solve(b)
    assert info["converged"] and info["restarts"] >= 2
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-8


def test_flexible_varying_preconditioner():
    """A preconditioner that changes every step (flexible GMRES) still
    converges to the unique solution and the estimate tracks the truth."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spla
    A, b = _problem(n=24, npml=4, seed=8)
    lu = spla.splu((A - 0.3j * sp.identity(A.shape[0])).tocsc())
    state = {"k": 0}

    def M(v):
        state["k"] += 1
        z = lu.solve(v)
        return z if state["k"] % 2 else np.tanh(np.abs(z)) * z  # nonlinear

    x, info = krylov.fgmres(lambda v: A @ v, b, precond=M, restart=30, tol=1e-10, max_iters=3000)
    xs = fdfd.DirectSolver(A).solve(b)
    assert info["converged"]
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-7
    assert fdfd.relres(A, x, b) <= 1e-10
