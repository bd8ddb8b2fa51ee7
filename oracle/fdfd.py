"""FDFD operator for 2D Ez (Eq. 1) with the stretched-coordinate PML of
Methods (UPML, Eq. 3-6); FP64, scipy.sparse, SuperLU.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Conventions (the paper's readings, all stated where they are used):
* time dependence e^{+j w t}: the UPML factor s = 1 + sigma/(j w eps0)
  (Methods) absorbs outgoing e^{-j k r} waves only under this convention;
* grid arrays are [ny][nx] (x fastest); cell (i, j) has its centre at
  x = (i + 1/2) dx and faces at x = i dx, x = (i + 1) dx;
* field outside the grid is zero (Dirichlet backing behind the PML);
* the linear system is Eq. 1 multiplied by dx^2, so
      A~ = L~x + L~y + (k0 dx)^2 diag(eps),    b~ = dx^2 j w mu0 J.

Parity: pinned by closed forms and invariants in tests/test_oracle_fdfd.py
(discrete sine-mode eigenvalues, dense brute force, 2D Hankel Green's
function with 2nd-order convergence, reciprocity, Poynting balance,
finite-difference gradient).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
from scipy import constants as C

MU0 = C.mu_0
EPS0 = C.epsilon_0
C0 = C.c
ETA0 = np.sqrt(MU0 / EPS0)


def omega_of(wavelength: float) -> float:
    return 2.0 * np.pi * C0 / wavelength


def k0dx_of(dx: float, wavelength: float) -> float:
    return 2.0 * np.pi * dx / wavelength


def pml_stretch(n: int, npml_lo: int, npml_hi: int, dx: float, wavelength: float,
                m: float = 3.0, lnR: float = -30.0):
    """UPML stretching factors along one axis (Methods, Eq. 6).

    s(zeta) = 1 + sigma(zeta) / (j w eps0),  sigma = sigma_max (zeta/d)^m,
    sigma_max = -(m+1) ln R / (2 eta0 d), d = npml * dx (the garbled
    "2 eta0 d zeta" read as 2 eta0 d).  zeta is the depth into the PML
    measured from its inner interface.  Returns (s_node[n], s_half[n+1]):
    s at cell centres (position i + 1/2) and at faces (position i).
    """
    w = omega_of(wavelength)
    s_node = np.ones(n, dtype=np.complex128)
    s_half = np.ones(n + 1, dtype=np.complex128)

    def sigma(depth, npml):
        d = npml * dx
        smax = -(m + 1.0) * lnR / (2.0 * ETA0 * d)
        return smax * (depth / npml) ** m

    for arr, offset in ((s_node, 0.5), (s_half, 0.0)):
        pos = np.arange(arr.size, dtype=np.float64) + offset
        sig = np.zeros(arr.size)
        if npml_lo > 0:
            dlo = np.maximum(0.0, npml_lo - pos)
            sig += np.where(dlo > 0, sigma(dlo, npml_lo), 0.0)
        if npml_hi > 0:
            dhi = np.maximum(0.0, pos - (n - npml_hi))
            sig += np.where(dhi > 0, sigma(dhi, npml_hi), 0.0)
        arr[:] = 1.0 + sig / (1j * w * EPS0)
    return s_node, s_half


def _gradient(n: int) -> sp.csr_matrix:
    """(n+1) x n difference from cell centres to faces, zero outside:
    (G x)_f = x_f - x_{f-1}, f = 0..n, with x_{-1} = x_n = 0."""
    rows = np.concatenate([np.arange(n), np.arange(1, n + 1)])
    cols = np.concatenate([np.arange(n), np.arange(n)])
    vals = np.concatenate([np.ones(n), -np.ones(n)])
    return sp.csr_matrix((vals, (rows, cols)), shape=(n + 1, n))


def laplacian_1d(s_node: np.ndarray, s_half: np.ndarray) -> sp.csr_matrix:
    """dx^2 (1/s) d/dzeta (1/s) d/dzeta as -S_node^-1 G^T S_half^-1 G."""
    n = s_node.size
    G = _gradient(n)
    return (-sp.diags(1.0 / s_node) @ G.T @ sp.diags(1.0 / s_half) @ G).tocsr()


def pml_factors(nx, ny, dx, wavelength, npml, m=3.0, lnR=-30.0):
    """npml = int or (x_lo, x_hi, y_lo, y_hi)."""
    if np.isscalar(npml):
        npml = (npml,) * 4
    sxn, sxh = pml_stretch(nx, npml[0], npml[1], dx, wavelength, m, lnR)
    syn, syh = pml_stretch(ny, npml[2], npml[3], dx, wavelength, m, lnR)
    return sxn, sxh, syn, syh


def assemble_operator(eps: np.ndarray, dx: float, wavelength: float, npml=20,
                      m: float = 3.0, lnR: float = -30.0) -> sp.csr_matrix:
    """A~ = I_y (x) L~x + L~y (x) I_x + (k0 dx)^2 diag(eps)  (Eq. 1 x dx^2).

    Unknowns ordered row-major over [ny][nx] (x fastest)."""
    ny, nx = eps.shape
    sxn, sxh, syn, syh = pml_factors(nx, ny, dx, wavelength, npml, m, lnR)
    Lx = laplacian_1d(sxn, sxh)
    Ly = laplacian_1d(syn, syh)
    k2 = k0dx_of(dx, wavelength) ** 2
    A = sp.kron(sp.identity(ny), Lx) + sp.kron(Ly, sp.identity(nx)) \
        + sp.diags(k2 * eps.astype(np.float64).ravel())
    return A.tocsr().astype(np.complex128)


def source_rhs(J: np.ndarray, dx: float, wavelength: float) -> np.ndarray:
    """b~ = dx^2 j w mu0 J (right-hand side of Eq. 1 under e^{+jwt},
    moved to the form  lap E + k^2 eps E = j w mu0 J, times dx^2)."""
    return (dx * dx * 1j * omega_of(wavelength) * MU0) * J.astype(np.complex128).ravel()


class DirectSolver:
    """SuperLU factorisation of A~ reused for forward and adjoint solves."""

    def __init__(self, A: sp.spmatrix):
        self.A = A.tocsc()
        self.lu = spla.splu(self.A, permc_spec="COLAMD")

    def solve(self, b: np.ndarray) -> np.ndarray:
        return self.lu.solve(np.asarray(b, dtype=np.complex128))

    def solve_transpose(self, g: np.ndarray) -> np.ndarray:
        """Solve A~^T lam = g (plain transpose, no conjugation)."""
        return self.lu.solve(np.asarray(g, dtype=np.complex128), trans="T")


def solve_direct(eps, J, dx, wavelength, npml=20):
    """E* = A~^{-1} b~ : the unique answer every iterative solve must reach."""
    A = assemble_operator(eps, dx, wavelength, npml)
    b = source_rhs(J, dx, wavelength)
    return DirectSolver(A).solve(b).reshape(eps.shape)


def relres(A, x, b) -> float:
    """True relative residual ||b - A x|| / ||b|| in FP64."""
    x = np.asarray(x, dtype=np.complex128).ravel()
    b = np.asarray(b, dtype=np.complex128).ravel()
    return float(np.linalg.norm(b - A @ x) / np.linalg.norm(b))


# --- adjoint-variable gradient (Sec. 2.2, inverse design) -----------------

def mode_overlap(E: np.ndarray, port_x: int, mode: np.ndarray, y0: int, dx: float) -> complex:
    """c = sum_port conj(m) E dx along the vertical port line x = port_x."""
    col = E[y0:y0 + mode.size, port_x]
    return complex(np.sum(np.conj(mode) * col) * dx)


def fom_and_adjoint_source(E: np.ndarray, port_x: int, mode: np.ndarray, y0: int, dx: float):
    """F = |c|^2 and dF/dE (holomorphic part) as an [ny][nx] array:
    F = c conj(c), dF/dE_p = conj(c) * conj(m_p) dx on the port line."""
    c = mode_overlap(E, port_x, mode, y0, dx)
    g = np.zeros(E.shape, dtype=np.complex128)
    g[y0:y0 + mode.size, port_x] = np.conj(c) * np.conj(mode) * dx
    return abs(c) ** 2, g


def grad_eps(E: np.ndarray, lam: np.ndarray, dx: float, wavelength: float) -> np.ndarray:
    """dF/deps_p for a real F(E) with A~(eps) E = b~ and A~^T lam = dF/dE:

        dF/deps_p = 2 Re( dF/dE . dE/deps_p ) = -2 Re( lam_p (k0 dx)^2 E_p )

    since dA~/deps_p = (k0 dx)^2 e_p e_p^T and dE/deps_p = -A~^{-1} dA~ E.
    """
    k2 = k0dx_of(dx, wavelength) ** 2
    return -2.0 * np.real(lam * k2 * E)


def slab_mode(eps_col: np.ndarray, dx: float, wavelength: float, y_lo: int, y_hi: int):
    """Fundamental mode of the 1D cross-section eps_col[y_lo:y_hi] (FP64
    finite-difference eigenproblem), normalised so that sum |m|^2 dx = 1."""
    seg = eps_col[y_lo:y_hi].astype(np.float64)
    n = seg.size
    k2 = k0dx_of(dx, wavelength) ** 2
    main = -2.0 * np.ones(n) + k2 * seg
    L = np.diag(main) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)
    w, v = np.linalg.eigh(L)
    m = v[:, -1]
    m = m * np.sign(m[np.argmax(np.abs(m))])
    m = m / np.sqrt(np.sum(m * m) * dx)
    return m.astype(np.complex128)
