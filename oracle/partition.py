"""The partitioner of Methods ("Two-level Schwarz method with coarse space"):
fixed-size overlapping windows, restriction, restricted prolongation, the
Robin traces of Eq. 2 and the local Robin boundary-value operator.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Window geometry (reading of "64 x 64 subdomains with 8-cell overlap"):
the grid (nx, ny multiples of 64, at least 128) is tiled by 64 x 64 cores;
core (a, b) covers x in [64a, 64a+64), y in [64b, 64b+64).  Its window is
80 x 80 cells, x0 = clamp(64a - 8, 0, nx - 80) (likewise y0), i.e. the core
plus 8 cells per side, shifted inward at the grid edge.  A window side that
lies on the grid edge keeps the global (Dirichlet-backed PML) rows; every
other side is an interface side carrying Robin data.

Robin data (Eq. 2, reading): with e^{+jwt} the transparent condition for
outgoing waves is  dE/dn + j k E = g,  k = k0 sqrt(eps_b) (PML stretching
ignored).  With the outward ghost cell o of boundary cell b and dE/dn ~
(E_o - E_b)/dx, the dx-scaled trace is
        g~ = E_o - E_b + j (k0 dx) sqrt(eps_b) E_b.
Trace slots per window: 4 sides x 80, side order (x-, x+, y-, y+), slot
index side*80 + t with t the coordinate along the side.

Parity: pinned in tests/test_oracle_partition.py (a local Robin solve fed
with the traces of the global solution reproduces that solution on the
window exactly; restriction / prolongation partition of unity).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fdfd

WIN = 80
CORE = 64
OVL = 8
SIDES = 4


class Windows:
    """Window table for an nx x ny grid."""

    def __init__(self, nx: int, ny: int):
        if nx % CORE or ny % CORE or nx < 2 * CORE or ny < 2 * CORE:
            raise ValueError("grid sides must be multiples of 64 and at least 128")
        self.nx, self.ny = nx, ny
        self.nwx, self.nwy = nx // CORE, ny // CORE
        self.n = self.nwx * self.nwy
        self.x0 = np.zeros(self.n, dtype=np.int64)
        self.y0 = np.zeros(self.n, dtype=np.int64)
        self.interface = np.zeros((self.n, SIDES), dtype=bool)
        for w in range(self.n):
            a, b = w % self.nwx, w // self.nwx
            self.x0[w] = min(max(CORE * a - OVL, 0), nx - WIN)
            self.y0[w] = min(max(CORE * b - OVL, 0), ny - WIN)
            self.interface[w] = [self.x0[w] > 0, self.x0[w] + WIN < nx,
                                 self.y0[w] > 0, self.y0[w] + WIN < ny]

    def core_offset(self, w: int):
        a, b = w % self.nwx, w // self.nwx
        return CORE * a - self.x0[w], CORE * b - self.y0[w]

    def owner(self, gx, gy):
        return (gy // CORE) * self.nwx + gx // CORE

    def side_cells(self, w: int, side: int):
        """Boundary cells b and ghost cells o (global x, y) of one side,
        in order of the along-side coordinate t = 0..79."""
        x0, y0 = int(self.x0[w]), int(self.y0[w])
        t = np.arange(WIN)
        if side == 0:
            bx, by, ox, oy = np.full(WIN, x0), y0 + t, np.full(WIN, x0 - 1), y0 + t
        elif side == 1:
            bx, by, ox, oy = np.full(WIN, x0 + WIN - 1), y0 + t, np.full(WIN, x0 + WIN), y0 + t
        elif side == 2:
            bx, by, ox, oy = x0 + t, np.full(WIN, y0), x0 + t, np.full(WIN, y0 - 1)
        else:
            bx, by, ox, oy = x0 + t, np.full(WIN, y0 + WIN - 1), x0 + t, np.full(WIN, y0 + WIN)
        return bx, by, ox, oy


def restrict(win: Windows, u: np.ndarray) -> np.ndarray:
    """R_w u for every window: [n_win][80][80]."""
    out = np.zeros((win.n, WIN, WIN), dtype=np.result_type(u.dtype, np.complex64))
    for w in range(win.n):
        x0, y0 = win.x0[w], win.y0[w]
        out[w] = u[y0:y0 + WIN, x0:x0 + WIN]
    return out


def prolong(win: Windows, loc: np.ndarray) -> np.ndarray:
    """Restricted (owner-core) assembly  u = sum_w R~_w^T u_w."""
    u = np.zeros((win.ny, win.nx), dtype=loc.dtype)
    for w in range(win.n):
        cx, cy = win.core_offset(w)
        a, b = w % win.nwx, w // win.nwx
        u[CORE * b:CORE * b + CORE, CORE * a:CORE * a + CORE] = loc[w, cy:cy + CORE, cx:cx + CORE]
    return u


def kd_map(eps: np.ndarray, dx: float, wavelength: float) -> np.ndarray:
    """(k0 dx) sqrt(eps) per cell: the dx-scaled Robin wavenumber."""
    return fdfd.k0dx_of(dx, wavelength) * np.sqrt(eps.astype(np.float64))


def traces(win: Windows, u: np.ndarray, eps: np.ndarray, dx: float, wavelength: float) -> np.ndarray:
    """Robin traces g~ = u_o - u_b + j kd_b u_b of a global field u on every
    interface side of every window: [n_win][4][80] (zero on grid-edge sides)."""
    kd = kd_map(eps, dx, wavelength)
    g = np.zeros((win.n, SIDES, WIN), dtype=np.complex128)
    bx, by, ox, oy, iface = _side_tables(win)
    ub = u[by[iface], bx[iface]]
    g[iface] = u[oy[iface], ox[iface]] - ub + 1j * kd[by[iface], bx[iface]] * ub
    return g


def _side_tables(win: Windows):
    """Boundary and ghost cells of every side of every window, [n_win][4][80]
    each, and the interface mask (side_cells stacked; cached on the table)."""
    if getattr(win, "_tables", None) is None:
        cells = np.zeros((4, win.n, SIDES, WIN), dtype=np.int64)
        for w in range(win.n):
            for s in range(SIDES):
                cells[:, w, s] = win.side_cells(w, s)
        iface = np.broadcast_to(win.interface[:, :, None], (win.n, SIDES, WIN))
        win._tables = (*cells, iface)
    return win._tables


def local_operator(win: Windows, w: int, A: sp.csr_matrix, eps: np.ndarray, dx: float,
                   wavelength: float):
    """Local Robin operator A_w (6400 x 6400) and the map from Robin data to
    the right-hand side.

    A_w is the global A~ restricted to the window's rows and columns, with
    each interface ghost eliminated through Eq. 2:  u_o = (1 - j kd_b) u_b + g~,
    so the row of b gains c_bo (1 - j kd_b) on its diagonal and its
    right-hand side loses c_bo g~ (c_bo is the global coupling b -> o).
    Returns (A_w as CSR, bnd) with bnd[side] = (local index of b, c_bo).
    """
    nx = win.nx
    x0, y0 = int(win.x0[w]), int(win.y0[w])
    gy, gx = np.meshgrid(np.arange(y0, y0 + WIN), np.arange(x0, x0 + WIN), indexing="ij")
    gidx = (gy * nx + gx).ravel()
    Aw = A[gidx][:, gidx].tolil()
    kd = kd_map(eps, dx, wavelength)
    bnd = {}
    for s in range(SIDES):
        if not win.interface[w, s]:
            continue
        bx, by, ox, oy = win.side_cells(w, s)
        lidx = (by - y0) * WIN + (bx - x0)
        c = np.asarray(A[by * nx + bx, oy * nx + ox]).ravel()
        for t in range(WIN):
            Aw[lidx[t], lidx[t]] += c[t] * (1.0 - 1j * kd[by[t], bx[t]])
        bnd[s] = (lidx, c)
    return Aw.tocsr(), bnd


def local_rhs(r_w: np.ndarray, g_w: np.ndarray, bnd: dict) -> np.ndarray:
    """Right-hand side of the local Robin problem: r - sum_sides c_bo g~."""
    rhs = np.array(r_w, dtype=np.complex128).ravel().copy()
    for s, (lidx, c) in bnd.items():
        np.add.at(rhs, lidx, -c * g_w[s])
    return rhs


def local_solve_exact(win: Windows, A: sp.csr_matrix, eps, dx, wavelength, r_loc, g_loc):
    """Exact local Robin solves (SuperLU) for every window: [n_win][80][80]."""
    out = np.zeros((win.n, WIN, WIN), dtype=np.complex128)
    for w in range(win.n):
        Aw, bnd = local_operator(win, w, A, eps, dx, wavelength)
        rhs = local_rhs(r_loc[w], g_loc[w], bnd)
        out[w] = spla.spsolve(Aw.tocsc(), rhs).reshape(WIN, WIN)
    return out
