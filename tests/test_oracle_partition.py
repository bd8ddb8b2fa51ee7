"""Pins of the partitioner oracle: window geometry, restricted assembly and
the exactness of the local Robin problem (Eq. 2) on global traces."""
import numpy as np
import scipy.sparse.linalg as spla

from oracle import fdfd, partition as P
from paper_2509_03622_gb300 import workloads as wl

LAM = 1.55e-6


def test_window_table_256():
    win = P.Windows(256, 256)
    assert win.n == 16
    assert sorted(set(win.x0.tolist())) == [0, 56, 120, 176]
    # corner window: interfaces only towards +x and +y
    assert win.interface[0].tolist() == [False, True, False, True]
    # interior window
    w = 1 * 4 + 1
    assert win.interface[w].tolist() == [True, True, True, True]
    assert win.core_offset(0) == (0, 0) and win.core_offset(w) == (8, 8)
    assert win.core_offset(15) == (16, 16)


def test_restrict_prolong_partition_of_unity():
    win = P.Windows(192, 128)
    u = wl.random_field(192, 128, 5).astype(np.complex128)
    assert np.array_equal(P.prolong(win, P.restrict(win, u)), u)


def test_local_robin_solve_reproduces_global_solution():
    """With Robin data taken from the global solution (traces of Eq. 2),
    each local problem's unique solution is the global field on its window."""
    n, dx = 192, LAM / 25
    eps = wl.rectangles_eps(n, n, npml=20, n_rect=12, seed=21)
    A = fdfd.assemble_operator(eps, dx, LAM, npml=20)
    J = wl.random_field(n, n, 6)
    b = fdfd.source_rhs(J, dx, LAM)
    E = fdfd.DirectSolver(A).solve(b).reshape(n, n)
    win = P.Windows(n, n)
    g = P.traces(win, E, eps, dx, LAM)
    r_loc = P.restrict(win, b.reshape(n, n))
    for w in [0, 1, 4, 8]:
        Aw, bnd = P.local_operator(win, w, A, eps, dx, LAM)
        rhs = P.local_rhs(r_loc[w], g[w], bnd)
        x = spla.spsolve(Aw.tocsc(), rhs).reshape(P.WIN, P.WIN)
        x0, y0 = win.x0[w], win.y0[w]
        ref = E[y0:y0 + P.WIN, x0:x0 + P.WIN]
        assert np.linalg.norm(x - ref) / np.linalg.norm(ref) < 1e-10


def test_trace_of_outgoing_wave_is_small():
    """For a 1D outgoing wave exp(-j k x) (discrete dispersion relation),
    the dx-scaled Robin trace on a +x side is -(k dx)^2/2 + O((k dx)^3)
    (the one-sided difference is first order at b) while on a -x side the
    wave is incoming and the trace is ~ 2 j k dx."""
    n = 256
    eps = np.ones((n, n), np.float32)
    dx = LAM / 40
    kd = 2 * np.pi / 40
    kdisc = 2 * np.arcsin(kd / 2)  # discrete wavenumber of the 1D stencil
    x = np.arange(n)
    u = np.tile(np.exp(-1j * kdisc * x), (n, 1))
    win = P.Windows(n, n)
    g = P.traces(win, u, eps, dx, LAM)
    ub_out = u[0, win.x0[0] + P.WIN - 1]
    ub_in = u[0, win.x0[1]]
    assert np.max(np.abs(g[0, 1] / ub_out + kd ** 2 / 2)) < 0.2 * kd ** 2   # outgoing
    assert np.max(np.abs(g[1, 0] / ub_in - 2j * kd)) < 0.1 * kd             # incoming
