"""Pins of the coarse-space oracle (Eq. 7-8, Algorithm 3) and trend pins of
the two-level preconditioner (Table 1: two-level needs fewer iterations)."""
import numpy as np
import pytest

from oracle import coarse, fdfd, krylov, partition as P, schwarz
from paper_2509_03622_gb300 import workloads as wl

LAM = 1.55e-6


def test_plane_wave_phase_homogeneous_window():
    """Homogeneous eps: the accumulated phase is exactly kd d.(r - r_corner)."""
    n = 192
    eps = np.full((n, n), 2.1, np.float32)
    dx = LAM / 25
    win = P.Windows(n, n)
    X = coarse.plane_wave_trials(win, eps, dx, LAM, 8)
    kd = 2 * np.pi / 25 * np.sqrt(np.float64(np.float32(2.1)))
    w = 4  # interior window (1, 1) of the 3 x 3 layout
    x0, y0 = win.x0[w], win.y0[w]
    for m in range(8):
        th = 2 * np.pi * m / 8
        for (s, t, gx, gy) in coarse.perimeter_walk(win, w):
            ph = kd * (np.cos(th) * (gx - x0) + np.sin(th) * (gy - y0))
            assert abs(X[w, m, s, t] - np.exp(-1j * ph)) < 1e-9


def test_gram_schmidt_orthonormal():
    g = wl.rng(0)
    X = g.standard_normal((3, 10, 4, 80)) + 1j * g.standard_normal((3, 10, 4, 80))
    X[1, :, 0] = 0  # a window with one grid-edge side
    Q = coarse.gram_schmidt(X).reshape(3, 10, -1)
    for w in range(3):
        G = Q[w].conj() @ Q[w].T
        assert np.allclose(G, np.eye(10), atol=1e-12)
    assert not np.any(Q.reshape(3, 10, 4, 80)[1, :, 0])


@pytest.fixture(scope="module")
def small_exact():
    n, dx = 192, LAM / 25
    eps = wl.rectangles_eps(n, n, npml=20, n_rect=10, seed=31)
    S = schwarz.Schwarz(eps, dx, LAM, 20, k_coarse=8, local="exact", coarse_form="normal")
    return S


@pytest.fixture(scope="module")
def small_galerkin():
    n, dx = 192, LAM / 25
    eps = wl.rectangles_eps(n, n, npml=20, n_rect=10, seed=31)
    return schwarz.Schwarz(eps, dx, LAM, 20, k_coarse=8, local="exact")


def test_galerkin_mismatch_orthogonal_to_trials(small_galerkin):
    """The Galerkin correction of a random mismatch e leaves, on every
    window's own slots, a mismatch with no component along any of that
    window's trial vectors.  The new mismatch is measured through the fields:
    the traces of the added basis fields minus the data Q z they were solved
    with (a transposed, conjugated or mis-signed coarse matrix fails)."""
    S = small_galerkin
    cs = S.coarse
    g = wl.rng(7)
    e = g.standard_normal((S.win.n, 4, 80)) + 1j * g.standard_normal((S.win.n, 4, 80))
    e[~S.win.interface] = 0.0
    z = cs.solve(e)
    tr = P.traces(S.win, cs.correction(z), S.eps, S.dx, S.wavelength)
    Qz = np.einsum("wm,wmst->wst", z.reshape(S.win.n, cs.k), cs.Q)
    left = (e + tr - Qz).reshape(S.win.n, -1)
    proj = np.einsum("wmt,wt->wm", cs.Q.reshape(S.win.n, cs.k, -1).conj(), left)
    assert np.max(np.abs(proj)) < 1e-9 * np.max(np.abs(e))
    assert np.max(np.abs(left)) > 1e-3 * np.max(np.abs(e))  # not trivially zero


def test_galerkin_recovers_a_mismatch_in_its_range(small_galerkin):
    """A mismatch produced by coefficients z0 (e = -C z0) is removed exactly."""
    cs = small_galerkin.coarse
    g = wl.rng(8)
    z0 = g.standard_normal(cs.C.shape[1]) + 1j * g.standard_normal(cs.C.shape[1])
    z0[cs.dropped] = 0.0
    assert np.allclose(cs.solve(-(cs.C @ z0)), z0, rtol=1e-8, atol=1e-10)


@pytest.mark.slow
def test_galerkin_two_level_fgmres_trend_table1():
    """Trend of Table 1 for FGMRES(30) with the two-level sweep, exact local
    solves, homogeneous medium at 24 cells per wavelength: from 4 x 4 to
    8 x 8 windows the one-level count grows more than twofold while the
    two-level count (Galerkin coarse equation, k = 36) stays nearly flat and
    several times smaller."""
    dx = LAM / 24
    its = {}
    for n in (256, 512):
        eps = np.ones((n, n), np.float32)
        b = fdfd.source_rhs(wl.point_source(n, n), dx, LAM)
        for k in (0, 36):
            S = schwarz.Schwarz(eps, dx, LAM, 20, k_coarse=k, local="exact")
            _, info = krylov.fgmres(lambda v: S.A @ v, b, precond=S, restart=30, tol=1e-6, max_iters=200)
            assert info["converged"]
            its[n, k] = info["iters"]
    assert its[512, 0] >= 2 * its[256, 0]
    assert its[512, 36] <= its[256, 36] + 4 <= 14
    assert 3 * its[512, 36] <= its[512, 0]


def test_normal_equations_equal_lstsq(small_exact):
    cs = small_exact.coarse
    e = wl.rng(1).standard_normal(cs.C.shape[0]) + 0j
    z = cs.solve(e)
    z_ls, *_ = np.linalg.lstsq(cs.C, -e, rcond=None)
    assert np.linalg.norm(z - z_ls) / np.linalg.norm(z_ls) < 1e-8


def test_correction_acts_through_traces(small_exact):
    """Trace(sum R~^T z Phi) - Q z equals C z for any z (C's columns are the
    traces of the restricted basis fields minus the window's own data), and
    a mismatch in the range of C is removed exactly."""
    S = small_exact
    cs = S.coarse
    z0 = wl.rng(2).standard_normal(cs.C.shape[1]) + 1j * wl.rng(3).standard_normal(cs.C.shape[1])
    z0[cs.dropped] = 0.0  # dropped trials carry no unknown
    corr = cs.correction(z0)
    tr = P.traces(S.win, corr, S.eps, S.dx, S.wavelength)
    Qz = np.einsum("wm,wmst->wst", z0.reshape(S.win.n, cs.k), cs.Q)
    assert np.allclose((tr - Qz).ravel(), cs.C @ z0, atol=1e-12 * np.max(np.abs(tr)))
    e_bc = -(cs.C @ z0)
    assert np.allclose(cs.solve(e_bc), z0, rtol=1e-7, atol=1e-9)


@pytest.mark.slow
def test_two_level_stationary_trend_table1():
    """Trend of Table 1 for the literal Algorithm 3 loop with exact local
    solves: on a homogeneous 256^2 grid at 24 cells per wavelength (4 x 4
    windows) the two-level loop (k = 36) needs several times fewer
    iterations than the one-level loop."""
    n, dx = 256, LAM / 24
    eps = np.ones((n, n), np.float32)
    b = fdfd.source_rhs(wl.point_source(n, n), dx, LAM)
    S1 = schwarz.Schwarz(eps, dx, LAM, 20, k_coarse=0, local="exact")
    S2 = schwarz.Schwarz(eps, dx, LAM, 20, k_coarse=36, local="exact")
    _, it1, r1 = schwarz.stationary_solve(S1, b, tol=1e-6, max_iters=80)
    _, it2, r2 = schwarz.stationary_solve(S2, b, tol=1e-6, max_iters=80)
    assert r1 <= 1e-6 and r2 <= 1e-6
    assert 3 * it2 <= it1


@pytest.mark.slow
def test_exact_oras_beats_jacobi_in_fgmres():
    """One-level ORAS with exact local Robin solves as the FGMRES
    preconditioner converges where Jacobi-GMRES(30) stagnates."""
    n, dx = 256, LAM / 25
    eps = np.ones((n, n), np.float32)
    A = fdfd.assemble_operator(eps, dx, LAM, 20)
    b = fdfd.source_rhs(wl.point_source(n, n), dx, LAM)
    S1 = schwarz.Schwarz(eps, dx, LAM, 20, k_coarse=0, local="exact")
    mv = lambda v: A @ v
    x, i1 = krylov.fgmres(mv, b, precond=S1, restart=30, tol=1e-6, max_iters=100)
    d = A.diagonal()
    _, ij = krylov.fgmres(mv, b, precond=lambda v: v / d, restart=30, tol=1e-6, max_iters=100)
    assert i1["converged"] and i1["iters"] < 40
    assert not ij["converged"]
    xs = fdfd.DirectSolver(A).solve(b)
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-4


@pytest.fixture(scope="module")
def ritz_pair():
    """The same layout and local solver without and with the Ritz step."""
    n, dx = 192, LAM / 25
    eps = wl.rectangles_eps(n, n, npml=20, n_rect=10, seed=31)
    f = "normal"
    S0 = schwarz.Schwarz(eps, dx, LAM, 20, k_coarse=8, local="exact", coarse_form=f)
    S1 = schwarz.Schwarz(eps, dx, LAM, 20, k_coarse=8, local="exact", ritz_tol=1e-12, coarse_form=f)
    S3 = schwarz.Schwarz(eps, dx, LAM, 20, k_coarse=8, local="exact", ritz_tol=0.3, coarse_form=f)
    return S0, S1, S3


def test_ritz_all_directions_keep_the_galerkin_correction():
    """Galerkin form: the kept Ritz vectors span the trial space, so both the
    trial and the test space are unchanged and so is the correction."""
    n, dx = 192, LAM / 25
    eps = wl.rectangles_eps(n, n, npml=20, n_rect=10, seed=31)
    c0 = schwarz.Schwarz(eps, dx, LAM, 20, k_coarse=8, local="exact").coarse
    c1 = schwarz.Schwarz(eps, dx, LAM, 20, k_coarse=8, local="exact", ritz_tol=1e-12).coarse
    e = wl.rng(9).standard_normal(c0.C.shape[0]) + 1j * wl.rng(10).standard_normal(c0.C.shape[0])
    u0, u1 = c0.correction(c0.solve(e)), c1.correction(c1.solve(e))
    assert np.linalg.norm(u1 - u0) / np.linalg.norm(u0) < 1e-8


def test_ritz_all_directions_keep_the_correction(ritz_pair):
    """Keeping every Ritz vector with a nonzero eigenvalue spans the same
    space as the trials, so the coarse correction of any mismatch is
    unchanged (Q, Phi and C are combined consistently)."""
    S0, S1, _ = ritz_pair
    c0, c1 = S0.coarse, S1.coarse
    assert np.array_equal(c0.dropped, c1.dropped)
    e = wl.rng(4).standard_normal(c0.C.shape[0]) + 1j * wl.rng(5).standard_normal(c0.C.shape[0])
    u0, u1 = c0.correction(c0.solve(e)), c1.correction(c1.solve(e))
    assert np.linalg.norm(u1 - u0) / np.linalg.norm(u0) < 1e-8


def test_ritz_truncation_is_least_squares_on_the_kept_span(ritz_pair):
    """With a threshold the kept directions are the Ritz vectors with
    |eta| >= tol; the correction is the least-squares fit of the mismatch
    over their columns of C alone (the others pinned to zero)."""
    _, S1, S3 = ritz_pair
    c1, c3 = S1.coarse, S3.coarse
    kept = ~c3.dropped
    assert kept.sum() == (np.abs(c3.eta) >= 0.3).sum() < (~c1.dropped).sum()
    e = wl.rng(6).standard_normal(c3.C.shape[0]) + 0j
    z = c3.solve(e)
    z_ls, *_ = np.linalg.lstsq(c3.C[:, kept], -e, rcond=None)
    assert np.all(z[~kept] == 0)
    assert np.linalg.norm(z[kept] - z_ls) / np.linalg.norm(z_ls) < 1e-8


def test_ritz_eigenvalues_of_a_lossless_layout():
    """Homogeneous lossless medium, exact local solves: no Robin-to-Robin
    mode grows (|eta| <= 1), the interior window hands most of a plane wave
    on (its largest |eta| is well above the corner windows'; reading the
    wrong side of a neighbour would leave it near zero)."""
    n, dx = 192, LAM / 24
    S = schwarz.Schwarz(np.ones((n, n), np.float32), dx, LAM, 20, k_coarse=8, local="exact", ritz_tol=1e-12)
    a = np.abs(S.coarse.eta)
    assert a.max() <= 1.0
    assert a[4].max() >= 0.5 and a[4].max() > 2 * a[0].max()


@pytest.mark.slow
def test_ritz_truncated_two_level_still_converges():
    """Algorithm 3 with the coarse space truncated at |eta| >= 0.05 (homogeneous
    256^2, k = 36, exact local solves) still converges to 1e-6 within 80
    iterations while keeping fewer than two thirds of the modes."""
    n, dx = 256, LAM / 24
    eps = np.ones((n, n), np.float32)
    b = fdfd.source_rhs(wl.point_source(n, n), dx, LAM)
    S = schwarz.Schwarz(eps, dx, LAM, 20, k_coarse=36, local="exact", ritz_tol=0.05)
    kept = (~S.coarse.dropped).sum()
    _, it, r = schwarz.stationary_solve(S, b, tol=1e-6, max_iters=80)
    assert r <= 1e-6 and kept < 2 * S.coarse.dropped.size / 3
