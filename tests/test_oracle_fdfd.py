"""Pins of the FDFD oracle (Eq. 1, UPML of Methods) against closed forms,
brute force and invariants -- never against the oracle itself."""
import numpy as np
import pytest
import scipy.special as ss

from oracle import fdfd
from paper_2509_03622_gb300 import workloads as wl

LAM = 1.55e-6


def test_sine_modes_are_eigenvectors():
    """No PML, eps = 1, Dirichlet: sin(p pi (i+1)/(nx+1)) sin(q pi (j+1)/(ny+1))
    has eigenvalue (k0dx)^2 - 4 sin^2(p pi/(2(nx+1))) - 4 sin^2(q pi/(2(ny+1)))."""
    nx, ny, dx = 13, 9, LAM / 25
    A = fdfd.assemble_operator(np.ones((ny, nx), np.float32), dx, LAM, npml=0)
    k2 = (2 * np.pi / 25) ** 2
    i = np.arange(nx)
    j = np.arange(ny)
    for p, q in [(1, 1), (2, 5), (13, 9), (7, 3)]:
        v = np.outer(np.sin(q * np.pi * (j + 1) / (ny + 1)), np.sin(p * np.pi * (i + 1) / (nx + 1)))
        lam = k2 - 4 * np.sin(p * np.pi / (2 * (nx + 1))) ** 2 - 4 * np.sin(q * np.pi / (2 * (ny + 1))) ** 2
        Av = (A @ v.ravel()).reshape(ny, nx)
        assert np.max(np.abs(Av - lam * v)) < 1e-12


def test_dense_brute_force_16x16():
    """SuperLU path equals a dense LAPACK solve on a 16 x 16 grid with PML 4."""
    eps = wl.rectangles_eps(16, 16, npml=4, n_rect=3, seed=7)
    A = fdfd.assemble_operator(eps, LAM / 25, LAM, npml=4)
    b = fdfd.source_rhs(wl.random_field(16, 16, 3), LAM / 25, LAM)
    x_dense = np.linalg.solve(A.toarray(), b)
    x_lu = fdfd.DirectSolver(A).solve(b)
    assert np.linalg.norm(x_lu - x_dense) / np.linalg.norm(x_dense) < 1e-12


def test_pml_profile_closed_form():
    """s at the outer face of a 20-cell PML equals 1 - j (m+1)(-lnR)/(2 k0 d)
    with d = 20 dx (sigma_max / (w eps0) = -(m+1) lnR c / (2 w d))."""
    dx = LAM / 25
    sn, sh = fdfd.pml_stretch(100, 20, 20, dx, LAM)
    k0 = 2 * np.pi / LAM
    expect = 1 - 1j * 4 * 30 / (2 * k0 * 20 * dx)
    assert abs(sh[0] - expect) < 1e-10 * abs(expect) and abs(sh[-1] - expect) < 1e-10 * abs(expect)
    assert np.all(sh[20:81] == 1) and np.all(sn[20:80] == 1)
    # cubic grading: depth 10 of 20 cells gives 1/8 of the maximum loss
    assert abs(sh[10].imag - expect.imag / 8) < 1e-10 * abs(expect)
    assert np.all(sn.imag <= 0)  # absorbing under e^{+jwt}


def _hankel_error(ppw):
    n_in = 4 * ppw
    n = n_in + 40
    dx = LAM / ppw
    eps = np.ones((n, n), np.float32)
    J = wl.point_source(n, n)
    E = fdfd.solve_direct(eps, J, dx, LAM, npml=20)
    c = n // 2
    w = fdfd.omega_of(LAM)
    k = 2 * np.pi / LAM
    I = dx * dx  # line current carried by the unit-density cell
    errs, refs = [], []
    for ang in np.linspace(0, 2 * np.pi, 16, endpoint=False):
        r_cells = 1.5 * ppw
        ix = int(round(c + r_cells * np.cos(ang)))
        iy = int(round(c + r_cells * np.sin(ang)))
        r = np.hypot(ix - c, iy - c) * dx
        G = -(w * fdfd.MU0 * I / 4) * ss.hankel2(0, k * r)
        errs.append(abs(E[iy, ix] - G))
        refs.append(abs(G))
    return np.linalg.norm(errs) / np.linalg.norm(refs)


def test_greens_function_hankel_second_order():
    """Homogeneous medium: E = -(w mu0 I / 4) H0^(2)(k r) (outgoing under
    e^{+jwt}); the discrete error falls ~4x per halving of dx."""
    e20, e40, e80 = _hankel_error(20), _hankel_error(40), _hankel_error(80)
    assert e80 < 0.01
    assert 3.0 < e20 / e40 < 5.5 and 3.0 < e40 / e80 < 5.5


def test_pml_operator_symmetrised_by_stretch_factors():
    """With D = diag(s_x s_y) at cell centres, D A~ is complex symmetric
    (the stretched Laplacian is -G^T S^-1 G per axis), so A~^T = D A~ D^-1:
    the adjoint of the PML operator is a diagonal similarity of it."""
    n, dx = 48, LAM / 25
    eps = wl.rectangles_eps(n, n, npml=8, n_rect=4, seed=2)
    A = fdfd.assemble_operator(eps, dx, LAM, npml=(8, 5, 6, 9))
    sxn, _, syn, _ = fdfd.pml_factors(n, n, dx, LAM, (8, 5, 6, 9))
    import scipy.sparse as sp
    DA = sp.diags(np.outer(syn, sxn).ravel()) @ A
    assert abs(DA - DA.T).max() < 1e-12 * abs(DA).max()
    assert abs(A - A.T).max() > 1e-3  # A~ itself is not symmetric in the PML


def test_reciprocity_heterogeneous():
    n = 96
    dx = LAM / 25
    eps = wl.rectangles_eps(n, n, npml=12, n_rect=10, seed=11)
    A = fdfd.assemble_operator(eps, dx, LAM, npml=12)
    S = fdfd.DirectSolver(A)
    a, b = (30, 41), (70, 55)
    ea = np.zeros(n * n, complex); ea[a[1] * n + a[0]] = 1
    eb = np.zeros(n * n, complex); eb[b[1] * n + b[0]] = 1
    Gab = S.solve(ea)[b[1] * n + b[0]]
    Gba = S.solve(eb)[a[1] * n + a[0]]
    assert abs(Gab - Gba) / abs(Gab) < 1e-10


def test_poynting_balance_lossless():
    """Im sum_R conj(E) b~ equals the discrete flux sum over edges leaving R
    of Im(conj(E_in) E_out), for any rectangle R outside the PML; nested
    rectangles around the source carry the same flux."""
    n = 96
    dx = LAM / 25
    eps = wl.rectangles_eps(n, n, npml=12, n_rect=8, seed=5)
    A = fdfd.assemble_operator(eps, dx, LAM, npml=12)
    J = wl.point_source(n, n)
    b = fdfd.source_rhs(J, dx, LAM)
    E = fdfd.DirectSolver(A).solve(b).reshape(n, n)
    bb = b.reshape(n, n)

    def flux(x0, x1, y0, y1):
        f = 0.0
        for y in range(y0, y1):
            f += np.imag(np.conj(E[y, x0]) * E[y, x0 - 1]) + np.imag(np.conj(E[y, x1 - 1]) * E[y, x1])
        for x in range(x0, x1):
            f += np.imag(np.conj(E[y0, x]) * E[y0 - 1, x]) + np.imag(np.conj(E[y1 - 1, x]) * E[y1, x])
        return f

    for (x0, x1, y0, y1) in [(20, 76, 20, 76), (40, 60, 30, 70)]:
        lhs = np.imag(np.sum(np.conj(E[y0:y1, x0:x1]) * bb[y0:y1, x0:x1]))
        assert abs(lhs - flux(x0, x1, y0, y1)) < 1e-9 * abs(lhs)
    # radiated power leaves the source: Re(E_s J) < 0 (P = -Re(E J*)/2 > 0)
    assert np.real(E[n // 2, n // 2]) < 0
    f1, f2 = flux(20, 76, 20, 76), flux(40, 60, 30, 70)
    assert abs(f1 - f2) < 1e-9 * abs(f1)


def test_adjoint_gradient_matches_central_differences():
    n = 64
    dx = LAM / 25
    eps0 = wl.rectangles_eps(n, n, npml=10, n_rect=6, seed=9).astype(np.float64)
    J = wl.point_source(n, n, x=20, y=32)
    mode = np.exp(-((np.arange(12) - 5.5) / 3.0) ** 2).astype(complex)

    def F_of(eps):
        E = fdfd.solve_direct(eps, J, dx, LAM, npml=10)
        return fdfd.fom_and_adjoint_source(E, 45, mode, 26, dx)[0]

    A = fdfd.assemble_operator(eps0, dx, LAM, npml=10)
    S = fdfd.DirectSolver(A)
    E = S.solve(fdfd.source_rhs(J, dx, LAM)).reshape(n, n)
    F, g = fdfd.fom_and_adjoint_source(E, 45, mode, 26, dx)
    lam = S.solve_transpose(g.ravel()).reshape(n, n)
    grad = fdfd.grad_eps(E, lam, dx, LAM)
    h = 1e-3
    gen = wl.rng(3)
    for _ in range(8):
        px, py = int(gen.integers(15, 50)), int(gen.integers(15, 50))
        ep = eps0.copy(); ep[py, px] += h
        em = eps0.copy(); em[py, px] -= h
        fd = (F_of(ep) - F_of(em)) / (2 * h)
        assert abs(fd - grad[py, px]) <= 1e-5 * abs(fd) + 1e-12 * abs(F)


def test_mode_overlap_definition():
    """c = dx sum conj(m) E on the port line: a field equal to a complex
    (phase-ramped) profile on that line and anything elsewhere overlaps it by
    dx sum |m|^2, real and positive (a missing conjugate would give
    dx sum m^2, complex here); a field orthogonal to it on the line gives 0;
    the adjoint source is conj(c) conj(m) dx on the line and zero elsewhere."""
    n, dx, x, y0 = 48, 2e-8, 31, 7
    m = np.exp(-((np.arange(20) - 9.5) / 4.0) ** 2) * np.exp(0.7j * np.arange(20))
    g = wl.rng(5)
    E = g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))
    E[y0:y0 + m.size, x] = m
    c = fdfd.mode_overlap(E, x, m, y0, dx)
    assert abs(c - dx * np.sum(np.abs(m) ** 2)) <= 1e-14 * abs(c)
    r = g.standard_normal(m.size) + 1j * g.standard_normal(m.size)
    v = r - (np.sum(np.conj(m) * r) / np.sum(np.abs(m) ** 2)) * m  # orthogonal to m
    E2 = E.copy()
    E2[y0:y0 + m.size, x] = v
    assert abs(fdfd.mode_overlap(E2, x, m, y0, dx)) <= 1e-14 * dx * np.linalg.norm(m) * np.linalg.norm(v)
    F, src = fdfd.fom_and_adjoint_source(E, x, m, y0, dx)
    assert abs(F - abs(c) ** 2) <= 1e-14 * F
    ref = np.zeros_like(E)
    ref[y0:y0 + m.size, x] = np.conj(c) * np.conj(m) * dx
    assert np.array_equal(src, ref)
