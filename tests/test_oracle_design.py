"""Pins of the inverse-design oracle (Sec. 2.2 inverse design: filtering,
projection, Adam ascent with adjoint gradients)."""
import numpy as np

from oracle import design as D, fdfd
from paper_2509_03622_gb300 import workloads as wl

LAM = 1.55e-6


def test_filter_passes_constants_and_is_local():
    rho = np.full((17, 23), 0.37)
    rf, S = D.filter_fwd(rho, 3.5)
    assert np.allclose(rf, 0.37, atol=1e-15)
    assert S[8, 11] > S[0, 0] > 0  # edge cells see fewer neighbours
    e = np.zeros((17, 23))
    e[8, 11] = 1.0
    rf, _ = D.filter_fwd(e, 3.5)
    assert np.all(rf[np.hypot(*np.mgrid[-8:9, -11:12]) >= 3.5] == 0) and rf[8, 11] > 0


def test_filter_adjoint_identity():
    g = wl.rng(7)
    x, y = g.random((19, 14)), g.random((19, 14))
    for R in (1.5, 2.0, 4.3):
        Wx, _ = D.filter_fwd(x, R)
        assert abs(np.sum(Wx * y) - np.sum(x * D.filter_adj(y, R))) < 1e-12 * np.sum(np.abs(Wx * y))


def test_projection_closed_forms():
    x = np.linspace(0, 1, 101)
    for beta, eta in ((8.0, 0.5), (32.0, 0.3)):
        p = D.project(x, beta, eta)
        assert abs(p[0]) < 1e-15 and abs(p[-1] - 1) < 1e-15 and np.all(np.diff(p) >= 0)
        h = 1e-6
        fd = (D.project(x + h, beta, eta) - D.project(x - h, beta, eta)) / (2 * h)
        assert np.allclose(D.project_grad(x, beta, eta), fd, rtol=1e-6, atol=1e-8)
    assert np.allclose(D.project(x, 1e-6, 0.5), x, atol=1e-9)


def test_rho_gradient_matches_finite_differences():
    g = wl.rng(8)
    rho = g.random((12, 15))
    c = g.standard_normal((12, 15))  # linear functional F = sum c * eps
    args = (2.5, 6.0, 0.5, 2.1, 12.25)
    grad = D.eps_grad_to_rho(c, rho, *args)
    h = 1e-6
    for (i, j) in ((0, 0), (5, 7), (11, 14), (6, 0)):
        rp, rm = rho.copy(), rho.copy()
        rp[i, j] += h
        rm[i, j] -= h
        fd = (np.sum(c * D.density_to_eps(rp, *args)[0]) - np.sum(c * D.density_to_eps(rm, *args)[0])) / (2 * h)
        assert abs(fd - grad[i, j]) < 1e-6 * max(1.0, abs(fd))


def test_adam_first_steps_closed_form():
    """Bias correction makes the first step lr * g / (|g| + eps), and a
    constant gradient keeps that step size."""
    opt = D.Adam((3,), lr=0.05)
    th = np.full(3, 0.5)
    g = np.array([2.0, -1e-3, 0.0])
    t1 = opt.step(th, g)
    assert np.allclose(t1 - th, 0.05 * g / (np.abs(g) + 1e-8), atol=1e-15)
    t2 = opt.step(t1, g)
    assert np.allclose(t2 - t1, 0.05 * g / (np.abs(g) + 1e-8), atol=1e-12)
    t = np.full(3, 0.99)
    for _ in range(5):
        t = opt.step(t, np.array([1.0, 1.0, 1.0]))
    assert np.all(t <= 1.0)


def _tiny_demux():
    """96^2 grid: input guide from the left, output guide to the right, a
    24 x 24 design square between them, one wavelength."""
    n, dx = 96, LAM / 25
    eps = np.full((n, n), 2.1, np.float32)
    eps[44:52, :36] = 12.25
    eps[44:52, 60:] = 12.25
    J = np.zeros((n, n), np.complex64)
    J[40:56, 26] = 1.0
    mode = fdfd.slab_mode(eps[:, 70], dx, LAM, 40, 56)
    return n, dx, eps, J, mode, (36, 36, 24, 24)


def _fom_and_grad(eps, J, dx, mode):
    A = fdfd.assemble_operator(eps, dx, LAM, 12)
    S = fdfd.DirectSolver(A)
    E = S.solve(fdfd.source_rhs(J, dx, LAM)).reshape(eps.shape)
    F, g = fdfd.fom_and_adjoint_source(E, 70, mode, 40, dx)
    lam = fdfd.DirectSolver(A.T).solve(g.ravel()).reshape(eps.shape)
    return F, fdfd.grad_eps(E, lam, dx, LAM)


def test_design_step_raises_the_figure_of_merit():
    """The chain rule through projection and filter gives the finite-
    difference derivative of the figure of merit in rho, and one Adam step
    along it raises the figure of merit."""
    n, dx, eps0, J, mode, (y0, x0, h, w) = _tiny_demux()
    args = (2.0, 4.0, 0.5, 2.1, 12.25)
    rho = np.full((h, w), 0.5) + 0.05 * wl.rng(9).standard_normal((h, w))

    def fom(r):
        e = eps0.copy()
        e[y0:y0 + h, x0:x0 + w] = D.density_to_eps(r, *args)[0]
        return _fom_and_grad(e, J, dx, mode)

    F0, g_eps = fom(rho)
    g_rho = D.eps_grad_to_rho(g_eps[y0:y0 + h, x0:x0 + w], rho, *args)
    hh = 1e-4
    for (i, j) in ((3, 4), (12, 12), (20, 2)):
        rp, rm = rho.copy(), rho.copy()
        rp[i, j] += hh
        rm[i, j] -= hh
        fd = (fom(rp)[0] - fom(rm)[0]) / (2 * hh)
        assert abs(fd - g_rho[i, j]) < 1e-3 * np.max(np.abs(g_rho))
    opt = D.Adam(rho.shape, lr=0.02)  # objective F / F0: Adam's eps assumes gradients well above 1e-8
    F1, _ = fom(opt.step(rho, g_rho / F0))
    assert F1 > 1.01 * F0
