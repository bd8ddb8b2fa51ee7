"""Differentiation pattern (Sec. 2.2, adjoint variable method) on the GPU:
dF/deps through torch.autograd over the library's forward solve, adjoint
solve on A~^T and dF/deps kernel, against the FP64 oracle's SuperLU adjoint
gradient (<= 1e-3 relative L2), itself checked by central differences."""
import os

import numpy as np
import pytest

from oracle import fdfd as OF
from paper_2509_03622_gb300 import workloads as wl

LAM = 1.55e-6
pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _weights():
    p = os.path.join(ROOT, "paper_2509_03622_gb300", "weights", "nno_trained.npy")
    return np.load(p) if os.path.exists(p) else wl.pack_weights(wl.nno_weights(0))


def test_adjoint_gradient_matches_oracle():
    import torch
    from paper_2509_03622_gb300 import fdfd as F
    from paper_2509_03622_gb300.autograd import fdfd_field, mode_overlap
    n, dx = 128, LAM / 30
    eps = wl.freeform_eps(n, n, seed=2128, hi=2.1)
    J = wl.point_source(n, n, x=40, y=64)
    port_x, y0, ny_m = 90, 52, 24
    mode = np.exp(-((np.arange(ny_m) - (ny_m - 1) / 2) / 5.0) ** 2).astype(np.complex64)
    S = F.Solver(torch.from_numpy(eps).cuda(), dx, LAM, npml=20)
    e_t = torch.from_numpy(eps).cuda().requires_grad_(True)
    E = fdfd_field(S, e_t, torch.from_numpy(J).cuda(), _weights(), restart=30, max_iters=3000, tol=1e-7,
                   precond=F.PRECOND_SCHWARZ, inner=8)
    c = mode_overlap(E, port_x, torch.from_numpy(mode).cuda(), y0, dx)
    Fv = (c.abs() ** 2)
    Fv.backward()
    g_gpu = e_t.grad.cpu().numpy().astype(np.float64)
    from paper_2509_03622_gb300.autograd import last_stats
    assert last_stats["forward"]["status"] == F.OK, last_stats
    assert last_stats["adjoint"]["status"] == F.OK, last_stats
    # oracle: SuperLU forward and adjoint, FP64
    A = OF.assemble_operator(eps, dx, LAM, 20)
    Sd = OF.DirectSolver(A)
    Eo = Sd.solve(OF.source_rhs(J, dx, LAM)).reshape(n, n)
    Fo, g = OF.fom_and_adjoint_source(Eo, port_x, mode.astype(complex), y0, dx)
    lam = Sd.solve_transpose(g.ravel()).reshape(n, n)
    g_ref = OF.grad_eps(Eo, lam, dx, LAM)
    assert abs(float(Fv.detach()) - Fo) <= 1e-4 * Fo
    inner = np.zeros((n, n), bool)
    inner[20:-20, 20:-20] = True
    err = np.linalg.norm((g_gpu - g_ref)[inner]) / np.linalg.norm(g_ref[inner])
    assert err < 1e-3, err
    # the oracle gradient itself against central differences on a few pixels
    h = 1e-3
    for (py, px) in [(60, 50), (70, 75)]:
        ep, em = eps.astype(np.float64).copy(), eps.astype(np.float64).copy()
        ep[py, px] += h
        em[py, px] -= h
        fp = OF.fom_and_adjoint_source(OF.solve_direct(ep, J, dx, LAM, 20), port_x, mode.astype(complex), y0, dx)[0]
        fm = OF.fom_and_adjoint_source(OF.solve_direct(em, J, dx, LAM, 20), port_x, mode.astype(complex), y0, dx)[0]
        assert abs((fp - fm) / (2 * h) - g_ref[py, px]) <= 1e-5 * abs(g_ref[py, px]) + 1e-9 * Fo


def _oracle_grad(eps, J, dx, lam_, port_x, mode, y0):
    """SuperLU forward and adjoint (FP64) and dF/deps of F = |c|^2."""
    n = eps.shape[0]
    A = OF.assemble_operator(eps, dx, lam_, 20)
    Sd = OF.DirectSolver(A)
    Eo = Sd.solve(OF.source_rhs(J, dx, lam_)).reshape(n, n)
    Fo, g = OF.fom_and_adjoint_source(Eo, port_x, mode.astype(complex), y0, dx)
    lam = Sd.solve_transpose(g.ravel()).reshape(n, n)
    return Fo, OF.grad_eps(Eo, lam, dx, lam_)


def _case():
    n, dx = 128, LAM / 30
    eps = wl.freeform_eps(n, n, seed=2128, hi=2.1)
    J = wl.point_source(n, n, x=40, y=64)
    mode = np.exp(-((np.arange(24) - 11.5) / 5.0) ** 2).astype(np.complex64)
    inner = np.zeros((n, n), bool)
    inner[20:-20, 20:-20] = True
    return n, dx, eps, J, mode, inner


def test_backward_after_another_forward_on_the_same_handle():
    """Two forward solves on one handle (the second at another permittivity),
    then the backward of the first: its gradient is the oracle's at the
    first permittivity, not at the one the handle last held."""
    import torch
    from paper_2509_03622_gb300 import fdfd as F
    from paper_2509_03622_gb300.autograd import fdfd_field, mode_overlap
    n, dx, eps, J, mode, inner = _case()
    eps2 = eps.copy()
    eps2[40:90, 60:100] = 2.1 - eps2[40:90, 60:100] + 1.0  # swap the two materials in a block
    S = F.Solver(torch.from_numpy(eps).cuda(), dx, LAM, npml=20)
    kw = dict(restart=30, max_iters=3000, tol=1e-7, precond=F.PRECOND_SCHWARZ, inner=8)
    Jt, mt = torch.from_numpy(J).cuda(), torch.from_numpy(mode).cuda()
    e1 = torch.from_numpy(eps).cuda().requires_grad_(True)
    e2 = torch.from_numpy(eps2).cuda().requires_grad_(True)
    F1 = mode_overlap(fdfd_field(S, e1, Jt, _weights(), **kw), 90, mt, 52, dx).abs() ** 2
    F2 = mode_overlap(fdfd_field(S, e2, Jt, _weights(), **kw), 90, mt, 52, dx).abs() ** 2
    F1.backward()
    _, g_ref = _oracle_grad(eps, J, dx, LAM, 90, mode, 52)
    g = e1.grad.cpu().numpy().astype(np.float64)
    err = np.linalg.norm((g - g_ref)[inner]) / np.linalg.norm(g_ref[inner])
    assert err < 1e-3, err
    F2.backward()  # and the second one still gets its own
    _, g_ref2 = _oracle_grad(eps2, J, dx, LAM, 90, mode, 52)
    g2 = e2.grad.cpu().numpy().astype(np.float64)
    err2 = np.linalg.norm((g2 - g_ref2)[inner]) / np.linalg.norm(g_ref2[inner])
    assert err2 < 1e-3, err2
    S.close()


def test_multi_wavelength_fdfdsolve_gradient():
    """FDFDSolve over three wavelengths: the gradient of sum |c_lambda|^2 is
    the sum of the oracle's adjoint gradients; close() frees the handles."""
    import torch
    from paper_2509_03622_gb300 import fdfd as F
    from paper_2509_03622_gb300.autograd import FDFDSolve, mode_overlap
    n, dx, eps, J, mode, inner = _case()
    lams = [1.50e-6, 1.55e-6, 1.60e-6]
    solve = FDFDSolve(dx, lams, _weights(), restart=30, max_iters=3000, tol=1e-7,
                      precond=F.PRECOND_SCHWARZ, inner=8)
    e_t = torch.from_numpy(eps).cuda().requires_grad_(True)
    Es = solve(e_t, torch.from_numpy(J).cuda())
    mt = torch.from_numpy(mode).cuda()
    Ftot = sum(mode_overlap(E, 90, mt, 52, dx).abs() ** 2 for E in Es)
    Ftot.backward()
    Fo, g_ref = 0.0, np.zeros((n, n))
    for lam_ in lams:
        f, g = _oracle_grad(eps, J, dx, lam_, 90, mode, 52)
        Fo += f
        g_ref += g
    assert abs(float(Ftot.detach()) - Fo) <= 1e-4 * Fo
    g = e_t.grad.cpu().numpy().astype(np.float64)
    err = np.linalg.norm((g - g_ref)[inner]) / np.linalg.norm(g_ref[inner])
    assert err < 1e-3, err
    assert len(solve.solvers) == 3
    solve.close()
    assert solve.solvers is None


@pytest.mark.parametrize("port_x,y0,nm", [(77, 11, 37), (127, 28, 100), (0, 0, 128)])
def test_overlap_kernels_match_oracle(port_x, y0, nm):
    """The figure of merit's kernels against the oracle's definitions on the
    same complex64 field: the overlap c (FP64 sums of exact products, so to
    1e-12), the chain rule for F = |c|^2 (G_c = 2c) followed by the adjoint
    right-hand side conj(G_E)/2, which must equal the oracle's adjoint source
    conj(c) conj(m) dx (complex64 output: 1e-6), zero off the port line; and
    accumulation adds.  Ports on the first and last column and a profile
    spanning every row cover the edges."""
    import torch
    from paper_2509_03622_gb300 import fdfd as F
    n, dx = 128, LAM / 30
    g = wl.rng(77)
    E = (g.standard_normal((n, n)) + 1j * g.standard_normal((n, n))).astype(np.complex64)
    m = (g.standard_normal(nm) + 1j * g.standard_normal(nm)).astype(np.complex64)
    Et, mt = torch.from_numpy(E).cuda(), torch.from_numpy(m).cuda()
    c = torch.empty(2, dtype=torch.float64, device="cuda")
    F.mode_overlap(Et, mt, port_x, y0, dx, c)
    torch.cuda.synchronize()
    cg = complex(c[0].item(), c[1].item())
    Fo, go = OF.fom_and_adjoint_source(E.astype(complex), port_x, m.astype(complex), y0, dx)
    c_ref = OF.mode_overlap(E.astype(complex), port_x, m.astype(complex), y0, dx)
    assert abs(cg - c_ref) <= 1e-12 * abs(c_ref)
    assert abs(abs(cg) ** 2 - Fo) <= 1e-12 * Fo
    S = F.Solver(torch.ones((n, n), device="cuda"), dx, LAM, npml=20)
    GE = torch.full((n, n), 7.0 + 3.0j, dtype=torch.complex64, device="cuda")  # overwritten
    F.mode_overlap_grad((n, n), mt, port_x, y0, dx, 2 * cg, GE)
    gt = torch.empty_like(GE)
    S.adjoint_rhs(GE, gt)
    torch.cuda.synchronize()
    gg = gt.cpu().numpy()
    assert np.linalg.norm(gg - go) <= 1e-6 * np.linalg.norm(go)
    off = np.ones((n, n), bool)
    off[y0:y0 + nm, port_x] = False
    assert not np.any(gg[off])
    F.mode_overlap_grad((n, n), mt, port_x, y0, dx, 2 * cg, GE, accumulate=True)
    S.adjoint_rhs(GE, GE)  # in place
    torch.cuda.synchronize()
    assert np.linalg.norm(GE.cpu().numpy() - 2 * go) <= 1e-6 * np.linalg.norm(2 * go)
    S.close()
