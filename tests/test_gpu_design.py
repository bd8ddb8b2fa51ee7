"""GPU parity of the inverse-design loop (Sec. 2.2: filtering, projection,
Adam ascent, gradients from the adjoint solve) against the FP64 oracle,
through the C-ABI."""
import os

import numpy as np
import pytest

from oracle import design as OD, fdfd as OF
from paper_2509_03622_gb300 import workloads as wl

LAM = 1.55e-6
pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PARAMS = dict(radius=2.5, beta=6.0, eta=0.5, eps_lo=2.1, eps_hi=12.25)


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _oargs(p=PARAMS):
    return (p["radius"], p["beta"], p["eta"], p["eps_lo"], p["eps_hi"])


def test_design_kernels_match_oracle():
    """Filter, projection and permittivity (FP32) and the chain rule back to
    rho on a ragged rectangle (37 x 53, touching no grid edge), random data."""
    import torch
    from paper_2509_03622_gb300 import fdfd as F
    from paper_2509_03622_gb300.design import Design
    n = 128
    S = F.Solver(_t(np.full((n, n), 2.1, np.float32)), LAM / 30, LAM, npml=20)
    x0, y0, w, h = 30, 41, 53, 37
    D = Design(S, x0, y0, w, h, **PARAMS)
    g = wl.rng(12)
    rho = g.random((h, w)).astype(np.float32)
    eps = torch.full((n, n), -1.0, dtype=torch.float32, device="cuda")
    D.eps(_t(rho), eps)
    e = eps.cpu().numpy()
    ref, rf_ref = OD.density_to_eps(rho.astype(np.float64), *_oargs())
    assert np.max(np.abs(e[y0:y0 + h, x0:x0 + w] - ref)) < 2e-5 * 12.25
    assert np.max(np.abs(D.rho_f.cpu().numpy() - rf_ref)) < 2e-6
    outside = np.ones((n, n), bool)
    outside[y0:y0 + h, x0:x0 + w] = False
    assert np.all(e[outside] == -1.0)
    g_eps = g.standard_normal((n, n)).astype(np.float32)
    g_rho = D.grad(_t(g_eps)).cpu().numpy()
    g_ref = OD.eps_grad_to_rho(g_eps[y0:y0 + h, x0:x0 + w].astype(np.float64), rho.astype(np.float64), *_oargs())
    assert np.max(np.abs(g_rho - g_ref)) < 1e-4 * np.max(np.abs(g_ref))


def test_adam_matches_oracle():
    import torch
    from paper_2509_03622_gb300 import fdfd as F
    from paper_2509_03622_gb300.design import Adam
    S = F.Solver(_t(np.full((128, 128), 2.1, np.float32)), LAM / 30, LAM, npml=20)
    g = wl.rng(13)
    th0 = g.random(1000)
    opt, ref = Adam(S, (1000,), lr=0.03), OD.Adam((1000,), lr=0.03)
    th, tr = _t(th0.astype(np.float32)), th0.copy()
    for _ in range(6):
        gr = g.standard_normal(1000) * 40.0
        opt.step(th, _t(gr.astype(np.float32)), scale=0.5)
        tr = ref.step(tr, 0.5 * gr)
    assert np.max(np.abs(th.cpu().numpy() - tr)) < 1e-5
    with pytest.raises(F.FDFDError):
        Adam(S, (4,), lr=-1.0).step(_t(np.zeros(4, np.float32)), _t(np.zeros(4, np.float32)))


def test_design_iteration_matches_oracle():
    """One iteration of the loop: density -> permittivity -> forward solve ->
    mode overlap -> adjoint solve -> dF/deps -> dF/drho (autograd over the
    library calls) against the oracle's SuperLU chain, then one Adam step."""
    import torch
    from paper_2509_03622_gb300 import fdfd as F
    from paper_2509_03622_gb300.autograd import fdfd_field, mode_overlap, last_stats
    from paper_2509_03622_gb300.design import Adam, Design, density_to_eps
    n, dx = 128, LAM / 30
    base = wl.freeform_eps(n, n, seed=2128, hi=2.1)
    J = wl.point_source(n, n, x=40, y=64)
    port_x, y0, ny_m = 90, 52, 24
    mode = np.exp(-((np.arange(ny_m) - (ny_m - 1) / 2) / 5.0) ** 2).astype(np.complex64)
    rx, ry, rw, rh = 52, 44, 32, 40
    rho0 = (0.5 + 0.1 * wl.rng(14).standard_normal((rh, rw))).clip(0, 1)
    S = F.Solver(_t(base), dx, LAM, npml=20)
    D = Design(S, rx, ry, rw, rh, **PARAMS)
    rho = _t(rho0.astype(np.float32)).requires_grad_(True)
    eps = density_to_eps(D, rho, _t(base))
    blob = np.load(os.path.join(ROOT, "paper_2509_03622_gb300", "weights", "nno_trained.npy"))
    E = fdfd_field(S, eps, _t(J), blob, restart=30, max_iters=3000, tol=1e-7, precond=F.PRECOND_SCHWARZ, inner=8)
    c = mode_overlap(E, port_x, _t(mode), y0, dx)
    Fv = c.abs() ** 2
    Fv.backward()
    assert last_stats["forward"]["status"] == F.OK and last_stats["adjoint"]["status"] == F.OK
    g_gpu = rho.grad.cpu().numpy().astype(np.float64)
    # oracle chain in FP64
    e_o = base.astype(np.float64).copy()
    e_o[ry:ry + rh, rx:rx + rw] = OD.density_to_eps(rho0, *_oargs())[0]
    A = OF.assemble_operator(e_o, dx, LAM, 20)
    Sd = OF.DirectSolver(A)
    Eo = Sd.solve(OF.source_rhs(J, dx, LAM)).reshape(n, n)
    Fo, g = OF.fom_and_adjoint_source(Eo, port_x, mode.astype(complex), y0, dx)
    lam = Sd.solve_transpose(g.ravel()).reshape(n, n)
    g_eps = OF.grad_eps(Eo, lam, dx, LAM)
    g_ref = OD.eps_grad_to_rho(g_eps[ry:ry + rh, rx:rx + rw], rho0, *_oargs())
    assert abs(float(Fv.detach()) - Fo) <= 1e-4 * Fo
    err = np.linalg.norm(g_gpu - g_ref) / np.linalg.norm(g_ref)
    print(f"design gradient: relative error {err:.2e}")
    assert err < 2e-3, err
    # one Adam step on the objective F / F0: equal wherever the gradient is
    # not close to zero (there rounding may flip its sign)
    th = rho.detach().clone()
    Adam(S, th.shape, lr=0.02).step(th, rho.grad, scale=1.0 / float(Fv.detach()))
    tr = OD.Adam(rho0.shape, lr=0.02).step(rho0, g_ref / Fo)
    big = np.abs(g_ref) > 1e-2 * np.max(np.abs(g_ref))
    assert big.mean() > 0.5
    assert np.max(np.abs(th.cpu().numpy() - tr)[big]) < 1e-5
