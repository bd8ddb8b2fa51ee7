"""GPU parity of the stencil, traces, gradient kernel and the FGMRES
machinery against the FP64 oracle, through the C-ABI."""
import numpy as np
import pytest

from oracle import fdfd as OF, krylov as OK, partition as OP
from paper_2509_03622_gb300 import workloads as wl

LAM = 1.55e-6
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import torch  # noqa: F401
    from paper_2509_03622_gb300 import fdfd
    return fdfd


def _t(a, dtype=None):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _solver(F, eps, dx, npml=20):
    return F.Solver(_t(eps.astype(np.float32)), dx, LAM, npml=npml)


@pytest.mark.parametrize("shape,npml,seed", [((128, 192), 20, 1), ((256, 256), 20, 2), ((320, 128), (10, 0, 5, 30), 3)])
def test_stencil_matches_oracle_csr(F, shape, npml, seed):
    ny, nx = shape
    dx = LAM / 25
    eps = wl.rectangles_eps(nx, ny, npml=20, n_rect=10, seed=seed)
    S = _solver(F, eps, dx, npml)
    A = OF.assemble_operator(eps, dx, LAM, npml)
    x = wl.random_field(nx, ny, seed + 10)
    import torch
    y = torch.empty_like(_t(x))
    for tr, M in ((False, A), (True, A.T.tocsr())):
        S.apply_A(_t(x), y, transpose=tr)
        ref = M @ x.astype(np.complex128).ravel()
        got = y.cpu().numpy().ravel()
        scale = np.abs(M) @ np.abs(x.astype(np.complex128).ravel())  # |A||x| per row
        assert np.all(np.abs(got - ref) <= 1e-6 * scale + 1e-30)
    S.close()


def test_traces_match_oracle(F):
    n = 256
    dx = LAM / 30
    eps = wl.freeform_eps(n, n, seed=7)
    S = _solver(F, eps, dx)
    u = wl.random_field(n, n, 4)
    import torch
    g = torch.empty((16, 4, 80), dtype=torch.complex64, device="cuda")
    S.trace_extract(_t(u), g)
    ref = OP.traces(OP.Windows(n, n), u.astype(np.complex128), eps, dx, LAM)
    got = g.cpu().numpy()
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref))
    assert not np.any(got[0, 0]) and not np.any(got[0, 2])  # grid-edge sides are empty


def test_grad_kernel_matches_oracle(F):
    n = 128
    dx = LAM / 25
    eps = wl.rectangles_eps(n, n, npml=10, n_rect=4, seed=2)
    S = _solver(F, eps, dx, 10)
    E = wl.random_field(n, n, 1)
    lam = wl.random_field(n, n, 2)
    import torch
    g = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    S.grad_eps(_t(E), _t(lam), g)
    S.grad_eps(_t(E), _t(lam), g, accumulate=True)
    ref = 2 * OF.grad_eps(E.astype(complex), lam.astype(complex), dx, LAM)
    assert np.allclose(g.cpu().numpy(), ref, rtol=1e-5, atol=1e-6 * np.max(np.abs(ref)))


@pytest.mark.parametrize("precond,transpose", [(1, False), (0, False), (1, True)])
def test_fgmres_history_matches_oracle(F, precond, transpose):
    """True residual after k Arnoldi steps (k within the first cycle) equals
    the oracle FGMRES least-squares residual history[k]."""
    n = 256
    dx = LAM / 25
    eps = wl.rectangles_eps(n, n, npml=20, seed=1000)
    S = _solver(F, eps, dx)
    A = OF.assemble_operator(eps, dx, LAM, 20)
    J = wl.random_field(n, n, 5)
    import torch
    d = A.diagonal()
    pre = (lambda v: v / d) if precond == 1 else None
    if transpose:
        # the library solves A~^T lam = g as A~ mu = D^-1 g, lam = D mu (D = s_x s_y)
        g = J.astype(np.complex128).ravel()
        sxn, _, syn, _ = OF.pml_factors(n, n, dx, LAM, 20)
        Dm = np.outer(syn, sxn).ravel()
        rhs = g / Dm
    else:
        rhs = OF.source_rhs(J, dx, LAM)
    _, info = OK.fgmres(lambda v: A @ v, rhs, precond=pre, restart=30, tol=1e-14, max_iters=30)
    E = torch.zeros((n, n), dtype=torch.complex64, device="cuda")
    for k in [1, 2, 3, 5, 8, 13, 21, 30]:
        if transpose:
            rc, st = S.solve_adjoint(_t(J), E, restart=30, max_iters=k, tol=1e-14, precond=precond)
            xk, _ = OK.fgmres(lambda v: A @ v, rhs, precond=pre, restart=30, tol=1e-14, max_iters=k)
            lam = Dm * xk
            ref = np.linalg.norm(g - A.T @ lam) / np.linalg.norm(g)
            got = OF.relres(A.T.tocsr(), E.cpu().numpy().ravel(), g)
        else:
            rc, st = S.solve(_t(J), E, restart=30, max_iters=k, tol=1e-14, precond=precond)
            ref = info["history"][k]
            got = OF.relres(A, E.cpu().numpy().ravel(), rhs)
        assert rc == F.NOT_CONVERGED and st["iters"] == k
        assert abs(st["relres_true"] - ref) <= 2e-4 * ref, (k, st, ref)
        # the returned field's residual (computed here in FP64 by the oracle's CSR)
        assert abs(got - st["relres_true"]) <= 1e-3 * st["relres_true"]


def test_solve_edge_cases(F):
    n = 128
    dx = LAM / 25
    eps = wl.rectangles_eps(n, n, npml=20, n_rect=4, seed=3)
    S = _solver(F, eps, dx)
    import torch
    E = torch.ones((n, n), dtype=torch.complex64, device="cuda")
    rc, st = S.solve(torch.zeros_like(E), E, max_iters=10, precond=1)
    assert rc == F.OK and not torch.any(E)
    J = torch.zeros_like(E)
    J[3, 4] = float("nan")
    with pytest.raises(F.FDFDError) as ex:
        S.solve(J, E, max_iters=5, precond=1)
    assert ex.value.code == F.ENUMERIC
    with pytest.raises(F.FDFDError):
        S.solve(J, E, restart=0)
    with pytest.raises(F.FDFDError) as ex:
        S.solve(torch.ones_like(E), E, precond=2)  # Schwarz needs set-up
    assert ex.value.code == F.ENOSETUP
    # host-buffer entry point equals the device one
    Jh = wl.random_field(n, n, 9)
    Eh = np.zeros_like(Jh)
    rc1, st1 = S.solve_host(Jh, Eh, max_iters=12, precond=1)
    rc2, st2 = S.solve(_t(Jh), E, max_iters=12, precond=1)
    assert rc1 == rc2 == F.NOT_CONVERGED
    assert np.array_equal(Eh, E.cpu().numpy())
