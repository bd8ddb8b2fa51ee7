"""Two-level Schwarz neural-operator FGMRES (Sec. 2.2, Algorithm 3 as the
flexible preconditioner, Galerkin coarse space) against the FP64 oracle:

* the coarse solve by block elimination over window rows equals a dense
  solve of the exported Galerkin matrix;
* converged fields on the 256^2 rectangles workload (4 x 4 windows, interior
  windows included) match SuperLU to 1e-5 relative L2, the two-level solve
  needing fewer outer iterations than the one-level one; on the 1024^2
  freeform workload the reported residual is pinned to the oracle's;
* the adjoint gradient on the 256^2 workload matches the SuperLU adjoint
  gradient to 1e-3;
* a lock-step batch of uneven problems at three wavelengths gives each
  problem's direct solution (batching pattern, Fig. 1a)."""
import os

import numpy as np
import pytest

from oracle import fdfd as OF
from paper_2509_03622_gb300 import workloads as wl

LAM = 1.55e-6
pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
K = 64       # coarse basis vectors per window
INNER = 16   # NN-FGMRES steps per local solve
FIELD_TOL = 1e-5


def _weights():
    return np.load(os.path.join(ROOT, "paper_2509_03622_gb300", "weights", "nno_trained.npy"))


def _dense_G(G, nwx, nwy, k):
    n = nwx * nwy * k
    D = np.zeros((n, n), complex)
    for i in range(nwx * nwy):
        a, b = i % nwx, i // nwx
        for j in range(9):
            a2, b2 = a + j % 3 - 1, b + j // 3 - 1
            if 0 <= a2 < nwx and 0 <= b2 < nwy:
                J = b2 * nwx + a2
                D[i * k:(i + 1) * k, J * k:(J + 1) * k] = G[i, j]
            else:
                assert not np.any(G[i, j])
    return D


@pytest.mark.parametrize("case", ["rect256", "freeform512"])
def test_coarse_block_solve_matches_dense_solve(case):
    """z = G^-1 (-Q^H e) by the forward/backward row sweeps vs
    numpy.linalg.solve of the same exported FP64 Galerkin matrix.  Bound:
    the sweeps read each inverted Schur complement stored as complex half
    (11 significant bits, relative rounding at most 2^-11 = 4.9e-4 per
    entry); with G close to -I the solution carries about that, times the
    few rows its error passes through, so 2e-3."""
    import torch
    from paper_2509_03622_gb300 import fdfd as F
    w = wl.workload(case)
    S = F.Solver(torch.from_numpy(w["eps"]).cuda(), w["dx"], w["wavelength"], npml=20)
    S.schwarz_setup(_weights(), k_coarse=K)
    inf = S.info()
    nw, nwx, nwy = inf["n_win"], inf["nwx"], inf["nwy"]
    Q, G = S.coarse_export()
    D = _dense_G(G, nwx, nwy, K)
    g = wl.rng(21)
    e = (g.standard_normal((nw, 4, 80)) + 1j * g.standard_normal((nw, 4, 80))).astype(np.complex64)
    z = torch.zeros((nw, K), dtype=torch.complex64, device="cuda")
    S.coarse_solve(torch.from_numpy(e).cuda(), z)
    rhs = -np.einsum("wmsl,wsl->wm", Q.conj(), e.astype(complex)).ravel()
    zr = np.linalg.solve(D, rhs)
    err = np.linalg.norm(z.cpu().numpy().ravel() - zr) / np.linalg.norm(zr)
    print(f"{case}: coarse block solve vs dense solve {err:.2e}")
    assert err < 2e-3, err
    S.close()


def _solve(case, k, inner, tol=1e-7, max_iters=4000):
    import torch
    from paper_2509_03622_gb300 import fdfd as F
    w = wl.workload(case)
    S = F.Solver(torch.from_numpy(w["eps"]).cuda(), w["dx"], w["wavelength"], npml=20)
    S.schwarz_setup(_weights(), k_coarse=k, inner_iters=inner)
    E = torch.zeros(w["eps"].shape, dtype=torch.complex64, device="cuda")
    rc, st = S.solve(torch.from_numpy(w["J"]).cuda(), E, restart=30, max_iters=max_iters, tol=tol)
    S.close()
    return w, rc, st, E.cpu().numpy()


@pytest.mark.parametrize("case", ["rect256"])
def test_two_level_solve_matches_direct_oracle(case):
    from paper_2509_03622_gb300 import fdfd as F
    w, rc, st, E = _solve(case, K, INNER)
    assert rc == F.OK, st
    Eo = OF.solve_direct(w["eps"], w["J"], w["dx"], w["wavelength"], 20)
    err = np.linalg.norm(E - Eo) / np.linalg.norm(Eo)
    print(f"{case}: two-level iterations {st['iters']}, field error vs SuperLU {err:.2e}")
    assert err < FIELD_TOL, (err, st)
    _, rc1, st1, _ = _solve(case, 0, INNER, max_iters=st["iters"])
    assert rc1 != F.OK and st1["relres_true"] > 1e-7  # one level is not there yet after as many steps


def test_two_level_freeform1024_residual_pinned():
    """The 1024^2 freeform workload (16 x 16 windows): the trained network's
    two-level FGMRES does not reach 1e-7 in a test-sized run, so this case is
    pinned by its residual: after 300 steps the FP64 relative residual the
    library reports equals the oracle's CSR residual of the returned field,
    and it is below the one-level residual after the same steps."""
    from paper_2509_03622_gb300 import fdfd as F
    w, rc, st, E = _solve("freeform1024", K, INNER, max_iters=300)
    A = OF.assemble_operator(w["eps"], w["dx"], w["wavelength"], 20)
    b = OF.source_rhs(w["J"], w["dx"], w["wavelength"])
    rr = OF.relres(A, E.ravel(), b)
    print(f"freeform1024: two-level relres after {st['iters']} steps {st['relres_true']:.3e} (oracle CSR {rr:.3e})")
    assert abs(rr - st["relres_true"]) <= 1e-3 * rr + 1e-7
    _, rc1, st1, _ = _solve("freeform1024", 0, INNER, max_iters=300)
    print(f"freeform1024: one-level relres after {st1['iters']} steps {st1['relres_true']:.3e}")
    assert st["relres_true"] < st1["relres_true"]


def test_two_level_adjoint_gradient_rect256():
    """dF/deps on the 256^2 rectangles workload through the library's forward
    and adjoint two-level solves vs the SuperLU adjoint gradient."""
    import torch
    from paper_2509_03622_gb300 import fdfd as F
    from paper_2509_03622_gb300.autograd import fdfd_field, mode_overlap, last_stats
    w = wl.workload("rect256")
    n, dx = 256, w["dx"]
    eps, J = w["eps"], w["J"]
    port_x, y0, nm = 200, 116, 24
    mode = np.exp(-((np.arange(nm) - (nm - 1) / 2) / 5.0) ** 2).astype(np.complex64)
    S = F.Solver(torch.from_numpy(eps).cuda(), dx, LAM, npml=20)
    e_t = torch.from_numpy(eps).cuda().requires_grad_(True)
    E = fdfd_field(S, e_t, torch.from_numpy(J).cuda(), _weights(), restart=30, max_iters=4000, tol=1e-7,
                   precond=F.PRECOND_SCHWARZ, k_coarse=K, inner=INNER)
    Fv = mode_overlap(E, port_x, torch.from_numpy(mode).cuda(), y0, dx).abs() ** 2
    Fv.backward()
    assert last_stats["forward"]["status"] == F.OK and last_stats["adjoint"]["status"] == F.OK, last_stats
    A = OF.assemble_operator(eps, dx, LAM, 20)
    Sd = OF.DirectSolver(A)
    Eo = Sd.solve(OF.source_rhs(J, dx, LAM)).reshape(n, n)
    Fo, g = OF.fom_and_adjoint_source(Eo, port_x, mode.astype(complex), y0, dx)
    lam = Sd.solve_transpose(g.ravel()).reshape(n, n)
    g_ref = OF.grad_eps(Eo, lam, dx, LAM)
    inner = np.zeros((n, n), bool)
    inner[20:-20, 20:-20] = True
    g_gpu = e_t.grad.cpu().numpy().astype(np.float64)
    err = np.linalg.norm((g_gpu - g_ref)[inner]) / np.linalg.norm(g_ref[inner])
    assert abs(float(Fv.detach()) - Fo) <= 1e-4 * Fo
    assert err < 1e-3, err
    S.close()


def test_batched_uneven_problems_match_direct_oracle():
    """Three problems of uneven grids (freeform recipe, fixed dx) at
    1.31 / 1.55 / 1.80 um solved in lock step, each with its own two-level
    preconditioner: every field matches its own SuperLU solution."""
    import torch
    from paper_2509_03622_gb300 import fdfd as F
    specs = [(256, 256, 1.31e-6), (320, 256, 1.55e-6), (256, 384, 1.80e-6)]
    dx = 1.55e-6 / 30
    solvers, Js, cases = [], [], []
    for i, (nx, ny, lam) in enumerate(specs):
        eps = wl.freeform_eps(nx, ny, seed=3000 + i)
        J = wl.point_source(nx, ny)
        S = F.Solver(torch.from_numpy(np.ascontiguousarray(eps)).cuda(), dx, lam, npml=20)
        S.schwarz_setup(_weights(), k_coarse=K, inner_iters=INNER)
        solvers.append(S)
        Js.append(torch.from_numpy(J).cuda())
        cases.append((eps, J, lam))
    B = F.Batch(solvers)
    Es = [torch.zeros_like(J) for J in Js]
    rc, stats = B.solve(Js, Es, restart=30, max_iters=4000, tol=1e-7, precond=F.PRECOND_SCHWARZ)
    for (eps, J, lam), E, st in zip(cases, Es, stats):
        assert st["status"] == F.OK, st
        Eo = OF.solve_direct(eps, J, dx, lam, 20)
        err = np.linalg.norm(E.cpu().numpy() - Eo) / np.linalg.norm(Eo)
        assert err < FIELD_TOL, (err, st)
    B.close()
    for S in solvers:
        S.close()


def _its(eps, dx, J, k, inner=16, tol=1e-6, max_iters=2000):
    import torch
    from paper_2509_03622_gb300 import fdfd as F
    S = F.Solver(torch.from_numpy(np.ascontiguousarray(eps)).cuda(), dx, LAM, npml=20)
    S.schwarz_setup(_weights(), k_coarse=k, inner_iters=inner)
    E = torch.zeros(eps.shape, dtype=torch.complex64, device="cuda")
    rc, st = S.solve(torch.from_numpy(J).cuda(), E, restart=30, max_iters=max_iters, tol=tol)
    S.close()
    assert rc == F.OK, st
    return st["iters"]


def test_table1_trend_homogeneous():
    """Table 1's trend with the library's kernels and the trained network:
    a homogeneous medium at 24 cells per wavelength with 4 x 4, 8 x 8 and
    16 x 16 windows, FGMRES(30) to 1e-6 with 16 NN-FGMRES steps per local
    solve.  The two-level solve (36 coarse vectors per window) needs fewer
    outer iterations than the one-level one at every size, and its count
    grows less from 4 x 4 to 16 x 16 (measured on GB300: one level 252 /
    345 / 482, two levels 186 / 211 / 240)."""
    one, two = [], []
    for n in (256, 512, 1024):
        eps = np.ones((n, n), np.float32)
        J = wl.point_source(n, n)
        one.append(_its(eps, LAM / 24, J, 0))
        two.append(_its(eps, LAM / 24, J, 36))
    print(f"homogeneous 4x4 / 8x8 / 16x16 windows: one level {one}, two levels {two}")
    assert all(b < a for a, b in zip(one, two)), (one, two)
    assert two[-1] / two[0] < one[-1] / one[0], (one, two)
    assert two[-1] / two[0] < 1.6, two


def test_demux512_two_level_converges():
    """The inverse-design workload (512^2 demultiplexer, 8 x 8 windows, the
    waveguide source): the two-level solve reaches 1e-6 and takes fewer outer
    iterations than the one-level one (measured on GB300: 878 vs 1195)."""
    base, mask, src_x, yin, port_x, port_rows = wl.demux_layout(512)
    J = np.zeros((512, 512), np.complex64)
    J[yin[0] - 4:yin[1] + 4, src_x] = 1.0
    two = _its(base, LAM / 30, J, 64)
    one = _its(base, LAM / 30, J, 0)
    print(f"demux512: two levels {two}, one level {one}")
    assert two < one, (two, one)
