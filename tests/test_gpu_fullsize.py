"""Parity at the bench's full size, in the bench's launch configuration:
the one-level Schwarz sweep on the freeform 4096x4096 workload (4096 windows,
every neural stage launched once over all windows) against the FP64 oracle's
neural local solve, computed window by window on a sample of windows (the
four corners, edge windows and seeded interior ones)."""
import numpy as np
import pytest

from oracle import fdfd as OF
from oracle import nno as ON
from oracle import partition as OP
from paper_2509_03622_gb300 import workloads as wl

pytestmark = pytest.mark.gpu
LAM = 1.55e-6
BF16_TOL = 3e-2  # relative L2, as for the smaller sweeps (seeded weights)


def test_precond_4096_sampled_windows_match_oracle():
    import torch
    from paper_2509_03622_gb300 import fdfd as F
    n, npml = 4096, 20
    dx = LAM / 30
    eps = wl.freeform_eps(n, n, seed=2000 + n)  # the bench's freeform4096 recipe
    w = wl.nno_weights(0)
    S = F.Solver(torch.from_numpy(eps).cuda(), dx, LAM, npml=npml)
    S.schwarz_setup(wl.pack_weights(w), k_coarse=0)
    v = wl.random_field(n, n, 4096)
    z = torch.empty((n, n), dtype=torch.complex64, device="cuda")
    S.precond_apply(torch.from_numpy(v).cuda(), z)
    zc = z.cpu().numpy()
    assert np.isfinite(zc).all()

    win = OP.Windows(n, n)
    sxn, _, syn, _ = OF.pml_factors(n, n, dx, LAM, npml)
    isx, isy = 1.0 / sxn, 1.0 / syn
    k2 = OF.k0dx_of(dx, LAM) ** 2
    nw = win.nwx
    rng = np.random.default_rng(7)
    sample = sorted({0, nw - 1, win.n - nw, win.n - 1, nw // 2, (nw // 2) * nw, *rng.integers(0, win.n, 6).tolist()})
    num = den = 0.0
    for wi in sample:
        x0, y0 = int(win.x0[wi]), int(win.y0[wi])
        r = v[y0:y0 + 80, x0:x0 + 80].astype(np.complex128)
        e = ON.solve(r, np.zeros((4, 80)), k2 * eps[y0:y0 + 80, x0:x0 + 80].astype(np.float64),
                     isx[x0:x0 + 80], isy[y0:y0 + 80], w)
        cx, cy = win.core_offset(wi)
        a, b = wi % nw, wi // nw
        ref = e[cy:cy + 64, cx:cx + 64]
        got = zc[64 * b:64 * b + 64, 64 * a:64 * a + 64]
        d = np.linalg.norm(got - ref) ** 2
        num += d
        den += np.linalg.norm(ref) ** 2
        assert np.sqrt(d) / np.linalg.norm(ref) < 2 * BF16_TOL, (wi, np.sqrt(d) / np.linalg.norm(ref))
    assert np.sqrt(num / den) < BF16_TOL, np.sqrt(num / den)


BENCH_K, BENCH_INNER = 64, 2  # the bench's two-level configuration


def _trained():
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    return np.load(os.path.join(root, "paper_2509_03622_gb300", "weights", "nno_trained.npy"))


def test_precond_4096_trained_inner_sampled_windows_match_oracle():
    """The bench's local solver at full size: the trained network inside
    BENCH_INNER steps of NN-FGMRES per window (one-level sweep, 4096 windows
    in each launch) vs the oracle's NN-FGMRES on the same windows."""
    import torch
    from oracle import krylov as OK
    from paper_2509_03622_gb300 import fdfd as F
    n, npml = 4096, 20
    dx = LAM / 30
    eps = wl.freeform_eps(n, n, seed=2000 + n)
    blob = _trained()
    w = wl.unpack_weights(blob)
    S = F.Solver(torch.from_numpy(eps).cuda(), dx, LAM, npml=npml)
    S.schwarz_setup(blob, k_coarse=0, inner_iters=BENCH_INNER)
    v = wl.random_field(n, n, 4097)
    z = torch.empty((n, n), dtype=torch.complex64, device="cuda")
    S.precond_apply(torch.from_numpy(v).cuda(), z)
    zc = z.cpu().numpy()
    assert np.isfinite(zc).all()
    A = OF.assemble_operator(eps, dx, LAM, npml)
    win = OP.Windows(n, n)
    sxn, _, syn, _ = OF.pml_factors(n, n, dx, LAM, npml)
    k2 = OF.k0dx_of(dx, LAM) ** 2
    nw = win.nwx
    rng = np.random.default_rng(8)
    sample = sorted({0, nw - 1, win.n - 1, (nw // 2) * nw + nw // 2, *rng.integers(0, win.n, 4).tolist()})
    num = den = 0.0
    for wi in sample:
        x0, y0 = int(win.x0[wi]), int(win.y0[wi])
        Aw, bnd = OP.local_operator(win, wi, A, eps, dx, LAM)
        rhs = v[y0:y0 + 80, x0:x0 + 80].astype(np.complex128).ravel()
        aux = (k2 * eps[y0:y0 + 80, x0:x0 + 80].astype(np.float64), 1 / sxn[x0:x0 + 80], 1 / syn[y0:y0 + 80])
        M = lambda q: ON.solve(q.reshape(80, 80), np.zeros((4, 80)), *aux, w).ravel()
        e, _ = OK.fgmres(lambda u: Aw @ u, rhs, precond=M, restart=BENCH_INNER, tol=0.0, max_iters=BENCH_INNER)
        e = e.reshape(80, 80)
        cx, cy = win.core_offset(wi)
        a, b = wi % nw, wi // nw
        ref = e[cy:cy + 64, cx:cx + 64]
        got = zc[64 * b:64 * b + 64, 64 * a:64 * a + 64]
        num += np.linalg.norm(got - ref) ** 2
        den += np.linalg.norm(ref) ** 2
    err = np.sqrt(num / den)
    print(f"trained network, {BENCH_INNER} inner steps, 4096^2 sampled windows: {err:.3e}")
    assert err < 2 * BF16_TOL, err


def test_coarse_4096_galerkin_residual():
    """The bench's coarse level at full size (4096 windows, k = 64): the
    solve by block elimination over the 64 window rows satisfies its
    Galerkin system, ||G z + Q^H e|| <= 2e-3 ||Q^H e|| (the sweeps read the
    inverted Schur complements stored as complex half, relative rounding
    at most 2^-11 = 4.9e-4 per entry), checked block by block against the
    exported FP64 blocks."""
    import torch
    from paper_2509_03622_gb300 import fdfd as F
    n, npml = 4096, 20
    dx = LAM / 30
    eps = wl.freeform_eps(n, n, seed=2000 + n)
    S = F.Solver(torch.from_numpy(eps).cuda(), dx, LAM, npml=npml)
    S.schwarz_setup(_trained(), k_coarse=BENCH_K, inner_iters=BENCH_INNER)
    inf = S.info()
    nw, nwx, nwy = inf["n_win"], inf["nwx"], inf["nwy"]
    g = wl.rng(99)
    e = (g.standard_normal((nw, 4, 80)) + 1j * g.standard_normal((nw, 4, 80))).astype(np.complex64)
    zt = torch.zeros((nw, BENCH_K), dtype=torch.complex64, device="cuda")
    S.coarse_solve(torch.from_numpy(e).cuda(), zt)
    z = zt.cpu().numpy().astype(np.complex128)
    Q, G = S.coarse_export()
    S.close()
    rhs = -np.einsum("wmsl,wsl->wm", Q.conj(), e.astype(np.complex128))
    Gz = np.zeros_like(rhs)
    a = np.arange(nw) % nwx
    b = np.arange(nw) // nwx
    for j in range(9):
        a2, b2 = a + j % 3 - 1, b + j // 3 - 1
        ok = (a2 >= 0) & (a2 < nwx) & (b2 >= 0) & (b2 < nwy)
        J = np.where(ok, b2 * nwx + a2, 0)
        Gz += np.where(ok[:, None], np.einsum("wpq,wq->wp", G[:, j], z[J]), 0)
    res = np.linalg.norm(Gz - rhs) / np.linalg.norm(rhs)
    print(f"coarse Galerkin residual at 4096 windows, k = {BENCH_K}: {res:.2e}")
    assert np.isfinite(z).all() and res < 2e-3, res
