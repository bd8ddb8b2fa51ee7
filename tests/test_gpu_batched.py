"""Batching pattern: lock-step solves of uneven problems at different
wavelengths, one neural pass over all their windows per Arnoldi step, give
the same iterates as the individual solves."""
import numpy as np
import pytest

from paper_2509_03622_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precond", [2, 1])
def test_batched_equals_individual(precond):
    import torch
    from paper_2509_03622_gb300 import fdfd as F
    specs = [(128, 128, 1.31e-6), (256, 192, 1.55e-6), (192, 256, 1.80e-6)]
    dx = 1.55e-6 / 30
    solvers, Js = [], []
    blob = wl.pack_weights(wl.nno_weights(2))
    for i, (nx, ny, lam) in enumerate(specs):
        eps = wl.freeform_eps(nx, ny, seed=300 + i)
        S = F.Solver(torch.from_numpy(np.ascontiguousarray(eps)).cuda(), dx, lam, npml=20)
        if precond == 2:
            S.schwarz_setup(blob, k_coarse=0)
        solvers.append(S)
        Js.append(torch.from_numpy(wl.random_field(nx, ny, 40 + i)).cuda())
    ref = []
    for S, J in zip(solvers, Js):
        E = torch.zeros_like(J)
        rc, st = S.solve(J, E, restart=8, max_iters=20, tol=1e-12, precond=precond)
        ref.append((E.cpu().numpy(), st))
    B = F.Batch(solvers, max_windows=7)  # forces several chunks of windows
    Es = [torch.zeros_like(J) for J in Js]
    rc, stats = B.solve(Js, Es, restart=8, max_iters=20, tol=1e-12, precond=precond)
    for (Er, sr), E, sb in zip(ref, Es, stats):
        assert sb["iters"] == sr["iters"] == 20
        assert abs(sb["relres_true"] - sr["relres_true"]) <= 1e-6 * sr["relres_true"]
        e = E.cpu().numpy()
        assert np.linalg.norm(e - Er) <= 1e-6 * np.linalg.norm(Er)
    B.close()
