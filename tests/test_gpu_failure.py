"""Failure detection without a GPU fault: a bounded device wait on a barrier
that nothing arrives on gives up and reports FDFD_ETIMEOUT with the context
still usable, and a neural operator marked failed (host-side injection, the
same flag a timed-out wait sets) stops the solve with FDFD_ETIMEOUT while a
fresh handle still solves."""
import time

import numpy as np
import pytest

from paper_2509_03622_gb300 import workloads as wl

LAM = 1.55e-6
pytestmark = pytest.mark.gpu


def _gemm_ok(F):
    import torch
    rng = np.random.default_rng(5)
    A = rng.standard_normal((128, 64)).astype(np.float32)
    B = rng.standard_normal((64, 64)).astype(np.float32)
    At = torch.from_numpy(A).to(torch.bfloat16).cuda().contiguous()
    Bt = torch.from_numpy(B).to(torch.bfloat16).cuda().contiguous()
    C = torch.zeros((128, 64), dtype=torch.float32, device="cuda")
    F.selftest_gemm(At, Bt, C)
    ref = At.float().cpu().numpy() @ Bt.float().cpu().numpy().T
    return np.max(np.abs(C.cpu().numpy() - ref)) / np.max(np.abs(ref))


def test_bounded_wait_gives_up_and_context_survives():
    from paper_2509_03622_gb300 import fdfd as F
    t0 = time.time()
    rc = F.selftest_wait()
    elapsed = time.time() - t0
    assert rc == F.ETIMEOUT, F.status_string(rc)
    assert elapsed < 30.0, elapsed
    # the CUDA context is intact: the tensor-core path still computes exactly
    assert _gemm_ok(F) < 1e-5


def test_failed_neural_operator_stops_the_solve():
    import torch
    from paper_2509_03622_gb300 import fdfd as F
    n = 128
    eps, dx = wl.freeform_eps(n, n, seed=2128), LAM / 30
    J = torch.from_numpy(wl.point_source(n, n)).cuda()
    blob = wl.pack_weights(wl.nno_weights(0))

    def solver():
        S = F.Solver(torch.from_numpy(eps).cuda(), dx, LAM, npml=20)
        S.schwarz_setup(blob, k_coarse=0)
        return S

    S = solver()
    E = torch.zeros((n, n), dtype=torch.complex64, device="cuda")
    rc, st = S.solve(J, E, restart=30, max_iters=60, tol=1e-12)
    assert rc >= 0, st  # a soft outcome: the healthy handle iterates
    S.nno_mark_failed()
    t0 = time.time()
    with pytest.raises(F.FDFDError) as e:
        S.solve(J, E, restart=30, max_iters=600, tol=1e-12)
    assert e.value.code == F.ETIMEOUT
    assert time.time() - t0 < 30.0
    # the flag stays set for this handle
    z = torch.zeros((n, n), dtype=torch.complex64, device="cuda")
    with pytest.raises(F.FDFDError) as e2:
        S.solve(J, z, restart=30, max_iters=60, tol=1e-12)
    assert e2.value.code == F.ETIMEOUT
    S.close()
    # a fresh handle is unaffected and the context is intact
    S2 = solver()
    E2 = torch.zeros((n, n), dtype=torch.complex64, device="cuda")
    rc2, st2 = S2.solve(J, E2, restart=30, max_iters=60, tol=1e-12)
    assert rc2 >= 0, st2
    assert np.isfinite(E2.cpu().numpy()).all()
    assert _gemm_ok(F) < 1e-5
