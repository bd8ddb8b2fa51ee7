"""fdfd_nno_solve_noalloc -- the neural local solve for callers that cannot
allocate device memory (inside a CUDA-graph capture, under their own memory
pool, or in a loop that cannot afford an allocation's synchronisation) --
gives the same results as fdfd_nno_solve, on two calls in a row, and
allocates nothing.  Collected last on purpose (file name)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
BF16_TOL = 3e-2  # the tolerance the neural-operator parity tests use
LAM = 1.55e-6


def _batch(seed, nwin):
    from paper_2509_03622_gb300 import workloads as wl
    g = wl.rng(seed)
    r = (g.standard_normal((nwin, 80, 80)) + 1j * g.standard_normal((nwin, 80, 80))).astype(np.complex64)
    gb = (g.standard_normal((nwin, 4, 80)) + 1j * g.standard_normal((nwin, 4, 80))).astype(np.complex64)
    return r, gb


def test_noalloc_nno_solve_matches_nno_solve():
    import torch
    from paper_2509_03622_gb300 import fdfd as F
    from paper_2509_03622_gb300 import workloads as wl
    n, dx = 256, LAM / 25
    eps = wl.rectangles_eps(n, n, seed=1000)
    S = F.Solver(torch.from_numpy(eps).cuda(), dx, LAM, npml=20)
    S.schwarz_setup(wl.pack_weights(wl.nno_weights(0)))
    cuda = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    for call, ids in enumerate([[0, 5, 15, 3], [10, 1, 6]]):  # two calls in a row, 4 then 3 windows
        ids = np.array(ids, dtype=np.int32)
        r, gb = _batch(100 + call, len(ids))
        e_ref = torch.empty((len(ids), 80, 80), dtype=torch.complex64, device="cuda")
        S.nno_solve(cuda(r), cuda(gb), cuda(ids), e_ref)
        e_na = torch.full_like(e_ref, float("nan"))
        args = (cuda(r), cuda(gb), cuda(ids), e_na)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        S.nno_solve_noalloc(*args)
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        a, b = e_ref.cpu().numpy(), e_na.cpu().numpy()
        assert np.all(np.isfinite(b))
        err = np.linalg.norm(b - a) / np.linalg.norm(a)
        assert err < BF16_TOL, (call, err)
        if call > 0:  # after the first call's one-time set-up nothing is allocated
            assert free_after == free_before
    # beyond the stated maximum: a clear error and no work
    r, gb = _batch(7, 5)
    ids = np.arange(5, dtype=np.int32)
    out = torch.zeros((5, 80, 80), dtype=torch.complex64, device="cuda")
    with pytest.raises(F.FDFDError) as ex:
        S.nno_solve_noalloc(cuda(r), cuda(gb), cuda(ids), out)
    assert ex.value.code == F.EINVAL
    assert not torch.any(out)
    S.close()
