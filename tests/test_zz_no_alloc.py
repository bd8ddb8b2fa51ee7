"""fdfd_nno_solve_noalloc -- the neural local solve for callers that cannot
allocate device memory (code bound to a memory budget its own pool allocator
hands out, or a loop that cannot afford the synchronisation an allocation may
cause) -- gives exactly the results of fdfd_nno_solve (the same kernels on
the same inputs), on two calls in a row, and allocates nothing.  Collected
last on purpose (file name)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
LAM = 1.55e-6


def _batch(seed, nwin):
    from paper_2509_03622_gb300 import workloads as wl
    g = wl.rng(seed)
    r = (g.standard_normal((nwin, 80, 80)) + 1j * g.standard_normal((nwin, 80, 80))).astype(np.complex64)
    gb = (g.standard_normal((nwin, 4, 80)) + 1j * g.standard_normal((nwin, 4, 80))).astype(np.complex64)
    return r, gb


def _solver():
    import torch
    from paper_2509_03622_gb300 import fdfd as F
    from paper_2509_03622_gb300 import workloads as wl
    n, dx = 256, LAM / 25
    eps = wl.rectangles_eps(n, n, seed=1000)
    S = F.Solver(torch.from_numpy(eps).cuda(), dx, LAM, npml=20)
    S.schwarz_setup(wl.pack_weights(wl.nno_weights(0)))
    return S


def _cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_noalloc_nno_solve_matches_nno_solve():
    import torch
    from paper_2509_03622_gb300 import fdfd as F
    S = _solver()
    ws = S.info()["workspace_bytes"]
    for call, ids in enumerate([[0, 5, 15, 3], [10, 1, 6]]):  # two calls in a row, 4 then 3 windows
        ids = np.array(ids, dtype=np.int32)
        r, gb = _batch(100 + call, len(ids))
        e_ref = torch.empty((len(ids), 80, 80), dtype=torch.complex64, device="cuda")
        S.nno_solve(_cuda(r), _cuda(gb), _cuda(ids), e_ref)
        e_na = torch.full_like(e_ref, float("nan"))
        args = (_cuda(r), _cuda(gb), _cuda(ids), e_na)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        torch_before = torch.cuda.memory_allocated()
        S.nno_solve_noalloc(*args)
        torch.cuda.synchronize()
        free_after = torch.cuda.mem_get_info()[0]
        a, b = e_ref.cpu().numpy(), e_na.cpu().numpy()
        assert np.all(np.isfinite(b))
        # same kernels, same variant, same inputs: identical to the last bit
        assert np.array_equal(a, b), (call, np.max(np.abs(a - b)))
        assert torch.cuda.memory_allocated() == torch_before
        assert S.info()["workspace_bytes"] == ws
        if call > 0:  # after the first call's one-time look-up nothing is allocated
            assert free_after == free_before
    # beyond the stated maximum: a clear error and no work
    r, gb = _batch(7, 5)
    ids = np.arange(5, dtype=np.int32)
    out = torch.zeros((5, 80, 80), dtype=torch.complex64, device="cuda")
    with pytest.raises(F.FDFDError) as ex:
        S.nno_solve_noalloc(_cuda(r), _cuda(gb), _cuda(ids), out)
    assert ex.value.code == F.EINVAL
    assert not torch.any(out)
    S.close()


def test_noalloc_reports_the_handles_failure():
    """After a neural pass of the handle gave up (injected on the host), the
    no-allocation call reports the same FDFD_ETIMEOUT as fdfd_nno_solve and
    writes nothing."""
    import torch
    from paper_2509_03622_gb300 import fdfd as F
    S = _solver()
    S.nno_mark_failed()
    r, gb = _batch(9, 2)
    ids = np.array([2, 7], dtype=np.int32)
    for fn in (S.nno_solve, S.nno_solve_noalloc):
        out = torch.zeros((2, 80, 80), dtype=torch.complex64, device="cuda")
        with pytest.raises(F.FDFDError) as ex:
            fn(_cuda(r), _cuda(gb), _cuda(ids), out)
        assert ex.value.code == F.ETIMEOUT
    assert not torch.any(out)  # the no-allocation call launched nothing
    S.close()
