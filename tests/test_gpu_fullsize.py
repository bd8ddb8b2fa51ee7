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
