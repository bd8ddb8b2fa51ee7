"""The PyTorch training twin (local Robin operator, UPML sampler, FNO
forward) agrees with the FP64 oracle on the CPU, so the trained weights
target the operator the solver actually uses."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import fdfd as OF, nno as ON, partition as OP
from paper_2509_03622_gb300 import train as T
from paper_2509_03622_gb300 import workloads as wl

LAM = 1.55e-6


def _P_from_oracle(n, dx, eps, win, w):
    sxn, sxh, syn, syh = OF.pml_factors(n, n, dx, LAM, 20)
    x0, y0 = int(win.x0[w]), int(win.y0[w])
    c = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(torch.complex64)[None]
    xlo = 1 / (sxn[x0:x0 + 80] * sxh[x0:x0 + 80])
    xhi = 1 / (sxn[x0:x0 + 80] * sxh[x0 + 1:x0 + 81])
    ylo = 1 / (syn[y0:y0 + 80] * syh[y0:y0 + 80])
    yhi = 1 / (syn[y0:y0 + 80] * syh[y0 + 1:y0 + 81])
    return dict(k0dx=torch.tensor([OF.k0dx_of(dx, LAM)], dtype=torch.float32),
                eps=torch.from_numpy(eps[y0:y0 + 80, x0:x0 + 80].copy())[None],
                sxn=c(sxn[x0:x0 + 80]), syn=c(syn[y0:y0 + 80]), xlo=c(xlo), xhi=c(xhi), ylo=c(ylo), yhi=c(yhi),
                robin=torch.tensor(win.interface[w][None]))


@pytest.mark.parametrize("w", [0, 1, 4, 8])
def test_local_operator_twin_matches_oracle(w):
    n, dx = 192, LAM / 25
    eps = wl.rectangles_eps(n, n, npml=20, n_rect=10, seed=4)
    A = OF.assemble_operator(eps, dx, LAM, 20)
    win = OP.Windows(n, n)
    Aw, bnd = OP.local_operator(win, w, A, eps, dx, LAM)
    P = _P_from_oracle(n, dx, eps, win, w)
    e = wl.random_field(80, 80, w)
    got = T.local_apply(torch, torch.from_numpy(e)[None], P)[0].numpy()
    ref = (Aw @ e.astype(complex).ravel()).reshape(80, 80)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-5
    g = wl.random_field(80, 4, 9)  # [4][80]
    gb = T.boundary_rhs(torch, torch.from_numpy(g)[None], P)[0].numpy()
    ref_b = OP.local_rhs(np.zeros((80, 80)), g * win.interface[w][:, None], bnd).reshape(80, 80)
    assert np.linalg.norm(gb - ref_b) <= 1e-5 * np.linalg.norm(ref_b) + 1e-12


def test_sampler_pml_matches_global_profile():
    """A window at the low grid edge gets the global UPML factors."""
    S = T.Sampler(torch, torch.device("cpu"), 64)
    torch.manual_seed(0)
    k0dx = torch.full((64,), 2 * np.pi / 25)
    sn, lo, hi, rl, rh = S.axis(k0dx)
    sxn, sxh = OF.pml_stretch(256, 20, 20, LAM / 25, LAM)
    m = (~rl).nonzero()[0, 0]
    assert np.allclose(sn[m].numpy(), sxn[:80], rtol=1e-5)
    assert np.allclose(lo[m].numpy(), 1 / (sxn[:80] * sxh[:80]), rtol=1e-5)
    m2 = (~rh).nonzero()[0, 0]
    assert np.allclose(sn[m2].numpy(), sxn[-80:], rtol=1e-5)
    assert np.allclose(hi[m2].numpy(), 1 / (sxn[-80:] * sxh[-80:]), rtol=1e-5)


def test_fno_twin_matches_oracle():
    w = wl.nno_weights(3)
    model = T.build_model(torch, w)
    x = wl.rng(5).standard_normal((2, 15, 80, 80)).astype(np.float32)
    with torch.no_grad():
        got = model(torch.from_numpy(x)).numpy()
    for i in range(2):
        ref = ON.forward(x[i], w)
        assert np.linalg.norm(got[i] - ref) / np.linalg.norm(ref) < 1e-4
    back = wl.unpack_weights(wl.pack_weights(model.export()))
    for k in w:
        assert np.array_equal(back[k], w[k])


def test_dense_operator_matches_stencil():
    """The dense local operator used for exact training targets equals the
    matrix-free local_apply (and hence the oracle's A_w)."""
    S = T.Sampler(torch, torch.device("cpu"), 2)
    torch.manual_seed(3)
    P = S.batch()
    A = T.dense_operator(torch, P)
    e = torch.randn(2, 80, 80, dtype=torch.complex64)
    y1 = (A @ e.reshape(2, -1, 1)).reshape(2, 80, 80)
    y2 = T.local_apply(torch, e, P)
    assert torch.allclose(y1, y2, rtol=1e-4, atol=1e-5 * y2.abs().max())


def test_modified_fno_twin_matches_oracle():
    """The training model of the modified FNO (modulation path, rank-8 R)
    equals the oracle's forward, and its export round-trips through the
    blob layout the library reads."""
    w = wl.nno_weights(3, rank=8, modulation=True)
    w["mod_fc_w"] *= 20.0
    m = T.build_model(torch, w).double()
    x = wl.rng(12).standard_normal((2, 15, 80, 80))
    out = m(torch.from_numpy(x)).detach().numpy()
    ref = np.stack([ON.forward(x[i], w) for i in range(2)])
    assert np.max(np.abs(out - ref)) < 1e-12 * np.max(np.abs(ref))
    back = wl.unpack_weights(wl.pack_weights(m.export()), rank=8, modulation=True)
    assert all(np.array_equal(back[k], w[k]) for k in w)


def test_exact_local_solve_by_row_elimination():
    """The training targets: block elimination over the window rows solves
    the local Robin problems of the sampler (residual at complex64 level)."""
    torch.manual_seed(1)
    S = T.Sampler(torch, torch.device("cpu"), 3)
    P = S.batch()
    rhs = torch.randn(3, 2, 80, 80, dtype=torch.complex64)
    x = T.exact_local_solve(torch, P, rhs)
    Pe = T.expand(P, 2)
    r = rhs.reshape(6, 80, 80) - T.local_apply(torch, x.reshape(6, 80, 80), Pe)
    rel = (r.abs() ** 2).sum((1, 2)).sqrt() / (rhs.reshape(6, 80, 80).abs() ** 2).sum((1, 2)).sqrt()
    assert float(rel.max()) < 1e-5


def test_sampler_window_kinds_match_large_grids():
    """Most windows of a large grid have no PML side: the sampler draws an
    interior axis (Robin data on both sides) 60% of the time and each grid
    edge 20%, so about 36% of its windows are fully interior, 64% have no PML
    on a given axis, and none has PML on both sides of one axis."""
    S = T.Sampler(torch, torch.device("cpu"), 4000)
    torch.manual_seed(1)
    k0dx = torch.full((4000,), 2 * np.pi / 25)
    _, _, _, rl, rh = S.axis(k0dx)
    interior = (rl & rh).float().mean().item()
    low, high = (~rl).float().mean().item(), (~rh).float().mean().item()
    assert abs(interior - 0.6) < 0.03, interior
    assert abs(low - 0.2) < 0.03 and abs(high - 0.2) < 0.03, (low, high)
    assert not bool(((~rl) & (~rh)).any())
    P = S.batch()
    full = P["robin"].all(1).float().mean().item()
    assert abs(full - 0.36) < 0.04, full
