"""Pins of the neural-operator oracle (Fig. 2): the FFT convolution against
explicit DFT sums, the mode-truncation projector, positive homogeneity."""
import numpy as np

from oracle import nno
from paper_2509_03622_gb300 import workloads as wl


def _brute_spectral(h, R):
    """Explicit sums: H[ky,kx] = sum h e^{-2 pi i (ky y + kx x)/80};
    inverse real DFT with Hermitian weights (1 for kx = 0, 2 otherwise,
    real part only)."""
    n = h.shape[-1]
    y = np.arange(n)
    rows = nno.retained_rows(n)
    Fy = np.exp(-2j * np.pi * np.outer(rows, y) / n)          # [32][80]
    Fx = np.exp(-2j * np.pi * np.outer(np.arange(16), y) / n)  # [16][80]
    H = np.einsum("qy,cyx,kx->cqk", Fy, h, Fx)
    Y = np.einsum("oiqk,iqk->oqk", R, H)
    T = np.einsum("yq,oqk->oyk", np.conj(Fy).T, Y) / n          # ifft along y
    wts = np.where(np.arange(16) == 0, 1.0, 2.0)
    ph = np.exp(2j * np.pi * np.outer(np.arange(16), y) / n)  # [16][80]
    return np.einsum("k,oyk,kx->oyx", wts, T, ph).real / n


def test_spectral_conv_matches_explicit_dft():
    g = wl.rng(3)
    h = g.standard_normal((3, 80, 80))
    R = g.standard_normal((2, 3, 32, 16)) + 1j * g.standard_normal((2, 3, 32, 16))
    a = nno.spectral_conv(h, R)
    b = _brute_spectral(h, R)
    assert np.max(np.abs(a - b)) < 1e-10 * np.max(np.abs(b))


def test_mode_truncation_is_a_projector():
    I = np.zeros((1, 1, 32, 16), complex)
    I[0, 0] = 1.0
    x = np.arange(80)
    # a real field made of retained modes (ky = 5, kx = 3) and (ky = -9, kx = 0)
    f = np.cos(2 * np.pi * (3 * x[None, :] + 5 * x[:, None]) / 80) + 0.5 * np.cos(2 * np.pi * 9 * x[:, None] / 80)
    assert np.allclose(nno.spectral_conv(f[None], I)[0], f, atol=1e-12)
    # a dropped mode (kx = 20) vanishes; a second application changes nothing
    g = np.cos(2 * np.pi * 20 * x[None, :] / 80) * np.ones((80, 1))
    assert np.max(np.abs(nno.spectral_conv(g[None], I))) < 1e-12
    # random real field band-limited to |ky| <= 15, kx <= 15 is reproduced
    # (ky = -16 at kx = 0 is kept without its Hermitian partner, so the
    # truncation is exactly a projector only on such fields)
    gen = wl.rng(1)
    F = np.zeros((80, 41), complex)
    rows = np.r_[0:16, 65:80]
    F[np.ix_(rows, np.arange(16))] = gen.standard_normal((31, 16)) + 1j * gen.standard_normal((31, 16))
    r = np.fft.irfft2(F, s=(80, 80))[None]
    assert np.allclose(nno.spectral_conv(r, I), r, atol=1e-12)


def test_zero_spectral_weights_reduce_to_pointwise_network():
    w = wl.nno_weights(seed=5)
    for b in range(4):
        w[f"R{b}_re"][:] = 0
        w[f"R{b}_im"][:] = 0
    x = wl.rng(2).standard_normal((15, 80, 80))
    out = nno.forward(x, w)
    for (py, px) in [(0, 0), (13, 71), (79, 40)]:
        h = w["lift_w"].astype(float) @ x[:, py, px] + w["lift_b"]
        for b in range(4):
            h = w[f"W{b}"].astype(float) @ h + w[f"b{b}"]
            if b < 3:
                h = np.maximum(h, 0.01 * h)
        q = w["p1_w"].astype(float) @ h + w["p1_b"]
        q = np.maximum(q, 0.01 * q)
        o = w["p2_w"].astype(float) @ q + w["p2_b"]
        assert np.allclose(out[:, py, px], o, rtol=1e-12, atol=1e-12)


def test_solve_is_positively_homogeneous_and_zero_safe():
    w = wl.nno_weights(seed=1)
    g = wl.rng(4)
    r = g.standard_normal((80, 80)) + 1j * g.standard_normal((80, 80))
    gb = g.standard_normal((4, 80)) + 1j * g.standard_normal((4, 80))
    k2e = 0.06 * np.ones((80, 80))
    isx = np.ones(80, complex)
    isy = np.ones(80, complex)
    e1 = nno.solve(r, gb, k2e, isx, isy, w)
    e2 = nno.solve(3.5 * r, 3.5 * gb, k2e, isx, isy, w)
    assert np.allclose(e2, 3.5 * e1, rtol=1e-12, atol=0)
    assert not np.any(nno.solve(0 * r, 0 * gb, k2e, isx, isy, w))
