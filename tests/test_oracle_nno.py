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


def _window_inputs(seed):
    g = wl.rng(seed)
    r = g.standard_normal((80, 80)) + 1j * g.standard_normal((80, 80))
    gb = g.standard_normal((4, 80)) + 1j * g.standard_normal((4, 80))
    k2e = 0.04 * np.where(g.random((80, 80)) > 0.5, 12.25, 1.0)
    isx = 1.0 / (1.0 - 0.3j * np.linspace(0, 1, 80) ** 3)
    isy = np.ones(80, complex)
    return r, gb, k2e, isx, isy


def test_zero_modulation_is_the_plain_fno():
    """With the fully connected layer at zero the modulation path leaves
    every block's R unchanged, whatever the convolution weights."""
    w = wl.nno_weights(4, modulation=True)
    w["mod_fc_w"][:] = 0.0
    w["mod_fc_b"][:] = 0.0
    plain = {k: v for k, v in w.items() if not k.startswith("mod_")}
    x, _ = nno.pack_inputs(*_window_inputs(5))
    assert np.max(np.abs(nno.forward(x, w) - nno.forward(x, plain))) == 0.0


def test_modulation_of_constant_auxiliary_inputs():
    """Constant auxiliary channels a_i: every convolution output is
    b_o + sum_i a_i sum_(dy,dx) k_{o,i,dy,dx}, so after leaky-ReLU and
    pooling each of the 144 features is that constant for its channel o, and
    the modulation is the fully connected layer applied to them."""
    w = wl.nno_weights(6, modulation=True)
    x = np.zeros((15, 80, 80))
    a = [0.3, -0.7, 0.2, 0.9, -0.1]
    for i, ch in enumerate(nno.MOD_AUX):
        x[ch] = a[i]
    cw, cb = w["mod_conv_w"].astype(float), w["mod_conv_b"].astype(float)
    per_o = [cb[o] + sum(a[i] * cw[o, i].sum() for i in range(5)) for o in range(16)]
    feat = np.repeat([v if v >= 0 else 0.01 * v for v in per_o], 9)  # [16 channels][3 x 3 cells]
    expect = w["mod_fc_w"].astype(float) @ feat + w["mod_fc_b"].astype(float)
    got = nno.modulation(x, w).ravel()
    assert np.allclose(got, expect, rtol=1e-12, atol=1e-14)


def test_modulation_is_a_strided_valid_convolution():
    """A single nonzero auxiliary pixel at (y, x) reaches only the conv
    outputs (Y, X) with 2Y <= y <= 2Y + 2, 2X <= x <= 2X + 2 (stride 2, no
    padding): moving it to another 13 x 13 pooling tile moves its effect on
    the pooled features to that tile (checked through a fully connected
    layer that reads one pooled feature)."""
    w = wl.nno_weights(7, modulation=True)
    w["mod_conv_b"][:] = 0.0
    w["mod_conv_w"][:] = 0.0
    w["mod_conv_w"][2, 0, 1, 1] = 1.0          # channel 2 copies aux channel 0 at offset (1, 1)
    w["mod_fc_b"][:] = 0.0
    w["mod_fc_w"][:] = 0.0
    w["mod_fc_w"][0, 2 * 9 + 1 * 3 + 2] = 1.0  # output 0 reads channel 2, pooled cell (1, 2)
    x = np.zeros((15, 80, 80))
    x[0, 2 * 20 + 1, 2 * 30 + 1] = 169.0       # conv output (20, 30): pooled cell (1, 2)
    assert np.isclose(nno.modulation(x, w).ravel()[0], 1.0)
    x[0] = 0.0
    x[0, 2 * 20 + 1, 2 * 5 + 1] = 169.0        # conv output (20, 5): pooled cell (1, 0)
    assert nno.modulation(x, w).ravel()[0] == 0.0


def test_full_rank_factorisation_is_the_plain_fno():
    """Rank 512 with V the identity over the retained modes: the expanded R
    is theta itself, so the network equals the plain FNO with R = theta."""
    w = wl.nno_weights(8, rank=512)
    eye = np.eye(512).reshape(512, 32, 16)
    w.update({f"R{b}_V_re": eye.astype(np.float32) for b in range(4)})
    w.update({f"R{b}_V_im": np.zeros((512, 32, 16), np.float32) for b in range(4)})
    plain = {k: v for k, v in w.items() if "theta" not in k and "_V_" not in k}
    for b in range(4):
        plain[f"R{b}_re"] = w[f"R{b}_theta_re"].reshape(32, 32, 32, 16)
        plain[f"R{b}_im"] = w[f"R{b}_theta_im"].reshape(32, 32, 32, 16)
    x, _ = nno.pack_inputs(*_window_inputs(9))
    assert np.max(np.abs(nno.forward(x, w) - nno.forward(x, plain))) < 1e-12


def test_modified_fno_solve_is_positively_homogeneous():
    """The modulation depends on the auxiliary inputs only: scaling the
    residual and Robin data by 3 scales the solve by 3."""
    w = wl.nno_weights(10, rank=8, modulation=True)
    r, gb, k2e, isx, isy = _window_inputs(11)
    e1 = nno.solve(r, gb, k2e, isx, isy, w)
    e3 = nno.solve(3 * r, 3 * gb, k2e, isx, isy, w)
    assert np.linalg.norm(e3 - 3 * e1) < 1e-10 * np.linalg.norm(e3)
