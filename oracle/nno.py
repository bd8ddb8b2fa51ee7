"""Subdomain Fourier neural operator (Sec. 2.1, Fig. 2), FP64 numpy.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper's modified FNO; without the optional parts below it is the plain
form:
    h0 = Lift x                                  (1x1, 15 -> 32)
    h_{b+1} = sigma( F^-1[ R_b . F[h_b] ] + W_b h_b + beta_b ),  b = 0..3
    out = P2 sigma(P1 h4 + p1) + p2              (32 -> 128 -> 2: Re, Im)
F is the 2D real FFT of the 80 x 80 window; R_b acts on the retained modes
ky in {0..15, -16..-1}, kx in {0..15} (the usual FNO corner blocks) as a
32 x 32 complex matrix per mode; all other modes are dropped; F^-1 is the
inverse real FFT onto 80 x 80.  sigma is leaky-ReLU (slope 0.01, Fig. 2
caption), not applied after the last Fourier block (the FNO convention;
the paper is silent).

Inputs (15 channels; readings of "eps, source and the four Robin edge
traces" plus the PML maps of Methods):
    0      (k0 dx)^2 eps
    1, 2   Re, Im of the window residual / rho
    3..10  Re, Im of the Robin data of sides x-, x+, y-, y+ divided by rho,
           broadcast along the side's normal
    11..14 Re, Im of 1/s_x (cell centres, broadcast along y) and of 1/s_y
rho^2 = (sum |r|^2 + sum |g|^2) / 6400 makes the solve 1-homogeneous:
e = rho * (out_re + j out_im), and e = 0 when rho = 0.

Modified FNO (Sec. 2.1, Fig. 2), both parts optional (readings: the paper
leaves the layer sizes to its supplement):
* modulation path: the five auxiliary channels (0 and 11..14, the
  permittivity and PML maps) of the window go through a 3 x 3 convolution
  with stride 2 and no padding (80 -> 39, 5 -> 16 channels), leaky-ReLU,
  average pooling over 13 x 13 tiles (39 -> 3) and a fully connected layer
  (144 -> 4 x 32 x 16) giving a real modulation tensor mod[b][ky][kx]; block
  b uses R*_b = R_b (1 + mod_b) element-wise (broadcast over the channel
  axes), i.e. it modulates the linearly transformed retained modes.  The
  residual form 1 + mod reduces to the plain FNO when the fully connected
  layer outputs zero.  mod depends on the auxiliary inputs only, not on the
  residual, so the solve stays 1-homogeneous;
* low-rank R: R_b[o][i][q] = sum_r theta_b[o][i][r] V_b[r][q] (q the 512
  retained modes): a linear layer V_b expands the rank-r tensor theta_b.

Parity: the FFT convolution is pinned in tests/test_oracle_nno.py by a
brute-force DFT on the retained modes, by the projector property of the
mode truncation, and by the reduction to a pointwise map when R = 0; the
modified FNO by its reduction to the plain one (zero modulation; rank 512
with V the identity), the closed-form modulation of constant auxiliary
inputs, and positive homogeneity with the modulation on.
"""
from __future__ import annotations

import numpy as np

WIN = 80
MY, MX = 32, 16
LEAK = 0.01


def leaky(x):
    return np.where(x >= 0, x, LEAK * x)


def retained_rows(n: int = WIN, my: int = MY):
    """Row (ky) indices of the retained modes: 0..my/2-1, then n-my/2..n-1."""
    h = my // 2
    return np.concatenate([np.arange(h), np.arange(n - h, n)])


def spectral_conv(h: np.ndarray, R: np.ndarray) -> np.ndarray:
    """F^-1[R . F[h]] for h [C][80][80] real, R [O][C][32][16] complex."""
    H = np.fft.rfft2(h, axes=(-2, -1))
    rows = retained_rows(h.shape[-2])
    Hk = H[:, rows, :MX]
    Y = np.einsum("oiyx,iyx->oyx", R, Hk)
    Yfull = np.zeros((R.shape[0], h.shape[-2], h.shape[-1] // 2 + 1), dtype=np.complex128)
    Yfull[:, rows, :MX] = Y
    return np.fft.irfft2(Yfull, s=h.shape[-2:], axes=(-2, -1))


def pointwise(Wm: np.ndarray, b: np.ndarray, h: np.ndarray) -> np.ndarray:
    return np.einsum("oi,iyx->oyx", Wm, h) + b[:, None, None]


MOD_AUX = (0, 11, 12, 13, 14)   # auxiliary input channels of the modulation path
MOD_CH = 16                     # convolution channels
MOD_OUT = 39                    # (80 - 3) / 2 + 1
MOD_POOL = 3                    # pooled grid (13 x 13 tiles)


def modulation(x: np.ndarray, w: dict, blocks: int = 4) -> np.ndarray:
    """mod[b][ky][kx] of one window from its auxiliary channels: 3 x 3
    convolution (stride 2, no padding), leaky-ReLU, 13 x 13 average pooling,
    fully connected layer."""
    a = np.asarray(x, dtype=np.float64)[list(MOD_AUX)]
    cw = w["mod_conv_w"].astype(np.float64)      # [16][5][3][3]
    cb = w["mod_conv_b"].astype(np.float64)      # [16]
    c = np.zeros((MOD_CH, MOD_OUT, MOD_OUT))
    for o in range(MOD_CH):
        acc = np.full((MOD_OUT, MOD_OUT), cb[o])
        for i in range(len(MOD_AUX)):
            for dy in range(3):
                for dx in range(3):
                    acc = acc + cw[o, i, dy, dx] * a[i, dy:dy + 2 * MOD_OUT - 1:2, dx:dx + 2 * MOD_OUT - 1:2]
        c[o] = acc
    t = MOD_OUT // MOD_POOL
    p = leaky(c).reshape(MOD_CH, MOD_POOL, t, MOD_POOL, t).mean(axis=(2, 4))
    m = w["mod_fc_w"].astype(np.float64) @ p.ravel() + w["mod_fc_b"].astype(np.float64)
    return m.reshape(blocks, MY, MX)


def spectral_weights(w: dict, b: int) -> np.ndarray:
    """R_b [32][32][32][16] complex: stored, or expanded from its rank-r
    factors theta_b [32][32][r] and V_b [r][32][16]."""
    if f"R{b}_theta_re" in w:
        th = w[f"R{b}_theta_re"].astype(np.float64) + 1j * w[f"R{b}_theta_im"].astype(np.float64)
        V = w[f"R{b}_V_re"].astype(np.float64) + 1j * w[f"R{b}_V_im"].astype(np.float64)
        return np.einsum("oir,ryx->oiyx", th, V)
    return w[f"R{b}_re"].astype(np.float64) + 1j * w[f"R{b}_im"].astype(np.float64)


def forward(x: np.ndarray, w: dict, blocks: int = 4) -> np.ndarray:
    """[15][80][80] -> [2][80][80] (Fig. 2)."""
    x = np.asarray(x, dtype=np.float64)
    mod = modulation(x, w, blocks) if "mod_fc_w" in w else None
    h = pointwise(w["lift_w"].astype(np.float64), w["lift_b"].astype(np.float64), x)
    for b in range(blocks):
        R = spectral_weights(w, b)
        if mod is not None:
            R = R * (1.0 + mod[b])[None, None]
        h = spectral_conv(h, R) + pointwise(w[f"W{b}"].astype(np.float64),
                                            w[f"b{b}"].astype(np.float64), h)
        if b < blocks - 1:
            h = leaky(h)
    q = leaky(pointwise(w["p1_w"].astype(np.float64), w["p1_b"].astype(np.float64), h))
    return pointwise(w["p2_w"].astype(np.float64), w["p2_b"].astype(np.float64), q)


def pack_inputs(r_w, g_w, k2eps_w, inv_sx_w, inv_sy_w):
    """Build the 15-channel input of one window and its scale rho.

    r_w [80][80] complex residual window, g_w [4][80] complex Robin data,
    k2eps_w [80][80] = (k0 dx)^2 eps, inv_sx_w [80] and inv_sy_w [80] the
    complex 1/s factors at the window's cell centres."""
    r_w = np.asarray(r_w, dtype=np.complex128)
    g_w = np.asarray(g_w, dtype=np.complex128)
    rho = np.sqrt((np.sum(np.abs(r_w) ** 2) + np.sum(np.abs(g_w) ** 2)) / (WIN * WIN))
    inv = 0.0 if rho == 0 else 1.0 / rho
    x = np.zeros((15, WIN, WIN))
    x[0] = k2eps_w
    x[1], x[2] = (r_w * inv).real, (r_w * inv).imag
    for s in range(4):
        gs = g_w[s] * inv
        if s < 2:   # x- / x+ sides: data varies along y, broadcast along x
            x[3 + 2 * s] = gs.real[:, None]
            x[4 + 2 * s] = gs.imag[:, None]
        else:       # y- / y+ sides: data varies along x, broadcast along y
            x[3 + 2 * s] = gs.real[None, :]
            x[4 + 2 * s] = gs.imag[None, :]
    x[11], x[12] = inv_sx_w.real[None, :], inv_sx_w.imag[None, :]
    x[13], x[14] = inv_sy_w.real[:, None], inv_sy_w.imag[:, None]
    return x, rho


def solve(r_w, g_w, k2eps_w, inv_sx_w, inv_sy_w, w: dict) -> np.ndarray:
    """Neural local solve: e = rho * NNO(inputs / rho) as an 80 x 80 complex field."""
    x, rho = pack_inputs(r_w, g_w, k2eps_w, inv_sx_w, inv_sy_w)
    if rho == 0:
        return np.zeros((WIN, WIN), dtype=np.complex128)
    out = forward(x, w)
    return rho * (out[0] + 1j * out[1])
