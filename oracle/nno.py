"""Subdomain Fourier neural operator (Sec. 2.1, Fig. 2), FP64 numpy.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The plain form of the paper's modified FNO (the modulation path and the
low-rank parameterisation of R are not part of this build):
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

Parity: the FFT convolution is pinned in tests/test_oracle_nno.py by a
brute-force DFT on the retained modes, by the projector property of the
mode truncation, and by the reduction to a pointwise map when R = 0.
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


def forward(x: np.ndarray, w: dict, blocks: int = 4) -> np.ndarray:
    """[15][80][80] -> [2][80][80] (Fig. 2)."""
    x = np.asarray(x, dtype=np.float64)
    h = pointwise(w["lift_w"].astype(np.float64), w["lift_b"].astype(np.float64), x)
    for b in range(blocks):
        R = w[f"R{b}_re"].astype(np.float64) + 1j * w[f"R{b}_im"].astype(np.float64)
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
