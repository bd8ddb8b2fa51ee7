"""Inverse-design parameterisation and optimiser (Sec. 2.2, inverse design:
density-based optimisation from a homogeneous grayscale start, differentiable
filtering and projection towards binary values, Adam ascent of the figure of
merit with adjoint gradients), FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper names the operations but prints no formulas; readings:
* design variable rho in [0, 1] on a rectangle of h x w cells;
* filter: cone of radius R cells, weights max(0, R - |d|) over the offsets d
  that stay inside the rectangle, each output divided by its own weight sum
  (so constants pass unchanged at the edges too): rho_f = W rho;
* projection: P(x) = (tanh(beta eta) + tanh(beta (x - eta))) /
  (tanh(beta eta) + tanh(beta (1 - eta))), P(0) = 0, P(1) = 1, and P -> x
  as beta -> 0;
* permittivity: eps = eps_lo + P(rho_f) (eps_hi - eps_lo) on the rectangle;
* the chain rule back to rho: g_rho = W^T (P'(rho_f) (eps_hi - eps_lo) g_eps);
* Adam (Kingma and Ba, 2015) with bias correction, ascending the figure of
  merit, rho clipped to [0, 1] after each step.

Parity: pinned in tests/test_oracle_design.py (constants pass the filter;
<W x, y> = <x, W^T y>; P(0) = 0, P(1) = 1, P -> identity as beta -> 0, P'
against central differences; the rho gradient against finite differences
of a linear functional of eps; Adam's first steps in closed form; one
design step raises the figure of merit of a small demultiplexer).
"""
from __future__ import annotations

import numpy as np


def cone_offsets(radius: float):
    """Offsets (dy, dx) with positive cone weight max(0, R - |d|)."""
    r = int(np.ceil(radius))
    out = []
    for dy in range(-r, r + 1):
        for dx in range(-r, r + 1):
            wgt = radius - np.hypot(dy, dx)
            if wgt > 0:
                out.append((dy, dx, wgt))
    return out


def filter_fwd(rho: np.ndarray, radius: float):
    """rho_f = W rho and the weight sums S (both h x w)."""
    h, w = rho.shape
    num = np.zeros((h, w))
    S = np.zeros((h, w))
    for (dy, dx, wgt) in cone_offsets(radius):
        for i in range(h):
            j0, j1 = max(0, -dx), min(w, w - dx)
            if not 0 <= i + dy < h or j0 >= j1:
                continue
            num[i, j0:j1] += wgt * rho[i + dy, j0 + dx:j1 + dx]
            S[i, j0:j1] += wgt
    return num / S, S


def filter_adj(t: np.ndarray, radius: float) -> np.ndarray:
    """W^T t: cell j collects w_ij t_i / S_i from every output i it feeds."""
    h, w = t.shape
    _, S = filter_fwd(np.zeros((h, w)), radius)
    q = t / S
    out = np.zeros((h, w))
    for (dy, dx, wgt) in cone_offsets(radius):
        # output i = j - d reads input j at offset d
        for j in range(h):
            i = j - dy
            if not 0 <= i < h:
                continue
            c0, c1 = max(0, dx), min(w, w + dx)
            if c0 >= c1:
                continue
            out[j, c0:c1] += wgt * q[i, c0 - dx:c1 - dx]
    return out


def project(x: np.ndarray, beta: float, eta: float) -> np.ndarray:
    a, b = np.tanh(beta * eta), np.tanh(beta * (1.0 - eta))
    return (a + np.tanh(beta * (x - eta))) / (a + b)


def project_grad(x: np.ndarray, beta: float, eta: float) -> np.ndarray:
    a, b = np.tanh(beta * eta), np.tanh(beta * (1.0 - eta))
    return beta * (1.0 - np.tanh(beta * (x - eta)) ** 2) / (a + b)


def density_to_eps(rho, radius, beta, eta, eps_lo, eps_hi):
    """Permittivity of the design rectangle, and the filtered density."""
    rf, _ = filter_fwd(rho, radius)
    return eps_lo + project(rf, beta, eta) * (eps_hi - eps_lo), rf


def eps_grad_to_rho(g_eps, rho, radius, beta, eta, eps_lo, eps_hi):
    """dF/drho from dF/deps on the design rectangle (chain rule above)."""
    rf, _ = filter_fwd(rho, radius)
    return filter_adj(project_grad(rf, beta, eta) * (eps_hi - eps_lo) * g_eps, radius)


class Adam:
    """Adam ascent with bias correction; the variable is clipped to [0, 1]."""

    def __init__(self, shape, lr=0.01, b1=0.9, b2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps
        self.m = np.zeros(shape)
        self.v = np.zeros(shape)
        self.t = 0

    def step(self, theta: np.ndarray, g: np.ndarray) -> np.ndarray:
        self.t += 1
        self.m = self.b1 * self.m + (1.0 - self.b1) * g
        self.v = self.b2 * self.v + (1.0 - self.b2) * g * g
        mh = self.m / (1.0 - self.b1 ** self.t)
        vh = self.v / (1.0 - self.b2 ** self.t)
        return np.clip(theta + self.lr * mh / (np.sqrt(vh) + self.eps), 0.0, 1.0)
