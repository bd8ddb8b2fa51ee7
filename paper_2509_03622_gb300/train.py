"""Offline training of the subdomain neural operator (Sec. 2.1; Methods,
Algorithm 2 and the physics-only data recipe).

This is the one piece of the project that runs in PyTorch: it produces the
weight blob that `schwarz_setup` consumes (layout of include/fdfd.h).  The
solve itself never calls it.

Model: the plain FNO of Fig. 2 (lift 15 -> 32, four Fourier blocks with 512
retained modes and 1x1 channel mixers, leaky-ReLU, projection 32 -> 128 ->
2).  Physics-only loss (Methods: random permittivity, Gaussian-noise sources
and Robin data, random PML placement, no ground truth): the network output
e for residual r and Robin data g must satisfy the local Robin problem
A_w e = r - B g (Eq. 1-2 on an 80 x 80 window).  Fixed-point recurrence of
Algorithm 2: x += M(r), r = rhs - A_w x with the gradient stopped through r,
loss = ||r||^2 / ||rhs||^2 after every step (clipped for stability).
"""
from __future__ import annotations

import argparse
import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

WIN = 80


def build_model(torch, w0: dict):
    nn = torch.nn

    class FNO(nn.Module):
        def __init__(self):
            super().__init__()
            P = lambda a: nn.Parameter(torch.tensor(np.asarray(a, dtype=np.float32)))
            self.lift_w, self.lift_b = P(w0["lift_w"]), P(w0["lift_b"])
            self.rank = int(w0["R0_theta_re"].shape[2]) if "R0_theta_re" in w0 else 0
            if self.rank:  # modified FNO: R_b = theta_b V_b (Sec. 2.1)
                self.Tr = nn.ParameterList([P(w0[f"R{b}_theta_re"]) for b in range(4)])
                self.Ti = nn.ParameterList([P(w0[f"R{b}_theta_im"]) for b in range(4)])
                self.Vr = nn.ParameterList([P(w0[f"R{b}_V_re"]) for b in range(4)])
                self.Vi = nn.ParameterList([P(w0[f"R{b}_V_im"]) for b in range(4)])
            else:
                self.Rr = nn.ParameterList([P(w0[f"R{b}_re"]) for b in range(4)])
                self.Ri = nn.ParameterList([P(w0[f"R{b}_im"]) for b in range(4)])
            self.mod = "mod_fc_w" in w0
            if self.mod:  # modulation path (Sec. 2.1, Fig. 2)
                self.mcw, self.mcb = P(w0["mod_conv_w"]), P(w0["mod_conv_b"])
                self.mfw, self.mfb = P(w0["mod_fc_w"]), P(w0["mod_fc_b"])
            self.W = nn.ParameterList([P(w0[f"W{b}"]) for b in range(4)])
            self.bb = nn.ParameterList([P(w0[f"b{b}"]) for b in range(4)])
            self.p1_w, self.p1_b = P(w0["p1_w"]), P(w0["p1_b"])
            self.p2_w, self.p2_b = P(w0["p2_w"]), P(w0["p2_b"])

        def spectral(self, b):
            if self.rank:
                return torch.einsum("oir,ryx->oiyx", torch.complex(self.Tr[b], self.Ti[b]),
                                    torch.complex(self.Vr[b], self.Vi[b]))
            return torch.complex(self.Rr[b], self.Ri[b])

        def modulation(self, x):  # [B][4][32][16]
            F_ = torch.nn.functional
            a = x[:, [0, 11, 12, 13, 14]]
            c = F_.leaky_relu(F_.conv2d(a, self.mcw, self.mcb, stride=2), 0.01)
            f = F_.avg_pool2d(c, 13).flatten(1)
            return (f @ self.mfw.t() + self.mfb).reshape(-1, 4, 32, 16)

        def forward(self, x):  # [B][15][80][80] -> [B][2][80][80]
            m = self.modulation(x) if self.mod else None
            h = torch.einsum("oi,biyx->boyx", self.lift_w, x) + self.lift_b[None, :, None, None]
            for b in range(4):
                H = torch.fft.rfft2(h)
                Hk = torch.cat([H[:, :, :16, :16], H[:, :, -16:, :16]], dim=2)
                if m is not None:  # R (1 + mod) on every channel pair = scaling the retained modes
                    Hk = Hk * (1.0 + m[:, b])[:, None]
                R = self.spectral(b)
                Y = torch.einsum("biyx,oiyx->boyx", Hk, R)
                Yf = torch.zeros(h.shape[0], 32, WIN, WIN // 2 + 1, dtype=Y.dtype, device=h.device)
                Yf[:, :, :16, :16] = Y[:, :, :16]
                Yf[:, :, -16:, :16] = Y[:, :, 16:]
                s = torch.fft.irfft2(Yf, s=(WIN, WIN))
                h = s + torch.einsum("oi,biyx->boyx", self.W[b], h) + self.bb[b][None, :, None, None]
                if b < 3:
                    h = torch.nn.functional.leaky_relu(h, 0.01)
            q = torch.nn.functional.leaky_relu(
                torch.einsum("oi,biyx->boyx", self.p1_w, h) + self.p1_b[None, :, None, None], 0.01)
            return torch.einsum("oi,biyx->boyx", self.p2_w, q) + self.p2_b[None, :, None, None]

        def export(self) -> dict:
            d = {"lift_w": self.lift_w, "lift_b": self.lift_b, "p1_w": self.p1_w, "p1_b": self.p1_b,
                 "p2_w": self.p2_w, "p2_b": self.p2_b}
            for b in range(4):
                if self.rank:
                    d[f"R{b}_theta_re"], d[f"R{b}_theta_im"] = self.Tr[b], self.Ti[b]
                    d[f"R{b}_V_re"], d[f"R{b}_V_im"] = self.Vr[b], self.Vi[b]
                else:
                    d[f"R{b}_re"], d[f"R{b}_im"] = self.Rr[b], self.Ri[b]
                d[f"W{b}"], d[f"b{b}"] = self.W[b], self.bb[b]
            if self.mod:
                d.update(mod_conv_w=self.mcw, mod_conv_b=self.mcb, mod_fc_w=self.mfw, mod_fc_b=self.mfb)
            return {k: v.detach().float().cpu().numpy() for k, v in d.items()}

    return FNO()


class Sampler:
    """Random 80 x 80 Robin windows (Methods: physics-only data)."""

    def __init__(self, torch, dev, batch, npml=20):
        self.t, self.dev, self.B, self.npml = torch, dev, batch, npml

    def smooth_noise(self, shape, sigma):
        t = self.t
        z = t.randn(*shape, dtype=t.complex64, device=self.dev)
        n = shape[-1]
        f = t.fft.fftfreq(n, device=self.dev)
        g = t.exp(-2 * (math.pi * f[:, None]) ** 2 * sigma[:, None, None] ** 2 - 2 * (math.pi * f[None, :]) ** 2
                  * sigma[:, None, None] ** 2) if len(shape) == 3 else None
        return t.fft.ifft2(t.fft.fft2(z) * g)

    def eps(self):
        t, B = self.t, self.B
        e = t.ones(B, WIN, WIN, device=self.dev)
        vals = t.tensor([1.0, 2.1, 12.25], device=self.dev)
        kind = t.randint(0, 3, (B,), device=self.dev)
        # rectangles
        for _ in range(6):
            w = t.randint(8, 48, (B,), device=self.dev)
            h = t.randint(8, 48, (B,), device=self.dev)
            x0 = t.randint(-20, WIN, (B,), device=self.dev)
            y0 = t.randint(-20, WIN, (B,), device=self.dev)
            v = vals[t.randint(0, 3, (B,), device=self.dev)]
            xs = t.arange(WIN, device=self.dev)
            mx = (xs[None, :] >= x0[:, None]) & (xs[None, :] < (x0 + w)[:, None])
            my = (xs[None, :] >= y0[:, None]) & (xs[None, :] < (y0 + h)[:, None])
            m = my[:, :, None] & mx[:, None, :] & (kind == 0)[:, None, None]
            e = t.where(m, v[:, None, None], e)
        # freeform: thresholded smooth noise
        sig = 2.0 + 4.0 * t.rand(B, device=self.dev)
        s = self.smooth_noise((B, WIN, WIN), sig).real
        hi = vals[1 + t.randint(0, 2, (B,), device=self.dev)]
        e = t.where((kind == 1)[:, None, None], t.where(s > 0, hi[:, None, None], t.ones_like(e)), e)
        # kind 2: homogeneous background of random value
        e = t.where((kind == 2)[:, None, None], vals[t.randint(0, 3, (B,), device=self.dev)][:, None, None]
                    * t.ones_like(e), e)
        return e

    def axis(self, k0dx):
        """Per-window 1D UPML factors and side kinds for one axis.
        mode 0: interior (both sides Robin), 1: grid edge at the low side
        (PML cells 0..npml-1, low side Dirichlet), 2: edge at the high side."""
        t, B, npml = self.t, self.B, self.npml
        # 60% interior (draws 0-2), 20% each grid edge (3 -> low side, 4 -> high
        # side): most windows of a large grid have no PML at all
        u = t.randint(0, 5, (B,), device=self.dev)
        mode = t.where(u < 3, t.zeros_like(u), u - 2)
        pn = t.arange(WIN, device=self.dev, dtype=t.float32) + 0.5
        ph = t.arange(WIN + 1, device=self.dev, dtype=t.float32)
        A = (4.0 * 30.0 / (2.0 * npml * k0dx))[:, None]  # -(m+1) lnR / (2 npml k0dx)

        def sig(p):
            dlo = (npml - p[None, :]).clamp(min=0) / npml
            dhi = (p[None, :] - (WIN - npml)).clamp(min=0) / npml
            lo = (mode == 1)[:, None].float() * dlo ** 3
            hi = (mode == 2)[:, None].float() * dhi ** 3
            return A * (lo + hi)

        sn = t.complex(t.ones(B, WIN, device=self.dev), -sig(pn))
        sh = t.complex(t.ones(B, WIN + 1, device=self.dev), -sig(ph))
        lo = 1.0 / (sn * sh[:, :-1])
        hi = 1.0 / (sn * sh[:, 1:])
        robin_lo = mode != 1
        robin_hi = mode != 2
        return sn, lo, hi, robin_lo, robin_hi

    def batch(self):
        t, B = self.t, self.B
        ppw = 20.0 + 20.0 * t.rand(B, device=self.dev)
        k0dx = 2 * math.pi / ppw
        eps = self.eps()
        sxn, xlo, xhi, rxl, rxh = self.axis(k0dx)
        syn, ylo, yhi, ryl, ryh = self.axis(k0dx)
        return dict(k0dx=k0dx, eps=eps, sxn=sxn, xlo=xlo, xhi=xhi, syn=syn, ylo=ylo, yhi=yhi,
                    robin=t.stack([rxl, rxh, ryl, ryh], 1))


def local_apply(t, e, P):
    """A_w e: 5-point UPML stencil with the Robin ghost elimination of Eq. 2
    on interface sides (u_o = (1 - j kd) u_b + g) and zero ghosts on grid
    sides.  e [B][80][80] complex."""
    xlo, xhi, ylo, yhi = P["xlo"], P["xhi"], P["ylo"], P["yhi"]
    k2 = (P["k0dx"] ** 2)[:, None, None]
    kd = P["k0dx"][:, None, None] * t.sqrt(P["eps"])
    z = t.zeros_like(e[:, :, :1])
    em = t.cat([z, e[:, :, :-1]], 2)
    ep = t.cat([e[:, :, 1:], z], 2)
    zr = t.zeros_like(e[:, :1, :])
    eym = t.cat([zr, e[:, :-1, :]], 1)
    eyp = t.cat([e[:, 1:, :], zr], 1)
    y = xlo[:, None, :] * em + xhi[:, None, :] * ep + ylo[:, :, None] * eym + yhi[:, :, None] * eyp
    dg = -(xlo + xhi)[:, None, :] - (ylo + yhi)[:, :, None] + k2 * P["eps"]
    y = y + dg * e
    rb = P["robin"]
    f = (1 - 1j * kd)
    add = t.zeros_like(e)
    add[:, :, 0] += rb[:, 0, None] * xlo[:, None, 0] * f[:, :, 0] * e[:, :, 0]
    add[:, :, -1] += rb[:, 1, None] * xhi[:, None, -1] * f[:, :, -1] * e[:, :, -1]
    add[:, 0, :] += rb[:, 2, None] * ylo[:, 0, None] * f[:, 0, :] * e[:, 0, :]
    add[:, -1, :] += rb[:, 3, None] * yhi[:, -1, None] * f[:, -1, :] * e[:, -1, :]
    return y + add


def boundary_rhs(t, g, P):
    """B g: contribution -c_bo g of the Robin data to the right-hand side."""
    out = t.zeros(g.shape[0], WIN, WIN, dtype=g.dtype, device=g.device)
    rb = P["robin"]
    out[:, :, 0] -= rb[:, 0, None] * P["xlo"][:, None, 0] * g[:, 0]
    out[:, :, -1] -= rb[:, 1, None] * P["xhi"][:, None, -1] * g[:, 1]
    out[:, 0, :] -= rb[:, 2, None] * P["ylo"][:, 0, None] * g[:, 2]
    out[:, -1, :] -= rb[:, 3, None] * P["yhi"][:, -1, None] * g[:, 3]
    return out


def dense_operator(t, P):
    """Dense A_w [B][6400][6400] of the local Robin problems (same stencil as
    local_apply), for exact training targets."""
    B = P["eps"].shape[0]
    n = WIN * WIN
    dev = P["eps"].device
    A = t.zeros(B, n, n, dtype=t.complex64, device=dev)
    idx = t.arange(n, device=dev)
    lx, ly = idx % WIN, idx // WIN
    xlo, xhi, ylo, yhi = P["xlo"], P["xhi"], P["ylo"], P["yhi"]
    k2 = (P["k0dx"] ** 2)[:, None]
    epsf = P["eps"].reshape(B, n)
    kd = P["k0dx"][:, None] * t.sqrt(epsf)
    f = 1 - 1j * kd
    dg = -(xlo + xhi)[:, lx] - (ylo + yhi)[:, ly] + k2 * epsf
    rb = P["robin"]
    dg = dg + t.where((lx == 0)[None] & rb[:, 0:1], xlo[:, lx] * f, t.zeros_like(dg))
    dg = dg + t.where((lx == WIN - 1)[None] & rb[:, 1:2], xhi[:, lx] * f, t.zeros_like(dg))
    dg = dg + t.where((ly == 0)[None] & rb[:, 2:3], ylo[:, ly] * f, t.zeros_like(dg))
    dg = dg + t.where((ly == WIN - 1)[None] & rb[:, 3:4], yhi[:, ly] * f, t.zeros_like(dg))
    A[:, idx, idx] = dg
    m = lx > 0
    A[:, idx[m], idx[m] - 1] = xlo[:, lx[m]]
    m = lx < WIN - 1
    A[:, idx[m], idx[m] + 1] = xhi[:, lx[m]]
    m = ly > 0
    A[:, idx[m], idx[m] - WIN] = ylo[:, ly[m]]
    m = ly < WIN - 1
    A[:, idx[m], idx[m] + WIN] = yhi[:, ly[m]]
    return A


def initial_weights(init, seed, rank=0, modulation=False):
    """Starting weights: a saved blob (plain, or of the requested layout) or
    the seeded initialisation.  From a plain blob the modified parts start
    where they change nothing or little: the modulation's fully connected
    layer at zero (the network is then the plain one) and each R split into
    rank-r factors by a truncated SVD along the mode axis."""
    from paper_2509_03622_gb300 import workloads as wl
    if not init:
        return wl.nno_weights(seed, rank=rank, modulation=modulation)
    blob = np.load(init)
    plain_n = wl.pack_weights(wl.nno_weights(0)).size
    if blob.size != plain_n:
        return wl.unpack_weights(blob, rank=rank, modulation=modulation)
    w = wl.unpack_weights(blob)
    if rank:
        for b in range(4):
            R = (w.pop(f"R{b}_re") + 1j * w.pop(f"R{b}_im")).astype(np.complex128).reshape(32 * 32, 512)
            U, sv, Vh = np.linalg.svd(R, full_matrices=False)
            th = (U[:, :rank] * sv[:rank]).reshape(32, 32, rank)
            V = Vh[:rank].reshape(rank, 32, 16)
            w[f"R{b}_theta_re"], w[f"R{b}_theta_im"] = th.real.astype(np.float32), th.imag.astype(np.float32)
            w[f"R{b}_V_re"], w[f"R{b}_V_im"] = V.real.astype(np.float32), V.imag.astype(np.float32)
    if modulation:
        m = wl.nno_weights(seed, modulation=True)
        for k in ("mod_conv_w", "mod_conv_b"):
            w[k] = m[k]
        w["mod_fc_w"] = np.zeros_like(m["mod_fc_w"])
        w["mod_fc_b"] = np.zeros_like(m["mod_fc_b"])
    return w


def row_blocks(t, P):
    """The local Robin operator A_w ordered by window rows: diagonal blocks
    D_y [B][80][80] (tridiagonal in x, Robin eliminations on interface
    sides) and the scalar couplings ylo[y], yhi[y] to the rows below and
    above (the same stencil as local_apply)."""
    B = P["eps"].shape[0]
    dev = P["eps"].device
    xlo, xhi, ylo, yhi = P["xlo"], P["xhi"], P["ylo"], P["yhi"]
    k2 = (P["k0dx"] ** 2)[:, None, None]
    kd = P["k0dx"][:, None, None] * t.sqrt(P["eps"])
    f = 1 - 1j * kd                                        # [B][y][x]
    rb = P["robin"]
    dg = -(xlo + xhi)[:, None, :] - (ylo + yhi)[:, :, None] + k2 * P["eps"]
    dg = dg.to(t.complex64)
    dg[:, :, 0] += rb[:, 0, None] * xlo[:, None, 0] * f[:, :, 0]
    dg[:, :, -1] += rb[:, 1, None] * xhi[:, None, -1] * f[:, :, -1]
    dg[:, 0, :] += rb[:, 2, None] * ylo[:, 0, None] * f[:, 0, :]
    dg[:, -1, :] += rb[:, 3, None] * yhi[:, -1, None] * f[:, -1, :]
    D = t.zeros(B, WIN, WIN, WIN, dtype=t.complex64, device=dev)  # [B][y][x][x']
    i = t.arange(WIN, device=dev)
    D[:, :, i, i] = dg
    D[:, :, i[1:], i[1:] - 1] = xlo[:, None, 1:].expand(B, WIN, WIN - 1)
    D[:, :, i[:-1], i[:-1] + 1] = xhi[:, None, :-1].expand(B, WIN, WIN - 1)
    return D, ylo, yhi


def exact_local_solve(t, P, rhs):
    """Exact solutions of the local Robin problems A_w x = rhs ([B][80][80],
    several right-hand sides per window allowed as rhs [B][R][80][80]) by
    block elimination over the 80 window rows: S_0 = D_0,
    S_y = D_y - ylo_y yhi_{y-1} S_{y-1}^-1 (the row couplings are scalar),
    then the forward and backward sweeps.  About 80 batched 80 x 80 inverses
    per window instead of a dense 6400 x 6400 factorisation."""
    D, ylo, yhi = row_blocks(t, P)
    # FP64 throughout: the row recursion amplifies rounding (and on GPUs
    # with TF32 matmuls enabled a complex64 einsum would lose bits)
    D, ylo, yhi = D.to(t.complex128), ylo.to(t.complex128), yhi.to(t.complex128)
    multi = rhs.dim() == 4
    b = (rhs if multi else rhs[:, None]).to(t.complex128)  # [B][R][y][x]
    Sinv = []
    prev = None
    for y in range(WIN):
        S = D[:, y]
        if prev is not None:
            S = S - (ylo[:, y] * yhi[:, y - 1])[:, None, None] * prev
        prev = t.linalg.inv(S)
        Sinv.append(prev)
    z = []
    zy = None
    for y in range(WIN):
        r = b[:, :, y, :]
        if zy is not None:
            r = r - ylo[:, y, None, None] * zy
        zy = t.einsum("bij,brj->bri", Sinv[y], r)
        z.append(zy)
    x = [None] * WIN
    x[WIN - 1] = z[WIN - 1]
    for y in range(WIN - 2, -1, -1):
        x[y] = z[y] - t.einsum("bij,brj->bri", Sinv[y], yhi[:, y, None, None] * x[y + 1])
    out = t.stack(x, 2).to(t.complex64)
    return out if multi else out[:, 0]


def plane_wave_data(t, P):
    """Robin data of a plane wave of random direction on every side,
    exp(-j kd (d . r)) at the side cells, kd from the mean permittivity of
    the window's boundary (the kind of data the coarse space's trials are)."""
    B = P["eps"].shape[0]
    dev = P["eps"].device
    th = 2 * math.pi * t.rand(B, device=dev)
    e = P["eps"]
    eb = t.cat([e[:, :, 0], e[:, :, -1], e[:, 0, :], e[:, -1, :]], 1).mean(1)
    kd = P["k0dx"] * t.sqrt(eb)
    s = t.arange(WIN, device=dev, dtype=t.float32)
    z, h = t.zeros_like(s), t.full_like(s, WIN - 1.0)
    xs = t.stack([z, h, s, s])                       # side cell coordinates [4][80]
    ys = t.stack([s, s, z, h])
    ph = kd[:, None, None] * (t.cos(th)[:, None, None] * xs + t.sin(th)[:, None, None] * ys)
    return t.polar(t.ones_like(ph), -ph)


def expand(P, reps):
    """Repeat each window's parameters `reps` times (several right-hand sides per window)."""
    return {k: v.repeat_interleave(reps, 0) for k, v in P.items()}


def train_data(minutes, windows, rhs_per_win, lr, seed, out, log_every, device, init, c_res=0.3, rank=0,
               modulation=False):
    """Supervised training on exact local solutions (block elimination over
    the window rows, several right-hand sides per window) plus the residual
    loss; second step trained on the residual of the first (Algorithm 2)."""
    import torch as t
    from paper_2509_03622_gb300 import workloads as wl
    dev = t.device(device)
    t.manual_seed(seed)
    t.backends.cuda.matmul.allow_tf32 = True
    w0 = initial_weights(init, seed, rank, modulation)
    model = build_model(t, w0).to(dev)
    opt = t.optim.Adam(model.parameters(), lr=lr)
    S = Sampler(t, dev, windows)
    val = validation_set(t, dev)
    print("validation before:", evaluate(t, model, val), flush=True)
    t0, it, hist = time.time(), 0, []
    R = rhs_per_win
    while time.time() - t0 < minutes * 60:
        frac = (time.time() - t0) / (minutes * 60)
        for gp in opt.param_groups:
            gp["lr"] = lr * 0.5 * (1 + math.cos(math.pi * min(frac, 1.0)))
        P = S.batch()
        Pe = expand(P, R)
        Bt = windows * R
        sig = t.rand(Bt, device=dev) * 6.0
        r = S.smooth_noise((Bt, WIN, WIN), sig) if hasattr(S, "smooth_noise") else None
        g = t.randn(Bt, 4, WIN, dtype=t.complex64, device=dev)
        g = t.where((t.rand(Bt, device=dev) < 0.5)[:, None, None], plane_wave_data(t, Pe), g)
        kindr = t.rand(Bt, device=dev)
        r = t.where((kindr < 0.25)[:, None, None], t.zeros_like(r), r)
        g = t.where((kindr > 0.5)[:, None, None], t.zeros_like(g), g)
        g = g * Pe["robin"][:, :, None]
        rhs = r + boundary_rhs(t, g, Pe)
        with t.no_grad():
            xs = exact_local_solve(t, P, rhs.reshape(windows, R, WIN, WIN)).reshape(Bt, WIN, WIN)
            # keep only samples the elimination solved accurately
            rr = (rhs - local_apply(t, xs, Pe)).abs().pow(2).sum((1, 2)) / \
                (rhs.abs() ** 2).sum((1, 2)).clamp(min=1e-30)
            good = (rr < 1e-6).float()
        nx_ = (xs.abs() ** 2).sum((1, 2)).clamp(min=1e-30)
        nr_ = (rhs.abs() ** 2).sum((1, 2)).clamp(min=1e-30)
        opt.zero_grad()
        e1 = solve(t, model, r, g, Pe)
        l1 = ((e1 - xs).abs() ** 2).sum((1, 2)) / nx_
        res1 = rhs - local_apply(t, e1, Pe)
        p1 = (res1.abs() ** 2).sum((1, 2)) / nr_
        res1d = res1.detach()
        e2 = solve(t, model, res1d, t.zeros_like(g), Pe)
        tgt2 = (xs - e1.detach())
        l2 = ((e2 - tgt2).abs() ** 2).sum((1, 2)) / (tgt2.abs() ** 2).sum((1, 2)).clamp(min=1e-30)
        # relative L2 errors (not squared, not clamped): bounded gradients
        # without switching off the samples a drifting network gets worst
        ng = good.sum().clamp(min=1.0)
        loss = ((good * l1.sqrt()).sum() + (good * l2.sqrt()).sum() + c_res * (good * p1.sqrt()).sum()) / ng / (2 + c_res)
        loss.backward()
        t.nn.utils.clip_grad_norm_(model.parameters(), 1.0)
        opt.step()
        it += 1
        hist.append((float(l1.detach().sqrt().mean()), float(l2.detach().sqrt().mean()),
                     float(p1.detach().sqrt().mean()), float(good.mean())))
        if it % log_every == 0:
            h = np.mean(hist[-log_every:], axis=0)
            print(f"it {it} t {time.time() - t0:.0f}s field-err1 {h[0]:.4f} field-err2 {h[1]:.4f} "
                  f"resid1 {h[2]:.4f} accepted {h[3]:.3f}", flush=True)
    np.save(out, wl.pack_weights(model.export()))
    print(f"saved {out} after {it} iterations")
    print("validation after:", evaluate(t, model, val), flush=True)


def validation_set(t, dev, windows=64, seed=12345):
    """A fixed batch of windows, residual-only right-hand sides and their
    exact solutions (same sampler as training, seeded)."""
    g = t.Generator(device=dev)
    state = t.random.get_rng_state() if dev.type == "cpu" else t.cuda.get_rng_state(dev)
    t.manual_seed(seed)
    S = Sampler(t, dev, windows)
    P = S.batch()
    sig = t.rand(windows, device=dev) * 6.0
    r = S.smooth_noise((windows, WIN, WIN), sig)
    with t.no_grad():
        xs = exact_local_solve(t, P, r)
    if dev.type == "cpu":
        t.random.set_rng_state(state)
    else:
        t.cuda.set_rng_state(state, dev)
    del g
    return P, r, xs


def evaluate(t, model, val):
    """Mean relative field error and local residual of one network
    application, and the residual after a second application to the first
    one's residual (fixed-point recurrence of Algorithm 2)."""
    P, r, xs = val
    with t.no_grad():
        zg = t.zeros(r.shape[0], 4, WIN, dtype=t.complex64, device=r.device)
        e1 = solve(t, model, r, zg, P)
        res1 = r - local_apply(t, e1, P)
        e2 = e1 + solve(t, model, res1, zg, P)
        res2 = r - local_apply(t, e2, P)
        nr = (r.abs() ** 2).sum((1, 2)).sqrt()
        ferr = ((e1 - xs).abs() ** 2).sum((1, 2)).sqrt() / (xs.abs() ** 2).sum((1, 2)).sqrt()
        return {"field_err": float(ferr.mean()), "resid1": float(((res1.abs() ** 2).sum((1, 2)).sqrt() / nr).mean()),
                "resid2": float(((res2.abs() ** 2).sum((1, 2)).sqrt() / nr).mean())}


def pack(t, r, g, P):
    rho = t.sqrt((r.abs() ** 2).sum((1, 2)) + (g.abs() ** 2).sum((1, 2))) / WIN
    inv = t.where(rho > 0, 1.0 / rho, t.zeros_like(rho))
    rn = r * inv[:, None, None]
    gn = g * inv[:, None, None]
    B = r.shape[0]
    x = t.zeros(B, 15, WIN, WIN, device=r.device)
    x[:, 0] = (P["k0dx"] ** 2)[:, None, None] * P["eps"]
    x[:, 1], x[:, 2] = rn.real, rn.imag
    for s in range(4):
        gs = gn[:, s]
        if s < 2:
            x[:, 3 + 2 * s] = gs.real[:, :, None].expand(B, WIN, WIN)
            x[:, 4 + 2 * s] = gs.imag[:, :, None].expand(B, WIN, WIN)
        else:
            x[:, 3 + 2 * s] = gs.real[:, None, :].expand(B, WIN, WIN)
            x[:, 4 + 2 * s] = gs.imag[:, None, :].expand(B, WIN, WIN)
    isx, isy = 1.0 / P["sxn"], 1.0 / P["syn"]
    x[:, 11], x[:, 12] = isx.real[:, None, :], isx.imag[:, None, :]
    x[:, 13], x[:, 14] = isy.real[:, :, None], isy.imag[:, :, None]
    return x, rho


def solve(t, model, r, g, P):
    x, rho = pack(t, r, g, P)
    out = model(x)
    return rho[:, None, None] * t.complex(out[:, 0], out[:, 1])


def train(minutes: float, batch: int, recur: int, lr: float, seed: int, out: str, log_every: int = 200,
          device: str = "cuda", init=None):
    import torch as t
    from paper_2509_03622_gb300 import workloads as wl
    dev = t.device(device)
    t.manual_seed(seed)
    t.backends.cuda.matmul.allow_tf32 = True
    w0 = wl.unpack_weights(np.load(init)) if init else wl.nno_weights(seed)
    model = build_model(t, w0).to(dev)
    opt = t.optim.Adam(model.parameters(), lr=lr)
    S = Sampler(t, dev, batch)
    t0 = time.time()
    it = 0
    hist = []
    while time.time() - t0 < minutes * 60:
        frac = (time.time() - t0) / (minutes * 60)
        for gp in opt.param_groups:
            gp["lr"] = lr * 0.5 * (1 + math.cos(math.pi * min(frac, 1.0)))
        P = S.batch()
        sig = t.rand(batch, device=dev) * 6.0
        r = S.smooth_noise((batch, WIN, WIN), sig)
        g = t.randn(batch, 4, WIN, dtype=t.complex64, device=dev)
        kindr = t.rand(batch, device=dev)
        r = t.where((kindr < 0.25)[:, None, None], t.zeros_like(r), r)           # boundary-data-only solves
        g = t.where((kindr > 0.5)[:, None, None], t.zeros_like(g), g)            # residual-only solves
        g = g * P["robin"][:, :, None]
        rhs = r + boundary_rhs(t, g, P)
        nrm = (rhs.abs() ** 2).sum((1, 2)).clamp(min=1e-30)
        x = t.zeros_like(rhs)
        res = rhs
        loss = 0.0
        opt.zero_grad()
        zg = t.zeros_like(g)
        for k in range(recur):
            # first step sees the source and the Robin data, later steps the residual only
            e = solve(t, model, r, g, P) if k == 0 else solve(t, model, res, zg, P)
            x = x + e
            res_new = rhs - local_apply(t, x, P)
            lk = ((res_new.abs() ** 2).sum((1, 2)) / nrm).clamp(max=4.0)
            loss = loss + lk.mean()
            res = res_new.detach()
            x = x.detach()
        loss = loss / recur
        loss.backward()
        t.nn.utils.clip_grad_norm_(model.parameters(), 1.0)
        opt.step()
        it += 1
        hist.append(float(loss))
        if it % log_every == 0:
            print(f"it {it} t {time.time() - t0:.0f}s loss {np.mean(hist[-log_every:]):.4f}", flush=True)
    w = model.export()
    np.save(out, wl.pack_weights(w))
    print(f"saved {out} after {it} iterations; final loss {np.mean(hist[-200:]):.4f}")
    return hist


if __name__ == "__main__":
    ap = argparse.ArgumentParser()
    ap.add_argument("--minutes", type=float, default=10.0)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--recur", type=int, default=3)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--out", default=os.path.join(HERE, "weights", "nno_trained.npy"))
    ap.add_argument("--device", default="cuda")
    ap.add_argument("--init", default=None, help="start from a saved weight blob")
    ap.add_argument("--log-every", type=int, default=200)
    ap.add_argument("--mode", default="physics", choices=["physics", "data"])
    ap.add_argument("--windows", type=int, default=4, help="data mode: windows factored per step")
    ap.add_argument("--rhs", type=int, default=16, help="data mode: right-hand sides per window")
    ap.add_argument("--rank", type=int, default=0, help="data mode: rank-r spectral weights (modified FNO)")
    ap.add_argument("--modulation", action="store_true", help="data mode: the modulation path (modified FNO)")
    a = ap.parse_args()
    os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
    if a.mode == "data":
        train_data(a.minutes, a.windows, a.rhs, a.lr, a.seed, a.out, a.log_every, a.device, a.init,
                   rank=a.rank, modulation=a.modulation)
    else:
        train(a.minutes, a.batch, a.recur, a.lr, a.seed, a.out, a.log_every, a.device, a.init)
