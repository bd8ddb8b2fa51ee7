"""Seeded synthetic inputs for the Schwarz neural-operator FDFD solver.

This module only draws inputs: permittivity maps, sources, neural-operator
weights and random test vectors.  It holds none of the solver's arithmetic
(no operator, no PML, no preconditioner), so both the CUDA path and the CPU
oracle can be fed from it without sharing any of the method.

The paper's own data (cropped freeform simulations, Methods "Training data
generation") is not available; the recipes below stand in for it with the
value ranges the paper uses (permittivity 1 to 12.25, feature sizes of at
least 8 cells, grids of 20 to 40 cells per wavelength).

Every generator takes an integer seed and uses numpy's PCG64.
"""
from __future__ import annotations

import numpy as np

# Physical scales shared by every workload (SI units).
WAVELENGTH_DEFAULT = 1.55e-6
NPML_DEFAULT = 20

# Neural-operator shape (Sec. 2.1, Fig. 2; width 32, 4 Fourier blocks,
# 16 x 16 retained modes, 80 x 80 windows = 64 x 64 core + 8 cells overlap).
NNO_CIN = 15
NNO_WIDTH = 32
NNO_BLOCKS = 4
NNO_MODES_Y = 32  # ky in {0..15} and {-16..-1}
NNO_MODES_X = 16  # kx in {0..15}
NNO_HIDDEN = 128
WIN = 80
CORE = 64
OVERLAP = 8


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def rectangles_eps(nx: int, ny: int, npml: int = NPML_DEFAULT, n_rect: int = 24,
                   seed: int = 1000, values=(2.1, 12.25)) -> np.ndarray:
    """Axis-aligned rectangles of permittivity drawn from `values` on a
    background of 1, sides uniform in 8..64 cells, clipped to the region
    inside the PML; later rectangles overwrite earlier ones."""
    g = rng(seed)
    eps = np.ones((ny, nx), dtype=np.float32)
    lo_x, hi_x = npml, nx - npml
    lo_y, hi_y = npml, ny - npml
    for _ in range(n_rect):
        w = int(g.integers(8, 65))
        h = int(g.integers(8, 65))
        x0 = int(g.integers(lo_x - w // 2, hi_x - w // 2))
        y0 = int(g.integers(lo_y - h // 2, hi_y - h // 2))
        v = values[int(g.integers(0, len(values)))]
        xa, xb = max(x0, lo_x), min(x0 + w, hi_x)
        ya, yb = max(y0, lo_y), min(y0 + h, hi_y)
        if xa < xb and ya < yb:
            eps[ya:yb, xa:xb] = v
    return eps


def _disk(radius: int) -> np.ndarray:
    r = np.arange(-radius, radius + 1)
    return (r[None, :] ** 2 + r[:, None] ** 2) <= radius * radius


def freeform_eps(nx: int, ny: int, npml: int = NPML_DEFAULT, seed: int = 2000,
                 sigma: float = 3.0, radius: int = 4, lo: float = 1.0,
                 hi: float = 12.25) -> np.ndarray:
    """Gaussian-smoothed white noise thresholded at zero, opened then closed
    with a disk of `radius` so features are at least 2*radius cells, mapped
    to {lo, hi}; PML cells are set to `lo`."""
    from scipy import ndimage
    g = rng(seed)
    noise = g.standard_normal((ny, nx))
    smooth = ndimage.gaussian_filter(noise, sigma, mode="wrap")
    mask = smooth > 0.0
    fp = _disk(radius)
    mask = ndimage.binary_opening(mask, structure=fp)
    mask = ndimage.binary_closing(mask, structure=fp)
    eps = np.where(mask, hi, lo).astype(np.float32)
    if npml > 0:
        eps[:npml, :] = lo
        eps[-npml:, :] = lo
        eps[:, :npml] = lo
        eps[:, -npml:] = lo
    return eps


def point_source(nx: int, ny: int, x: int | None = None, y: int | None = None) -> np.ndarray:
    """Unit current density (1 A/m^2) in one cell, default at the centre."""
    J = np.zeros((ny, nx), dtype=np.complex64)
    J[ny // 2 if y is None else y, nx // 2 if x is None else x] = 1.0
    return J


def random_field(nx: int, ny: int, seed: int, dtype=np.complex64) -> np.ndarray:
    g = rng(seed)
    v = g.standard_normal((ny, nx)) + 1j * g.standard_normal((ny, nx))
    return v.astype(dtype)


def demux_layout(n: int = 512, npml: int = NPML_DEFAULT, design: int = 200,
                 guide_w: int = 8, seed: int = 4000):
    """Three-port wavelength demultiplexer (one input guide on the left,
    outputs on the right at y = 156/256/356 for n = 512), cladding 2.1,
    guides 12.25, design region `design` x `design` at the centre with
    permittivity uniform in [2.1, 12.25].

    Returns (eps, design_mask, src_x, src_rows, port_x, port_rows) where the
    rows are (y_lo, y_hi) of each guide.
    """
    g = rng(seed)
    eps = np.full((n, n), 2.1, dtype=np.float32)
    c = n // 2
    d0, d1 = c - design // 2, c + design // 2
    yin = (c - guide_w // 2, c + guide_w // 2)
    eps[yin[0]:yin[1], :d0] = 12.25
    outs = [c - 100, c, c + 100]
    port_rows = []
    for yc in outs:
        r = (yc - guide_w // 2, yc + guide_w // 2)
        port_rows.append(r)
        eps[r[0]:r[1], d1:] = 12.25
    mask = np.zeros((n, n), dtype=bool)
    mask[d0:d1, d0:d1] = True
    eps[mask] = g.uniform(2.1, 12.25, size=design * design).astype(np.float32)
    src_x = npml + 20
    port_x = n - npml - 20
    return eps, mask, src_x, yin, port_x, port_rows


MOD_CH, MOD_AUX, MOD_FEAT = 16, 5, 144   # modulation path: conv channels, aux inputs, pooled features


def nno_weights(seed: int = 0, width: int = NNO_WIDTH, cin: int = NNO_CIN,
                hidden: int = NNO_HIDDEN, blocks: int = NNO_BLOCKS,
                my: int = NNO_MODES_Y, mx: int = NNO_MODES_X, rank: int = 0,
                modulation: bool = False) -> dict:
    """Seeded initialisation of the Fourier neural operator (Fig. 2).

    Spectral weights follow the usual FNO recipe (uniform in [0, 1) times
    1/(in*out), real and imaginary parts drawn independently); 1x1 layers
    are uniform in +-1/sqrt(fan_in).  rank > 0: R_b is given by the factors
    theta_b [width][width][rank] (FNO recipe) and V_b [rank][my][mx]
    (uniform +-1/sqrt(rank)).  modulation: the modulation path's
    convolution (uniform +-1/sqrt(45)) and fully connected layer (uniform
    +-0.1/sqrt(144), so the seeded modulation is small).  Arrays are float32.
    """
    g = rng(seed)

    def lin(o, i):
        b = 1.0 / np.sqrt(i)
        return (g.uniform(-b, b, size=(o, i)).astype(np.float32),
                g.uniform(-b, b, size=(o,)).astype(np.float32))

    w = {}
    w["lift_w"], w["lift_b"] = lin(width, cin)
    scale = 1.0 / (width * width)
    for b in range(blocks):
        if rank:
            w[f"R{b}_theta_re"] = (scale * g.random((width, width, rank))).astype(np.float32)
            w[f"R{b}_theta_im"] = (scale * g.random((width, width, rank))).astype(np.float32)
            v = 1.0 / np.sqrt(rank)
            w[f"R{b}_V_re"] = g.uniform(-v, v, size=(rank, my, mx)).astype(np.float32)
            w[f"R{b}_V_im"] = g.uniform(-v, v, size=(rank, my, mx)).astype(np.float32)
        else:
            w[f"R{b}_re"] = (scale * g.random((width, width, my, mx))).astype(np.float32)
            w[f"R{b}_im"] = (scale * g.random((width, width, my, mx))).astype(np.float32)
        w[f"W{b}"], w[f"b{b}"] = lin(width, width)
    w["p1_w"], w["p1_b"] = lin(hidden, width)
    w["p2_w"], w["p2_b"] = lin(2, hidden)
    if modulation:
        c = 1.0 / np.sqrt(MOD_AUX * 9)
        w["mod_conv_w"] = g.uniform(-c, c, size=(MOD_CH, MOD_AUX, 3, 3)).astype(np.float32)
        w["mod_conv_b"] = g.uniform(-c, c, size=(MOD_CH,)).astype(np.float32)
        f = 0.1 / np.sqrt(MOD_FEAT)
        w["mod_fc_w"] = g.uniform(-f, f, size=(blocks * my * mx, MOD_FEAT)).astype(np.float32)
        w["mod_fc_b"] = g.uniform(-f, f, size=(blocks * my * mx,)).astype(np.float32)
    return w


def weight_rank(w: dict) -> int:
    """Rank of the spectral weights' factorisation (0 = full R)."""
    return int(w["R0_theta_re"].shape[2]) if "R0_theta_re" in w else 0


# Order of tensors in the flat float32 weight blob handed to the library.
def weight_order(blocks: int = NNO_BLOCKS, rank: int = 0, modulation: bool = False):
    names = ["lift_w", "lift_b"]
    for b in range(blocks):
        if rank:
            names += [f"R{b}_theta_re", f"R{b}_theta_im", f"R{b}_V_re", f"R{b}_V_im"]
        else:
            names += [f"R{b}_re", f"R{b}_im"]
        names += [f"W{b}", f"b{b}"]
    names += ["p1_w", "p1_b", "p2_w", "p2_b"]
    if modulation:
        names += ["mod_conv_w", "mod_conv_b", "mod_fc_w", "mod_fc_b"]
    return names


def pack_weights(w: dict) -> np.ndarray:
    """Flatten a weight dict into the blob layout the C-ABI expects."""
    order = weight_order(rank=weight_rank(w), modulation="mod_fc_w" in w)
    return np.concatenate([np.ascontiguousarray(w[n], dtype=np.float32).ravel() for n in order])


def weight_shapes(width: int = NNO_WIDTH, cin: int = NNO_CIN, hidden: int = NNO_HIDDEN,
                  blocks: int = NNO_BLOCKS, my: int = NNO_MODES_Y, mx: int = NNO_MODES_X, rank: int = 0):
    shapes = {"lift_w": (width, cin), "lift_b": (width,),
              "p1_w": (hidden, width), "p1_b": (hidden,),
              "p2_w": (2, hidden), "p2_b": (2,),
              "mod_conv_w": (MOD_CH, MOD_AUX, 3, 3), "mod_conv_b": (MOD_CH,),
              "mod_fc_w": (blocks * my * mx, MOD_FEAT), "mod_fc_b": (blocks * my * mx,)}
    for b in range(blocks):
        shapes[f"R{b}_re"] = (width, width, my, mx)
        shapes[f"R{b}_im"] = (width, width, my, mx)
        shapes[f"R{b}_theta_re"] = shapes[f"R{b}_theta_im"] = (width, width, rank)
        shapes[f"R{b}_V_re"] = shapes[f"R{b}_V_im"] = (rank, my, mx)
        shapes[f"W{b}"] = (width, width)
        shapes[f"b{b}"] = (width,)
    return shapes


def unpack_weights(blob: np.ndarray, rank: int = 0, modulation: bool = False, **kw) -> dict:
    shapes = weight_shapes(rank=rank, **kw)
    out, off = {}, 0
    for n in weight_order(rank=rank, modulation=modulation):
        sz = int(np.prod(shapes[n]))
        out[n] = blob[off:off + sz].reshape(shapes[n]).astype(np.float32)
        off += sz
    assert off == blob.size, (off, blob.size)
    return out


# Workloads named by what they are (grid, wavelength, resolution, medium).
def workload(name: str) -> dict:
    """Seeded synthetic workloads (problem definitions only)."""
    lam = WAVELENGTH_DEFAULT
    if name == "rect256":  # 256^2, lambda/25, rectangles, centre line source
        n = 256
        return dict(nx=n, ny=n, dx=lam / 25, wavelength=lam, npml=NPML_DEFAULT,
                    eps=rectangles_eps(n, n, seed=1000), J=point_source(n, n), k_coarse=36)
    if name.startswith("freeform"):  # freeform<N>, lambda/30
        n = int(name[len("freeform"):])
        return dict(nx=n, ny=n, dx=lam / 30, wavelength=lam, npml=NPML_DEFAULT,
                    eps=freeform_eps(n, n, seed=2000 + n), J=point_source(n, n), k_coarse=36)
    raise KeyError(name)
