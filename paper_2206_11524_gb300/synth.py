"""Seeded synthetic inputs (geometry, wettability and initial densities).

This module builds input arrays only: bounce-back fraction fields ``ns``,
per-node adhesion parameters ``gads2`` (G_ads,2; G_ads,1 = -G_ads,2), and
initial component densities.  It holds none of the lattice Boltzmann
arithmetic, so both the CUDA library's tests and the CPU oracle can be fed
from it.  All arrays are float32/float64 numpy in ``[z, y, x]`` order.

Stand-ins for the paper's data: the 3D cathode reconstruction (40 % porosity,
Sec. 4) and the binder/separator images are not available, so
``electrode`` draws a Boolean model of overlapping spheres (radius 6-12 lu)
until the solid fraction reaches 60 %, plus gray binder blobs (a thresholded
Gaussian random field filling 21 % of the volume inside the pore space, each
connected blob with its own n_s drawn from U[0.2, 0.9]).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# Table 1 densities (majority / dissolved) and the interaction strength.
RHO_MAJOR = 0.99
RHO_DIS = 0.01
G_TABLE1 = 1.75


@dataclass
class Case:
    """One synthetic problem: geometry, wettability, initial densities and
    the reservoir faces {face: (layers, rho_1, rho_2)}."""
    name: str
    shape: tuple            # (nz, ny, nx)
    ns: np.ndarray
    gads2: np.ndarray
    rho_a: np.ndarray
    rho_b: np.ndarray
    reservoirs: dict
    tau: tuple = (1.0, 1.0)
    G: float = G_TABLE1
    F_ext: tuple = (0.0, 0.0, 0.0)
    steps: int = 0

    @property
    def n_nodes(self) -> int:
        nz, ny, nx = self.shape
        return nx * ny * nz


def gray_slab(nx=32, ny=16, nz=16, ns_slab=0.5, x0=12, x1=19, major=1.0,
              minor=0.03, G=G_TABLE1, force=(1e-5, 0.0, 0.0), steps=500):
    """Gray slab of uniform n_s at x0..x1 (inclusive); fluid 1 fills x < nx/2,
    fluid 2 fills x >= nx/2; periodic on every axis; a body force."""
    shape = (nz, ny, nx)
    x = np.arange(nx)
    ns = np.zeros(shape)
    ns[..., (x >= x0) & (x <= x1)] = ns_slab
    left = np.broadcast_to(x < nx // 2, shape)
    rho_a = np.where(left, major, minor)
    rho_b = np.where(left, minor, major)
    return Case("gray_slab", shape, ns, np.zeros(shape), rho_a, rho_b, {},
                G=G, F_ext=tuple(force), steps=steps)


def droplet(n=128, radius=20.0, ns=0.0, G=G_TABLE1, hi=RHO_MAJOR, lo=RHO_DIS,
            steps=20000):
    """Sphere of fluid 1 (radius in lu, centred) in fluid 2, periodic cube,
    homogeneous gray medium."""
    shape = (n, n, n)
    c = n / 2 - 0.5
    z, y, x = np.meshgrid(*(np.arange(n),) * 3, indexing="ij")
    inside = (x - c) ** 2 + (y - c) ** 2 + (z - c) ** 2 < radius ** 2
    rho_a = np.where(inside, hi, lo)
    rho_b = np.where(inside, lo, hi)
    return Case(f"droplet_R{radius:g}", shape, np.full(shape, float(ns)),
                np.zeros(shape), rho_a, rho_b, {}, G=G, steps=steps)


def random_state(shape, seed, rho=(0.8, 0.2), spread=0.3):
    """Random positive populations, layout [2, 19, nz, ny, nx]: each value is
    rho_sigma / 19 times U[1 - spread, 1 + spread]."""
    rng = np.random.default_rng(seed)
    base = np.array(rho)[:, None, None, None, None] / 19.0
    return base * rng.uniform(1 - spread, 1 + spread, (2, 19) + tuple(shape))


def random_geometry(shape, seed, gads_max=0.3):
    """Random n_s in [0, 1] with exact 0 and 1 cells, random G_ads,2."""
    rng = np.random.default_rng(seed)
    ns = rng.uniform(0, 1, shape)
    ns.flat[::5] = 0.0
    ns.flat[::7] = 1.0
    gads = rng.uniform(-gads_max, gads_max, shape)
    return ns, gads


_OFFSETS = {}


def _offsets(r):
    """Integer offset grids (dz, dy, dx) of the cube [-r, r]^3, built once
    per radius."""
    g = _OFFSETS.get(r)
    if g is None:
        offs = np.arange(-r, r + 1)
        g = _OFFSETS[r] = np.meshgrid(offs, offs, offs, indexing="ij")
    return g


def _periodic_ball_indices(center, radius, shape):
    nz, ny, nx = shape
    r = int(math.ceil(radius))
    dz, dy, dx = _offsets(r)
    fz = center[0] - math.floor(center[0])
    fy = center[1] - math.floor(center[1])
    fx = center[2] - math.floor(center[2])
    inside = (dz - fz) ** 2 + (dy - fy) ** 2 + (dx - fx) ** 2 <= radius ** 2
    z0, y0, x0 = (int(math.floor(v)) for v in center)
    return ((dz[inside] + z0) % nz, (dy[inside] + y0) % ny,
            (dx[inside] + x0) % nx)


def _gaussian_field(shape, sigma, rng):
    """White noise smoothed by a periodic Gaussian (real FFT)."""
    noise = rng.standard_normal(shape)
    kz = np.fft.fftfreq(shape[0])[:, None, None]
    ky = np.fft.fftfreq(shape[1])[None, :, None]
    kx = np.fft.rfftfreq(shape[2])[None, None, :]
    filt = np.exp(-2 * (math.pi * sigma) ** 2 * (kx ** 2 + ky ** 2 + kz ** 2))
    return np.fft.irfftn(np.fft.rfftn(noise) * filt, s=shape)


def _label_components(mask):
    """Connected components (6-neighbourhood) of a boolean mask."""
    from scipy import ndimage
    labels, n = ndimage.label(mask)
    return labels, n


def electrode(n=(256, 256, 256), seed=2206, solid_fraction=0.60,
              r_min=6.0, r_max=12.0, binder_fraction=0.21, binder_sigma=3.0,
              gads_active=0.0, gads_binder=0.214375, res_layers=4,
              rho_in=(1.04, 0.01), rho_out=(0.01, 0.99), G=G_TABLE1,
              steps=50000):
    """Synthetic electrode: solid spheres (n_s = 1, G_ads,2 = gads_active),
    gray binder blobs (n_s ~ U[0.2, 0.9] per blob, G_ads,2 = gads_binder),
    reservoirs of `res_layers` layers at x = 0 (electrolyte, fluid 1) and at
    x = nx - 1 (gas, fluid 2); periodic in y and z.  The pore space starts
    filled with gas (Sec. 4).  The default binder G_ads,2 corresponds to
    theta = 60 deg under Table 1's parameters."""
    nz, ny, nx = n
    shape = (nz, ny, nx)
    rng = np.random.default_rng(seed)
    solid = np.zeros(shape, dtype=bool)
    # Boolean model: add spheres until the target solid fraction is reached.
    target = solid_fraction * solid.size
    count = 0
    mean_ball = 4.0 / 3.0 * math.pi * (r_max ** 4 - r_min ** 4) / (4 * (r_max - r_min))
    while count < target:
        batch = max(1, min(64, int((target - count) / mean_ball)))
        centers = rng.uniform(0, 1, (batch, 3)) * np.array(shape)
        radii = rng.uniform(r_min, r_max, batch)
        for c, r in zip(centers, radii):
            zi, yi, xi = _periodic_ball_indices(c, r, shape)
            # cells this ball adds (its own index list has no repeats)
            count += int(np.count_nonzero(~solid[zi, yi, xi]))
            solid[zi, yi, xi] = True
    # Gray binder: Gaussian random field thresholded inside the pore space.
    field = _gaussian_field(shape, binder_sigma, rng)
    pore = ~solid
    want = binder_fraction * solid.size
    if want > 0 and pore.any():
        vals = field[pore]
        k = min(int(want), vals.size - 1)
        # the (k+1)-th largest pore value is the threshold
        thr = np.partition(vals, vals.size - 1 - k)[vals.size - 1 - k]
        binder = pore & (field >= thr)
    else:
        binder = np.zeros(shape, bool)
    ns = np.where(solid, 1.0, 0.0)
    gads = np.where(solid, gads_active, 0.0)
    labels, nlab = _label_components(binder)
    blob_ns = rng.uniform(0.2, 0.9, nlab + 1)
    ns = np.where(binder, blob_ns[labels], ns)
    gads = np.where(binder, gads_binder, gads)
    # Reservoir layers are open fluid.
    ns[..., :res_layers] = 0.0
    ns[..., nx - res_layers:] = 0.0
    gads[..., :res_layers] = 0.0
    gads[..., nx - res_layers:] = 0.0
    rho_a = np.full(shape, RHO_DIS)
    rho_b = np.full(shape, RHO_MAJOR)
    rho_a[..., :res_layers] = rho_in[0]
    rho_b[..., :res_layers] = rho_in[1]
    rho_a[..., nx - res_layers:] = rho_out[0]
    rho_b[..., nx - res_layers:] = rho_out[1]
    res = {0: (res_layers, rho_in[0], rho_in[1]),
           1: (res_layers, rho_out[0], rho_out[1])}
    return Case(f"electrode_{nx}x{ny}x{nz}", shape, ns, gads, rho_a, rho_b,
                res, G=G, steps=steps)
