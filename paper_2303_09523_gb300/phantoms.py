"""Seeded synthetic slice stacks shaped like the paper's spine and brain MRI series.

The paper validates on private T2 spine and brain stacks (512x512 slices,
Sec. 5) that are not available; these phantoms stand in for them.  Each
phantom is a piecewise-constant anatomy defined in continuous coordinates of
the fine (output) grid, where known slice j sits at z = j*g.  Only the known
slices (plus noise) are handed to the interpolator; the noise-free fine slices
at the missing z are the ground truth for quality metrics.

This module holds no kriging arithmetic: it is the one input generator that
both the CUDA library's tests/benchmark and the oracle consume.
Randomness: ``numpy.random.Generator(PCG64(seed))``.
"""
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

SEED_BASE = 230309523


@dataclass
class Volume:
    """One synthetic known-slice stack and its interpolation settings."""
    name: str
    slices: np.ndarray            # (n, H, W) in its storage dtype (float64 / float32 / uint16)
    zfactor: int                  # g: output slices per gap
    half_w: int                   # r: neighbourhood half-width (K = 2 (2r+1)^2)
    n_sub_blocks: int             # k: Z sub-blocks
    model: str                    # "spherical" | "exponential"
    nugget: float
    sill: float
    range: float
    in_scale: float = 1.0         # uint16 storage: value = float32(u16) * in_scale
    truth: Optional[np.ndarray] = field(default=None, repr=False)  # noise-free fine volume, if built

    @property
    def n(self):
        return self.slices.shape[0]

    @property
    def H(self):
        return self.slices.shape[1]

    @property
    def W(self):
        return self.slices.shape[2]

    @property
    def n_out(self):
        return (self.n - 1) * self.zfactor + 1

    @property
    def n_missing(self):
        return (self.n - 1) * (self.zfactor - 1) * self.H * self.W

    def values_f64(self) -> np.ndarray:
        """The exact values the interpolator sees, widened to float64."""
        if self.slices.dtype == np.uint16:
            return (self.slices.astype(np.float32) * np.float32(self.in_scale)).astype(np.float64)
        return self.slices.astype(np.float64)

    def variogram(self):
        return dict(model=self.model, nugget=self.nugget, sill=self.sill, range=self.range)


# --------------------------------------------------------------------------
# anatomy, evaluated on a (z, y, x) grid in fine-voxel units
# --------------------------------------------------------------------------

def _grid(H, W, zs):
    z = np.asarray(zs, dtype=np.float64)[:, None, None]
    y = np.arange(H, dtype=np.float64)[None, :, None]
    x = np.arange(W, dtype=np.float64)[None, None, :]
    return z, y, x


def _ellipsoid(z, y, x, c, ax):
    return ((x - c[0]) / ax[0]) ** 2 + ((y - c[1]) / ax[1]) ** 2 + ((z - c[2]) / ax[2]) ** 2 <= 1.0


def _rounded_box(z, y, x, c, half, rad):
    qx = np.abs(x - c[0]) - half[0]
    qy = np.abs(y - c[1]) - half[1]
    qz = np.abs(z - c[2]) - half[2]
    outside = np.sqrt(np.maximum(qx, 0) ** 2 + np.maximum(qy, 0) ** 2 + np.maximum(qz, 0) ** 2)
    inside = np.minimum(np.maximum(np.maximum(qx, qy), qz), 0.0)
    return outside + inside - rad <= 0.0


def ellipsoids_anatomy(H, W, depth, zs):
    """Three nested ellipsoids: 0.2 (outer), 0.6, 1.0 (inner) on 0."""
    z, y, x = _grid(H, W, zs)
    c = ((W - 1) / 2.0, (H - 1) / 2.0, (depth - 1) / 2.0)
    v = np.zeros(np.broadcast_shapes(z.shape, y.shape, x.shape))
    for scale, val in ((0.45, 0.2), (0.30, 0.6), (0.15, 1.0)):
        ax = (scale * W, scale * H * 0.8, scale * depth * 1.6)
        v = np.where(_ellipsoid(z, y, x, c, ax), val, v)
    return v


def spine_anatomy(H, W, depth, zs, rng_geom):
    """Stacked rounded-box vertebrae (1.0), discs (0.5), cord cylinder (0.3), background 0.1.

    The spine runs along y; slices are taken along z (sagittal-like stack).
    """
    z, y, x = _grid(H, W, zs)
    v = np.full(np.broadcast_shapes(z.shape, y.shape, x.shape), 0.1)
    cx, cz = 0.45 * W, (depth - 1) / 2.0
    n_vert = 7
    pitch = H / (n_vert + 0.5)
    jit = rng_geom.uniform(-0.04, 0.04, size=(n_vert, 3))
    for k in range(n_vert):
        cy = pitch * (k + 0.75)
        c = (cx * (1 + jit[k, 0]), cy, cz * (1 + jit[k, 2]))
        half = (0.13 * W, 0.30 * pitch, 0.22 * depth)
        v = np.where(_rounded_box(z, y, x, c, half, 0.06 * pitch), 1.0, v)
        if k + 1 < n_vert:
            cd = (c[0], cy + 0.5 * pitch, c[2])
            halfd = (0.12 * W, 0.10 * pitch, 0.20 * depth)
            v = np.where(_rounded_box(z, y, x, cd, halfd, 0.04 * pitch), 0.5, v)
    # spinal cord: cylinder along y, posterior to the vertebral bodies
    rc = 0.05 * W
    cord = ((x - (cx + 0.22 * W)) / rc) ** 2 + ((z - cz) / (rc * depth / W * 1.5 + 1e-9)) ** 2 <= 1.0
    v = np.where(cord & (y >= 0), 0.3, v)
    return v


def brain_anatomy(H, W, depth, zs, rng_geom):
    """Skull shell, grey/white-matter ellipsoids and ventricles, with a smooth multiplicative bias field."""
    z, y, x = _grid(H, W, zs)
    shape = np.broadcast_shapes(z.shape, y.shape, x.shape)
    c = ((W - 1) / 2.0, (H - 1) / 2.0, (depth - 1) / 2.0)
    v = np.zeros(shape)
    sk = (0.46 * W, 0.40 * H, 0.48 * depth)
    v = np.where(_ellipsoid(z, y, x, c, sk), 0.9, v)                       # skull
    v = np.where(_ellipsoid(z, y, x, c, (sk[0] * 0.92, sk[1] * 0.92, sk[2] * 0.92)), 0.15, v)  # CSF gap
    v = np.where(_ellipsoid(z, y, x, c, (sk[0] * 0.88, sk[1] * 0.88, sk[2] * 0.88)), 0.6, v)   # grey matter
    v = np.where(_ellipsoid(z, y, x, c, (sk[0] * 0.70, sk[1] * 0.66, sk[2] * 0.70)), 0.8, v)   # white matter
    for side in (-1, 1):                                                   # lateral ventricles
        cv = (c[0] + side * 0.08 * W, c[1] - 0.02 * H, c[2])
        v = np.where(_ellipsoid(z, y, x, cv, (0.05 * W, 0.16 * H, 0.18 * depth)), 1.0, v)
    # smooth bias field: 1 + low-order polynomial, within about +-10 %
    a = rng_geom.uniform(-1.0, 1.0, size=6)
    u, w_, s = (x - c[0]) / W, (y - c[1]) / H, (z - c[2]) / max(depth, 1)
    bias = a[0] * u + a[1] * w_ + a[2] * s + a[3] * u * w_ + a[4] * u * u + a[5] * w_ * w_
    bias = 1.0 + 0.1 * bias / max(np.abs(a).sum() * 0.5, 1e-9)
    return v * bias


# --------------------------------------------------------------------------
# noise and storage
# --------------------------------------------------------------------------

def rician(v, sigma, rng):
    n1 = rng.normal(0.0, sigma, size=v.shape)
    n2 = rng.normal(0.0, sigma, size=v.shape)
    return np.sqrt((v + n1) ** 2 + n2 ** 2)


def to_u16(v):
    """uint16 storage: clamp(round(v * 32767), 0, 65535); value = float32(u16) * float32(1/32767)."""
    return np.clip(np.rint(v * 32767.0), 0, 65535).astype(np.uint16), float(np.float32(1.0 / 32767.0))


def population_variance(a) -> float:
    a = np.asarray(a, dtype=np.float64)
    return float(a.var(ddof=0))


# --------------------------------------------------------------------------
# the five configurations
# --------------------------------------------------------------------------

def tiny_ellipsoids(n=9, H=64, W=64, g=4, k=2, seed=SEED_BASE + 0, with_truth=False) -> Volume:
    """9 known 64x64 float64 slices, nested ellipsoids, Rician 0.02; g 4; 18 points; spherical, range 8."""
    rng = np.random.Generator(np.random.PCG64(seed))
    depth = (n - 1) * g + 1
    known = ellipsoids_anatomy(H, W, depth, [j * g for j in range(n)])
    sl = rician(known, 0.02, rng)
    vol = Volume("tiny_ellipsoids_%dx%dx%d_g%d" % (n, H, W, g), sl.astype(np.float64), g, 1, k,
                 "spherical", 0.0, population_variance(sl), 8.0)
    if with_truth:
        vol.truth = ellipsoids_anatomy(H, W, depth, range(depth))
    return vol


def spine(n=24, H=256, W=256, g=4, k=4, half_w=1, seed=SEED_BASE + 1, with_truth=False) -> Volume:
    """24 known 256x256 slices, spine anatomy, Rician 0.03, stored uint16; g 4; 18 points; spherical."""
    rng = np.random.Generator(np.random.PCG64(seed))
    geom = np.random.Generator(np.random.PCG64(seed + 7))
    depth = (n - 1) * g + 1
    known = spine_anatomy(H, W, depth, [j * g for j in range(n)], geom)
    sl = rician(known, 0.03, rng)
    u16, scale = to_u16(sl)
    vol = Volume("spine_%dx%dx%d_g%d_u16" % (n, H, W, g), u16, g, half_w, k, "spherical", 0.0, 0.0, 8.0,
                 in_scale=scale)
    vol.sill = population_variance(vol.values_f64())
    if with_truth:
        vol.truth = spine_anatomy(H, W, depth, range(depth), np.random.Generator(np.random.PCG64(seed + 7)))
    return vol


def brain(n=32, H=512, W=512, g=6, k=8, half_w=2, seed=SEED_BASE + 2, with_truth=False, dtype=np.float32) -> Volume:
    """32 known 512x512 float32 slices, brain anatomy with bias field, Gaussian 0.02; g 6; 50 points; exponential."""
    rng = np.random.Generator(np.random.PCG64(seed))
    geom = np.random.Generator(np.random.PCG64(seed + 7))
    depth = (n - 1) * g + 1
    known = brain_anatomy(H, W, depth, [j * g for j in range(n)], geom)
    sl = (known + rng.normal(0.0, 0.02, size=known.shape)).astype(dtype)
    vol = Volume("brain_%dx%dx%d_g%d" % (n, H, W, g), sl, g, half_w, k, "exponential", 0.0,
                 population_variance(sl), 8.0)
    if with_truth:
        vol.truth = brain_anatomy(H, W, depth, range(depth), np.random.Generator(np.random.PCG64(seed + 7)))
    return vol


def batch_mix(count=16, seed=SEED_BASE + 3, max_side=512) -> List[Volume]:
    """16 seeded spine/brain float32 phantoms: sides 128..512 step 64, 12-40 slices, g 2-6, 18 or 50 points."""
    vols = []
    for i in range(count):
        rng = np.random.Generator(np.random.PCG64(seed + 100 * i))
        sides = [s for s in range(128, max_side + 1, 64)]
        side = int(rng.choice(sides))
        n = int(rng.integers(12, 41))
        g = int(rng.integers(2, 7))
        r = int(rng.choice([1, 2]))
        k = int(rng.choice([2, 4, 8]))
        k = min(k, n - 1)
        s = int(rng.integers(0, 2**31 - 1))
        if i % 2 == 0:
            v = spine(n=n, H=side, W=side, g=g, k=k, half_w=r, seed=s)
            vals = v.values_f64().astype(np.float32)
            vol = Volume("mix%02d_spine_%dx%dx%d_g%d_r%d" % (i, n, side, side, g, r), vals, g, r, k,
                         "spherical", 0.0, population_variance(vals), 8.0)
        else:
            v = brain(n=n, H=side, W=side, g=g, k=k, half_w=r, seed=s)
            vol = Volume("mix%02d_brain_%dx%dx%d_g%d_r%d" % (i, n, side, side, g, r), v.slices, g, r, k,
                         "exponential", 0.0, population_variance(v.slices), 8.0)
        vols.append(vol)
    return vols


def random_stack(n, H, W, g, r, k=1, seed=0, dtype=np.float32, model="spherical", rng_range=8.0) -> Volume:
    """Small smooth random stack for parity cases with ragged sizes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    base = rng.normal(size=(n, H, W))
    # smooth a little so the variogram is meaningful
    sm = base.copy()
    for ax in (1, 2):
        sm = (sm + np.roll(sm, 1, axis=ax) + np.roll(sm, -1, axis=ax)) / 3.0
    sl = (0.5 + 0.2 * sm).astype(dtype)
    return Volume("random_%dx%dx%d_g%d_r%d" % (n, H, W, g, r), sl, g, r, k, model, 0.0,
                  population_variance(sl), rng_range)
