"""Seeded synthetic inputs shared by the tests, the bench and the oracle runs.

This module generates *inputs only*: optical parameter sets, voxelised
phantoms and noise.  It contains none of the imaging model's arithmetic (no
pupils, transfer functions, FFTs or solves), so the oracle and the CUDA path
can both consume its arrays without sharing any method code.

The paper's experiments use microscopy datasets that are not available; these
phantoms stand in for them with the shapes and value distributions of the
workloads the method is evaluated on:

* widefield z-stack, 16 x 64 x 64, 20 spheres (radius U[0.5, 2] um,
  index increment U[0.005, 0.03]);
* joint phase + absorption + fluorescence volume, 96 x 512 x 512, 2000 spheres
  plus 200 random ellipsoidal shells, absorption U[0, 0.01], fluorophore
  density log-normal(0, 1) per object;
* shift-variant field 48 x 2048 x 2048 cut into a 16 x 16 grid of tiles, each
  with its own defocus U[-1, 1] um, illumination tilt U[-0.1, 0.1] NA per axis
  and illumination NA U[0.7, 0.95].

Conventions: arrays are (Z, Y, X) with x contiguous; voxel (k, j, i) sits at
(k*dz, j*p, i*p) micrometres.
"""
from __future__ import annotations

import numpy as np

OPTICS_KEYS = ("lambda_um", "n_medium", "pixel_um", "z_step_um", "na_det",
               "na_ill", "tilt_x", "tilt_y", "defocus_um")

# Widefield optics shared by the three volumetric workloads.
WIDEFIELD_OPTICS = dict(lambda_um=0.532, n_medium=1.33, pixel_um=0.1,
                        z_step_um=0.25, na_det=1.2, na_ill=0.9,
                        tilt_x=0.0, tilt_y=0.0, defocus_um=0.0)

# Low-NA phase-from-defocus optics used for the auto-tuned 2D phase
# reconstructions of the pooled-screen data (Methods, "Cell-scale optical
# pooled screen data": 450 nm, NA_det 0.15, NA_ill 0.1, n = 1.0).
POOLED_SCREEN_OPTICS = dict(lambda_um=0.45, n_medium=1.0, pixel_um=0.65,
                            z_step_um=2.0, na_det=0.15, na_ill=0.1,
                            tilt_x=0.0, tilt_y=0.0, defocus_um=0.0)

SHAPE_SMALL = (16, 64, 64)
SHAPE_WIDEFIELD = (96, 512, 512)
FIELD_SHAPE = (48, 2048, 2048)
TILE_CORE = 128
TILE_HALO = 32


def optics(**overrides) -> dict:
    """A copy of the widefield optics with some fields replaced.  The flag
    smooth_source=True selects the smooth-edged source pupil (a model flag,
    not an optics field)."""
    o = dict(WIDEFIELD_OPTICS)
    for k, v in overrides.items():
        if k == "smooth_source":
            o[k] = bool(v)
            continue
        if k not in OPTICS_KEYS:
            raise KeyError(k)
        o[k] = float(v)
    return o


def tile_optics(rng: np.random.Generator, n_tiles: int, base: dict | None = None) -> list[dict]:
    """Per-tile parameter vectors theta for the shift-variant field.

    defocus U[-1, 1] um, tilt_x and tilt_y U[-0.1, 0.1] NA, NA_ill U[0.7, 0.95].
    """
    base = dict(WIDEFIELD_OPTICS if base is None else base)
    out = []
    for _ in range(n_tiles):
        o = dict(base)
        o["defocus_um"] = float(rng.uniform(-1.0, 1.0))
        o["tilt_x"] = float(rng.uniform(-0.1, 0.1))
        o["tilt_y"] = float(rng.uniform(-0.1, 0.1))
        o["na_ill"] = float(rng.uniform(0.7, 0.95))
        out.append(o)
    return out


def _box(center, half, spacing, shape):
    """Index ranges of the voxels whose centres can lie within `half` um of `center`."""
    lo = [max(0, int(np.floor((c - h) / s))) for c, h, s in zip(center, half, spacing)]
    hi = [min(n, int(np.ceil((c + h) / s)) + 1) for c, h, s, n in zip(center, half, spacing, shape)]
    return lo, hi


def _local_coords(lo, hi, spacing, center):
    axes = [np.arange(l, h) * s - c for l, h, s, c in zip(lo, hi, spacing, center)]
    return np.meshgrid(*axes, indexing="ij")


def add_spheres(vols, rng, n, r_range, values, shape, spacing):
    """Rasterise `n` spheres: voxel centre inside -> add the object's values.

    `values` maps a volume name to a callable rng -> value drawn per object.
    Centres are uniform in the box; no wrap; clipped at the borders; overlaps add.
    """
    extent = [n_ * s for n_, s in zip(shape, spacing)]
    for _ in range(n):
        c = [rng.uniform(0.0, e) for e in extent]
        r = rng.uniform(*r_range)
        vals = {k: f(rng) for k, f in values.items()}
        lo, hi = _box(c, (r, r, r), spacing, shape)
        if any(h <= l for l, h in zip(lo, hi)):
            continue
        zz, yy, xx = _local_coords(lo, hi, spacing, c)
        inside = zz * zz + yy * yy + xx * xx <= r * r
        sl = tuple(slice(l, h) for l, h in zip(lo, hi))
        for k, v in vals.items():
            vols[k][sl] += v * inside


def random_rotation(rng) -> np.ndarray:
    """Uniform random rotation from a normalised Gaussian quaternion."""
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


def add_shells(vols, rng, n, axes_range, thickness, values, shape, spacing):
    """Rasterise `n` randomly rotated ellipsoidal shells of the given thickness.

    A voxel belongs to the shell when its centre is inside the outer ellipsoid
    (semi-axes a) and outside the inner one (semi-axes a - thickness).
    """
    extent = [n_ * s for n_, s in zip(shape, spacing)]
    for _ in range(n):
        c = [rng.uniform(0.0, e) for e in extent]
        a = np.array([rng.uniform(*axes_range) for _ in range(3)])
        rot = random_rotation(rng)
        vals = {k: f(rng) for k, f in values.items()}
        rmax = float(a.max())
        lo, hi = _box(c, (rmax, rmax, rmax), spacing, shape)
        if any(h <= l for l, h in zip(lo, hi)):
            continue
        zz, yy, xx = _local_coords(lo, hi, spacing, c)
        pts = np.stack([zz, yy, xx], axis=-1) @ rot  # body-frame coordinates
        outer = np.sum((pts / a) ** 2, axis=-1) <= 1.0
        ai = np.maximum(a - thickness, 1e-6)
        inner = np.sum((pts / ai) ** 2, axis=-1) <= 1.0
        shell = outer & ~inner
        sl = tuple(slice(l, h) for l, h in zip(lo, hi))
        for k, v in vals.items():
            vols[k][sl] += v * shell


def spacing_of(o: dict):
    return (o["z_step_um"], o["pixel_um"], o["pixel_um"])


def sphere_phantom(seed: int, shape=SHAPE_SMALL, o: dict | None = None, n_spheres: int = 20,
                   r_range=(0.5, 2.0), dn_range=(0.005, 0.03)) -> np.ndarray:
    """Index-increment volume of `n_spheres` spheres (float64)."""
    o = WIDEFIELD_OPTICS if o is None else o
    rng = np.random.default_rng(seed)
    vols = {"dn": np.zeros(shape)}
    add_spheres(vols, rng, n_spheres, r_range, {"dn": lambda g: g.uniform(*dn_range)},
                shape, spacing_of(o))
    return vols["dn"]


def widefield_phantom(seed: int, shape=SHAPE_WIDEFIELD, o: dict | None = None,
                      n_spheres: int = 2000, n_shells: int = 200) -> dict:
    """Joint phase + absorption + fluorescence phantom (float64 volumes).

    Spheres: radius U[0.5, 2] um; shells: semi-axes U[1, 4] um, thickness
    0.3 um, uniform random rotation.  Every object draws its own index increment
    U[0.005, 0.03], absorption U[0, 0.01] and log-normal(0, 1) fluorophore density.
    """
    o = WIDEFIELD_OPTICS if o is None else o
    rng = np.random.default_rng(seed)
    vols = {k: np.zeros(shape) for k in ("dn", "kappa", "rho")}
    vals = {"dn": lambda g: g.uniform(0.005, 0.03),
            "kappa": lambda g: g.uniform(0.0, 0.01),
            "rho": lambda g: g.lognormal(0.0, 1.0)}
    add_spheres(vols, rng, n_spheres, (0.5, 2.0), vals, shape, spacing_of(o))
    add_shells(vols, rng, n_shells, (1.0, 4.0), 0.3, vals, shape, spacing_of(o))
    return vols


def gaussian_noise(seed: int, shape, sigma: float) -> np.ndarray:
    """N(0, sigma^2) noise, float64."""
    return np.random.default_rng(seed).normal(0.0, sigma, size=shape)


def uniform_volume(seed: int, shape, lo=-1.0, hi=1.0) -> np.ndarray:
    return np.random.default_rng(seed).uniform(lo, hi, size=shape)


def thin_sphere_params(seed: int, shape2d, o: dict | None = None, n_spheres: int = 40,
                       r_range=(0.5, 2.0), dn_range=(0.005, 0.03)) -> np.ndarray:
    """Sphere parameters of a thin specimen, (n_spheres, 4) float64 rows of
    (centre y, centre x, radius, dn) in um: centres uniform over the periodic
    tile, radius and dn as in ``sphere_phantom``."""
    o = WIDEFIELD_OPTICS if o is None else o
    rng = np.random.default_rng(seed)
    Y, X = shape2d
    p = o["pixel_um"]
    out = np.zeros((n_spheres, 4))
    for i in range(n_spheres):
        out[i] = (rng.uniform(0, Y * p), rng.uniform(0, X * p), rng.uniform(*r_range), rng.uniform(*dn_range))
    return out


def thin_phantom_from_params(params: np.ndarray, shape2d, o: dict | None = None) -> np.ndarray:
    """Spheres projected along z onto the object plane, as the index increment
    of one plane of thickness z_step: sum dn 2 sqrt(r^2 - rho^2) / z_step
    (float64 (Y, X), periodic minimum-image distances)."""
    o = WIDEFIELD_OPTICS if o is None else o
    Y, X = shape2d
    p = o["pixel_um"]
    yy, xx = np.meshgrid(np.arange(Y) * p, np.arange(X) * p, indexing="ij")
    out = np.zeros((Y, X))
    for cy, cx, r, dn in params:
        dy = (yy - cy + 0.5 * Y * p) % (Y * p) - 0.5 * Y * p
        dx = (xx - cx + 0.5 * X * p) % (X * p) - 0.5 * X * p
        rho2 = dy * dy + dx * dx
        out += dn * 2.0 * np.sqrt(np.maximum(r * r - rho2, 0.0)) / o["z_step_um"]
    return out


def thin_phantom(seed: int, shape2d, o: dict | None = None, n_spheres: int = 40,
                 r_range=(0.5, 2.0), dn_range=(0.005, 0.03)) -> np.ndarray:
    """Thin specimen for the 2D (phase-from-defocus) model: spheres projected
    along z onto the object plane (``thin_sphere_params`` then
    ``thin_phantom_from_params``)."""
    return thin_phantom_from_params(thin_sphere_params(seed, shape2d, o, n_spheres, r_range, dn_range), shape2d, o)


def aperture_optics(n_apertures: int = 9, ring_na: float = 0.6, na_ill: float = 0.15,
                    base: dict | None = None) -> list[dict]:
    """Illumination apertures for multi-aperture fusion: one on axis and
    n_apertures - 1 evenly spaced on a ring of radius ring_na (NA units), each
    of numerical aperture na_ill."""
    base = WIDEFIELD_OPTICS if base is None else base
    out = [dict(base, na_ill=na_ill, tilt_x=0.0, tilt_y=0.0)]
    for i in range(n_apertures - 1):
        a = 2.0 * np.pi * i / (n_apertures - 1)
        out.append(dict(base, na_ill=na_ill, tilt_x=ring_na * np.cos(a), tilt_y=ring_na * np.sin(a)))
    return out
