"""Tiling and blending for shift-variant restoration, float64 (test infrastructure).

The field of view is divided into overlapping, approximately shift-invariant
tiles, each reconstructed with its own parameters (Results, "Physics-guided ML
auto-tunes multi-contrast blind deconvolution"; Fig. 2a), and the tiles are
stitched back with linearly weighted blending (Methods, "Organelle-scale
optical pooled screen data": linearly weighted EDT-based blending).

Readings (the paper gives no formulas):
* a tile = a core of `core` x `core` pixels on a regular grid plus a halo of
  `halo` pixels on each side, so neighbouring tiles overlap by 2*halo;
* halo pixels outside the field are mirror-padded (index -i for i < 0,
  2(n-1) - i for i >= n; no edge repetition);
* the blend weight of a tile pixel is the separable product of 1D linear
  ramps w(u) = min(1, (u + 1/2) / (2 halo), (E - u - 1/2) / (2 halo)), E the
  tile extent - the distance-to-edge weight of a rectangle taken per axis;
* field = sum_t w_t tile_t / sum_t w_t over the tiles covering each pixel.
All z planes are carried through unchanged (tiling is transverse).
"""
from __future__ import annotations

import numpy as np


def mirror(i: np.ndarray, n: int) -> np.ndarray:
    """Reflect indices into [0, n): -i for i < 0, 2(n-1) - i for i >= n."""
    i = np.where(i < 0, -i, i)
    return np.where(i >= n, 2 * (n - 1) - i, i)


def tile_origin(ty: int, tx: int, core: int, halo: int):
    """Field coordinates of a tile's first pixel (may be negative)."""
    return ty * core - halo, tx * core - halo


def gather(field: np.ndarray, tiles_y: int, tiles_x: int, core: int, halo: int) -> np.ndarray:
    """Cut (Z, Yf, Xf) into tiles (tiles_y*tiles_x, Z, E, E), row-major tile order."""
    Z, Yf, Xf = field.shape
    E = core + 2 * halo
    out = np.empty((tiles_y * tiles_x, Z, E, E), dtype=field.dtype)
    for ty in range(tiles_y):
        for tx in range(tiles_x):
            y0, x0 = tile_origin(ty, tx, core, halo)
            ys = mirror(np.arange(y0, y0 + E), Yf)
            xs = mirror(np.arange(x0, x0 + E), Xf)
            out[ty * tiles_x + tx] = field[:, ys][:, :, xs]
    return out


def ramp(E: int, halo: int) -> np.ndarray:
    """1D blend weight of a tile axis of extent E with overlap 2*halo."""
    u = np.arange(E) + 0.5
    w = np.minimum(np.minimum(1.0, u / (2 * halo)), (E - u) / (2 * halo))
    return w


def blend(tiles: np.ndarray, tiles_y: int, tiles_x: int, core: int, halo: int) -> np.ndarray:
    """Stitch tiles (T, Z, E, E) into the field (Z, tiles_y*core, tiles_x*core)."""
    T, Z, E, _ = tiles.shape
    Yf, Xf = tiles_y * core, tiles_x * core
    acc = np.zeros((Z, Yf, Xf))
    wsum = np.zeros((Yf, Xf))
    w1 = ramp(E, halo)
    w2 = np.outer(w1, w1)
    for ty in range(tiles_y):
        for tx in range(tiles_x):
            y0, x0 = tile_origin(ty, tx, core, halo)
            ya, yb = max(y0, 0), min(y0 + E, Yf)
            xa, xb = max(x0, 0), min(x0 + E, Xf)
            wt = w2[ya - y0: yb - y0, xa - x0: xb - x0]
            acc[:, ya:yb, xa:xb] += wt[None] * tiles[ty * tiles_x + tx][:, ya - y0: yb - y0, xa - x0: xb - x0]
            wsum[ya:yb, xa:xb] += wt
    return acc / wsum[None]


# ------------------------------------------------------------------ padding
PAD_MODES = ("zero", "mirror", "edge")


def pad_index(i: np.ndarray, n: int, mode: str) -> np.ndarray:
    """Source index of position i of an axis of length n padded on both sides
    (-1: a zero).  mirror: reflection about the edge samples, -i and
    2(n-1) - i, repeated with period 2(n-1); edge: the nearest sample."""
    i = np.asarray(i)
    inside = (i >= 0) & (i < n)
    if mode == "zero":
        return np.where(inside, i, -1)
    if mode == "edge":
        return np.clip(i, 0, n - 1)
    if n == 1:
        return np.zeros_like(i)
    p = 2 * (n - 1)
    r = np.mod(i, p)
    return np.where(r < n, r, p - r)


def pad(vol: np.ndarray, shape_p, mode: str) -> np.ndarray:
    """(..., Z, Y, X) -> (..., Zp, Yp, Xp): the input at offset ((Zp-Z)//2,
    (Yp-Y)//2, (Xp-X)//2), the margin filled per ``mode`` (padding in place
    of circular boundaries)."""
    out = np.asarray(vol)
    for ax, n_p in zip((-3, -2, -1), shape_p):
        n = out.shape[ax]
        idx = pad_index(np.arange(n_p) - (n_p - n) // 2, n, mode)
        taken = np.take(out, np.maximum(idx, 0), axis=ax)
        mask_shape = [1] * out.ndim
        mask_shape[ax] = n_p
        out = np.where((idx >= 0).reshape(mask_shape), taken, 0.0)
    return out


def crop(vol: np.ndarray, shape) -> np.ndarray:
    """The window of ``shape`` at the offset ``pad`` uses."""
    Zp, Yp, Xp = vol.shape[-3:]
    Z, Y, X = shape
    oz, oy, ox = (Zp - Z) // 2, (Yp - Y) // 2, (Xp - X) // 2
    return vol[..., oz:oz + Z, oy:oy + Y, ox:ox + X]
