"""Learned optics estimator, float64 reference (test infrastructure).

A small convolutional network maps features of a tile's spectra to its four
optics parameters (defocus, tilt_x, tilt_y, NA_ill), as the starting point of
auto-tuning.  The paper has no such estimator; the workload asks for one.
This module is the plain definition of what the library's kernels compute:

Features (``tile_features``), a 3 x 64 x 64 image per tile, from the per-plane
2D spectra D_j of the brightfield stack (mean removed), planes in natural
order (rows, padded to 64) and 64 radial bins of |nu| up to 2 NA_det/lambda
(columns):
  ch0[r, b] = log(1 + P[r, b] / mean(P)),  P[r, b] = sum_{nu in bin b} |D_r(nu)|^2
  ch1[r, b] = sum Im(D_{r+1} conj(D_r)) nu_x/|nu| / sum |D_{r+1}| |D_r|
  ch2[r, b] = the same with nu_y
The per-plane power profile locates the in-focus plane (the defocus, with its
sign, from the plane order) and its width; the cross-plane phase asymmetry
is the lateral image drift with defocus that oblique illumination causes.
A z-averaged magnitude spectrum cannot carry the defocus sign, which is why
per-plane statistics are used.

Network (``forward``): four 3x3 convolutions (3->32 stride 1, 32->64, 64->96,
96->128 stride 2, zero padding 1, ReLU), a global average pool and a linear
layer to 4 outputs.  Weights are rounded to bfloat16 before use (the
library stores them so), sums are float64 here.  ``backward`` is the
gradient of the mean squared error by the chain rule; ``adam`` one Adam step
on float32 master weights.
"""
from __future__ import annotations

import numpy as np

LAYERS = ((3, 32, 1), (32, 64, 2), (64, 96, 2), (96, 128, 2))  # (in, out, stride)
N_OUT = 4
SIDE = 64


def param_shapes():
    shapes = []
    for ci, co, _ in LAYERS:
        shapes += [(co, ci, 3, 3), (co,)]
    shapes += [(N_OUT, LAYERS[-1][1]), (N_OUT,)]
    return shapes


def n_params() -> int:
    return int(sum(np.prod(s) for s in param_shapes()))


def unpack(flat: np.ndarray):
    out, i = [], 0
    for s in param_shapes():
        k = int(np.prod(s))
        out.append(flat[i:i + k].reshape(s))
        i += k
    return out


def bf16(x: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), as float64."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


# ------------------------------------------------------------------ features
def natural_plane(r: int, Z: int) -> int:
    """Storage index (FFT order) of the plane in natural row r."""
    return (r - Z // 2) % Z


def tile_features(d: np.ndarray, o: dict) -> np.ndarray:
    """(3, 64, 64) features of a brightfield stack d (Z, Y, X), Z <= 64."""
    Z, Y, X = d.shape
    D = np.fft.fft2(np.asarray(d, dtype=np.float64) - np.mean(d), axes=(1, 2))
    fy = np.fft.fftfreq(Y, o["pixel_um"])[:, None] * np.ones((1, X))
    fx = np.fft.fftfreq(X, o["pixel_um"])[None, :] * np.ones((Y, 1))
    r = np.sqrt(fx * fx + fy * fy)
    cut = 2.0 * o["na_det"] / o["lambda_um"]
    b = np.floor(r / cut * SIDE).astype(int)
    ok = b < SIDE
    ux = np.where(r > 0, fx / np.where(r > 0, r, 1.0), 0.0)
    uy = np.where(r > 0, fy / np.where(r > 0, r, 1.0), 0.0)
    f = np.zeros((3, SIDE, SIDE))
    P = np.zeros((SIDE, SIDE))
    for row in range(Z):
        Dr = D[natural_plane(row, Z)]
        P[row] = np.bincount(b[ok], weights=np.abs(Dr[ok]) ** 2, minlength=SIDE)
        if row + 1 < Z:
            Dn = D[natural_plane(row + 1, Z)]
            C = Dn * np.conj(Dr)
            den = np.bincount(b[ok], weights=(np.abs(Dn) * np.abs(Dr))[ok], minlength=SIDE)
            sx = np.bincount(b[ok], weights=(np.imag(C) * ux)[ok], minlength=SIDE)
            sy = np.bincount(b[ok], weights=(np.imag(C) * uy)[ok], minlength=SIDE)
            f[1, row] = np.where(den > 0, sx / np.where(den > 0, den, 1.0), 0.0)
            f[2, row] = np.where(den > 0, sy / np.where(den > 0, den, 1.0), 0.0)
    m = P[:Z].mean()
    f[0, :Z] = np.log1p(P[:Z] / m) if m > 0 else 0.0
    return f


# ------------------------------------------------------------------ network
def _conv(x, w, bias, stride):
    """x (B, Ci, H, W), w (Co, Ci, 3, 3): zero-padded 3x3 cross-correlation."""
    B, Ci, H, W = x.shape
    Co = w.shape[0]
    Ho, Wo = (H + stride - 1) // stride, (W + stride - 1) // stride
    xp = np.zeros((B, Ci, H + 2, W + 2))
    xp[:, :, 1:-1, 1:-1] = x
    y = np.zeros((B, Co, Ho, Wo)) + bias[None, :, None, None]
    for kh in range(3):
        for kw in range(3):
            patch = xp[:, :, kh:kh + stride * Ho:stride, kw:kw + stride * Wo:stride]
            y += np.einsum("bchw,oc->bohw", patch, w[:, :, kh, kw])
    return y


def forward(flat: np.ndarray, x: np.ndarray):
    """Outputs (B, 4) and the activations (for ``backward``)."""
    p = [bf16(q) if q.ndim > 1 else np.asarray(q, dtype=np.float64) for q in unpack(flat)]
    acts = [np.asarray(x, dtype=np.float64)]
    h = acts[0]
    for li, (_, _, s) in enumerate(LAYERS):
        h = np.maximum(_conv(h, p[2 * li], p[2 * li + 1], s), 0.0)
        acts.append(h)
    pooled = h.mean(axis=(2, 3))
    acts.append(pooled)
    out = pooled @ p[-2].T + p[-1]
    return out, acts


def loss(flat, x, target) -> float:
    out, _ = forward(flat, x)
    return float(np.mean((out - target) ** 2))


def backward(flat: np.ndarray, x: np.ndarray, target: np.ndarray, masks=None):
    """Loss and d(mean squared error)/d(parameters), float64, flattened.

    ``masks`` (optional, one boolean array per convolution layer, the shape
    of its output) gives the ReLU decisions to differentiate through; by
    default they are this forward pass's (activation > 0).  A pre-activation
    within float rounding of zero can be decided either way, so a comparison
    with float32 kernels passes their decisions here."""
    p = [bf16(q) if q.ndim > 1 else np.asarray(q, dtype=np.float64) for q in unpack(flat)]
    out, acts = forward(flat, x)
    B = x.shape[0]
    g_out = 2.0 * (out - target) / (B * N_OUT)
    grads = [None] * len(p)
    pooled = acts[-1]
    grads[-2] = g_out.T @ pooled
    grads[-1] = g_out.sum(0)
    h = acts[-2]
    g = (g_out @ p[-2])[:, :, None, None] * np.ones_like(h) / (h.shape[2] * h.shape[3])
    for li in range(len(LAYERS) - 1, -1, -1):
        ci, co, s = LAYERS[li]
        g = g * ((acts[li + 1] > 0) if masks is None else masks[li])
        xin = acts[li]
        Bn, Ci, H, W = xin.shape
        Ho, Wo = g.shape[2], g.shape[3]
        xp = np.zeros((Bn, Ci, H + 2, W + 2))
        xp[:, :, 1:-1, 1:-1] = xin
        gw = np.zeros_like(p[2 * li])
        gxp = np.zeros_like(xp)
        for kh in range(3):
            for kw in range(3):
                sl = (slice(None), slice(None), slice(kh, kh + s * Ho, s), slice(kw, kw + s * Wo, s))
                gw[:, :, kh, kw] = np.einsum("bohw,bchw->oc", g, xp[sl])
                gxp[sl] += np.einsum("bohw,oc->bchw", g, p[2 * li][:, :, kh, kw])
        grads[2 * li] = gw
        grads[2 * li + 1] = g.sum(axis=(0, 2, 3))
        g = gxp[:, :, 1:-1, 1:-1]
    L = float(np.mean((out - target) ** 2))
    return L, np.concatenate([q.ravel() for q in grads])


def adam(w, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma and Ba, 2015) on float32 master weights; step
    is the 1-based step count.  Returns the new (w, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v
