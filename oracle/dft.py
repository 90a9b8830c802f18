"""Discrete Fourier transforms written from their definition (test infrastructure).

X[k] = sum_n x[n] exp(-2 pi i k.n / N)  (forward, unnormalised)
x[n] = (1/N) sum_k X[k] exp(+2 pi i k.n / N)  (inverse)

The Fourier form of the shift-invariant model (Methods, "Linear
contrast-separable shift-invariant imaging systems") is written with these
transforms.  ``bruteforce_dft`` evaluates the multi-dimensional sum directly
and is used to pin numpy.fft; ``dft_coefficient`` evaluates one coefficient of
a large volume without any FFT.
"""
from __future__ import annotations

import numpy as np


def bruteforce_dft(x: np.ndarray, inverse: bool = False) -> np.ndarray:
    """Full N-D DFT as an explicit sum over every (k, n) pair (O(N^2)).

    Only for tiny arrays (a few thousand elements).
    """
    x = np.asarray(x, dtype=np.complex128)
    shape = x.shape
    # Index vectors of every element, and the phase k.n/N summed over axes.
    grids = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    idx = np.stack([g.ravel() for g in grids], axis=1).astype(np.float64)  # (M, d)
    frac = np.zeros((idx.shape[0], idx.shape[0]))
    for ax, n in enumerate(shape):
        frac += np.outer(idx[:, ax], idx[:, ax]) / n
    sign = 1.0 if inverse else -1.0
    kernel = np.exp(sign * 2j * np.pi * frac)
    out = kernel @ x.ravel()
    if inverse:
        out /= x.size
    return out.reshape(shape)


def dft_coefficient(vol: np.ndarray, k) -> complex:
    """One coefficient X[k] of a 3D volume, from the definition.

    The triple sum is evaluated axis by axis (x, then y, then z), which is the
    same sum reordered; no FFT is used.  Cost O(volume) per coefficient.
    """
    vol = np.asarray(vol)
    Z, Y, X = vol.shape
    kz, ky, kx = (int(v) for v in k)
    ex = np.exp(-2j * np.pi * kx * np.arange(X) / X)
    ey = np.exp(-2j * np.pi * ky * np.arange(Y) / Y)
    ez = np.exp(-2j * np.pi * kz * np.arange(Z) / Z)
    s = vol.astype(np.float64) @ ex if not np.iscomplexobj(vol) else vol.astype(np.complex128) @ ex
    s = s @ ey
    return complex(s @ ez)
