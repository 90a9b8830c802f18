"""Auto-tuning objective for the per-tile defocus, float64 (test infrastructure).

The paper auto-tunes each tile's parameter vector theta by back-propagating a
scalar loss through the transfer-function build and the Tikhonov
reconstruction of a phase-from-defocus model (Results, "Physics-guided ML
auto-tunes multi-contrast blind deconvolution"; Fig. 2a(iv); Ext. Data
Fig. 3; Methods, "Cell-scale optical pooled screen data": 2D phase from a
z-stack, Adam, eta fixed at 1e-2).

Reading used here (a data-fidelity loss): for the 2D thin-object model (every
plane j of the stack sees the per-plane TF H_j of the object at the reference
plane), the Tikhonov objective at its minimiser,

    L(theta) = min_f ||d - b - H_theta f||^2 + eta ||f||^2
             = ||d - b - H_theta f_hat||^2 + eta ||f_hat||^2,

with a fixed absolute eta, the channel mean as background and theta the
tile's defocus z_offset.  (For the 3D model the same loss does not identify
the defocus: with one free unknown per 3D frequency the fit is exact wherever
H != 0.)  ``objective`` evaluates the definition - reconstruct, predict,
form the residual in real space.  ``gradient_fd`` is its central finite
difference.  ``tf_defocus_derivative`` is dH/d(defocus) of the 3D phase TF.
``midband_objective`` is the paper's own image-quality loss (minus the
mid-band power of the reconstruction), for comparison.
"""
from __future__ import annotations

import numpy as np

from . import model, optics


def band_limit(o: dict, d: np.ndarray, nu_max: float) -> np.ndarray:
    """The stack with every plane's transverse frequencies |nu| > nu_max
    (cycles/um) removed (an ideal low-pass; the mean is kept)."""
    Z, Y, X = d.shape
    ky, kx = optics.transverse_grid(Y, X, o["pixel_um"])
    keep = ky ** 2 + kx ** 2 <= float(nu_max) ** 2
    return np.real(np.fft.ifft2(np.fft.fft2(np.asarray(d, dtype=np.float64), axes=(1, 2)) * keep, axes=(1, 2)))


def objective(o: dict, d: np.ndarray, eta: float, nu_max: float | None = None) -> float:
    """L(theta) for one tile; d is the (Z, Y, X) brightfield stack.  With
    nu_max, the loss of the band-limited stack (``band_limit``)."""
    shape = d.shape
    Hj = optics.plane_tfs(o, shape, ("phase",))["phase"]
    modes = [dict(channels=[0], props=[0], H=[[Hj]])]
    dd = np.asarray(d, dtype=np.float64)[None]
    if nu_max is not None:
        dd = band_limit(o, dd[0], nu_max)[None]
    f_hat = model.reconstruct_2d(modes, dd, eta, background=None, relative=False)[0]
    b = float(np.mean(dd[0]))
    pred = np.real(np.fft.ifft2(Hj * np.fft.fft2(f_hat)[None], axes=(1, 2))) + b
    r = dd[0] - pred
    return float(np.sum(r * r) + eta * np.sum(f_hat * f_hat))


def midband_mask(o: dict, Y: int, X: int) -> np.ndarray:
    """Transverse frequencies with c/8 <= |nu| <= c/4, c = (NA_det + NA_ill)/lambda
    (the transverse cutoff of the label-free transfer functions)."""
    ky, kx = optics.transverse_grid(Y, X, o["pixel_um"])
    r = np.sqrt(ky * ky + kx * kx)
    c = (o["na_det"] + o["na_ill"]) / o["lambda_um"]
    return (r >= c / 8) & (r <= c / 4)


def midband_objective(o: dict, d: np.ndarray, eta: float) -> float:
    """The paper's image-quality loss (Results, auto-tuning; Methods, optical
    pooled screen data): minus the power of the 2D phase reconstruction in the
    mid band of transverse frequencies, read as sum |F|^2 / N_perp over
    c/8 <= |nu| <= c/4.  Evaluated by its definition: reconstruct (absolute
    eta, channel-mean background), transform, sum the band."""
    shape = d.shape
    Hj = optics.plane_tfs(o, shape, ("phase",))["phase"]
    modes = [dict(channels=[0], props=[0], H=[[Hj]])]
    f_hat = model.reconstruct_2d(modes, np.asarray(d, dtype=np.float64)[None], eta, background=None,
                                 relative=False)[0]
    F = np.fft.fft2(f_hat)
    m = midband_mask(o, shape[1], shape[2])
    return float(-np.sum(np.abs(F[m]) ** 2) / (shape[1] * shape[2]))


def midband_objective_at(o: dict, d: np.ndarray, eta: float, defocus: float) -> float:
    return midband_objective(dict(o, defocus_um=float(defocus)), d, eta)


def midband_gradient_fd(o: dict, d: np.ndarray, eta: float, h: float = 1e-4) -> float:
    z = o["defocus_um"]
    return (midband_objective_at(o, d, eta, z + h) - midband_objective_at(o, d, eta, z - h)) / (2 * h)


def objective_at(o: dict, d: np.ndarray, eta: float, defocus: float, nu_max: float | None = None) -> float:
    return objective(dict(o, defocus_um=float(defocus)), d, eta, nu_max)


def gradient_fd(o: dict, d: np.ndarray, eta: float, h: float = 1e-4, nu_max: float | None = None) -> float:
    """dL/d(defocus) by a central difference of the objective."""
    z = o["defocus_um"]
    return (objective_at(o, d, eta, z + h, nu_max) - objective_at(o, d, eta, z - h, nu_max)) / (2 * h)


def plane_tf_defocus_derivative(o: dict, shape) -> np.ndarray:
    """dH_phase,j/d(defocus) of the per-plane 2D phase TFs (complex128, (Z, Y, X)).

    The defocus enters both arms through e^{i2pi eta z_j}, so
    d/dz [sum_nu A*(nu) B(nu+q)] = sum_nu A*(nu) B'(nu+q) + sum_nu A'*(nu) B(nu+q)
    with A' = i 2 pi eta A and B' = i 2 pi eta B; Table 1's combination is
    linear and carries over unchanged.
    """
    Z, Y, X = shape
    A, B = optics.arms(o, shape)
    eta = optics.axial_frequency(o, Y, X)[None]
    Ad, Bd = 2j * np.pi * eta * A, 2j * np.pi * eta * B
    S = optics.source_pupil(o, Y, X)
    P = optics.detection_pupil(o, Y, X)
    c = optics.labelfree_prefactor(o) / np.sum(S * P * P)
    dH1 = c * (optics.correlate(A, Bd) + optics.correlate(Ad, B))
    dH2 = np.conj(optics.reflect(dH1))
    T = optics.TABLE1_LABELFREE
    return T[0, 0] * dH1 + T[0, 1] * dH2


def tf_defocus_derivative(o: dict, shape) -> np.ndarray:
    """dH_phase/d(defocus) of the 3D phase TF: the z-DFT of the per-plane derivative."""
    return optics.stack_to_3d(plane_tf_defocus_derivative(o, shape))


def plane_tf_source_derivatives(o: dict, shape) -> dict:
    """d H_phase,j / d theta of the per-plane 2D phase TFs for theta = tilt_x,
    tilt_y, NA_ill under the smooth source pupil (complex128, (Z, Y, X) each).

    Only the direct arm A = S P e^{i2pi eta z_j} and the normalisation
    D = sum S P^2 depend on the source, so with A_theta = (dS/dtheta) P e^{...}
    and D_theta = sum (dS/dtheta) P^2:
    dH1/dtheta = c [sum A_theta* B(.+q)] / D - H1 D_theta / D,
    and Table 1's combination carries over.
    """
    assert o.get("smooth_source", False), "the derivatives exist for the smooth source pupil"
    Z, Y, X = shape
    A, B = optics.arms(o, shape)
    S = optics.source_pupil(o, Y, X)
    P = optics.detection_pupil(o, Y, X)
    eta = optics.axial_frequency(o, Y, X)
    z = optics.plane_displacements(Z, o["z_step_um"], o["defocus_um"])
    prop = np.exp(2j * np.pi * eta[None] * z[:, None, None])
    D = np.sum(S * P * P)
    c = optics.labelfree_prefactor(o)
    H1 = c * optics.correlate(A, B) / D
    T = optics.TABLE1_LABELFREE
    out = {}
    for k, dS in optics.source_pupil_derivatives(o, Y, X).items():
        At = (dS * optics.detection_pupil_complex(o, Y, X))[None] * prop
        Dt = np.sum(dS * P * P)
        dH1 = c * optics.correlate(At, B) / D - H1 * Dt / D
        out[k] = T[0, 0] * dH1 + T[0, 1] * np.conj(optics.reflect(dH1))
    return out


PARAMS = ("defocus_um", "tilt_x", "tilt_y", "na_ill")


def gradient_fd_params(o: dict, d: np.ndarray, eta: float, h: float = 1e-4, loss: str = "data") -> np.ndarray:
    """dL/d(defocus, tilt_x, tilt_y, NA_ill) by central differences of the
    objective (data-fidelity or mid-band)."""
    f = objective if loss == "data" else midband_objective
    g = np.zeros(len(PARAMS))
    for i, k in enumerate(PARAMS):
        g[i] = (f(dict(o, **{k: o[k] + h}), d, eta) - f(dict(o, **{k: o[k] - h}), d, eta)) / (2 * h)
    return g
