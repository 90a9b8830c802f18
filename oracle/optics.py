"""Scalar weak-object transfer functions, float64 (test infrastructure).

Follows Methods, "Label-free and fluorescence contrast in a unified
framework", "Summary of transfer functions" and Table 1 (scalar column):

* label-free:   [H_re; H_im] = [[1, 1], [i, -i]] . [H1; H2], where H1 is the
  scatter-direct correlation of the detection pupil with the illuminated
  detection pupil and H2 its direct-scatter mirror;
* fluorescence: H_fl = [P * P], the autocorrelation of the detection pupil.

The Supplement that fixes the explicit pupil, Green's-function and
normalisation formulas is not available, so the following readings are used
(scalar first-Born scattering with the Weyl plane-wave expansion of the
Green's function, e^{ikr}/(4 pi r) = (i/4pi) Int d^2nu e^{i2pi(nu.r + eta|z|)}/eta):

* frequencies nu = k / (N p) in FFT order; k_m = n_medium / lambda;
  eta(nu) = sqrt(k_m^2 - |nu|^2) (axial frequency on the Ewald shell);
* source pupil S = 1[|nu - t/lambda| <= NA_ill/lambda] (closed disk, t the tilt
  in NA units), or with a logistic edge one frequency bin wide for tuning the
  illumination; detection pupil P = 1[|nu| <= NA_det/lambda], times
  e^{i 2 pi W} for an aberrated detection pupil (Ext. Data Fig. 3b), W the sum
  of Zernike polynomials in Noll's order and normalisation over the unit
  pupil rho = |nu| lambda / NA_det, coefficients in waves;
* the scattered arm carries the scalar Green's spectrum G = i/eta;
* plane j of a stack sits at focal displacement z_j = k_j dz + defocus with
  k_j in FFT order, and every arm is propagated by e^{+i 2 pi eta z_j};
* label-free prefactor c = 2 pi n_medium dz / lambda^2 for an object given as
  index increment (phase) and extinction index (absorption) per voxel, and
  the direct-direct background is normalised to 1 by dividing by sum(S P^2);
* the fluorescence TF is normalised to H_fl(0) = 1.

Pins: tests/test_oracle_pins.py (thin-slab closed form, Beer-Lambert,
Hermitian/parity symmetry, source-point field summation, PSF route).
"""
from __future__ import annotations

import numpy as np

KINDS = ("phase", "absorption", "fluor")


# --------------------------------------------------------------------- grids
def fft_indices(n: int) -> np.ndarray:
    """Signed integer frequency index of each FFT bin: 0..ceil(n/2)-1, then -floor(n/2)..-1."""
    k = np.arange(n)
    return np.where(k < (n + 1) // 2, k, k - n)


def frequency_axis(n: int, spacing: float) -> np.ndarray:
    """Spatial frequencies (cycles/um) of an n-point axis sampled every `spacing` um.

    Computed as k / (n * spacing) in float64 (the CUDA side evaluates the same
    expression so that pupil-edge decisions agree bit for bit).
    """
    return fft_indices(n).astype(np.float64) / (float(n) * spacing)


def transverse_grid(Y: int, X: int, pixel: float):
    nu_y = frequency_axis(Y, pixel)[:, None] * np.ones((1, X))
    nu_x = frequency_axis(X, pixel)[None, :] * np.ones((Y, 1))
    return nu_y, nu_x


def plane_displacements(Z: int, dz: float, defocus: float) -> np.ndarray:
    """Focal-plane displacement z_j of stack plane j relative to the object plane."""
    return fft_indices(Z).astype(np.float64) * dz + defocus


# -------------------------------------------------------------------- pupils
def _disk(nu_y, nu_x, cy, cx, radius):
    dy = nu_y - cy
    dx = nu_x - cx
    r2 = dx * dx + dy * dy
    return (r2 <= radius * radius).astype(np.float64)


def source_edge_width(o: dict, Y: int, X: int) -> float:
    """Edge width of the smooth source pupil: one frequency bin of the coarser axis."""
    return 1.0 / (min(Y, X) * o["pixel_um"])


def source_pupil(o: dict, Y: int, X: int) -> np.ndarray:
    """Illumination model S (Methods, "Summary of transfer functions", item 1).

    Binary disk of radius NA_ill/lambda centred on the tilt (tilt_x, tilt_y)/lambda.
    With o["smooth_source"] the edge is a logistic ramp instead,
    S = 1 / (1 + exp(-(R - |nu - t/lambda|) / w)), w = ``source_edge_width``:
    the model in which the tilt and NA_ill have derivatives (auto-tuning of
    the illumination parameters).
    """
    lam = o["lambda_um"]
    nu_y, nu_x = transverse_grid(Y, X, o["pixel_um"])
    if not o.get("smooth_source", False):
        return _disk(nu_y, nu_x, o["tilt_y"] / lam, o["tilt_x"] / lam, o["na_ill"] / lam)
    d = np.sqrt((nu_x - o["tilt_x"] / lam) ** 2 + (nu_y - o["tilt_y"] / lam) ** 2)
    w = source_edge_width(o, Y, X)
    return 1.0 / (1.0 + np.exp(-(o["na_ill"] / lam - d) / w))


def source_pupil_derivatives(o: dict, Y: int, X: int) -> dict:
    """dS/d(tilt_x), dS/d(tilt_y), dS/d(NA_ill) of the smooth source pupil
    (the chain rule through the logistic edge; zero at the disk centre for
    the tilts by symmetry)."""
    lam = o["lambda_um"]
    nu_y, nu_x = transverse_grid(Y, X, o["pixel_um"])
    ux, uy = nu_x - o["tilt_x"] / lam, nu_y - o["tilt_y"] / lam
    d = np.sqrt(ux * ux + uy * uy)
    w = source_edge_width(o, Y, X)
    S = 1.0 / (1.0 + np.exp(-(o["na_ill"] / lam - d) / w))
    ds = S * (1.0 - S) / w  # dS/dx times dx/d(R - d)
    safe = np.where(d > 0, d, 1.0)
    return {"tilt_x": np.where(d > 0, ds * ux / (safe * lam), 0.0),
            "tilt_y": np.where(d > 0, ds * uy / (safe * lam), 0.0),
            "na_ill": ds / lam}


def detection_pupil(o: dict, Y: int, X: int) -> np.ndarray:
    """Detection model P (item 3): binary disk of radius NA_det/lambda."""
    lam = o["lambda_um"]
    nu_y, nu_x = transverse_grid(Y, X, o["pixel_um"])
    return _disk(nu_y, nu_x, 0.0, 0.0, o["na_det"] / lam)


def noll_nm(j: int):
    """Radial order n and signed azimuthal order m of Noll's index j >= 1.

    Orders are taken n = 0, 1, 2, ... and within an order |m| increasing; an
    |m| > 0 takes two consecutive indices, the even one for cos(|m| phi)
    (m > 0) and the odd one for sin(|m| phi) (m < 0).
    """
    if j < 1:
        raise ValueError("Noll indices start at 1")
    nxt = 1
    n = 0
    while True:
        for am in range(n % 2, n + 1, 2):
            idx = [nxt] if am == 0 else [nxt, nxt + 1]
            nxt += len(idx)
            for i in idx:
                if i == j:
                    return n, (0 if am == 0 else (am if i % 2 == 0 else -am))
        n += 1


def zernike_radial(n: int, am: int, rho):
    """R_n^|m|(rho) = sum_s (-1)^s (n-s)! / (s! ((n+|m|)/2-s)! ((n-|m|)/2-s)!) rho^(n-2s)."""
    from math import factorial
    rho = np.asarray(rho, dtype=np.float64)
    out = np.zeros_like(rho)
    for s_ in range((n - am) // 2 + 1):
        c = (-1) ** s_ * factorial(n - s_) / (factorial(s_) * factorial((n + am) // 2 - s_) *
                                               factorial((n - am) // 2 - s_))
        out = out + c * rho ** (n - 2 * s_)
    return out


def zernike(j: int, rho, phi):
    """Noll's Z_j(rho, phi) with unit RMS over the unit disk:
    sqrt(n+1) R_n^0 for m = 0, sqrt(2(n+1)) R_n^|m| cos(m phi) or sin(|m| phi)."""
    n, m = noll_nm(j)
    R = zernike_radial(n, abs(m), rho)
    if m == 0:
        return np.sqrt(n + 1.0) * R
    ang = np.cos(m * phi) if m > 0 else np.sin(-m * phi)
    return np.sqrt(2.0 * (n + 1.0)) * R * ang


def aberration_phase(o: dict, Y: int, X: int) -> np.ndarray:
    """W(nu) = sum_j c_j Z_j(|nu| lambda / NA_det, atan2(nu_y, nu_x)) in waves,
    c_j = o["zernike"][j - 1]; zero without coefficients and outside P."""
    coef = np.asarray(o.get("zernike", ()), dtype=np.float64)
    W = np.zeros((Y, X))
    if coef.size == 0:
        return W
    nu_y, nu_x = transverse_grid(Y, X, o["pixel_um"])
    rho = np.sqrt(nu_x * nu_x + nu_y * nu_y) * o["lambda_um"] / o["na_det"]
    phi = np.arctan2(nu_y, nu_x)
    for j, c in enumerate(coef, start=1):
        if c != 0.0:
            W += c * zernike(j, rho, phi)
    return W * detection_pupil(o, Y, X)


def detection_pupil_complex(o: dict, Y: int, X: int) -> np.ndarray:
    """The (possibly aberrated) detection pupil P e^{i 2 pi W} (complex128).
    |P e^{i 2 pi W}|^2 = P^2, so the normalisations keep the binary P."""
    return detection_pupil(o, Y, X) * np.exp(2j * np.pi * aberration_phase(o, Y, X))


def axial_frequency(o: dict, Y: int, X: int) -> np.ndarray:
    """eta(nu) = sqrt(k_m^2 - |nu|^2); set to 0 outside the shell (never used there)."""
    km = o["n_medium"] / o["lambda_um"]
    nu_y, nu_x = transverse_grid(Y, X, o["pixel_um"])
    return np.sqrt(np.maximum(km * km - (nu_x * nu_x + nu_y * nu_y), 0.0))


def pupil_boundary_ties(o: dict, Y: int, X: int, rel: float = 1e-9) -> int:
    """Number of grid points within `rel` (relative) of either pupil edge.

    Such points could flip between float32 and float64 predicates; both sides
    evaluate the predicate in float64, and this count lets a test assert that
    a configuration has none.
    """
    lam = o["lambda_um"]
    nu_y, nu_x = transverse_grid(Y, X, o["pixel_um"])
    n = 0
    for cy, cx, rad in ((o["tilt_y"] / lam, o["tilt_x"] / lam, o["na_ill"] / lam),
                        (0.0, 0.0, o["na_det"] / lam)):
        r2 = (nu_x - cx) ** 2 + (nu_y - cy) ** 2
        n += int(np.sum(np.abs(r2 - rad * rad) <= rel * max(rad * rad, 1e-300)))
    return n


# ---------------------------------------------------------------------- arms
def arms(o: dict, shape):
    """Defocused direct arm A_j = S P e^{i2pi eta z_j} and scattered arm
    B_j = P (i/eta) e^{i2pi eta z_j} for every plane j (complex128, (Z, Y, X))."""
    Z, Y, X = shape
    S = source_pupil(o, Y, X)
    P = detection_pupil(o, Y, X)
    Pc = detection_pupil_complex(o, Y, X)
    eta = axial_frequency(o, Y, X)
    z = plane_displacements(Z, o["z_step_um"], o["defocus_um"])
    prop = np.exp(2j * np.pi * eta[None, :, :] * z[:, None, None])
    inv_eta = np.where(P > 0, 1.0 / np.where(eta > 0, eta, 1.0), 0.0)
    A = (S * Pc)[None] * prop
    B = (Pc * 1j * inv_eta)[None] * prop
    return A, B


def fluor_arm(o: dict, shape):
    """Defocused detection pupil P_j = P e^{i2pi eta z_j} (complex128, (Z, Y, X))."""
    Z, Y, X = shape
    P = detection_pupil_complex(o, Y, X)
    eta = axial_frequency(o, Y, X)
    z = plane_displacements(Z, o["z_step_um"], o["defocus_um"])
    return P[None] * np.exp(2j * np.pi * eta[None, :, :] * z[:, None, None])


# ------------------------------------------------------------ correlations
def correlate(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Circular cross-correlation per plane: C(q) = sum_nu conj(A(nu)) B(nu + q).

    Evaluated with the correlation theorem, C = N * FFT2(conj(IFFT2 A) * IFFT2 B)
    (a library FFT as one step); pinned against ``correlate_direct``.
    """
    n = A.shape[-1] * A.shape[-2]
    a = np.fft.ifft2(A, axes=(-2, -1))
    b = np.fft.ifft2(B, axes=(-2, -1))
    return n * np.fft.fft2(np.conj(a) * b, axes=(-2, -1))


def correlate_direct(A: np.ndarray, B: np.ndarray, qy: int, qx: int) -> np.ndarray:
    """sum_nu conj(A(nu)) B(nu + q) for one integer shift q, every plane (definition)."""
    Bq = np.roll(B, shift=(-qy, -qx), axis=(-2, -1))  # Bq(nu) = B(nu + q)
    return np.sum(np.conj(A) * Bq, axis=(-2, -1))


def reflect(H: np.ndarray, axes=(-2, -1)) -> np.ndarray:
    """H(-nu) on an FFT-ordered grid: index k -> (-k) mod n along each axis."""
    out = H
    for ax in axes:
        n = H.shape[ax]
        out = np.take(out, (-np.arange(n)) % n, axis=ax)
    return out


def labelfree_prefactor(o: dict) -> float:
    """c = 2 pi n_medium dz / lambda^2 (first-Born potential of a dz-thick voxel slab)."""
    return 2.0 * np.pi * o["n_medium"] * o["z_step_um"] / o["lambda_um"] ** 2


TABLE1_LABELFREE = np.array([[1.0, 1.0], [1.0j, -1.0j]])  # Table 1, scalar label-free row


def labelfree_plane_tfs(o: dict, shape):
    """Per-plane 2D label-free TFs (H_re_j, H_im_j), each (Z, Y, X) complex128.

    H1_j(q) = c sum_nu A_j*(nu) B_j(nu+q) / sum(S P^2);  H2_j(q) = H1_j(-q)*;
    [H_re_j; H_im_j] = [[1, 1], [i, -i]] [H1_j; H2_j]   (Table 1, scalar).
    """
    Z, Y, X = shape
    A, B = arms(o, shape)
    S = source_pupil(o, Y, X)
    P = detection_pupil(o, Y, X)
    norm = np.sum(S * P * P)
    if norm <= 0:
        raise ValueError("illumination pupil does not overlap the detection pupil")
    H1 = labelfree_prefactor(o) * correlate(A, B) / norm
    H2 = np.conj(reflect(H1))
    Hre = TABLE1_LABELFREE[0, 0] * H1 + TABLE1_LABELFREE[0, 1] * H2
    Him = TABLE1_LABELFREE[1, 0] * H1 + TABLE1_LABELFREE[1, 1] * H2
    return Hre, Him


def fluor_plane_tfs(o: dict, shape) -> np.ndarray:
    """Per-plane 2D fluorescence TFs Hfl_j = [P_j * P_j] / (Z sum P^2) (Table 1, scalar).

    The constant makes the 3D TF equal 1 at zero frequency.
    """
    Z, Y, X = shape
    Pj = fluor_arm(o, shape)
    P = detection_pupil(o, Y, X)
    return correlate(Pj, Pj) / (Z * np.sum(P * P))


def stack_to_3d(Hj: np.ndarray) -> np.ndarray:
    """3D TF from per-plane 2D TFs: unnormalised DFT over the plane index j."""
    return np.fft.fft(Hj, axis=0)


def plane_tfs(o: dict, shape, kinds=KINDS) -> dict:
    """Per-plane 2D TFs for the requested kinds (used by the 2D reconstruction)."""
    out = {}
    if "phase" in kinds or "absorption" in kinds:
        Hre, Him = labelfree_plane_tfs(o, shape)
        if "phase" in kinds:
            out["phase"] = Hre
        if "absorption" in kinds:
            out["absorption"] = Him
    if "fluor" in kinds:
        out["fluor"] = fluor_plane_tfs(o, shape)
    return out


def transfer_functions(o: dict, shape, kinds=KINDS) -> dict:
    """3D TFs (full spectrum, complex128, (Z, Y, X)) for the requested kinds."""
    return {k: stack_to_3d(v) for k, v in plane_tfs(o, shape, kinds).items()}


def tf_at(o: dict, shape, kind: str, k3) -> complex:
    """One 3D TF value at integer frequency index (kz, ky, kx), from the definition.

    Uses ``correlate_direct`` per plane (O(Z Y X) work), so it serves as a
    sampled check of full-size transfer functions.
    """
    Z, Y, X = shape
    kz, ky, kx = (int(v) for v in k3)
    if kind == "fluor":
        Pj = fluor_arm(o, shape)
        P = detection_pupil(o, Y, X)
        Hj = correlate_direct(Pj, Pj, ky, kx) / (Z * np.sum(P * P))
    else:
        A, B = arms(o, shape)
        S = source_pupil(o, Y, X)
        P = detection_pupil(o, Y, X)
        c = labelfree_prefactor(o) / np.sum(S * P * P)
        H1 = c * correlate_direct(A, B, ky, kx)
        H2 = np.conj(c * correlate_direct(A, B, -ky, -kx))
        row = 0 if kind == "phase" else 1
        Hj = TABLE1_LABELFREE[row, 0] * H1 + TABLE1_LABELFREE[row, 1] * H2
    j = np.arange(Z)
    return complex(np.sum(Hj * np.exp(-2j * np.pi * kz * j / Z)))


def tf_samples(o: dict, shape, kind: str, ks) -> np.ndarray:
    """3D TF values at several integer frequencies, from the definition.

    Same sums as ``tf_at`` (direct per-plane correlations, then the DFT over
    planes) with the arms computed once; O(Z Y X) per frequency.
    """
    Z, Y, X = shape
    j = np.arange(Z)
    out = np.zeros(len(ks), dtype=np.complex128)
    if kind == "fluor":
        Pj = fluor_arm(o, shape)
        norm = Z * np.sum(detection_pupil(o, Y, X) ** 2)
        for i, (kz, ky, kx) in enumerate(ks):
            Hj = correlate_direct(Pj, Pj, int(ky), int(kx)) / norm
            out[i] = np.sum(Hj * np.exp(-2j * np.pi * int(kz) * j / Z))
        return out
    A, B = arms(o, shape)
    S = source_pupil(o, Y, X)
    P = detection_pupil(o, Y, X)
    c = labelfree_prefactor(o) / np.sum(S * P * P)
    row = 0 if kind == "phase" else 1
    for i, (kz, ky, kx) in enumerate(ks):
        H1 = c * correlate_direct(A, B, int(ky), int(kx))
        H2 = np.conj(c * correlate_direct(A, B, -int(ky), -int(kx)))
        Hj = TABLE1_LABELFREE[row, 0] * H1 + TABLE1_LABELFREE[row, 1] * H2
        out[i] = np.sum(Hj * np.exp(-2j * np.pi * int(kz) * j / Z))
    return out


def half_spectrum(H: np.ndarray) -> np.ndarray:
    """The non-redundant half (last axis 0..X/2) of a Hermitian spectrum."""
    return H[..., : H.shape[-1] // 2 + 1]
