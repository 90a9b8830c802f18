"""Forward model, adjoint and Tikhonov reconstruction, float64 (test infrastructure).

* Forward (Eq. fwd, Eq. fwd_block and its shift-invariant Fourier form):
  D_c(nu) = sum_p H_cp(nu) F_p(nu) + b_c delta(nu), i.e.
  d_c = IFFT3(sum_p H_cp FFT3(f_p)) + b_c with circular boundaries.
* Adjoint: f_p = IFFT3(sum_c conj(H_cp) FFT3(d_c - b_c)).
* Reconstruction (Eq. recon, "Reconstructing object properties"): for each
  contrast mode m the minimiser of ||d - b - H f||^2 + eta ||f||^2.  For a
  shift-invariant H this is, frequency by frequency, the P x P normal
  equations (H^H H + eta I) F = H^H D~ - the plain definition of the
  minimiser; Eq. tls_solution (the SVD form) is the same operator and is
  checked against it in the pins.

Readings where the paper is silent:
* eta is relative by default: eta_abs = eta * max_nu sum_{c,p} |H_cp(nu)|^2,
  computed per contrast mode ("we choose a different regularization parameter
  for each contrast mode"); ``relative=False`` takes eta as absolute.
* The background b_c is given, or defaults to the channel mean; the DC bin of
  the residual is D_c(0) - N b_c.
* 2D phase-from-defocus (Methods, "Cell-scale optical pooled screen data";
  Ext. Data Fig. 3d): a thin object at the reference plane seen through the
  per-plane 2D TFs H_j; per transverse frequency the stack of planes is a
  multi-channel system, F = (sum_j H_j^H H_j + eta I)^-1 sum_j H_j^H D_j, with
  eta_abs = eta * max_nu sum_j sum_{c,p} |H_cp,j|^2.

Systems are described as a list of contrast modes; each mode is a dict with
``channels`` (indices into d), ``props`` (indices into f) and ``H`` (a
nested list H[c][p] of arrays, all of one shape).
"""
from __future__ import annotations

import numpy as np


def widefield_system(tfs: dict, kinds) -> tuple[list, list, list]:
    """The label-free + fluorescence system of the widefield workloads.

    Properties, in order: index increment (phase), extinction index
    (absorption), fluorophore density - those present in ``kinds``.
    Channels: a brightfield stack if any label-free kind is present, then a
    fluorescence stack if 'fluor' is.  Two contrast modes (block-diagonal,
    Eq. fwd_block): label-free C = 1 x P <= 2, fluorescence 1 x 1.
    Returns (modes, property_names, channel_names).
    """
    props = [k for k in ("phase", "absorption", "fluor") if k in kinds]
    lf = [k for k in ("phase", "absorption") if k in kinds]
    channels = []
    modes = []
    if lf:
        channels.append("brightfield")
        modes.append(dict(channels=[0], props=[props.index(k) for k in lf],
                          H=[[tfs[k] for k in lf]]))
    if "fluor" in kinds:
        channels.append("fluorescence")
        modes.append(dict(channels=[len(channels) - 1], props=[props.index("fluor")],
                          H=[[tfs["fluor"]]]))
    return modes, props, channels


def _fftn(x):
    return np.fft.fftn(x)


def _ifftn(X):
    return np.fft.ifftn(X)


def forward(modes, f: np.ndarray, background) -> np.ndarray:
    """d_c = IFFT3(sum_p H_cp FFT3(f_p)) + b_c, for every channel of every mode."""
    n_ch = 1 + max(c for m in modes for c in m["channels"])
    F = [_fftn(fp) for fp in f]
    d = np.zeros((n_ch,) + f.shape[1:])
    for m in modes:
        for ci, c in enumerate(m["channels"]):
            D = np.zeros(f.shape[1:], dtype=np.complex128)
            for pi, p in enumerate(m["props"]):
                D += m["H"][ci][pi] * F[p]
            d[c] = np.real(_ifftn(D)) + background[c]
    return d


def adjoint(modes, d: np.ndarray, background) -> np.ndarray:
    """f_p = IFFT3(sum_c conj(H_cp) FFT3(d_c - b_c))."""
    n_p = 1 + max(p for m in modes for p in m["props"])
    f = np.zeros((n_p,) + d.shape[1:])
    for m in modes:
        Dc = [_fftn(d[c] - background[c]) for c in m["channels"]]
        for pi, p in enumerate(m["props"]):
            F = np.zeros(d.shape[1:], dtype=np.complex128)
            for ci in range(len(m["channels"])):
                F += np.conj(m["H"][ci][pi]) * Dc[ci]
            f[p] = np.real(_ifftn(F))
    return f


def residual_spectrum(d_c: np.ndarray, b_c, axes) -> np.ndarray:
    """FFT of one channel with the background removed from the DC bin:
    D~(0) = D(0) - N b, b defaulting to the channel mean."""
    D = np.fft.fftn(d_c, axes=axes)
    n = int(np.prod([d_c.shape[a] for a in axes]))
    b = float(np.mean(d_c)) if b_c is None else float(b_c)
    transformed = {a % d_c.ndim for a in axes}
    idx = tuple(0 if a in transformed else slice(None) for a in range(d_c.ndim))
    D[idx] = D[idx] - n * b
    return D


def eta_absolute(Hm, eta: float, relative: bool, sum_axes=()) -> float:
    """eta_abs = eta * max_nu sum_{c,p} |H_cp(nu)|^2 (relative) or eta (absolute).

    ``sum_axes`` are summed before the maximum (the plane axis in 2D mode).
    """
    if not relative:
        return float(eta)
    tot = sum(np.abs(Hcp) ** 2 for row in Hm for Hcp in row)
    if sum_axes:
        tot = np.sum(tot, axis=sum_axes)
    return float(eta) * float(np.max(tot))


def _normal_solve(Hm, Dm, eta_abs):
    """Per-frequency (H^H H + eta I) F = H^H D for stacked frequencies.

    Hm[c][p] and Dm[c] are arrays over the same frequency grid.
    """
    C = len(Hm)
    P = len(Hm[0])
    shape = Dm[0].shape
    M = np.zeros(shape + (P, P), dtype=np.complex128)
    r = np.zeros(shape + (P,), dtype=np.complex128)
    for p in range(P):
        for q in range(P):
            for c in range(C):
                M[..., p, q] += np.conj(Hm[c][p]) * Hm[c][q]
        M[..., p, p] += eta_abs
        for c in range(C):
            r[..., p] += np.conj(Hm[c][p]) * Dm[c]
    if P == 1:
        return [r[..., 0] / M[..., 0, 0]]
    F = np.linalg.solve(M, r[..., None])[..., 0]
    return [F[..., p] for p in range(P)]


def reconstruct(modes, d: np.ndarray, eta: float, background=None, relative=True) -> np.ndarray:
    """3D Tikhonov reconstruction of every property, mode by mode (Eq. recon).

    Returns f_hat (P_total, Z, Y, X) float64.  ``background`` is a per-channel
    sequence or None (channel means).
    """
    n_p = 1 + max(p for m in modes for p in m["props"])
    out = np.zeros((n_p,) + d.shape[1:])
    for m in modes:
        Dm = [residual_spectrum(d[c], None if background is None else background[c], (0, 1, 2))
              for c in m["channels"]]
        ea = eta_absolute(m["H"], eta, relative)
        F = _normal_solve(m["H"], Dm, ea)
        for pi, p in enumerate(m["props"]):
            out[p] = np.real(np.fft.ifftn(F[pi]))
    return out


def reconstruct_2d(plane_modes, d: np.ndarray, eta: float, background=None, relative=True) -> np.ndarray:
    """2D thin-object reconstruction from a z-stack through per-plane 2D TFs.

    ``plane_modes`` has the layout of ``modes`` with H[c][p] the per-plane 2D
    TF stacks (Z, Y, X).  Every plane of every channel acts as one channel of
    a multi-channel system at each transverse frequency.  Returns (P, Y, X).
    """
    n_p = 1 + max(p for m in plane_modes for p in m["props"])
    Z, Y, X = d.shape[1:]
    out = np.zeros((n_p, Y, X))
    for m in plane_modes:
        Hm, Dm = [], []
        for ci, c in enumerate(m["channels"]):
            Dc = residual_spectrum(d[c], None if background is None else background[c], (1, 2))
            for j in range(Z):
                Hm.append([Hcp[j] for Hcp in m["H"][ci]])
                Dm.append(Dc[j])
        if relative:
            tot = sum(np.sum(np.abs(Hcp) ** 2, axis=0) for row in m["H"] for Hcp in row)
            ea = float(eta) * float(np.max(tot))
        else:
            ea = float(eta)
        F = _normal_solve(Hm, Dm, ea)
        for pi, p in enumerate(m["props"]):
            out[p] = np.real(np.fft.ifft2(F[pi]))
    return out


# ------------------------------------------- single-frequency solver forms
def solve_normal(H: np.ndarray, D: np.ndarray, eta: float) -> np.ndarray:
    """(H^H H + eta I)^-1 H^H D for one frequency (H is C x P)."""
    P = H.shape[1]
    return np.linalg.solve(H.conj().T @ H + eta * np.eye(P), H.conj().T @ D)


def solve_pushthrough(H: np.ndarray, D: np.ndarray, eta: float) -> np.ndarray:
    """H^H (H H^H + eta I)^-1 D (push-through identity form)."""
    C = H.shape[0]
    return H.conj().T @ np.linalg.solve(H @ H.conj().T + eta * np.eye(C), D)


def solve_svd(H: np.ndarray, D: np.ndarray, eta: float) -> np.ndarray:
    """Eq. tls_solution: sum_i s_i / (s_i^2 + eta) v_i u_i^H D."""
    U, s, Vh = np.linalg.svd(H, full_matrices=False)
    return (Vh.conj().T * (s / (s * s + eta))) @ (U.conj().T @ D)


def solve_lstsq(H: np.ndarray, D: np.ndarray, eta: float) -> np.ndarray:
    """Least squares on the stacked system [H; sqrt(eta) I] f = [D; 0]."""
    P = H.shape[1]
    A = np.vstack([H, np.sqrt(eta) * np.eye(P)])
    b = np.concatenate([D, np.zeros(P)])
    return np.linalg.lstsq(A, b, rcond=None)[0]
