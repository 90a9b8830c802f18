"""Pins that tie the FP64 oracle to the paper and to closed forms (CPU only).

Each test checks the oracle against something other than itself: a brute-force
definition, a textbook closed form, an identity of linear algebra, an
independent physical route, or a value printed in the paper.  A dropped term,
wrong sign, transposed operand or wrong index anywhere in ``oracle/`` should
fail at least one of them.
"""
import json
import os

import numpy as np
import pytest

import phantom as ph
from oracle import dft, model, optics as O, tiles
from conftest import rel_l2

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")


# ------------------------------------------------------------------ P1 FFT
@pytest.mark.parametrize("shape", [(8, 8, 8), (6, 10, 12)])
def test_numpy_fft_matches_bruteforce_dft(shape):
    x = np.random.default_rng(1).normal(size=shape) + 1j * np.random.default_rng(2).normal(size=shape)
    ref = dft.bruteforce_dft(x)
    assert np.abs(np.fft.fftn(x) - ref).max() <= 1e-12 * np.abs(ref).max()
    back = dft.bruteforce_dft(ref, inverse=True)
    assert np.abs(back - x).max() <= 1e-12
    # Parseval: sum |x|^2 = (1/N) sum |X|^2
    assert abs(np.sum(np.abs(x) ** 2) - np.sum(np.abs(ref) ** 2) / x.size) <= 1e-10 * np.sum(np.abs(x) ** 2)


def test_dft_coefficient_matches_bruteforce():
    x = np.random.default_rng(3).normal(size=(6, 10, 12))
    ref = dft.bruteforce_dft(x)
    for k in [(0, 0, 0), (1, 3, 5), (5, 9, 11), (3, 0, 7)]:
        assert abs(dft.dft_coefficient(x, k) - ref[k]) <= 1e-12 * np.abs(ref).max()


# ------------------------------------------------------------ pupils (a1)
def test_pupil_radius_and_tilt_on_grid():
    # pixel 0.1 um, X = Y = 40 -> grid step 1/(40*0.1) = 0.25 /um.  lambda = 0.5.
    o = ph.optics(lambda_um=0.5, pixel_um=0.1, na_det=0.375, na_ill=0.0, tilt_x=0.25, tilt_y=0.0)
    # Detection cutoff NA/lambda = 0.75 /um = exactly 3 grid steps (closed disk).
    P = O.detection_pupil(o, 40, 40)
    assert P[0, 3] == 1 and P[0, 4] == 0 and P[3, 0] == 1 and P[0, -3] == 1 and P[0, -4] == 0
    assert P[2, 2] == 1 and P[2, 3] == 0  # 2^2+2^2 = 8 <= 9 < 13
    # A point source tilted by tilt_x = 0.25 NA sits at nu_x = 0.25/0.5 = 0.5 /um = +2 steps.
    S = O.source_pupil(o, 40, 40)
    assert S.sum() == 1 and S[0, 2] == 1
    o2 = dict(o, tilt_x=0.0, tilt_y=-0.125)  # -1 step along y
    S2 = O.source_pupil(o2, 40, 40)
    assert S2.sum() == 1 and S2[-1, 0] == 1


def test_correlation_theorem_matches_direct_sum():
    A, B = O.arms(ph.optics(na_ill=0.6, tilt_x=0.05), (3, 16, 20))
    C = O.correlate(A, B)
    for qy, qx in [(0, 0), (1, 3), (-2, 5), (7, -9), (8, 10)]:
        assert np.abs(C[:, qy % 16, qx % 20] - O.correlate_direct(A, B, qy, qx)).max() <= 1e-12 * np.abs(C).max()


def test_table1_matrix_is_the_papers():
    g = json.load(open(GOLDEN))["table1_scalar_labelfree_matrix"]
    m = np.array(g["re"]) + 1j * np.array(g["im"])
    assert np.array_equal(O.TABLE1_LABELFREE, m)


# ----------------------------------------------- P2 thin slab closed forms
@pytest.mark.parametrize("defocus", [0.0, 0.37])
def test_thin_slab_born_closed_form(defocus):
    """On-axis point source, one-voxel slab: each plane's TF is
    -2 (c/eta) sin(2 pi z (eta - k_m)) P for index and -2 (c/eta) cos(...) P for
    absorption (textbook defocus CTF; k_m = n/lambda, c = 2 pi n dz / lambda^2)."""
    o = ph.optics(na_ill=0.0, defocus_um=defocus)
    shape = (8, 32, 32)
    Hre, Him = O.labelfree_plane_tfs(o, shape)
    lam, n, dz = o["lambda_um"], o["n_medium"], o["z_step_um"]
    km = n / lam
    c = 2 * np.pi * n * dz / lam ** 2
    ky = np.fft.fftfreq(32, d=o["pixel_um"])
    rho2 = ky[:, None] ** 2 + ky[None, :] ** 2
    inside = rho2 <= (o["na_det"] / lam) ** 2
    eta = np.sqrt(np.where(inside, km ** 2 - rho2, 1.0))
    z = np.array([0, 1, 2, 3, -4, -3, -2, -1]) * dz + defocus
    phase = 2 * np.pi * z[:, None, None] * (eta[None] - km)
    exp_re = np.where(inside, -2 * c / eta * np.sin(phase), 0.0)
    exp_im = np.where(inside, -2 * c / eta * np.cos(phase), 0.0)
    assert np.abs(Hre - exp_re).max() <= 1e-12 * np.abs(exp_im).max()
    assert np.abs(Him - exp_im).max() <= 1e-12 * np.abs(exp_im).max()
    # Beer-Lambert at zero frequency: transmitted intensity drops by 2 k0 kappa dz.
    k0 = 2 * np.pi / lam
    assert np.allclose(Him[:, 0, 0], -2 * k0 * dz, rtol=1e-13)
    # Phase of a uniform slab is invisible.
    assert np.abs(Hre[:, 0, 0]).max() <= 1e-12


def test_beer_lambert_oblique_partially_coherent():
    """A uniform absorbing slab under a tilted partially coherent source dims
    every plane by the source average of 2 k0 kappa dz / cos(theta_s), with
    cos(theta_s) = eta(s)/k_m (oblique rays cross the slab on a longer path)."""
    o = ph.optics(na_ill=0.7, tilt_x=0.08, tilt_y=-0.05, defocus_um=0.3)
    shape = (6, 24, 24)
    tfs = O.transfer_functions(o, shape, ("phase", "absorption"))
    modes, _, _ = model.widefield_system(tfs, ("phase", "absorption"))
    kappa = 1e-3
    f = np.zeros((2,) + shape)
    f[1, 2] = kappa  # one voxel-thick uniform slab in plane 2
    d = model.forward(modes, f, [0.0])[0]
    # closed form from the source points
    lam, n, dz = o["lambda_um"], o["n_medium"], o["z_step_um"]
    km, k0 = n / lam, 2 * np.pi / lam
    nu = np.fft.fftfreq(24, d=o["pixel_um"])
    vy, vx = nu[:, None] * np.ones((1, 24)), nu[None, :] * np.ones((24, 1))
    S = ((vx - 0.08 / lam) ** 2 + (vy + 0.05 / lam) ** 2) <= (0.7 / lam) ** 2
    P = (vx ** 2 + vy ** 2) <= (o["na_det"] / lam) ** 2
    src = S & P
    cos_t = np.sqrt(km ** 2 - vx[src] ** 2 - vy[src] ** 2) / km
    expected = -np.mean(2 * k0 * kappa * dz / cos_t)
    assert np.allclose(d, expected, rtol=1e-12, atol=0)
    # a uniform index slab changes nothing
    f2 = np.zeros((2,) + shape)
    f2[0, 1] = 0.01
    assert np.abs(model.forward(modes, f2, [0.0])[0]).max() <= 1e-14


# ------------------------------------------------------------ P3 symmetry
@pytest.mark.parametrize("tilt", [0.0, 0.07])
def test_parity_and_hermitian(tilt):
    """Odd Z, so that every plane j has its mirror -j: phase TF odd (purely
    imaginary), absorption TF even (real), fluorescence TF real, even, max at
    DC; all Hermitian (Methods, Summary of transfer functions)."""
    o = ph.optics(na_ill=0.5, tilt_x=tilt, tilt_y=-0.03)
    T = O.transfer_functions(o, (9, 32, 32))
    R = lambda H: O.reflect(H, axes=(0, 1, 2))
    for k, H in T.items():
        s = np.abs(H).max()
        assert np.abs(H - np.conj(R(H))).max() <= 1e-13 * s, k
    assert np.abs(T["phase"] + R(T["phase"])).max() <= 1e-13 * np.abs(T["phase"]).max()
    assert np.abs(T["phase"].real).max() <= 1e-13 * np.abs(T["phase"]).max()
    assert np.abs(T["absorption"] - R(T["absorption"])).max() <= 1e-13 * np.abs(T["absorption"]).max()
    assert np.abs(T["absorption"].imag).max() <= 1e-13 * np.abs(T["absorption"]).max()
    Hf = T["fluor"]
    assert np.abs(Hf.imag).max() <= 1e-13 and np.abs(Hf - R(Hf)).max() <= 1e-13
    assert abs(Hf[0, 0, 0] - 1.0) <= 1e-13 and np.abs(Hf).max() <= 1.0 + 1e-13


def test_hermitian_with_even_z_and_defocus():
    o = ph.optics(na_ill=0.8, tilt_x=-0.06, defocus_um=-0.6)
    T = O.transfer_functions(o, (8, 16, 24))
    for k, H in T.items():
        assert np.abs(H - np.conj(O.reflect(H, axes=(0, 1, 2)))).max() <= 1e-13 * np.abs(H).max(), k


# ----------------------------------------------- P4 independent routes
def _field_route(o, shape, m, dn_plane, kappa_plane, pupil=None):
    """First-Born fields per source point, summed incoherently.

    For each source point s (inside S and P) and data plane i the detector sees
    the direct plane wave u0 = e^{i2pi(s.r + eta(s) z)} and the scattered field
    us = IDFT2[P(nu) (i c / eta(nu)) e^{i2pi eta(nu) z} F(nu - s)], with z the
    displacement between focus and the object plane m, and F the 2D spectrum of
    dn + i kappa.  Label-free contrast is 2 Re(u0* us) summed over the source
    (Methods, unified framework), normalised by the direct background.
    ``pupil``: a complex detection pupil (an aberrated one) applied to both
    the direct wave, u0 -> pupil(s) u0, and the scattered field.
    """
    Z, Y, X = shape
    S = O.source_pupil(o, Y, X)
    P = O.detection_pupil(o, Y, X)
    Pc = P if pupil is None else pupil
    eta = O.axial_frequency(o, Y, X)
    inv_eta = np.where(P > 0, 1.0 / np.where(eta > 0, eta, 1.0), 0.0)
    z = O.plane_displacements(Z, o["z_step_um"], o["defocus_um"])
    c = 2 * np.pi * o["n_medium"] * o["z_step_um"] / o["lambda_um"] ** 2
    F = np.fft.fft2(dn_plane + 1j * kappa_plane)
    ky, kx = O.fft_indices(Y), O.fft_indices(X)
    yy, xx = np.meshgrid(np.arange(Y), np.arange(X), indexing="ij")
    out = np.zeros(shape)
    count = 0.0
    for sy, sx in zip(*np.nonzero(S * P)):
        wgt = S[sy, sx] * P[sy, sx]  # 1 for the binary source, the edge weight for the smooth one
        count += wgt
        Fs = np.roll(F, shift=(sy, sx), axis=(0, 1))  # F(nu - s)
        for i in range(Z):
            zi = z[(i - m) % Z]
            u0 = Pc[sy, sx] * np.exp(2j * np.pi * (ky[sy] * yy / Y + kx[sx] * xx / X + eta[sy, sx] * zi))
            us = np.fft.ifft2(Pc * 1j * c * inv_eta * np.exp(2j * np.pi * eta * zi) * Fs)
            out[i] += wgt * 2.0 * np.real(np.conj(u0) * us)
    return out / count


@pytest.mark.parametrize("m,na_ill,tilt_x", [(0, 0.55, 0.06), (2, 0.55, 0.06), (1, 1.15, 0.12)])
def test_labelfree_forward_equals_source_point_field_sum(m, na_ill, tilt_x):
    # the last case has source points outside the detection pupil (no direct light)
    o = ph.optics(na_ill=na_ill, tilt_x=tilt_x, tilt_y=0.02, defocus_um=0.2)
    shape = (5, 20, 24)
    rng = np.random.default_rng(7)
    dn = rng.normal(size=shape[1:]) * 1e-2
    kap = rng.normal(size=shape[1:]) * 1e-3
    tfs = O.transfer_functions(o, shape, ("phase", "absorption"))
    modes, _, _ = model.widefield_system(tfs, ("phase", "absorption"))
    f = np.zeros((2,) + shape)
    f[0, m] = dn
    f[1, m] = kap
    d = model.forward(modes, f, [1.0])[0] - 1.0
    ref = _field_route(o, shape, m, dn, kap)
    assert rel_l2(d, ref) <= 1e-12


def test_fluorescence_forward_of_point_is_psf():
    """Forward of a point emitter = |sum_nu P_j(nu) e^{i2pi nu.r}|^2 per plane,
    normalised to unit sum (explicit inverse-DFT matrices, no FFT)."""
    o = ph.optics(defocus_um=0.4)
    shape = (6, 16, 20)
    Z, Y, X = shape
    tfs = O.transfer_functions(o, shape, ("fluor",))
    modes, _, _ = model.widefield_system(tfs, ("fluor",))
    f = np.zeros((1,) + shape)
    f[0, 0, 0, 0] = 1.0
    d = model.forward(modes, f, [0.0])[0]
    P = O.detection_pupil(o, Y, X)
    eta = O.axial_frequency(o, Y, X)
    z = O.plane_displacements(Z, o["z_step_um"], o["defocus_um"])
    Ey = np.exp(2j * np.pi * np.outer(np.arange(Y), O.fft_indices(Y)) / Y)
    Ex = np.exp(2j * np.pi * np.outer(np.arange(X), O.fft_indices(X)) / X)
    psf = np.stack([np.abs(Ey @ (P * np.exp(2j * np.pi * eta * z[j])) @ Ex.T) ** 2 for j in range(Z)])
    psf /= psf.sum()
    assert rel_l2(d, psf) <= 1e-12


def test_tf_at_matches_full_build():
    o = ph.optics(na_ill=0.7, tilt_x=0.04, defocus_um=-0.3)
    shape = (6, 16, 20)
    T = O.transfer_functions(o, shape)
    for kind in O.KINDS:
        for k in [(0, 0, 0), (1, 2, 3), (5, 15, 19), (3, 8, 10), (2, 13, 4)]:
            assert abs(O.tf_at(o, shape, kind, k) - T[kind][k]) <= 1e-12 * np.abs(T[kind]).max()


def test_tf_samples_match_full_build():
    o = ph.optics(na_ill=0.8, tilt_y=-0.05, defocus_um=0.25)
    shape = (5, 12, 16)
    T = O.transfer_functions(o, shape)
    ks = [(0, 0, 0), (4, 11, 15), (2, 5, 3), (1, 0, 8)]
    for kind in O.KINDS:
        got = O.tf_samples(o, shape, kind, ks)
        ref = np.array([T[kind][k] for k in ks])
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(T[kind]).max()


# -------------------------------------------------- P5 linearity, adjoint
def test_adjoint_dot_product():
    o = ph.optics(na_ill=0.6, tilt_y=0.05)
    shape = (6, 12, 16)
    tfs = O.transfer_functions(o, shape)
    modes, props, chans = model.widefield_system(tfs, O.KINDS)
    rng = np.random.default_rng(11)
    f = rng.normal(size=(3,) + shape)
    d = rng.normal(size=(2,) + shape)
    b = [0.7, -0.2]
    Af = model.forward(modes, f, b) - np.array(b)[:, None, None, None]
    Ahd = model.adjoint(modes, d + np.array(b)[:, None, None, None], b)
    assert abs(np.vdot(Af, d) - np.vdot(f, Ahd)) <= 1e-12 * np.linalg.norm(Af) * np.linalg.norm(d)
    # linearity
    f2 = rng.normal(size=f.shape)
    lhs = model.forward(modes, 2 * f - 3 * f2, [0, 0])
    rhs = 2 * model.forward(modes, f, [0, 0]) - 3 * model.forward(modes, f2, [0, 0])
    assert np.abs(lhs - rhs).max() <= 1e-12 * np.abs(lhs).max()


# ------------------------------------------------------ P6 solver forms
@pytest.mark.parametrize("C,P", [(1, 1), (1, 2), (2, 1), (3, 2), (2, 3), (4, 4)])
def test_solver_identities(C, P):
    rng = np.random.default_rng(C * 10 + P)
    for _ in range(5):
        H = rng.normal(size=(C, P)) + 1j * rng.normal(size=(C, P))
        D = rng.normal(size=C) + 1j * rng.normal(size=C)
        eta = 10 ** rng.uniform(-3, 0)
        a = model.solve_normal(H, D, eta)
        for other in (model.solve_pushthrough, model.solve_svd, model.solve_lstsq):
            assert np.abs(other(H, D, eta) - a).max() <= 1e-10 * max(1.0, np.abs(a).max())
        # the minimiser: gradient of ||D - H f||^2 + eta ||f||^2 vanishes
        g = H.conj().T @ (H @ a - D) + eta * a
        assert np.abs(g).max() <= 1e-10 * max(1.0, np.abs(D).max())


def test_batched_normal_solve_matches_single_frequency_forms():
    rng = np.random.default_rng(5)
    C, P, n = 2, 2, 7
    Hm = [[rng.normal(size=n) + 1j * rng.normal(size=n) for _ in range(P)] for _ in range(C)]
    Dm = [rng.normal(size=n) + 1j * rng.normal(size=n) for _ in range(C)]
    F = model._normal_solve(Hm, Dm, 0.3)
    for i in range(n):
        H = np.array([[Hm[c][p][i] for p in range(P)] for c in range(C)])
        D = np.array([Dm[c][i] for c in range(C)])
        assert np.abs(np.array([F[p][i] for p in range(P)]) - model.solve_svd(H, D, 0.3)).max() <= 1e-12


# ----------------------------------------------------- P7 exact recovery
@pytest.mark.parametrize("kind", ["phase", "fluor"])
def test_exact_recovery_band_limited(kind):
    o = ph.optics(na_ill=0.6)
    shape = (8, 16, 16)
    tfs = O.transfer_functions(o, shape, (kind,))
    modes, _, _ = model.widefield_system(tfs, (kind,))
    H = tfs[kind]
    tau = 0.05
    mask = np.abs(H) ** 2 >= tau * np.max(np.abs(H) ** 2)
    f0 = np.random.default_rng(9).normal(size=shape)
    f = np.real(np.fft.ifftn(np.fft.fftn(f0) * mask))[None]
    d = model.forward(modes, f, [1.0])
    eta = 1e-10
    fh = model.reconstruct(modes, d, eta, background=[1.0])
    assert rel_l2(fh, f) <= 2 * eta / tau + 1e-12


def test_exact_recovery_2d_pooled_screen_optics():
    """2D phase-from-defocus at the pooled-screen optics printed in Methods."""
    g = json.load(open(GOLDEN))["pooled_screen_autotune"]
    o = dict(ph.POOLED_SCREEN_OPTICS)
    assert (o["lambda_um"], o["na_det"], o["na_ill"], o["n_medium"]) == (
        g["wavelength_um"], g["na_det"], g["na_ill"], g["n_medium"])
    shape = (7, 32, 32)
    pt = O.plane_tfs(o, shape, ("phase",))
    Hj = pt["phase"]
    tot = np.sum(np.abs(Hj) ** 2, axis=0)
    tau = 0.05
    mask = tot >= tau * tot.max()
    f2 = np.real(np.fft.ifft2(np.fft.fft2(np.random.default_rng(4).normal(size=shape[1:])) * mask))
    # thin object at the reference plane -> every data plane j sees H_j
    d = np.real(np.fft.ifft2(Hj * np.fft.fft2(f2)[None])) + 1.0
    plane_modes = [dict(channels=[0], props=[0], H=[[Hj]])]
    eta = 1e-10
    fh = model.reconstruct_2d(plane_modes, d[None], eta, background=[1.0])
    assert rel_l2(fh[0], f2) <= 2 * eta / tau + 1e-12


# ----------------------------------------- P8 dense operator, brute force
def _dense_operator(apply, n_in, out_size):
    A = np.zeros((out_size, n_in))
    e = np.zeros(n_in)
    for i in range(n_in):
        e[:] = 0.0
        e[i] = 1.0
        A[:, i] = apply(e).ravel()
    return A


@pytest.mark.parametrize("kinds,bg", [(("phase",), [1.3]), (("phase", "absorption"), [0.9]),
                                      (("fluor",), None), (("phase", "absorption", "fluor"), [1.1, 0.4])])
def test_dense_tikhonov_equals_fourier_reconstruction(kinds, bg):
    o = ph.optics(na_ill=0.7, tilt_x=0.05, defocus_um=0.1)
    shape = (8, 8, 8)
    n = int(np.prod(shape))
    tfs = O.transfer_functions(o, shape, kinds)
    modes, props, chans = model.widefield_system(tfs, kinds)
    rng = np.random.default_rng(21)
    d = 1.0 + 0.05 * rng.normal(size=(len(chans),) + shape)
    eta = 0.37
    fh = model.reconstruct(modes, d, eta, background=bg, relative=False)
    for m in modes:
        P = len(m["props"])
        sub = dict(channels=list(range(len(m["channels"]))), props=list(range(P)), H=m["H"])

        def apply(x, sub=sub, P=P):
            return model.forward([sub], x.reshape((P,) + shape), [0.0] * len(sub["channels"]))

        A = _dense_operator(apply, P * n, len(m["channels"]) * n)
        dm = np.stack([d[c] - (np.mean(d[c]) if bg is None else bg[c]) for c in m["channels"]]).ravel()
        x = np.linalg.solve(A.T @ A + eta * np.eye(P * n), A.T @ dm)
        got = np.stack([fh[p] for p in m["props"]]).ravel()
        assert np.abs(got - x).max() <= 1e-9 * np.abs(x).max()


def test_dense_tikhonov_equals_2d_reconstruction():
    o = ph.optics(na_ill=0.5, defocus_um=-0.2)
    shape = (5, 8, 8)
    Z, Y, X = shape
    pt = O.plane_tfs(o, shape, ("phase", "absorption"))
    tf3 = {k: O.stack_to_3d(v) for k, v in pt.items()}
    modes3, _, _ = model.widefield_system(tf3, ("phase", "absorption"))
    plane_modes = [dict(channels=[0], props=[0, 1], H=[[pt["phase"], pt["absorption"]]])]

    def apply(x):  # thin object in plane 0 of the 3D model
        f = np.zeros((2,) + shape)
        f[:, 0] = x.reshape(2, Y, X)
        return model.forward(modes3, f, [0.0])
    A = _dense_operator(apply, 2 * Y * X, Z * Y * X)
    rng = np.random.default_rng(8)
    d = 1.0 + 0.05 * rng.normal(size=(1,) + shape)
    eta = 0.2
    x = np.linalg.solve(A.T @ A + eta * np.eye(2 * Y * X), A.T @ (d[0] - np.mean(d[0])).ravel())
    fh = model.reconstruct_2d(plane_modes, d, eta, background=None, relative=False)
    assert np.abs(fh.ravel() - x).max() <= 1e-9 * np.abs(x).max()


def test_relative_eta_definition():
    o = ph.optics()
    shape = (4, 8, 8)
    tfs = O.transfer_functions(o, shape, ("phase", "absorption"))
    modes, _, _ = model.widefield_system(tfs, ("phase", "absorption"))
    d = 1.0 + 0.01 * np.random.default_rng(2).normal(size=(1,) + shape)
    mx = np.max(np.abs(tfs["phase"]) ** 2 + np.abs(tfs["absorption"]) ** 2)
    a = model.reconstruct(modes, d, 1e-3, relative=True)
    b = model.reconstruct(modes, d, 1e-3 * mx, relative=False)
    assert np.abs(a - b).max() <= 1e-14 * np.abs(a).max()


def test_relative_eta_is_eta_times_the_forward_operators_squared_norm():
    # Reading (v) without the per-frequency formula: the relative eta scales
    # eta by the largest squared singular value of the forward model as a map
    # of real volumes, taken here from its dense matrix (the real-space forward
    # model applied to every unit voxel of every property) by an SVD
    o = ph.optics(na_ill=0.5, tilt_x=0.1, defocus_um=0.2)
    shape = (4, 8, 8)
    kinds = ("phase", "absorption")
    tfs = O.transfer_functions(o, shape, kinds)
    modes, props, _ = model.widefield_system(tfs, kinds)
    n, P = int(np.prod(shape)), len(props)
    A = np.empty((n, P * n))
    for col in range(P * n):
        f = np.zeros((P,) + shape)
        f.flat[col] = 1.0
        A[:, col] = model.forward(modes, f, [0.0])[0].ravel()
    smax2 = np.linalg.norm(A, 2) ** 2
    got = model.eta_absolute(modes[0]["H"], 1e-3, True)
    assert abs(got - 1e-3 * smax2) <= 1e-10 * 1e-3 * smax2


def test_relative_eta_2d_is_the_3d_plane_sum_by_parseval():
    # 2D mode: eta_abs = eta * max over nu_perp of sum_j |H_j|^2 over the
    # planes; by Parseval over z that is (1/Z) sum over k_z of the 3D TF's
    # |H|^2, an independent route through the z-DFT
    o = ph.optics(na_ill=0.6, defocus_um=0.3)
    shape = (6, 16, 16)
    Z = shape[0]
    Hj = O.plane_tfs(o, shape, ("phase",))["phase"]
    H3 = O.transfer_functions(o, shape, ("phase",))["phase"]
    mx = float(np.max(np.sum(np.abs(H3) ** 2, axis=0) / Z))
    modes = [dict(channels=[0], props=[0], H=[[Hj]])]
    d = 1.0 + 0.01 * np.random.default_rng(4).normal(size=(1,) + shape)
    a = model.reconstruct_2d(modes, d, 1e-2, relative=True)
    b = model.reconstruct_2d(modes, d, 1e-2 * mx, relative=False)
    assert np.abs(a - b).max() <= 1e-12 * np.abs(a).max()


# ------------------------------------------------------------ tiles (a8)
def test_mirror_index():
    assert tiles.mirror(np.arange(-2, 7), 5).tolist() == [2, 1, 0, 1, 2, 3, 4, 3, 2]


def test_ramp_partition_of_unity():
    E, halo, core = 192, 32, 128
    w = tiles.ramp(E, halo)
    assert np.allclose(w[core:] + w[: E - core], 1.0, atol=1e-15)
    assert np.all(w[2 * halo: E - 2 * halo] == 1.0) and w.min() > 0


@pytest.mark.parametrize("ty,tx,core,halo", [(2, 3, 16, 4), (1, 1, 8, 2), (3, 2, 12, 6)])
def test_gather_then_blend_is_identity(ty, tx, core, halo):
    field = np.random.default_rng(3).normal(size=(3, ty * core, tx * core))
    t = tiles.gather(field, ty, tx, core, halo)
    assert t.shape == (ty * tx, 3, core + 2 * halo, core + 2 * halo)
    # a tile's core is the field's block
    assert np.array_equal(t[ty * tx - 1][:, halo:halo + core, halo:halo + core],
                          field[:, (ty - 1) * core:ty * core, (tx - 1) * core:tx * core])
    back = tiles.blend(t, ty, tx, core, halo)
    assert np.abs(back - field).max() <= 1e-14


def test_blend_of_constant_tiles_is_convex():
    ty, tx, core, halo = 2, 2, 16, 4
    vals = np.array([1.0, 2.0, 3.0, 4.0])
    t = np.broadcast_to(vals[:, None, None, None], (4, 1, core + 2 * halo, core + 2 * halo)).copy()
    out = tiles.blend(t, ty, tx, core, halo)[0]
    assert out[0, 0] == 1.0 and out[-1, -1] == 4.0 and out[0, -1] == 2.0
    assert out.min() >= 1.0 and out.max() <= 4.0
    # at the shared corner all four tiles weigh equally
    assert abs(out[core - 1: core + 1, core - 1: core + 1].mean() - 2.5) <= 1e-12


# ------------------------------------------------ auto-tuning objective
def test_tuning_objective_equals_rank_one_closed_form():
    """min_F sum_j |D_j - H_j F|^2 + eta |F|^2 = sum_j |D_j|^2 - |H^H D|^2 / (||H||^2 + eta)
    per transverse frequency (Parseval over the transform); the oracle
    evaluates the definition (reconstruct, residual in real space)."""
    from oracle import tuning
    o = ph.optics(na_ill=0.6, tilt_x=0.04, defocus_um=0.3)
    shape = (8, 32, 24)
    d = 1 + 0.01 * np.random.default_rng(1).normal(size=shape)
    eta = 1e-2
    Hj = O.plane_tfs(o, shape, ("phase",))["phase"]
    Dj = np.fft.fft2(d - d.mean(), axes=(1, 2))
    q = (np.sum(np.abs(Dj) ** 2, 0)
         - np.abs(np.sum(np.conj(Hj) * Dj, 0)) ** 2 / (np.sum(np.abs(Hj) ** 2, 0) + eta))
    assert abs(tuning.objective(o, d, eta) - np.sum(q) / (32 * 24)) <= 1e-12 * np.sum(q)


def test_tf_defocus_derivative_matches_finite_difference():
    from oracle import tuning
    o = ph.optics(na_ill=0.7, tilt_y=-0.03, defocus_um=-0.2)
    shape = (6, 24, 32)
    h = 1e-5
    Hp = O.transfer_functions(dict(o, defocus_um=-0.2 + h), shape, ("phase",))["phase"]
    Hm = O.transfer_functions(dict(o, defocus_um=-0.2 - h), shape, ("phase",))["phase"]
    dH = tuning.tf_defocus_derivative(o, shape)
    assert np.abs(dH - (Hp - Hm) / (2 * h)).max() <= 1e-7 * np.abs(dH).max()


def test_tuning_objective_is_minimal_at_the_true_defocus():
    """A thin band-limited object imaged at defocus z0 (noiseless): the loss
    is smallest at z0 and its derivative vanishes there."""
    from oracle import tuning
    o = ph.optics(na_ill=0.5)
    shape = (12, 48, 48)
    Z, Y, X = shape
    rng = np.random.default_rng(3)
    ky, kx = np.fft.fftfreq(Y)[:, None], np.fft.fftfreq(X)[None, :]
    f2 = 0.05 * np.real(np.fft.ifft2(np.fft.fft2(rng.normal(size=(Y, X))) * np.exp(-(ky ** 2 + kx ** 2) / 0.02)))
    z0 = 0.35
    Hj = O.plane_tfs(dict(o, defocus_um=z0), shape, ("phase",))["phase"]
    d = np.real(np.fft.ifft2(Hj * np.fft.fft2(f2)[None], axes=(1, 2))) + 1.0
    eta = 1e-6
    L0 = tuning.objective_at(o, d, eta, z0)
    for dz in (-0.1, -0.03, 0.03, 0.1):
        assert tuning.objective_at(o, d, eta, z0 + dz) > L0
    g = tuning.gradient_fd(dict(o, defocus_um=z0), d, eta, h=1e-4)
    g_off = tuning.gradient_fd(dict(o, defocus_um=z0 + 0.1), d, eta, h=1e-4)
    assert abs(g) <= 1e-3 * abs(g_off)


def test_band_limited_objective_is_the_closed_form_over_the_band():
    """Restricting the data to |nu| <= nu_max restricts the per-frequency sum
    of the closed form to those frequencies (every frequency is solved on its
    own), and a band above every grid frequency changes nothing."""
    from oracle import tuning
    o = ph.optics(na_ill=0.8, defocus_um=-0.2)
    shape = (6, 40, 32)
    Z, Y, X = shape
    d = 1 + 0.02 * np.random.default_rng(4).normal(size=shape)
    eta, nu_max = 1e-2, 1.37
    Hj = O.plane_tfs(o, shape, ("phase",))["phase"]
    Dj = np.fft.fft2(d - d.mean(), axes=(1, 2))
    q = (np.sum(np.abs(Dj) ** 2, 0)
         - np.abs(np.sum(np.conj(Hj) * Dj, 0)) ** 2 / (np.sum(np.abs(Hj) ** 2, 0) + eta))
    fy = np.fft.fftfreq(Y, o["pixel_um"])[:, None]
    fx = np.fft.fftfreq(X, o["pixel_um"])[None, :]
    band = fy ** 2 + fx ** 2 <= nu_max ** 2
    assert 10 < band.sum() < Y * X // 2
    want = np.sum(q[band]) / (Y * X)
    assert abs(tuning.objective(o, d, eta, nu_max) - want) <= 1e-12 * want
    assert abs(tuning.objective(o, d, eta, 1e3) - tuning.objective(o, d, eta)) <= 1e-12 * want


def test_midband_objective_closed_form_and_band():
    """Minus the mid-band power equals -sum_band |sum_j H_j* D_j|^2 /
    (sum_j |H_j|^2 + eta)^2 / N_perp (the 2D solve written out), and the band
    is the annulus c/8 <= |nu| <= c/4 with c = (NA_det + NA_ill)/lambda."""
    from oracle import tuning
    o = ph.optics(na_ill=0.7, defocus_um=0.25, tilt_y=0.05)
    shape = (6, 40, 48)
    Z, Y, X = shape
    d = 1 + 0.02 * np.random.default_rng(8).normal(size=shape)
    eta = 1e-2
    Hj = O.plane_tfs(o, shape, ("phase",))["phase"]
    Dj = np.fft.fft2(d - d.mean(), axes=(1, 2))
    F = np.sum(np.conj(Hj) * Dj, 0) / (np.sum(np.abs(Hj) ** 2, 0) + eta)
    fy = np.fft.fftfreq(Y, o["pixel_um"])[:, None]
    fx = np.fft.fftfreq(X, o["pixel_um"])[None, :]
    c = (o["na_det"] + o["na_ill"]) / o["lambda_um"]
    r = np.sqrt(fy ** 2 + fx ** 2)
    band = (r >= c / 8) & (r <= c / 4)
    assert 20 < band.sum() < Y * X // 4
    want = -np.sum(np.abs(F[band]) ** 2) / (Y * X)
    assert abs(tuning.midband_objective(o, d, eta) - want) <= 1e-12 * abs(want)
    assert np.array_equal(tuning.midband_mask(o, Y, X), band)


# ------------------------------------------------ smooth source pupil (illumination tuning)
def test_smooth_source_edge_values():
    """The logistic edge is 1/2 on the circle, within 1e-4 of the disk five
    edge widths inside and outside, and reduces to the disk away from it."""
    o = ph.optics(na_ill=0.7, tilt_x=0.05, smooth_source=True)
    Y, X = 32, 40
    S = O.source_pupil(o, Y, X)
    Sh = O.source_pupil(dict(o, smooth_source=False), Y, X)
    lam = o["lambda_um"]
    ky, kx = O.transverse_grid(Y, X, o["pixel_um"])
    d = np.sqrt((kx - o["tilt_x"] / lam) ** 2 + ky ** 2)
    w = O.source_edge_width(o, Y, X)
    far = np.abs(d - o["na_ill"] / lam) > 10 * w
    assert np.abs(S - Sh)[far].max() <= 1e-4
    o2 = dict(o, na_ill=float(d[3, 4] * lam))  # a grid point exactly on the edge
    assert abs(O.source_pupil(o2, Y, X)[3, 4] - 0.5) <= 1e-12
    # the edge width is one frequency bin of the coarser axis: 1 / (32 * 0.1 um)
    # = 0.3125 /um here, so a grid point that far outside the circle has
    # S = 1 / (1 + e)
    o3 = dict(o, na_ill=float((d[3, 4] - 0.3125) * lam))
    assert abs(O.source_pupil(o3, Y, X)[3, 4] - 1.0 / (1.0 + np.e)) <= 1e-12


def test_smooth_source_derivatives_match_finite_differences():
    o = ph.optics(na_ill=0.6, tilt_x=0.07, tilt_y=-0.04, smooth_source=True)
    Y, X = 24, 32
    dS = O.source_pupil_derivatives(o, Y, X)
    h = 1e-6
    for k in ("tilt_x", "tilt_y", "na_ill"):
        fd = (O.source_pupil(dict(o, **{k: o[k] + h}), Y, X) - O.source_pupil(dict(o, **{k: o[k] - h}), Y, X)) / (2 * h)
        assert np.abs(dS[k] - fd).max() <= 1e-6 * np.abs(fd).max(), k


def test_smooth_source_forward_equals_weighted_source_point_sum():
    """The correlation route with the smooth source equals the incoherent sum
    of source-point fields weighted by S (independent of the correlation)."""
    o = ph.optics(na_ill=0.55, tilt_x=0.06, tilt_y=0.02, defocus_um=0.2, smooth_source=True)
    shape = (5, 20, 24)
    rng = np.random.default_rng(11)
    dn = rng.normal(size=shape[1:]) * 1e-2
    kap = rng.normal(size=shape[1:]) * 1e-3
    tfs = O.transfer_functions(o, shape, ("phase", "absorption"))
    modes, _, _ = model.widefield_system(tfs, ("phase", "absorption"))
    f = np.zeros((2,) + shape)
    f[0, 1] = dn
    f[1, 1] = kap
    d = model.forward(modes, f, [1.0])[0] - 1.0
    assert rel_l2(d, _field_route(o, shape, 1, dn, kap)) <= 1e-12


def test_source_tf_derivatives_match_finite_differences():
    from oracle import tuning
    o = ph.optics(na_ill=0.65, tilt_x=0.05, tilt_y=-0.03, defocus_um=0.3, smooth_source=True)
    shape = (6, 24, 32)
    dH = tuning.plane_tf_source_derivatives(o, shape)
    h = 1e-5
    for k in ("tilt_x", "tilt_y", "na_ill"):
        Hp = O.plane_tfs(dict(o, **{k: o[k] + h}), shape, ("phase",))["phase"]
        Hm = O.plane_tfs(dict(o, **{k: o[k] - h}), shape, ("phase",))["phase"]
        fd = (Hp - Hm) / (2 * h)
        assert np.abs(dH[k] - fd).max() <= 1e-6 * np.abs(fd).max(), k


# ------------------------------------------------ learned estimator (reference network and features)
def test_estimator_conv_equals_scipy_correlation():
    """The network's 3x3 zero-padded strided convolution equals a sum of
    scipy.signal.correlate2d results, subsampled."""
    from scipy.signal import correlate2d
    from oracle import estimator as E
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 3, 10, 12))
    w = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    for s in (1, 2):
        y = E._conv(x, w, b, s)
        for bi in range(2):
            for co in range(4):
                full = sum(correlate2d(x[bi, ci], w[co, ci], mode="same", boundary="fill") for ci in range(3))
                assert np.allclose(y[bi, co], full[::s, ::s] + b[co], atol=1e-12)


def test_estimator_bf16_rounding_matches_torch():
    import torch
    from oracle import estimator as E
    vals = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -9, -2.7182817, 3.1415927e-5, 65504.0, 1e-40], dtype=np.float32)
    want = torch.tensor(vals).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(E.bf16(vals), want)


def test_estimator_backward_matches_finite_differences(monkeypatch):
    """The hand-derived backward pass equals central differences of the loss
    for weights and biases of every layer.  The bfloat16 rounding of the
    weights makes the loss piecewise constant in them, so the check runs
    with the rounding replaced by the identity (the backward pass is the
    gradient with respect to the rounded values)."""
    from oracle import estimator as E
    monkeypatch.setattr(E, "bf16", lambda v: np.asarray(v, dtype=np.float64))
    rng = np.random.default_rng(1)
    flat = rng.normal(size=E.n_params()) * 0.05
    x = rng.normal(size=(2, 3, 16, 16))
    t = rng.normal(size=(2, 4))
    L, g = E.backward(flat, x, t)
    assert abs(L - E.loss(flat, x, t)) <= 1e-14 * abs(L)
    offs = np.cumsum([0] + [int(np.prod(sh)) for sh in E.param_shapes()])
    h = 1e-6
    for k in range(len(offs) - 1):  # a few entries of every parameter array
        for i in rng.integers(offs[k], offs[k + 1], size=3):
            fp, fm = flat.copy(), flat.copy()
            fp[i] += h
            fm[i] -= h
            fd = (E.loss(fp, x, t) - E.loss(fm, x, t)) / (2 * h)
            assert abs(g[i] - fd) <= 1e-6 * (abs(fd) + 1e-4), (k, i, g[i], fd)


def test_estimator_backward_with_given_relu_decisions():
    """Passing the forward pass's own ReLU decisions reproduces the default
    gradient exactly; flipping the decision of one output that is exactly zero
    before the ReLU changes only gradients of that layer and below."""
    from oracle import estimator as E
    rng = np.random.default_rng(4)
    flat = rng.normal(size=E.n_params()) * 0.05
    x = rng.normal(size=(2, 3, 16, 16))
    t = rng.normal(size=(2, 4))
    _, acts = E.forward(flat, x)
    masks = [a > 0 for a in acts[1:5]]
    L0, g0 = E.backward(flat, x, t)
    L1, g1 = E.backward(flat, x, t, masks=masks)
    assert L0 == L1 and np.array_equal(g0, g1)
    # an inactive output of the last convolution layer switched on: its
    # activation is 0 either way, so the forward pass and the head's
    # gradients stay, while the layers below see one more path
    m = [q.copy() for q in masks]
    i = np.argwhere(~m[3])[0]
    m[3][tuple(i)] = True
    _, g2 = E.backward(flat, x, t, masks=m)
    offs = np.cumsum([0] + [int(np.prod(sh)) for sh in E.param_shapes()])
    assert np.array_equal(g2[offs[8]:], g0[offs[8]:])          # the linear head
    assert not np.array_equal(g2[offs[6]:offs[7]], g0[offs[6]:offs[7]])  # the last conv's weights


def test_estimator_features_properties():
    """Plane-to-plane drift shows in the cross channels with its sign and
    axis; reversing the plane order mirrors the rows and flips the drift;
    the power channel does not see the data's scale."""
    from oracle import estimator as E
    o = ph.optics()
    rng = np.random.default_rng(2)
    Z, Y, X = 8, 32, 32
    base = rng.normal(size=(Y, X))
    same = np.stack([base] * Z)
    f = E.tile_features(same, o)
    assert np.abs(f[1:]).max() <= 1e-12
    # +1 pixel in x per plane; an image even in y has no drift signal along y
    def stack_drift(img, axis):  # natural plane r shifted by r pixels, stored in FFT order
        out = np.zeros((Z,) + img.shape)
        for r in range(Z):
            out[E.natural_plane(r, Z)] = np.roll(img, r, axis=axis)
        return out

    sym_y = base + np.roll(base[::-1], 1, axis=0)
    xs = stack_drift(sym_y, 1)
    f = E.tile_features(xs, o)
    band = f[0, 0] > 0
    band[0] = False  # bin 0 holds only the zero frequency, which has no direction
    assert np.all(f[1, : Z - 1][:, band] < 0) and np.abs(f[2]).max() <= 1e-12
    sym_x = base + np.roll(base[:, ::-1], 1, axis=1)
    ys = stack_drift(sym_x, 0)
    f = E.tile_features(ys, o)
    assert np.all(f[2, : Z - 1][:, band] < 0) and np.abs(f[1]).max() <= 1e-12
    # plane order reversed (row r <-> Z-1-r in natural order): drift flips sign
    stack = rng.normal(size=(Z, Y, X))
    nat = np.stack([stack[E.natural_plane(r, Z)] for r in range(Z)])
    rev = nat[::-1]
    back = np.zeros_like(stack)
    for r in range(Z):
        back[E.natural_plane(r, Z)] = rev[r]
    fa, fb = E.tile_features(stack, o), E.tile_features(back, o)
    assert np.allclose(fb[0, :Z], fa[0, :Z][::-1], atol=1e-12)
    assert np.allclose(fb[1, : Z - 1], -fa[1, : Z - 1][::-1], atol=1e-12)
    assert np.allclose(E.tile_features(1 + 3.0 * (stack - 1), o)[0], fa[0], atol=1e-12)


def test_adam_first_steps_move_by_the_learning_rate():
    # Kingma and Ba (2015): with bias correction the first step is lr * sign(g)
    # for |g| >> eps, and so is every step of a constant gradient
    from oracle import estimator as E
    g = np.array([3.0, -0.5, 1e-3, -200.0])
    w, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    for step in (1, 2, 3):
        w1, m, v = E.adam(w, g, m, v, step, 0.01)
        assert np.allclose(w1 - w, -0.01 * np.sign(g), rtol=1e-4, atol=0)
        w = w1


def test_estimator_feature_bins_floor():
    # a plane wave at k_x = 7 on a 64-pixel, 0.1 um grid: |nu| = 7 / 6.4 um^-1,
    # which is 15.52 in units of (2 NA / lambda) / 64 at NA 1.2, lambda
    # 0.532 um, so all its power sits in radial bin 15
    from oracle import estimator as E
    o = ph.optics()
    Z, Y, X = 4, 64, 64
    x = np.arange(X)
    d = np.stack([np.cos(2 * np.pi * 7 * x / X + 0.3 * j)[None, :] * np.ones((Y, 1)) for j in range(Z)])
    f = E.tile_features(d, o)
    p = np.expm1(f[0, :Z])  # power per bin over the mean power per bin
    assert np.all(p[:, 15] > 0) and np.abs(np.delete(p, 15, axis=1)).max() <= 1e-12


@pytest.mark.parametrize("Z", [1, 3, 4, 6, 8])
def test_estimator_rows_are_the_planes_in_axial_order(Z):
    # natural row r holds the plane displaced by (r - Z//2) steps: the storage
    # index (FFT order) whose signed index is r - Z//2
    from oracle import estimator as E
    k = O.fft_indices(Z)
    for r in range(Z):
        assert k[E.natural_plane(r, Z)] == r - Z // 2


# ------------------------------------------------- aberrated detection pupils
def _unit_pupil(o, Y, X):
    nu_y, nu_x = O.transverse_grid(Y, X, o["pixel_um"])
    R = o["na_det"] / o["lambda_um"]
    return nu_x / R, nu_y / R


def test_zernike_matches_nolls_table():
    """Noll (1976), Table 1: the closed forms of the first polynomials."""
    rng = np.random.default_rng(3)
    rho = np.sqrt(rng.uniform(0, 1, 200))
    phi = rng.uniform(-np.pi, np.pi, 200)
    r, c, s_ = rho, np.cos, np.sin
    table = {
        1: np.ones_like(r), 2: 2 * r * c(phi), 3: 2 * r * s_(phi), 4: np.sqrt(3) * (2 * r**2 - 1),
        5: np.sqrt(6) * r**2 * s_(2 * phi), 6: np.sqrt(6) * r**2 * c(2 * phi),
        7: np.sqrt(8) * (3 * r**3 - 2 * r) * s_(phi), 8: np.sqrt(8) * (3 * r**3 - 2 * r) * c(phi),
        9: np.sqrt(8) * r**3 * s_(3 * phi), 10: np.sqrt(8) * r**3 * c(3 * phi),
        11: np.sqrt(5) * (6 * r**4 - 6 * r**2 + 1),
        12: np.sqrt(10) * (4 * r**4 - 3 * r**2) * c(2 * phi), 13: np.sqrt(10) * (4 * r**4 - 3 * r**2) * s_(2 * phi),
        14: np.sqrt(10) * r**4 * c(4 * phi), 15: np.sqrt(10) * r**4 * s_(4 * phi),
        16: np.sqrt(12) * (10 * r**5 - 12 * r**3 + 3 * r) * c(phi),
        17: np.sqrt(12) * (10 * r**5 - 12 * r**3 + 3 * r) * s_(phi),
        22: np.sqrt(7) * (20 * r**6 - 30 * r**4 + 12 * r**2 - 1),
    }
    for j, want in table.items():
        assert np.abs(O.zernike(j, rho, phi) - want).max() <= 1e-12, j


def test_zernike_orthonormal_on_the_unit_disk():
    """<Z_i, Z_j> = pi delta_ij for the first 36 (Gauss-Legendre in rho, exact
    for these degrees; a uniform grid in phi, exact for trigonometric degree < 64)."""
    xg, wg = np.polynomial.legendre.leggauss(16)
    rho = 0.5 * (xg + 1.0)
    w_r = 0.5 * wg * rho  # rho d rho
    phi = np.arange(64) * 2 * np.pi / 64
    R, PH = np.meshgrid(rho, phi, indexing="ij")
    W = w_r[:, None] * (2 * np.pi / 64)
    Zs = np.stack([O.zernike(j, R, PH) for j in range(1, 37)])
    G = np.einsum("iab,jab,ab->ij", Zs, Zs, W) / np.pi
    assert np.abs(G - np.eye(36)).max() <= 1e-12
    # every (n, m) with n <= 7 and n - |m| even, exactly once
    nm = [O.noll_nm(j) for j in range(1, 37)]
    assert sorted(nm) == sorted((n, m) for n in range(8) for m in range(-n, n + 1, 2))


def test_piston_leaves_every_tf_unchanged():
    o = ph.optics(na_ill=0.6, tilt_x=0.05, defocus_um=0.3)
    shape = (6, 24, 32)
    ref = O.transfer_functions(o, shape)
    got = O.transfer_functions(dict(o, zernike=[0.37]), shape)
    for k in O.KINDS:
        assert rel_l2(got[k], ref[k]) <= 1e-13, k


@pytest.mark.parametrize("axis,shift", [("x", 2), ("y", -3)])
def test_tilt_zernike_is_a_lateral_shift(axis, shift):
    """W = c_2 Z_2 = 2 c_2 nu_x lambda / NA_det: the pupil gains e^{i 2 pi s nu_x}
    with s = 2 c_2 lambda / NA_det, every PSF moves by -s, and every TF is
    multiplied by e^{i 2 pi s q_x}.  With s a whole number of pixels that is
    exact on the periodic grid (Z_3 likewise along y)."""
    o = ph.optics(na_ill=0.5, tilt_x=0.04, tilt_y=-0.03, defocus_um=-0.2)
    shape = (6, 24, 32)
    Z, Y, X = shape
    c = shift * o["pixel_um"] * o["na_det"] / (2.0 * o["lambda_um"])
    coef = [0.0, c, 0.0] if axis == "x" else [0.0, 0.0, c]
    ref = O.transfer_functions(o, shape)
    got = O.transfer_functions(dict(o, zernike=coef), shape)
    k = O.fft_indices(X)[None, None, :] if axis == "x" else O.fft_indices(Y)[None, :, None]
    n = X if axis == "x" else Y
    ramp = np.exp(2j * np.pi * shift * k / n)
    for kind in O.KINDS:
        assert rel_l2(got[kind], ref[kind] * ramp) <= 1e-12, kind


def test_aberrated_forward_equals_source_point_field_sum():
    """Astigmatism and coma (closed forms typed here, Cartesian) through the
    field route against the TF model with the same Noll coefficients."""
    o = ph.optics(na_ill=0.55, tilt_x=0.06, tilt_y=0.02, defocus_um=0.2)
    shape = (5, 20, 24)
    Z, Y, X = shape
    c6, c8 = 0.21, -0.13
    ux, uy = _unit_pupil(o, Y, X)
    W = c6 * np.sqrt(6) * (ux * ux - uy * uy) + c8 * np.sqrt(8) * (3 * (ux * ux + uy * uy) - 2) * ux
    P = O.detection_pupil(o, Y, X)
    pupil = P * np.exp(2j * np.pi * W)
    rng = np.random.default_rng(11)
    dn = rng.normal(size=shape[1:]) * 1e-2
    kap = rng.normal(size=shape[1:]) * 1e-3
    oa = dict(o, zernike=[0, 0, 0, 0, 0, c6, 0, c8])
    tfs = O.transfer_functions(oa, shape, ("phase", "absorption"))
    modes, _, _ = model.widefield_system(tfs, ("phase", "absorption"))
    f = np.zeros((2,) + shape)
    f[0, 1] = dn
    f[1, 1] = kap
    d = model.forward(modes, f, [1.0])[0] - 1.0
    assert rel_l2(d, _field_route(o, shape, 1, dn, kap, pupil)) <= 1e-12
    # and the aberration matters: the unaberrated model is far from it
    tf0 = O.transfer_functions(o, shape, ("phase", "absorption"))
    d0 = model.forward(model.widefield_system(tf0, ("phase", "absorption"))[0], f, [1.0])[0] - 1.0
    assert rel_l2(d0, d) >= 0.05


def test_aberrated_fluorescence_point_is_psf():
    """Spherical aberration (Z_11, typed here): the image of a point emitter is
    |IDFT2(P e^{i 2 pi W} e^{i 2 pi eta z_j})|^2 per plane, unit sum."""
    o = ph.optics(defocus_um=0.3)
    shape = (6, 16, 20)
    Z, Y, X = shape
    c11 = 0.3
    ux, uy = _unit_pupil(o, Y, X)
    r2 = ux * ux + uy * uy
    W = c11 * np.sqrt(5) * (6 * r2 * r2 - 6 * r2 + 1)
    tfs = O.transfer_functions(dict(o, zernike=[0] * 10 + [c11]), shape, ("fluor",))
    modes, _, _ = model.widefield_system(tfs, ("fluor",))
    f = np.zeros((1,) + shape)
    f[0, 0, 0, 0] = 1.0
    d = model.forward(modes, f, [0.0])[0]
    P = O.detection_pupil(o, Y, X) * np.exp(2j * np.pi * W)
    eta = O.axial_frequency(o, Y, X)
    z = O.plane_displacements(Z, o["z_step_um"], o["defocus_um"])
    Ey = np.exp(2j * np.pi * np.outer(np.arange(Y), O.fft_indices(Y)) / Y)
    Ex = np.exp(2j * np.pi * np.outer(np.arange(X), O.fft_indices(X)) / X)
    psf = np.stack([np.abs(Ey @ (P * np.exp(2j * np.pi * eta * z[j])) @ Ex.T) ** 2 for j in range(Z)])
    psf /= psf.sum()
    assert rel_l2(d, psf) <= 1e-12
    assert abs(np.sum(tfs["fluor"][0, 0, 0]) - 1.0) <= 1e-12  # H_fl(0) = 1 still


# ------------------------------------------------------------------ padding
@pytest.mark.parametrize("mode,np_mode", [("zero", "constant"), ("edge", "edge"), ("mirror", "reflect")])
def test_padding_matches_numpy_pad(mode, np_mode):
    """numpy.pad with the centred split of the margin; the mirror case includes
    margins wider than the axis (numpy reflects repeatedly)."""
    v = np.random.default_rng(0).normal(size=(2, 5, 6, 7))
    for sp in ((9, 10, 11), (5, 16, 8), (21, 6, 30), (5, 6, 7)):
        widths = [(0, 0)] + [((p - n) // 2, p - n - (p - n) // 2) for p, n in zip(sp, v.shape[1:])]
        assert np.array_equal(tiles.pad(v, sp, mode), np.pad(v, widths, mode=np_mode)), sp
        assert np.array_equal(tiles.crop(tiles.pad(v, sp, mode), v.shape[1:]), v)
    one = np.arange(3.0).reshape(1, 1, 3)
    assert np.array_equal(tiles.pad(one, (3, 1, 3), "mirror")[:, 0, :], np.tile(one[0], (3, 1)))


def test_zero_padding_in_place_of_circular_boundaries_helps():
    """A stack cut out of a larger world is not periodic: reconstructing it
    with circular boundaries wraps the missing planes around.  Zero padding
    of the background-free window (to twice the planes, 1.5 times the
    width) brings the error well down towards that of the full world."""
    o = ph.optics(na_ill=0.7)
    world, win = (24, 48, 48), (12, 32, 32)

    def recon(data, shape):
        md, _, _ = model.widefield_system(O.transfer_functions(o, shape, ("phase",)), ("phase",))
        return model.reconstruct(md, data[None], 1e-3)[0]

    for seed in range(3):
        rng = np.random.default_rng(seed)
        f = ph.sphere_phantom(seed, world, o, n_spheres=30)
        md, _, _ = model.widefield_system(O.transfer_functions(o, world, ("phase",)), ("phase",))
        d = model.forward(md, f[None], [1.0])[0] + rng.normal(size=world) * 1e-3
        dw, fw = tiles.crop(d, win), tiles.crop(f, win)
        circular = rel_l2(recon(dw, win), fw)
        padded = rel_l2(tiles.crop(recon(tiles.pad(dw - dw.mean(), world, "zero"), world), win), fw)
        assert padded <= 0.75 * circular, (seed, padded, circular)
