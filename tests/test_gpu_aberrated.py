"""Aberrated detection pupils (Noll Zernike phase) through the C ABI against
the float64 oracle: every kind of TF bank, the derivative banks, the forward
model, and the whole bank at the widefield workload's full size."""
import numpy as np
import pytest

import phantom as ph
from conftest import rel_l2
from oracle import model as OM, optics as OO, tuning as OT

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2412_09775_gb300.build import build
    build()
    from paper_2412_09775_gb300 import binding
    return binding, torch, torch.device("cuda:0")


def coefficient_sets(n_tiles, seed=5):
    """Tile 0: defocus, astigmatism, coma and spherical; tile 1: all 36 terms
    small and random; tile 2 (if asked): several waves (phase wrapping)."""
    rng = np.random.default_rng(seed)
    sets = [[0.0, 0.0, 0.0, 0.1, -0.15, 0.2, 0.08, -0.12, 0.0, 0.0, 0.1],
            list(rng.uniform(-0.1, 0.1, 36)),
            [0.4, 0.3, -0.2, 2.3, 0.0, 1.1, 0.0, 0.0, 0.0, 0.0, -1.7]]
    width = max(len(s) for s in sets[:n_tiles])
    return [s + [0.0] * (width - len(s)) for s in sets[:n_tiles]]


def build(env, optics_list, zern, shape, kinds):
    B, torch, dev = env
    Z, Y, X = shape
    n = len(optics_list)
    tf = torch.empty(B.wo_tf_bytes(n, Z, Y, X, kinds), dtype=torch.uint8, device=dev)
    ws = torch.empty(B.wo_aberrated_workspace_bytes(n, Z, Y, X, kinds), dtype=torch.uint8, device=dev)
    B.wo_build_tf_aberrated(optics_list, zern, n, Z, Y, X, kinds, tf, ws)
    torch.cuda.synchronize()
    return tf, ws


def with_zernike(optics_list, zern):
    return [dict(o, zernike=z) for o, z in zip(optics_list, zern)]


def check_bank(env, optics_list, zern, shape, kinds):
    B, torch, dev = env
    Z, Y, X = shape
    tf, _ = build(env, optics_list, zern, shape, kinds)
    spec = B.tf_views(tf, len(optics_list), Z, Y, X, kinds)[0].cpu().numpy()
    names = [k for k in OO.KINDS if B.KIND_BITS[k] & kinds]
    for t, o in enumerate(with_zernike(optics_list, zern)):
        ref = OO.transfer_functions(o, shape, names)
        for s, k in enumerate(names):
            mode = ("fluor",) if k == "fluor" else [q for q in ("phase", "absorption") if q in names]
            den = np.sqrt(sum(np.linalg.norm(OO.half_spectrum(ref[q])) ** 2 for q in mode))
            e = np.linalg.norm(spec[t, s] - OO.half_spectrum(ref[k])) / den
            assert e <= TOL, (t, k, e)


@pytest.mark.parametrize("kinds", [1, 2, 4, 3, 7])
def test_aberrated_tf_kinds_match_oracle(env, kinds):
    ol = [ph.optics(na_ill=0.8, tilt_x=0.04, tilt_y=-0.02, defocus_um=0.3),
          ph.optics(na_ill=0.6, defocus_um=-0.5),
          ph.optics(na_ill=0.9, tilt_y=0.05, defocus_um=0.1)]
    check_bank(env, ol, coefficient_sets(3), (8, 32, 48), kinds)


@pytest.mark.parametrize("shape", [(16, 64, 64), (12, 48, 96), (1, 16, 16), (3, 12, 24), (4, 192, 24),
                                   (6, 96, 48)])
def test_aberrated_tf_shapes(env, shape):
    ol = [ph.optics(na_ill=0.6, tilt_y=0.05, defocus_um=-0.4), ph.optics(na_ill=0.7, tilt_x=-0.03)]
    check_bank(env, ol, coefficient_sets(2, seed=len(shape) + shape[1]), shape, 7)


def test_aberrated_smooth_source_bank(env):
    B = env[0]
    ol = [dict(ph.optics(na_ill=0.75, tilt_x=0.06, defocus_um=0.2), smooth_source=True)]
    check_bank(env, ol, coefficient_sets(1), (8, 32, 48), B.WO_TF_PHASE | B.WO_TF_ABSORPTION | B.WO_TF_SMOOTH_SOURCE)


def test_no_coefficients_is_the_plain_build(env):
    B, torch, dev = env
    shape = (8, 32, 48)
    Z, Y, X = shape
    ol = [ph.optics(na_ill=0.8, tilt_x=0.04, defocus_um=0.3), ph.optics(na_ill=0.5)]
    tf_a, _ = build(env, ol, [[], []], shape, 7)
    tf_p, ws_p = B.alloc(2, Z, Y, X, 7, dev)
    B.wo_build_tf(ol, 2, Z, Y, X, 7, tf_p, ws_p)
    torch.cuda.synchronize()
    assert torch.equal(tf_a, tf_p)


@pytest.mark.parametrize("planes", [False, True])
def test_aberrated_defocus_derivative_bank(env, planes):
    B, torch, dev = env
    shape = (8, 32, 48)
    Z, Y, X = shape
    ol = [ph.optics(defocus_um=0.4, na_ill=0.6), ph.optics(defocus_um=-0.7, tilt_x=0.05, na_ill=0.8)]
    zern = coefficient_sets(2, seed=9)
    kinds = B.WO_TF_PHASE_DZ | (B.WO_TF_PLANES if planes else 0)
    tf, _ = build(env, ol, zern, shape, kinds)
    spec = B.tf_views(tf, 2, Z, Y, X, kinds)[0].cpu().numpy()
    for t, o in enumerate(with_zernike(ol, zern)):
        if planes:
            H, dH = OO.plane_tfs(o, shape, ("phase",))["phase"], OT.plane_tf_defocus_derivative(o, shape)
        else:
            H, dH = OO.transfer_functions(o, shape, ("phase",))["phase"], OT.tf_defocus_derivative(o, shape)
        assert rel_l2(spec[t, 0], OO.half_spectrum(H)) <= TOL, t
        assert rel_l2(spec[t, 1], OO.half_spectrum(dH)) <= TOL, t


def test_aberrated_gradient_bank(env):
    """The five per-plane slots (H and its derivatives in defocus, tilt_x,
    tilt_y, NA_ill) with an aberrated detection pupil."""
    B, torch, dev = env
    shape = (6, 64, 64)
    Z, Y, X = shape
    ol = [dict(ph.optics(defocus_um=0.3, na_ill=0.7, tilt_x=0.04), smooth_source=True),
          dict(ph.optics(defocus_um=-0.5, na_ill=0.85, tilt_y=-0.06), smooth_source=True)]
    zern = coefficient_sets(2, seed=13)
    kinds = B.WO_TF_PHASE_GRAD | B.WO_TF_PLANES
    tf, _ = build(env, ol, zern, shape, kinds)
    spec = B.tf_views(tf, 2, Z, Y, X, kinds)[0].cpu().numpy()
    for t, o in enumerate(with_zernike(ol, zern)):
        refs = [OO.plane_tfs(o, shape, ("phase",))["phase"], OT.plane_tf_defocus_derivative(o, shape)]
        src = OT.plane_tf_source_derivatives(o, shape)
        refs += [src["tilt_x"], src["tilt_y"], src["na_ill"]]
        for q, ref in enumerate(refs):
            assert rel_l2(spec[t, q], OO.half_spectrum(ref)) <= TOL, (t, q)


def test_aberrated_forward_and_adjoint_match_oracle(env):
    B, torch, dev = env
    shape = (8, 32, 48)
    Z, Y, X = shape
    ol = [ph.optics(na_ill=0.7, tilt_x=0.03, defocus_um=0.2), ph.optics(na_ill=0.5, defocus_um=-0.3)]
    zern = coefficient_sets(2, seed=17)
    kinds = 7
    tf, ws = build(env, ol, zern, shape, kinds)
    f = ph.uniform_volume(5, (2, 3) + shape, -0.02, 0.02).astype(np.float32)
    bg = [1.0, 0.3]
    data = torch.empty((2, 2) + shape, dtype=torch.float32, device=dev)
    B.wo_forward(tf, kinds, torch.from_numpy(f).to(dev), bg, data, 2, Z, Y, X, ws)
    dd = ph.uniform_volume(6, (2, 2) + shape, 0.5, 1.5).astype(np.float32)
    fo = torch.empty((2, 3) + shape, dtype=torch.float32, device=dev)
    B.wo_forward_adjoint(tf, kinds, torch.from_numpy(dd).to(dev), bg, fo, 2, Z, Y, X, ws)
    got, got_adj = data.cpu().numpy(), fo.cpu().numpy()
    b = np.array(bg)[:, None, None, None]
    for t, o in enumerate(with_zernike(ol, zern)):
        modes, _, _ = OM.widefield_system(OO.transfer_functions(o, shape, OO.KINDS), OO.KINDS)
        ref = OM.forward(modes, f[t].astype(np.float64), bg)
        assert rel_l2(got[t] - b, ref - b) <= TOL, t
        assert rel_l2(got_adj[t], OM.adjoint(modes, dd[t].astype(np.float64), bg)) <= TOL, t


def test_aberrated_full_size(env):
    """The widefield workload's size (96 x 512 x 512), all three kinds, an
    aberration of several waves: the whole bank against the oracle."""
    B, torch, dev = env
    shape = (96, 512, 512)
    Z, Y, X = shape
    o = ph.optics()
    zern = [coefficient_sets(3, seed=21)[2]]
    tf, _ = build(env, [o], zern, shape, 7)
    spec = B.tf_views(tf, 1, Z, Y, X, 7)[0].cpu().numpy()
    ref = OO.transfer_functions(dict(o, zernike=zern[0]), shape, OO.KINDS)
    for s, k in enumerate(OO.KINDS):
        mode = ("fluor",) if k == "fluor" else ("phase", "absorption")
        den = np.sqrt(sum(np.linalg.norm(OO.half_spectrum(ref[q])) ** 2 for q in mode))
        assert np.linalg.norm(spec[0, s] - OO.half_spectrum(ref[k])) / den <= TOL, k
