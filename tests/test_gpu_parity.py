"""Parity of the CUDA path (through the C ABI) with the float64 oracle.

Both sides take the same seeded inputs; the GPU result must match the oracle
to a relative L2 error of 1e-4 (the tolerance the workloads fix for float32
reconstructions), element by element at sizes the oracle handles in seconds,
and on sampled outputs or the whole transfer-function bank at the widefield
workload's full size.
"""
import numpy as np
import pytest

import phantom as ph
from conftest import rel_l2
from oracle import dft as OD, model as OM, optics as OO, tiles as OT

pytestmark = pytest.mark.gpu

TOL = 1e-4
KIND_SETS = [("phase",), ("absorption",), ("fluor",), ("phase", "absorption"), ("phase", "fluor"),
             ("absorption", "fluor"), ("phase", "absorption", "fluor")]


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2412_09775_gb300.build import build
    build()
    from paper_2412_09775_gb300 import binding
    return binding, torch, torch.device("cuda:0")


def gpu_tf(env, optics_list, shape, kinds):
    B, torch, dev = env
    Z, Y, X = shape
    n = len(optics_list)
    tf, ws = B.alloc(n, Z, Y, X, kinds, dev)
    B.wo_build_tf(optics_list, n, Z, Y, X, kinds, tf, ws)
    torch.cuda.synchronize()
    spec, stats = B.tf_views(tf, n, Z, Y, X, kinds)
    return tf, ws, spec.cpu().numpy(), stats.cpu().numpy()


def oracle_tf(o, shape, kinds):
    return OO.transfer_functions(o, shape, kinds)


def check_tf(env, optics_list, shape, kinds, tol=TOL):
    tf, ws, spec, stats = gpu_tf(env, optics_list, shape, kinds)
    for t, o in enumerate(optics_list):
        ref = oracle_tf(o, shape, kinds)
        for s, k in enumerate([k for k in OO.KINDS if k in kinds]):
            # error relative to the norm of the TFs of the same contrast mode: the
            # phase TF alone vanishes identically in symmetric cases (one in-focus
            # plane, or a pupil holding only the zero frequency)
            mode = ("fluor",) if k == "fluor" else [q for q in ("phase", "absorption") if q in kinds]
            den = np.sqrt(sum(np.linalg.norm(OO.half_spectrum(ref[q])) ** 2 for q in mode))
            e = np.linalg.norm(spec[t, s] - OO.half_spectrum(ref[k])) / den
            assert e <= tol, (t, k, e)
        lf = [k for k in ("phase", "absorption") if k in kinds]
        if lf:
            tot = sum(np.abs(ref[k]) ** 2 for k in lf)
            assert abs(stats[t, 0] / tot.max() - 1) <= 1e-5
            assert abs(stats[t, 1] / np.sum(tot, axis=0).max() - 1) <= 1e-5
        if "fluor" in kinds:
            tot = np.abs(ref["fluor"]) ** 2
            assert abs(stats[t, 2] / tot.max() - 1) <= 1e-5
            assert abs(stats[t, 3] / np.sum(tot, axis=0).max() - 1) <= 1e-5
    return tf, ws


# ------------------------------------------------------------ TF build
@pytest.mark.parametrize("kinds", KIND_SETS)
def test_tf_kinds(env, kinds):
    check_tf(env, [ph.optics(na_ill=0.8, tilt_x=0.04, tilt_y=-0.02, defocus_um=0.3)], (8, 32, 48), kinds)


@pytest.mark.parametrize("shape", [(16, 64, 64), (12, 48, 96), (6, 24, 32), (1, 16, 16), (2, 4, 4),
                                   (3, 12, 24), (24, 96, 16), (4, 192, 24)])
def test_tf_shapes(env, shape):
    check_tf(env, [ph.optics(na_ill=0.6, tilt_y=0.05, defocus_um=-0.4)], shape, OO.KINDS)


def test_tf_tiles_each_with_own_optics(env):
    optics = ph.tile_optics(np.random.default_rng(3), 3)
    check_tf(env, optics, (8, 32, 32), OO.KINDS)


@pytest.mark.parametrize("shape", [(3, 3, 32), (3, 3, 64), (3, 3, 96), (1, 3, 128), (1, 3, 192), (3, 3, 512),
                                   (1, 3, 256)])
@pytest.mark.parametrize("kinds", [("fluor",), ("absorption",), ("phase", "fluor"), ("phase", "absorption", "fluor")])
def test_tf_odd_rows_per_tile(env, shape, kinds):
    # Z*Y odd with three tiles: consecutive rows that share a transform belong
    # to different tiles, and the batch ends on a row without a partner
    optics = ph.tile_optics(np.random.default_rng(11), 3)
    check_tf(env, optics, shape, kinds)


@pytest.mark.parametrize("shape,kinds", [((3, 3, 64), OO.KINDS), ((2, 16, 128), ("phase",)),
                                         ((1, 3, 512), ("fluor",))])
def test_tf_tiles_with_different_sampling_host_and_device_optics(env, shape, kinds):
    # tiles with their own pixel size (the middle one samples the pupils more
    # coarsely) in batches whose blocks hold rows of several tiles; host and
    # device optics must give the same bank
    B, torch, dev = env
    Z, Y, X = shape
    optics = [ph.optics(na_ill=0.5), ph.optics(na_ill=0.5, pixel_um=0.13, defocus_um=0.2),
              ph.optics(na_ill=0.5, tilt_x=0.05)]
    tf_h, _ = check_tf(env, optics, shape, kinds)
    tf_d, ws_d = B.alloc(3, Z, Y, X, kinds, dev)
    B.wo_build_tf_device(B.optics_tensor(optics, dev), 3, Z, Y, X, kinds, tf_d, ws_d)
    torch.cuda.synchronize()
    # with host optics the y and z passes stop at the batch's largest support
    # radius (+2 bins); compare the columns both paths transform
    r = max((2 * o["na_det"] if "fluor" in kinds else o["na_det"] + min(o["na_det"], o["na_ill"] + np.hypot(
        o["tilt_x"], o["tilt_y"]))) / o["lambda_um"] * X * o["pixel_um"] for o in optics)
    xc = min(X // 2 + 1, int(np.ceil(r)) + 3)
    sh, _ = B.tf_views(tf_h, 3, Z, Y, X, kinds)
    sd, _ = B.tf_views(tf_d, 3, Z, Y, X, kinds)
    assert torch.equal(sd[..., :xc], sh[..., :xc])


def test_tf_point_source_and_pooled_screen_optics(env):
    check_tf(env, [ph.optics(na_ill=0.0)], (8, 32, 32), ("phase", "absorption"))
    check_tf(env, [dict(ph.POOLED_SCREEN_OPTICS, tilt_x=0.03)], (5 + 1, 64, 64), ("phase",))


def test_tf_largest_lengths(env):
    check_tf(env, [ph.optics(na_ill=0.5)], (2, 8, 2048), ("phase", "fluor"))
    check_tf(env, [ph.optics(na_ill=0.5)], (2, 2048, 8), ("absorption",))
    check_tf(env, [ph.optics(na_ill=0.5)], (2048, 8, 8), ("phase",))


# ------------------------------------------------ forward / adjoint
def run_forward(env, tf, ws, kinds, f, bg, shape, n=1):
    B, torch, dev = env
    Z, Y, X = shape
    nc = (1 if set(kinds) & {"phase", "absorption"} else 0) + (1 if "fluor" in kinds else 0)
    fd = torch.from_numpy(np.ascontiguousarray(f, dtype=np.float32)).to(dev)
    dd = torch.empty((n, nc, Z, Y, X), dtype=torch.float32, device=dev)
    B.wo_forward(tf, kinds, fd, bg, dd, n, Z, Y, X, ws)
    return dd.cpu().numpy()


@pytest.mark.parametrize("kinds", KIND_SETS)
def test_forward_and_adjoint(env, kinds):
    B, torch, dev = env
    shape = (8, 32, 48)
    o = ph.optics(na_ill=0.7, tilt_x=-0.03, defocus_um=0.15)
    tf, ws = check_tf(env, [o], shape, kinds)
    modes, props, chans = OM.widefield_system(oracle_tf(o, shape, kinds), kinds)
    f = ph.uniform_volume(5, (1, len(props)) + shape, -0.02, 0.02).astype(np.float32)
    bg = [1.0, 0.3][: len(chans)]
    d = run_forward(env, tf, ws, kinds, f, bg, shape)[0]
    ref = OM.forward(modes, f[0].astype(np.float64), bg)
    b = np.array(bg)[:, None, None, None]
    assert rel_l2(d - b, ref - b) <= TOL
    # adjoint on an arbitrary data stack
    dd = ph.uniform_volume(6, (len(chans),) + shape, 0.5, 1.5).astype(np.float32)
    Z, Y, X = shape
    din = torch.from_numpy(dd[None]).to(dev)
    fo = torch.empty((1, len(props)) + shape, dtype=torch.float32, device=dev)
    B.wo_forward_adjoint(tf, kinds, din, bg, fo, 1, Z, Y, X, ws)
    ref = OM.adjoint(modes, dd.astype(np.float64), bg)
    assert rel_l2(fo.cpu().numpy()[0], ref) <= TOL


# ------------------------------------------------------ reconstruct
def run_recon(env, tf, ws, kinds, d, bg, eta, flag, mode, shape, n=1):
    B, torch, dev = env
    Z, Y, X = shape
    P = len(kinds)
    din = torch.from_numpy(np.ascontiguousarray(d, dtype=np.float32)).to(dev)
    out_shape = (n, P) + ((Z, Y, X) if mode == B.WO_MODE_3D else (Y, X))
    fo = torch.empty(out_shape, dtype=torch.float32, device=dev)
    B.wo_reconstruct(tf, kinds, din, bg, eta, flag, mode, fo, n, Z, Y, X, ws)
    return fo.cpu().numpy()


def test_reconstruct_small_widefield_stack(env):
    """16 x 64 x 64 stack of 20 spheres, forward + 1e-3 noise, phase-only Tikhonov with eta = 1e-3."""
    B = env[0]
    shape = (16, 64, 64)
    o = ph.optics()
    dn = ph.sphere_phantom(1, shape, o)
    tfs = oracle_tf(o, shape, ("phase",))
    modes, _, _ = OM.widefield_system(tfs, ("phase",))
    d = OM.forward(modes, dn[None], [1.0])
    d = (d + ph.gaussian_noise(101, d.shape, 1e-3 * d.mean())).astype(np.float32)
    tf, ws = check_tf(env, [o], shape, ("phase",))
    got = run_recon(env, tf, ws, ("phase",), d[None], None, [1e-3], B.WO_ETA_RELATIVE, B.WO_MODE_3D, shape)
    ref = OM.reconstruct(modes, d.astype(np.float64), 1e-3)
    assert rel_l2(got[0], ref) <= TOL


@pytest.mark.parametrize("kinds,mode", [(("phase",), 0), (("phase",), 1), (("phase", "absorption", "fluor"), 0),
                                        (("phase", "absorption"), 1)])
def test_reconstruct_batch_sharing_one_tf_bank(env, kinds, mode):
    """A batch of independent small stacks (16 x 64 x 64) with the same optics
    reconstructed from one TF bank (wo_reconstruct_shared_tf): every stack
    against the oracle, and bit for bit equal to wo_reconstruct with the bank
    replicated per stack."""
    B, torch, dev = env
    shape = (16, 64, 64)
    Z, Y, X = shape
    n = 5
    o = ph.optics(na_ill=0.8, tilt_x=0.03, defocus_um=0.1)
    tf1, _ = check_tf(env, [o], shape, kinds)
    tfn, ws = B.alloc(n, Z, Y, X, kinds, dev)
    B.wo_build_tf([o] * n, n, Z, Y, X, kinds, tfn, ws)
    modes, props, chans = OM.widefield_system(oracle_tf(o, shape, kinds), kinds)
    d = ph.uniform_volume(21, (n, len(chans)) + shape, 0.9, 1.1).astype(np.float32)
    eta = [1e-3, 2e-3][: len(modes)]
    din = torch.from_numpy(d).to(dev)
    out_shape = (n, len(props)) + ((Z, Y, X) if mode == B.WO_MODE_3D else (Y, X))
    got = torch.empty(out_shape, dtype=torch.float32, device=dev)
    rep = torch.empty_like(got)
    B.wo_reconstruct_shared_tf(tf1, kinds, din, None, eta, B.WO_ETA_RELATIVE, mode, got, n, Z, Y, X, ws)
    B.wo_reconstruct(tfn, kinds, din, None, eta, B.WO_ETA_RELATIVE, mode, rep, n, Z, Y, X, ws)
    got, rep = got.cpu().numpy(), rep.cpu().numpy()
    assert np.array_equal(got, rep)
    if mode == B.WO_MODE_2D:
        modes = OM.widefield_system(OO.plane_tfs(o, shape, kinds), kinds)[0]
    solve = OM.reconstruct if mode == B.WO_MODE_3D else OM.reconstruct_2d
    for t in range(n):
        for m, e in zip(modes, eta):
            r = solve([m], d[t].astype(np.float64), e)
            for p in m["props"]:
                assert rel_l2(got[t, p], r[p]) <= TOL, (t, p)


def test_reconstruct_shared_tf_full_batch(env):
    """The small-stack workload's launch configuration: 4096 stacks of
    16 x 64 x 64 sharing one phase TF bank; the first and last stacks against
    the oracle."""
    B, torch, dev = env
    shape = (16, 64, 64)
    Z, Y, X = shape
    n = 4096
    o = ph.optics()
    tf1, _ = check_tf(env, [o], shape, ("phase",))
    ws = torch.empty(B.wo_workspace_bytes(n, Z, Y, X, ("phase",)), dtype=torch.uint8, device=dev)
    modes, _, _ = OM.widefield_system(oracle_tf(o, shape, ("phase",)), ("phase",))
    d = ph.uniform_volume(22, (n, 1) + shape, 0.95, 1.05).astype(np.float32)
    din = torch.from_numpy(d).to(dev)
    got = torch.empty((n, 1) + shape, dtype=torch.float32, device=dev)
    B.wo_reconstruct_shared_tf(tf1, ("phase",), din, None, [1e-3], B.WO_ETA_RELATIVE, B.WO_MODE_3D, got, n, Z, Y, X,
                               ws)
    for t in (0, n - 1):
        ref = OM.reconstruct(modes, d[t].astype(np.float64), 1e-3)
        assert rel_l2(got[t, 0].cpu().numpy(), ref[0]) <= TOL, t


@pytest.mark.parametrize("kinds", KIND_SETS)
@pytest.mark.parametrize("bg,flag", [(None, 0), ("given", 0), ("given", 1)])
def test_reconstruct_3d(env, kinds, bg, flag):
    B = env[0]
    shape = (12, 48, 32)
    o = ph.optics(na_ill=0.75, tilt_y=0.04, defocus_um=-0.2)
    tf, ws = check_tf(env, [o], shape, kinds)
    modes, props, chans = OM.widefield_system(oracle_tf(o, shape, kinds), kinds)
    d = ph.uniform_volume(9, (len(chans),) + shape, 0.9, 1.1).astype(np.float32)
    b = [1.0, 0.8][: len(chans)] if bg == "given" else None
    n_modes = len(modes)
    eta = [1e-3, 3e-3][:n_modes] if flag == 0 else [0.5, 2e-4][:n_modes]
    got = run_recon(env, tf, ws, kinds, d[None], b, eta, flag, B.WO_MODE_3D, shape)[0]
    ref = np.zeros_like(got, dtype=np.float64)
    for m, e in zip(modes, eta):
        r = OM.reconstruct([m], d.astype(np.float64), e, background=b, relative=(flag == 0))
        for p in m["props"]:
            ref[p] = r[p]
    for p in range(len(props)):
        assert rel_l2(got[p], ref[p]) <= TOL, (props[p], rel_l2(got[p], ref[p]))


@pytest.mark.parametrize("kinds", [("phase",), ("phase", "absorption"), ("phase", "absorption", "fluor"),
                                   ("fluor",)])
@pytest.mark.parametrize("bg,flag", [(None, 0), ("given", 1)])
def test_reconstruct_2d_phase_from_defocus(env, kinds, bg, flag):
    B = env[0]
    shape = (8, 64, 48)
    o = ph.optics(na_ill=0.5, tilt_x=0.06, defocus_um=0.4)
    tf, ws = check_tf(env, [o], shape, kinds)
    plane = OO.plane_tfs(o, shape, kinds)
    modes, props, chans = OM.widefield_system(plane, kinds)
    d = ph.uniform_volume(12, (len(chans),) + shape, 0.9, 1.1).astype(np.float32)
    b = [1.0, 0.8][: len(chans)] if bg == "given" else None
    eta = [1e-3, 1e-2][: len(modes)] if flag == 0 else [0.3, 1e-3][: len(modes)]
    got = run_recon(env, tf, ws, kinds, d[None], b, eta, flag, B.WO_MODE_2D, shape)[0]
    ref = np.zeros(got.shape)
    for m, e in zip(modes, eta):
        r = OM.reconstruct_2d([m], d.astype(np.float64), e, background=b, relative=(flag == 0))
        for p in m["props"]:
            ref[p] = r[p]
    for p in range(len(props)):
        assert rel_l2(got[p], ref[p]) <= TOL, (props[p], rel_l2(got[p], ref[p]))


@pytest.mark.parametrize("shape", [(1, 32, 32), (2, 4, 4), (3, 24, 96), (16, 16, 2048 // 8)])
def test_reconstruct_edge_shapes(env, shape):
    B = env[0]
    kinds = ("phase", "absorption", "fluor")
    o = ph.optics(na_ill=0.6)
    tf, ws = check_tf(env, [o], shape, kinds)
    modes, props, chans = OM.widefield_system(oracle_tf(o, shape, kinds), kinds)
    d = ph.uniform_volume(13, (2,) + shape, 0.9, 1.1).astype(np.float32)
    got = run_recon(env, tf, ws, kinds, d[None], [1.0, 1.0], [1e-2, 1e-2], 0, B.WO_MODE_3D, shape)[0]
    ref = np.zeros(got.shape)
    for m in modes:
        r = OM.reconstruct([m], d.astype(np.float64), 1e-2, background=[1.0, 1.0])
        for p in m["props"]:
            ref[p] = r[p]
    assert rel_l2(got, ref) <= TOL


def test_exact_recovery_band_limited_fp32(env):
    """Noiseless band-limited object, eta_rel = 1e-6: float32 recovery within 1e-4.

    The data carry no background: with a background of 1 the float32 rounding
    of the input (6e-8) is itself amplified by the near-singular inverse and
    dominates, whatever computes the reconstruction."""
    B = env[0]
    shape = (16, 64, 64)
    o = ph.optics()
    tfs = oracle_tf(o, shape, ("phase",))
    H = tfs["phase"]
    mask = np.abs(H) ** 2 >= 0.05 * np.max(np.abs(H) ** 2)
    f = np.real(np.fft.ifftn(np.fft.fftn(ph.uniform_volume(2, shape, -1, 1)) * mask)) * 0.01
    modes, _, _ = OM.widefield_system(tfs, ("phase",))
    d = OM.forward(modes, f[None], [0.0]).astype(np.float32)
    tf, ws = check_tf(env, [o], shape, ("phase",))
    got = run_recon(env, tf, ws, ("phase",), d[None], [0.0], [1e-6], 0, B.WO_MODE_3D, shape)[0, 0]
    assert rel_l2(got, f) <= TOL


# ------------------------------------------------------------ tiles
def test_tiles_gather_blend(env):
    B, torch, dev = env
    ty, tx, core, halo, Z = 2, 3, 32, 8, 4
    field = ph.uniform_volume(4, (Z, ty * core, tx * core)).astype(np.float32)
    E = core + 2 * halo
    fd = torch.from_numpy(field).to(dev)
    td = torch.empty((ty * tx, Z, E, E), dtype=torch.float32, device=dev)
    B.wo_tile_gather(fd, Z, ty, tx, core, halo, td)
    ref = OT.gather(field, ty, tx, core, halo)
    assert np.array_equal(td.cpu().numpy(), ref)  # a pure copy: bit exact
    td2 = torch.from_numpy(ph.uniform_volume(5, ref.shape).astype(np.float32)).to(dev)
    out = torch.empty_like(fd)
    B.wo_tile_blend(td2, Z, ty, tx, core, halo, out)
    ref2 = OT.blend(td2.cpu().numpy().astype(np.float64), ty, tx, core, halo)
    assert np.abs(out.cpu().numpy() - ref2).max() <= 1e-6


def test_shift_variant_pipeline_four_tiles(env):
    """Field 48 x 256 x 256, 2 x 2 tiles of 128-px cores with 32-px halos
    (48 x 192 x 192 tiles, each with its own theta), phase reconstruction, blend."""
    B, torch, dev = env
    ty, tx, core, halo, Z = 2, 2, 128, 32, 48
    E = core + 2 * halo
    o_list = ph.tile_optics(np.random.default_rng(7), ty * tx)
    field = (1.0 + ph.sphere_phantom(3, (Z, ty * core, tx * core), n_spheres=150)
             + ph.gaussian_noise(4, (Z, ty * core, tx * core), 1e-3)).astype(np.float32)
    fd = torch.from_numpy(field).to(dev)
    td = torch.empty((ty * tx, Z, E, E), dtype=torch.float32, device=dev)
    B.wo_tile_gather(fd, Z, ty, tx, core, halo, td)
    tf, ws = B.alloc(ty * tx, Z, E, E, ("phase",), dev)
    B.wo_build_tf(o_list, ty * tx, Z, E, E, ("phase",), tf, ws)
    rec = torch.empty_like(td)
    B.wo_reconstruct(tf, ("phase",), td, None, [1e-3], B.WO_ETA_RELATIVE, B.WO_MODE_3D, rec, ty * tx, Z, E, E, ws)
    out = torch.empty_like(fd)
    B.wo_tile_blend(rec, Z, ty, tx, core, halo, out)
    got = out.cpu().numpy()
    tiles = OT.gather(field.astype(np.float64), ty, tx, core, halo)
    rec_ref = np.empty_like(tiles)
    for t, o in enumerate(o_list):
        modes, _, _ = OM.widefield_system(oracle_tf(o, (Z, E, E), ("phase",)), ("phase",))
        rec_ref[t] = OM.reconstruct(modes, tiles[t][None], 1e-3)[0]
    ref = OT.blend(rec_ref, ty, tx, core, halo)
    assert rel_l2(got, ref) <= TOL


# --------------------------------------------- full widefield workload
def test_widefield_full_size(env):
    """96 x 512 x 512, phase + absorption + fluorescence: the whole TF bank
    against the oracle, and the reconstruction at sampled frequencies (direct
    DFT coefficients of the GPU's input and output)."""
    B, torch, dev = env
    shape = (96, 512, 512)
    Z, Y, X = shape
    kinds = ("phase", "absorption", "fluor")
    o = ph.optics()
    tf, ws, spec, stats = gpu_tf(env, [o], shape, kinds)
    ref = oracle_tf(o, shape, kinds)
    for s, k in enumerate(kinds):
        assert rel_l2(spec[0, s], OO.half_spectrum(ref[k])) <= TOL, k
    tot_lf = np.abs(ref["phase"]) ** 2 + np.abs(ref["absorption"]) ** 2
    assert abs(stats[0, 0] / tot_lf.max() - 1) <= 1e-5
    # input stacks: brightfield-like and fluorescence-like volumes from a phantom
    vols = ph.widefield_phantom(2, shape, o, n_spheres=300, n_shells=30)
    d = np.stack([1.0 + vols["dn"] + ph.gaussian_noise(5, shape, 1e-3),
                  0.2 + 0.05 * vols["rho"] + ph.gaussian_noise(6, shape, 1e-3)]).astype(np.float32)
    eta = [1e-3, 1e-3]
    got = run_recon(env, tf, ws, kinds, d[None], None, eta, 0, B.WO_MODE_3D, shape)[0]
    eta_lf = eta[0] * tot_lf.max()
    eta_fl = eta[1] * (np.abs(ref["fluor"]) ** 2).max()
    rng = np.random.default_rng(0)
    ks = [(0, 0, 0), (1, 5, 7)] + [tuple(int(rng.integers(0, n)) for n in shape) for _ in range(4)]
    for k in ks:
        D = [OD.dft_coefficient(d[c].astype(np.float64), k) for c in range(2)]
        if k == (0, 0, 0):
            D = [0.0, 0.0]  # background = channel mean
        H = [ref[kk][k] for kk in kinds]
        Hm = np.array([[H[0], H[1]]])
        F_lf = OM.solve_normal(Hm, np.array([D[0]]), eta_lf)
        F_fl = np.conj(H[2]) * D[1] / (abs(H[2]) ** 2 + eta_fl)
        want = [F_lf[0], F_lf[1], F_fl]
        for p in range(3):
            have = OD.dft_coefficient(got[p].astype(np.float64), k)
            # typical coefficient magnitude sqrt(N) * rms(f): 1e-4 of it is the
            # per-coefficient analogue of a 1e-4 relative L2 error
            typical = np.sqrt(got[p].size) * np.sqrt(np.mean(got[p].astype(np.float64) ** 2))
            assert abs(have - want[p]) <= 1e-4 * typical + 1e-4 * abs(want[p]), (k, p, have, want[p], typical)


def test_launch_counter_and_profiler(env):
    B, torch, dev = env
    shape = (8, 32, 32)
    B.wo_profile_enable(True)
    n0 = B.wo_launch_count()
    check_tf(env, [ph.optics()], shape, ("phase",))
    prof = B.wo_profile_read()
    B.wo_profile_enable(False)
    assert B.wo_launch_count() - n0 >= 5
    assert {"tf_pupil_record", "tf_arms", "tf_psf_rows", "tf_ypass", "tf_zpass"} <= set(prof)
    assert all(ms > 0 for _, ms in prof.values())


# ------------------------------------------- device optics, graph capture
def test_build_tf_device_matches_host_and_flags_bad_tiles(env):
    B, torch, dev = env
    shape = (8, 32, 48)
    Z, Y, X = shape
    good = ph.tile_optics(np.random.default_rng(5), 2)
    bad = dict(good[0], na_det=1.4)          # NA_det > n: invalid
    under = dict(good[0], pixel_um=0.2)       # pupil correlation aliases
    optics = [good[0], bad, good[1], under]
    tf_h, ws = B.alloc(2, Z, Y, X, OO.KINDS, dev)
    B.wo_build_tf(good, 2, Z, Y, X, OO.KINDS, tf_h, ws)
    tf_d, ws4 = B.alloc(4, Z, Y, X, OO.KINDS, dev)
    B.wo_build_tf_device(B.optics_tensor(optics, dev), 4, Z, Y, X, OO.KINDS, tf_d, ws4)
    torch.cuda.synchronize()
    sh, sth = B.tf_views(tf_h, 2, Z, Y, X, OO.KINDS)
    sd, std_ = B.tf_views(tf_d, 4, Z, Y, X, OO.KINDS)
    assert torch.equal(sd[0], sh[0]) and torch.equal(sd[2], sh[1])
    assert torch.count_nonzero(sd[1]) == 0 and torch.count_nonzero(sd[3]) == 0
    status = std_.view(torch.int32)[:, 4].cpu().tolist()
    assert status == [0, B.STATUS_CODES["WO_ERR_OPTICS"], 0, B.STATUS_CODES["WO_ERR_UNDERSAMPLED"]]
    # reconstruction of a flagged tile is zero, the others match the host bank
    d = torch.from_numpy(ph.uniform_volume(3, (4, 2) + shape, 0.9, 1.1).astype(np.float32)).to(dev)
    out = torch.empty((4, 3) + shape, dtype=torch.float32, device=dev)
    B.wo_reconstruct(tf_d, OO.KINDS, d, None, [1e-3, 1e-3], 0, 0, out, 4, Z, Y, X, ws4)
    ref = torch.empty((2, 3) + shape, dtype=torch.float32, device=dev)
    B.wo_reconstruct(tf_h, OO.KINDS, d[[0, 2]].contiguous(), None, [1e-3, 1e-3], 0, 0, ref, 2, Z, Y, X, ws)
    torch.cuda.synchronize()
    assert torch.count_nonzero(out[1]) == 0 and torch.count_nonzero(out[3]) == 0
    assert torch.equal(out[0], ref[0]) and torch.equal(out[2], ref[1])


def test_tile_pipeline_under_cuda_graph(env):
    """gather -> TF build (device optics) -> reconstruct -> blend captured once
    and replayed; the replay equals the eager calls and follows new inputs."""
    B, torch, dev = env
    ty, tx, core, halo, Z = 2, 2, 32, 8, 12
    E = core + 2 * halo
    n = ty * tx
    optics = B.optics_tensor(ph.tile_optics(np.random.default_rng(9), n), dev)
    field = torch.from_numpy((1.0 + ph.sphere_phantom(2, (Z, ty * core, tx * core), n_spheres=30)).astype(np.float32)).to(dev)
    tiles = torch.empty((n, Z, E, E), dtype=torch.float32, device=dev)
    tf, ws = B.alloc(n, Z, E, E, ("phase",), dev)
    rec = torch.empty_like(tiles)
    out = torch.empty_like(field)

    def pipeline():
        B.wo_tile_gather(field, Z, ty, tx, core, halo, tiles)
        B.wo_build_tf_device(optics, n, Z, E, E, ("phase",), tf, ws)
        B.wo_reconstruct(tf, ("phase",), tiles, None, [1e-3], 0, 0, rec, n, Z, E, E, ws)
        B.wo_tile_blend(rec, Z, ty, tx, core, halo, out)

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        pipeline()  # warm-up outside capture (one-time kernel attributes)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    eager = out.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        pipeline()
    out.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(out, eager)
    field.mul_(1.5).add_(0.1)
    g.replay()
    with torch.cuda.stream(s):
        pipeline()
    torch.cuda.synchronize()
    graph_out = out.clone()
    with torch.cuda.stream(s):
        pipeline()
    torch.cuda.synchronize()
    assert torch.equal(graph_out, out) and not torch.equal(graph_out, eager)


# ------------------------------------------------ multi-aperture fusion
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("bg,flag", [(None, 0), ("given", 1)])
def test_nine_aperture_fusion(env, mode, bg, flag):
    """C = 9 illumination apertures fused into one phase volume (3D) or one
    thin-object phase image (2D): the GPU matches the oracle's C x 1
    multi-channel Tikhonov solve, for 2 tiles at once."""
    B, torch, dev = env
    C, n = 9, 2
    Z, Y, X = (12, 48, 64)
    apertures = ph.aperture_optics(C, ring_na=0.6, na_ill=0.15)
    optics = []
    for t in range(n):
        optics += [dict(o, defocus_um=0.2 * t) for o in apertures]
    tf, _ = B.alloc(n * C, Z, Y, X, ("phase",), dev)
    ws_build = B.alloc(n * C, Z, Y, X, ("phase",), dev)[1]
    B.wo_build_tf(optics, n * C, Z, Y, X, ("phase",), tf, ws_build)
    rng_f = ph.sphere_phantom(5, (Z, Y, X), ph.optics(), n_spheres=10)
    d = np.zeros((n, C, Z, Y, X))
    want = []
    for t in range(n):
        if mode == 0:
            H = [OO.transfer_functions(optics[t * C + c], (Z, Y, X), ("phase",))["phase"] for c in range(C)]
            m = [dict(channels=list(range(C)), props=[0], H=[[h] for h in H])]
            dt = OM.forward(m, rng_f[None], [1.0] * C)
        else:
            Hj = [OO.plane_tfs(optics[t * C + c], (Z, Y, X), ("phase",))["phase"] for c in range(C)]
            f2 = ph.thin_phantom(7 + t, (Y, X), ph.optics(), n_spheres=8)
            dt = np.stack([1.0 + np.real(np.fft.ifft2(h * np.fft.fft2(f2)[None], axes=(1, 2))) for h in Hj])
            m = [dict(channels=list(range(C)), props=[0], H=[[h] for h in Hj])]
        dt = dt + ph.gaussian_noise(30 + t, dt.shape, 1e-3)
        d[t] = dt.astype(np.float32)
        b = None if bg is None else [1.0] * C
        eta = 1e-3 if flag == 0 else 1e-2
        if mode == 0:
            want.append(OM.reconstruct(m, d[t], eta, background=b, relative=(flag == 0))[0])
        else:
            want.append(OM.reconstruct_2d(m, d[t], eta, background=b, relative=(flag == 0))[0])
    wsb = B.wo_fused_workspace_bytes(C, n, Z, Y, X)
    ws = torch.empty(wsb, dtype=torch.uint8, device=dev)
    out_shape = (n, Z, Y, X) if mode == 0 else (n, Y, X)
    f = torch.empty(out_shape, dtype=torch.float32, device=dev)
    B.wo_reconstruct_fused(tf, C, torch.tensor(d, dtype=torch.float32, device=dev),
                           None if bg is None else [1.0] * C, 1e-3 if flag == 0 else 1e-2, flag, mode, f,
                           n, Z, Y, X, ws)
    got = f.cpu().numpy()
    for t in range(n):
        assert rel_l2(got[t], want[t]) <= TOL, t


# ------------------------------------------------ column engines and the autotuner
@pytest.mark.parametrize("engine", [1, 2])
@pytest.mark.parametrize("shape", [(8, 64, 48), (6, 128, 64), (4, 192, 32), (4, 256, 32), (2, 512, 16),
                                   (6, 96, 48), (4, 48, 64), (4, 32, 32)])
def test_column_engines_match_oracle(env, shape, engine):
    """Forward + reconstruction with the y transforms pinned to each engine
    (shared-memory Stockham, hybrid register-resident) match the oracle."""
    B, torch, dev = env
    Z, Y, X = shape
    try:
        B.wo_schedule_set(B.WO_PASS_COLS, Y, engine)
        assert B.wo_schedule_get(B.WO_PASS_COLS, Y) == engine
        o = ph.optics(na_ill=0.6, defocus_um=0.2)
        kinds = ("phase", "absorption")
        tf, ws = check_tf(env, [o], shape, kinds)
        f = ph.uniform_volume(3, (2,) + shape, -0.01, 0.01)
        tfs = OO.transfer_functions(o, shape, kinds)
        modes, _, _ = OM.widefield_system(tfs, kinds)
        want = OM.forward(modes, f, [1.0])
        d = torch.empty((1, 1) + shape, dtype=torch.float32, device=dev)
        B.wo_forward(tf, kinds, torch.tensor(f[None], dtype=torch.float32, device=dev), [1.0], d, 1, Z, Y, X, ws)
        got = d.cpu().numpy()[0]
        assert rel_l2(got[0] - 1.0, want[0] - 1.0) <= TOL
    finally:
        B.wo_schedule_set(B.WO_PASS_COLS, Y, 0)


def test_autotune_keeps_results(env):
    """The autotuner times the engines on the workspace and records one per
    length; the reconstruction afterwards matches the oracle as before."""
    B, torch, dev = env
    Z, Y, X = 16, 128, 64
    o = ph.optics(na_ill=0.7)
    kinds = ("phase",)
    tf, ws = B.alloc(2, Z, Y, X, kinds, dev)
    try:
        B.wo_autotune(2, Z, Y, X, kinds, ws)
        assert B.wo_schedule_get(B.WO_PASS_COLS, Y) in (1, 2)
        assert B.wo_schedule_get(B.WO_PASS_COLS, Z) in (1, 2)
        B.wo_build_tf([o, o], 2, Z, Y, X, kinds, tf, ws)
        d = 1.0 + 0.01 * ph.uniform_volume(9, (Z, Y, X))
        out = torch.empty((2, Z, Y, X), dtype=torch.float32, device=dev)
        dd = torch.tensor(np.stack([d, d])[:, None], dtype=torch.float32, device=dev)
        B.wo_reconstruct(tf, kinds, dd, None, 1e-3, 0, 0, out, 2, Z, Y, X, ws)
        modes, _, _ = OM.widefield_system(OO.transfer_functions(o, (Z, Y, X), kinds), kinds)
        want = OM.reconstruct(modes, d[None].astype(np.float32).astype(np.float64), 1e-3)[0]
        got = out.cpu().numpy()
        assert rel_l2(got[0], want) <= TOL and rel_l2(got[1], want) <= TOL
    finally:
        B.wo_schedule_set(B.WO_PASS_COLS, Y, 0)
        B.wo_schedule_set(B.WO_PASS_COLS, Z, 0)


def test_shift_variant_field_full_size(env):
    """The shift-variant workload at its full size, in the calls the bench
    times: a 48 x 2048 x 2048 field cut into 256 tiles of 48 x 192 x 192
    (128-px cores, 32-px halos), each tile's TF built from its own optics on
    the device, reconstructed, and blended back.  Checked on samples the
    oracle computes one by one: three whole tiles (gather bit for bit, the
    reconstruction within 1e-4), and blended field values at pixels on tile
    cores, overlaps and the field's edges."""
    B, torch, dev = env
    ty = tx = 16
    core, halo = 128, 32
    Z, E = 48, core + 2 * halo
    n = ty * tx
    o_list = ph.tile_optics(np.random.default_rng(3), n)
    field_np = (1.0 + ph.uniform_volume(21, (Z, ty * core, tx * core), -0.01, 0.01)).astype(np.float32)
    field = torch.from_numpy(field_np).to(dev)
    optics = B.optics_tensor(o_list, dev)
    tiles = torch.empty((n, Z, E, E), dtype=torch.float32, device=dev)
    rec = torch.empty_like(tiles)
    out = torch.empty_like(field)
    tf, ws = B.alloc(n, Z, E, E, ("phase",), dev)
    B.wo_tile_gather(field, Z, ty, tx, core, halo, tiles)
    B.wo_build_tf_device(optics, n, Z, E, E, ("phase",), tf, ws)
    B.wo_reconstruct(tf, ("phase",), tiles, None, [1e-3], B.WO_ETA_RELATIVE, B.WO_MODE_3D, rec, n, Z, E, E, ws)
    B.wo_tile_blend(rec, Z, ty, tx, core, halo, out)
    # the in-place reconstruction the bench's step runs gives the same tiles, bit for bit
    rec2 = torch.empty_like(rec)
    B.wo_reconstruct_field_tiles(tf, ("phase",), field, Z, ty, tx, core, halo, None, [1e-3], B.WO_ETA_RELATIVE,
                                 B.WO_MODE_3D, rec2, ws)
    assert torch.equal(rec2, rec)
    del rec2
    torch.cuda.synchronize()
    for t in (0, 17, 255):  # a corner, an interior tile, the opposite corner
        y0, x0 = OT.tile_origin(t // tx, t % tx, core, halo)
        ys = OT.mirror(np.arange(y0, y0 + E), ty * core)
        xs = OT.mirror(np.arange(x0, x0 + E), tx * core)
        want_tile = field_np[:, ys][:, :, xs]
        got_tile = tiles[t].cpu().numpy()
        assert np.array_equal(got_tile, want_tile), t
        modes, _, _ = OM.widefield_system(OO.transfer_functions(o_list[t], (Z, E, E), ("phase",)), ("phase",))
        want = OM.reconstruct(modes, want_tile[None].astype(np.float64), 1e-3)[0]
        assert rel_l2(rec[t].cpu().numpy(), want) <= TOL, t
    w1 = OT.ramp(E, halo)
    for z, y, x in ((0, 0, 0), (5, 64, 1000), (17, 127, 128), (31, 160, 96), (47, 2047, 2047), (23, 1024, 900),
                    (40, 96, 2040)):
        acc = wsum = 0.0
        for a in range(ty):
            for b in range(tx):
                y0, x0 = OT.tile_origin(a, b, core, halo)
                if y0 <= y < y0 + E and x0 <= x < x0 + E:
                    wgt = w1[y - y0] * w1[x - x0]
                    acc += wgt * float(rec[a * tx + b, z, y - y0, x - x0].item())
                    wsum += wgt
        got = float(out[z, y, x].item())
        assert abs(got - acc / wsum) <= 1e-6 * max(1.0, abs(acc / wsum)), (z, y, x, got, acc / wsum)


@pytest.mark.parametrize("engine", [1, 2])
@pytest.mark.parametrize("shape", [(4, 8, 64), (6, 12, 96), (4, 16, 128), (8, 6, 192), (4, 8, 256), (3, 4, 384),
                                   (4, 8, 512), (2, 4, 1024)])
def test_row_engines_match_oracle(env, shape, engine):
    """The x passes pinned to each engine (shared-memory rows, register rows):
    forward with backgrounds, adjoint, 3D and 2D reconstruction with the
    channel-mean background, and wo_spectrum, against the oracle."""
    B, torch, dev = env
    Z, Y, X = shape
    n = X // 2
    kinds = OO.KINDS
    try:
        B.wo_schedule_set(B.WO_PASS_ROWS, n, engine)
        assert B.wo_schedule_get(B.WO_PASS_ROWS, n) == engine
        o = ph.optics(na_ill=0.7, tilt_y=0.04, defocus_um=-0.2)
        tf, ws = check_tf(env, [o], shape, kinds)
        modes, props, chans = OM.widefield_system(oracle_tf(o, shape, kinds), kinds)
        f = ph.uniform_volume(9, (1, 3) + shape, -0.02, 0.02).astype(np.float32)
        bg = [1.0, 0.0]
        b = np.array(bg)[:, None, None, None]
        d = run_forward(env, tf, ws, kinds, f, bg, shape)[0]
        assert rel_l2(d - b, OM.forward(modes, f[0].astype(np.float64), bg) - b) <= TOL
        dd = ph.uniform_volume(10, (2,) + shape, 0.5, 1.5).astype(np.float32)
        fo = torch.empty((1, 3) + shape, dtype=torch.float32, device=dev)
        B.wo_forward_adjoint(tf, kinds, torch.from_numpy(dd[None]).to(dev), bg, fo, 1, Z, Y, X, ws)
        assert rel_l2(fo.cpu().numpy()[0], OM.adjoint(modes, dd.astype(np.float64), bg)) <= TOL
        got = run_recon(env, tf, ws, kinds, dd[None], None, [1e-3, 1e-3], B.WO_ETA_RELATIVE, B.WO_MODE_3D, shape)
        ref = OM.reconstruct(modes, dd.astype(np.float64), 1e-3)
        for p in range(3):
            assert rel_l2(got[0, p], ref[p]) <= TOL, p
        pm, _, _ = OM.widefield_system(OO.plane_tfs(o, shape, kinds), kinds)
        got2 = run_recon(env, tf, ws, kinds, dd[None], None, [1e-3, 1e-3], B.WO_ETA_RELATIVE, B.WO_MODE_2D, shape)
        ref2 = OM.reconstruct_2d(pm, dd.astype(np.float64), 1e-3)
        for p in range(3):
            assert rel_l2(got2[0, p], ref2[p]) <= TOL, p
        spec = torch.empty((1, Z, Y, X // 2 + 1), dtype=torch.complex64, device=dev)
        B.wo_spectrum(torch.from_numpy(dd[:1]).to(dev), None, B.WO_MODE_2D, spec, 1, Z, Y, X)
        want = OM.residual_spectrum(dd[0].astype(np.float64), float(np.mean(dd[0])), (1, 2))
        assert rel_l2(spec.cpu().numpy()[0], want[..., : X // 2 + 1]) <= 1e-5
    finally:
        B.wo_schedule_set(B.WO_PASS_ROWS, n, 0)


@pytest.mark.parametrize("shape", [(1, 16, 16), (2, 2048, 8), (2, 8, 2048), (3, 4, 6), (1, 1, 2), (2048, 2, 4)])
def test_operators_at_degenerate_and_largest_lengths(env, shape):
    """Forward, adjoint and 3D reconstruction at a single plane, a single
    row, the smallest transform and the largest lengths of each axis."""
    B, torch, dev = env
    Z, Y, X = shape
    kinds = ("phase", "absorption", "fluor")
    o = ph.optics(na_ill=0.6, tilt_x=0.02, defocus_um=0.1)
    tf, ws = check_tf(env, [o], shape, kinds)
    modes, props, chans = OM.widefield_system(oracle_tf(o, shape, kinds), kinds)
    f = ph.uniform_volume(31, (1, 3) + shape, -0.02, 0.02).astype(np.float32)
    bg = [1.0, 0.0]
    b = np.array(bg)[:, None, None, None]
    d = run_forward(env, tf, ws, kinds, f, bg, shape)[0]
    ref = OM.forward(modes, f[0].astype(np.float64), bg)
    assert rel_l2(d - b, ref - b) <= TOL
    dd = ph.uniform_volume(32, (2,) + shape, 0.5, 1.5).astype(np.float32)
    fo = torch.empty((1, 3) + shape, dtype=torch.float32, device=dev)
    B.wo_forward_adjoint(tf, kinds, torch.from_numpy(dd[None]).to(dev), bg, fo, 1, Z, Y, X, ws)
    assert rel_l2(fo.cpu().numpy()[0], OM.adjoint(modes, dd.astype(np.float64), bg)) <= TOL
    got = run_recon(env, tf, ws, kinds, dd[None], None, [1e-3, 1e-3], B.WO_ETA_RELATIVE, B.WO_MODE_3D, shape)[0]
    want = OM.reconstruct(modes, dd.astype(np.float64), 1e-3)
    # per contrast mode, relative to the mode's norm, plus float32 rounding of
    # data-sized values where the mode's TFs vanish off the zero frequency (a
    # grid holding only the DC inside the pupil, whose data term the channel
    # mean removes, so the exact answer is zero)
    for ps in ((0, 1), (2,)):
        err = np.linalg.norm((got[list(ps)] - want[list(ps)]).ravel())
        tol = TOL * np.linalg.norm(want[list(ps)].ravel()) + 1e-6 * np.linalg.norm(dd.ravel())
        assert err <= tol, (ps, err, tol)
