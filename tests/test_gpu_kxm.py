"""kx-major TF banks (WO_TF_KX_MAJOR) and the plane engine (wo_plane.cu).

* A kx-major bank holds the same transfer functions as the standard bank of
  the same optics, stored [tile][k_x][z][y]: compared through the binding's
  permuted view, for every supported (Z, Y) shape and each kind, with host
  and device optics; and directly against the oracle.
* The field tiles reconstructed through the plane engine (x pass transposing
  into the kx-major spectrum, one y-z-operator pass per plane, x pass
  transposing back) against the five-pass path with the standard bank and
  against the oracle, on border and interior tiles, both background rules.
* The forward model, its adjoint and the 3D reconstruction of plain tiles
  (a bank per tile, and one bank shared by a batch) on the plane engine
  against the same calls with the standard bank and against the oracle.
* The uses such a bank does not serve (the 2D solve, the fused blend) are
  refused with WO_ERR_ARG.
"""
import numpy as np
import pytest

import phantom as ph
from conftest import rel_l2
from oracle import model as OM, optics as OO, tiles as OT

pytestmark = pytest.mark.gpu

TOL = 1e-4      # against the float64 oracle (the parity bound of every GPU path)
ENGINE = 2e-6   # between the two float32 engines (transform order only), relative eta 1e-3


def engine_tol(flag, m3):
    """Bound between the engines' reconstructions.  The Tikhonov inverse
    multiplies a TF error by up to 1 / (2 sqrt(eta)) (times max |H|): with the
    relative eta (eta = 1e-3 max |H|^2) that is 1 / (2 sqrt(1e-3)) whatever
    the TF's scale, with the absolute eta 1e-3 it is max |H| = sqrt(m3) times
    larger, so the two banks' rounding differences (their y and z transforms
    run in different orders) grow by about that factor; twice the bound per
    unit of gain, since the weakly regularised inverse brings a band of
    frequencies near its peak gain, not one."""
    return ENGINE if flag == 0 else 2.0 * ENGINE * max(1.0, float(np.sqrt(m3)))

SHAPES = [(48, 192), (48, 128), (48, 64), (32, 192), (32, 128), (32, 64), (16, 64)]


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2412_09775_gb300.build import build
    build()
    from paper_2412_09775_gb300 import binding
    return binding, torch, torch.device("cuda:0")


def build_bank(env, ol, Z, E, kinds, device_optics):
    B, torch, dev = env
    n = len(ol)
    tf, ws = B.alloc(n, Z, E, E, kinds, dev)
    if device_optics:
        B.wo_build_tf_device(B.optics_tensor(ol, dev), n, Z, E, E, kinds, tf, ws)
    else:
        B.wo_build_tf(ol, n, Z, E, E, kinds, tf, ws)
    assert B.wo_sync_status(ws)[0] == 0
    return tf, ws


@pytest.mark.parametrize("kind", ["phase", "absorption", "fluor"])
@pytest.mark.parametrize("Z,E", SHAPES)
def test_kx_major_bank_equals_standard_bank(env, Z, E, kind):
    B, torch, dev = env
    n = 3
    ol = ph.tile_optics(np.random.default_rng(Z + E), n)
    device_optics = (Z + E) % 3 == 0  # half of the shapes with device-side optics (every column transformed)
    base = B.kinds_mask((kind,))
    tf0, _ = build_bank(env, ol, Z, E, base, device_optics)
    tf1, _ = build_bank(env, ol, Z, E, base | B.WO_TF_KX_MAJOR, device_optics)
    s0, st0 = B.tf_views(tf0, n, Z, E, E, base)
    s1, st1 = B.tf_views(tf1, n, Z, E, E, base | B.WO_TF_KX_MAJOR)
    s0, s1 = s0.cpu().numpy(), s1.cpu().numpy()
    st0, st1 = st0.cpu().numpy(), st1.cpu().numpy()
    for t in range(n):
        assert rel_l2(s1[t], s0[t]) <= ENGINE, t
    w = slice(2, 4) if kind == "fluor" else slice(0, 2)
    assert np.allclose(st1[:, w], st0[:, w], rtol=1e-5, atol=0), (st1[:, w], st0[:, w])
    assert np.array_equal(st1[:, 4:6], st0[:, 4:6])  # optics status, support radius


@pytest.mark.parametrize("Z,E,kinds", [(48, 192, ("phase",)), (32, 64, ("fluor",)), (48, 128, ("absorption",))])
def test_kx_major_bank_matches_oracle(env, Z, E, kinds):
    B, torch, dev = env
    n = 2
    ol = [ph.optics(na_ill=0.6, tilt_y=0.05, defocus_um=-0.4), ph.tile_optics(np.random.default_rng(4), 1)[0]]
    m = B.kinds_mask(kinds) | B.WO_TF_KX_MAJOR
    tf, _ = build_bank(env, ol, Z, E, m, False)
    spec, stats = B.tf_views(tf, n, Z, E, E, m)
    spec, stats = spec.cpu().numpy(), stats.cpu().numpy()
    k = kinds[0]
    for t, o in enumerate(ol):
        ref = OO.transfer_functions(o, (Z, E, E), kinds)[k]
        assert rel_l2(spec[t, 0], OO.half_spectrum(ref)) <= TOL, t
        tot = np.abs(ref) ** 2
        w = 2 if k == "fluor" else 0
        assert abs(stats[t, w] / tot.max() - 1) <= 1e-5
        assert abs(stats[t, w + 1] / np.sum(tot, axis=0).max() - 1) <= 1e-5


def field_case(env, Z, ty, tx, core, halo, kinds, bg, flag, seed, device_optics):
    B, torch, dev = env
    E = core + 2 * halo
    n = ty * tx
    field_np = (1.0 + ph.sphere_phantom(seed, (Z, ty * core, tx * core), n_spheres=40)
                + ph.gaussian_noise(seed + 1, (Z, ty * core, tx * core), 1e-3)).astype(np.float32)
    field = torch.from_numpy(field_np).to(dev)
    ol = ph.tile_optics(np.random.default_rng(seed), n)
    base = B.kinds_mask(kinds)
    eta = [1e-3]
    out = []
    m3 = 0.0
    for m in (base, base | B.WO_TF_KX_MAJOR):
        tf, ws = build_bank(env, ol, Z, E, m, device_optics)
        st = B.tf_views(tf, n, Z, E, E, m)[1].cpu().numpy()
        m3 = max(m3, float(st[:, 2 if kinds == ("fluor",) else 0].max()))
        rec = torch.full((n, 1, Z, E, E), float("nan"), dtype=torch.float32, device=dev)
        B.wo_reconstruct_field_tiles(tf, m, field, Z, ty, tx, core, halo, bg, eta, flag, B.WO_MODE_3D, rec, ws)
        assert B.wo_sync_status(ws)[0] == 0
        out.append(rec.cpu().numpy()[:, 0])
    return field_np, ol, out[0], out[1], m3


@pytest.mark.parametrize("geom", [(48, 2, 2, 128, 32), (48, 2, 3, 96, 16), (32, 3, 2, 48, 8), (32, 2, 2, 160, 16)])
@pytest.mark.parametrize("bg,flag", [(None, 0), ([1.0], 1)])
def test_field_tiles_plane_engine(env, geom, bg, flag):
    """Plane engine against the five passes (every tile) and the oracle (a
    corner tile and the last tile)."""
    B, torch, dev = env
    Z, ty, tx, core, halo = geom
    E = core + 2 * halo
    field_np, ol, want, got, m3 = field_case(env, Z, ty, tx, core, halo, ("phase",), bg, flag, 11 + core,
                                             core % 3 == 0)
    assert np.all(np.isfinite(got))
    for t in range(ty * tx):
        assert rel_l2(got[t], want[t]) <= engine_tol(flag, m3), (t, m3)
    tiles = OT.gather(field_np.astype(np.float64), ty, tx, core, halo)
    for t in (0, ty * tx - 1):
        modes, _, _ = OM.widefield_system(OO.transfer_functions(ol[t], (Z, E, E), ("phase",)), ("phase",))
        ref = OM.reconstruct(modes, tiles[t][None], 1e-3, background=bg, relative=(flag == 0))[0]
        assert rel_l2(got[t], ref) <= TOL, t


@pytest.mark.parametrize("kinds", [("absorption",), ("fluor",)])
def test_field_tiles_plane_engine_other_kinds(env, kinds):
    B, torch, dev = env
    Z, ty, tx, core, halo = 32, 2, 2, 48, 8
    E = core + 2 * halo
    field_np, ol, want, got, _ = field_case(env, Z, ty, tx, core, halo, kinds, None, 0, 5, False)
    tiles = OT.gather(field_np.astype(np.float64), ty, tx, core, halo)
    for t in range(ty * tx):
        assert rel_l2(got[t], want[t]) <= ENGINE, t
        modes, _, _ = OM.widefield_system(OO.transfer_functions(ol[t], (Z, E, E), kinds), kinds)
        ref = OM.reconstruct(modes, tiles[t][None], 1e-3)[0]
        assert rel_l2(got[t], ref) <= TOL, t


def test_field_workload_tiles_plane_engine(env):
    """The field workload's tile geometry (48 x 192 x 192 tiles, 128-px cores,
    32-px halos) on a 4 x 4 grid with device optics: every tile against the
    five passes, an interior tile against the oracle."""
    B, torch, dev = env
    Z, ty, tx, core, halo = 48, 4, 4, 128, 32
    E = core + 2 * halo
    field_np, ol, want, got, _ = field_case(env, Z, ty, tx, core, halo, ("phase",), None, 0, 3, True)
    for t in range(ty * tx):
        assert rel_l2(got[t], want[t]) <= ENGINE, t
    tiles = OT.gather(field_np.astype(np.float64), ty, tx, core, halo)
    t = 5
    modes, _, _ = OM.widefield_system(OO.transfer_functions(ol[t], (Z, E, E), ("phase",)), ("phase",))
    ref = OM.reconstruct(modes, tiles[t][None], 1e-3)[0]
    assert rel_l2(got[t], ref) <= TOL


@pytest.mark.parametrize("Z,E,n", [(16, 64, 5), (32, 128, 2), (48, 192, 3)])
def test_operators_on_tiles_plane_engine(env, Z, E, n):
    """wo_forward (with a background), wo_forward_adjoint, wo_reconstruct
    (relative and absolute eta) and wo_reconstruct_shared_tf on plain tiles
    with a kx-major bank: against the standard bank (every tile) and the
    oracle (the first tile)."""
    B, torch, dev = env
    ol = ph.tile_optics(np.random.default_rng(Z + n), n)
    base = B.WO_TF_PHASE
    kx = base | B.WO_TF_KX_MAJOR
    tfs, wss = build_bank(env, ol, Z, E, base, False)
    tfk, wsk = build_bank(env, ol, Z, E, kx, False)
    m3 = float(B.tf_views(tfs, n, Z, E, E, base)[1][:, 0].max())
    f = torch.from_numpy(ph.uniform_volume(3, (n, 1, Z, E, E), -0.02, 0.02).astype(np.float32)).to(dev)
    d = torch.from_numpy((1.0 + ph.uniform_volume(4, (n, Z, E, E), -0.02, 0.02)).astype(np.float32)).to(dev)

    def both(fn):
        outs = []
        for tf, ws, m in ((tfs, wss, base), (tfk, wsk, kx)):
            outs.append(fn(tf, ws, m))
            assert B.wo_sync_status(ws)[0] == 0
        return outs[0].cpu().numpy(), outs[1].cpu().numpy()

    def fwd(tf, ws, m):
        out = torch.full((n, Z, E, E), float("nan"), device=dev)
        B.wo_forward(tf, m, f, [1.0], out, n, Z, E, E, ws)
        return out

    def adj(tf, ws, m):
        out = torch.full((n, 1, Z, E, E), float("nan"), device=dev)
        B.wo_forward_adjoint(tf, m, d, [1.0], out, n, Z, E, E, ws)
        return out

    def rec(flag, bg):
        def run(tf, ws, m):
            out = torch.full((n, 1, Z, E, E), float("nan"), device=dev)
            B.wo_reconstruct(tf, m, d, bg, [1e-3], flag, B.WO_MODE_3D, out, n, Z, E, E, ws)
            return out
        return run

    modes, _, _ = OM.widefield_system(OO.transfer_functions(ol[0], (Z, E, E), ("phase",)), ("phase",))
    want, got = both(fwd)
    for t in range(n):
        assert rel_l2(got[t] - 1.0, want[t] - 1.0) <= ENGINE, ("forward", t)
    ref = OM.forward(modes, f[0].cpu().numpy().astype(np.float64), [1.0])[0]
    assert rel_l2(got[0] - 1.0, ref - 1.0) <= TOL
    want, got = both(adj)
    for t in range(n):
        assert rel_l2(got[t], want[t]) <= ENGINE, ("adjoint", t)
    ref = OM.adjoint(modes, d[0:1].cpu().numpy().astype(np.float64), [1.0])[0]
    assert rel_l2(got[0, 0], ref) <= TOL
    for flag, bg in ((0, None), (1, [1.0])):
        want, got = both(rec(flag, bg))
        # white-noise data: unlike the phantoms above, every frequency near the
        # inverse's peak gain carries signal, so twice the phantoms' bound
        for t in range(n):
            assert rel_l2(got[t], want[t]) <= 2.0 * engine_tol(flag, m3), ("reconstruct", flag, t)
        ref = OM.reconstruct(modes, d[0:1].cpu().numpy().astype(np.float64), 1e-3, background=bg,
                             relative=(flag == 0))[0]
        assert rel_l2(got[0, 0], ref) <= TOL, ("reconstruct", flag)
    # one bank (tile 0's) shared by the whole batch
    tf1s, ws1s = build_bank(env, ol[:1], Z, E, base, False)
    tf1k, ws1k = build_bank(env, ol[:1], Z, E, kx, False)
    outs = []
    for tf, m in ((tf1s, base), (tf1k, kx)):
        ws = torch.empty(B.wo_workspace_bytes(n, Z, E, E, m), dtype=torch.uint8, device=dev)
        ws[:256].zero_()
        out = torch.full((n, 1, Z, E, E), float("nan"), device=dev)
        B.wo_reconstruct_shared_tf(tf, m, d, None, [1e-3], 0, B.WO_MODE_3D, out, n, Z, E, E, ws)
        assert B.wo_sync_status(ws)[0] == 0
        outs.append(out.cpu().numpy())
    for t in range(n):
        assert rel_l2(outs[1][t], outs[0][t]) <= 2.0 * ENGINE, ("shared", t)  # white-noise data, as above
    ref = OM.reconstruct(modes, d[n - 1:n].cpu().numpy().astype(np.float64), 1e-3)[0]
    assert rel_l2(outs[1][n - 1, 0], ref) <= TOL


def test_kx_major_bank_refused_elsewhere(env):
    B, torch, dev = env
    Z, ty, tx, core, halo = 32, 2, 2, 48, 8
    E = core + 2 * halo
    n = ty * tx
    m = B.WO_TF_PHASE | B.WO_TF_KX_MAJOR
    ol = ph.tile_optics(np.random.default_rng(2), n)
    tf, ws = build_bank(env, ol, Z, E, m, False)
    field = torch.ones((Z, ty * core, tx * core), dtype=torch.float32, device=dev)
    tiles = torch.ones((n, Z, E, E), dtype=torch.float32, device=dev)
    out = torch.empty((n, 1, Z, E, E), dtype=torch.float32, device=dev)
    calls = [
        lambda: B.wo_reconstruct(tf, m, tiles, None, [1e-3], 0, B.WO_MODE_2D, out[:, :, 0].contiguous(), n, Z, E,
                                 E, ws),
        lambda: B.wo_reconstruct_field_tiles(tf, m, field, Z, ty, tx, core, halo, None, [1e-3], 0, B.WO_MODE_2D,
                                             out[:, :, 0].contiguous(), ws),
        lambda: B.wo_restore_field(tf, m, field, Z, ty, tx, core, halo, None, [1e-3], 0, B.WO_MODE_3D,
                                   torch.empty_like(field), ws),
    ]
    for c in calls:
        with pytest.raises(B.WoError) as e:
            c()
        assert e.value.status == B.STATUS_CODES["WO_ERR_ARG"]
    assert B.wo_sync_status(ws)[0] == 0


def test_tf_outside_support_is_never_read(env):
    """The plane engine reads no TF value outside a tile's support disk:
    filling every such entry of a kx-major bank (whole planes k_x outside the
    disk, and the z columns (k_y, k_x) outside it in the planes inside) with
    NaN leaves the field tiles' reconstruction bit for bit the same.  The
    disk is the library's own test, (k_y / Y)^2 + (k_x / X)^2 > r^2 in
    float32 with r from the bank's statistics (word 5); entries within 1e-6
    of the circle are left as they are."""
    B, torch, dev = env
    Z, ty, tx, core, halo = 48, 2, 2, 128, 32
    E = core + 2 * halo
    n = ty * tx
    m = B.WO_TF_PHASE | B.WO_TF_KX_MAJOR
    ol = ph.tile_optics(np.random.default_rng(8), n)
    tf, ws = build_bank(env, ol, Z, E, m, True)
    field = torch.from_numpy((1.0 + ph.sphere_phantom(9, (Z, ty * core, tx * core), n_spheres=30))
                             .astype(np.float32)).to(dev)

    def recon():
        rec = torch.empty((n, 1, Z, E, E), dtype=torch.float32, device=dev)
        B.wo_reconstruct_field_tiles(tf, m, field, Z, ty, tx, core, halo, None, [1e-3], B.WO_ETA_RELATIVE,
                                     B.WO_MODE_3D, rec, ws)
        assert B.wo_sync_status(ws)[0] == 0
        return rec.clone()

    want = recon()
    spec, stats = B.tf_views(tf, n, Z, E, E, m)  # spec: a permuted view of the kx-major storage
    r = stats[:, 5].cpu().numpy().astype(np.float32)
    ky = np.arange(E)
    fy = (np.where(ky < (E + 1) // 2, ky, ky - E).astype(np.float32) / np.float32(E)).astype(np.float32)
    fx = (np.arange(E // 2 + 1).astype(np.float32) / np.float32(E)).astype(np.float32)
    planted = 0
    for t in range(n):
        # outside by a margin (the device may fuse the sum into an FMA, so entries
        # within an ulp of the circle are left alone)
        out = (fy[:, None] * fy[:, None] + fx[None, :] * fx[None, :]) > r[t] * r[t] * np.float32(1 + 1e-6)
        mask = torch.from_numpy(np.broadcast_to(out, (Z,) + out.shape).copy()).to(dev)
        spec[t, 0][mask] = complex(float("nan"), float("nan"))
        planted += int(out.sum())
    assert planted > 0
    got = recon()
    assert torch.equal(got, want)
