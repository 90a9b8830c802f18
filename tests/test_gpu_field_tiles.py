"""wo_reconstruct_field_tiles: the tiles of a field reconstructed without
gathering them first must equal, bit for bit, wo_tile_gather followed by
wo_reconstruct — on grids with border tiles (mirror-padded halos), for the
one-channel kinds, both background rules and both modes."""
import numpy as np
import pytest

import phantom as ph

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2412_09775_gb300.build import build
    build()
    from paper_2412_09775_gb300 import binding
    return binding, torch, torch.device("cuda:0")


def gathered_and_in_place(env, Z, ty, tx, core, halo, kinds, bg, flag, mode, seed):
    B, torch, dev = env
    E = core + 2 * halo
    n = ty * tx
    field = torch.from_numpy((1.0 + ph.uniform_volume(seed, (Z, ty * core, tx * core), -0.02, 0.02))
                             .astype(np.float32)).to(dev)
    ol = ph.tile_optics(np.random.default_rng(seed), n)
    tf, ws = B.alloc(n, Z, E, E, kinds, dev)
    B.wo_build_tf(ol, n, Z, E, E, kinds, tf, ws)
    tiles = torch.empty((n, Z, E, E), dtype=torch.float32, device=dev)
    B.wo_tile_gather(field, Z, ty, tx, core, halo, tiles)
    P = len([k for k in kinds])
    shape = (n, P, Z, E, E) if mode == B.WO_MODE_3D else (n, P, E, E)
    want = torch.empty(shape, dtype=torch.float32, device=dev)
    got = torch.full(shape, float("nan"), dtype=torch.float32, device=dev)
    eta = [1e-3] * 2
    B.wo_reconstruct(tf, kinds, tiles, bg, eta, flag, mode, want, n, Z, E, E, ws)
    B.wo_reconstruct_field_tiles(tf, kinds, field, Z, ty, tx, core, halo, bg, eta, flag, mode, got, ws)
    assert B.wo_sync_status(ws)[0] == 0
    return got, want


@pytest.mark.parametrize("kinds", [("phase",), ("fluor",), ("phase", "absorption")])
@pytest.mark.parametrize("bg,flag", [(None, 0), ([1.0], 1)])
def test_field_tiles_equal_gathered_tiles(env, kinds, bg, flag):
    B, torch, _ = env
    # 2 x 3 tiles of 56-px cores and 4-px halos (64 x 64 tiles): every tile
    # touches a field edge, where the halo is mirrored
    got, want = gathered_and_in_place(env, 16, 2, 3, 56, 4, kinds, bg, flag, B.WO_MODE_3D, 5)
    assert torch.equal(got, want)


def test_field_tiles_2d_mode_and_192_tiles(env):
    B, torch, _ = env
    got, want = gathered_and_in_place(env, 16, 2, 2, 48, 8, ("phase",), None, 0, B.WO_MODE_2D, 6)
    assert torch.equal(got, want)
    # the field workload's tiles: 128-px cores, 32-px halos, an interior tile among border ones
    got, want = gathered_and_in_place(env, 48, 3, 3, 128, 32, ("phase",), None, 0, B.WO_MODE_3D, 7)
    assert torch.equal(got, want)


@pytest.mark.parametrize("kinds", [("phase",), ("phase", "absorption")])
@pytest.mark.parametrize("geom", [(16, 2, 3, 56, 4), (16, 2, 2, 50, 7), (48, 3, 3, 128, 32)])
@pytest.mark.parametrize("mode", [0, 1])
def test_restore_field_equals_tiles_then_blend(env, kinds, geom, mode):
    """wo_restore_field (tiles read in place, blended by the last pass) against
    wo_reconstruct_field_tiles followed by wo_tile_blend of each property: bit
    for bit, with and without the 4-pixel vector path (halo 7) and in both
    modes."""
    B, torch, dev = env
    Z, ty, tx, core, halo = geom
    m = (B.WO_MODE_3D, B.WO_MODE_2D)[mode]
    E = core + 2 * halo
    n = ty * tx
    P = len(kinds)
    field = torch.from_numpy((1.0 + ph.uniform_volume(8, (Z, ty * core, tx * core), -0.02, 0.02))
                             .astype(np.float32)).to(dev)
    ol = ph.tile_optics(np.random.default_rng(9), n)
    tf, ws = B.alloc(n, Z, E, E, kinds, dev)
    B.wo_build_tf(ol, n, Z, E, E, kinds, tf, ws)
    zf = Z if m == B.WO_MODE_3D else 1
    rec = torch.empty((n, P, zf, E, E), dtype=torch.float32, device=dev)
    B.wo_reconstruct_field_tiles(tf, kinds, field, Z, ty, tx, core, halo, None, [1e-3, 1e-3], B.WO_ETA_RELATIVE, m,
                                 rec, ws)
    want = torch.empty((P, zf, ty * core, tx * core), dtype=torch.float32, device=dev)
    for p in range(P):
        B.wo_tile_blend(rec[:, p].contiguous(), zf, ty, tx, core, halo, want[p])
    got = torch.full_like(want, float("nan"))
    B.wo_restore_field(tf, kinds, field, Z, ty, tx, core, halo, None, [1e-3, 1e-3], B.WO_ETA_RELATIVE, m, got, ws)
    assert B.wo_sync_status(ws)[0] == 0
    assert torch.equal(got, want)
