"""Padding in place of circular boundaries through the C ABI: wo_pad and
wo_crop bit for bit against the oracle, and a padded reconstruction (pad ->
TF build and Tikhonov solve on the padded grid -> crop) against the
oracle's."""
import numpy as np
import pytest

import phantom as ph
from conftest import rel_l2
from oracle import model as OM, optics as OO, tiles as OT

pytestmark = pytest.mark.gpu

MODES = {"zero": 0, "mirror": 1, "edge": 2}


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2412_09775_gb300.build import build
    build()
    from paper_2412_09775_gb300 import binding
    return binding, torch, torch.device("cuda:0")


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("shape,shape_p", [((5, 6, 7), (9, 10, 11)), ((5, 6, 7), (21, 6, 30)), ((1, 1, 3), (3, 2, 9)),
                                           ((12, 32, 32), (24, 48, 48)), ((7, 33, 65), (7, 33, 65)),
                                           ((16, 100, 130), (32, 128, 192))])
def test_pad_and_crop_bit_exact(env, mode, shape, shape_p):
    B, torch, dev = env
    n = 3
    v = np.random.default_rng(1).normal(size=(n,) + shape).astype(np.float32)
    vin = torch.from_numpy(v).to(dev)
    out = torch.full((n,) + shape_p, float("nan"), dtype=torch.float32, device=dev)
    B.wo_pad(vin, n, *shape, *shape_p, MODES[mode], out)
    got = out.cpu().numpy()
    assert np.array_equal(got, OT.pad(v, shape_p, mode).astype(np.float32))
    back = torch.full((n,) + shape, float("nan"), dtype=torch.float32, device=dev)
    B.wo_crop(out, n, *shape_p, *shape, back)
    assert np.array_equal(back.cpu().numpy(), v)


def test_padded_reconstruction_matches_oracle(env):
    """A 12 x 32 x 32 window of a brightfield stack, background removed, zero
    padded to 24 x 48 x 48, reconstructed there and cropped back."""
    B, torch, dev = env
    o = ph.optics(na_ill=0.7)
    world, win = (24, 48, 48), (12, 32, 32)
    f = ph.sphere_phantom(0, world, o, n_spheres=30)
    md, _, _ = OM.widefield_system(OO.transfer_functions(o, world, ("phase",)), ("phase",))
    d = OM.forward(md, f[None], [1.0])[0] + np.random.default_rng(0).normal(size=world) * 1e-3
    dw = (OT.crop(d, win) - OT.crop(d, win).mean()).astype(np.float32)
    # oracle
    md_p, _, _ = OM.widefield_system(OO.transfer_functions(o, world, ("phase",)), ("phase",))
    ref = OT.crop(OM.reconstruct(md_p, OT.pad(dw.astype(np.float64), world, "zero")[None], 1e-3)[0], win)
    # library
    Z, Y, X = world
    din = torch.from_numpy(dw[None]).to(dev)
    dp = torch.empty((1,) + world, dtype=torch.float32, device=dev)
    B.wo_pad(din, 1, *win, *world, B.WO_PAD_ZERO, dp)
    tf, ws = B.alloc(1, Z, Y, X, ("phase",), dev)
    B.wo_build_tf([o], 1, Z, Y, X, ("phase",), tf, ws)
    fp = torch.empty((1, 1) + world, dtype=torch.float32, device=dev)
    B.wo_reconstruct(tf, ("phase",), dp, None, [1e-3], B.WO_ETA_RELATIVE, B.WO_MODE_3D, fp, 1, Z, Y, X, ws)
    fw = torch.empty((1,) + win, dtype=torch.float32, device=dev)
    B.wo_crop(fp, 1, *world, *win, fw)
    assert rel_l2(fw.cpu().numpy()[0], ref) <= 1e-4
