"""The fused x-y kernels (WO_PASS_XY, a cluster of two CTAs per plane) against
the separate x and y passes, on every entry point that runs them: the 3D and
2D reconstructions, the forward model with a given background (the inverse's
per-channel constant), the adjoint, the data spectra and the reconstruction
gradient; plus the spectra against numpy's FFT in float64.
"""
import numpy as np
import pytest

import phantom as ph
from conftest import rel_l2

pytestmark = pytest.mark.gpu

SHAPES = [(16, 64, 64), (48, 128, 128), (48, 192, 192)]


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2412_09775_gb300.build import build
    build()
    from paper_2412_09775_gb300 import binding
    return binding, torch, torch.device("cuda:0")


def on_engine(B, Y, e, fn):
    B.wo_schedule_set(B.WO_PASS_XY, Y, e)
    try:
        return fn()
    finally:
        B.wo_schedule_set(B.WO_PASS_XY, Y, B.WO_ENGINE_DEFAULT)


def both(B, Y, fn):
    """fn() on the fused kernels and on the separate passes."""
    a = on_engine(B, Y, B.WO_ENGINE_HYBRID, fn)
    b = on_engine(B, Y, B.WO_ENGINE_SMEM, fn)
    return a, b


@pytest.mark.parametrize("shape", SHAPES)
def test_fused_xy_matches_separate_passes(env, shape):
    B, torch, dev = env
    Z, Y, X = shape
    n = 3  # an odd number of tiles: ragged plane counts for every batch below
    ol = ph.tile_optics(np.random.default_rng(11), n)
    tf, ws = B.alloc(n, Z, Y, X, ("phase",), dev)
    B.wo_build_tf(ol, n, Z, Y, X, ("phase",), tf, ws)
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    d = 1.0 + 0.05 * torch.randn((n, Z, Y, X), generator=g, device=dev)
    f = 0.1 * torch.randn((n, 1, Z, Y, X), generator=g, device=dev)

    def recon(mode, flag, bg):
        def run():
            out = torch.empty((n, 1, Z, Y, X) if mode == B.WO_MODE_3D else (n, 1, Y, X), device=dev)
            B.wo_reconstruct(tf, ("phase",), d, bg, [1e-3], flag, mode, out, n, Z, Y, X, ws)
            assert B.wo_sync_status(ws)[0] == 0
            return out.clone()
        return run

    for mode, flag, bg in ((B.WO_MODE_3D, B.WO_ETA_RELATIVE, None), (B.WO_MODE_3D, B.WO_ETA_ABSOLUTE, [1.0]),
                           (B.WO_MODE_2D, B.WO_ETA_RELATIVE, None)):
        a, b = both(B, Y, recon(mode, flag, bg))
        assert rel_l2(a.cpu().numpy(), b.cpu().numpy()) <= 2e-6, (mode, flag, bg)

    def forward():
        out = torch.empty((n, Z, Y, X), device=dev)
        B.wo_forward(tf, ("phase",), f, [1.0], out, n, Z, Y, X, ws)
        return out.clone()
    a, b = both(B, Y, forward)
    assert rel_l2(a.cpu().numpy(), b.cpu().numpy()) <= 2e-6

    def adjoint():
        out = torch.empty((n, 1, Z, Y, X), device=dev)
        B.wo_forward_adjoint(tf, ("phase",), d, None, out, n, Z, Y, X, ws)
        return out.clone()
    a, b = both(B, Y, adjoint)
    assert rel_l2(a.cpu().numpy(), b.cpu().numpy()) <= 2e-6

    def spectrum():
        spec = torch.empty((n, Z, Y, X // 2 + 1), dtype=torch.complex64, device=dev)
        B.wo_spectrum(d, None, B.WO_MODE_2D, spec, n, Z, Y, X)
        return spec.clone()
    a, b = both(B, Y, spectrum)
    a, b = a.cpu().numpy(), b.cpu().numpy()
    assert rel_l2(a, b) <= 2e-6
    # against numpy's 2D real transform in float64, per plane (the DC bin is the
    # plane's centred value: compare the rest)
    want = np.fft.rfft2(d.cpu().numpy().astype(np.float64), axes=(-2, -1))
    a[..., 0, 0] = 0
    want[..., 0, 0] = 0
    assert rel_l2(a, want) <= 2e-6
