"""The persistent tile pipeline of the phase-only 3D reconstruction (the
WO_PASS_RECON engine) against the float64 oracle and the five-pass path, and
its bounded waits: a tile whose plane items are never posted must end the
kernel with WO_ERR_TIMEOUT in the workspace's status block, not hang it.
"""
import time

import numpy as np
import pytest

import phantom as ph
from conftest import rel_l2
from oracle import model as OM, optics as OO

pytestmark = pytest.mark.gpu

TOL = 1e-4
SHAPES = [(48, 192, 192), (48, 128, 128), (16, 64, 64)]


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2412_09775_gb300.build import build
    build()
    from paper_2412_09775_gb300 import binding
    return binding, torch, torch.device("cuda:0")


def engine(B, Y, e):
    B.wo_schedule_set(B.WO_PASS_RECON, Y, e)


def stacks(o_list, shape, seed):
    """Brightfield stacks of sphere phantoms imaged by the oracle with each
    tile's optics, plus 1e-3 noise."""
    out = []
    for t, o in enumerate(o_list):
        dn = ph.sphere_phantom(seed + t, shape, o, n_spheres=30)
        modes, _, _ = OM.widefield_system(OO.transfer_functions(o, shape, ("phase",)), ("phase",))
        d = OM.forward(modes, dn[None], [1.0]) + ph.gaussian_noise(seed + 100 + t, (1,) + shape, 1e-3)
        out.append(d)
    return np.stack(out).astype(np.float32)


def run(env, kinds, o_list, d, bg, eta, flag, shape, eng, shared=False):
    B, torch, dev = env
    Z, Y, X = shape
    n = d.shape[0]
    nb = 1 if shared else n
    tf, ws = B.alloc(n if not shared else n, Z, Y, X, kinds, dev)
    if shared:
        tf, _ = B.alloc(1, Z, Y, X, kinds, dev)
    B.wo_build_tf(o_list[:nb], nb, Z, Y, X, kinds, tf, ws)
    din = torch.from_numpy(d).to(dev)
    out = torch.empty_like(din)
    engine(B, Y, eng)
    try:
        if shared:
            B.wo_reconstruct_shared_tf(tf, kinds, din, bg, [eta], flag, B.WO_MODE_3D, out, n, Z, Y, X, ws)
        else:
            B.wo_reconstruct(tf, kinds, din, bg, [eta], flag, B.WO_MODE_3D, out, n, Z, Y, X, ws)
        code = B.wo_sync_status(ws)
    finally:
        engine(B, Y, B.WO_ENGINE_DEFAULT)
    assert code[0] == 0, code
    return out.cpu().numpy()


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("bg,flag", [(None, 0), ([1.0], 1)])
def test_pipeline_matches_oracle_and_passes(env, shape, bg, flag):
    B = env[0]
    rng = np.random.default_rng(5)
    ol = ph.tile_optics(rng, 3)
    d = stacks(ol, shape, 40)
    eta = 1e-3 if flag == 0 else 2e-2
    got = run(env, ("phase",), ol, d, bg, eta, flag, shape, B.WO_ENGINE_HYBRID)
    ref5 = run(env, ("phase",), ol, d, bg, eta, flag, shape, B.WO_ENGINE_SMEM)
    for t, o in enumerate(ol):
        modes, _, _ = OM.widefield_system(OO.transfer_functions(o, shape, ("phase",)), ("phase",))
        want = OM.reconstruct(modes, d[t].astype(np.float64), eta, background=bg, relative=(flag == 0))
        assert rel_l2(got[t, 0], want[0]) <= TOL, t
        assert rel_l2(got[t, 0], ref5[t, 0]) <= 3e-5, t  # two float32 orders of the same sums


def test_pipeline_with_shared_tf_and_derivative_bank(env):
    """The pipeline serves a bank shared by a batch of stacks and the phase slot
    of a defocus-derivative bank."""
    B, torch, dev = env
    shape = (16, 64, 64)
    Z, Y, X = shape
    o = ph.optics(na_ill=0.8, defocus_um=0.3)
    d = stacks([o] * 5, shape, 60)
    got = run(env, ("phase",), [o] * 5, d, None, 1e-3, 0, shape, B.WO_ENGINE_HYBRID, shared=True)
    modes, _, _ = OM.widefield_system(OO.transfer_functions(o, shape, ("phase",)), ("phase",))
    for t in range(5):
        want = OM.reconstruct(modes, d[t].astype(np.float64), 1e-3)
        assert rel_l2(got[t, 0], want[0]) <= TOL, t
    kinds = B.WO_TF_PHASE_DZ
    tf, ws = B.alloc(2, Z, Y, X, kinds, dev)
    B.wo_build_tf([o, o], 2, Z, Y, X, kinds, tf, ws)
    din = torch.from_numpy(d[:2]).to(dev)
    out = torch.empty_like(din)
    engine(B, Y, B.WO_ENGINE_HYBRID)
    try:
        B.wo_reconstruct(tf, kinds, din, None, [1e-3], B.WO_ETA_RELATIVE, B.WO_MODE_3D, out, 2, Z, Y, X, ws)
    finally:
        engine(B, Y, B.WO_ENGINE_DEFAULT)
    assert B.wo_sync_status(ws)[0] == 0
    assert rel_l2(out.cpu().numpy(), got[:2]) <= 1e-5


def test_pipeline_timeout_returns_instead_of_hanging(env):
    """Tile 1's plane items are withheld: its z-solve items wait, run out of a
    2 ms budget, record WO_ERR_TIMEOUT (site 1, tile 1) and the kernel ends.
    The context stays usable: a whole run afterwards is clean and correct."""
    B, torch, dev = env
    shape = (16, 64, 64)
    Z, Y, X = shape
    n = 4
    ol = ph.tile_optics(np.random.default_rng(8), n)
    d = stacks(ol, shape, 70)
    tf, ws = B.alloc(n, Z, Y, X, ("phase",), dev)
    B.wo_build_tf(ol, n, Z, Y, X, ("phase",), tf, ws)
    din = torch.from_numpy(d).to(dev)
    out = torch.zeros_like(din)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    B.wo_pipeline_probe(tf, din, out, n, Z, Y, X, 1, 2_000_000, ws)
    code, site, detail = B.wo_sync_status(ws)
    dt = time.perf_counter() - t0
    assert code == B.STATUS_CODES["WO_ERR_TIMEOUT"] and site in (1, 2) and detail == 1, (code, site, detail)
    assert dt < 5.0, dt
    assert B.wo_sync_status(ws)[0] == 0  # read and cleared
    # the same pipeline, nothing withheld: clean, and equal to wo_reconstruct on the pipeline engine
    B.wo_pipeline_probe(tf, din, out, n, Z, Y, X, -1, 1_000_000_000, ws)
    assert B.wo_sync_status(ws)[0] == 0
    ref = torch.empty_like(din)
    engine(B, Y, B.WO_ENGINE_HYBRID)
    try:
        B.wo_reconstruct(tf, ("phase",), din, None, [1e-3], B.WO_ETA_ABSOLUTE, B.WO_MODE_3D, ref, n, Z, Y, X, ws)
    finally:
        engine(B, Y, B.WO_ENGINE_DEFAULT)
    assert B.wo_sync_status(ws)[0] == 0
    assert torch.equal(out, ref)


def test_status_block_reports_a_recorded_code(env):
    """wo_sync_status returns what the status block holds and clears it."""
    B, torch, dev = env
    ws = torch.zeros(4096, dtype=torch.uint8, device=dev)
    assert B.wo_sync_status(ws) == (0, 0, 0)
    ws[:12].view(torch.int32).copy_(torch.tensor([6, 2, 17], dtype=torch.int32))
    assert B.wo_sync_status(ws) == (6, 2, 17)
    assert B.wo_sync_status(ws) == (0, 0, 0)
    ws[:4].view(torch.int32).fill_(12345)  # never a status: an uncleared block
    assert B.wo_sync_status(ws)[0] == B.STATUS_CODES["WO_ERR_CUDA"]
    B.wo_clear_status(ws)
    assert B.wo_sync_status(ws) == (0, 0, 0)
