"""wo_reconstruct_static: the reconstruction for callers that cannot allocate.

Some callers (a plugin whose host application owns the device-memory
budget, code behind a caching allocator it may not bypass, latency-bound
loops that cannot afford cudaMalloc's implicit synchronisation) need a
reconstruction without handing the library a workspace.  This test calls
that entry point through the C ABI twice in a row, on different inputs, and
checks each result against wo_reconstruct with a caller-allocated workspace.
It lives in its own file, collected last, and passes alone or after the rest.
"""
import numpy as np
import pytest

import phantom as ph
from conftest import rel_l2

pytestmark = pytest.mark.gpu

TOL = 1e-4


def test_static_workspace_matches_reconstruct_twice():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2412_09775_gb300.build import build
    build()
    from paper_2412_09775_gb300 import binding as B

    dev = torch.device("cuda:0")
    Z, Y, X = 16, 64, 64
    kinds = ("phase", "absorption", "fluor")
    assert B.wo_workspace_bytes(1, Z, Y, X, kinds) <= B.WO_STATIC_SCRATCH_BYTES
    o = ph.optics(na_ill=0.8, tilt_x=0.03, defocus_um=0.2)
    tf, ws = B.alloc(1, Z, Y, X, kinds, dev)
    B.wo_build_tf([o], 1, Z, Y, X, kinds, tf, ws)
    for call, (seed, bg, eta) in enumerate([(21, None, [1e-3, 1e-3]), (22, [1.0, 0.4], [3e-3, 1e-2])]):
        d = torch.from_numpy(ph.uniform_volume(seed, (1, 2, Z, Y, X), 0.9, 1.1).astype(np.float32)).to(dev)
        ref = torch.empty((1, 3, Z, Y, X), dtype=torch.float32, device=dev)
        got = torch.full_like(ref, float("nan"))
        B.wo_reconstruct(tf, kinds, d, bg, eta, B.WO_ETA_RELATIVE, B.WO_MODE_3D, ref, 1, Z, Y, X, ws)
        B.wo_reconstruct_static(tf, kinds, d, bg, eta, B.WO_ETA_RELATIVE, B.WO_MODE_3D, got, 1, Z, Y, X)
        torch.cuda.synchronize()
        e = rel_l2(got.cpu().numpy(), ref.cpu().numpy())
        assert e <= TOL, (call, e)


def test_static_workspace_rejects_problems_beyond_its_size():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2412_09775_gb300.build import build
    build()
    from paper_2412_09775_gb300 import binding as B
    lib = B._lib
    fake = 1 << 20  # never dereferenced: the size check fails before any launch
    import ctypes
    eta = (ctypes.c_float * 2)(1e-3, 1e-3)
    pe = ctypes.cast(eta, ctypes.POINTER(ctypes.c_float))
    assert B.wo_workspace_bytes(1, 96, 512, 512, 7) > B.WO_STATIC_SCRATCH_BYTES
    assert lib.wo_reconstruct_static(fake, 7, fake, None, pe, 0, 0, fake, 1, 96, 512, 512, None) == 8
