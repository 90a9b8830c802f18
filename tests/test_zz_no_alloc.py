"""wo_reconstruct_static: the reconstruction for callers that cannot allocate.

Some callers (a plugin whose host application owns the device-memory
budget, code behind a caching allocator it may not bypass, latency-bound
loops that cannot afford cudaMalloc's implicit synchronisation) need a
reconstruction without handing the library a workspace.  This test first
fills the library's shared scratch array with the spectra of an unrelated,
larger problem, then calls the entry point through the C ABI twice in a row
on different inputs (three kinds through the five passes, and the phase-only
case through the tile pipeline) and checks each result against the float64
oracle and against wo_reconstruct with a caller-allocated workspace; the
device's free memory must not change across those calls.  One more call is
captured in a CUDA graph in global capture mode, which rejects any device
allocation or release made while the capture is open, and replayed: it must
give the first call's result bit for bit.  It lives in its own file,
collected last, and passes alone or after the rest.
"""
import numpy as np
import pytest

import phantom as ph
from conftest import rel_l2
from oracle import model as OM, optics as OO

pytestmark = pytest.mark.gpu

TOL = 1e-4


def oracle_recon(o, shape, kinds, d, bg, eta):
    modes, props, _ = OM.widefield_system(OO.transfer_functions(o, shape, kinds), kinds)
    out = np.zeros((len(props),) + shape)
    for m, e in zip(modes, eta):
        r = OM.reconstruct([m], d.astype(np.float64), e, background=bg)
        for p in m["props"]:
            out[p] = r[p]
    return out


def test_static_workspace_matches_reconstruct_twice():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2412_09775_gb300.build import build
    build()
    from paper_2412_09775_gb300 import binding as B

    dev = torch.device("cuda:0")
    Z, Y, X = 16, 64, 64
    o = ph.optics(na_ill=0.8, tilt_x=0.03, defocus_um=0.2)
    # an unrelated, larger problem leaves non-zero garbage in the shared scratch
    Zb, Yb, Xb = 48, 128, 128
    assert B.wo_workspace_bytes(1, Zb, Yb, Xb, ("phase",)) <= B.WO_STATIC_SCRATCH_BYTES
    tfb, wsb = B.alloc(1, Zb, Yb, Xb, ("phase",), dev)
    B.wo_build_tf([ph.optics()], 1, Zb, Yb, Xb, ("phase",), tfb, wsb)
    junk = torch.from_numpy(ph.uniform_volume(5, (1, 1, Zb, Yb, Xb), -1e4, 1e4).astype(np.float32)).to(dev)
    junk_out = torch.empty_like(junk)
    B.wo_reconstruct_static(tfb, ("phase",), junk, [0.0], [1e-3], B.WO_ETA_ABSOLUTE, B.WO_MODE_3D, junk_out, 1, Zb,
                            Yb, Xb)
    torch.cuda.synchronize()
    cases = [(("phase", "absorption", "fluor"), 21, None, [1e-3, 1e-3]),
             (("phase",), 22, [1.0], [3e-3])]
    prepared = []
    for kinds, seed, bg, eta in cases:
        assert B.wo_workspace_bytes(1, Z, Y, X, kinds) <= B.WO_STATIC_SCRATCH_BYTES
        tf, ws = B.alloc(1, Z, Y, X, kinds, dev)
        B.wo_build_tf([o], 1, Z, Y, X, kinds, tf, ws)
        nc = 2 if "fluor" in kinds else 1
        d_np = ph.uniform_volume(seed, (1, nc, Z, Y, X), 0.9, 1.1).astype(np.float32)
        d = torch.from_numpy(d_np).to(dev)
        ref = torch.empty((1, len(kinds), Z, Y, X), dtype=torch.float32, device=dev)
        got = torch.full_like(ref, float("nan"))
        B.wo_reconstruct(tf, kinds, d, bg, eta, B.WO_ETA_RELATIVE, B.WO_MODE_3D, ref, 1, Z, Y, X, ws)
        prepared.append((kinds, d_np, d, bg, eta, tf, ref, got))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    for kinds, d_np, d, bg, eta, tf, ref, got in prepared:
        B.wo_reconstruct_static(tf, kinds, d, bg, eta, B.WO_ETA_RELATIVE, B.WO_MODE_3D, got, 1, Z, Y, X)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(dev)[0] == free0  # nothing was allocated on the device
    for call, (kinds, d_np, d, bg, eta, tf, ref, got) in enumerate(prepared):
        g = got.cpu().numpy()
        assert rel_l2(g, ref.cpu().numpy()) <= TOL, call
        want = oracle_recon(o, (Z, Y, X), kinds, d_np[0], bg, eta)
        assert rel_l2(g[0], want) <= TOL, call
    # the first case once more, captured and replayed: an allocation on this
    # path would make the capture fail
    kinds, d_np, d, bg, eta, tf, ref, got = prepared[0]
    replayed = torch.full_like(ref, float("nan"))
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, capture_error_mode="global"):
        B.wo_reconstruct_static(tf, kinds, d, bg, eta, B.WO_ETA_RELATIVE, B.WO_MODE_3D, replayed, 1, Z, Y, X)
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(replayed, got)


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
