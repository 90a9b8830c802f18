"""Small, valid calls of every kernel family, run by tests/test_gpu_check_build.py
with the normal library and with its WO_CHECK variant (each kernel testing the
indices of its global accesses).  Returns the outputs and the status codes
that wo_sync_status read after each call."""
import numpy as np

import phantom as ph


def run(B, torch, dev):
    out, codes = {}, []

    def sync(name, ws):
        codes.append((name,) + tuple(B.wo_sync_status(ws)))

    kinds = ("phase", "absorption", "fluor")
    for shape in ((8, 32, 48), (6, 24, 96), (4, 16, 192)):
        Z, Y, X = shape
        ol = [ph.optics(na_ill=0.7, tilt_x=0.04, defocus_um=0.2), ph.optics(na_ill=0.5, defocus_um=-0.3)]
        tf, ws = B.alloc(2, Z, Y, X, kinds, dev)
        B.wo_build_tf(ol, 2, Z, Y, X, kinds, tf, ws)
        sync(f"build {shape}", ws)
        f = torch.from_numpy(ph.uniform_volume(3, (2, 3) + shape, -0.01, 0.01).astype(np.float32)).to(dev)
        d = torch.empty((2, 2) + shape, dtype=torch.float32, device=dev)
        B.wo_forward(tf, kinds, f, [1.0, 0.5], d, 2, Z, Y, X, ws)
        sync(f"forward {shape}", ws)
        fa = torch.empty_like(f)
        B.wo_forward_adjoint(tf, kinds, d, [1.0, 0.5], fa, 2, Z, Y, X, ws)
        sync(f"adjoint {shape}", ws)
        r3 = torch.empty_like(f)
        B.wo_reconstruct(tf, kinds, d, None, [1e-3, 1e-3], B.WO_ETA_RELATIVE, B.WO_MODE_3D, r3, 2, Z, Y, X, ws)
        sync(f"reconstruct 3D {shape}", ws)
        r2 = torch.empty((2, 3, Y, X), dtype=torch.float32, device=dev)
        B.wo_reconstruct(tf, kinds, d, [1.0, 0.5], [1e-3, 1e-3], B.WO_ETA_ABSOLUTE, B.WO_MODE_2D, r2, 2, Z, Y, X, ws)
        sync(f"reconstruct 2D {shape}", ws)
        out[f"tf {shape}"] = tf.cpu().numpy()
        for k, v in (("d", d), ("fa", fa), ("r3", r3), ("r2", r2)):
            out[f"{k} {shape}"] = v.cpu().numpy()
    # tiles: gather and blend of a 3 x 2 grid (core 32, halo 8)
    field = torch.from_numpy(ph.uniform_volume(4, (4, 96, 64), 0.0, 1.0).astype(np.float32)).to(dev)
    tiles = torch.empty((6, 4, 48, 48), dtype=torch.float32, device=dev)
    B.wo_tile_gather(field, 4, 3, 2, 32, 8, tiles)
    back = torch.empty_like(field)
    B.wo_tile_blend(tiles, 4, 3, 2, 32, 8, back)
    ws = torch.zeros(4096, dtype=torch.uint8, device=dev)
    sync("tiles", ws)
    out["tiles"] = tiles.cpu().numpy()
    out["blend"] = back.cpu().numpy()
    # the tile pipeline (16 x 64 x 64 tiles)
    Z, Y, X = 16, 64, 64
    ol = ph.tile_optics(np.random.default_rng(2), 3)
    tf, ws = B.alloc(3, Z, Y, X, ("phase",), dev)
    B.wo_build_tf(ol, 3, Z, Y, X, ("phase",), tf, ws)
    d = torch.from_numpy(ph.uniform_volume(5, (3, Z, Y, X), 0.9, 1.1).astype(np.float32)).to(dev)
    r = torch.empty_like(d)
    B.wo_pipeline_probe(tf, d, r, 3, Z, Y, X, -1, 10 ** 9, ws)
    sync("pipeline", ws)
    out["pipeline"] = r.cpu().numpy()
    # the plane engine: a kx-major bank (16 x 64 x 64), the operators on
    # tiles, and a 2 x 2 field's tiles read in place (core 48, halo 8)
    kx = B.WO_TF_PHASE | B.WO_TF_KX_MAJOR
    tfk, wsk = B.alloc(3, Z, Y, X, kx, dev)
    B.wo_build_tf(ol, 3, Z, Y, X, kx, tfk, wsk)
    sync("kx-major build", wsk)
    fk = torch.from_numpy(ph.uniform_volume(6, (3, 1, Z, Y, X), -0.02, 0.02).astype(np.float32)).to(dev)
    dk = torch.empty((3, Z, Y, X), dtype=torch.float32, device=dev)
    B.wo_forward(tfk, kx, fk, [1.0], dk, 3, Z, Y, X, wsk)
    ak = torch.empty_like(fk)
    B.wo_forward_adjoint(tfk, kx, d, [1.0], ak, 3, Z, Y, X, wsk)
    rk = torch.empty_like(fk)
    B.wo_reconstruct(tfk, kx, d, None, [1e-3], B.WO_ETA_RELATIVE, B.WO_MODE_3D, rk, 3, Z, Y, X, wsk)
    sync("kx-major operators", wsk)
    fld = torch.from_numpy(ph.uniform_volume(7, (Z, 96, 96), 0.9, 1.1).astype(np.float32)).to(dev)
    tf4, ws4 = B.alloc(4, Z, Y, X, kx, dev)
    B.wo_build_tf(ph.tile_optics(np.random.default_rng(3), 4), 4, Z, Y, X, kx, tf4, ws4)
    rf = torch.empty((4, 1, Z, Y, X), dtype=torch.float32, device=dev)
    B.wo_reconstruct_field_tiles(tf4, kx, fld, Z, 2, 2, 48, 8, None, [1e-3], B.WO_ETA_RELATIVE, B.WO_MODE_3D, rf, ws4)
    sync("kx-major field tiles", ws4)
    for k, v in (("kx tf", tfk), ("kx forward", dk), ("kx adjoint", ak), ("kx reconstruct", rk), ("kx field", rf)):
        out[k] = v.cpu().numpy()
    return out, codes
