"""Host-side checks of the C ABI (CPU only; no compute call reaches a GPU).

Every call below is built to fail validation, so nothing is ever launched on
the placeholder pointers it passes.

The library must load without a GPU, export every symbol include/wo.h
declares, size its buffers consistently, and reject invalid arguments with
the documented status before launching anything.
"""
import ctypes
import os
import re

import pytest

import phantom as ph

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def B():
    from paper_2412_09775_gb300.build import build
    build()
    from paper_2412_09775_gb300 import binding
    return binding


def header_functions():
    src = open(os.path.join(ROOT, "include", "wo.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(wo_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(B):
    names = header_functions()
    assert len(names) >= 13
    for n in names:
        assert hasattr(B._lib, n), n
        assert n in B.EXPORTED, n


def test_supported_sizes(B):
    ok = [1, 2, 3, 4, 6, 8, 12, 16, 24, 48, 64, 96, 192, 512, 1536, 2048]
    bad = [0, 5, 7, 9, 10, 18, 36, 100, 3072, 4096, -4]
    assert all(B.wo_size_supported(n) for n in ok)
    assert not any(B.wo_size_supported(n) for n in bad)


def test_buffer_sizes(B):
    n, Z, Y, X = 3, 16, 64, 96
    Xh = X // 2 + 1
    for kinds, nk in ((1, 1), (3, 2), (4, 1), (7, 3)):
        spec = n * nk * Z * Y * Xh * 8
        assert B.wo_tf_bytes(n, Z, Y, X, kinds) == ((spec + 255) // 256) * 256 + n * 32
        assert B.wo_workspace_bytes(n, Z, Y, X, kinds) > 0
    assert B.wo_tf_bytes(1, 16, 64, 63, 1) == 0          # odd X
    assert B.wo_workspace_bytes(1, 10, 64, 64, 1) == 0   # Z not supported
    assert B.wo_tf_bytes(1, 16, 64, 64, 0) == 0          # no kinds
    # phase_dz: two TF slots per tile (phase TF and its defocus derivative)
    assert B.wo_tf_bytes(n, Z, Y, X, 8) == ((n * 2 * Z * Y * Xh * 8 + 255) // 256) * 256 + n * 32
    assert B.wo_workspace_bytes(n, Z, Y, X, 8) >= n * 4 * Z * Y * X * 8  # four pupil arms
    assert B.wo_tf_bytes(1, 16, 64, 1024, 8) == 0 and B.wo_tf_bytes(1, 16, 64, 64, 12) == 0


def test_build_tf_validation(B):
    lib = B._lib
    good = B.optics_array([ph.optics()])
    fake = 1 << 20  # 16-byte aligned non-null address; never dereferenced
    big = 1 << 40
    cases = [
        (B.optics_array([ph.optics(na_det=1.33)]), 1, 16, 64, 64, 1, fake, fake, big, 7),  # NA_det >= n
        (B.optics_array([ph.optics(na_ill=0.5, tilt_x=1.0)]), 1, 16, 64, 64, 1, fake, fake, big, 7),
        (B.optics_array([ph.optics(lambda_um=-1.0)]), 1, 16, 64, 64, 1, fake, fake, big, 7),
        (B.optics_array([ph.optics(pixel_um=0.2)]), 1, 16, 64, 64, 1, fake, fake, big, 4),  # aliasing
        (B.optics_array([ph.optics(z_step_um=0.4)]), 1, 16, 64, 64, 1, fake, fake, big, 4),  # axial
        (good, 1, 16, 64, 62, 1, fake, fake, big, 3),   # X/2 = 31
        (good, 1, 16, 64, 63, 1, fake, fake, big, 2),   # odd X
        (good, 1, 16, 64, 64, 16, fake, fake, big, 1),  # bad kinds
        (good, 1, 16, 64, 64, 9, fake, fake, big, 1),   # phase_dz or-ed with phase
        (good, 1, 16, 64, 1024, 8, fake, fake, big, 3),  # phase_dz beyond X = 768
        (good, 0, 16, 64, 64, 1, fake, fake, big, 1),   # no tiles
        (good, 1, 16, 64, 64, 1, fake + 4, fake, big, 1),  # misaligned
        (good, 1, 16, 64, 64, 1, None, fake, big, 1),   # null
        (good, 1, 16, 64, 64, 1, fake, fake, 1024, 8),  # workspace too small
    ]
    for arr, n, Z, Y, X, kinds, tf, ws, wsb, want in cases:
        assert lib.wo_build_tf(arr, n, Z, Y, X, kinds, tf, ws, wsb, None) == want


def test_aberrated_build_validation(B):
    lib = B._lib
    good = B.optics_array([ph.optics(), ph.optics()])
    fake = 1 << 20
    big = 1 << 40
    D = ctypes.c_double
    z = (D * 8)(0.0, 0.0, 0.0, 0.1, 0.0, 0.05, 0.0, 0.0)
    nan = (D * 8)(0.0, 0.0, 0.0, float("nan"), 0.0, 0.0, 0.0, 0.0)
    ws_plain = B.wo_workspace_bytes(2, 16, 64, 64, 1)
    ws_ab = B.wo_aberrated_workspace_bytes(2, 16, 64, 64, 1)
    assert ws_ab > ws_plain > 0  # the aberration record and the coefficients
    assert B.wo_aberrated_workspace_bytes(2, 16, 64, 64, 0) == 0
    f = lib.wo_build_tf_aberrated
    assert f(good, z, 37, 2, 16, 64, 64, 1, fake, fake, big, None) == 1     # more than WO_MAX_ZERNIKE
    assert f(good, z, -1, 2, 16, 64, 64, 1, fake, fake, big, None) == 1
    assert f(good, None, 4, 2, 16, 64, 64, 1, fake, fake, big, None) == 1   # coefficients missing
    assert f(good, nan, 4, 2, 16, 64, 64, 1, fake, fake, big, None) == 1    # non-finite coefficient
    assert f(good, z, 4, 2, 16, 64, 64, 1, fake, fake, ws_ab - 1, None) == 8  # workspace too small
    assert f(good, z, 4, 2, 16, 64, 40, 1, fake, fake, big, None) == 3      # X/2 = 20 unsupported
    assert B.WO_MAX_ZERNIKE == 36


def test_op_validation(B):
    lib = B._lib
    fake = 1 << 20
    eta = (ctypes.c_float * 2)(1e-3, 1e-3)
    neg = (ctypes.c_float * 2)(-1.0, 1e-3)
    pe = ctypes.cast(eta, ctypes.POINTER(ctypes.c_float))
    pn = ctypes.cast(neg, ctypes.POINTER(ctypes.c_float))
    big = 1 << 40
    assert lib.wo_reconstruct(fake, 7, fake, None, None, 0, 0, fake, 1, 16, 64, 64, fake, big, None) == 1
    assert lib.wo_reconstruct(fake, 7, fake, None, pn, 0, 0, fake, 1, 16, 64, 64, fake, big, None) == 1
    assert lib.wo_reconstruct(fake, 7, fake, None, pe, 2, 0, fake, 1, 16, 64, 64, fake, big, None) == 1
    assert lib.wo_reconstruct(fake, 7, fake, None, pe, 0, 5, fake, 1, 16, 64, 64, fake, big, None) == 1
    assert lib.wo_reconstruct(fake, 7, fake, None, pe, 0, 0, fake, 1, 16, 64, 64, fake, 16, None) == 8
    assert lib.wo_reconstruct_shared_tf(fake, 7, fake, None, None, 0, 0, fake, 4, 16, 64, 64, fake, big, None) == 1
    assert lib.wo_reconstruct_shared_tf(fake, 7, fake, None, pe, 0, 0, fake, 4, 16, 64, 64, fake, 16, None) == 8
    assert lib.wo_reconstruct_shared_tf(fake, 7, fake, None, pe, 0, 0, fake, 4, 16, 64, 60, fake, big, None) == 3
    assert lib.wo_forward(fake, 7, fake + 8, None, fake, 1, 16, 64, 64, fake, big, None) == 1
    assert lib.wo_forward_adjoint(fake, 7, fake, None, fake, 1, 16, 64, 100, fake, big, None) == 3


def test_tuning_validation(B):
    lib = B._lib
    fake = 1 << 20
    big = 1 << 40
    d = ctypes.c_double
    obj = lib.wo_tune_objective
    K = 8  # WO_TF_PHASE_DZ
    assert obj(fake, K, fake, fake, 0, 1e-3, 0.0, None, None, 1, 16, 64, 64, fake, big, None) == 1  # no output
    assert obj(fake, K, fake, fake, 0, -1.0, 0.0, fake, fake, 1, 16, 64, 64, fake, big, None) == 1  # eta < 0
    assert obj(fake, K, fake + 4, fake, 0, 1e-3, 0.0, fake, fake, 1, 16, 64, 64, fake, big, None) == 1
    assert obj(fake, K, fake, fake, 0, 1e-3, 0.0, fake, fake + 4, 1, 16, 64, 64, fake, big, None) == 1
    assert obj(fake, K, fake, fake, 0, 1e-3, float("nan"), fake, fake, 1, 16, 64, 64, fake, big, None) == 1
    assert obj(fake, K, fake, fake, 0, 1e-3, 0.0, fake, fake, 1, 16, 64, 64, fake, 16, None) == 8
    assert obj(fake, K | 16, fake, fake, 0, 1e-3, 0.0, fake, fake, 1, 16, 64, 64, fake, 16, None) == 8
    assert obj(fake, K, fake, fake, 0, 1e-3, 0.0, fake, fake, 1, 16, 64, 1024, fake, big, None) == 3
    assert obj(fake, K, fake, fake, 0, 1e-3, 0.0, fake, fake, 1, 16, 64, 63, fake, big, None) == 2
    assert obj(fake, 1, fake, fake, 0, 1e-3, 0.0, fake, fake, 1, 16, 64, 64, fake, big, None) == 1  # not a dz bank
    assert obj(fake, 16, fake, fake, 0, 1e-3, 0.0, fake, fake, 1, 16, 64, 64, fake, big, None) == 1
    assert obj(fake, K, fake, fake, 2, 1e-3, 0.0, fake, fake, 1, 16, 64, 64, fake, big, None) == 1  # bad loss
    adam = lib.wo_adam_optics
    lr1 = (ctypes.c_double * 1)(0.02)
    lr4 = (ctypes.c_double * 4)(0.02, 0.005, 0.005, 0.005)
    neg = (ctypes.c_double * 4)(0.02, -0.005, 0.005, 0.005)
    assert adam(fake, fake, 1, fake, 0, lr1, d(0.9), d(0.999), d(1e-8), None) == 1      # no tiles
    assert adam(fake, fake, 2, fake, 4, lr4, d(0.9), d(0.999), d(1e-8), None) == 1      # 2 parameters
    assert adam(fake, fake, 4, fake, 4, neg, d(0.9), d(0.999), d(1e-8), None) == 1      # lr < 0
    assert adam(fake, fake, 1, fake, 4, lr1, d(1.0), d(0.999), d(1e-8), None) == 1      # beta1 = 1
    assert adam(fake, fake, 1, fake, 4, lr1, d(0.9), d(0.999), d(0.0), None) == 1       # eps = 0
    assert adam(None, fake, 1, fake, 4, lr1, d(0.9), d(0.999), d(1e-8), None) == 1
    assert adam(fake, fake, 1, fake + 4, 4, lr1, d(0.9), d(0.999), d(1e-8), None) == 1
    assert adam(fake, fake, 4, fake, 4, None, d(0.9), d(0.999), d(1e-8), None) == 1
    spec = lib.wo_spectrum
    assert spec(fake, None, 0, fake, 1, 16, 64, 63, None) == 2
    assert spec(fake, None, 0, fake, 1, 10, 64, 64, None) == 3
    assert spec(fake + 8, None, 1, fake, 1, 16, 64, 64, None) == 1
    assert spec(fake, None, 0, fake, 0, 16, 64, 64, None) == 1
    assert spec(fake, None, 2, fake, 1, 16, 64, 64, None) == 1  # bad mode
    # per-plane banks: only with the derivative kinds; the operators reject them
    assert B.wo_tf_bytes(1, 16, 64, 64, 16) == 0 and B.wo_tf_bytes(1, 16, 64, 64, 17) == 0
    assert B.wo_tf_bytes(1, 16, 64, 64, 24) == B.wo_tf_bytes(1, 16, 64, 64, 8)
    assert lib.wo_forward(fake, 24, fake, None, fake, 1, 16, 64, 64, fake, big, None) == 1
    # the gradient bank: per plane only, five slots, register row pass lengths only
    assert B.wo_tf_bytes(1, 16, 64, 64, 64) == 0                 # needs WO_TF_PLANES
    assert B.wo_tf_bytes(1, 16, 64, 64, 64 | 16) == ((5 * 16 * 64 * 33 * 8 + 255) // 256) * 256 + 32
    assert B.wo_tf_bytes(1, 16, 64, 64, 64 | 16 | 32) == B.wo_tf_bytes(1, 16, 64, 64, 64 | 16)
    assert B.wo_tf_bytes(1, 16, 64, 96, 64 | 16) > 0             # 96- and 192-point rows (the field's tiles)
    assert B.wo_tf_bytes(1, 16, 192, 192, 64 | 16) > 0
    assert B.wo_tf_bytes(1, 16, 64, 384, 64 | 16) == 0           # 384-point rows: no gradient bank
    assert B.wo_tf_bytes(1, 16, 64, 64, 64 | 8 | 16) == 0        # two derivative banks at once
    assert B.wo_tf_bytes(1, 16, 64, 64, 4 | 32) == 0             # smooth source without label-free kinds
    assert B.wo_tf_bytes(1, 16, 64, 64, 1 | 32) == B.wo_tf_bytes(1, 16, 64, 64, 1)
    assert obj(fake, 64 | 16, fake, fake, 0, 1e-3, 0.0, fake, fake, 1, 16, 64, 64, fake, 16, None) == 8


def test_schedule_table(B):
    lib = B._lib
    assert lib.wo_schedule_set(4, 128, 1) == 1        # unknown pass
    assert lib.wo_schedule_set(1, 1024, 2) == 3       # no register row engine for 1024 points
    assert lib.wo_schedule_get(4, 128) == -1
    # the fused x-y kernels, keyed by Y for square planes: 64, 128 and 192 only
    for n in (64, 128, 192):
        assert lib.wo_schedule_get(3, n) == 1                                     # default: two passes
        assert lib.wo_schedule_set(3, n, 2) == 0 and lib.wo_schedule_get(3, n) == 2
        assert lib.wo_schedule_set(3, n, 0) == 0 and lib.wo_schedule_get(3, n) == 1
    assert lib.wo_schedule_set(3, 512, 2) == 3 and lib.wo_schedule_get(3, 512) == 1
    # the reconstruction engine, keyed by Y: the tile pipeline at 64, 128 and 192 only
    for n in (64, 128, 192):
        assert lib.wo_schedule_get(2, n) == 1                                     # default: the five passes
        assert lib.wo_schedule_set(2, n, 2) == 0 and lib.wo_schedule_get(2, n) == 2
        assert lib.wo_schedule_set(2, n, 0) == 0 and lib.wo_schedule_get(2, n) == 1
    assert lib.wo_schedule_set(2, 512, 2) == 3 and lib.wo_schedule_get(2, 512) == 1
    for n in (96, 256, 512):  # the x passes
        assert lib.wo_schedule_set(1, n, 2) == 0 and lib.wo_schedule_get(1, n) == 2
        assert lib.wo_schedule_set(1, n, 1) == 0 and lib.wo_schedule_get(1, n) == 1
        assert lib.wo_schedule_set(1, n, 0) == 0 and lib.wo_schedule_get(1, n) in (1, 2)
    assert lib.wo_schedule_get(1, 24) == 1
    assert lib.wo_schedule_set(0, 0, 1) == 1          # bad length
    assert lib.wo_schedule_set(0, 128, 7) == 1        # bad engine
    assert lib.wo_schedule_set(0, 1024, 2) == 3       # no hybrid engine for 1024
    assert lib.wo_schedule_get(0, 5000) == -1
    for n in (128, 512):
        assert lib.wo_schedule_set(0, n, 2) == 0 and lib.wo_schedule_get(0, n) == 2
        assert lib.wo_schedule_set(0, n, 1) == 0 and lib.wo_schedule_get(0, n) == 1
        assert lib.wo_schedule_set(0, n, 0) == 0 and lib.wo_schedule_get(0, n) in (1, 2)
    assert lib.wo_schedule_get(0, 1024) == 1
    fake = 1 << 20
    assert lib.wo_autotune(1, 16, 64, 64, 1, fake, 16, None) == 8       # workspace too small
    assert lib.wo_autotune(1, 16, 64, 63, 1, fake, 1 << 40, None) == 1  # bad shape
    assert lib.wo_autotune(1, 16, 64, 64, 1, fake + 4, 1 << 40, None) == 1


def test_tile_validation(B):
    lib = B._lib
    fake = 1 << 20
    assert lib.wo_tile_gather(fake, 4, 2, 2, 16, 9, fake, None) == 2   # 2*halo > core
    assert lib.wo_tile_gather(fake, 4, 0, 2, 16, 4, fake, None) == 2
    assert lib.wo_tile_blend(None, 4, 2, 2, 16, 4, fake, None) == 1
    assert lib.wo_tile_blend(fake, 4, 2, 2, 16, -1, fake, None) == 2


def test_pad_validation(B):
    lib = B._lib
    fake, other = 1 << 20, 1 << 21
    assert lib.wo_pad(fake, 1, 4, 4, 4, 8, 8, 8, 3, other, None) == 1     # unknown mode
    assert lib.wo_pad(fake, 1, 4, 4, 4, 8, 8, 8, 0, fake, None) == 1      # in place
    assert lib.wo_pad(None, 1, 4, 4, 4, 8, 8, 8, 0, other, None) == 1
    assert lib.wo_pad(fake, 1, 4, 4, 4, 8, 3, 8, 1, other, None) == 2     # padded axis shorter
    assert lib.wo_pad(fake, 0, 4, 4, 4, 8, 8, 8, 1, other, None) == 2
    assert lib.wo_crop(fake, 1, 8, 8, 8, 4, 9, 4, other, None) == 2       # window larger than the volume
    assert lib.wo_crop(fake, 1, 8, 8, 8, 4, 4, 4, fake, None) == 1


def test_status_block_entry_points(B):
    lib = B._lib
    # the status block leads every workspace: the sizes grow by it
    n, Z, Y, X = 2, 16, 64, 64
    assert B.wo_workspace_bytes(n, Z, Y, X, 1) >= 256 + 2 * n * Z * Y * (X // 2 + 1) * 8
    assert B.wo_fused_workspace_bytes(3, n, Z, Y, X) >= 256 + 4 * n * Z * Y * (X // 2 + 1) * 8
    info = (ctypes.c_int * 2)()
    assert lib.wo_sync_status(None, info, None) == 1
    assert lib.wo_sync_status((1 << 20) + 8, info, None) == 1   # misaligned
    assert lib.wo_clear_status(None, None) == 1
    fake, big = 1 << 20, 1 << 40
    probe = lib.wo_pipeline_probe
    assert probe(fake, fake, fake, 2, 48, 192, 192, 2, 10 ** 6, fake, big, None) == 1      # withhold >= n_tiles
    assert probe(fake, fake, fake, 2, 48, 192, 192, -2, 10 ** 6, fake, big, None) == 1
    assert probe(fake, fake, fake, 2, 48, 192, 192, 0, 10, fake, big, None) == 1           # budget below 1 us
    assert probe(fake, fake, fake, 2, 48, 96, 96, 0, 10 ** 6, fake, big, None) == 3        # no pipeline for 96
    assert probe(fake, fake, fake, 2, 48, 192, 192, 0, 10 ** 6, fake, 1024, None) == 8     # workspace
    assert probe(fake + 4, fake, fake, 2, 48, 192, 192, 0, 10 ** 6, fake, big, None) == 1  # misaligned
    assert B.STATUS[9] == "WO_ERR_BOUNDS" and "WO_CHECK" in B.wo_status_string(9)


def test_status_strings(B):
    for s in range(9):
        assert B.wo_status_string(s)
    assert B.wo_status_string(99) == "unknown status"


def test_device_optics_build_validation(B):
    lib = B._lib
    fake = 1 << 20
    big = 1 << 40
    f = lib.wo_build_tf_device
    assert f(fake + 4, 1, 16, 64, 64, 1, fake, fake, big, None) == 1   # optics not 8-byte aligned
    assert f(None, 1, 16, 64, 64, 1, fake, fake, big, None) == 1
    assert f(fake, 1, 16, 64, 64, 1, fake + 8, fake, big, None) == 1   # TF bank not 16-byte aligned
    assert f(fake, 1, 16, 64, 63, 1, fake, fake, big, None) == 2       # odd X
    assert f(fake, 1, 16, 64, 62, 1, fake, fake, big, None) == 3       # X/2 = 31
    assert f(fake, 1, 16, 64, 64, 1, fake, fake, 1024, None) == 8      # workspace too small


def test_fusion_validation(B):
    lib = B._lib
    fake = 1 << 20
    big = 1 << 40
    Z, Y, X = 16, 64, 64
    half = Z * Y * (X // 2 + 1) * 8

    def a256(n):
        return (n + 255) // 256 * 256

    # nine apertures of two tiles: the status block, all channel spectra, one fused spectrum per tile, two
    # floats per tile
    assert B.wo_fused_workspace_bytes(9, 2, Z, Y, X) == 256 + a256(18 * half) + a256(2 * half) + a256(2 * 2 * 4)
    assert B.wo_fused_workspace_bytes(17, 1, Z, Y, X) == 0     # more than 16 channels
    assert B.wo_fused_workspace_bytes(9, 7282, Z, Y, X) == 0   # more than 65535 TF entries
    assert B.wo_fused_workspace_bytes(9, 1, Z, Y, 63) == 0     # odd X
    g = lib.wo_reconstruct_fused
    F = ctypes.c_float
    nan_bg = (F * 9)(*([1.0] * 8 + [float("nan")]))
    pb = ctypes.cast(nan_bg, ctypes.POINTER(F))
    ok = (fake, 9, fake, None, 1e-3, 0, 0, fake, 1, Z, Y, X, fake, big, None)

    def call(**kw):
        names = ("tf", "C", "d", "bg", "eta", "flag", "mode", "f", "n", "Z", "Y", "X", "ws", "wsb", "s")
        args = dict(zip(names, ok))
        args.update(kw)
        return g(*[args[n] for n in names])

    assert call(C=0) == 1 and call(C=17) == 1
    assert call(flag=2) == 1 and call(mode=5) == 1
    assert call(eta=-1.0) == 1 and call(eta=float("nan")) == 1 and call(eta=float("inf")) == 1
    assert call(bg=pb) == 1                       # a non-finite background
    assert call(d=fake + 4) == 1 and call(f=None) == 1
    assert call(X=63) == 2 and call(X=62) == 3
    assert call(wsb=1024) == 8


def test_estimator_validation(B):
    lib = B._lib
    from oracle import estimator as E
    # conv 3->32->64->96->128 (3x3, with biases), linear 128->4: the header's
    # network, counted by hand, and the oracle's parameter list agree
    n = sum(ci * co * 9 + co for ci, co in ((3, 32), (32, 64), (64, 96), (96, 128))) + 128 * 4 + 4
    assert B._lib.wo_est_param_count() == n == E.n_params() == 186020
    ws1, ws64 = lib.wo_est_workspace_bytes(1), lib.wo_est_workspace_bytes(64)
    assert 0 < ws1 < ws64 and lib.wo_est_workspace_bytes(4096) > ws64
    assert lib.wo_est_workspace_bytes(0) == 0 and lib.wo_est_workspace_bytes(4097) == 0
    fake = 1 << 20
    big = 1 << 40
    F = ctypes.c_float
    sc = (F * 4)(1.0, 1.0, 1.0, 1.0)
    off = (F * 4)(0.0, 0.0, 0.0, 0.0)
    zero = (F * 4)(1.0, 0.0, 1.0, 1.0)
    ps, po, pz = (ctypes.cast(a, ctypes.POINTER(F)) for a in (sc, off, zero))
    fwd = lib.wo_est_forward
    assert fwd(fake, fake, fake, 0, ps, po, fake, fake, big, None) == 1       # batch 0
    assert fwd(fake, fake, fake, 4097, ps, po, fake, fake, big, None) == 1    # batch above 4096
    assert fwd(fake, fake, fake + 8, 4, ps, po, fake, fake, big, None) == 1   # misaligned features
    assert fwd(fake, fake, fake, 4, pz, po, fake, fake, big, None) == 1       # a zero scale
    assert fwd(fake, fake, fake, 4, None, po, fake, fake, big, None) == 1
    assert fwd(fake, fake, fake, 4, ps, po, fake, fake, ws1, None) == 8       # workspace for one tile
    bwd = lib.wo_est_backward
    assert bwd(fake, fake, fake, fake + 4, 4, ps, po, None, None, fake, big, None) == 1  # misaligned targets
    assert bwd(fake, fake, fake, fake, 4, ps, po, fake + 4, None, fake, big, None) == 1  # misaligned gradient
    step = lib.wo_est_train_step
    assert step(fake, fake, fake, fake, fake, fake, 4, ps, po, 0, 1e-3, None, fake, big, None) == 1  # step 0
    assert step(fake, fake, fake, fake, fake, fake, 4, ps, po, 1, -1e-3, None, fake, big, None) == 1
    assert step(fake, fake, fake, fake, fake, fake, 4, ps, po, 1, float("nan"), None, fake, big, None) == 1
    assert step(fake, fake, fake + 8, fake, fake, fake, 4, ps, po, 1, 1e-3, None, fake, big, None) == 1
    assert lib.wo_est_sync_bf16(fake + 8, fake, None) == 1
    feat = lib.wo_est_features
    assert feat(fake, fake, 4, 1, 64, 64, fake, None) == 2     # one plane
    assert feat(fake, fake, 4, 65, 64, 64, fake, None) == 2    # more than 64 planes
    assert feat(fake, fake, 4, 16, 64, 63, fake, None) == 2    # odd X
    assert feat(fake, fake + 4, 4, 16, 64, 64, fake, None) == 1
    ph_ = lib.wo_thin_phantom
    assert ph_(fake, 4, -1, 64, 64, 0.1, 0.25, fake, None) == 2
    assert ph_(fake, 4, 8, 64, 64, 0.0, 0.25, fake, None) == 1
    assert ph_(fake, 4, 8, 64, 64, 0.1, float("nan"), fake, None) == 1
    assert ph_(fake + 4, 4, 8, 64, 64, 0.1, 0.25, fake, None) == 1


def test_launch_counter_is_host_side(B):
    # counting needs no device: failed validations launch nothing
    n0 = B._lib.wo_launch_count()
    assert B._lib.wo_forward(1 << 20, 7, (1 << 20) + 8, None, 1 << 20, 1, 16, 64, 64, 1 << 20, 1 << 40, None) == 1
    assert B._lib.wo_launch_count() == n0


def test_field_tiles_validation(B):
    # the in-place field-tile reconstruction rejects what it cannot do before launching
    lib = B._lib
    fake = 1 << 20
    big = 1 << 40
    eta = B._floats([1e-3, 1e-3])

    def call(kinds, Z, ty, tx, core, halo):
        return lib.wo_reconstruct_field_tiles(fake, kinds, fake, Z, ty, tx, core, halo, None, eta[0], 0, 0, fake,
                                              fake, big, None)
    assert call(1 | 4, 16, 2, 2, 48, 8) == 1      # two data channels
    assert call(1, 16, 2, 2, 48, 25) == 1         # 2 halo > core
    assert call(1, 16, 0, 2, 48, 8) == 1          # no tiles
    assert call(1, 16, 2, 2, 52, 4) == 3          # E = 60: no 30-point register rows


def test_restore_field_validation(B):
    lib = B._lib
    fake = 1 << 20
    big = 1 << 40
    eta = B._floats([1e-3, 1e-3])

    def call(kinds, ty, tx, core, halo, out=fake + 256):
        return lib.wo_restore_field(fake, kinds, fake, 16, ty, tx, core, halo, None, eta[0], 0, 0, out, fake, big,
                                    None)
    assert call(1, 2, 2, 48, 8, out=fake) == 1    # output over the input field
    assert call(1, 2, 65, 48, 8) == 1             # more than 64 tiles across
    assert call(1 | 4, 2, 2, 48, 8) == 1          # two data channels
    assert call(1, 2, 2, 52, 4) == 3              # E = 60: no 30-point register rows


def test_kx_major_validation(B):
    """WO_TF_KX_MAJOR: one kind, 3D TFs, the plane engine's shapes; same bank
    size as the standard layout; the 2D solve and the fused blend refuse it
    before launching anything."""
    K = B.WO_TF_KX_MAJOR
    for Z, E in ((48, 192), (48, 128), (48, 64), (32, 192), (32, 128), (32, 64), (16, 64)):
        for kind in (1, 2, 4):
            assert B.wo_tf_bytes(3, Z, E, E, kind | K) == B.wo_tf_bytes(3, Z, E, E, kind) > 0
    assert B.wo_tf_bytes(1, 48, 192, 192, 1 | 32 | K) > 0          # smooth source
    assert B.wo_tf_bytes(1, 48, 192, 192, 1 | 2 | K) == 0          # two kinds
    assert B.wo_tf_bytes(1, 48, 192, 192, 8 | K) == 0              # derivative banks
    assert B.wo_tf_bytes(1, 48, 192, 192, 8 | 16 | K) == 0
    assert B.wo_tf_bytes(1, 48, 192, 192, K) == 0                  # no kind
    assert B.wo_tf_bytes(1, 16, 128, 128, 1 | K) == 0              # 16 planes: 64-point planes only
    assert B.wo_tf_bytes(1, 96, 192, 192, 1 | K) == 0
    assert B.wo_tf_bytes(1, 48, 256, 256, 1 | K) == 0              # Y outside the plane engine
    assert B.wo_tf_bytes(1, 48, 96, 96, 1 | K) == 0
    assert B.wo_tf_bytes(1, 48, 192, 256, 1 | K) == 0              # 256-point PSF rows
    assert B.wo_tf_bytes(1, 48, 128, 192, 1 | K) == 0              # planes not square
    assert B.wo_tf_bytes(1, 48, 192, 192, 1 | 256) == 0            # unknown bit
    lib = B._lib
    fake = 1 << 20
    big = 1 << 40
    eta = B._floats([1e-3, 1e-3])
    n0 = lib.wo_launch_count()
    m = 1 | K
    assert lib.wo_reconstruct(fake, m, fake, None, eta[0], 0, 1, fake, 4, 32, 64, 64, fake, big, None) == 1  # 2D
    assert lib.wo_forward(fake, m, fake, None, fake, 4, 32, 64, 128, fake, big, None) == 3  # not square
    assert lib.wo_reconstruct_field_tiles(fake, m, fake, 32, 2, 2, 48, 8, None, eta[0], 0, 1, fake, fake, big,
                                          None) == 1               # 2D mode
    assert lib.wo_restore_field(fake, m, fake, 32, 2, 2, 48, 8, None, eta[0], 0, 0, fake + 256, fake, big,
                                None) == 1
    assert lib.wo_reconstruct_field_tiles(fake, m, fake, 64, 2, 2, 48, 8, None, eta[0], 0, 0, fake, fake, big,
                                          None) == 3               # Z = 64: no plane engine
    assert lib.wo_launch_count() == n0
