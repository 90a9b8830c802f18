"""ctypes binding of the C ABI in include/wo.h (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: it converts torch tensors to device pointers and
the current torch stream to a cudaStream_t, calls the library, and raises
``WoError`` on a non-zero status.  The library is loaded from the in-tree
build (``paper_2412_09775_gb300/lib/libwo_gb300.so``, or its WO_CHECK variant
``libwo_gb300_check.so`` when the environment sets WO_LIB=check); if it is
missing the import of this module fails loudly - there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libwo_gb300_check.so" if os.environ.get("WO_LIB") == "check"
                        else "libwo_gb300.so")

WO_TF_PHASE, WO_TF_ABSORPTION, WO_TF_FLUOR = 1, 2, 4
WO_TF_PHASE_DZ = 8
WO_TF_PLANES = 16
WO_TF_SMOOTH_SOURCE = 32
WO_TF_PHASE_GRAD = 64
WO_TF_KX_MAJOR = 128
WO_MODE_3D, WO_MODE_2D = 0, 1
WO_ETA_RELATIVE, WO_ETA_ABSOLUTE = 0, 1
WO_LOSS_DATA, WO_LOSS_MIDBAND = 0, 1
WO_PASS_COLS, WO_PASS_ROWS, WO_PASS_RECON, WO_PASS_XY = 0, 1, 2, 3
WO_ENGINE_DEFAULT, WO_ENGINE_SMEM, WO_ENGINE_HYBRID = 0, 1, 2
WO_MAX_ZERNIKE = 36
WO_PAD_ZERO, WO_PAD_MIRROR, WO_PAD_EDGE = 0, 1, 2
KIND_BITS = {"phase": WO_TF_PHASE, "absorption": WO_TF_ABSORPTION, "fluor": WO_TF_FLUOR,
             "phase_dz": WO_TF_PHASE_DZ, "planes": WO_TF_PLANES, "smooth_source": WO_TF_SMOOTH_SOURCE,
             "phase_grad": WO_TF_PHASE_GRAD, "kx_major": WO_TF_KX_MAJOR}
STATUS = {0: "WO_OK", 1: "WO_ERR_ARG", 2: "WO_ERR_SHAPE", 3: "WO_ERR_UNSUPPORTED_SIZE",
          4: "WO_ERR_UNDERSAMPLED", 5: "WO_ERR_CUDA", 6: "WO_ERR_TIMEOUT", 7: "WO_ERR_OPTICS",
          8: "WO_ERR_WORKSPACE", 9: "WO_ERR_BOUNDS"}

STATUS_CODES = {v: k for k, v in STATUS.items()}

OPTICS_FIELDS = ("lambda_um", "n_medium", "pixel_um", "z_step_um", "na_det", "na_ill",
                 "tilt_x", "tilt_y", "defocus_um")


class wo_optics(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in OPTICS_FIELDS]


class WoError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} ({_string(status)})")


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run paper_2412_09775_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i, u, sz, f = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint, ctypes.c_size_t, ctypes.c_float
    fp = ctypes.POINTER(ctypes.c_float)
    sig = {
        "wo_size_supported": (i, [i]),
        "wo_tf_bytes": (sz, [i, i, i, i, u]),
        "wo_workspace_bytes": (sz, [i, i, i, i, u]),
        "wo_build_tf": (i, [ctypes.POINTER(wo_optics), i, i, i, i, u, vp, vp, sz, vp]),
        "wo_build_tf_device": (i, [vp, i, i, i, i, u, vp, vp, sz, vp]),
        "wo_aberrated_workspace_bytes": (sz, [i, i, i, i, u]),
        "wo_build_tf_aberrated": (i, [ctypes.POINTER(wo_optics), ctypes.POINTER(ctypes.c_double), i, i, i, i, i, u,
                                      vp, vp, sz, vp]),
        "wo_forward": (i, [vp, u, vp, fp, vp, i, i, i, i, vp, sz, vp]),
        "wo_forward_adjoint": (i, [vp, u, vp, fp, vp, i, i, i, i, vp, sz, vp]),
        "wo_reconstruct": (i, [vp, u, vp, fp, fp, i, i, vp, i, i, i, i, vp, sz, vp]),
        "wo_reconstruct_static": (i, [vp, u, vp, fp, fp, i, i, vp, i, i, i, i, vp]),
        "wo_reconstruct_shared_tf": (i, [vp, u, vp, fp, fp, i, i, vp, i, i, i, i, vp, sz, vp]),
        "wo_reconstruct_field_tiles": (i, [vp, u, vp, i, i, i, i, i, fp, fp, i, i, vp, vp, sz, vp]),
        "wo_restore_field": (i, [vp, u, vp, i, i, i, i, i, fp, fp, i, i, vp, vp, sz, vp]),
        "wo_clear_status": (i, [vp, vp]),
        "wo_sync_status": (i, [vp, ctypes.POINTER(ctypes.c_int), vp]),
        "wo_check_build": (i, []),
        "wo_pipeline_probe": (i, [vp, vp, vp, i, i, i, i, i, ctypes.c_longlong, vp, sz, vp]),
        "wo_spectrum": (i, [vp, fp, i, vp, i, i, i, i, vp]),
        "wo_tune_objective": (i, [vp, u, vp, vp, i, f, f, vp, vp, i, i, i, i, vp, sz, vp]),
        "wo_reconstruct_vjp": (i, [vp, u, vp, vp, f, i, vp, i, i, i, i, vp, sz, vp]),
        "wo_adam_optics": (i, [vp, vp, i, vp, i, ctypes.POINTER(ctypes.c_double), ctypes.c_double,
                               ctypes.c_double, ctypes.c_double, vp]),
        "wo_fused_workspace_bytes": (sz, [i, i, i, i, i]),
        "wo_reconstruct_fused": (i, [vp, i, vp, fp, f, i, i, vp, i, i, i, i, vp, sz, vp]),
        "wo_est_param_count": (sz, []),
        "wo_est_workspace_bytes": (sz, [i]),
        "wo_est_activation_offset": (sz, [i, i]),
        "wo_est_sync_bf16": (i, [vp, vp, vp]),
        "wo_est_forward": (i, [vp, vp, vp, i, fp, fp, vp, vp, sz, vp]),
        "wo_est_backward": (i, [vp, vp, vp, vp, i, fp, fp, vp, vp, vp, sz, vp]),
        "wo_est_train_step": (i, [vp, vp, vp, vp, vp, vp, i, fp, fp, i, f, vp, vp, sz, vp]),
        "wo_est_features": (i, [vp, vp, i, i, i, i, vp, vp]),
        "wo_thin_phantom": (i, [vp, i, i, i, i, ctypes.c_double, ctypes.c_double, vp, vp]),
        "wo_schedule_set": (i, [i, i, i]),
        "wo_schedule_get": (i, [i, i]),
        "wo_autotune": (i, [i, i, i, i, u, vp, sz, vp]),
        "wo_tile_gather": (i, [vp, i, i, i, i, i, vp, vp]),
        "wo_tile_blend": (i, [vp, i, i, i, i, i, vp, vp]),
        "wo_pad": (i, [vp, i, i, i, i, i, i, i, i, vp, vp]),
        "wo_crop": (i, [vp, i, i, i, i, i, i, i, vp, vp]),
        "wo_status_string": (ctypes.c_char_p, [i]),
        "wo_profile_enable": (None, [i]),
        "wo_profile_read": (i, [ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_longlong),
                                ctypes.POINTER(ctypes.c_double), i]),
        "wo_launch_count": (ctypes.c_longlong, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()
EXPORTED = ("wo_size_supported", "wo_tf_bytes", "wo_workspace_bytes", "wo_build_tf", "wo_build_tf_device",
            "wo_aberrated_workspace_bytes", "wo_build_tf_aberrated",
            "wo_forward",
            "wo_forward_adjoint", "wo_reconstruct", "wo_reconstruct_static", "wo_reconstruct_shared_tf",
            "wo_reconstruct_field_tiles", "wo_restore_field", "wo_clear_status", "wo_sync_status", "wo_check_build", "wo_pipeline_probe", "wo_spectrum",
            "wo_tune_objective", "wo_reconstruct_vjp", "wo_adam_optics", "wo_fused_workspace_bytes", "wo_reconstruct_fused",
            "wo_est_param_count", "wo_est_workspace_bytes", "wo_est_activation_offset", "wo_est_sync_bf16", "wo_est_forward", "wo_est_backward",
            "wo_est_train_step", "wo_est_features", "wo_thin_phantom",
            "wo_schedule_set", "wo_schedule_get", "wo_autotune", "wo_tile_gather", "wo_tile_blend",
            "wo_pad", "wo_crop",
            "wo_status_string", "wo_profile_enable", "wo_profile_read", "wo_launch_count")


def _string(status: int) -> str:
    return _lib.wo_status_string(int(status)).decode()


def _check(status: int, where: str):
    if status != 0:
        raise WoError(status, where)


def _ptr(x):
    """Device pointer of a tensor (or an int address); None -> NULL."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _nbytes(x) -> int:
    return x.numel() * x.element_size()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


def _floats(vals):
    if vals is None:
        return None
    arr = (ctypes.c_float * len(vals))(*[float(v) for v in vals])
    return ctypes.cast(arr, ctypes.POINTER(ctypes.c_float)), arr


def kinds_mask(kinds) -> int:
    if isinstance(kinds, int):
        return kinds
    if isinstance(kinds, str):
        kinds = (kinds,)
    m = 0
    for k in kinds:
        m |= KIND_BITS[k]
    return m


def optics_array(optics_list):
    arr = (wo_optics * len(optics_list))()
    for i, o in enumerate(optics_list):
        for k in OPTICS_FIELDS:
            setattr(arr[i], k, float(o[k]))
    return arr


# ------------------------------------------------------------- entry points
def wo_size_supported(n: int) -> bool:
    return bool(_lib.wo_size_supported(int(n)))


def wo_tf_bytes(n_tiles, Z, Y, X, kinds) -> int:
    return int(_lib.wo_tf_bytes(n_tiles, Z, Y, X, kinds_mask(kinds)))


def wo_workspace_bytes(n_tiles, Z, Y, X, kinds) -> int:
    return int(_lib.wo_workspace_bytes(n_tiles, Z, Y, X, kinds_mask(kinds)))


def wo_build_tf(optics_list, n_tiles, Z, Y, X, kinds, tf, ws, stream=None):
    arr = optics_array(optics_list)
    if len(optics_list) != n_tiles:
        raise ValueError("one optics entry per tile")
    _check(_lib.wo_build_tf(arr, n_tiles, Z, Y, X, kinds_mask(kinds), _ptr(tf), _ptr(ws),
                            _nbytes(ws), _stream(stream)), "wo_build_tf")


def wo_build_tf_device(d_optics, n_tiles, Z, Y, X, kinds, tf, ws, stream=None):
    """TF build with the optics in device memory (a float64 tensor [n_tiles, 9])."""
    _check(_lib.wo_build_tf_device(_ptr(d_optics), n_tiles, Z, Y, X, kinds_mask(kinds), _ptr(tf), _ptr(ws),
                                   _nbytes(ws), _stream(stream)), "wo_build_tf_device")


def wo_aberrated_workspace_bytes(n_tiles, Z, Y, X, kinds) -> int:
    return int(_lib.wo_aberrated_workspace_bytes(n_tiles, Z, Y, X, kinds_mask(kinds)))


def wo_build_tf_aberrated(optics_list, zernike, n_tiles, Z, Y, X, kinds, tf, ws, stream=None):
    """TF build with aberrated detection pupils: ``zernike`` [n_tiles, n_zernike]
    Noll coefficients in waves (c_1 first)."""
    if len(optics_list) != n_tiles:
        raise ValueError("one optics entry per tile")
    arr = optics_array(optics_list)
    nz = len(zernike[0]) if n_tiles > 0 and len(zernike) > 0 else 0
    if len(zernike) != n_tiles or any(len(row) != nz for row in zernike):
        raise ValueError("zernike: one row of equal length per tile")
    flat = (ctypes.c_double * max(n_tiles * nz, 1))(*[float(v) for row in zernike for v in row])
    _check(_lib.wo_build_tf_aberrated(arr, flat, nz, n_tiles, Z, Y, X, kinds_mask(kinds), _ptr(tf), _ptr(ws),
                                      _nbytes(ws), _stream(stream)), "wo_build_tf_aberrated")


def optics_tensor(optics_list, device="cuda"):
    """Device array of optics structs (float64 [n, 9], field order of wo_optics)."""
    import torch
    return torch.tensor([[float(o[k]) for k in OPTICS_FIELDS] for o in optics_list], dtype=torch.float64,
                        device=device)


def wo_forward(tf, kinds, f, background, data, n_tiles, Z, Y, X, ws, stream=None):
    bg = _floats(background)
    _check(_lib.wo_forward(_ptr(tf), kinds_mask(kinds), _ptr(f), bg[0] if bg else None, _ptr(data),
                           n_tiles, Z, Y, X, _ptr(ws), _nbytes(ws), _stream(stream)), "wo_forward")


def wo_forward_adjoint(tf, kinds, data, background, f, n_tiles, Z, Y, X, ws, stream=None):
    bg = _floats(background)
    _check(_lib.wo_forward_adjoint(_ptr(tf), kinds_mask(kinds), _ptr(data), bg[0] if bg else None,
                                   _ptr(f), n_tiles, Z, Y, X, _ptr(ws), _nbytes(ws), _stream(stream)),
           "wo_forward_adjoint")


def wo_reconstruct(tf, kinds, data, background, eta, eta_flag, mode, f, n_tiles, Z, Y, X, ws, stream=None):
    bg = _floats(background)
    et = _floats(eta if isinstance(eta, (list, tuple)) else [eta])
    _check(_lib.wo_reconstruct(_ptr(tf), kinds_mask(kinds), _ptr(data), bg[0] if bg else None, et[0],
                               int(eta_flag), int(mode), _ptr(f), n_tiles, Z, Y, X, _ptr(ws), _nbytes(ws),
                               _stream(stream)), "wo_reconstruct")


def wo_reconstruct_field_tiles(tf, kinds, field, Z, tiles_y, tiles_x, core, halo, background, eta, eta_flag, mode,
                               f, ws, stream=None):
    """wo_reconstruct of the tiles of `field` [Z][tiles_y*core][tiles_x*core]
    (f: [tiles][P][Z][E][E], E = core + 2 halo) without gathering them first."""
    bg = _floats(background)
    et = _floats(eta if isinstance(eta, (list, tuple)) else [eta])
    _check(_lib.wo_reconstruct_field_tiles(_ptr(tf), kinds_mask(kinds), _ptr(field), int(Z), int(tiles_y),
                                           int(tiles_x), int(core), int(halo), bg[0] if bg else None, et[0],
                                           int(eta_flag), int(mode), _ptr(f), _ptr(ws), _nbytes(ws), _stream(stream)),
           "wo_reconstruct_field_tiles")


def wo_restore_field(tf, kinds, field, Z, tiles_y, tiles_x, core, halo, background, eta, eta_flag, mode, out, ws,
                     stream=None):
    """Reconstruct the tiles of `field` read in place and blend them into
    `out` [P][Z][tiles_y*core][tiles_x*core] in one call."""
    bg = _floats(background)
    et = _floats(eta if isinstance(eta, (list, tuple)) else [eta])
    _check(_lib.wo_restore_field(_ptr(tf), kinds_mask(kinds), _ptr(field), int(Z), int(tiles_y), int(tiles_x),
                                 int(core), int(halo), bg[0] if bg else None, et[0], int(eta_flag), int(mode),
                                 _ptr(out), _ptr(ws), _nbytes(ws), _stream(stream)), "wo_restore_field")


def wo_reconstruct_shared_tf(tf, kinds, data, background, eta, eta_flag, mode, f, n_tiles, Z, Y, X, ws,
                             stream=None):
    """wo_reconstruct of n_tiles stacks with one TF bank (built for one tile) shared by all of them."""
    bg = _floats(background)
    et = _floats(eta if isinstance(eta, (list, tuple)) else [eta])
    _check(_lib.wo_reconstruct_shared_tf(_ptr(tf), kinds_mask(kinds), _ptr(data), bg[0] if bg else None, et[0],
                                         int(eta_flag), int(mode), _ptr(f), n_tiles, Z, Y, X, _ptr(ws), _nbytes(ws),
                                         _stream(stream)), "wo_reconstruct_shared_tf")


WO_STATIC_SCRATCH_BYTES = 32 * 1024 * 1024


def wo_reconstruct_static(tf, kinds, data, background, eta, eta_flag, mode, f, n_tiles, Z, Y, X, stream=None):
    """wo_reconstruct with the library's own fixed device workspace (no allocation)."""
    bg = _floats(background)
    et = _floats(eta if isinstance(eta, (list, tuple)) else [eta])
    _check(_lib.wo_reconstruct_static(_ptr(tf), kinds_mask(kinds), _ptr(data), bg[0] if bg else None, et[0],
                                      int(eta_flag), int(mode), _ptr(f), n_tiles, Z, Y, X, _stream(stream)),
           "wo_reconstruct_static")


def wo_clear_status(ws, stream=None):
    """Zero the status block at the start of a workspace (once, before its first use)."""
    _check(_lib.wo_clear_status(_ptr(ws), _stream(stream)), "wo_clear_status")


def wo_sync_status(ws, stream=None):
    """Wait for the stream, read and clear the workspace's status block:
    (status code, site, detail); code 0 when no device-side error was recorded."""
    info = (ctypes.c_int * 2)()
    code = int(_lib.wo_sync_status(_ptr(ws), info, _stream(stream)))
    return code, int(info[0]), int(info[1])


def wo_check_build() -> bool:
    """True for the WO_CHECK variant of the library (kernels test their indices)."""
    return bool(_lib.wo_check_build())


def wo_pipeline_probe(tf, data, f, n_tiles, Z, Y, X, withhold, budget_ns, ws, stream=None):
    """The tile pipeline with one tile's plane items withheld and a wait budget (diagnostic)."""
    _check(_lib.wo_pipeline_probe(_ptr(tf), _ptr(data), _ptr(f), n_tiles, Z, Y, X, int(withhold), int(budget_ns),
                                  _ptr(ws), _nbytes(ws), _stream(stream)), "wo_pipeline_probe")


def wo_spectrum(data, background, mode, spec, n_tiles, Z, Y, X, stream=None):
    """Half spectra [n, Z, Y, X/2+1] (complex64 tensor `spec`) of brightfield stacks, 3D or per plane."""
    bg = _floats(background)
    _check(_lib.wo_spectrum(_ptr(data), bg[0] if bg else None, int(mode), _ptr(spec), n_tiles, Z, Y, X,
                            _stream(stream)), "wo_spectrum")


def wo_tune_objective(tf, kinds, d_optics, spec, loss, eta, nu_max, value, grad, n_tiles, Z, Y, X, ws,
                      stream=None):
    """Per-tile loss [n] and derivatives [n, n_params] (float64 tensors or None) from a derivative bank."""
    _check(_lib.wo_tune_objective(_ptr(tf), kinds_mask(kinds), _ptr(d_optics), _ptr(spec), int(loss), float(eta),
                                  float(nu_max), _ptr(value), _ptr(grad), n_tiles, Z, Y, X, _ptr(ws), _nbytes(ws),
                                  _stream(stream)), "wo_tune_objective")


def wo_reconstruct_vjp(tf, kinds, spec, gout, eta, mode, grad, n_tiles, Z, Y, X, ws, stream=None):
    """dL/dtheta [n, n_params] (float64 tensor `grad`) of the phase reconstruction for an upstream gradient gout."""
    _check(_lib.wo_reconstruct_vjp(_ptr(tf), kinds_mask(kinds), _ptr(spec), _ptr(gout), float(eta), int(mode),
                                   _ptr(grad), n_tiles, Z, Y, X, _ptr(ws), _nbytes(ws), _stream(stream)),
           "wo_reconstruct_vjp")


def wo_adam_optics(d_optics, grad, n_params, state, n_tiles, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """One on-device Adam step on each tile's tuned parameters (state: float64 [n, n_params, 3], zeroed first)."""
    lrs = lr if isinstance(lr, (list, tuple)) else [lr] * n_params
    arr = (ctypes.c_double * n_params)(*[float(v) for v in lrs])
    _check(_lib.wo_adam_optics(_ptr(d_optics), _ptr(grad), int(n_params), _ptr(state), n_tiles, arr, float(beta1),
                               float(beta2), float(eps), _stream(stream)), "wo_adam_optics")


def wo_fused_workspace_bytes(n_channels, n_tiles, Z, Y, X) -> int:
    return int(_lib.wo_fused_workspace_bytes(n_channels, n_tiles, Z, Y, X))


def wo_reconstruct_fused(tf, n_channels, data, background, eta, eta_flag, mode, f, n_tiles, Z, Y, X, ws,
                         stream=None):
    """One property from n_channels data channels, each through its own phase TF (bank of n_tiles*C entries)."""
    bg = _floats(background)
    _check(_lib.wo_reconstruct_fused(_ptr(tf), int(n_channels), _ptr(data), bg[0] if bg else None, float(eta),
                                     int(eta_flag), int(mode), _ptr(f), n_tiles, Z, Y, X, _ptr(ws), _nbytes(ws),
                                     _stream(stream)), "wo_reconstruct_fused")


def wo_est_param_count() -> int:
    return int(_lib.wo_est_param_count())


def wo_est_workspace_bytes(batch) -> int:
    return int(_lib.wo_est_workspace_bytes(int(batch)))


def wo_est_activation_offset(batch, layer) -> int:
    return int(_lib.wo_est_activation_offset(int(batch), int(layer)))


def wo_est_sync_bf16(w32, wbf16, stream=None):
    _check(_lib.wo_est_sync_bf16(_ptr(w32), _ptr(wbf16), _stream(stream)), "wo_est_sync_bf16")


def wo_est_forward(wbf16, w32, feat, batch, scale, offset, out, ws, stream=None):
    sc, off = _floats(scale), _floats(offset)
    _check(_lib.wo_est_forward(_ptr(wbf16), _ptr(w32), _ptr(feat), int(batch), sc[0], off[0], _ptr(out), _ptr(ws),
                               _nbytes(ws), _stream(stream)), "wo_est_forward")


def wo_est_backward(wbf16, w32, feat, target, batch, scale, offset, grad, loss, ws, stream=None):
    sc, off = _floats(scale), _floats(offset)
    _check(_lib.wo_est_backward(_ptr(wbf16), _ptr(w32), _ptr(feat), _ptr(target), int(batch), sc[0], off[0],
                                _ptr(grad), _ptr(loss), _ptr(ws), _nbytes(ws), _stream(stream)), "wo_est_backward")


def wo_est_train_step(w32, wbf16, m, v, feat, target, batch, scale, offset, step, lr, loss, ws, stream=None):
    sc, off = _floats(scale), _floats(offset)
    _check(_lib.wo_est_train_step(_ptr(w32), _ptr(wbf16), _ptr(m), _ptr(v), _ptr(feat), _ptr(target), int(batch),
                                  sc[0], off[0], int(step), float(lr), _ptr(loss), _ptr(ws), _nbytes(ws),
                                  _stream(stream)), "wo_est_train_step")


def wo_est_features(spec, d_optics, n_tiles, Z, Y, X, feat, stream=None):
    _check(_lib.wo_est_features(_ptr(spec), _ptr(d_optics), n_tiles, Z, Y, X, _ptr(feat), _stream(stream)),
           "wo_est_features")


def wo_thin_phantom(params, n_tiles, n_spheres, Y, X, pixel_um, z_step_um, out, stream=None):
    _check(_lib.wo_thin_phantom(_ptr(params), n_tiles, n_spheres, Y, X, float(pixel_um), float(z_step_um), _ptr(out),
                                _stream(stream)), "wo_thin_phantom")


def wo_schedule_set(pass_, n, engine):
    _check(_lib.wo_schedule_set(int(pass_), int(n), int(engine)), "wo_schedule_set")


def wo_schedule_get(pass_, n) -> int:
    return int(_lib.wo_schedule_get(int(pass_), int(n)))


def wo_autotune(n_tiles, Z, Y, X, kinds, ws, stream=None):
    """Time the engines of the column transforms for these shapes and keep the fastest (destroys ws)."""
    _check(_lib.wo_autotune(n_tiles, Z, Y, X, kinds_mask(kinds), _ptr(ws), _nbytes(ws), _stream(stream)),
           "wo_autotune")


def wo_tile_gather(field, Z, tiles_y, tiles_x, core, halo, tiles, stream=None):
    _check(_lib.wo_tile_gather(_ptr(field), Z, tiles_y, tiles_x, core, halo, _ptr(tiles), _stream(stream)),
           "wo_tile_gather")


def wo_tile_blend(tiles, Z, tiles_y, tiles_x, core, halo, field, stream=None):
    _check(_lib.wo_tile_blend(_ptr(tiles), Z, tiles_y, tiles_x, core, halo, _ptr(field), _stream(stream)),
           "wo_tile_blend")


def wo_pad(vol, n_vol, Z, Y, X, Zp, Yp, Xp, mode, out, stream=None):
    _check(_lib.wo_pad(_ptr(vol), n_vol, Z, Y, X, Zp, Yp, Xp, int(mode), _ptr(out), _stream(stream)), "wo_pad")


def wo_crop(vol, n_vol, Zp, Yp, Xp, Z, Y, X, out, stream=None):
    _check(_lib.wo_crop(_ptr(vol), n_vol, Zp, Yp, Xp, Z, Y, X, _ptr(out), _stream(stream)), "wo_crop")


def wo_status_string(status: int) -> str:
    return _string(status)


def wo_profile_enable(on: bool):
    _lib.wo_profile_enable(1 if on else 0)


def wo_profile_read(cap: int = 64) -> dict:
    names = (ctypes.c_char_p * cap)()
    cnt = (ctypes.c_longlong * cap)()
    ms = (ctypes.c_double * cap)()
    n = _lib.wo_profile_read(names, cnt, ms, cap)
    return {names[i].decode(): (int(cnt[i]), float(ms[i])) for i in range(min(n, cap))}


def wo_launch_count() -> int:
    return int(_lib.wo_launch_count())


# ------------------------------------------------------------- views
def tf_views(tf, n_tiles, Z, Y, X, kinds):
    """(spectra, stats) views of a TF bank tensor: complex64 [n][k][Z][Y][X/2+1], float32 [n][8].
    A kx-major bank's spectra are stored [n][k][X/2+1][Z][Y]; the view is
    permuted back to [n][k][Z][Y][X/2+1] (not contiguous)."""
    import torch
    m = kinds_mask(kinds)
    core = m & ~(WO_TF_PLANES | WO_TF_SMOOTH_SOURCE | WO_TF_KX_MAJOR)
    nk = 2 if core == WO_TF_PHASE_DZ else (5 if core == WO_TF_PHASE_GRAD else bin(core).count("1"))
    Xh = X // 2 + 1
    n_spec = n_tiles * nk * Z * Y * Xh
    raw = tf.view(torch.uint8)
    if m & WO_TF_KX_MAJOR:
        spec = raw[: n_spec * 8].view(torch.complex64).view(n_tiles, nk, Xh, Z, Y).permute(0, 1, 3, 4, 2)
    else:
        spec = raw[: n_spec * 8].view(torch.complex64).view(n_tiles, nk, Z, Y, Xh)
    off = ((n_spec * 8 + 255) // 256) * 256
    stats = raw[off: off + n_tiles * 32].view(torch.float32).view(n_tiles, 8)
    return spec, stats


def alloc(n_tiles, Z, Y, X, kinds, device="cuda"):
    """Allocate a TF bank and a workspace (torch uint8 tensors) for these shapes."""
    import torch
    tfb = wo_tf_bytes(n_tiles, Z, Y, X, kinds)
    wsb = wo_workspace_bytes(n_tiles, Z, Y, X, kinds)
    if tfb == 0 or wsb == 0:
        raise ValueError("invalid shape or kinds")
    ws = torch.empty(wsb, dtype=torch.uint8, device=device)
    ws[:256].zero_()  # the status block starts cleared
    return torch.empty(tfb, dtype=torch.uint8, device=device), ws
