"""Benchmark of the hot path: transfer-function build + Tikhonov reconstruction.

Default line (``--workload field``): the shift-variant field, 48 x 2048 x 2048,
cut into 256 overlapping tiles of 48 x 192 x 192, each with its own optics
(defocus, illumination tilt, NA_ill).  One step = gather the tiles, build
every tile's phase transfer function from its device-side optics, reconstruct
every tile (3D Tikhonov, relative eta 1e-3, channel-mean background) and blend
the tiles back into the field: 12 launches in one CUDA graph.  The value is
field voxels/s (tiles/s beside it).  Inputs are synthetic (seeded sphere
phantom forward-simulated per tile with its tile's optics, 1e-3 Gaussian
noise) and resident in HBM; the working set (field 805 MB, tiles 1.8 GB, TFs
1.8 GB) exceeds the 129 MB L2, so no flush is needed between steps.

The same line carries the metric's other parts as legs:
* "autotune": auto-tuning of (defocus, tilt_x, tilt_y, NA_ill) of the same 256
  tiles of 48 x 192 x 192, 50 Adam steps each through the library's adjoint
  in one CUDA graph, as tiles/s with the parameter errors reached;
* "widefield": the 96 x 512 x 512 widefield step (phase + absorption +
  fluorescence TF build and 3D reconstruction);
* "small_stacks": one 16 x 64 x 64 reconstruction call (latency) and a batch
  of 4096 such stacks sharing one TF bank;
* "estimator": the learned optics estimator (training on 10^5 synthetic tiles
  of 48 x 128 x 128, then a network start plus 10 refinement steps against
  50 plain tuning steps on 4096 test tiles, errors against the true optics).
``--workload tiles|widefield|autotune|estimator`` prints one of them alone.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
N > 1 runs under torchrun: every rank restores its own field (weak scaling,
no data-path collective); the reported value is the total over ranks.
"""
from __future__ import annotations

import os

os.environ.setdefault("OMP_NUM_THREADS", "1")        # the CPU oracle baseline runs single-threaded
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("MKL_NUM_THREADS", "1")

import argparse
import hashlib
import json
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "recon voxels/s & auto-tuned tiles/s at fixed error; % of HBM roofline"
SHAPE = (96, 512, 512)
KINDS = ("phase", "absorption", "fluor")
ETA = [1e-3, 1e-3]
WORKLOAD = "widefield 96x512x512: TF build (phase+absorption+fluorescence) + 3D Tikhonov reconstruction"
# CPU sample for the oracle baseline: the same optics, kinds and eta on a
# 96 x 256 x 256 sub-volume (1/4 of the voxels, a quarter of the objects).
CPU_SAMPLE = (96, 256, 256)

# Last ncu capture of DRAM traffic per launch (bytes) of a workload's dominant
# kernels, keyed by (workload, kernel family), with the digest of the kernel's
# sources at capture time (reported as null once a source changes).  Field
# entries: read + written bytes per launch on 64 tiles of 48x192x192 (an
# 8x8-tile field; the full 256-tile workload is too large for a full
# capture), scaled by 4 to the 256 tiles of a launch of the bench's field
# (the traffic grows with the tiles).
NCU_TRAFFIC = {
    ("field", "tf_arms"): {"bytes": 4 * (54528000 + 772520960), "digest": "451b42818bf0103a"},
    ("field", "tf_psf_rows"): {"bytes": 4 * (906436096 + 440025600), "digest": "cf4d832d91af6988"},
}


def kernel_digest(name: str) -> str:
    """Digest of the sources a kernel family is built from."""
    tf = ["wo_tf.cu", "wo_tf.cuh"]
    src = {"z_fused": ["wo_zops.cuh", "wo_zops_a.cu", "wo_zops_b.cu", "wo_zreg.cu", "wo_regfft.cuh"],
           "z_solve2d": ["wo_zops.cuh", "wo_zops_a.cu"], "rows_r2c": ["wo_rows.cu"], "rows_c2r": ["wo_rows.cu"],
           "xy_fwd": ["wo_xy.cu", "wo_rowsplit.cuh", "wo_regfft.cuh"], "xy_inv": ["wo_xy.cu", "wo_rowsplit.cuh", "wo_regfft.cuh"],
           "y_fwd": ["wo_cols.cu"], "y_inv": ["wo_cols.cu"], "tf_ypass": ["wo_cols.cu"], "tf_arms": tf + ["wo_armsreg.cu", "wo_regfft.cuh"],
           # the register-resident row kernel (rows of 32..512 points; wo_tf.cu holds only the
           # shared-memory fallback for other lengths)
           "tf_psf_rows": ["wo_psf.cu", "wo_regfft.cuh", "wo_tf.cuh"],
           "tf_zpass": tf + ["wo_zops.cuh"],
           "tf_pupil_record": tf, "tune_cols": ["wo_tune.cu"],
           "tf_yz": ["wo_plane.cu", "wo_bulk.cuh", "wo_regfft.cuh", "wo_zops.cuh"],
           "yz_op": ["wo_plane.cu", "wo_bulk.cuh", "wo_regfft.cuh", "wo_zops.cuh"]}.get(name)
    if src is None:
        return ""
    h = hashlib.sha256()
    for f in src + ["wo_fft.cuh"]:
        with open(os.path.join(ROOT, "paper_2412_09775_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def band_columns(o, X):
    """x columns inside the detection band |nu_x| <= NA_det/lambda (the arms are
    exactly zero elsewhere and are neither stored nor read)."""
    R = o["na_det"] / o["lambda_um"]
    k = 0
    while k + 1 <= X // 2 and ((k + 1) / (X * o["pixel_um"])) ** 2 <= R * R:
        k += 1
    return min(X, 2 * k + 1)


def support_columns(o, kinds, Y, X):
    """(k_y, k_x) columns of the half spectrum inside the TFs' support disk,
    (k_y/Y)^2 + (k_x/X)^2 <= r^2 with r = R p + 2/min(Y, X) (cycles per pixel;
    R = (NA_det + min(NA_det, NA_ill + |t|))/lambda label-free, 2 NA_det/lambda
    fluorescence): the z passes read and transform only these, the others are
    written as zeros."""
    lam = o["lambda_um"]
    tilt = float(np.hypot(o["tilt_x"], o["tilt_y"]))
    R = 0.0
    if {"phase", "absorption"} & set(kinds):
        R = o["na_det"] + min(o["na_det"], o["na_ill"] + tilt)
    if "fluor" in kinds:
        R = max(R, 2 * o["na_det"])
    r = R / lam * o["pixel_um"] + 2.0 / min(Y, X)
    ky = np.where(np.arange(Y) < (Y + 1) // 2, np.arange(Y), np.arange(Y) - Y) / Y
    kx = np.arange(X // 2 + 1) / X
    return int(np.sum(ky[:, None] ** 2 + kx[None, :] ** 2 <= r * r))


def support_planes(o, kinds, X):
    """Half-spectrum columns k_x whose (k_x, k_y = 0) lies inside the TFs'
    support disk (the planes the plane engine reads; the others are written
    as zeros without being read)."""
    lam = o["lambda_um"]
    tilt = float(np.hypot(o["tilt_x"], o["tilt_y"]))
    R = 0.0
    if {"phase", "absorption"} & set(kinds):
        R = o["na_det"] + min(o["na_det"], o["na_ill"] + tilt)
    if "fluor" in kinds:
        R = max(R, 2 * o["na_det"])
    r = R / lam * o["pixel_um"] + 2.0 / X
    kx = np.arange(X // 2 + 1) / X
    return int(np.sum(kx ** 2 <= r * r))


def support_xcols(o, kinds, X):
    """Half-spectrum columns the TF build's y and z passes transform (the
    support radius in x plus two bins, as the library computes it)."""
    import math
    tilt = float(np.hypot(o["tilt_x"], o["tilt_y"]))
    R = 0.0
    if {"phase", "absorption"} & set(kinds):
        R = o["na_det"] + min(o["na_det"], o["na_ill"] + tilt)
    if "fluor" in kinds:
        R = max(R, 2 * o["na_det"])
    return min(X // 2 + 1, math.ceil(R / o["lambda_um"] * X * o["pixel_um"]) + 3)


def algorithmic_bytes(shape, kinds, o):
    """Compulsory HBM bytes per launch of each kernel family for one step."""
    Z, Y, X = shape
    Xh = X // 2 + 1
    nk = len(kinds)
    lf = 1 if {"phase", "absorption"} & set(kinds) else 0
    C = lf + (1 if "fluor" in kinds else 0)
    P = nk
    n_arms = 2 * lf + (1 if "fluor" in kinds else 0)
    real = Z * Y * X * 4
    half = Z * Y * Xh * 8
    inside = Z * support_columns(o, kinds, Y, X) * 8  # bytes of one volume inside the support
    tf_cols = Z * Y * support_xcols(o, kinds, X) * 8  # bytes of one TF slot the build's y/z passes touch
    arms = n_arms * Z * Y * band_columns(o, X) * 8
    return {
        "tf_pupil_record": Y * X * 16,
        "tf_arms": arms,
        "tf_psf_rows": arms + nk * half,
        "tf_ypass": 2 * nk * tf_cols,
        "tf_zpass": 2 * nk * tf_cols,
        "rows_r2c": C * (real + half),
        "y_fwd": 2 * C * half,
        "xy_fwd": C * (real + half),  # the fused x-y kernels (square planes)
        "xy_inv": P * (half + real),
        "z_fused": (C + nk) * inside + P * half,
        "y_inv": 2 * P * half,
        "rows_c2r": P * (half + real),
    }


def engines_recon(Y):
    from paper_2412_09775_gb300 import binding as B
    return {1: "five passes", 2: "tile pipeline"}.get(B.wo_schedule_get(B.WO_PASS_RECON, Y), "?")


def engines_xy(n):
    from paper_2412_09775_gb300 import binding as B
    return {1: "x and y passes", 2: "fused x-y kernels"}.get(B.wo_schedule_get(B.WO_PASS_XY, n), "?")


def pin_rows_engine(args, B, n):
    """Pin the x passes' engine for n complex points (engine comparisons)."""
    if args.rows_engine != "default":
        B.wo_schedule_set(B.WO_PASS_ROWS, n, {"smem": 1, "hybrid": 2}[args.rows_engine])


def engines(*lengths, rows=None):
    from paper_2412_09775_gb300 import binding as B
    names = {1: "smem", 2: "hybrid"}
    out = {f"cols_{n}": names.get(B.wo_schedule_get(B.WO_PASS_COLS, n), "?") for n in sorted(set(lengths))}
    if rows is not None:
        out[f"rows_{rows}"] = names.get(B.wo_schedule_get(B.WO_PASS_ROWS, rows), "?")
    return out


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------------ clocks
class NvmlClockSampler:
    """Polls SM clock and clock-event reasons through NVML (read-only queries)
    from a background thread every ~2 ms while the timed region runs."""
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, torch_device):
        import ctypes
        import threading
        self.ok = False
        self.samples = []
        self._stop = threading.Event()
        try:
            nv = ctypes.CDLL("libnvidia-ml.so.1")
            if nv.nvmlInit_v2() != 0:
                return
            h = ctypes.c_void_p()
            bus = None
            try:
                import torch
                p = torch.cuda.get_device_properties(torch_device)
                bus = f"{p.pci_domain_id:08x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0".encode()
            except Exception:
                bus = None
            if bus is None or nv.nvmlDeviceGetHandleByPciBusId_v2(bus, ctypes.byref(h)) != 0:
                if nv.nvmlDeviceGetHandleByIndex_v2(0, ctypes.byref(h)) != 0:
                    return
            self.nv, self.h, self.ct = nv, h, ctypes
            mx = ctypes.c_uint()
            self.max_mhz = float(mx.value) if nv.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx)) == 0 else None
            fn = getattr(nv, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                getattr(nv, "nvmlDeviceGetCurrentClocksThrottleReasons")
            self.reason_fn = fn
            self.ok = True
            self.thread = threading.Thread(target=self._run, daemon=True)
        except OSError:
            self.ok = False

    def _run(self):
        ct = self.ct
        clk = ct.c_uint()
        rs = ct.c_ulonglong()
        while not self._stop.is_set():
            a = self.nv.nvmlDeviceGetClockInfo(self.h, 1, ct.byref(clk))
            b = self.reason_fn(self.h, ct.byref(rs))
            if a == 0:
                self.samples.append((float(clk.value), int(rs.value) if b == 0 else 0))
            self._stop.wait(0.002)

    def __enter__(self):
        if self.ok:
            self.thread.start()
        return self

    def __exit__(self, *exc):
        if self.ok:
            self._stop.set()
            self.thread.join()

    def summary(self):
        if not self.samples:
            return None
        reasons = set()
        for _, r in self.samples:
            for bit, name in self.REASONS.items():
                if r & bit:
                    reasons.add(name)
        return {"sm_mhz": statistics.median([c for c, _ in self.samples]), "sm_max_mhz": self.max_mhz,
                "reasons": sorted(reasons), "samples": len(self.samples), "source": "nvml"}


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in getattr(self, "lines", []):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for name, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ inputs
def make_inputs(shape, seed=2):
    import phantom as ph
    o = ph.optics()
    vols = ph.widefield_phantom(seed, shape, o)
    f = np.stack([vols["dn"], vols["kappa"], vols["rho"]]).astype(np.float32)
    return o, f


# ------------------------------------------------------------------ CPU oracle
def oracle_step(o, d):
    from oracle import model as OM, optics as OO
    shape = d.shape[1:]
    tfs = OO.transfer_functions(o, shape, KINDS)
    modes, _, _ = OM.widefield_system(tfs, KINDS)
    out = np.zeros((3,) + shape)
    for m, e in zip(modes, ETA):
        r = OM.reconstruct([m], d, e)
        for p in m["props"]:
            out[p] = r[p]
    return out


def oracle_sample_inputs():
    """Seeded data for the CPU sample (oracle forward of a phantom + noise)."""
    import phantom as ph
    from oracle import model as OM, optics as OO
    o = ph.optics()
    shape = CPU_SAMPLE
    vols = ph.widefield_phantom(3, shape, o, n_spheres=2000 // 4, n_shells=200 // 4)
    f = np.stack([vols["dn"], vols["kappa"], vols["rho"]])
    modes, _, _ = OM.widefield_system(OO.transfer_functions(o, shape, KINDS), KINDS)
    d = OM.forward(modes, f, [1.0, 0.1])
    for c in range(2):
        d[c] += ph.gaussian_noise(10 + c, shape, 1e-3 * abs(d[c].mean()))
    return o, d.astype(np.float32).astype(np.float64)


def cpu_baseline(steps=2):
    o, d = oracle_sample_inputs()
    t0 = time.perf_counter()
    for _ in range(steps):
        oracle_step(o, d)
    dt = (time.perf_counter() - t0) / steps
    vox = float(np.prod(CPU_SAMPLE))
    return {"value": vox / dt, "unit": "voxels/s", "cores": 1, "kind": "oracle",
            "sample": f"numpy float64 oracle, TF build + reconstruction of a {CPU_SAMPLE[0]}x{CPU_SAMPLE[1]}x"
                      f"{CPU_SAMPLE[2]} sub-volume (1/4 of the voxels, same optics/kinds/eta), "
                      f"{dt:.1f} s per step, single thread", "seconds_per_step": dt,
            "host_cpus": os.cpu_count()}


# ------------------------------------------------------------------ GPU arm
def run_gpu(args, rank, world, local_rank):
    """The widefield workload as its own line (``--workload widefield``)."""
    line = widefield_leg(args, rank, world, local_rank, with_tune=not args.no_autotune)
    if rank == 0:
        print(json.dumps(line), flush=True)


def widefield_leg(args, rank, world, local_rank, with_tune=False):
    """The widefield 96x512x512 step (TF build + reconstruction) with its
    e2e, torch.fft comparison and CPU baseline; returns the line (rank 0)."""
    import torch
    from paper_2412_09775_gb300.build import build
    build()
    from paper_2412_09775_gb300 import binding as B
    import phantom as ph

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    Z, Y, X = SHAPE
    o, f = make_inputs(SHAPE, seed=2 + rank)
    tf, ws = B.alloc(1, Z, Y, X, KINDS, dev)
    if not args.default_engines:
        B.wo_autotune(1, Z, Y, X, KINDS, ws)  # engine per column-transform length, timed on these shapes
    pin_rows_engine(args, B, X // 2)
    # synthetic data: forward model of the phantom (on the GPU) + seeded noise
    f_d = torch.from_numpy(f).to(dev)
    data = torch.empty((1, 2, Z, Y, X), dtype=torch.float32, device=dev)
    B.wo_build_tf([o], 1, Z, Y, X, KINDS, tf, ws)
    B.wo_forward(tf, KINDS, f_d, [1.0, 0.1], data, 1, Z, Y, X, ws)
    torch.cuda.synchronize()
    mean = data.mean(dim=(2, 3, 4)).cpu().numpy()[0]
    for c in range(2):
        noise = ph.gaussian_noise(100 + 10 * rank + c, SHAPE, 1e-3 * abs(float(mean[c]))).astype(np.float32)
        data[0, c] += torch.from_numpy(noise).to(dev)
    del f_d
    out = torch.empty((1, 3, Z, Y, X), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        B.wo_build_tf([o], 1, Z, Y, X, KINDS, tf, ws)
        B.wo_reconstruct(tf, KINDS, data, None, ETA, B.WO_ETA_RELATIVE, B.WO_MODE_3D, out, 1, Z, Y, X, ws)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    # the timed steps run with the library's profiler off; per-kernel times
    # come from a separate profiled pass over the same number of steps
    n0 = B.wo_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nvml = NvmlClockSampler(dev)
    with ClockSampler(local_rank) as smi, nvml:
        ev0.record(stream)
        for _ in range(args.steps):
            step()
        ev1.record(stream)
        torch.cuda.synchronize()
    clk = nvml.summary() or smi.summary()
    launches = B.wo_launch_count() - n0
    barrier()
    from paper_2412_09775_gb300.shard import max_over_ranks
    ms_max = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, device=dev)
    prof = profiled_pass(B, step, args.steps)

    # end to end through the public API: host (pinned) in, host out
    if args.no_e2e:
        e2e_ms = (float("nan"), float("nan"))
    else:
        e2e_ms = run_e2e(args, B, o, data, out, tf, ws, stream, barrier, world, dev)
    lib = None if args.no_library_fft else library_leg(args, B, tf, ws, data, out, stream, dev)
    del tf, ws, data, out
    torch.cuda.empty_cache()
    tune = autotune_leg(args, rank, world, local_rank) if with_tune else None
    if rank != 0:
        return None
    return report(args, world, ms_max, e2e_ms, prof, launches, clk, tune, lib)


def profiled_pass(B, step, n):
    """Per-kernel launches and milliseconds over n eager steps with the
    library's event profiler on (a pass of its own, outside the timed one)."""
    import torch
    torch.cuda.synchronize()
    B.wo_profile_read()  # drop anything recorded so far
    B.wo_profile_enable(True)
    for _ in range(n):
        step()
    torch.cuda.synchronize()
    B.wo_profile_enable(False)
    return B.wo_profile_read()


def run_e2e(args, B, o, data, out, tf, ws, stream, barrier, world, dev):
    """Steps through the public API from pinned host buffers: each step copies
    its two input stacks to the device, builds the TFs, reconstructs and
    copies the three property volumes back.  Measured twice: serially on one
    stream, and with consecutive steps going round `args.e2e_streams` streams
    (each with its own device buffers), so one step's copies overlap the
    others' kernels, as a serving loop would run them.  Returns (pipelined, serial)
    ms per step."""
    import torch
    Z, Y, X = SHAPE
    h_in = torch.empty((1, 2, Z, Y, X), dtype=torch.float32, pin_memory=True)
    h_in.copy_(data.cpu())
    lanes = [dict(s=stream, d_in=torch.empty_like(data), out=out, tf=tf, ws=ws)]
    for _ in range(1, args.e2e_streams):
        tf_l, ws_l = B.alloc(1, Z, Y, X, KINDS, dev)
        lanes.append(dict(s=torch.cuda.Stream(device=dev), d_in=torch.empty_like(data), out=torch.empty_like(out),
                          tf=tf_l, ws=ws_l))
    for ln in lanes:
        ln["h_out"] = torch.empty((1, 3, Z, Y, X), dtype=torch.float32, pin_memory=True)

    def e2e_step(ln):
        with torch.cuda.stream(ln["s"]):
            ln["d_in"].copy_(h_in, non_blocking=True)
            B.wo_build_tf([o], 1, Z, Y, X, KINDS, ln["tf"], ln["ws"], stream=ln["s"])
            B.wo_reconstruct(ln["tf"], KINDS, ln["d_in"], None, ETA, B.WO_ETA_RELATIVE, B.WO_MODE_3D, ln["out"],
                             1, Z, Y, X, ln["ws"], stream=ln["s"])
            ln["h_out"].copy_(ln["out"], non_blocking=True)

    def timed(n_lanes):
        for i in range(max(1, args.warmup)):
            e2e_step(lanes[i % n_lanes])
        torch.cuda.synchronize()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for ln in lanes[1:n_lanes]:
            ln["s"].wait_stream(stream)  # the timed region starts before any lane's first copy
        for i in range(args.steps):
            e2e_step(lanes[i % n_lanes])
        for ln in lanes[1:n_lanes]:
            stream.wait_stream(ln["s"])
        e1.record(stream)
        torch.cuda.synchronize()
        from paper_2412_09775_gb300.shard import max_over_ranks
        return max_over_ranks(e0.elapsed_time(e1) / args.steps, device=dev)

    serial = timed(1)
    return timed(len(lanes)), serial


def torch_fft_forward(H, f, bg):
    """The widefield forward model written with torch.fft and torch elementwise
    ops: H the (phase, absorption, fluorescence) half-spectrum TFs (3, Z, Y, Xh),
    f the three property volumes (3, Z, Y, X); returns the brightfield and
    fluorescence stacks (2, Z, Y, X) with backgrounds bg added."""
    import torch
    dims = (-3, -2, -1)
    F = torch.fft.rfftn(f, dim=dims)
    D = torch.stack((H[0] * F[0] + H[1] * F[1], H[2] * F[2]))
    d = torch.fft.irfftn(D, s=tuple(f.shape[-3:]), dim=dims)
    d[0] += bg[0]
    d[1] += bg[1]
    return d


def torch_fft_eta(H, eta):
    """Absolute eta per contrast mode (relative eta times the mode's largest
    sum of |H|^2), as device scalars: formed once per TF bank, as the library
    forms its regulariser maxima in the TF build."""
    return (float(eta[0]) * ((H[0].abs() ** 2) + (H[1].abs() ** 2)).max(), float(eta[1]) * (H[2].abs() ** 2).max())


def torch_fft_reconstruct(H, d, w):
    """The widefield 3D Tikhonov reconstruction written the same way: channel
    means as backgrounds, absolute eta w = (label-free, fluorescence) from
    torch_fft_eta, the label-free 1 x 2 block by its push-through form and the
    fluorescence 1 x 1 block."""
    import torch
    dims = (-3, -2, -1)
    w_re, w_fl = w
    D = torch.fft.rfftn(d - d.mean(dim=dims, keepdim=True), dim=dims)
    g = D[0] / ((H[0].abs() ** 2) + (H[1].abs() ** 2) + w_re)
    F = torch.stack((H[0].conj() * g, H[1].conj() * g, H[2].conj() * D[1] / ((H[2].abs() ** 2) + w_fl)))
    return torch.fft.irfftn(F, s=tuple(d.shape[-3:]), dim=dims)


def library_leg(args, B, tf, ws, data, out, stream, dev):
    """The same forward model and reconstruction written with torch.fft (cuFFT)
    and torch elementwise ops on the same TF bank and shapes - the style of a
    PyTorch implementation of the method - timed beside the library's calls.
    Timed only, for context: nothing here is on the library's path.  Returns
    ms per call for both and the relative L2 difference of their outputs."""
    import torch
    Z, Y, X = SHAPE
    Xh = X // 2 + 1
    spectra = tf[: 3 * Z * Y * Xh * 8]  # the bank's spectra; its per-tile statistics block follows them
    H = torch.view_as_complex(spectra.view(torch.float32).view(3, Z, Y, Xh, 2))  # phase, absorption, fluorescence
    bg = [1.0, 0.1]
    f_vol = torch.empty((1, 3, Z, Y, X), dtype=torch.float32, device=dev)
    f_vol.copy_(out)
    d_lib = torch.empty((1, 2, Z, Y, X), dtype=torch.float32, device=dev)

    def torch_forward():
        return torch_fft_forward(H, f_vol[0], bg)

    w_abs = torch_fft_eta(H, ETA)

    def torch_reconstruct():
        return torch_fft_reconstruct(H, data[0], w_abs)

    def lib_forward():
        B.wo_forward(tf, KINDS, f_vol, bg, d_lib, 1, Z, Y, X, ws)

    def lib_reconstruct():
        B.wo_reconstruct(tf, KINDS, data, None, ETA, B.WO_ETA_RELATIVE, B.WO_MODE_3D, out, 1, Z, Y, X, ws)

    def timed(fn):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / args.steps

    def rel(a, b):
        return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))

    t_fwd, l_fwd = timed(torch_forward), timed(lib_forward)
    diff_fwd = rel(torch_forward(), d_lib[0])
    t_rec, l_rec = timed(torch_reconstruct), timed(lib_reconstruct)
    diff_rec = rel(torch_reconstruct(), out[0])
    return {"forward": {"torch_fft_ms": round(t_fwd, 4), "library_ms": round(l_fwd, 4),
                        "speedup": round(t_fwd / l_fwd, 2), "rel_l2_diff": float(f"{diff_fwd:.3g}")},
            "reconstruct": {"torch_fft_ms": round(t_rec, 4), "library_ms": round(l_rec, 4),
                            "speedup": round(t_rec / l_rec, 2), "rel_l2_diff": float(f"{diff_rec:.3g}")},
            "note": "torch.fft (cuFFT) + torch elementwise ops on the same TF bank, 96x512x512, three "
                    "properties / two stacks, CUDA events; timed only, not on the library's path"}


def report(args, world, ms_max, e2e_ms, prof, launches, clk, tune=None, lib=None):
    Z, Y, X = SHAPE
    from paper_2412_09775_gb300.shard import job_throughput
    vox = float(Z * Y * X)
    value = job_throughput(vox, world, ms_max)
    import phantom as ph
    algo = algorithmic_bytes(SHAPE, KINDS, ph.optics())
    per_kernel = {}
    for name, (cnt, tot) in prof.items():
        avg = tot / cnt if cnt else 0.0
        b = algo.get(name)
        per_kernel[name] = {"launches": cnt, "avg_ms": round(avg, 4),
                            "share": round(tot / max(1e-9, sum(v[1] for v in prof.values())), 4),
                            "algo_bytes": b,
                            "gbs": round(b / (avg * 1e-3) / 1e9, 1) if b and avg > 0 else None}
    dom = max(prof.items(), key=lambda kv: kv[1][1])[0]
    peak, peak_kind = peaks()
    dk = per_kernel[dom]
    traffic = None
    rec = NCU_TRAFFIC.get(("widefield", dom))
    if rec and rec.get("digest") == kernel_digest(dom):
        traffic = rec["bytes"]
    roofline = {"bound": "hbm", "kernel": dom, "achieved": dk["gbs"], "peak": peak, "unit": "GB/s",
                "frac": round(dk["gbs"] / peak, 4) if dk["gbs"] else None, "traffic": traffic,
                "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                else "fallback 6.8 TB/s"}
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "voxels/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (seeded phantom: 2000 spheres + 200 shells, GPU forward model + 1e-3 noise)",
        "config": {"workload": WORKLOAD if SHAPE == (96, 512, 512) else f"profiling case {Z}x{Y}x{X}", "Z": Z, "Y": Y, "X": X, "kinds": list(KINDS), "eta_relative": ETA,
                   "background": "channel mean", "tiles": 1, "parallelism": f"replicas x{world}",
                   "l2": "working set > L2 (no flush needed): data 201 MB, TF 303 MB, workspace 606 MB",
                   "schedule": engines(Y, Z, rows=X // 2)},
        "roofline": roofline,
        "kernels": per_kernel,
        "gpu_launches": int(launches),
        "clocks": clk,
        "e2e": None if e2e_ms[0] != e2e_ms[0] else {
                "value": round(job_throughput(vox, world, e2e_ms[0]), 1), "unit": "voxels/s",
                "ms_per_step": round(e2e_ms[0], 4),
                "h2d_bytes_per_step": int(2 * vox * 4 + 72), "d2h_bytes_per_step": int(3 * vox * 4),
                "streams": args.e2e_streams, "serial_ms_per_step": round(e2e_ms[1], 4),
                "serial_value": round(job_throughput(vox, world, e2e_ms[1]), 1),
                "note": "pinned host stacks in, pinned host volumes out, every step; consecutive steps "
                        "go round the streams, each with its own device buffers (copies of one step "
                        "overlap the others' kernels); serial_*: the same steps on one stream"},
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if lib is not None:
        line["library_fft"] = lib  # cuFFT-based composition of the same calls, timed beside them
    if tune is not None:
        line["autotune"] = tune  # the metric's second half: auto-tuned tiles/s at fixed error
    return line


# ------------------------------------------------------------------ tiles
TILE_GRID = (16, 16)
TILE_CORE, TILE_HALO = 128, 32
FIELD_Z = 48
TILES_WORKLOAD = ("shift-variant field 48x2048x2048: 16x16 tiles of 48x192x192 (128-px cores, 32-px halos), "
                  "per-tile optics; TF build (phase) + 3D Tikhonov of the tiles read in place from the field "
                  "+ blend, one CUDA graph")


def make_field(o_list, dev, seed=4):
    """Synthetic shift-variant field: a sphere phantom whose 16x16 regions are
    each forward-simulated (on the GPU) with their tile's optics, then blended."""
    import torch
    import phantom as ph
    from paper_2412_09775_gb300 import binding as B
    ty, tx = TILE_GRID
    Z, E = FIELD_Z, TILE_CORE + 2 * TILE_HALO
    n = ty * tx
    obj = ph.sphere_phantom(seed, (Z, ty * TILE_CORE, tx * TILE_CORE), ph.optics(), n_spheres=16000 * n // 256)
    obj_d = torch.from_numpy(obj.astype(np.float32)).to(dev)
    t_obj = torch.empty((n, Z, E, E), dtype=torch.float32, device=dev)
    B.wo_tile_gather(obj_d, Z, ty, tx, TILE_CORE, TILE_HALO, t_obj)
    tf, ws = B.alloc(n, Z, E, E, ("phase",), dev)
    B.wo_build_tf(o_list, n, Z, E, E, ("phase",), tf, ws)
    t_dat = torch.empty_like(t_obj)
    B.wo_forward(tf, ("phase",), t_obj, [1.0], t_dat, n, Z, E, E, ws)
    field = torch.empty_like(obj_d)
    B.wo_tile_blend(t_dat, Z, ty, tx, TILE_CORE, TILE_HALO, field)
    torch.cuda.synchronize()
    noise = ph.gaussian_noise(seed + 1, field.shape, 1e-3).astype(np.float32)
    field += torch.from_numpy(noise).to(dev)
    del tf, ws, t_obj, t_dat, obj_d
    torch.cuda.empty_cache()
    return field


def field_algorithmic_bytes(o_list, Z, E, field_vox):
    """Compulsory HBM bytes per launch of each kernel family of one field step:
    the phase TF build from device optics (every half-spectrum column), the
    3D reconstruction, whose first pass reads the tiles from the field (4 B
    per tile voxel), and the blend; summed over the tiles, each with its own
    detection band and TF support.  (tile_gather: the separate gather launch,
    for runs that use it.)"""
    Xh = E // 2 + 1
    real, half = Z * E * E * 4, Z * E * Xh * 8
    out = {k: 0 for k in ("tf_pupil_record", "tf_arms", "tf_psf_rows", "tf_ypass", "tf_zpass", "tf_yz", "rows_r2c",
                          "y_fwd", "xy_fwd", "z_fused", "yz_op", "y_inv", "rows_c2r", "xy_inv")}
    for o in o_list:
        arms = 2 * Z * E * band_columns(o, E) * 8
        inside = Z * support_columns(o, ("phase",), E, E) * 8
        planes_in = support_planes(o, ("phase",), E)
        out["tf_pupil_record"] += E * E * 16
        out["tf_arms"] += arms
        out["tf_psf_rows"] += arms + half
        out["tf_ypass"] += 2 * half
        out["tf_zpass"] += 2 * half
        out["tf_yz"] += 2 * planes_in * Z * E * 8  # the plane engine: the TF planes inside the support in and out
        # the plane engine's operator pass: the data planes inside the support
        # disk in, the TF columns inside it in, every plane out
        out["yz_op"] += planes_in * Z * E * 8 + inside + half
        out["rows_r2c"] += real + half
        out["y_fwd"] += 2 * half
        out["xy_fwd"] += real + half
        out["z_fused"] += 2 * inside + half
        out["y_inv"] += 2 * half
        out["rows_c2r"] += half + real
        out["xy_inv"] += half + real
    tiles = len(o_list) * Z * E * E * 4
    # the tile pipeline: every tile's data in, its phase TF in, its result out
    # (the spectra between its items stay in L2)
    out["tile_pipeline"] = len(o_list) * (2 * real + half)
    out["tile_gather"] = 4 * field_vox + tiles
    out["tile_blend"] = tiles + 4 * field_vox
    return out


def kernel_table(prof, algo, per):
    """Per kernel family: launches, average ms, share of the profiled time,
    algorithmic bytes per launch and the GB/s they give."""
    tot = sum(v[1] for v in prof.values()) or 1e-9
    out = {}
    for name, (cnt, t) in prof.items():
        avg = t / cnt if cnt else 0.0
        b = algo.get(name)
        out[name] = {per: cnt, "avg_ms": round(avg, 4), "share": round(t / tot, 4), "algo_bytes": b,
                     "gbs": round(b / (avg * 1e-3) / 1e9, 1) if b and avg > 0 else None}
    return out


def roofline_of(kern, prof, workload=None):
    """The roofline entry of the kernel family with the largest share."""
    dom = max(prof.items(), key=lambda kv: kv[1][1])[0]
    peak, peak_kind = peaks()
    gbs = kern[dom]["gbs"]
    traffic = None
    rec = NCU_TRAFFIC.get((workload, dom))
    if rec and rec.get("digest") == kernel_digest(dom):
        traffic = rec["bytes"]
    return {"bound": "hbm", "kernel": dom, "achieved": gbs, "peak": peak, "unit": "GB/s",
            "frac": round(gbs / peak, 4) if gbs else None, "traffic": traffic,
            "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
            else "fallback 6.8 TB/s"}


def run_tiles(args, rank, world, local_rank):
    """The shift-variant field as the headline line, with the auto-tuning,
    widefield, small-stack and learned-estimator legs unless --field-only."""
    import torch
    line = field_leg(args, rank, world, local_rank)
    if not args.field_only:
        tune = None if args.no_autotune else autotune_leg(args, rank, world, local_rank)
        wide = widefield_leg(args, rank, world, local_rank)
        small = small_stack_leg(args, rank, world, local_rank)
        est = None if args.no_estimator else estimator_leg(args, rank, world, local_rank)
        if rank == 0:
            if tune is not None:
                line["autotune"] = tune  # the metric's second half: auto-tuned tiles/s at fixed error
            line["widefield"] = wide
            line["small_stacks"] = small
            if est is not None:  # learned start + 10 refinement steps against 50 plain steps
                line["estimator"] = {k: est[k] for k in ("value", "unit", "ms_per_step", "config", "learned",
                                                         "plain", "speedup_vs_plain",
                                                         "learned_with_training_s_per_tile", "break_even_tiles",
                                                         "training")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    torch.cuda.synchronize()


def field_leg(args, rank, world, local_rank):
    import torch
    import phantom as ph
    from paper_2412_09775_gb300.build import build
    from paper_2412_09775_gb300.shard import job_throughput, max_over_ranks
    build()
    from paper_2412_09775_gb300 import binding as B
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    ty, tx = TILE_GRID
    n = ty * tx
    Z, E = FIELD_Z, TILE_CORE + 2 * TILE_HALO
    o_list = ph.tile_optics(np.random.default_rng(3 + rank), n)
    field = make_field(o_list, dev, seed=4 + rank)
    optics = B.optics_tensor(o_list, dev)
    tiles = None  # the step reads the tiles from the field in place
    rec = torch.empty((n, Z, E, E), dtype=torch.float32, device=dev)
    out = torch.empty_like(field)
    tf, ws = B.alloc(n, Z, E, E, ("phase",), dev)
    if not args.default_engines:
        B.wo_autotune(n, Z, E, E, ("phase",), ws)
    pin_rows_engine(args, B, E // 2)
    # planes: a kx-major phase bank (WO_TF_KX_MAJOR), whose build and
    # reconstruction run their y and z transforms (and the operator between
    # them) one (tile, k_x) plane per CTA; passes: the standard bank and the
    # separate y pass, z pass and inverse y pass
    field_kinds = {"planes": B.WO_TF_PHASE | B.WO_TF_KX_MAJOR, "passes": B.WO_TF_PHASE}

    def make_step_on(kinds):
        def step_on(fld, dst, tl, rc, tfb, wsb, opt):
            # the reconstruction's first pass reads each tile's rows from the field
            # (wo_reconstruct_field_tiles: the same tiles wo_tile_gather would copy);
            # the separate blend is faster than wo_restore_field's fused last pass
            B.wo_build_tf_device(opt, n, Z, E, E, kinds, tfb, wsb)
            B.wo_reconstruct_field_tiles(tfb, kinds, fld, Z, ty, tx, TILE_CORE, TILE_HALO, None, [1e-3],
                                         B.WO_ETA_RELATIVE, B.WO_MODE_3D, rc, wsb)
            B.wo_tile_blend(rc, Z, ty, tx, TILE_CORE, TILE_HALO, dst)
        return step_on

    step_on = make_step_on(field_kinds[args.field_engine])
    other_engine = "passes" if args.field_engine == "planes" else "planes"
    other_step_on = make_step_on(field_kinds[other_engine])

    def step():
        step_on(field, out, tiles, rec, tf, ws, optics)

    s = torch.cuda.Stream(device=dev)
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        for _ in range(max(1, args.warmup)):
            step()
    torch.cuda.synchronize()
    n0 = B.wo_launch_count()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        step()
    per_step_launches = B.wo_launch_count() - n0
    for _ in range(args.warmup):
        g.replay()
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nvml = NvmlClockSampler(dev)
    with ClockSampler(local_rank) as smi, nvml:
        ev0.record()
        for _ in range(args.steps):
            g.replay()
        ev1.record()
        torch.cuda.synchronize()
    clk = nvml.summary() or smi.summary()
    ms_max = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, device=dev)
    # per-kernel times from eager profiled steps (the events do not enter a graph)
    with torch.cuda.stream(s):
        prof = profiled_pass(B, step, args.steps)
    def alt_step_ms(pass_, engine, step_fn=step):
        """The step timed the same way with one schedule entry pinned (context
        for the engine choices); the entry is restored afterwards."""
        saved = B.wo_schedule_get(pass_, E)
        B.wo_schedule_set(pass_, E, engine)
        g5 = torch.cuda.CUDAGraph()
        with torch.cuda.stream(s):
            step_fn()
        torch.cuda.synchronize()
        with torch.cuda.graph(g5, stream=s):
            step_fn()
        B.wo_schedule_set(pass_, E, saved)
        for _ in range(args.warmup):
            g5.replay()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            g5.replay()
        e1.record()
        torch.cuda.synchronize()
        del g5
        return e0.elapsed_time(e1) / args.steps

    # the reconstruction on the persistent tile pipeline instead of the five
    # passes, and the x-y transforms as separate passes instead of fused
    # (the other field engine; with the passes, also the persistent tile
    # pipeline instead of the five passes and the other x-y engine)
    def other_step():
        other_step_on(field, out, tiles, rec, tf, ws, optics)

    passes_step = step if args.field_engine == "passes" else other_step
    other_ms = alt_step_ms(B.WO_PASS_RECON, B.wo_schedule_get(B.WO_PASS_RECON, E), other_step)
    pipe_ms = alt_step_ms(B.WO_PASS_RECON, B.WO_ENGINE_HYBRID, passes_step)
    other_xy = B.WO_ENGINE_SMEM if B.wo_schedule_get(B.WO_PASS_XY, E) == B.WO_ENGINE_HYBRID else B.WO_ENGINE_HYBRID
    xy_ms = alt_step_ms(B.WO_PASS_XY, other_xy, passes_step)
    code = B.wo_sync_status(ws)
    vox = float(field.numel())
    kern = kernel_table(prof, field_algorithmic_bytes(o_list, Z, E, vox), "launches")
    e2e = None if args.no_e2e else field_e2e(args, B, step_on, field, o_list, n, Z, E, world, dev)
    if rank != 0:
        return None
    line = {
        "metric": METRIC, "value": round(job_throughput(vox, world, ms_max), 1), "unit": "voxels/s",
        "tiles_per_s": round(job_throughput(n, world, ms_max), 1), "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32",
        "data": "synthetic (sphere phantom forward-simulated per tile with its own optics + 1e-3 noise)",
        "config": {"workload": TILES_WORKLOAD if (ty, tx) == (16, 16) else f"profiling case: {ty}x{tx} tiles",
                   "field": [Z, ty * TILE_CORE, tx * TILE_CORE], "tiles": n,
                   "tile": [Z, E, E], "eta_relative": 1e-3, "parallelism": f"replicas x{world}",
                   "l2": "working set > L2, no flush needed (field 805 MB, tiles 1.8 GB, TF 1.8 GB)",
                   "schedule": engines(E, Z, rows=E // 2)},
        "roofline": roofline_of(kern, prof, "field" if (ty, tx) == (16, 16) else None), "kernels": kern,
        "gpu_launches": int(per_step_launches * args.steps), "clocks": clk,
        "e2e": e2e,
        "recon_engine": {"field_engine": args.field_engine,
                         f"step_ms_with_{other_engine}": round(other_ms, 4),
                         "passes": {"engine": engines_recon(E), "step_ms_with_tile_pipeline": round(pipe_ms, 4),
                                    "xy": engines_xy(E), "step_ms_with_other_xy_engine": round(xy_ms, 4)},
                         "device_status": list(code)},
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = field_cpu_baseline(field, o_list)
    del tiles, rec, tf, ws, field, out
    torch.cuda.empty_cache()
    return line


def field_e2e(args, B, step_on, field, o_list, n, Z, E, world, dev):
    """The field step through the public API from pinned host memory: the
    48x2048x2048 field copied in, TF build + reconstruction of the tiles read
    in place from the field + blend,
    the restored field copied out, every step.  Consecutive steps go round
    ``args.e2e_streams`` streams, each with its own device buffers, so one
    step's copies overlap the others' kernels; also timed serially."""
    import torch
    from paper_2412_09775_gb300.shard import job_throughput, max_over_ranks
    stream = torch.cuda.current_stream()
    h_in = torch.empty(field.shape, dtype=torch.float32, pin_memory=True)
    h_in.copy_(field.cpu())
    lanes = []
    for i in range(max(1, args.e2e_streams)):
        tfb, wsb = B.alloc(n, Z, E, E, ("phase",), dev)
        lanes.append(dict(s=torch.cuda.Stream(device=dev), d_in=torch.empty_like(field), d_out=torch.empty_like(field),
                          tl=None, rc=torch.empty((n, Z, E, E), dtype=torch.float32, device=dev), tf=tfb,
                          ws=wsb,
                          opt=B.optics_tensor(o_list, dev),
                          h_out=torch.empty(field.shape, dtype=torch.float32, pin_memory=True)))

    def e2e_step(ln):
        with torch.cuda.stream(ln["s"]):
            ln["d_in"].copy_(h_in, non_blocking=True)
            step_on(ln["d_in"], ln["d_out"], ln["tl"], ln["rc"], ln["tf"], ln["ws"], ln["opt"])
            ln["h_out"].copy_(ln["d_out"], non_blocking=True)

    def timed(n_lanes):
        for i in range(max(1, args.warmup)):
            e2e_step(lanes[i % n_lanes])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for ln in lanes[:n_lanes]:
            ln["s"].wait_stream(stream)  # the timed region starts before any lane's first copy
        for i in range(args.steps):
            e2e_step(lanes[i % n_lanes])
        for ln in lanes[:n_lanes]:
            stream.wait_stream(ln["s"])
        e1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(e0.elapsed_time(e1) / args.steps, device=dev)

    serial = timed(1)
    piped = timed(len(lanes))
    vox = float(field.numel())
    ok = bool(torch.equal(lanes[0]["h_out"], lanes[-1]["h_out"]))
    del lanes
    torch.cuda.empty_cache()
    best = min(serial, piped)
    return {"value": round(job_throughput(vox, world, best), 1), "unit": "voxels/s", "ms_per_step": round(best, 4),
            "h2d_bytes_per_step": int(vox * 4), "d2h_bytes_per_step": int(vox * 4),
            "mode": "serial" if serial <= piped else f"{args.e2e_streams} streams",
            "serial_ms_per_step": round(serial, 4), "streams_ms_per_step": round(piped, 4),
            "lanes_agree": ok,
            "note": "pinned host field in, pinned host field out, every step, through the binding's calls "
                    "(gather, TF build from device optics, reconstruction, blend); timed serially on one stream "
                    "and with consecutive steps going round the streams, each with its own device buffers; the "
                    "value is the faster of the two"}


def _oracle_tile(job):
    """Worker of the CPU baseline: the float64 oracle's phase TF build and 3D
    Tikhonov reconstruction of one tile (relative eta 1e-3, channel mean)."""
    from oracle import model as OM, optics as OO
    o, d = job
    tfs = OO.transfer_functions(o, d.shape, ("phase",))
    modes, _, _ = OM.widefield_system(tfs, ("phase",))
    return OM.reconstruct(modes, d[None].astype(np.float64), 1e-3)[0].astype(np.float32)


def _pool_map(jobs, workers):
    """The oracle over `jobs` in a pool of `workers` processes (spawned, so no
    worker inherits the CUDA context); returns the results and the seconds."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        pool.map(_oracle_tile, jobs[:workers], chunksize=1)  # start-up and imports outside the clock
        t0 = time.perf_counter()
        res = pool.map(_oracle_tile, jobs, chunksize=1)
        dt = time.perf_counter() - t0
    return res, dt


def field_cpu_baseline(field, o_list):
    """The float64 oracle on the host cores for the field workload: gather,
    per-tile TF build + reconstruction, blend.  One core over 8 tiles, and a
    pool of one worker per host core over the tiles (all 256 with 16 or more
    cores, else 16 per core), both scaled to the whole field."""
    from oracle import tiles as OTl
    ty, tx = TILE_GRID
    n = ty * tx
    fld = field.cpu().numpy()
    t0 = time.perf_counter()
    tl = OTl.gather(fld, ty, tx, TILE_CORE, TILE_HALO)
    t_gather = time.perf_counter() - t0
    jobs = [(o_list[t], tl[t]) for t in range(n)]
    t0 = time.perf_counter()
    for j in jobs[:8]:
        _oracle_tile(j)
    t_one = (time.perf_counter() - t0) / 8
    cores = os.cpu_count() or 1
    m = n if cores >= 16 else min(n, 16 * cores)
    res, t_pool = _pool_map(jobs[:m], cores)
    out_tiles = tl.copy()
    for t in range(m):
        out_tiles[t] = res[t]
    t0 = time.perf_counter()
    OTl.blend(out_tiles, ty, tx, TILE_CORE, TILE_HALO)
    t_blend = time.perf_counter() - t0
    vox = float(fld.size)
    pool_s = t_gather + t_pool * n / m + t_blend
    one_s = t_gather + t_one * n + t_blend
    return {"value": round(vox / pool_s, 1), "unit": "voxels/s", "cores": cores, "kind": "oracle",
            "sample": f"numpy float64 oracle on the field workload: gather and blend of the whole "
                      f"48x2048x2048 field in the main process ({t_gather:.1f} s, {t_blend:.1f} s), TF build + "
                      f"3D Tikhonov of {m} of the 256 tiles in a pool of {cores} processes ({t_pool:.1f} s), "
                      f"scaled to 256 tiles: {pool_s:.1f} s per field",
            "single_core": {"value": round(vox / one_s, 1), "unit": "voxels/s", "cores": 1,
                            "s_per_tile": round(t_one, 3),
                            "sample": "the same oracle on one core over 8 tiles, scaled to 256 tiles plus gather "
                                      f"and blend: {one_s:.1f} s per field"}}


# ------------------------------------------------------------------ small stacks
SMALL_SHAPE = (16, 64, 64)
SMALL_BATCH = 4096
SMALL_WORKLOAD = ("small stacks 16x64x64 (20 spheres, phase-only, relative eta 1e-3): one wo_reconstruct call "
                  "(single-call latency, TF prebuilt) and a batch of 4096 stacks sharing one TF bank "
                  "(wo_reconstruct_shared_tf)")


def small_cpu_baseline(o, d):
    """The oracle on one host core: the phase TF of a 16x64x64 stack and its
    3D reconstruction (relative eta 1e-3), as for the GPU's single call, and
    the reconstruction alone with the TF built once (as the GPU batch shares
    one bank), each timed over 1 s or more."""
    from oracle import model as OM, optics as OO
    Z, Y, X = SMALL_SHAPE
    d64 = d.astype(np.float64)

    def per_call(fn):
        n, t0 = 0, time.perf_counter()
        while True:
            fn()
            n += 1
            dt = time.perf_counter() - t0
            if dt >= 1.0:
                return dt / n

    def build_and_solve():
        modes, _, _ = OM.widefield_system(OO.transfer_functions(o, SMALL_SHAPE, ("phase",)), ("phase",))
        OM.reconstruct(modes, d64, 1e-3, relative=True)
    t_call = per_call(build_and_solve)
    modes, _, _ = OM.widefield_system(OO.transfer_functions(o, SMALL_SHAPE, ("phase",)), ("phase",))
    t_solve = per_call(lambda: OM.reconstruct(modes, d64, 1e-3, relative=True))
    vox = Z * Y * X
    return {"value": round(vox / t_solve, 1), "unit": "voxels/s", "cores": 1, "kind": "oracle",
            "sample": f"numpy float64 oracle on one core: reconstruction of one 16x64x64 stack with a prebuilt TF "
                      f"({1e3 * t_solve:.1f} ms per stack, the batch's per-stack work); with the TF build "
                      f"{1e3 * t_call:.1f} ms per call ({vox / t_call:.0f} voxels/s)"}


def small_stack_leg(args, rank, world, local_rank):
    """Config of the 16x64x64 stack: the latency of one reconstruction call
    (its 0.8 MB sit in L2) and the throughput of 4096 stacks sharing one TF
    bank (compulsory 8 B per voxel: data in, volume out; the 0.27 MB bank
    stays in L2)."""
    import torch
    import phantom as ph
    from paper_2412_09775_gb300 import binding as B
    from paper_2412_09775_gb300.shard import job_throughput, max_over_ranks
    dev = torch.device("cuda", local_rank)
    Z, Y, X = SMALL_SHAPE
    o = ph.optics()
    dn = ph.sphere_phantom(1 + rank, SMALL_SHAPE, o, n_spheres=20)
    tf1, ws1 = B.alloc(1, Z, Y, X, ("phase",), dev)
    B.wo_build_tf([o], 1, Z, Y, X, ("phase",), tf1, ws1)
    f = torch.from_numpy(dn.astype(np.float32)).to(dev).view(1, 1, Z, Y, X)
    d1 = torch.empty_like(f)
    B.wo_forward(tf1, ("phase",), f, [1.0], d1, 1, Z, Y, X, ws1)
    g = torch.Generator(device=dev)
    g.manual_seed(11 + rank)
    d1 += 1e-3 * torch.randn(d1.shape, generator=g, device=dev)
    o1 = torch.empty_like(d1)
    stream = torch.cuda.current_stream()
    # the plane engine: the same TF in a kx-major bank (the standard bank's
    # calls are timed beside it as context)
    kx = B.WO_TF_PHASE | B.WO_TF_KX_MAJOR
    tf1k, ws1k = B.alloc(1, Z, Y, X, kx, dev)
    B.wo_build_tf([o], 1, Z, Y, X, kx, tf1k, ws1k)

    def one():
        B.wo_reconstruct(tf1k, kx, d1, None, [1e-3], B.WO_ETA_RELATIVE, B.WO_MODE_3D, o1, 1, Z, Y, X, ws1k)

    def one_std():
        B.wo_reconstruct(tf1, ("phase",), d1, None, [1e-3], B.WO_ETA_RELATIVE, B.WO_MODE_3D, o1, 1, Z, Y, X, ws1)

    def timed(fn, k):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return max_over_ranks(e0.elapsed_time(e1) / k, device=dev)

    lat = timed(one, max(50, args.steps))
    lat_std = timed(one_std, max(50, args.steps))
    nb = SMALL_BATCH
    data = d1.expand(nb, 1, Z, Y, X).contiguous()
    data += 1e-3 * torch.randn(data.shape, generator=g, device=dev)  # every stack its own noise
    outb = torch.empty_like(data)
    wsb = torch.empty(B.wo_workspace_bytes(nb, Z, Y, X, ("phase",)), dtype=torch.uint8, device=dev)
    if not args.default_engines:
        B.wo_autotune(nb, Z, Y, X, ("phase",), wsb)  # engines timed on these shapes (the batch's workspace)

    def batch():
        B.wo_reconstruct_shared_tf(tf1k, kx, data, None, [1e-3], B.WO_ETA_RELATIVE, B.WO_MODE_3D, outb, nb, Z, Y, X,
                                   wsb)

    def batch_std():
        B.wo_reconstruct_shared_tf(tf1, ("phase",), data, None, [1e-3], B.WO_ETA_RELATIVE, B.WO_MODE_3D, outb, nb, Z,
                                   Y, X, wsb)

    ms = timed(batch, args.steps)
    ms_std = timed(batch_std, args.steps)
    prof = profiled_pass(B, batch, args.steps)
    vox = float(nb * Z * Y * X)
    half = Z * Y * (X // 2 + 1) * 8
    inside = Z * support_columns(o, ("phase",), Y, X) * 8
    real = Z * Y * X * 4
    planes_in = support_planes(o, ("phase",), X)
    algo = {"tile_pipeline": nb * 2 * real + half, "yz_op": nb * (planes_in * Z * Y * 8 + inside + half),
            "rows_r2c": nb * (real + half), "y_fwd": 2 * nb * half, "z_fused": nb * (inside + half),
            "y_inv": 2 * nb * half, "rows_c2r": nb * (half + real), "xy_fwd": nb * (real + half),
            "xy_inv": nb * (half + real)}
    kern = kernel_table(prof, algo, "launches")
    peak, _ = peaks()
    compulsory = 8.0 * vox
    out = {"workload": SMALL_WORKLOAD, "single_call_ms": round(lat, 4),
           "single_call_voxels_per_s": round(job_throughput(Z * Y * X, world, lat), 1),
           "batch": nb, "value": round(job_throughput(vox, world, ms), 1), "unit": "voxels/s",
           "ms_per_batch": round(ms, 4),
           "engine": "plane engine (kx-major bank shared by the batch)",
           "single_call_ms_with_passes": round(lat_std, 4), "ms_per_batch_with_passes": round(ms_std, 4),
           "compulsory_gbs": round(compulsory / (ms * 1e-3) / 1e9, 1),
           "compulsory_frac": round(compulsory / (ms * 1e-3) / 1e9 / peak, 4),
           "roofline": roofline_of(kern, prof), "kernels": kern,
           "schedule": dict(engines(Y, Z, rows=X // 2), xy=engines_xy(Y)),
           "l2": "batch data 268 MB in, 268 MB out (> L2); the shared TF bank 0.27 MB stays in L2"}
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = small_cpu_baseline(o, d1[0].cpu().numpy())
    del data, outb, wsb, tf1k, ws1k
    torch.cuda.empty_cache()
    return out if rank == 0 else None


# ------------------------------------------------------------------ auto-tuning
TUNE_TILES = 256
TUNE_SHAPE = (48, 192, 192)  # the shift-variant field's tiles
EST_SHAPE = (48, 128, 128)   # the learned estimator's tiles
TUNE_ETA = 1e-3
TUNE_WORKLOAD = {
    "all": ("auto-tuning of (defocus, tilt_x, tilt_y, NA_ill), 256 tiles of 48x192x192 with their own optics, "
            "smooth-edged source pupil: 50 Adam steps per tile from nominal (defocus 0, no tilt, NA_ill 0.825; 25 "
            "on the loss band-limited to 0.12 NA_det/lambda, 25 on the full loss with fresh moments); each step = "
            "per-plane build of the phase TF and its 4 derivatives + 2D thin-object loss and adjoint + Adam, one "
            "CUDA graph"),
    "defocus": ("defocus auto-tuning, 256 tiles of 48x192x192, per-tile optics: 50 Adam steps per tile from "
                "defocus 0 (25 on the loss band-limited to 0.12 NA_det/lambda, lr 0.08->0.02 um; 25 on the full "
                "loss with fresh moments, lr 0.02->0 um); each step = per-plane TF pair build (phase TF + d/d "
                "defocus) + 2D thin-object loss and adjoint + Adam, one CUDA graph")}


def tune_algorithmic_bytes(o, n, n_params):
    """Compulsory HBM bytes per launch of each kernel family of one Adam step
    over n tiles: 4 arms and 2 per-plane TF slots for the defocus alone, 7
    arms and 5 slots for the four parameters (no z transform)."""
    Z, Y, X = TUNE_SHAPE
    half = Z * Y * (X // 2 + 1) * 8
    n_arms, n_slots = (4, 2) if n_params == 1 else (7, 5)
    arms = n_arms * Z * Y * band_columns(o, X) * 8
    return {k: n * v for k, v in {
        "tf_pupil_record": Y * X * (16 if n_params == 1 else 32), "tf_arms": arms,
        "tf_psf_rows": arms + n_slots * half, "tf_ypass": 2 * n_slots * half,
        "tune_cols": (1 + n_slots) * half}.items()}


def make_tune_data(o_list, dev, seed=5, smooth=False):
    """Thin specimens (projected spheres) imaged at each tile's true optics by
    the 2D model: the 3D forward model of an object held in plane 0 alone
    (its z-DFT is flat, so plane j sees H_j of that plane), + 1e-3 noise."""
    import torch
    import phantom as ph
    from paper_2412_09775_gb300 import binding as B
    n = len(o_list)
    Z, Y, X = TUNE_SHAPE
    f = torch.zeros((n, Z, Y, X), dtype=torch.float32, device=dev)
    for t in range(n):
        f[t, 0] = torch.from_numpy(ph.thin_phantom(seed * 100003 + t, (Y, X), o_list[t], n_spheres=20)
                                   .astype(np.float32)).to(dev)
    kinds = B.WO_TF_PHASE | (B.WO_TF_SMOOTH_SOURCE if smooth else 0)
    tf, ws = B.alloc(n, Z, Y, X, kinds, dev)
    B.wo_build_tf(o_list, n, Z, Y, X, kinds, tf, ws)
    data = torch.empty_like(f)
    B.wo_forward(tf, kinds, f, [1.0], data, n, Z, Y, X, ws)
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    data += 1e-3 * torch.randn(data.shape, generator=g, device=dev, dtype=torch.float32)
    torch.cuda.synchronize()
    del f, tf, ws
    torch.cuda.empty_cache()
    return data


def tune_cpu_baseline(o, start, d, schedule, params, max_steps=4):
    """The oracle tuning one tile: the first `max_steps` of the same Adam
    schedule, each with the oracle's loss at theta +/- 1e-4 per parameter
    (central differences: the oracle has no adjoint); the time is scaled to
    the whole schedule."""
    from oracle import tuning as OT
    keys = OT.PARAMS[: len(params)]
    total = sum(ph_.steps for ph_ in schedule)
    done = 0
    t0 = time.perf_counter()
    th = np.array([start[k] for k in keys])
    m = np.zeros_like(th)
    v = np.zeros_like(th)
    k = 0
    for ph_ in schedule:
        if ph_.reset:
            m[:], v[:], k = 0.0, 0.0, 0
        for i in range(ph_.steps):
            if done >= max_steps:
                break
            done += 1
            lr = np.array(ph_.lr_at(i), dtype=float).reshape(-1)
            nu = ph_.nu_max if ph_.nu_max > 0 else None
            cur = dict(start, **dict(zip(keys, th)))
            g = np.zeros_like(th)
            for q, key in enumerate(keys):
                g[q] = (OT.objective(dict(cur, **{key: cur[key] + 1e-4}), d, TUNE_ETA, nu)
                        - OT.objective(dict(cur, **{key: cur[key] - 1e-4}), d, TUNE_ETA, nu)) / 2e-4
            k += 1
            m = 0.9 * m + 0.1 * g
            v = 0.999 * v + 0.001 * g * g
            th = th - lr * (m / (1 - 0.9 ** k)) / (np.sqrt(v / (1 - 0.999 ** k)) + 1e-8)
    dt = (time.perf_counter() - t0) * total / max(done, 1)
    return {"value": 1.0 / dt, "unit": "tiles/s", "cores": 1, "kind": "oracle",
            "sample": f"numpy float64 oracle tuning 1 of the 256 tiles ({'x'.join(map(str, TUNE_SHAPE))}): the first {done} of the "
                      f"{total} Adam steps of the same schedule with central-difference gradients "
                      f"({2 * len(keys)} loss evaluations per step), timed and scaled to {total} steps "
                      f"({dt:.1f} s per tile), single thread"}


def autotune_leg(args, rank, world, local_rank, with_cpu=True):
    """Times the whole 50-step tuning of 256 tiles; returns the summary dict."""
    import torch
    import phantom as ph
    from paper_2412_09775_gb300 import autotune as A, binding as B
    from paper_2412_09775_gb300.shard import job_throughput, max_over_ranks
    dev = torch.device("cuda", local_rank)
    n = args.tune_tiles
    Z, Y, X = TUNE_SHAPE
    four = args.tune_params == "all"
    truth = ph.tile_optics(np.random.default_rng(7 + rank), n)
    if four:
        truth = [dict(o, smooth_source=True) for o in truth]
        start = [dict(o, defocus_um=0.0, tilt_x=0.0, tilt_y=0.0, na_ill=0.825) for o in truth]
    else:
        start = [dict(o, defocus_um=0.0) for o in truth]
    data = make_tune_data(truth, dev, seed=5 + rank, smooth=four)
    pb = A.TuningProblem(data, start, TUNE_ETA, params=args.tune_params)
    if not args.default_engines:
        B.wo_autotune(n, Z, Y, X, pb.kinds, pb.ws)  # the workspace is scratch between calls
    sched = A.default_schedule4(truth[0]) if four else A.default_schedule(truth[0])
    n_adam = sum(p.steps for p in sched)
    # per-kernel times of one eager Adam step on the full loss
    B.wo_profile_read()
    B.wo_profile_enable(True)
    pb.step(0.0, 0.0)
    torch.cuda.synchronize()
    B.wo_profile_enable(False)
    prof = B.wo_profile_read()
    per_adam_step = sum(c for c, _ in prof.values())  # library launches of one Adam step
    pb.run(sched, graph=True)  # captures (and replays once)
    per_run = n_adam * per_adam_step
    for _ in range(args.warmup):
        pb.reset()
        pb.run(sched, graph=True)
    torch.cuda.synchronize()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream()
    nvml = NvmlClockSampler(dev)
    with nvml:
        ev0.record(stream)
        for _ in range(args.steps):
            pb.reset()
            pb.run(sched, graph=True)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, device=dev)
    keys = ("defocus_um", "tilt_x", "tilt_y", "na_ill")[: pb.n_params]
    errs = np.abs(pb.params().cpu().numpy() - np.array([[o[k] for k in keys] for o in truth]))
    err = errs[:, 0]
    # end to end: host stacks in (pinned), tuned defocus out
    h_in = torch.empty(data.shape, dtype=torch.float32, pin_memory=True)
    h_in.copy_(data.cpu())
    h_out = torch.empty(n, dtype=torch.float64, pin_memory=True)
    d_in = torch.empty_like(data)

    def e2e_step():
        d_in.copy_(h_in, non_blocking=True)
        pb.set_data(d_in)
        pb.reset()
        pb.run(sched, graph=True)
        h_out.copy_(pb.defocus, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, device=dev)
    algo = tune_algorithmic_bytes(truth[0], n, pb.n_params)
    tot = sum(v[1] for v in prof.values())
    kern = {}
    for name, (cnt, t) in prof.items():
        b = algo.get(name)
        kern[name] = {"launches_per_adam_step": cnt, "avg_ms": round(t / cnt, 4), "share": round(t / tot, 4),
                      "algo_bytes": b, "gbs": round(b / (t / cnt * 1e-3) / 1e9, 1) if b else None}
    dom = max(prof.items(), key=lambda kv: kv[1][1])[0]
    peak, peak_kind = peaks()
    out = {
        "value": round(job_throughput(n, world, ms), 2), "unit": "tiles/s", "ms_per_step": round(ms, 3),
        "workload": TUNE_WORKLOAD[args.tune_params] if n == TUNE_TILES else f"profiling case: {n} tiles",
        "adam_steps": n_adam, "ms_per_adam_step": round(ms / n_adam, 4),
        "defocus_error_um": {"max": round(float(err.max()), 4), "median": round(float(np.median(err)), 4),
                             "frac_within_0.05": round(float(np.mean(err <= 0.05)), 4)},
        "param_error_max": {k: round(float(errs[:, i].max()), 5) for i, k in enumerate(keys)},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": kern[dom]["gbs"], "peak": peak, "unit": "GB/s",
                     "frac": round(kern[dom]["gbs"] / peak, 4) if kern[dom]["gbs"] else None, "traffic": None,
                     "peak_source": peak_kind},
        "kernels": kern, "gpu_launches": int(per_run * args.steps), "clocks": nvml.summary(),
        "e2e": {"value": round(job_throughput(n, world, e2e_ms), 2), "unit": "tiles/s",
                "ms_per_step": round(e2e_ms, 3), "h2d_bytes_per_step": int(data.numel() * 4),
                "d2h_bytes_per_step": int(n * 8)},
        "l2": "working set > L2: arms 6.4 GB, TF pair 1.6 GB, spectra 0.8 GB",
        "schedule": engines(Y, Z, rows=X // 2),
    }
    if with_cpu and rank == 0 and not args.no_cpu_baseline:
        d0 = data[0].double().cpu().numpy()
        out["cpu_baseline"] = tune_cpu_baseline(truth[0], start[0], d0, sched, keys)
    del pb, data, d_in
    torch.cuda.empty_cache()
    return out


def run_autotune(args, rank, world, local_rank):
    import torch
    from paper_2412_09775_gb300.build import build
    build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    r = autotune_leg(args, rank, world, local_rank)
    if rank != 0:
        return
    line = {"metric": METRIC, "value": r["value"], "unit": "tiles/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (thin sphere-projection specimens, GPU forward model at each tile's optics + "
                    "1e-3 noise)",
            "config": {"workload": r["workload"], "tiles": args.tune_tiles, "tile": list(TUNE_SHAPE), "eta": TUNE_ETA,
                       "parallelism": f"replicas x{world}", "l2": r["l2"], "schedule": r["schedule"]}}
    for k in ("defocus_error_um", "param_error_max", "roofline", "kernels", "gpu_launches", "clocks", "e2e",
              "cpu_baseline", "ms_per_adam_step"):
        if k in r:
            line[k] = r[k]
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ learned estimator
EST_TRAIN = 100000
EST_TEST = 4096
EST_FALLBACK = 2.0  # refined loss above this multiple of the batch median: the 50-step schedule for that tile
EST_WORKLOAD = ("learned optics estimator: conv net (4 conv 3x3 + pool + linear, 186k bfloat16 weights, float32 "
                "sums) trained on forward-simulated tiles of 48x128x128, then inference on 4096 tiles + 10 "
                "refinement Adam steps (tiles whose refined loss stays above 2x the batch median get the "
                "50-step schedule), against 50-step auto-tuning from nominal on the same tiles")


def estimator_leg(args, rank, world, local_rank):
    import torch
    import phantom as ph
    from paper_2412_09775_gb300.build import build
    build()
    from paper_2412_09775_gb300 import autotune as A, binding as B, estimator as E
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    base = ph.optics()
    shape = EST_SHAPE
    Z, Y, X = shape

    def clock(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = fn()
        torch.cuda.synchronize()
        return r, time.perf_counter() - t0

    (feat, truth), t_gen = clock(lambda: E.generate(args.est_train, shape, base, seed=100 + rank, device=dev))
    est = E.Estimator(dev, seed=rank, batch=256)
    losses, t_train = clock(lambda: est.train(feat, truth, epochs=args.est_epochs, lr=2e-3))
    # per-kernel times of training steps (the library's event profiler, a pass of its own)
    f0, t0_ = feat[:256].contiguous(), truth[:256].contiguous()

    def train_step():
        B.wo_est_train_step(est.w32, est.wbf, est.m, est.v, f0, t0_, 256, E.SCALE, E.OFFSET, est.step + 1, 0.0,
                            est.loss, est.ws)
    step_prof = profiled_pass(B, train_step, 5)
    step_kern = {k: {"launches_per_step": c // 5, "ms_per_step": round(t / 5, 4)} for k, (c, t) in step_prof.items()}
    n_steps = args.est_epochs * (args.est_train // 256)
    del feat
    torch.cuda.empty_cache()
    # test tiles: stacks kept for the refinement, in chunks of 256
    rng = np.random.default_rng(200 + rank)
    gen = torch.Generator(device=dev)
    gen.manual_seed(200 + rank)
    sim = E.Simulator(shape, 256, dev)
    n_test = args.est_test
    stacks, optics, truths = [], [], []
    for i0 in range(0, n_test, 256):
        m = min(256, n_test - i0)
        ol = E.random_optics(rng, m, base)
        stacks.append(sim.stacks(ol, E.sphere_params(rng, m, shape[1:], base["pixel_um"]), 1e-3, gen))
        optics.append(ol)
        truths.append(np.array([[o["defocus_um"], o["tilt_x"], o["tilt_y"], o["na_ill"]] for o in ol]))
    nominal = [dict(o, defocus_um=0.0, tilt_x=0.0, tilt_y=0.0, na_ill=0.825) for o in optics[0]]
    refine, plain = A.refine_schedule(10), A.default_schedule4(base)

    def new_problem(data, start):
        q = A.TuningProblem(data, start, TUNE_ETA, params="all")
        if not args.default_engines:
            B.wo_autotune(q.n, Z, Y, X, q.kinds, q.ws)
        for sch in (refine, plain):  # capture both graphs outside the timed regions
            q.run(sch, graph=True)
            q.reset()
        return q

    pb = new_problem(stacks[0], nominal)
    fb = new_problem(stacks[0], nominal)  # fallback batch: plain tuning of the tiles the refinement did not fit
    feats = torch.empty((256, 3, 64, 64), dtype=torch.float32, device=dev)
    t_feat = t_inf = t_ref = t_plain = t_fb = 0.0
    est_err, ref_err, plain_err = [], [], []
    flagged = []  # (chunk, tile) whose refined loss stays above EST_FALLBACK x the chunk's median
    for c, data in enumerate(stacks):
        m = data.shape[0]
        ol = optics[c]
        nom = [dict(o, defocus_um=0.0, tilt_x=0.0, tilt_y=0.0, na_ill=0.825) for o in ol]
        _, dt = clock(lambda: sim.features(data, B.optics_tensor(nom, dev), feats[:m]))
        t_feat += dt
        pred, dt = clock(lambda: est.predict(feats[:m]))
        t_inf += dt
        p = pred.cpu().numpy().astype(np.float64)
        est_err.append(np.abs(p - truths[c]))
        start = [dict(o, defocus_um=float(q[0]), tilt_x=float(q[1]), tilt_y=float(q[2]),
                      na_ill=float(np.clip(q[3], 0.5, 1.0))) for o, q in zip(nom, p)]
        if m != pb.n:
            pb = new_problem(data, start)
        pb.set_data(data)
        pb.restart(start)

        def refine_and_check():
            pb.run(refine, graph=True)
            pb.evaluate()  # the loss at the refined optics
            return pb.value.cpu().numpy()
        val, dt = clock(refine_and_check)
        t_ref += dt
        ref_err.append(np.abs(pb.params().cpu().numpy() - truths[c]))
        flagged += [(c, i) for i in np.nonzero(val > EST_FALLBACK * np.median(val))[0]]
        pb.restart(nom)
        _, dt = clock(lambda: pb.run(plain, graph=True))
        t_plain += dt
        plain_err.append(np.abs(pb.params().cpu().numpy() - truths[c]))
    # fallback: the flagged tiles, in batches of 256, get the plain schedule
    n_flag = len(flagged)
    for f0 in range(0, n_flag, 256):
        part = flagged[f0:f0 + 256]

        def fallback():
            batch = [stacks[c][i] for c, i in part]
            batch += [batch[-1]] * (256 - len(batch))  # pad to the captured batch size
            fb.set_data(torch.stack(batch))
            starts = [dict(optics[c][i], defocus_um=0.0, tilt_x=0.0, tilt_y=0.0, na_ill=0.825) for c, i in part]
            fb.restart(starts + [starts[-1]] * (256 - len(starts)))
            fb.run(plain, graph=True)
            return fb.params().cpu().numpy()
        res, dt = clock(fallback)
        t_fb += dt
        for k, (c, i) in enumerate(part):
            ref_err[c][i] = np.abs(res[k] - truths[c][i])
    est_err, ref_err, plain_err = (np.concatenate(e) for e in (est_err, ref_err, plain_err))
    if rank != 0:
        return None

    def summary(err):
        return {"defocus_max_um": round(float(err[:, 0].max()), 4),
                "defocus_median_um": round(float(np.median(err[:, 0])), 4),
                "frac_defocus_within_0.05": round(float(np.mean(err[:, 0] <= 0.05)), 4),
                "illumination_max_na": [round(float(err[:, k].max()), 4) for k in (1, 2, 3)]}

    learned_s = (t_feat + t_inf + t_ref + t_fb) / n_test
    plain_s = t_plain / n_test
    line = {"metric": METRIC, "value": round(1.0 / learned_s, 2), "unit": "tiles/s", "n_gpus": world,
            "steps": 1, "warmup": 1, "ms_per_step": round(1e3 * (t_feat + t_inf + t_ref + t_fb), 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16 weights, f32 sums",
            "data": "synthetic (thin sphere-projection specimens, forward model with the smooth source, 1e-3 noise)",
            "config": {"workload": EST_WORKLOAD, "train_tiles": args.est_train, "epochs": args.est_epochs,
                       "test_tiles": n_test, "tile": list(shape), "parallelism": f"replicas x{world}"},
            "learned": {"s_per_tile": learned_s, "features_s": t_feat, "inference_s": t_inf, "refine_10_s": t_ref,
                        "fallback_s": t_fb, "fallback_tiles": n_flag,
                        "estimate_error": summary(est_err), "refined_error": summary(ref_err)},
            "plain": {"s_per_tile": plain_s, "tune_50_s": t_plain, "error": summary(plain_err)},
            "speedup_vs_plain": round(plain_s / learned_s, 2),
            # the one-off cost of training, spread over the test tiles, and the
            # number of tiles after which it has paid for itself
            "learned_with_training_s_per_tile": (t_gen + t_train) / n_test + learned_s,
            "break_even_tiles": (round((t_gen + t_train) / (plain_s - learned_s)) if plain_s > learned_s
                                 else None),
            "training": {"generate_s": round(t_gen, 2), "train_s": round(t_train, 2), "steps": n_steps,
                         "ms_per_step": round(1e3 * t_train / max(n_steps, 1), 3), "step_kernels": step_kern,
                         "loss_per_epoch": [round(v, 5) for v in losses], "params": est.n}}
    return line


def run_estimator(args, rank, world, local_rank):
    line = estimator_leg(args, rank, world, local_rank)
    if line is not None:
        print(json.dumps(line), flush=True)


def _oracle_field_tile(job):
    """Worker: one tile of the field workload made on the host - a sphere
    phantom region (the field's sphere density, 140 spheres per 48x192x192
    tile) imaged by the oracle's forward model with the tile's optics, plus
    1e-3 Gaussian noise."""
    import phantom as ph
    from oracle import model as OM, optics as OO
    o, seed = job
    shape = (FIELD_Z, TILE_CORE + 2 * TILE_HALO, TILE_CORE + 2 * TILE_HALO)
    dn = ph.sphere_phantom(seed, shape, o, n_spheres=140)
    modes, _, _ = OM.widefield_system(OO.transfer_functions(o, shape, ("phase",)), ("phase",))
    d = OM.forward(modes, dn[None], [1.0])[0] + ph.gaussian_noise(seed + 1, shape, 1e-3)
    return d.astype(np.float32)


def run_reference(args, rank, world):
    """The float64 oracle timed on the host cores on the field workload: each
    step reconstructs (TF build + 3D Tikhonov) one tile per host core in a pool
    of spawned processes; the value is field voxels/s scaled from the tiles
    done (256 tiles per field; gather and blend left out, a few % of the
    oracle's time)."""
    if rank != 0:
        return
    import multiprocessing as mp
    import phantom as ph
    cores = os.cpu_count() or 1
    n = TILE_GRID[0] * TILE_GRID[1]
    o_list = ph.tile_optics(np.random.default_rng(3), n)
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        tiles = pool.map(_oracle_field_tile, [(o_list[t], 1000 + t) for t in range(cores)], chunksize=1)
        jobs = [(o_list[t], tiles[t]) for t in range(cores)]
        for _ in range(args.warmup):
            pool.map(_oracle_tile, jobs, chunksize=1)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            pool.map(_oracle_tile, jobs, chunksize=1)
        dt = (time.perf_counter() - t0) / max(1, args.steps)
    field_vox = float(FIELD_Z * (TILE_GRID[0] * TILE_CORE) * (TILE_GRID[1] * TILE_CORE))
    value = field_vox * (cores / n) / dt
    sample = (f"numpy float64 oracle (no reference code exists: the paper ships none) on the field workload: "
              f"per step, TF build + 3D Tikhonov of {cores} of the 256 tiles of 48x192x192 (one per process, "
              f"{cores} spawned processes), {dt:.2f} s per step, scaled to field voxels/s")
    line = {"impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": "voxels/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": TILES_WORKLOAD, "tiles_per_step": cores},
            "cpu_baseline": {"value": round(value, 1), "unit": "voxels/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 1), "unit": "voxels/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg")
    ap.add_argument("--no-library-fft", action="store_true",
                    help="skip timing the torch.fft composition of the forward model and reconstruction")
    ap.add_argument("--workload", choices=["field", "tiles", "widefield", "autotune", "estimator", "small"],
                    default="field",
                    help="field (default): the shift-variant field as the headline with the auto-tuning, widefield "
                         "and small-stack legs; tiles: the field line alone; small: the small-stack leg alone")
    ap.add_argument("--field-only", action="store_true", help="field workload without the other legs")
    ap.add_argument("--no-estimator", action="store_true", help="default run without the learned-estimator leg")
    ap.add_argument("--default-engines", action="store_true",
                    help="skip the engine autotuner (built-in engine choices; for runs under a profiler, whose "
                         "serialised launches would mislead the autotuner's timings)")
    ap.add_argument("--field-engine", choices=["planes", "passes"], default="planes",
                    help="field step: kx-major TF bank and one y-z pass per (tile, k_x) plane (planes), or the "
                         "standard bank and separate y, z and inverse y passes (passes); the other is timed as context")
    ap.add_argument("--est-train", type=int, default=EST_TRAIN, help="estimator training tiles")
    ap.add_argument("--est-epochs", type=int, default=12, help="estimator training epochs")
    ap.add_argument("--est-test", type=int, default=EST_TEST, help="estimator test tiles")
    ap.add_argument("--no-autotune", action="store_true",
                    help="widefield workload: skip the auto-tuning summary leg")
    ap.add_argument("--tune-tiles", type=int, default=TUNE_TILES,
                    help="auto-tuning tiles (fewer only for profiler captures)")
    ap.add_argument("--tune-params", choices=["all", "defocus"], default="all",
                    help="auto-tuning of (defocus, tilt_x, tilt_y, NA_ill) or of the defocus alone")
    ap.add_argument("--e2e-streams", type=int, default=3,
                    help="streams the end-to-end leg's consecutive steps go round (1: serial)")
    ap.add_argument("--rows-engine", choices=["default", "smem", "hybrid"], default="default",
                    help="engine of the x passes (default: the library's choice)")
    ap.add_argument("--shape", type=int, nargs=3, default=None,
                    help="override Z Y X (smaller cases for profiler captures only)")
    ap.add_argument("--tile-grid", type=int, nargs=2, default=None,
                    help="field workload: tiles along y and x (smaller cases for profiler captures only)")
    args = ap.parse_args()
    if args.shape:
        global SHAPE
        SHAPE = tuple(args.shape)
    if args.tile_grid:
        global TILE_GRID
        TILE_GRID = tuple(args.tile_grid)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    try:
        if args.workload in ("field", "tiles"):
            if args.workload == "tiles":
                args.field_only = True
            run_tiles(args, rank, world, local_rank)
        elif args.workload == "autotune":
            run_autotune(args, rank, world, local_rank)
        elif args.workload == "estimator":
            run_estimator(args, rank, world, local_rank)
        elif args.workload == "small":  # the small-stack leg alone
            import torch
            from paper_2412_09775_gb300.build import build
            build()
            torch.cuda.set_device(local_rank)
            out = small_stack_leg(args, rank, world, local_rank)
            if rank == 0:
                print(json.dumps(out), flush=True)
        else:
            run_gpu(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
