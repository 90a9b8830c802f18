"""The learned optics estimator: training data from the forward model, the
network's training and inference, all in the library's kernels.

A tile's optics (defocus, tilt_x, tilt_y, NA_ill) are estimated from
features of its spectra (wo_est_features) by a small convolutional network
with bfloat16 weights (wo_est_forward / wo_est_train_step), as the starting
point of a short auto-tuning run (autotune.TuningProblem).  Training tiles
are thin specimens (wo_thin_phantom) imaged by the forward model with the
smooth-edged source pupil (wo_build_tf, wo_forward) at seeded random optics.
The host only draws the random optics and sphere parameters and moves
arguments; every array operation runs in the library.
"""
from __future__ import annotations

import numpy as np
import torch

from . import binding as B

# standardisation of the outputs: optics = SCALE * net + OFFSET
SCALE = (1.0, 0.1, 0.1, 0.125)
OFFSET = (0.0, 0.0, 0.0, 0.825)
KINDS = B.WO_TF_PHASE | B.WO_TF_SMOOTH_SOURCE


def random_optics(rng: np.random.Generator, n: int, base: dict) -> list:
    """Seeded optics draws of the shift-variant tiles: defocus U[-1, 1] um,
    tilt U[-0.1, 0.1] NA per axis, NA_ill U[0.7, 0.95]."""
    out = []
    for _ in range(n):
        out.append(dict(base, defocus_um=rng.uniform(-1, 1), tilt_x=rng.uniform(-0.1, 0.1),
                        tilt_y=rng.uniform(-0.1, 0.1), na_ill=rng.uniform(0.7, 0.95), smooth_source=True))
    return out


def sphere_params(rng: np.random.Generator, n: int, shape2d, pixel_um: float, n_spheres: int = 20):
    """(n, n_spheres, 4) float32: centre y, centre x (uniform on the tile),
    radius U[0.5, 2] um, index increment U[0.005, 0.03]."""
    Y, X = shape2d
    p = np.empty((n, n_spheres, 4), dtype=np.float32)
    p[..., 0] = rng.uniform(0, Y * pixel_um, (n, n_spheres))
    p[..., 1] = rng.uniform(0, X * pixel_um, (n, n_spheres))
    p[..., 2] = rng.uniform(0.5, 2.0, (n, n_spheres))
    p[..., 3] = rng.uniform(0.005, 0.03, (n, n_spheres))
    return p


class Simulator:
    """Brightfield stacks of thin specimens at given optics (forward model,
    smooth source), in batches of at most `batch` tiles."""

    def __init__(self, shape, batch: int, device):
        self.Z, self.Y, self.X = shape
        self.batch = batch
        self.dev = device
        Z, Y, X = shape
        self.tf, self.ws = B.alloc(batch, Z, Y, X, KINDS, device)
        self.obj = torch.zeros((batch, Z, Y, X), dtype=torch.float32, device=device)
        self.plane = torch.empty((batch, Y, X), dtype=torch.float32, device=device)
        self.spec = torch.empty((batch, Z, Y, X // 2 + 1), dtype=torch.complex64, device=device)

    def stacks(self, optics, params, noise: float, gen: torch.Generator):
        """Stacks [n, Z, Y, X] for n = len(optics) <= batch tiles."""
        n = len(optics)
        Z, Y, X = self.Z, self.Y, self.X
        par = torch.from_numpy(params).to(self.dev)
        # the specimen in plane 0 alone: its z-DFT is flat, so plane j sees H_j
        B.wo_thin_phantom(par, n, params.shape[1], Y, X, optics[0]["pixel_um"], optics[0]["z_step_um"], self.plane)
        self.obj[:n, 0].copy_(self.plane[:n])
        B.wo_build_tf(optics, n, Z, Y, X, KINDS, self.tf, self.ws)
        data = torch.empty((n, Z, Y, X), dtype=torch.float32, device=self.dev)
        B.wo_forward(self.tf, KINDS, self.obj[:n], [1.0], data, n, Z, Y, X, self.ws)
        data += noise * torch.randn(data.shape, generator=gen, device=self.dev, dtype=torch.float32)
        return data

    def features(self, data, d_optics, out):
        n = data.shape[0]
        B.wo_spectrum(data, None, B.WO_MODE_2D, self.spec[:n], n, self.Z, self.Y, self.X)
        B.wo_est_features(self.spec[:n], d_optics, n, self.Z, self.Y, self.X, out)


def generate(n: int, shape, base: dict, seed: int, device, batch: int = 256, noise: float = 1e-3):
    """Features [n, 3, 64, 64] and true optics [n, 4] (float32, on the device)
    of n seeded forward-simulated tiles."""
    rng = np.random.default_rng(seed)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    sim = Simulator(shape, batch, device)
    feat = torch.empty((n, 3, 64, 64), dtype=torch.float32, device=device)
    truth = torch.empty((n, 4), dtype=torch.float32, device=device)
    for i0 in range(0, n, batch):
        m = min(batch, n - i0)
        ol = random_optics(rng, m, base)
        par = sphere_params(rng, m, shape[1:], base["pixel_um"])
        data = sim.stacks(ol, par, noise, gen)
        sim.features(data, B.optics_tensor(ol, device), feat[i0:i0 + m])
        truth[i0:i0 + m] = torch.tensor([[o["defocus_um"], o["tilt_x"], o["tilt_y"], o["na_ill"]] for o in ol],
                                        dtype=torch.float32, device=device)
    return feat, truth


class Estimator:
    """The network's float32 master weights, bfloat16 copy and Adam moments."""

    def __init__(self, device, seed: int = 0, batch: int = 256):
        n = B.wo_est_param_count()
        self.n, self.batch, self.dev = n, batch, device
        rng = np.random.default_rng(seed)
        w = np.zeros(n, dtype=np.float32)
        off = 0
        for ci, co in ((3, 32), (32, 64), (64, 96), (96, 128)):  # He-normal weights, zero biases
            k = co * ci * 9
            w[off:off + k] = rng.normal(0.0, np.sqrt(2.0 / (ci * 9)), k)
            off += k + co
        w[off:off + 4 * 128] = rng.normal(0.0, np.sqrt(1.0 / 128), 4 * 128)
        self.w32 = torch.from_numpy(w).to(device)
        self.wbf = torch.empty(n, dtype=torch.int16, device=device)
        self.m = torch.zeros(n, dtype=torch.float32, device=device)
        self.v = torch.zeros(n, dtype=torch.float32, device=device)
        self.ws = torch.empty(B.wo_est_workspace_bytes(batch), dtype=torch.uint8, device=device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=device)
        self.step = 0
        B.wo_est_sync_bf16(self.w32, self.wbf)

    def train(self, feat, truth, epochs: int, lr: float = 1e-3, seed: int = 0):
        """Mini-batch Adam over shuffled batches; returns the last batch loss of every epoch."""
        n = feat.shape[0]
        gen = torch.Generator(device=self.dev)
        gen.manual_seed(seed)
        losses = []
        for ep in range(epochs):
            order = torch.randperm(n, generator=gen, device=self.dev)
            rate = lr * 0.5 * (1.0 + np.cos(np.pi * ep / max(epochs, 1)))  # cosine decay over epochs
            for i0 in range(0, n - self.batch + 1, self.batch):
                idx = order[i0:i0 + self.batch]
                f = feat.index_select(0, idx)
                t = truth.index_select(0, idx)
                self.step += 1
                B.wo_est_train_step(self.w32, self.wbf, self.m, self.v, f, t, self.batch, SCALE, OFFSET, self.step,
                                    rate, self.loss, self.ws)
            losses.append(float(self.loss.item()))
        return losses

    def predict(self, feat):
        """Optics [n, 4] (defocus_um, tilt_x, tilt_y, na_ill) of n tiles."""
        n = feat.shape[0]
        out = torch.empty((n, 4), dtype=torch.float32, device=self.dev)
        for i0 in range(0, n, self.batch):
            m = min(self.batch, n - i0)
            B.wo_est_forward(self.wbf, self.w32, feat[i0:i0 + m], m, SCALE, OFFSET, out[i0:i0 + m], self.ws)
        return out
