"""Per-tile defocus auto-tuning through the library's hand-written adjoint.

The paper tunes each tile's optical parameters by gradient descent on a scalar
loss of the reconstruction (Results, physics-guided auto-tuning; Fig. 2a(iv);
Ext. Data Fig. 3).  Here the loss is the 2D thin-object Tikhonov fit
(wo_defocus_objective) and the parameter is the tile's defocus; every step of
the arithmetic runs in the library's kernels:

* ``DefocusProblem`` holds the device buffers of one batch of tiles: their
  optics (float64 [n, 9], the device array the TF build reads), the data
  spectra (wo_spectrum, computed once), a WO_TF_PHASE_DZ bank (per plane by
  default: the loss needs no z transform, by Parseval), the workspace,
  and the per-tile loss, gradient and Adam state.
* ``DefocusLoss`` is a torch.autograd.Function over the defocus vector: its
  forward builds the TF pair and evaluates loss and derivative in one pass,
  its backward returns that derivative times the incoming gradient.
* ``DefocusProblem.run`` applies a schedule of ``Phase``s of Adam steps
  (wo_adam_defocus, state on the device), eagerly or replayed from one
  captured CUDA graph.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

from . import binding as B

PHASE_DZ = B.WO_TF_PHASE_DZ


class DefocusProblem:
    """``planes`` (default): per-plane TF banks and 2D data spectra, so no z
    transform runs per step; otherwise 3D banks and spectra (the same loss by
    Parseval over z).  ``loss``: the data-fidelity loss (default) or the
    paper's mid-band power loss (WO_LOSS_MIDBAND)."""

    def __init__(self, data: torch.Tensor, optics_list, eta: float, background=None, planes: bool = True,
                 loss: int = B.WO_LOSS_DATA):
        if data.dim() != 4 or data.dtype != torch.float32 or not data.is_cuda:
            raise ValueError("data: float32 CUDA tensor [n_tiles, Z, Y, X]")
        self.n, self.Z, self.Y, self.X = (int(s) for s in data.shape)
        if len(optics_list) != self.n:
            raise ValueError("one optics entry per tile")
        dev = data.device
        self.eta = float(eta)
        self.loss = int(loss)
        self.kinds = PHASE_DZ | (B.WO_TF_PLANES if planes else 0)
        self.mode = B.WO_MODE_2D if planes else B.WO_MODE_3D
        self.optics = B.optics_tensor(optics_list, dev)
        self.optics0 = self.optics.clone()
        self.tf, self.ws = B.alloc(self.n, self.Z, self.Y, self.X, self.kinds, dev)
        self.spec = torch.empty((self.n, self.Z, self.Y, self.X // 2 + 1), dtype=torch.complex64, device=dev)
        self.background = background
        self.set_data(data)
        self.value = torch.zeros(self.n, dtype=torch.float64, device=dev)
        self.grad = torch.zeros_like(self.value)
        self.state = torch.zeros((self.n, 3), dtype=torch.float64, device=dev)
        self._graph = None
        self._graph_key = None

    def set_data(self, data: torch.Tensor):
        """New stacks for the same tiles (the spectra are recomputed)."""
        B.wo_spectrum(data.contiguous(), self.background, self.mode, self.spec, self.n, self.Z, self.Y, self.X)

    @property
    def defocus(self) -> torch.Tensor:
        return self.optics[:, 8]

    def reset(self):
        """Back to the starting optics, Adam state cleared."""
        self.optics.copy_(self.optics0)
        self.state.zero_()

    def evaluate(self, nu_max: float = 0.0):
        """Loss and defocus derivative of every tile at the current optics."""
        n, Z, Y, X = self.n, self.Z, self.Y, self.X
        B.wo_build_tf_device(self.optics, n, Z, Y, X, self.kinds, self.tf, self.ws)
        B.wo_defocus_objective(self.tf, self.kinds, self.optics, self.spec, self.loss, self.eta, nu_max, self.value,
                               self.grad, n, Z, Y, X, self.ws)

    def step(self, lr: float, nu_max: float = 0.0, beta1=0.9, beta2=0.999, eps=1e-8):
        self.evaluate(nu_max)
        B.wo_adam_defocus(self.optics, self.grad, self.state, self.n, lr, beta1, beta2, eps)

    def _queue(self, schedule):
        for ph in schedule:
            if ph.reset:
                self.state.zero_()
            for i in range(ph.steps):
                self.step(ph.lr_at(i), ph.nu_max)

    def run(self, schedule, graph: bool = True):
        """Apply ``schedule`` (a sequence of ``Phase``) of Adam steps.

        With ``graph`` the whole schedule is captured once into a CUDA graph
        (after one eager pass that sets up the kernels, undone afterwards)
        and replayed; the Adam state lives on the device, so the replay
        continues from wherever the optics stand.
        """
        key = tuple(schedule)
        if not graph:
            self._queue(key)
            return
        if self._graph is None or self._graph_key != key:
            saved_o, saved_s = self.optics.clone(), self.state.clone()
            self._queue(key[:1])  # first launch of every kernel, outside the capture
            torch.cuda.synchronize()
            self.optics.copy_(saved_o)
            self.state.copy_(saved_s)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                self._queue(key)
            self._graph, self._graph_key = g, key
        self._graph.replay()


@dataclass(frozen=True)
class Phase:
    """``steps`` Adam steps on the loss restricted to |nu| <= nu_max (0: the
    full loss), the step size going from lr_start to lr_end (um) along half a
    cosine; ``reset`` clears the Adam moments first (a new loss)."""
    steps: int
    lr_start: float
    lr_end: float
    nu_max: float = 0.0
    reset: bool = False

    def lr_at(self, i: int) -> float:
        if self.steps <= 1:
            return self.lr_start
        w = 0.5 * (1.0 + math.cos(math.pi * i / self.steps))
        return self.lr_end + (self.lr_start - self.lr_end) * w


def default_schedule(o) -> tuple:
    """50 Adam steps from a nominal defocus: 25 on the loss band-limited to
    |nu| <= 0.12 NA_det/lambda (a wide basin; lr 0.08 -> 0.02 um), then 25 on
    the full loss with fresh moments (lr 0.02 -> 0 um)."""
    nu = 0.12 * o["na_det"] / o["lambda_um"]
    return (Phase(25, 0.08, 0.02, nu), Phase(25, 0.02, 0.0, 0.0, reset=True))


class DefocusLoss(torch.autograd.Function):
    """loss[t] = L_t(defocus[t]) with dL/d(defocus) from the library's adjoint."""

    @staticmethod
    def forward(ctx, defocus: torch.Tensor, problem: DefocusProblem, nu_max: float = 0.0):
        problem.optics[:, 8].copy_(defocus.detach())
        problem.evaluate(nu_max)
        ctx.save_for_backward(problem.grad.clone())
        return problem.value.clone()

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out * g, None, None


def defocus_loss(defocus: torch.Tensor, problem: DefocusProblem, nu_max: float = 0.0) -> torch.Tensor:
    return DefocusLoss.apply(defocus, problem, nu_max)
