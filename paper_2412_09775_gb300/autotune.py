"""Per-tile auto-tuning of the optics through the library's hand-written adjoint.

The paper tunes each tile's optical parameters by gradient descent on a scalar
loss of the reconstruction (Results, physics-guided auto-tuning; Fig. 2a(iv);
Ext. Data Fig. 3).  Here the loss is the 2D thin-object Tikhonov fit or the
paper's mid-band power (wo_tune_objective) and the parameters are the tile's
defocus, or defocus, illumination tilt (x, y) and NA_ill under the smooth
source pupil; every step of the arithmetic runs in the library's kernels:

* ``TuningProblem`` holds the device buffers of one batch of tiles: their
  optics (float64 [n, 9], the device array the TF build reads), the data
  spectra (wo_spectrum, computed once), a derivative bank (per plane by
  default: the loss needs no z transform, by Parseval), the workspace, and
  the per-tile loss, gradient and Adam state.
* ``TuneLoss`` is a torch.autograd.Function over the tuned parameters: its
  forward builds the TF and its derivatives and evaluates loss and gradient
  in one pass, its backward returns that gradient times the incoming one.
* ``TuningProblem.run`` applies a schedule of ``Phase``s of Adam steps
  (wo_adam_optics, state on the device), eagerly or replayed from one
  captured CUDA graph; ``state_dict`` / ``load_state_dict`` checkpoint and
  resume the optics and the Adam state.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

from . import binding as B

# parameter order of the gradient and of the Adam state
PARAMS = ("defocus_um", "tilt_x", "tilt_y", "na_ill")
_COLUMN = {"defocus_um": 8, "tilt_x": 6, "tilt_y": 7, "na_ill": 5}  # wo_optics field index


class TuningProblem:
    """``params``: "defocus" (the defocus alone) or "all" (defocus, tilt_x,
    tilt_y, NA_ill; the smooth-edged source pupil, per-plane banks).
    ``planes`` (defocus only; default): per-plane TF banks and 2D data
    spectra, so no z transform runs per step; otherwise 3D banks and spectra
    (the same loss by Parseval over z).  ``smooth``: the smooth source pupil
    for the defocus-only bank too.  ``loss``: the data-fidelity loss (default)
    or the paper's mid-band power loss (WO_LOSS_MIDBAND)."""

    def __init__(self, data: torch.Tensor, optics_list, eta: float, background=None, planes: bool = True,
                 loss: int = B.WO_LOSS_DATA, params: str = "defocus", smooth: bool = False):
        if data.dim() != 4 or data.dtype != torch.float32 or not data.is_cuda:
            raise ValueError("data: float32 CUDA tensor [n_tiles, Z, Y, X]")
        if params not in ("defocus", "all"):
            raise ValueError("params: 'defocus' or 'all'")
        self.n, self.Z, self.Y, self.X = (int(s) for s in data.shape)
        if len(optics_list) != self.n:
            raise ValueError("one optics entry per tile")
        dev = data.device
        self.eta = float(eta)
        self.loss = int(loss)
        self.n_params = 1 if params == "defocus" else 4
        if self.n_params == 4:
            self.kinds = B.WO_TF_PHASE_GRAD | B.WO_TF_PLANES
            planes = True
        else:
            self.kinds = B.WO_TF_PHASE_DZ | (B.WO_TF_PLANES if planes else 0) | (B.WO_TF_SMOOTH_SOURCE if smooth else 0)
        self.mode = B.WO_MODE_2D if planes else B.WO_MODE_3D
        self.optics = B.optics_tensor(optics_list, dev)
        self.optics0 = self.optics.clone()
        self.tf, self.ws = B.alloc(self.n, self.Z, self.Y, self.X, self.kinds, dev)
        self.spec = torch.empty((self.n, self.Z, self.Y, self.X // 2 + 1), dtype=torch.complex64, device=dev)
        self.background = background
        self.set_data(data)
        self.value = torch.zeros(self.n, dtype=torch.float64, device=dev)
        self.grad = torch.zeros((self.n, self.n_params), dtype=torch.float64, device=dev)
        self.state = torch.zeros((self.n, self.n_params, 3), dtype=torch.float64, device=dev)
        self._graphs = {}  # schedule -> captured CUDA graph

    def set_data(self, data: torch.Tensor):
        """New stacks for the same tiles (the spectra are recomputed)."""
        B.wo_spectrum(data.contiguous(), self.background, self.mode, self.spec, self.n, self.Z, self.Y, self.X)

    @property
    def defocus(self) -> torch.Tensor:
        return self.optics[:, 8]

    def params(self) -> torch.Tensor:
        """The tuned parameters [n, n_params] (a copy)."""
        return torch.stack([self.optics[:, _COLUMN[k]] for k in PARAMS[: self.n_params]], dim=1)

    def set_params(self, p: torch.Tensor):
        for i, k in enumerate(PARAMS[: self.n_params]):
            self.optics[:, _COLUMN[k]].copy_(p[:, i])

    def restart(self, optics_list):
        """New starting optics for the same tiles (e.g. an estimator's output)."""
        self.optics0.copy_(B.optics_tensor(optics_list, self.optics.device))
        self.reset()

    def reset(self):
        """Back to the starting optics, Adam state cleared."""
        self.optics.copy_(self.optics0)
        self.state.zero_()

    def state_dict(self) -> dict:
        """Checkpoint of the tuning state as host arrays: the current and the
        starting optics (float64 [n, 9], wo_optics field order) and the Adam
        state (float64 [n, n_params, 3]: m, v and the step count per
        parameter).  Take it between calls of ``run``: a schedule runs to its
        end within one call (one graph replay), so a checkpoint holds the
        state after whole schedules; split a long schedule into its phases to
        checkpoint between them."""
        return {"optics": self.optics.cpu().numpy().copy(), "optics0": self.optics0.cpu().numpy().copy(),
                "adam": self.state.cpu().numpy().copy()}

    def load_state_dict(self, sd: dict):
        """Resume from a ``state_dict`` of a problem over the same tiles and
        parameters.  The arrays are copied into the existing device buffers,
        so graphs captured by ``run`` stay valid and continue from there."""
        for name, t in (("optics", self.optics), ("optics0", self.optics0), ("adam", self.state)):
            a = torch.as_tensor(sd[name], dtype=t.dtype)
            if tuple(a.shape) != tuple(t.shape):
                raise ValueError(f"{name}: shape {tuple(a.shape)}, expected {tuple(t.shape)}")
            t.copy_(a)

    def evaluate(self, nu_max: float = 0.0):
        """Loss and gradient of every tile at the current optics."""
        n, Z, Y, X = self.n, self.Z, self.Y, self.X
        B.wo_build_tf_device(self.optics, n, Z, Y, X, self.kinds, self.tf, self.ws)
        B.wo_tune_objective(self.tf, self.kinds, self.optics, self.spec, self.loss, self.eta, nu_max, self.value,
                            self.grad, n, Z, Y, X, self.ws)

    def step(self, lr, nu_max: float = 0.0, beta1=0.9, beta2=0.999, eps=1e-8):
        self.evaluate(nu_max)
        B.wo_adam_optics(self.optics, self.grad, self.n_params, self.state, self.n, lr, beta1, beta2, eps)

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
        continues from wherever the optics stand.  Graphs are kept per
        schedule and stay valid across ``set_data`` and ``restart``, which
        only rewrite the problem's buffers.
        """
        key = tuple(schedule)
        if not graph:
            self._queue(key)
            return
        if key not in self._graphs:
            saved_o, saved_s = self.optics.clone(), self.state.clone()
            self._queue(key[:1])  # first launch of every kernel, outside the capture
            torch.cuda.synchronize()
            self.optics.copy_(saved_o)
            self.state.copy_(saved_s)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g):
                self._queue(key)
            self._graphs[key] = g
        self._graphs[key].replay()


@dataclass(frozen=True)
class Phase:
    """``steps`` Adam steps on the loss restricted to |nu| <= nu_max (0: the
    full loss), the step size going from lr_start to lr_end along half a
    cosine; a step size is one number (every parameter) or a tuple with one
    per tuned parameter.  ``reset`` clears the Adam moments first (a new
    loss)."""
    steps: int
    lr_start: float | tuple
    lr_end: float | tuple
    nu_max: float = 0.0
    reset: bool = False

    def lr_at(self, i: int):
        w = 1.0 if self.steps <= 1 else 0.5 * (1.0 + math.cos(math.pi * i / self.steps))
        if isinstance(self.lr_start, tuple):
            return [e + (s - e) * w for s, e in zip(self.lr_start, self.lr_end)]
        return self.lr_end + (self.lr_start - self.lr_end) * w


def default_schedule(o) -> tuple:
    """50 Adam steps from a nominal defocus: 25 on the loss band-limited to
    |nu| <= 0.12 NA_det/lambda (a wide basin; lr 0.08 -> 0.02 um), then 25 on
    the full loss with fresh moments (lr 0.02 -> 0 um)."""
    nu = 0.12 * o["na_det"] / o["lambda_um"]
    return (Phase(25, 0.08, 0.02, nu), Phase(25, 0.02, 0.0, 0.0, reset=True))


def default_schedule4(o) -> tuple:
    """50 Adam steps on (defocus, tilt_x, tilt_y, NA_ill) from nominal: 25 on
    the band-limited loss (lr 0.08 -> 0.02 um for the defocus, 0.01 -> 0.003
    NA for the illumination), then 25 on the full loss with fresh moments
    (0.02 -> 0 um, 0.005 -> 0 NA)."""
    nu = 0.12 * o["na_det"] / o["lambda_um"]
    return (Phase(25, (0.08, 0.01, 0.01, 0.01), (0.02, 0.003, 0.003, 0.003), nu),
            Phase(25, (0.02, 0.005, 0.005, 0.005), (0.0, 0.0, 0.0, 0.0), 0.0, reset=True))


def refine_schedule(steps: int = 10) -> tuple:
    """A short run on the full loss from a good starting point (an
    estimator's output): lr 0.01 -> 0 um for the defocus, 0.002 -> 0 NA for
    the illumination."""
    return (Phase(steps, (0.01, 0.002, 0.002, 0.002), (0.0, 0.0, 0.0, 0.0), 0.0),)


class TuneLoss(torch.autograd.Function):
    """loss[t] = L_t(theta[t]) with dL/dtheta from the library's adjoint;
    theta [n, n_params] in the order of PARAMS."""

    @staticmethod
    def forward(ctx, theta: torch.Tensor, problem: TuningProblem, nu_max: float = 0.0):
        problem.set_params(theta.detach().reshape(problem.n, problem.n_params))
        problem.evaluate(nu_max)
        ctx.save_for_backward(problem.grad.clone())
        return problem.value.clone()

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out[:, None] * g, None, None


def tune_loss(theta: torch.Tensor, problem: TuningProblem, nu_max: float = 0.0) -> torch.Tensor:
    return TuneLoss.apply(theta, problem, nu_max)


class Reconstruction:
    """The phase reconstruction of a batch of stacks as a differentiable
    function of each tile's tuned optics (Ext. Data Fig. 3: a loss of the
    reconstruction is back-propagated to the parameters).

    ``mode``: B.WO_MODE_3D (the 3D reconstruction; ``params="defocus"``) or
    B.WO_MODE_2D (the thin-object reconstruction from the z-stack;
    ``params="defocus"`` or ``"all"`` = defocus, tilt_x, tilt_y, NA_ill under
    the smooth source pupil).  The regulariser ``eta`` is absolute; the
    background is each stack's mean.  ``forward(theta)`` builds the phase
    transfer function from the device optics and reconstructs (wo_reconstruct);
    ``vjp(grad_out)`` builds the derivative bank at the same optics and returns
    dL/dtheta for the upstream gradient dL/df (wo_reconstruct_vjp).
    ``ReconstructFn`` wraps both for autograd."""

    def __init__(self, data: torch.Tensor, optics_list, eta: float, mode: int = B.WO_MODE_3D,
                 params: str = "defocus"):
        if data.dim() != 4 or data.dtype != torch.float32 or not data.is_cuda:
            raise ValueError("data: float32 CUDA tensor [n_tiles, Z, Y, X]")
        if params not in ("defocus", "all") or (mode == B.WO_MODE_3D and params != "defocus"):
            raise ValueError("params: 'defocus' (3D or 2D) or 'all' (2D)")
        self.n, self.Z, self.Y, self.X = (int(s) for s in data.shape)
        if len(optics_list) != self.n:
            raise ValueError("one optics entry per tile")
        dev = data.device
        self.data = data.contiguous()
        self.eta, self.mode = float(eta), int(mode)
        self.n_params = 1 if params == "defocus" else 4
        smooth = B.WO_TF_SMOOTH_SOURCE if self.n_params == 4 else 0
        self.kinds_fwd = (B.WO_TF_PHASE_DZ if mode == B.WO_MODE_3D else B.WO_TF_PHASE) | smooth
        if mode == B.WO_MODE_3D:
            self.kinds_vjp = B.WO_TF_PHASE_DZ
        else:
            self.kinds_vjp = (B.WO_TF_PHASE_GRAD if self.n_params == 4 else B.WO_TF_PHASE_DZ) | B.WO_TF_PLANES
        self.optics = B.optics_tensor(optics_list, dev)
        n, Z, Y, X = self.n, self.Z, self.Y, self.X
        self.tf_fwd, ws1 = B.alloc(n, Z, Y, X, self.kinds_fwd, dev)
        self.tf_vjp, ws2 = B.alloc(n, Z, Y, X, self.kinds_vjp, dev)
        self.ws = ws1 if ws1.numel() >= ws2.numel() else ws2
        self.spec = torch.empty((n, Z, Y, X // 2 + 1), dtype=torch.complex64, device=dev)
        B.wo_spectrum(self.data, None, self.mode, self.spec, n, Z, Y, X)
        shape = (n, Z, Y, X) if mode == B.WO_MODE_3D else (n, Y, X)
        self.out = torch.empty(shape, dtype=torch.float32, device=dev)
        self.grad = torch.zeros((n, self.n_params), dtype=torch.float64, device=dev)

    def set_params(self, theta: torch.Tensor):
        for i, k in enumerate(PARAMS[: self.n_params]):
            self.optics[:, _COLUMN[k]].copy_(theta[:, i])

    def forward(self, theta: torch.Tensor) -> torch.Tensor:
        n, Z, Y, X = self.n, self.Z, self.Y, self.X
        self.set_params(theta.detach().reshape(n, self.n_params).to(torch.float64))
        B.wo_build_tf_device(self.optics, n, Z, Y, X, self.kinds_fwd, self.tf_fwd, self.ws)
        B.wo_reconstruct(self.tf_fwd, self.kinds_fwd, self.data, None, [self.eta], B.WO_ETA_ABSOLUTE, self.mode,
                         self.out, n, Z, Y, X, self.ws)
        return self.out.clone()

    def vjp(self, grad_out: torch.Tensor) -> torch.Tensor:
        n, Z, Y, X = self.n, self.Z, self.Y, self.X
        g = grad_out.detach().to(torch.float32).contiguous()
        B.wo_build_tf_device(self.optics, n, Z, Y, X, self.kinds_vjp, self.tf_vjp, self.ws)
        B.wo_reconstruct_vjp(self.tf_vjp, self.kinds_vjp, self.spec, g, self.eta, self.mode, self.grad, n, Z, Y, X,
                             self.ws)
        return self.grad.clone()


class ReconstructFn(torch.autograd.Function):
    """f = R(theta) for a ``Reconstruction``: theta [n, n_params] (float64, in
    the order of PARAMS) -> the reconstructed phase [n, Z, Y, X] (3D) or
    [n, Y, X] (2D); backward returns the library's vector-Jacobian product."""

    @staticmethod
    def forward(ctx, theta: torch.Tensor, problem: Reconstruction):
        ctx.problem = problem
        ctx.save_for_backward(theta.detach().clone())
        return problem.forward(theta)

    @staticmethod
    def backward(ctx, grad_out):
        (theta,) = ctx.saved_tensors
        p = ctx.problem
        p.set_params(theta.reshape(p.n, p.n_params).to(torch.float64))  # the optics this output was made at
        return p.vjp(grad_out).to(theta.dtype), None


def reconstruct(theta: torch.Tensor, problem: Reconstruction) -> torch.Tensor:
    return ReconstructFn.apply(theta, problem)
