"""Defocus auto-tuning on the GPU against the float64 oracle.

The TF pair bank (phase TF and its defocus derivative), the data spectra, the
per-tile loss and its hand-written adjoint gradient are compared with the
oracle (oracle/tuning.py); the gradient is also checked against central
differences of the GPU loss (step 1e-3 um), and the on-device Adam loop must
bring every tile to within 0.05 um of its true defocus.  Data are thin
specimens imaged by the oracle's 2D model at each tile's true defocus.
"""
import numpy as np
import pytest

import phantom as ph
from conftest import rel_l2
from oracle import model as OM, optics as OO, tuning as OT

pytestmark = pytest.mark.gpu

SHAPE = (48, 128, 128)  # tiles of 48 planes of 128 x 128
SHAPE192 = (48, 192, 192)  # the shift-variant field's tiles (128-px cores with 32-px halos)


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2412_09775_gb300.build import build
    build()
    from paper_2412_09775_gb300 import autotune, binding
    return binding, autotune, torch, torch.device("cuda:0")


def thin_stack(o_true, shape, seed, noise=1e-3):
    """Brightfield stack of a thin specimen at o_true's defocus (oracle 2D model)."""
    Z, Y, X = shape
    f2 = ph.thin_phantom(seed, (Y, X), o_true, n_spheres=20)
    Hj = OO.plane_tfs(o_true, shape, ("phase",))["phase"]
    d = 1.0 + np.real(np.fft.ifft2(Hj * np.fft.fft2(f2)[None], axes=(1, 2)))
    return d + ph.gaussian_noise(seed + 1000, shape, noise)


def tiles(n, seed):
    rng = np.random.default_rng(seed)
    return ph.tile_optics(rng, n)


def nominal(o):
    return dict(o, defocus_um=0.0)


# ------------------------------------------------------------ TF pair
@pytest.mark.parametrize("planes", [False, True])
@pytest.mark.parametrize("shape", [(8, 32, 48), (12, 64, 64), (6, 24, 96)])
def test_phase_dz_bank_matches_oracle(env, shape, planes):
    B, _, torch, dev = env
    Z, Y, X = shape
    ol = [ph.optics(defocus_um=0.4, na_ill=0.6), ph.optics(defocus_um=-0.7, tilt_x=0.05, tilt_y=-0.08, na_ill=0.8),
          ph.optics(defocus_um=0.0, na_ill=0.9)]
    n = len(ol)
    kinds = B.WO_TF_PHASE_DZ | (B.WO_TF_PLANES if planes else 0)
    tf, ws = B.alloc(n, Z, Y, X, kinds, dev)
    B.wo_build_tf(ol, n, Z, Y, X, kinds, tf, ws)
    torch.cuda.synchronize()
    spec, stats = B.tf_views(tf, n, Z, Y, X, kinds)
    spec, stats = spec.cpu().numpy(), stats.cpu().numpy()
    for t, o in enumerate(ol):
        if planes:  # per-plane 2D TFs, no z-DFT
            H = OO.plane_tfs(o, shape, ("phase",))["phase"]
            dH = OT.plane_tf_defocus_derivative(o, shape)
        else:
            H = OO.transfer_functions(o, shape, ("phase",))["phase"]
            dH = OT.tf_defocus_derivative(o, shape)
        assert rel_l2(spec[t, 0], OO.half_spectrum(H)) <= 1e-4, t
        assert rel_l2(spec[t, 1], OO.half_spectrum(dH)) <= 1e-4, t
        if not planes:
            assert abs(stats[t, 0] / np.max(np.abs(H) ** 2) - 1) <= 1e-5


def test_phase_dz_bank_reconstructs_like_a_phase_bank(env):
    B, _, torch, dev = env
    Z, Y, X = 16, 64, 64
    o = ph.optics(defocus_um=0.3, na_ill=0.7)
    d = torch.tensor(1.0 + 0.01 * ph.uniform_volume(5, (Z, Y, X)), dtype=torch.float32, device=dev)
    outs, tfs = [], []
    for kinds in ("phase", "phase_dz"):
        tf, ws = B.alloc(1, Z, Y, X, kinds, dev)
        B.wo_build_tf([o], 1, Z, Y, X, kinds, tf, ws)
        f = torch.empty((Z, Y, X), dtype=torch.float32, device=dev)
        B.wo_reconstruct(tf, kinds, d, None, 1e-3, B.WO_ETA_RELATIVE, B.WO_MODE_3D, f, 1, Z, Y, X, ws)
        outs.append(f.cpu().numpy())
        tfs.append(B.tf_views(tf, 1, Z, Y, X, kinds)[0][0, 0].cpu().numpy())
    # the same phase TF up to float32 rounding (the derivative bank transforms
    # Re g and Re g' as one complex row, the phase bank transforms g) ...
    assert rel_l2(tfs[1], tfs[0]) <= 2e-6
    # ... and the same reconstruction within the parity bar
    assert rel_l2(outs[1], outs[0]) <= 1e-4


# ------------------------------------------------------------ spectra
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("bg", [None, 0.97])
def test_spectrum_matches_oracle(env, bg, mode):
    """3D spectra (DC: D(0) - N b) and per-plane 2D spectra (every plane's DC:
    D_j(0) - N_perp b), b given or the stack mean."""
    B, _, torch, dev = env
    n, Z, Y, X = 2, 12, 48, 64
    d = 1.0 + 0.05 * ph.uniform_volume(7, (n, Z, Y, X))
    spec = torch.empty((n, Z, Y, X // 2 + 1), dtype=torch.complex64, device=dev)
    B.wo_spectrum(torch.tensor(d, dtype=torch.float32, device=dev), None if bg is None else [bg], mode, spec,
                  n, Z, Y, X)
    got = spec.cpu().numpy()
    for t in range(n):
        if mode == 0:
            want = OM.residual_spectrum(d[t], bg, (0, 1, 2))
        else:
            b = float(np.mean(d[t])) if bg is None else bg
            want = OM.residual_spectrum(d[t], b, (1, 2))
        assert rel_l2(got[t], want[..., : X // 2 + 1]) <= 1e-5


# ------------------------------------------------------------ loss and adjoint
def problem(env, ol_true, start, eta, seed=11, planes=True):
    B, A, torch, dev = env
    d = np.stack([thin_stack(o, SHAPE, seed + 17 * t) for t, o in enumerate(ol_true)])
    data = torch.tensor(d, dtype=torch.float32, device=dev)
    return A.TuningProblem(data, start, eta, planes=planes), d


def cutoff(o):
    return o["na_det"] / o["lambda_um"]


@pytest.mark.parametrize("planes", [True, False])
@pytest.mark.parametrize("band", [None, 0.3])
def test_loss_and_gradient_match_the_oracle_on_eight_tiles(env, band, planes):
    """Value within 1e-4 and adjoint gradient within 1e-3 (relative) of the
    float64 oracle's loss and its central-difference derivative, from
    per-plane and from 3D banks."""
    B, A, torch, dev = env
    ol = tiles(8, 21)
    offs = np.array([0.2, -0.15, 0.12, -0.18, 0.1, -0.2, 0.16, -0.1])
    start = [dict(o, defocus_um=o["defocus_um"] + s) for o, s in zip(ol, offs)]
    eta = 1e-3
    pb, d = problem(env, ol, start, eta, planes=planes)
    nu = 0.0 if band is None else band * cutoff(ol[0]) + 1e-3  # off the frequency grid
    pb.evaluate(nu)
    torch.cuda.synchronize()
    val, grad = pb.value.cpu().numpy(), pb.grad[:, 0].cpu().numpy()
    for t in range(8):
        nm = None if band is None else nu
        want = OT.objective(start[t], d[t], eta, nm)
        gwant = OT.gradient_fd(start[t], d[t], eta, h=1e-4, nu_max=nm)
        assert abs(val[t] - want) <= 1e-4 * abs(want), (t, val[t], want)
        assert abs(grad[t] - gwant) <= 1e-3 * abs(gwant), (t, grad[t], gwant)


@pytest.mark.parametrize("planes", [True, False])
def test_midband_loss_and_gradient_match_the_oracle(env, planes):
    """The paper's mid-band power loss and its derivative through the solve."""
    B, A, torch, dev = env
    ol = tiles(6, 31)
    offs = np.array([0.2, -0.15, 0.12, -0.18, 0.1, -0.2])
    start = [dict(o, defocus_um=o["defocus_um"] + s) for o, s in zip(ol, offs)]
    eta = 1e-3
    _, d = problem(env, ol, start, eta, seed=90)
    data = torch.tensor(d, dtype=torch.float32, device=dev)
    pb = A.TuningProblem(data, start, eta, planes=planes, loss=B.WO_LOSS_MIDBAND)
    pb.evaluate()
    torch.cuda.synchronize()
    val, grad = pb.value.cpu().numpy(), pb.grad[:, 0].cpu().numpy()
    for t in range(len(ol)):
        want = OT.midband_objective(start[t], d[t], eta)
        gwant = OT.midband_gradient_fd(start[t], d[t], eta, h=1e-4)
        assert abs(val[t] - want) <= 1e-4 * abs(want), (t, val[t], want)
        assert abs(grad[t] - gwant) <= 1e-3 * abs(gwant), (t, grad[t], gwant)


def test_gradient_matches_central_difference_of_the_gpu_loss(env):
    B, A, torch, dev = env
    ol = tiles(8, 22)
    start = [dict(o, defocus_um=o["defocus_um"] + (0.2 if t % 2 else -0.25)) for t, o in enumerate(ol)]
    pb, _ = problem(env, ol, start, 1e-3, seed=40)
    pb.evaluate()
    g = pb.grad[:, 0].clone()
    h = 1e-3
    z0 = pb.defocus.clone()
    vals = []
    for s in (+1, -1):
        pb.optics[:, 8] = z0 + s * h
        pb.evaluate()
        vals.append(pb.value.clone())
    fd = ((vals[0] - vals[1]) / (2 * h)).cpu().numpy()
    g = g.cpu().numpy()
    assert np.all(np.abs(g - fd) <= 1e-3 * np.abs(fd)), (g, fd)


def test_autograd_function_returns_the_adjoint_gradient(env):
    B, A, torch, dev = env
    ol = tiles(4, 23)
    start = [dict(o, defocus_um=o["defocus_um"] - 0.2) for o in ol]
    pb, d = problem(env, ol, start, 1e-3, seed=60)
    z = torch.tensor([[o["defocus_um"]] for o in start], dtype=torch.float64, device=dev, requires_grad=True)
    w = torch.tensor([1.0, -2.0, 0.5, 3.0], dtype=torch.float64, device=dev)
    loss = (A.tune_loss(z, pb) * w).sum()
    loss.backward()
    pb.evaluate()
    assert torch.allclose(z.grad, w[:, None] * pb.grad, rtol=0, atol=0)
    want = sum(float(w[t]) * OT.objective(start[t], d[t], 1e-3) for t in range(4))
    assert abs(float(loss.detach()) - want) <= 1e-4 * abs(want)


def test_adam_reaches_the_true_defocus_under_a_cuda_graph(env):
    """50 Adam steps from nominal (defocus 0): 25 on the band-limited loss
    (|nu| <= 0.12 of the detection cutoff, lr 0.08 -> 0.02 um), then with
    fresh moments 25 on the full loss (lr 0.02 -> 0 um); every tile ends
    within 0.05 um of its true defocus, and the graph replay gives the same
    result, bit for bit, as the eager loop."""
    B, A, torch, dev = env
    ol = tiles(8, 24)
    truth = np.array([o["defocus_um"] for o in ol])
    pb, _ = problem(env, ol, [nominal(o) for o in ol], 1e-3, seed=80)
    schedule = A.default_schedule(ol[0])
    assert sum(p.steps for p in schedule) == 50
    pb.run(schedule, graph=True)
    torch.cuda.synchronize()
    z_graph = pb.defocus.cpu().numpy().copy()
    assert np.all(np.abs(z_graph - truth) <= 0.05), (z_graph, truth)
    pb.reset()
    pb.run(schedule, graph=False)
    torch.cuda.synchronize()
    assert np.array_equal(pb.defocus.cpu().numpy(), z_graph)
    # a second replay continues from where the first ended (state on the device)
    pb.reset()
    pb.run(schedule, graph=True)
    torch.cuda.synchronize()
    assert np.array_equal(pb.defocus.cpu().numpy(), z_graph)


# ------------------------------------------------ smooth source, four parameters
def smooth_tiles(n, seed):
    return [dict(o, smooth_source=True) for o in tiles(n, seed)]


def test_smooth_source_bank_matches_oracle(env):
    B, _, torch, dev = env
    shape = (8, 32, 48)
    Z, Y, X = shape
    ol = smooth_tiles(3, 41)
    kinds = B.WO_TF_PHASE | B.WO_TF_ABSORPTION | B.WO_TF_SMOOTH_SOURCE
    tf, ws = B.alloc(3, Z, Y, X, kinds, dev)
    B.wo_build_tf(ol, 3, Z, Y, X, kinds, tf, ws)
    spec = B.tf_views(tf, 3, Z, Y, X, kinds)[0].cpu().numpy()
    for t, o in enumerate(ol):
        ref = OO.transfer_functions(o, shape, ("phase", "absorption"))
        den = np.sqrt(sum(np.linalg.norm(OO.half_spectrum(ref[k])) ** 2 for k in ref))
        for s_, k in enumerate(("phase", "absorption")):
            assert np.linalg.norm(spec[t, s_] - OO.half_spectrum(ref[k])) / den <= 1e-4, (t, k)


@pytest.mark.parametrize("shape", [(8, 32, 48), (6, 64, 64), (4, 24, 128), (6, 48, 96), (4, 24, 192), (3, 192, 192)])
def test_gradient_bank_matches_oracle(env, shape):
    """The five per-plane slots: H, dH/d(defocus, tilt_x, tilt_y, NA_ill)."""
    B, _, torch, dev = env
    Z, Y, X = shape
    ol = smooth_tiles(3, 42)
    kinds = B.WO_TF_PHASE_GRAD | B.WO_TF_PLANES
    tf, ws = B.alloc(3, Z, Y, X, kinds, dev)
    B.wo_build_tf(ol, 3, Z, Y, X, kinds, tf, ws)
    spec = B.tf_views(tf, 3, Z, Y, X, kinds)[0].cpu().numpy()
    for t, o in enumerate(ol):
        refs = [OO.plane_tfs(o, shape, ("phase",))["phase"], OT.plane_tf_defocus_derivative(o, shape)]
        src = OT.plane_tf_source_derivatives(o, shape)
        refs += [src["tilt_x"], src["tilt_y"], src["na_ill"]]
        for q, ref in enumerate(refs):
            assert rel_l2(spec[t, q], OO.half_spectrum(ref)) <= 1e-4, (t, q)


def assert_gradient(grad, gwant, what):
    """Every component of the adjoint gradient within 1e-3 of the oracle's
    central difference, relative to that component (no absolute slack)."""
    err = np.abs(np.asarray(grad) - gwant) / np.abs(gwant)
    assert np.all(err <= 1e-3), (what, grad, gwant, err)


@pytest.mark.parametrize("shape", [SHAPE, SHAPE192])
@pytest.mark.parametrize("loss", [0, 1])
def test_four_parameter_gradient_matches_oracle(env, loss, shape):
    """Loss and its gradient in (defocus, tilt_x, tilt_y, NA_ill) against the
    oracle's loss and central differences, data from the smooth-source model."""
    B, A, torch, dev = env
    ol = smooth_tiles(4, 43)
    offs = [(0.15, 0.02, -0.03, 0.05), (-0.12, -0.04, 0.02, -0.06), (0.1, 0.03, 0.03, 0.04),
            (-0.18, -0.02, -0.04, -0.05)]
    start = [dict(o, defocus_um=o["defocus_um"] + a, tilt_x=o["tilt_x"] + b, tilt_y=o["tilt_y"] + c,
                  na_ill=o["na_ill"] + e) for o, (a, b, c, e) in zip(ol, offs)]
    eta = 1e-3
    d = np.stack([thin_stack(o, shape, 70 + 17 * t) for t, o in enumerate(ol)])
    data = torch.tensor(d, dtype=torch.float32, device=dev)
    pb = A.TuningProblem(data, start, eta, params="all", loss=loss)
    pb.evaluate()
    torch.cuda.synchronize()
    val, grad = pb.value.cpu().numpy(), pb.grad.cpu().numpy()
    name = "data" if loss == 0 else "midband"
    for t in range(len(ol)):
        want = (OT.objective if loss == 0 else OT.midband_objective)(start[t], d[t], eta)
        gwant = OT.gradient_fd_params(start[t], d[t], eta, h=1e-4, loss=name)
        assert abs(val[t] - want) <= 1e-4 * abs(want), (t, val[t], want)
        assert_gradient(grad[t], gwant, t)


@pytest.mark.parametrize("shape", [SHAPE, SHAPE192])
def test_four_parameter_adam_from_nominal_under_a_cuda_graph(env, shape):
    """50 Adam steps on (defocus, tilt_x, tilt_y, NA_ill) from defocus 0, no
    tilt and NA_ill 0.825: every tile within 0.05 um in defocus and 0.01 NA in
    tilt and NA_ill of its true optics (smooth-source data)."""
    B, A, torch, dev = env
    ol = smooth_tiles(8, 24)
    d = np.stack([thin_stack(o, shape, 80 + 17 * t) for t, o in enumerate(ol)])
    data = torch.tensor(d, dtype=torch.float32, device=dev)
    truth = np.array([[o["defocus_um"], o["tilt_x"], o["tilt_y"], o["na_ill"]] for o in ol])
    start = [dict(o, defocus_um=0.0, tilt_x=0.0, tilt_y=0.0, na_ill=0.825) for o in ol]
    pb = A.TuningProblem(data, start, 1e-3, params="all")
    pb.run(A.default_schedule4(ol[0]), graph=True)
    err = np.abs(pb.params().cpu().numpy() - truth)
    assert np.all(err[:, 0] <= 0.05) and np.all(err[:, 1:] <= 0.01), err


def test_checkpoint_between_runs_resumes_exactly(env):
    """A run split by a checkpoint (state_dict after the first phase, a fresh
    problem over the same tiles loading it, the second phase there) ends on
    the same optics as the run in one problem, bit for bit; the first phase
    and the second each run as their own captured graph in both."""
    B, A, torch, dev = env
    shape = (16, 64, 64)
    ol = smooth_tiles(4, 31)
    d = np.stack([thin_stack(o, shape, 90 + 5 * t) for t, o in enumerate(ol)])
    data = torch.tensor(d, dtype=torch.float32, device=dev)
    start = [dict(o, defocus_um=0.0, tilt_x=0.0, tilt_y=0.0, na_ill=0.825) for o in ol]
    first, second = A.default_schedule4(ol[0])
    whole = A.TuningProblem(data, start, 1e-3, params="all")
    whole.run((first,), graph=True)
    whole.run((second,), graph=True)
    part = A.TuningProblem(data, start, 1e-3, params="all")
    part.run((first,), graph=True)
    sd = part.state_dict()
    resumed = A.TuningProblem(data, start, 1e-3, params="all")
    resumed.load_state_dict(sd)
    resumed.run((second,), graph=True)
    assert np.array_equal(resumed.params().cpu().numpy(), whole.params().cpu().numpy())
    assert np.array_equal(resumed.state_dict()["adam"], whole.state_dict()["adam"])


@pytest.mark.parametrize("shape", [SHAPE, SHAPE192])
def test_four_parameter_gradient_full_batch(env, shape):
    """The auto-tuning workload's launch configuration: 256 tiles of
    48 x 192 x 192 (the shift-variant field's tiles; also 48 x 128 x 128) with
    their own optics in one batch (per-plane gradient bank, smooth source,
    data-fidelity loss).  Loss and gradient of two sampled tiles (the first
    and the last) against the oracle's loss and its central differences."""
    B, A, torch, dev = env
    n = 256
    ol = [dict(o, smooth_source=True) for o in tiles(n, 77)]
    start = [dict(o, defocus_um=0.0, tilt_x=0.0, tilt_y=0.0, na_ill=0.825) for o in ol]
    eta = 1e-3
    d = (1.0 + ph.uniform_volume(78, (n,) + shape, -0.01, 0.01)).astype(np.float32)
    for t in (0, n - 1):  # physically consistent stacks where the oracle checks
        d[t] = thin_stack(ol[t], shape, 79 + t).astype(np.float32)
    pb = A.TuningProblem(torch.from_numpy(d).to(dev), start, eta, params="all")
    pb.evaluate()
    torch.cuda.synchronize()
    val, grad = pb.value.cpu().numpy(), pb.grad.cpu().numpy()
    assert np.all(np.isfinite(val)) and np.all(np.isfinite(grad))
    for t in (0, n - 1):
        dt = d[t].astype(np.float64)
        want = OT.objective(start[t], dt, eta)
        gwant = OT.gradient_fd_params(start[t], dt, eta, h=1e-4, loss="data")
        assert abs(val[t] - want) <= 1e-4 * abs(want), (t, val[t], want)
        assert_gradient(grad[t], gwant, t)
