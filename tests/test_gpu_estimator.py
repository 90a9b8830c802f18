"""The learned optics estimator on the GPU against the float64 reference
(oracle/estimator.py): features, the thin-specimen generator, the network's
forward pass, its gradient and the Adam step; then a short training run
that must learn the defocus from forward-simulated tiles."""
import numpy as np
import pytest

import phantom as ph
from conftest import rel_l2
from oracle import estimator as OE, optics as OO

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2412_09775_gb300.build import build
    build()
    from paper_2412_09775_gb300 import binding, estimator
    return binding, estimator, torch, torch.device("cuda:0")


def test_thin_phantom_kernel_matches_reference(env):
    B, E, torch, dev = env
    o = ph.optics()
    Y, X = 48, 64
    pars = [ph.thin_sphere_params(s, (Y, X), o, n_spheres=12) for s in (1, 2, 3)]
    p = torch.tensor(np.stack(pars), dtype=torch.float32, device=dev)
    out = torch.empty((3, Y, X), dtype=torch.float32, device=dev)
    B.wo_thin_phantom(p, 3, 12, Y, X, o["pixel_um"], o["z_step_um"], out)
    got = out.cpu().numpy()
    for t in range(3):
        want = ph.thin_phantom_from_params(np.stack(pars)[t].astype(np.float32).astype(np.float64), (Y, X), o)
        assert np.abs(got[t] - want).max() <= 1e-4 * np.abs(want).max()


@pytest.mark.parametrize("shape", [(16, 64, 64), (48, 128, 128)])
def test_features_match_reference(env, shape):
    B, E, torch, dev = env
    Z, Y, X = shape
    rng = np.random.default_rng(4)
    ol = [dict(o, smooth_source=True) for o in ph.tile_optics(rng, 2)]
    d = np.stack([1 + 0.01 * ph.uniform_volume(10 + t, shape) for t in range(2)]).astype(np.float32)
    data = torch.tensor(d, device=dev)
    spec = torch.empty((2, Z, Y, X // 2 + 1), dtype=torch.complex64, device=dev)
    B.wo_spectrum(data, None, B.WO_MODE_2D, spec, 2, Z, Y, X)
    feat = torch.empty((2, 3, 64, 64), dtype=torch.float32, device=dev)
    B.wo_est_features(spec, B.optics_tensor(ol, dev), 2, Z, Y, X, feat)
    got = feat.cpu().numpy()
    for t in range(2):
        want = OE.tile_features(d[t].astype(np.float64), ol[t])
        assert np.abs(got[t, 0] - want[0]).max() <= 1e-4 * max(1.0, np.abs(want[0]).max())
        assert np.abs(got[t, 1:] - want[1:]).max() <= 1e-3


def random_net(env, seed=3):
    B, E, torch, dev = env
    est = E.Estimator(dev, seed=seed, batch=4)
    flat = est.w32.cpu().numpy().astype(np.float64)
    # nonzero biases, so that they are tested too
    rng = np.random.default_rng(seed)
    flat += np.where(np.abs(flat) == 0, rng.normal(0, 0.05, flat.size), 0.0)
    est.w32.copy_(torch.tensor(flat, dtype=torch.float32))
    B.wo_est_sync_bf16(est.w32, est.wbf)
    return est, est.w32.cpu().numpy().astype(np.float64)


def test_network_forward_matches_reference(env):
    B, E, torch, dev = env
    est, flat = random_net(env)
    x = np.random.default_rng(5).normal(size=(4, 3, 64, 64)).astype(np.float32)
    out = est.predict(torch.tensor(x, device=dev)).cpu().numpy()
    want, _ = OE.forward(flat, x.astype(np.float64))
    want = want * np.array(E.SCALE) + np.array(E.OFFSET)
    assert rel_l2(out, want) <= 1e-4


def test_network_gradient_and_adam_match_reference(env):
    B, E, torch, dev = env
    est, flat = random_net(env, seed=6)
    rng = np.random.default_rng(7)
    x = rng.normal(size=(4, 3, 64, 64)).astype(np.float32)
    phys = (np.array(E.OFFSET) + np.array(E.SCALE) * rng.normal(size=(4, 4))).astype(np.float32)
    t_std = (phys.astype(np.float64) - np.array(E.OFFSET)) / np.array(E.SCALE)
    grad = torch.empty(est.n, dtype=torch.float32, device=dev)
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    xd, td = torch.tensor(x, device=dev), torch.tensor(phys, device=dev)
    B.wo_est_backward(est.wbf, est.w32, xd, td, 4, E.SCALE, E.OFFSET, grad, loss, est.ws)
    # the ReLU decisions the kernels took in float32: a pre-activation within
    # float rounding of zero can go either way, and one such decision moves
    # the first layer's weight gradient by ~1e-3, so the reference
    # differentiates through the same decisions
    masks = []
    for layer, (ci, co, s) in enumerate(OE.LAYERS, start=1):
        side = 64 // (2 ** (layer - 1)) if layer > 1 else 64
        off = B.wo_est_activation_offset(4, layer)
        n_el = 4 * co * side * side
        act = est.ws[off: off + 4 * n_el].view(torch.float32).view(4, co, side, side)
        masks.append(act.cpu().numpy() > 0)
    L, g = OE.backward(flat, x.astype(np.float64), t_std, masks=masks)
    assert abs(float(loss.item()) - L) <= 1e-4 * L
    gg = grad.cpu().numpy()
    offs = np.cumsum([0] + [int(np.prod(s)) for s in OE.param_shapes()])
    for k in range(len(offs) - 1):
        a, b = gg[offs[k]:offs[k + 1]], g[offs[k]:offs[k + 1]]
        assert rel_l2(a, b) <= 1e-3, k
    # one Adam step from zero moments equals the reference update with the GPU's gradient
    w0 = est.w32.cpu().numpy().astype(np.float64)
    B.wo_est_train_step(est.w32, est.wbf, est.m, est.v, xd, td, 4, E.SCALE, E.OFFSET, 1, 1e-3, loss, est.ws)
    w1, _, _ = OE.adam(w0, gg.astype(np.float64), np.zeros_like(w0), np.zeros_like(w0), 1, 1e-3)
    assert np.abs(est.w32.cpu().numpy() - w1).max() <= 1e-6
    assert np.array_equal(est.wbf.cpu().numpy().view(np.uint16),
                          (OE.bf16(est.w32.cpu().numpy()).astype(np.float32).view(np.uint32) >> 16).astype(np.uint16))


def test_training_learns_the_defocus(env):
    """A short training run on forward-simulated 16 x 64 x 64 tiles brings the
    held-out defocus error far below the spread of the draws."""
    B, E, torch, dev = env
    base = ph.optics()
    shape = (16, 64, 64)
    feat, truth = E.generate(3072, shape, base, seed=1, device=dev)
    vf, vt = E.generate(512, shape, base, seed=2, device=dev)
    est = E.Estimator(dev, seed=0, batch=128)
    losses = est.train(feat, truth, epochs=8, lr=2e-3)
    assert losses[-1] < losses[0]
    pred = est.predict(vf).cpu().numpy()
    err = np.sqrt(np.mean((pred - vt.cpu().numpy()) ** 2, axis=0))
    assert err[0] <= 0.15, err   # defocus draws have a spread of 0.58 um
