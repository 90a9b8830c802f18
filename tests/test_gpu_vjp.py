"""The hand-written adjoint of the phase reconstruction with respect to the
optics (wo_reconstruct_vjp, autotune.ReconstructFn) against the float64
oracle: for a seeded random upstream gradient g (a specimen-like image),
dL/dtheta of L = <g, f(theta)> must match the oracle's central differences of
the same contraction (h = 1e-3) within 1e-3 relative, per parameter, on 8
tiles; the forward reconstruction must match the oracle's within 1e-4.
"""
import numpy as np
import pytest

import phantom as ph
from conftest import rel_l2
from oracle import model as OM, optics as OO

pytestmark = pytest.mark.gpu

KEYS = ("defocus_um", "tilt_x", "tilt_y", "na_ill")
ETA = 1e-3


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2412_09775_gb300.build import build
    build()
    from paper_2412_09775_gb300 import autotune, binding
    return binding, autotune, torch, torch.device("cuda:0")


def oracle_f(o, d, mode, smooth):
    o = dict(o, smooth_source=smooth)
    if mode == 0:
        modes, _, _ = OM.widefield_system(OO.transfer_functions(o, d.shape, ("phase",)), ("phase",))
        return OM.reconstruct(modes, d[None], ETA, relative=False)[0]
    modes, _, _ = OM.widefield_system(OO.plane_tfs(o, d.shape, ("phase",)), ("phase",))
    return OM.reconstruct_2d(modes, d[None], ETA, relative=False)[0]


def oracle_grad(o, d, g, mode, smooth, keys, h=1e-3):
    """Central differences of <g, f> at step h with one Richardson step (h and
    h/2: the h^2 term, up to 6e-4 of the derivative here, cancels)."""
    def L(oo):
        return float(np.sum(g * oracle_f(oo, d, mode, smooth)))
    out = []
    for k in keys:
        c = [(L(dict(o, **{k: o[k] + s})) - L(dict(o, **{k: o[k] - s}))) / (2 * s) for s in (h, h / 2)]
        out.append((4 * c[1] - c[0]) / 3)
    return np.array(out)


def stacks(o_list, shape, seed, smooth):
    out = []
    for t, o in enumerate(o_list):
        dn = ph.sphere_phantom(seed + t, shape, o, n_spheres=25)
        oo = dict(o, smooth_source=smooth)
        modes, _, _ = OM.widefield_system(OO.transfer_functions(oo, shape, ("phase",)), ("phase",))
        out.append(OM.forward(modes, dn[None], [1.0])[0] + ph.gaussian_noise(seed + 50 + t, shape, 1e-3))
    return np.stack(out).astype(np.float32)


CASES = [  # (mode, params, shape, tiles)
    (0, "defocus", (24, 64, 64), 8),
    (1, "defocus", (24, 64, 64), 8),
    (1, "all", (24, 64, 64), 8),
    (0, "defocus", (48, 128, 128), 2),
    (1, "all", (48, 192, 192), 2),
]


@pytest.mark.parametrize("mode,params,shape,n", CASES)
def test_reconstruction_vjp_matches_oracle_central_differences(env, mode, params, shape, n):
    B, A, torch, dev = env
    smooth = params == "all"
    truth = ph.tile_optics(np.random.default_rng(90 + n), n)
    d = stacks(truth, shape, 300, smooth)
    # the parameters the derivative is taken at: off the truth
    rng = np.random.default_rng(91)
    at = [dict(o, defocus_um=o["defocus_um"] + rng.uniform(-0.2, 0.2), tilt_x=o["tilt_x"] + rng.uniform(-0.03, 0.03),
               tilt_y=o["tilt_y"] + rng.uniform(-0.03, 0.03), na_ill=o["na_ill"] + rng.uniform(-0.05, 0.05))
          for o in truth]
    keys = KEYS[: 4 if smooth else 1]
    pb = A.Reconstruction(torch.from_numpy(d).to(dev), at, ETA, mode=mode, params=params)
    theta = torch.tensor([[o[k] for k in keys] for o in at], dtype=torch.float64, device=dev, requires_grad=True)
    f = A.reconstruct(theta, pb)
    # the upstream gradient: a seeded random specimen-like image per tile (a
    # sphere phantom).  Uniform white noise makes <g, df> a sum whose terms
    # cancel by factors of 10^2 - 10^3, below which the float32 TF bank's own
    # rounding (1e-4 relative) shows; image-like gradients, as a loss of the
    # reconstruction produces, cancel by factors of 2 - 30
    if mode == 0:
        g = np.stack([ph.sphere_phantom(500 + t, shape, at[t], n_spheres=25) for t in range(n)])
    else:
        g = np.stack([ph.thin_phantom(500 + t, shape[1:], at[t], n_spheres=20) for t in range(n)])
    g = g.astype(np.float32)
    loss = (f * torch.from_numpy(g).to(dev)).sum()
    loss.backward()
    grad = theta.grad.cpu().numpy()
    f_np = f.detach().cpu().numpy()
    for t in range(n):
        assert rel_l2(f_np[t], oracle_f(at[t], d[t].astype(np.float64), mode, smooth)) <= 1e-4, t
        want = oracle_grad(at[t], d[t].astype(np.float64), g[t].astype(np.float64), mode, smooth, keys)
        err = np.abs(grad[t] - want) / np.abs(want)
        assert np.all(err <= 1e-3), (t, grad[t], want, err)


def test_vjp_is_linear_in_the_upstream_gradient(env):
    """vjp(a g1 + b g2) = a vjp(g1) + b vjp(g2) (float rounding)."""
    B, A, torch, dev = env
    shape = (24, 64, 64)
    ol = ph.tile_optics(np.random.default_rng(93), 3)
    d = stacks(ol, shape, 400, True)
    pb = A.Reconstruction(torch.from_numpy(d).to(dev), ol, ETA, mode=1, params="all")
    theta = torch.tensor([[o[k] for k in KEYS] for o in ol], dtype=torch.float64, device=dev)
    pb.forward(theta)
    g1 = torch.randn((3,) + shape[1:], device=dev, generator=torch.Generator(device=dev).manual_seed(1))
    g2 = torch.randn((3,) + shape[1:], device=dev, generator=torch.Generator(device=dev).manual_seed(2))
    v1, v2, v12 = pb.vjp(g1), pb.vjp(g2), pb.vjp(2.0 * g1 - 0.5 * g2)
    assert torch.allclose(v12, 2.0 * v1 - 0.5 * v2, rtol=1e-4, atol=1e-6 * float(v12.abs().max()))
