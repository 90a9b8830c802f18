"""Host-side logic of bench.py and the auto-tuning driver (CPU only): the
column limits and algorithmic byte counts behind the roofline figures, the
torch.fft composition timed beside the library, the reference arm's JSON
line, and the tuning state's checkpoint round trip.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import bench
import phantom as ph
from oracle import model as OM, optics as OO

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_band_columns_count_the_detection_band():
    for X, p in ((512, 0.1), (192, 0.1), (128, 0.1), (64, 0.05)):
        o = ph.optics(pixel_um=p)
        nu = np.abs(np.fft.fftfreq(X, p))
        assert bench.band_columns(o, X) == int(np.sum(nu <= o["na_det"] / o["lambda_um"]))


@pytest.mark.parametrize("kinds", [("phase",), ("phase", "absorption"), ("fluor",), ("phase", "absorption", "fluor")])
def test_skipped_columns_hold_no_transfer_function(kinds):
    # the columns the bench counts as skipped (beyond support_xcols in k_x,
    # outside support_columns in (k_y, k_x)) carry none of the oracle's TFs
    shape = (4, 48, 64)
    Z, Y, X = shape
    o = ph.optics(pixel_um=0.05, na_ill=0.6, tilt_x=0.05)
    T = OO.transfer_functions(o, shape, kinds)
    xc = bench.support_xcols(o, kinds, X)
    n_sup = bench.support_columns(o, kinds, Y, X)
    assert xc < X // 2 + 1 and n_sup < Y * (X // 2 + 1)
    for k in kinds:
        H = OO.half_spectrum(T[k])
        peak = np.abs(H).max()
        assert np.abs(H[..., xc:]).max() <= 1e-12 * peak
        # the n_sup columns of largest energy hold all of it
        e = np.sort((np.abs(H) ** 2).sum(axis=0).ravel())[::-1]
        assert e[n_sup:].sum() <= 1e-20 * e.sum()


def test_widefield_algorithmic_bytes():
    o = ph.optics()
    Z, Y, X = bench.SHAPE
    Xh = X // 2 + 1
    b = bench.algorithmic_bytes(bench.SHAPE, bench.KINDS, o)
    band = int(np.sum(np.abs(np.fft.fftfreq(X, o["pixel_um"])) <= o["na_det"] / o["lambda_um"]))
    # three arms in the detection band in, three TF half spectra out (8-byte complex)
    assert b["tf_psf_rows"] == 3 * Z * Y * band * 8 + 3 * Z * Y * Xh * 8 == 575668224
    assert b["tf_arms"] == 3 * Z * Y * band * 8
    # x passes: two real stacks in and their half spectra out; three back
    assert b["rows_r2c"] == 2 * (Z * Y * X * 4 + Z * Y * Xh * 8)
    assert b["rows_c2r"] == 3 * (Z * Y * Xh * 8 + Z * Y * X * 4)
    assert all(v > 0 for v in b.values())


def test_torch_fft_composition_matches_the_oracle():
    torch = pytest.importorskip("torch")
    shape = (8, 16, 24)
    o = ph.optics(na_ill=0.7, tilt_y=0.03, defocus_um=0.2)
    kinds = ("phase", "absorption", "fluor")
    T = OO.transfer_functions(o, shape, kinds)
    modes, _, _ = OM.widefield_system(T, kinds)
    H = torch.from_numpy(np.stack([OO.half_spectrum(T[k]) for k in kinds]))
    rng = np.random.default_rng(7)
    f = rng.uniform(-0.02, 0.02, (3,) + shape)
    d = bench.torch_fft_forward(H, torch.from_numpy(f), [1.0, 0.1]).numpy()
    want = OM.forward(modes, f, [1.0, 0.1])
    assert np.linalg.norm(d - want) <= 1e-12 * np.linalg.norm(want)
    data = want + rng.normal(0.0, 1e-3, want.shape)
    got = bench.torch_fft_reconstruct(H, torch.from_numpy(data), bench.torch_fft_eta(H, [1e-3, 1e-3])).numpy()
    ref = OM.reconstruct(modes, data, 1e-3)
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


def test_reference_arm_prints_its_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                       cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "voxels/s" and line["value"] > 0
    assert line["metric"] == bench.METRIC and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_tuning_state_checkpoint_round_trip():
    # host logic of TuningProblem.state_dict / load_state_dict on CPU tensors
    torch = pytest.importorskip("torch")
    from paper_2412_09775_gb300.autotune import TuningProblem
    p = TuningProblem.__new__(TuningProblem)
    rng = np.random.default_rng(3)
    p.optics = torch.from_numpy(rng.normal(size=(5, 9)))
    p.optics0 = torch.from_numpy(rng.normal(size=(5, 9)))
    p.state = torch.from_numpy(rng.normal(size=(5, 4, 3)))
    sd = p.state_dict()
    want = {k: v.copy() for k, v in sd.items()}
    p.optics.zero_(), p.optics0.zero_(), p.state.zero_()
    # the checkpoint holds copies: clearing the buffers left it unchanged
    assert all(np.array_equal(sd[k], want[k]) for k in want)
    p.load_state_dict(sd)
    assert np.array_equal(p.optics.numpy(), want["optics"]) and np.array_equal(p.state.numpy(), want["adam"])
    assert np.array_equal(p.optics0.numpy(), want["optics0"])
    with pytest.raises(ValueError):
        p.load_state_dict(dict(want, adam=np.zeros((5, 1, 3))))


def test_traffic_records_match_their_kernels_sources():
    # a DRAM-traffic record is reported only while the kernel's sources are
    # the ones it was captured from; a record that no longer matches would
    # never be reported, so none is kept
    assert bench.NCU_TRAFFIC
    for (workload, family), rec in bench.NCU_TRAFFIC.items():
        assert rec["bytes"] > 0
        assert rec["digest"] == bench.kernel_digest(family), (workload, family)
