"""Preprocessing (Sect. 2.2, Eqs. 1-3) on the GPU against the oracle: far field, source-cube
convolution, screen smoothing, through the C ABI."""
import math

import numpy as np
import pytest
import torch

from oracle import gateau_oracle as O
from paper_2604_23305_b300 import prep
from paper_2604_23305_b300 import _lib as L

pytestmark = pytest.mark.gpu

AS = math.pi / (180 * 3600)


def test_far_field_matches_oracle():
    nu = np.array([220e9, 330e9, 440e9])
    F = prep.beam_far_field(nu, 128, 64, 3 * AS, 4 * AS, 5.0, -12.0).cpu().numpy()
    for k, v in enumerate(nu):
        want = O.beam_far_field(float(v), 128, 64, 3 * AS, 4 * AS, 5.0, -12.0)
        err = np.abs(F[k] - want).max()
        print(f"far field {v / 1e9:.0f} GHz: max |dF| {err:.2e}")
        assert err < 2e-6                      # FP32 transforms of a peak-1 pattern


def test_source_convolution_matches_oracle():
    rng = np.random.default_rng(12)
    n_az, n_el, n_f = 32, 16, 6
    I = rng.uniform(0.0, 1e-18, (n_az, n_el, n_f)).astype(np.float32)
    I[7, 5, :] += 5e-17                        # a bright compact source on top
    nu = np.linspace(200e9, 420e9, n_f)
    d = 5 * AS
    P = prep.convolve_source(torch.from_numpy(I).cuda(), nu, 0.83, d, d, 5.0, -10.0).cpu().numpy()
    want = O.convolve_source(I.astype(np.float64), nu, 0.83, d, d, 5.0, -10.0)
    scale = np.abs(want).max(axis=(0, 1))
    err = (np.abs(P - want).max(axis=(0, 1)) / scale).max()
    print(f"source convolution: max |dP| / max P {err:.2e}")
    assert err < 1e-5


def test_screen_smoothing_matches_oracle():
    rng = np.random.default_rng(5)
    scr = rng.normal(1.0, 0.05, (64, 128)).astype(np.float32)
    out = prep.smooth_screen(torch.from_numpy(scr).cuda(), 0.5, 5.0, -10.0).cpu().numpy()
    want = O.smooth_screen(scr.astype(np.float64), 0.5, 5.0, -10.0)
    err = np.abs(out - want).max()
    print(f"screen smoothing: max |d| {err:.2e} mm")
    assert err < 4e-6 * np.abs(want).max()


def test_preprocessing_rejects_bad_sizes():
    with pytest.raises(L.GateauError):
        prep.beam_far_field([300e9], 100, 64, AS, AS, 5.0, -10.0)
    with pytest.raises(L.GateauError):
        prep.smooth_screen(torch.zeros((48, 64), device="cuda"), 0.5, 5.0, -10.0)


@pytest.mark.parametrize("shape", [(8, 8192), (4096, 16), (2048, 2)])
def test_screen_smoothing_long_sides(shape):
    """Sides up to 4096 points take one shared-memory pass per dimension (1-16 vectors per block);
    longer sides (8192) take the global Stockham passes and transposes."""
    rng = np.random.default_rng(9)
    scr = rng.normal(0.9, 0.02, shape).astype(np.float32)
    out = prep.smooth_screen(torch.from_numpy(scr).cuda(), 0.5, 3.0, -10.0).cpu().numpy()
    want = O.smooth_screen(scr.astype(np.float64), 0.5, 3.0, -10.0)
    err = np.abs(out - want).max()
    print(f"screen smoothing {shape}: max |d| {err:.2e} mm")
    assert err < 4e-6 * np.abs(want).max()
