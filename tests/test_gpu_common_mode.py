"""Common-mode reduction (Sect. 4.3, Eqs. 25-26) and the observation's mean zenith PWV on the
GPU against the oracle, through the C ABI.  The reduced TOD is a seeded synthetic brightness-
temperature array given to both sides (no input comes from the CUDA path)."""
import math

import numpy as np
import pytest
import torch

from oracle import gateau_oracle as O
from paper_2604_23305_b300 import Plan, workloads as W
from paper_2604_23305_b300 import _lib as L

pytestmark = pytest.mark.gpu

ARCSEC = math.pi / (180 * 3600)
F32_EPS = 2.0 ** -23


def _scenario(nt):
    sc = W.scenario("single_pixel_small", nt_total=nt)
    sc["pix_offsets"] = O.hex_offsets(2, 30 * ARCSEC)                      # 19 spaxels, 30" apart
    sc["scan"] = dict(sc["scan"], kind="daisy", params=(20 * ARCSEC, 1.0, 0.1))
    return sc


def test_mean_zenith_pwv_matches_oracle():
    sc = _scenario(700)
    p = Plan(sc, precision="fp32")
    got = p.mean_zenith_pwv(700)
    want = O.mean_zenith_pwv(sc, 700)
    print(f"mean zenith PWV {got:.9f} vs {want:.9f} mm")
    assert abs(got / want - 1.0) < 1e-6


@pytest.mark.parametrize("t0", [0, 137])
def test_common_mode_matches_oracle(t0):
    nt = 200
    sc = _scenario(t0 + nt)
    p = Plan(sc, precision="bf16x3")
    n_pix, n_ch = p.n_pix, p.n_ch
    rng = np.random.default_rng(19 + t0)
    tb = rng.uniform(5.0, 40.0, (nt, n_pix, n_ch)).astype(np.float32)
    pwv, r_out = 1.3, 45 * ARCSEC
    got = p.common_mode(t0, torch.from_numpy(tb).cuda(), pwv, r_out).cpu().numpy().astype(np.float64)
    torch.cuda.synchronize()
    want = O.common_mode_reduction(sc, tb.astype(np.float64), t0, pwv, r_out)
    # float rounding of T_b / eta and of (1 - eta) C / eta, C the common term (<= max T_b / (1 - eta_max))
    inst = O.build_instrument(sc)
    atm = sc["atmosphere"]
    tau = O.zenith_opacity(O.opacity_table(sc), atm["pwv_min"], atm["dpwv"], np.array([pwv]))[0]
    hw = inst.eta_filt * inst.w
    eta_z = (hw @ np.exp(-tau)) / hw.sum(axis=1)
    nn, ii = np.meshgrid(np.arange(t0, t0 + nt), np.arange(n_pix), indexing="ij")
    _, _, el, _ = O.row_geometry(sc, nn.ravel(), ii.ravel())
    eta = eta_z[None, None, :] ** (1.0 / np.sin(el)).reshape(nt, n_pix)[:, :, None]
    cmax = (tb.max(axis=1, keepdims=True) / (1.0 - eta.max(axis=1, keepdims=True)))
    bound = 64 * F32_EPS * (np.abs(tb) + (1.0 - eta) * cmax) / eta
    err = np.abs(got - want)
    print(f"t0={t0}: max |dT| {err.max():.3e} K, max ratio to bound {np.max(err / bound):.3f}")
    assert np.all(err <= bound)


def test_common_mode_in_place_and_rejections():
    nt = 64
    sc = _scenario(nt)
    p = Plan(sc, precision="bf16x3")
    tb = torch.from_numpy(np.random.default_rng(3).uniform(5, 40, (nt, p.n_pix, p.n_ch)).astype(np.float32)).cuda()
    ref = p.common_mode(0, tb, 1.1, 45 * ARCSEC)
    same = tb.clone()
    p.common_mode(0, same, 1.1, 45 * ARCSEC, out=same)
    torch.cuda.synchronize()
    assert torch.equal(ref, same)
    with pytest.raises(L.GateauError):                    # no spaxel beyond r_out
        p.common_mode(0, tb, 1.1, 3600 * ARCSEC)
