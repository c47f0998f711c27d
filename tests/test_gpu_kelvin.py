"""Brightness-temperature output (Sect. 2.7): the device skydip fit and the K-mode TOD against
the oracle, through the C ABI."""
import numpy as np
import pytest
import torch

from oracle import gateau_oracle as O
from paper_2604_23305_b300 import Plan, workloads as W
from paper_2604_23305_b300 import _lib as L

pytestmark = pytest.mark.gpu

SIGNAL_TOL = {"fp32": 1e-5, "bf16x3": 1e-3}
DIP = (0.4, 2.4, 16)
F32_EPS = 2.0 ** -23


def _scenario(nt):
    sc = W.scenario("single_pixel_small", nt_total=nt)
    sc["output"] = dict(units="K", skydip=DIP)
    return sc


def _run(sc, precision, nt, white, pink, chunks=None):
    p = Plan(sc, precision=precision, white=white, pink=pink)
    if chunks is None:
        out = p.run(0, nt)
    else:
        parts, a = [], 0
        for c in chunks:
            parts.append(p.run(a, c))
            a += c
        out = torch.cat(parts)
    torch.cuda.synchronize()
    assert p.status() & ~L.STATUS_PWV_CLAMPED == 0
    return out.cpu().numpy().astype(np.float64), p


def test_skydip_fit_matches_oracle():
    sc = _scenario(64)
    p = Plan(sc, precision="bf16x3")
    p.prepare()
    n_ch = p.n_ch
    a = p.get_vector(L.VEC_TB_A, n_ch)
    b = p.get_vector(L.VEC_TB_B, n_ch)
    cal = O.skydip_calibration(sc, None, *DIP)
    print(f"skydip a rel err {np.max(np.abs(a / cal['a'] - 1)):.2e}, b abs err {np.max(np.abs(b - cal['b'])):.2e} K")
    np.testing.assert_allclose(a, cal["a"], rtol=1e-6)
    np.testing.assert_allclose(b, cal["b"], rtol=1e-6, atol=1e-6 * np.abs(cal["t_b"]).max())


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_kelvin_tod_noiseless_matches_oracle(precision):
    """|K_gpu - K_oracle| <= a (tol_W P) + float rounding of the map, tol_W the W-mode signal bound."""
    nt = 300
    sc = _scenario(nt)
    got, _ = _run(sc, precision, nt, white=False, pink=False)
    inst = O.build_instrument(sc)
    cal = O.skydip_calibration(sc, inst, *DIP)
    parts = O.simulate(sc, 0, nt, inst, white=False, pink=False, return_parts=True)
    want = cal["a"] * parts["total"] + cal["b"]
    bound = SIGNAL_TOL[precision] * np.abs(cal["a"] * parts["total"]) + 4 * F32_EPS * (
        np.abs(cal["a"] * parts["total"]) + np.abs(cal["b"]))
    err = np.abs(got - want)
    print(f"{precision}: max |dK| {err.max():.3e} K, max ratio to bound {np.max(err / bound):.3f}")
    assert np.all(err <= bound)


@pytest.mark.parametrize("precision", ["fp32", "bf16x3"])
def test_kelvin_tod_with_noise_is_the_affine_map_of_watts(precision):
    """With white and pink noise, in chunks: the K-mode TOD equals a P_tot + b of the same plan
    in W to float rounding (the pink term enters through residues scaled by a)."""
    nt = 400
    chunks = [77, 123, 200]
    sc = _scenario(nt)
    k, p = _run(sc, precision, nt, white=True, pink=True, chunks=chunks)
    a = p.get_vector(L.VEC_TB_A, p.n_ch)
    b = p.get_vector(L.VEC_TB_B, p.n_ch)
    scw = W.scenario("single_pixel_small", nt_total=nt)
    w, _ = _run(scw, precision, nt, white=True, pink=True, chunks=chunks)
    want = a * w + b
    bound = 8 * F32_EPS * (np.abs(a * w) + np.abs(b)) + 1e-5 * np.abs(a) * np.std(w, axis=0)
    err = np.abs(k - want)
    print(f"{precision}: max |K - (a W + b)| {err.max():.3e} K, max ratio to bound {np.max(err / bound):.3f}")
    assert np.all(err <= bound)
