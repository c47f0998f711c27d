"""Exact (Timmer-Koenig) pink noise (Sect. 2.6) on the GPU against the oracle, through the C ABI.

The pink term is isolated as the difference of two runs of the same plan configuration with
and without GATEAU_NOISE_PINK (everything else is deterministic and identical)."""
import numpy as np
import pytest
import torch

from oracle import gateau_oracle as O
from paper_2604_23305_b300 import Plan, workloads as W
from paper_2604_23305_b300 import _lib as L

pytestmark = pytest.mark.gpu

F32_EPS = 2.0 ** -23


def _tod(sc, nt, pink, chunks=None, precision="bf16x3"):
    p = Plan(sc, precision=precision, white=False, pink=pink)
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
    return out.cpu().numpy().astype(np.float64)


def _check(pink, base, want, label):
    """|got - want| <= 1e-5 rms_ch(want) + 4 eps |TOD| (FP32 FFT of 2^k points, float TOD)."""
    got = pink - base
    rms = np.sqrt(np.mean(want ** 2, axis=0))
    bound = 1e-5 * rms + 4 * F32_EPS * np.abs(pink)
    err = np.abs(got - want)
    print(f"{label}: max |d| / rms {np.max(err / np.maximum(rms, 1e-300)):.2e}, max ratio to bound {np.max(err / bound):.3f}")
    assert np.all(err <= bound)


@pytest.mark.parametrize("nt", [300, 1000, 2000])      # M = 512 (8^3), 1024 (8^3 2), 2048 (8^3 4)
def test_tk_pink_matches_oracle(nt):
    sc = W.scenario("single_pixel_small", nt_total=nt)
    sc["noise"] = dict(sc["noise"], pink_tk=nt)
    base = _tod(sc, nt, pink=False)
    pink = _tod(sc, nt, pink=True)
    parts = O.simulate(sc, 0, nt, white=False, pink=True, pink_tk=nt, return_parts=True)
    _check(pink, base, parts["p_pn"], f"N={nt}")


def test_tk_chunks_equal_one_pass():
    nt = 1000
    sc = W.scenario("single_pixel_small", nt_total=nt)
    sc["noise"] = dict(sc["noise"], pink_tk=nt)
    one = _tod(sc, nt, pink=True)
    parts = _tod(sc, nt, pink=True, chunks=[77, 123, 800])
    assert np.array_equal(one, parts)


def test_tk_run_past_the_realisation_is_rejected():
    sc = W.scenario("single_pixel_small", nt_total=300)
    sc["noise"] = dict(sc["noise"], pink_tk=200)
    p = Plan(sc, precision="bf16x3", white=False, pink=True)
    with pytest.raises(L.GateauError):
        p.run(0, 300)


def test_tk_full_size_sampled_series():
    """ifu25 (25 spaxels x 347 channels x 192000 samples, M = 262144): three whole series
    against the oracle's realisation of the same (spaxel, channel)."""
    sc = W.scenario("ifu25")
    nt = sc["nt_total"]
    sc["noise"] = dict(sc["noise"], pink_tk=nt)
    picks = [(0, 0), (12, 173), (24, 346)]
    series = {}
    for pink in (False, True):
        p = Plan(sc, precision="bf16x3", white=False, pink=pink)
        out = p.run(0, nt)
        torch.cuda.synchronize()
        assert p.status() & ~L.STATUS_PWV_CLAMPED == 0
        series[pink] = [out[:, i, ch].cpu().numpy().astype(np.float64) for i, ch in picks]
        del out, p
        torch.cuda.empty_cache()
    noise = sc["noise"]
    inst_A = O.build_instrument(sc).pink_A          # the knee at 1 Hz: A = the planned white level
    for k, (i, ch) in enumerate(picks):
        want = O.pink_tk_realisation(noise["seed"], float(inst_A[ch]), float(noise["pink_alpha"][ch]),
                                     sc["f_sample"], nt, i, ch)
        _check(series[True][k][:, None], series[False][k][:, None], want[:, None], f"ifu25 ({i}, {ch})")
