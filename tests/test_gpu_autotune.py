"""The fused kernel's tile choices and the project's tile autotuner on the GPU.

Every channel split and pipeline depth computes the same contraction: each
choice is checked against the FP64 oracle within the split-BF16 tolerance.  The
autotuner times the candidates, keeps the fastest, and serves the next plan of
the same shape class from its cache.
"""
import numpy as np
import pytest
import torch

from oracle import gateau_oracle as O
from paper_2604_23305_b300 import Plan, workloads as W

pytestmark = pytest.mark.gpu

_ref = {}


def _oracle(name, nt):
    if (name, nt) not in _ref:
        sc = W.scenario(name, nt_total=nt)
        _ref[(name, nt)] = (sc, O.simulate(sc, 0, nt, white=False, pink=False, return_parts=True))
    return _ref[(name, nt)]


@pytest.mark.parametrize("n_groups,ring_b", [(0, 0), (2, 2), (2, 6), (3, 4), (3, 6), (4, 3)])
def test_every_tile_choice_matches_the_oracle(n_groups, ring_b):
    """347 channels: 2 groups (2-CTA clusters, the default), 3 or 4 groups (independent CTAs),
    B rings of 2 to 6 stages."""
    sc, ref = _oracle("ifu25", 300)
    p = Plan(sc, precision="bf16x3", white=False, pink=False)
    p.set_tiles(n_groups, ring_b)
    got = p.run(0, 300)
    torch.cuda.synchronize()
    info = p.info()
    assert info.tile_groups == (n_groups or 2)
    assert 2 <= info.ring_b <= 6 and info.ring_b <= info.ring_a
    if ring_b:
        assert info.ring_b <= ring_b
    err = float(np.max(np.abs(got.double().cpu().numpy() - ref["p_kid"]) / np.abs(ref["p_kid"])))
    print(f"groups {info.tile_groups} x {info.tile_half}, rings A {info.ring_a} B {info.ring_b}: max rel err {err:.3e}")
    assert err < 1e-3
    assert p.status() & ~1 == 0


def test_autotune_times_candidates_then_serves_the_shape_class_from_cache():
    sc, ref = _oracle("single_pixel_small", 256)
    p = Plan(sc, precision="bf16x3", white=False, pink=False)
    ch = p.autotune(nt_sample=1024)
    print("autotune:", ch)
    assert ch["candidates"] >= 3
    assert ch["ms"] > 0 and ch["default_ms"] > 0 and ch["ms"] <= ch["default_ms"]
    info = p.info()
    assert (info.tile_groups, info.ring_b) == (ch["n_groups"], ch["ring_b"]) and info.tune_ms == ch["ms"]
    # the tuned plan still matches the oracle, and its run state was not touched by the tuning
    assert info.next_t0 == 0
    got = p.run(0, 256)
    torch.cuda.synchronize()
    err = float(np.max(np.abs(got.double().cpu().numpy() - ref["p_kid"]) / np.abs(ref["p_kid"])))
    assert err < 1e-3
    # a second plan of the same shape class takes the cached choice without timing
    q = Plan(sc, precision="bf16x3", white=False, pink=False)
    ch2 = q.autotune(nt_sample=1024)
    assert ch2["candidates"] == 0
    assert (ch2["n_groups"], ch2["ring_b"]) == (ch["n_groups"], ch["ring_b"])


def test_autotune_keeps_the_pink_state_of_a_running_scan():
    """Tuning in the middle of a chunked scan leaves the next chunk identical to an untuned plan's
    (the tuning sample neither advances the scan nor resets the pink-filter states)."""
    sc = W.scenario("single_pixel_small", nt_total=600)
    a = Plan(sc, precision="bf16x3", white=True, pink=True)
    b = Plan(sc, precision="bf16x3", white=True, pink=True)
    a.run(0, 300)
    b.run(0, 300)
    torch.cuda.synchronize()
    a.autotune(nt_sample=512)
    ta, tb = a.run(300, 300), b.run(300, 300)
    torch.cuda.synchronize()
    # same noise draws and pink states; the signal may differ by the split-BF16 rounding only
    x, y = ta.double().cpu().numpy(), tb.double().cpu().numpy()
    assert np.max(np.abs(x - y) / np.abs(y)) < 1e-4
