"""Shared persistent launches over several plans (gateau_run_batch) on the GPU.

A batch puts the split-BF16 contractions of all its plans into shared launches of
the fused kernel (one for plans with two channel groups, one for the others).
Each plan's arithmetic is the same as when it runs alone, so every output must
be bit-identical to gateau_run of a fresh plan over the same chunks, whatever
the mix of spaxel counts, channel counts and spectral grids; one plan is also
checked against the oracle.
"""
import numpy as np
import pytest
import torch

from oracle import gateau_oracle as O
from paper_2604_23305_b300 import Plan, run_batch
from paper_2604_23305_b300.serve import ServingInputs

pytestmark = pytest.mark.gpu

# uneven requests: 1-19 spaxels, 60-347 channels (one and two channel groups), 1000-6000 points
SHAPES = [dict(R_hex=0, n_pix=1, n_ch=347, n_freq=1500, nt=700),
          dict(R_hex=1, n_pix=7, n_ch=100, n_freq=1000, nt=300),
          dict(R_hex=2, n_pix=19, n_ch=213, n_freq=2000, nt=260),
          dict(R_hex=1, n_pix=7, n_ch=60, n_freq=6000, nt=200),
          dict(R_hex=0, n_pix=1, n_ch=176, n_freq=3000, nt=129),
          dict(R_hex=1, n_pix=7, n_ch=290, n_freq=1000, nt=1000)]


def _scenarios(seed):
    inp = ServingInputs(seed=seed)
    return [inp.scenario(r, i) for i, r in enumerate(SHAPES)]


def _alone(sc, precision, chunks):
    p = Plan(sc, precision=precision, white=True, pink=True)
    outs, t0 = [], 0
    for c in chunks:
        outs.append(p.run(t0, c))
        t0 += c
    torch.cuda.synchronize()
    assert p.status() & ~1 == 0
    return torch.cat(outs).cpu().numpy()


@pytest.mark.parametrize("precision", ["bf16x3", "fp32"])
def test_batch_equals_plans_run_alone(precision):
    scs = _scenarios(7)
    # two chunks per plan: a first batch, then a second that continues every plan's pink state
    firsts = [max(1, r["nt"] // 3) for r in SHAPES]
    plans = [Plan(sc, precision=precision, white=True, pink=True) for sc in scs]
    a = run_batch(plans, [0] * len(plans), firsts)
    b = run_batch(plans, firsts, [r["nt"] - f for r, f in zip(SHAPES, firsts)])
    torch.cuda.synchronize()
    for k, (sc, r) in enumerate(zip(scs, SHAPES)):
        got = torch.cat([a[k], b[k]]).cpu().numpy()
        want = _alone(sc, precision, [firsts[k], r["nt"] - firsts[k]])
        assert np.array_equal(got, want), f"plan {k} ({r}) differs in the batch"
        assert plans[k].status() & ~1 == 0


def test_batch_matches_the_oracle():
    """The 19-spaxel, 213-channel request of a mixed batch against the FP64 oracle (noiseless)."""
    scs = _scenarios(8)
    plans = [Plan(sc, precision="bf16x3", white=False, pink=False) for sc in scs]
    outs = run_batch(plans, [0] * len(plans), [r["nt"] for r in SHAPES])
    torch.cuda.synchronize()
    k = 2
    ref = O.simulate(scs[k], 0, SHAPES[k]["nt"], white=False, pink=False, return_parts=True)
    got = outs[k].double().cpu().numpy()
    err = float(np.max(np.abs(got - ref["p_kid"]) / np.abs(ref["p_kid"])))
    print(f"batched plan {k}: max rel err {err:.3e}")
    assert err < 1e-3


def test_batch_launch_count():
    """The contractions of a batch are two launches (one per launch mode), not one per plan."""
    scs = _scenarios(9)
    plans = [Plan(sc, precision="bf16x3", white=True, pink=False) for sc in scs]
    for p in plans:
        p.get_timing()
    run_batch(plans, [0] * len(plans), [r["nt"] for r in SHAPES])
    torch.cuda.synchronize()
    launches = sum(p.get_timing()[2] for p in plans)
    # per plan: row setup (+ cube scaling on the first run); shared: 2 fused launches
    n_scale = len(plans)
    assert launches == len(plans) + n_scale + 2
