"""A prepared plan's runs captured into a CUDA graph and replayed.

Once a plan is prepared and its buffers are sized by a first run, gateau_run
enqueues stream work only, so a sequence of chunk runs can be captured into a
CUDA graph (torch's stream capture) and replayed: the replay repeats the same
chunks -- the chunk at t0 = 0 resets the pink-filter states inside the graph --
and reproduces the direct runs bit for bit.
"""
import pytest
import torch

from paper_2604_23305_b300 import Plan, workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["bf16x3", "fp32"])
def test_chunked_runs_captured_in_a_cuda_graph_replay_bit_identically(precision):
    sc = W.scenario("single_pixel_small", nt_total=512)
    p = Plan(sc, precision=precision, white=True, pink=True)
    chunks = [(0, 200), (200, 56), (256, 256)]
    ref = torch.cat([p.run(t0, n) for t0, n in chunks])           # direct runs (they also size the buffers)
    torch.cuda.synchronize()
    out = torch.zeros_like(ref)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        for t0, n in chunks:
            p.run(t0, n, out[t0:t0 + n])
    for _ in range(2):
        out.zero_()
        g.replay()
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    assert p.status() & ~1 == 0
