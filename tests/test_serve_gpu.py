"""The serving runtime on the GPU: results do not depend on the mix.

A request's TOD must be the same whether it runs alone on the server or
admitted together with others whose chunks are in flight on other streams at
the same time, and the same as gateau_run of a fresh plan over the same chunk
boundaries (bit for bit: every request's arithmetic is independent of the
others', and chunks of one request run in order on one stream).
"""
import numpy as np
import pytest
import torch

from paper_2604_23305_b300 import Plan
from paper_2604_23305_b300.serve import Server, ServingInputs, build_requests

pytestmark = pytest.mark.gpu

CHUNK = 512


def shapes():
    # four small, different requests: spaxels 1/7/19, 100-347 channels, 1000-2000 points, 2-8 chunks
    return [dict(R_hex=0, n_pix=1, n_ch=347, n_freq=1500, nt=1800),
            dict(R_hex=1, n_pix=7, n_ch=100, n_freq=1000, nt=1100),
            dict(R_hex=2, n_pix=19, n_ch=213, n_freq=2000, nt=700),
            dict(R_hex=1, n_pix=7, n_ch=290, n_freq=1000, nt=4000)]


def outputs(reqs):
    return [np.zeros((r["nt"], r["n_pix"], r["n_ch"]), dtype=np.float32) for r in reqs]


def test_request_results_are_the_same_alone_and_in_the_mix():
    assert torch.cuda.is_available()
    inputs = ServingInputs(seed=3)
    scs, reqs = build_requests(shapes(), inputs, CHUNK)
    make = lambda i: Plan(scs[i], precision="bf16x3", device_inputs=False)

    alone = []
    for i in range(len(reqs)):
        srv = Server(budget_bytes=8 << 30, max_active=1, chunk_samples=CHUNK, max_chunk_bytes=16 << 20)
        out = outputs([reqs[i]])[0]
        st = srv.run([dict(reqs[i], host_out=out)], lambda k, i=i: make(i))
        assert st["n_done"] == 1, st
        alone.append((out, srv.result(0)["checksum"]))
        srv.close()

    # the mix: four requests at once, plans built on the server thread (all four then have chunks
    # in flight together) and on three builder threads (they start as their plans are ready); chunks
    # on the requests' own streams, or in rounds whose contractions share persistent fused launches
    for builders, shared in ((0, False), (3, False), (0, True), (3, True)):
        srv = Server(budget_bytes=8 << 30, max_active=4, chunk_samples=CHUNK, max_chunk_bytes=16 << 20,
                     n_streams=4, n_builders=builders, shared_launches=shared)
        outs = outputs(reqs)
        st = srv.run([dict(r, host_out=o) for r, o in zip(reqs, outs)], make)
        assert st["n_done"] == 4 and st["n_failed"] == 0
        assert st["peak_active"] == 4
        if builders == 0:
            assert st["overlap"] > 1.0                   # requests had chunks in flight together
        if shared and builders == 0:
            assert st["mean_round"] > 1.0                # rounds held several requests' chunks
        assert 0 < st["p50_latency_s"] <= st["p99_latency_s"] <= st["max_latency_s"]
        for i in range(4):
            assert np.array_equal(outs[i], alone[i][0]), \
                f"request {i} differs in the mix ({builders} builders, shared launches {shared})"
            assert srv.result(i)["checksum"] == alone[i][1]
            assert np.isfinite(outs[i]).all() and np.abs(outs[i]).max() > 0
        srv.close()


def test_server_tod_equals_plan_runs_over_the_same_chunks():
    inputs = ServingInputs(seed=4)
    scs, reqs = build_requests(shapes()[:2], inputs, CHUNK)
    srv = Server(budget_bytes=8 << 30, max_active=2, chunk_samples=CHUNK, max_chunk_bytes=16 << 20)
    outs = outputs(reqs)
    st = srv.run([dict(r, host_out=o) for r, o in zip(reqs, outs)],
                 lambda i: Plan(scs[i], precision="bf16x3", device_inputs=False))
    assert st["n_done"] == 2
    for i, r in enumerate(reqs):
        p = Plan(scs[i], precision="bf16x3", device_inputs=False)
        ref = torch.empty((r["nt"], r["n_pix"], r["n_ch"]), dtype=torch.float32, device="cuda")
        for t0 in range(0, r["nt"], CHUNK):
            n = min(CHUNK, r["nt"] - t0)
            p.run(t0, n, ref[t0:t0 + n])
        torch.cuda.synchronize()
        assert np.array_equal(outs[i], ref.cpu().numpy())
        want = ref.double()
        cs = srv.result(i)["checksum"]
        assert cs[0] == pytest.approx(float(want.sum()), rel=1e-9, abs=1e-30)
        assert cs[1] == pytest.approx(float((want * want).sum()), rel=1e-9)
        p.close()


def test_budget_serialises_admission_on_the_gpu():
    # three requests of one shape; the budget holds exactly one of them (plan + two chunk buffers
    # + the checksum scratch, as the server counts it)
    inputs = ServingInputs(seed=5)
    scs, reqs = build_requests([shapes()[2]] * 3, inputs, CHUNK)
    r = reqs[0]
    need = r["device_bytes"] + 2 * min(CHUNK, r["nt"]) * r["n_pix"] * r["n_ch"] * 4 + 2 * (2 * 148 + 2) * 8
    assert all(q["device_bytes"] == r["device_bytes"] for q in reqs)
    srv = Server(budget_bytes=need, max_active=3, chunk_samples=CHUNK, max_chunk_bytes=16 << 20)
    st = srv.run(reqs, lambda i: Plan(scs[i], precision="bf16x3", device_inputs=False))
    assert st["n_done"] == 3
    assert st["peak_active"] == 1
    assert st["peak_bytes"] == need
    admitted = [srv.result(i)["admitted_s"] for i in range(3)]
    assert admitted[0] <= admitted[1] <= admitted[2]
