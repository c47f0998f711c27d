"""Host tests of the serving scheduler (gateau_server_* in dry-run mode: no GPU).

In a dry run the server makes the same admission, slot, stream and budget
decisions as on the GPU, but a chunk of D detector samples occupies its stream
for D * dry_seconds_per_sample on a virtual clock, so latencies are exact
numbers that can be worked out by hand.
"""
import numpy as np
import pytest

from paper_2604_23305_b300 import _lib as L
from paper_2604_23305_b300.serve import Server

SPS = 1e-3   # virtual seconds per detector sample


def req(arrival=0.0, nt=100, n_pix=1, n_ch=10, device_bytes=1000):
    return dict(arrival_s=arrival, nt=nt, n_pix=n_pix, n_ch=n_ch, device_bytes=device_bytes)


def dry(**kw):
    args = dict(budget_bytes=10**12, max_active=4, chunk_samples=50, max_chunk_bytes=1 << 20, n_streams=1,
                dry_run=True, dry_seconds_per_sample=SPS)
    args.update(kw)
    return Server(**args)


def test_one_stream_serialises_chunks_in_launch_order():
    # two requests of 2 chunks x 500 detector samples (0.5 s each) on one stream
    s = dry()
    st = s.run([req(), req()], lambda i: 1)
    assert st["n_done"] == 2 and st["n_failed"] == 0
    assert s.result(0)["latency_s"] == pytest.approx(1.0)
    assert s.result(1)["latency_s"] == pytest.approx(2.0)
    assert st["p50_latency_s"] == pytest.approx(1.5)
    assert st["p99_latency_s"] == pytest.approx(1.99)
    assert st["makespan_s"] == pytest.approx(2.0)
    assert st["throughput"] == pytest.approx(2000 / 2.0)
    assert st["peak_active"] == 2


def test_two_streams_overlap_requests():
    s = dry(n_streams=2)
    st = s.run([req(), req()], lambda i: 1)
    assert [s.result(i)["latency_s"] for i in range(2)] == pytest.approx([1.0, 1.0])
    assert st["overlap"] > 1.0


def test_slots_bound_admission_first_come_first_served():
    s = dry(max_active=1, n_streams=1)
    st = s.run([req(), req(), req()], lambda i: 1)
    assert st["peak_active"] == 1
    assert [s.result(i)["admitted_s"] for i in range(3)] == pytest.approx([0.0, 1.0, 2.0])
    assert [s.result(i)["latency_s"] for i in range(3)] == pytest.approx([1.0, 2.0, 3.0])


def test_budget_bounds_admission():
    chunk_bytes = 50 * 10 * 4
    need = 1000 + 2 * chunk_bytes + 2 * (2 * 148 + 2) * 8     # device bytes + 2 chunks + checksum scratch
    s = dry(budget_bytes=2 * need, max_active=8, n_streams=8)
    st = s.run([req() for _ in range(5)], lambda i: 1)
    assert st["n_done"] == 5
    assert st["peak_active"] == 2
    assert st["peak_bytes"] <= 2 * need
    # two at a time, 1 s each on their own streams
    assert sorted(s.result(i)["latency_s"] for i in range(5)) == pytest.approx([1, 1, 2, 2, 3])


def test_requests_that_cannot_run_fail_and_others_complete():
    s = dry(budget_bytes=100_000)
    reqs = [req(), req(device_bytes=10**9), req(), req()]
    st = s.run(reqs, lambda i: None if i == 2 else 1)       # 1: over budget, 2: factory fails
    assert st["n_done"] == 2 and st["n_failed"] == 2
    assert [s.result(i)["state"] for i in range(4)] == [2, 3, 3, 2]


def test_latency_counts_from_arrival():
    s = dry(n_streams=1)
    st = s.run([req(), req(arrival=10.0)], lambda i: 1)
    assert s.result(1)["admitted_s"] == pytest.approx(10.0)
    assert s.result(1)["latency_s"] == pytest.approx(1.0)
    assert st["makespan_s"] == pytest.approx(11.0)


def test_percentiles_match_linear_interpolation():
    rng = np.random.default_rng(5)
    arrivals = np.sort(rng.uniform(0, 20, 40))
    reqs = [req(arrival=float(a), nt=int(rng.integers(10, 400)), n_pix=int(rng.integers(1, 8)),
                n_ch=int(rng.integers(5, 40))) for a in arrivals]
    s = dry(max_active=6, n_streams=3, chunk_samples=64)
    st = s.run(reqs, lambda i: 1)
    lat = np.array([s.result(i)["latency_s"] for i in range(len(reqs))])
    assert st["n_done"] == len(reqs)
    assert st["p50_latency_s"] == pytest.approx(np.percentile(lat, 50))
    assert st["p99_latency_s"] == pytest.approx(np.percentile(lat, 99))
    assert st["mean_latency_s"] == pytest.approx(lat.mean())
    work = sum(r["nt"] * r["n_pix"] * r["n_ch"] for r in reqs)
    assert st["detector_samples"] == pytest.approx(work)


def test_invalid_arguments_are_refused():
    with pytest.raises(L.GateauError):
        Server(budget_bytes=1, max_active=0, dry_run=True)
    s = dry()
    with pytest.raises(L.GateauError):
        s.run([req(arrival=1.0), req(arrival=0.5)], lambda i: 1)     # arrivals must not decrease
    with pytest.raises(L.GateauError):
        s.run([req(nt=0)], lambda i: 1)


def test_plan_memory_estimate_covers_the_inputs_and_grows_with_the_chunk():
    from paper_2604_23305_b300 import workloads as W
    from paper_2604_23305_b300.plan import estimate_bytes
    sc = W.scenario("single_pixel_small")
    kp = (sc["n_freq"] + 31) // 32 * 32
    cube = np.asarray(sc["source"]["cube"])
    floor = (2 * cube.shape[0] * cube.shape[1] * kp * 4                      # cube as set + scaled
             + np.asarray(sc["atmosphere"]["screen"]).size * 4
             + 2 * np.asarray(sc["atmosphere"]["table"]).shape[0] * kp * 4)  # interleaved opacity rows
    small, large = estimate_bytes(sc, 128), estimate_bytes(sc, 4096)
    assert small > floor
    assert large - small >= (4096 - 128) * 32                              # 32-byte row records per sample
    assert estimate_bytes(sc, 128, precision="fp32") > small                # FP32 operands + spectrum chunk
    with pytest.raises(L.GateauError):
        estimate_bytes(sc, 0)


def test_shared_launch_rounds_batch_every_active_request():
    # rounds of one chunk per request on one compute stream, two rounds in flight: requests 0 and 1
    # (2 chunks x 0.5 s) share rounds [0, 1] and [1, 2]; request 2 arrives at 0.5 and waits for a
    # round slot (both in flight until 1.0), then runs its chunks in rounds [2, 2.5] and [2.5, 3]
    s = dry(shared_launches=True)
    st = s.run([req(), req(), req(arrival=0.5)], lambda i: 1)
    assert st["n_done"] == 3 and st["n_failed"] == 0
    assert [s.result(i)["latency_s"] for i in range(3)] == pytest.approx([2.0, 2.0, 2.5])
    assert st["rounds"] == 4
    assert st["mean_round"] == pytest.approx(6 / 4)
    assert st["makespan_s"] == pytest.approx(3.0)


def test_shared_launch_rounds_respect_slots_and_budget():
    s = dry(shared_launches=True, max_active=2)
    st = s.run([req() for _ in range(5)], lambda i: 1)
    assert st["n_done"] == 5 and st["peak_active"] == 2
    assert st["mean_round"] <= 2.0
