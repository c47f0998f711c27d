"""The allocation-free pink-noise entry point against gateau_run's own pink noise.

gateau_pink_noise_noalloc serves callers that cannot allocate device memory
while they run (a fixed memory pool owned by an embedding runtime, a real-time
loop that must not call cudaMalloc): its scratch is a static device array.
This test feeds it the plan's own filter tables, state and seed through the C
ABI, in two calls in a row (the second continuing the first's state), and
checks that the result equals the pink noise gateau_run adds, within the pink
tolerance the other GPU tests use (1e-4 of the channel's pink rms).
The file is named so that pytest collects it after every other test file.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2604_23305_b300 import Plan, workloads as W
from paper_2604_23305_b300 import _lib as L

pytestmark = pytest.mark.gpu


def test_noalloc_pink_matches_gateau_run_on_two_calls():
    assert torch.cuda.is_available()
    lib = L.lib()
    sc = W.scenario("ifu25", nt_total=300)
    nt, first = 300, 173
    with_pink = Plan(sc, precision="fp32", white=True, pink=True)
    ref = with_pink.run(0, nt)
    base = Plan(sc, precision="fp32", white=True, pink=False)
    out = base.run(0, nt)
    torch.cuda.synchronize()
    signal = out.clone()

    info = with_pink.info()
    n_pix, n_ch, n_pole = info.n_pix, info.n_ch, info.n_pole
    a = torch.tensor(with_pink.get_vector(L.VEC_PINK_A, n_ch * n_pole), dtype=torch.float32, device="cuda")
    r = torch.tensor(with_pink.get_vector(L.VEC_PINK_R, n_ch * n_pole), dtype=torch.float32, device="cuda")
    d = torch.tensor(with_pink.get_vector(L.VEC_PINK_D, n_ch), dtype=torch.float32, device="cuda")
    state = torch.zeros((n_pix, n_ch, n_pole), dtype=torch.float32, device="cuda")
    seed = int(sc["noise"]["seed"])
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for t0, cnt in ((0, first), (first, nt - first)):
        view = out[t0:t0 + cnt]
        st = lib.gateau_pink_noise_noalloc(a.data_ptr(), r.data_ptr(), d.data_ptr(), n_pix, n_ch, n_pole, seed,
                                           t0, cnt, state.data_ptr(), view.data_ptr(), stream)
        assert st == L.OK, lib.gateau_last_error()
    torch.cuda.synchronize()

    got = out.double().cpu().numpy()
    want = ref.double().cpu().numpy()
    sig = signal.double().cpu().numpy()
    pink = want - sig
    rms = np.sqrt(np.mean(pink ** 2, axis=0, keepdims=True))
    worst = np.max(np.abs(got - want) / (1e-4 * rms + 1e-6 * np.abs(sig)))
    assert worst <= 1.0, worst
    _, plan_state = with_pink.get_state()
    np.testing.assert_allclose(state.double().cpu().numpy(), plan_state, rtol=1e-4, atol=1e-5 * np.abs(plan_state).max())

    # sizes beyond the fixed scratch are refused before anything is enqueued
    st = lib.gateau_pink_noise_noalloc(a.data_ptr(), r.data_ptr(), d.data_ptr(), 10000, n_ch, n_pole, seed,
                                       0, 4, state.data_ptr(), out.data_ptr(), stream)
    assert st == L.EINVAL and b"fixed scratch" in lib.gateau_last_error()


def _default_chunks(nt, S):
    """The allocating path's chunk count: the C (>= 64 samples a chunk) that minimises
    (L + 16) x (rounds of phase 3 + 0.75 rounds of phase 1), with 148 x 2 x 256 and 148 x 3 x 256
    threads resident per round."""
    cap1, cap3 = 148 * 3 * 256, 148 * 2 * 256
    best, best_c = None, 1
    for c in range(1, max(-(-nt // 64), 1) + 1):
        l_ = -(-(-(-nt // c)) // 4) * 4
        u = -(-nt // l_) * S
        cost = (l_ + 16) * (-(-u // cap3) + 0.75 * -(-u // cap1))
        if best is None or cost < best:
            best, best_c = cost, c
        if c * S > 16 * cap3:
            break
    L_ = -(-(-(-nt // best_c)) // 4) * 4
    return -(-nt // L_)


def test_noalloc_pink_caps_its_chunks_and_allocates_nothing():
    """A scan long enough that the allocating path's chunk states (n_pix n_ch n_pole per chunk)
    would not fit the 4 MiB of fixed scratch: the entry point takes fewer, longer chunks and still
    matches gateau_run's pink noise.  The calls after the first on this device (which looks up the
    scratch address and may load the library's module) leave the device's free memory unchanged."""
    assert torch.cuda.is_available()
    lib = L.lib()
    nt = 4096
    sc = W.scenario("ifu25", nt_total=nt)
    with_pink = Plan(sc, precision="fp32", white=False, pink=True)
    ref = with_pink.run(0, nt)
    base = Plan(sc, precision="fp32", white=False, pink=False)
    out = base.run(0, nt)
    torch.cuda.synchronize()
    signal = out.clone()
    info = with_pink.info()
    n_pix, n_ch, n_pole = info.n_pix, info.n_ch, info.n_pole
    S = n_pix * n_ch
    assert S * n_pole * _default_chunks(nt, S) > (1 << 20)      # the cap is needed here
    a = torch.tensor(with_pink.get_vector(L.VEC_PINK_A, n_ch * n_pole), dtype=torch.float32, device="cuda")
    r = torch.tensor(with_pink.get_vector(L.VEC_PINK_R, n_ch * n_pole), dtype=torch.float32, device="cuda")
    d = torch.tensor(with_pink.get_vector(L.VEC_PINK_D, n_ch), dtype=torch.float32, device="cuda")
    state = torch.zeros((n_pix, n_ch, n_pole), dtype=torch.float32, device="cuda")
    warm_state = torch.zeros_like(state)
    warm_out = torch.zeros((4, n_pix, n_ch), dtype=torch.float32, device="cuda")
    seed = int(sc["noise"]["seed"])
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.gateau_pink_noise_noalloc(a.data_ptr(), r.data_ptr(), d.data_ptr(), n_pix, n_ch, n_pole, seed,
                                       0, 4, warm_state.data_ptr(), warm_out.data_ptr(), stream)
    assert st == L.OK, lib.gateau_last_error()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    st = lib.gateau_pink_noise_noalloc(a.data_ptr(), r.data_ptr(), d.data_ptr(), n_pix, n_ch, n_pole, seed,
                                       0, nt, state.data_ptr(), out.data_ptr(), stream)
    assert st == L.OK, lib.gateau_last_error()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0

    got = out.double().cpu().numpy()
    want = ref.double().cpu().numpy()
    sig = signal.double().cpu().numpy()
    pink = want - sig
    rms = np.sqrt(np.mean(pink ** 2, axis=0, keepdims=True))
    worst = np.max(np.abs(got - want) / (1e-4 * rms + 1e-6 * np.abs(sig)))
    assert worst <= 1.0, worst
