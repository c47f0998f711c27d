"""Serving many simulations on one GPU through the native server (gateau_server_*).

The scheduling -- admission by slots and device-memory budget, chunked runs
on several streams, copies to the host, latency statistics -- runs in the
library (csrc/serve.cu); this module marshals requests and turns Python plan
objects into the factory / release callbacks the server calls.
"""
from __future__ import annotations

import ctypes as C
import math
import traceback

import numpy as np

from . import _lib as L
from . import workloads as W
from .plan import Plan, estimate_bytes, hex_offsets

ARCSEC = math.pi / (180.0 * 3600.0)
DEG = math.pi / 180.0

_STAT_FIELDS = [f for f, _ in L.ServerStats._fields_]


class Server:
    """A gateau_server: `run` plays a list of requests through it in real time."""

    def __init__(self, budget_bytes: int, max_active: int = 16, chunk_samples: int = 4096,
                 max_chunk_bytes: int = 32 << 20, n_streams: int | None = None, dry_run: bool = False,
                 dry_seconds_per_sample: float = 0.0, n_builders: int = 0, shared_launches: bool = False):
        self._lib = L.lib()
        d = L.ServerDesc()
        d.budget_bytes = int(budget_bytes)
        d.max_active = int(max_active)
        d.chunk_samples = int(chunk_samples)
        d.max_chunk_bytes = int(max_chunk_bytes)
        d.n_streams = int(n_streams if n_streams is not None else max_active)
        d.dry_run = 1 if dry_run else 0
        d.dry_seconds_per_sample = float(dry_seconds_per_sample)
        d.n_builders = int(n_builders)
        d.shared_launches = 1 if shared_launches else 0
        self._h = L.ServerP()
        L.check(self._lib.gateau_server_create(C.byref(d), C.byref(self._h)))
        self.n = 0

    def run(self, requests: list[dict], make_plan) -> dict:
        """requests[i]: arrival_s, nt, n_pix, n_ch, device_bytes, optional host_out (float32
        [nt, n_pix, n_ch]); make_plan(i) returns the request's Plan (or a raw handle in a dry
        run, or None for a failed request).  Returns the server statistics as a dict."""
        n = len(requests)
        arr = (L.Request * max(n, 1))()
        keep = []
        for i, r in enumerate(requests):
            q = arr[i]
            q.arrival_s = float(r["arrival_s"])
            q.nt = int(r["nt"])
            q.n_pix, q.n_ch = int(r["n_pix"]), int(r["n_ch"])
            q.device_bytes = int(r.get("device_bytes", 0))
            out = r.get("host_out")
            if out is not None:
                assert out.dtype == np.float32 and out.flags.c_contiguous and out.size == q.nt * q.n_pix * q.n_ch
                keep.append(out)
                q.host_out = out.ctypes.data
            else:
                q.host_out = None
        live: dict[int, object] = {}

        def factory(_user, i):
            try:
                p = make_plan(i)
            except Exception:
                traceback.print_exc()
                return None
            if p is None:
                return None
            live[i] = p
            return p._h.value if isinstance(p, Plan) else int(p)

        def release(_user, i, _plan):
            p = live.pop(i, None)
            if isinstance(p, Plan):
                p.close()

        cf, cr = L.PLAN_FACTORY(factory), L.PLAN_RELEASE(release)
        stats = L.ServerStats()
        st = self._lib.gateau_server_run(self._h, arr, n, cf, cr, None, C.byref(stats))
        for p in list(live.values()):
            if isinstance(p, Plan):
                p.close()
        live.clear()
        L.check(st)
        self.n = n
        del keep
        return {f: getattr(stats, f) for f in _STAT_FIELDS}

    def result(self, i: int) -> dict:
        state, lat, adm = C.c_int(0), C.c_double(0), C.c_double(0)
        cs = (C.c_double * 2)()
        L.check(self._lib.gateau_server_request_result(self._h, int(i), C.byref(state), C.byref(lat),
                                                       C.byref(adm), cs))
        return dict(state=state.value, latency_s=lat.value, admitted_s=adm.value, checksum=(cs[0], cs[1]))

    def close(self):
        if self._h:
            self._lib.gateau_server_destroy(self._h)
            self._h = L.ServerP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------- serving workload

def serving_requests(n: int = 256, seed: int = 2, f_sample: float = 160.0) -> list[dict]:
    """Request shapes of the serving workload: hexagonal IFUs of R = 0..4 rings (1, 7, 19, 37,
    61 spaxels), 100-347 channels, 1000-6000 spectral points (steps of 500), scans of 10 s to
    10 min (log-uniform) at 160 Hz."""
    rng = np.random.default_rng(seed)
    R = rng.integers(0, 5, n)
    n_ch = rng.integers(100, 348, n)
    n_freq = rng.integers(2, 13, n) * 500
    dur = np.exp(rng.uniform(math.log(10.0), math.log(600.0), n))
    nt = np.maximum(16, np.round(dur * f_sample)).astype(np.int64)
    return [dict(R_hex=int(R[i]), n_pix=1 + 3 * int(R[i]) * (int(R[i]) + 1), n_ch=int(n_ch[i]),
                 n_freq=int(n_freq[i]), nt=int(nt[i])) for i in range(n)]


class ServingInputs:
    """Seeded inputs of serving requests; the screen is shared, tables and cubes are cached per
    spectral grid (they depend only on it)."""

    def __init__(self, seed: int = 2, cube_side: int = 24):
        self.seed = seed
        self.cube_side = cube_side
        self.screen = W.pwv_screen(256, 256, 0.5, 1.0, 0.02, seed)
        self._grid = {}

    def _grid_inputs(self, n_freq: int):
        if n_freq not in self._grid:
            nu = np.linspace(220e9, 440e9, n_freq)
            tab, pmin, dp = W.opacity_table(nu)
            cube, grid = W.point_source_cube(nu, self.cube_side, self.cube_side, 70 * ARCSEC, 47.8 * DEG)
            self._grid[n_freq] = (tab, pmin, dp, cube, grid)
        return self._grid[n_freq]

    def scenario(self, req: dict, index: int) -> dict:
        n_freq, n_ch, nt = req["n_freq"], req["n_ch"], req["nt"]
        tab, pmin, dp, cube, grid = self._grid_inputs(n_freq)
        fs = 160.0
        sc = W._base(n_freq, 220e9, 440e9, fs, hex_offsets(req["R_hex"], 15 * ARCSEC), nt)
        w = 2 * math.pi * 1.54
        sc.update(
            atmosphere=dict(screen=self.screen, pitch=0.5, is_epl=False, pwv0=0.0, h_column=W.ASTE["h_column"],
                            wind=10.0, T_atm=W.ASTE["T_atm"], table=tab, table_is_opacity=True, pwv_min=pmin,
                            dpwv=dp),
            source=dict(cube=cube, az0=grid["az0"], daz=grid["daz"], el0=grid["el0"], **{"del": grid["d_el"]}),
            scan=dict(kind="daisy", params=(65 * ARCSEC, w, w / 50.0), phi0=0.0, theta0=47.8 * DEG),
            cascade=W.table1_cascade(),
            dispersive=dict(kind="filterbank", f_c=W.geometric_channels(220e9, 440e9, n_ch),
                            R=np.full(n_ch, 500.0), eta_peak=np.full(n_ch, 0.16)),
        )
        _, alpha = W.pink_levels(n_ch, self.seed + 7 + index)
        sc["noise"] = dict(seed=1000 + index, pink_A=None, pink_alpha=alpha, pink_f_min=fs / nt)
        return sc


def build_requests(shapes: list[dict], inputs: ServingInputs, chunk_samples: int, arrivals=None,
                   precision: str = "bf16x3"):
    """Scenarios, memory estimates and request records of a serving workload."""
    scs = [inputs.scenario(r, i) for i, r in enumerate(shapes)]
    reqs = []
    for i, (r, sc) in enumerate(zip(shapes, scs)):
        reqs.append(dict(arrival_s=0.0 if arrivals is None else float(arrivals[i]), nt=r["nt"], n_pix=r["n_pix"],
                         n_ch=r["n_ch"], device_bytes=estimate_bytes(sc, chunk_samples, precision)))
    return scs, reqs
