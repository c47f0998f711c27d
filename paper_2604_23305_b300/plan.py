"""Python handle on a simulator plan: marshals numpy / torch buffers into the C ABI.

Every step of the simulation runs in libgateau_b300.so; this module only passes
pointers, sizes and streams.  torch supplies device memory and streams.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L

_PREC = {"fp32": L.PREC_FP32, "bf16x3": L.PREC_BF16X3}
_SCAN = {"stare": L.SCAN_STARE, "daisy": L.SCAN_DAISY, "raster": L.SCAN_RASTER, "custom": L.SCAN_CUSTOM}
_DISP = {"filterbank": L.DISP_FILTERBANK, "lorentzian": L.DISP_LORENTZIAN, "custom": L.DISP_CUSTOM}


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(L.dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _stage_structs(stages, n_freq):
    keep = []
    arr = (L.Stage * max(len(stages), 1))()
    for s, st in enumerate(stages):
        T = st.get("T")
        t_k = L.T_SKY if (isinstance(T, str) and T == "sky") else float(T)
        x = arr[s]
        kind = st["kind"]
        if kind == "reflective":
            x.kind = L.STAGE_REFLECTIVE
            eta = np.asarray(st["eta"], dtype=np.float64)
            if eta.ndim == 0:
                x.eta = float(eta)
                x.eta_nu = None
            else:
                e = _f64(np.broadcast_to(eta, (n_freq,)))
                keep.append(e)
                x.eta_nu = _dptr(e)
        elif kind == "ohmic":
            x.kind = L.STAGE_OHMIC
            x.eps_ref = st["eps_ref"]
            x.nu_ref_hz = st["nu_ref"]
        elif kind == "refractive":
            x.kind = L.STAGE_REFRACTIVE
            x.d_m, x.n_index, x.tan_delta = st["d"], st["n"], st["tan_delta"]
            Tr = st.get("T_refl", T)
            x.T_refl_K = L.T_SKY if (isinstance(Tr, str) and Tr == "sky") else float(Tr)
            x.ar_coated = 1 if st.get("ar", False) else 0
        else:
            raise ValueError(f"unknown stage kind {kind!r}")
        x.T_K = t_k
    return arr, keep


def _plan_desc(sc: dict, pix: np.ndarray, precision: str, white: bool, pink: bool) -> L.PlanDesc:
    """gateau_plan_desc of a scenario (pix must stay alive while the struct is used)."""
    noise = sc.get("noise", {})
    d = L.PlanDesc()
    d.n_freq = int(sc["n_freq"])
    d.f_lo_hz, d.f_hi_hz, d.f_sample_hz = sc["f_lo"], sc["f_hi"], sc["f_sample"]
    d.n_pix = pix.shape[0]
    d.pix_offsets_rad = _dptr(pix)
    atm = sc["atmosphere"]
    d.T_atm_K, d.T_cmb_K = atm["T_atm"], sc["T_cmb"]
    d.h_column_m, d.wind_mps = atm["h_column"], atm["wind"]
    d.eta_taper, d.rho_surf_m, d.eta_pol = sc["eta_taper"], sc["rho_surf"], sc["eta_pol"]
    d.delta_al_J, d.eta_pb = sc["delta_al"], sc["eta_pb"]
    d.seed = int(noise.get("seed", 0))
    d.precision = _PREC[precision]
    d.noise_flags = (L.NOISE_WHITE if white else 0) | (L.NOISE_PINK if pink else 0)
    d.pink_f_min_hz = float(noise.get("pink_f_min", 1e-3))
    return d


def estimate_bytes(sc: dict, chunk_samples: int, precision: str = "bf16x3", white: bool = True,
                   pink: bool = True) -> int:
    """gateau_plan_estimate_bytes for a scenario: device memory its plan holds, upper bound."""
    pix = _f64(sc["pix_offsets"]).reshape(-1, 2)
    d = _plan_desc(sc, pix, precision, white, pink)
    atm, src = sc["atmosphere"], sc["source"]
    cube = np.asarray(src["cube"])
    scr = np.asarray(atm["screen"])
    custom = sc["scan"].get("custom")
    out = C.c_size_t(0)
    L.check(L.lib().gateau_plan_estimate_bytes(C.byref(d), int(np.asarray(sc["dispersive"]["f_c"]).size),
                                               cube.shape[0], cube.shape[1], scr.shape[1], scr.shape[0],
                                               np.asarray(atm["table"]).shape[0], int(chunk_samples),
                                               0 if custom is None else int(np.asarray(custom).shape[0]),
                                               C.byref(out)))
    return int(out.value)


class Plan:
    """A configured simulation (one instrument, one sky, one scan)."""

    def __init__(self, sc: dict, precision: str = "bf16x3", white: bool = True, pink: bool = True,
                 device_inputs: bool = True, upload: bool = True):
        self._lib = L.lib()
        self.sc = sc
        self.n_freq = int(sc["n_freq"])
        self.pix = _f64(sc["pix_offsets"]).reshape(-1, 2)
        self.n_pix = self.pix.shape[0]
        noise = sc.get("noise", {})
        atm = sc["atmosphere"]
        d = _plan_desc(sc, self.pix, precision, white, pink)
        self.precision = precision
        self._h = L.PlanP()
        L.check(self._lib.gateau_plan_create(C.byref(d), C.byref(self._h)))
        disp = sc["dispersive"]
        self.n_ch = int(np.asarray(disp["f_c"]).size)
        self.set_cascade(sc["cascade"])
        self.set_dispersive(disp)
        if "pink_alpha" in noise:
            # no level given: the library sets the knee at 1 Hz (A = the planned white level NEP^2)
            A = noise.get("pink_A")
            A = None if A is None else _f64(A)
            al = _f64(noise["pink_alpha"])
            L.check(self._lib.gateau_set_pink_noise(self._h, None if A is None else _dptr(A), _dptr(al)))
        if noise.get("pink_tk"):
            self.set_pink_timmer_koenig(int(noise["pink_tk"]))
        if upload:
            self.set_scan(sc["scan"], device=device_inputs)
            self.set_source(sc["source"], device=device_inputs)
            self.set_screen(atm, device=device_inputs)
            self.set_table(atm, device=device_inputs)
        out = sc.get("output")
        if out is not None and out.get("units", "W") == "K":
            self.set_output_kelvin(*out.get("skydip", (0.5, 2.0, 16)))

    # ---------------------------------------------------------------- setters
    def set_output_kelvin(self, pwv_lo: float = 0.5, pwv_hi: float = 2.0, n_pwv: int = 16, enable: bool = True):
        """Brightness-temperature output by a simulated skydip over n_pwv zenith PWVs (mm)."""
        L.check(self._lib.gateau_set_output_kelvin(self._h, 1 if enable else 0, float(pwv_lo), float(pwv_hi),
                                                   int(n_pwv)))

    def set_pink_timmer_koenig(self, n_total: int):
        """Exact (Timmer-Koenig) pink noise over samples [0, n_total); 0 restores the filter."""
        L.check(self._lib.gateau_set_pink_timmer_koenig(self._h, int(n_total)))

    def set_cascade(self, stages):
        arr, keep = _stage_structs(stages, self.n_freq)
        L.check(self._lib.gateau_set_cascade(self._h, len(stages), arr))
        del keep

    def set_dispersive(self, disp):
        kind = _DISP[disp["kind"]]
        f_c = _f64(disp["f_c"])
        R = _f64(np.broadcast_to(np.asarray(disp.get("R", 1.0), dtype=np.float64), f_c.shape))
        ep = _f64(np.broadcast_to(np.asarray(disp.get("eta_peak", 1.0), dtype=np.float64), f_c.shape))
        custom = disp.get("custom")
        cptr = _dptr(_f64(custom).reshape(-1)) if custom is not None else None
        keep = _f64(custom).reshape(-1) if custom is not None else None
        if keep is not None:
            cptr = _dptr(keep)
        L.check(self._lib.gateau_set_dispersive_element(self._h, kind, f_c.size, _dptr(f_c), _dptr(R), _dptr(ep), cptr))

    def _buffer(self, arr, dtype, device):
        a = np.ascontiguousarray(np.asarray(arr, dtype=dtype))
        if device:
            import torch
            t = torch.from_numpy(a).cuda()
            return t, t.data_ptr(), L.MEM_DEVICE
        return a, a.ctypes.data, L.MEM_HOST

    def set_source(self, src, device=True):
        keep, ptr, mem = self._buffer(src["cube"], np.float32, device)
        n_az, n_el = keep.shape[0], keep.shape[1]
        L.check(self._lib.gateau_set_source_cube(self._h, ptr, n_az, n_el, src["az0"], src["daz"], src["el0"],
                                                 src["del"], mem))

    def set_screen(self, atm, device=True):
        keep, ptr, mem = self._buffer(atm["screen"], np.float32, device)
        ny, nx = keep.shape
        L.check(self._lib.gateau_set_atmosphere_screen(self._h, ptr, nx, ny, atm["pitch"], int(atm.get("is_epl", False)),
                                                       float(atm.get("pwv0", 0.0)), mem))

    def set_table(self, atm, device=True):
        keep, ptr, mem = self._buffer(atm["table"], np.float32, device)
        L.check(self._lib.gateau_set_atmosphere_table(self._h, ptr, keep.shape[0], atm["pwv_min"], atm["dpwv"],
                                                      int(atm.get("table_is_opacity", True)), mem))

    def set_scan(self, scan, device=True):
        kind = _SCAN[scan["kind"]]
        params = _f64(scan.get("params", ()) or [0.0])
        n_params = len(scan.get("params", ()) or ())
        custom = scan.get("custom")
        if custom is not None:
            keep, ptr, mem = self._buffer(custom, np.float64, device)
            n_custom = keep.shape[0]
        else:
            keep, ptr, mem, n_custom = None, None, L.MEM_HOST, 0
        L.check(self._lib.gateau_set_scan(self._h, kind, _dptr(params), n_params, scan["phi0"], scan["theta0"], ptr,
                                          n_custom, mem))

    # ---------------------------------------------------------------- running
    def prepare(self):
        """Build and upload everything derived from the setters (gateau_plan_prepare)."""
        L.check(self._lib.gateau_plan_prepare(self._h))

    def run(self, t0: int, nt: int, out=None, stream=None):
        """Enqueue samples [t0, t0+nt) into a device tensor [nt, n_pix, n_ch] (float32, W)."""
        import torch
        if out is None:
            out = torch.empty((nt, self.n_pix, self.n_ch), dtype=torch.float32, device="cuda")
        s = stream if stream is not None else torch.cuda.current_stream()
        L.check(self._lib.gateau_run(self._h, t0, nt, out.data_ptr(), C.c_void_p(s.cuda_stream)))
        return out

    def run_host(self, t0: int, nt: int, out: np.ndarray | None = None, stream=None):
        """Simulate into host memory (numpy float32 [nt, n_pix, n_ch]); returns when complete."""
        import torch
        if out is None:
            out = np.empty((nt, self.n_pix, self.n_ch), dtype=np.float32)
        s = stream if stream is not None else torch.cuda.current_stream()
        L.check(self._lib.gateau_run_host(self._h, t0, nt, out.ctypes.data, C.c_void_p(s.cuda_stream)))
        return out

    def mean_zenith_pwv(self, n_total: int) -> float:
        """Zenith PWV averaged over the observation's first n_total samples (Sect. 4.3)."""
        v = C.c_double(0.0)
        L.check(self._lib.gateau_mean_zenith_pwv(self._h, int(n_total), C.byref(v)))
        return v.value

    def common_mode(self, t0: int, tb, pwv_mean: float, r_out: float, out=None, stream=None):
        """Common-mode reduction (Eqs. 25-26) of a device TOD tb [nt, n_pix, n_ch] in K."""
        import torch
        assert tb.is_cuda and tb.dtype == torch.float32 and tb.is_contiguous()
        if out is None:
            out = torch.empty_like(tb)
        s = stream if stream is not None else torch.cuda.current_stream()
        L.check(self._lib.gateau_common_mode(self._h, int(t0), int(tb.shape[0]), tb.data_ptr(), out.data_ptr(),
                                             float(pwv_mean), float(r_out), C.c_void_p(s.cuda_stream)))
        return out

    def status(self) -> int:
        flags = C.c_uint(0)
        L.check(self._lib.gateau_plan_status(self._h, C.byref(flags)))
        return flags.value

    def info(self) -> L.PlanInfo:
        info = L.PlanInfo()
        L.check(self._lib.gateau_plan_get_info(self._h, C.byref(info)))
        return info

    def get_vector(self, which: int, size: int) -> np.ndarray:
        out = np.empty(size, dtype=np.float64)
        L.check(self._lib.gateau_plan_get_vector(self._h, which, _dptr(out), size))
        return out

    def get_state(self):
        info = self.info()
        st = np.empty((self.n_pix, self.n_ch, info.n_pole), dtype=np.float64)
        t0 = C.c_longlong(0)
        L.check(self._lib.gateau_plan_get_state(self._h, C.byref(t0), _dptr(st)))
        return t0.value, st

    def set_state(self, next_t0: int, pink_state=None):
        ptr = _dptr(_f64(pink_state)) if pink_state is not None else None
        keep = _f64(pink_state) if pink_state is not None else None
        if keep is not None:
            ptr = _dptr(keep)
        L.check(self._lib.gateau_plan_set_state(self._h, next_t0, ptr))

    def set_tiles(self, n_groups: int = 0, ring_b: int = 0):
        """Fused-kernel tiles: channel groups (0: the fewest) and the deepest B ring (0: the default)."""
        L.check(self._lib.gateau_plan_set_tiles(self._h, int(n_groups), int(ring_b)))

    def autotune(self, nt_sample: int = 1024, stream=None) -> dict:
        """Time the candidate tiles on the first nt_sample samples and keep the fastest (cached per
        shape class for the process).  Returns the choice."""
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        ch = L.TileChoice()
        L.check(self._lib.gateau_plan_autotune(self._h, int(nt_sample), C.c_void_p(s.cuda_stream), C.byref(ch)))
        return {f: getattr(ch, f) for f, _ in L.TileChoice._fields_}

    def set_wait_budget(self, cycles: int):
        """Budget of each pipeline wait of the fused kernel in SM clock cycles (default 4e9)."""
        L.check(self._lib.gateau_plan_set_wait_budget(self._h, int(cycles)))

    def set_timing(self, enable: bool = True):
        L.check(self._lib.gateau_plan_set_timing(self._h, 1 if enable else 0))

    def get_timing(self):
        """(ms per phase [rows, spectrum, contract, pink], runs, kernel launches) since the last call."""
        ms = np.zeros(L.PHASE_COUNT, dtype=np.float64)
        runs, launches = C.c_longlong(0), C.c_longlong(0)
        L.check(self._lib.gateau_plan_get_timing(self._h, _dptr(ms), C.byref(runs), C.byref(launches)))
        return ms, runs.value, launches.value

    def close(self):
        if self._h:
            self._lib.gateau_plan_destroy(self._h)
            self._h = L.PlanP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def run_batch(plans, t0s, nts, outs=None, stream=None):
    """gateau_run_batch: every plan's chunk [t0, t0 + nt) in one batch on one stream; the split-BF16
    contractions share persistent fused launches.  Returns the device output tensors."""
    import torch
    n = len(plans)
    if outs is None:
        outs = [torch.empty((nt, p.n_pix, p.n_ch), dtype=torch.float32, device="cuda") for p, nt in zip(plans, nts)]
    s = stream if stream is not None else torch.cuda.current_stream()
    hp = (L.PlanP * n)(*[p._h for p in plans])
    a0 = (C.c_longlong * n)(*[int(t) for t in t0s])
    an = (C.c_longlong * n)(*[int(t) for t in nts])
    ao = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
    L.check(L.lib().gateau_run_batch(hp, a0, an, ao, n, C.c_void_p(s.cuda_stream)))
    return outs


def hex_offsets(R_hex: int, spacing_rad: float) -> np.ndarray:
    n = 1 + 3 * R_hex * (R_hex + 1)
    out = np.empty((n, 2), dtype=np.float64)
    n_out = C.c_int(0)
    L.check(L.lib().gateau_hex_offsets(R_hex, spacing_rad, _dptr(out), n, C.byref(n_out)))
    return out
