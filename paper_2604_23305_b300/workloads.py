"""Seeded synthetic inputs shaped like the paper's workloads.

This module only *makes input data*: it holds none of the simulator's
arithmetic (no cascade, no filter curves, no noise model).  It is the one
module that both the CUDA path's callers and the FP64 oracle's callers use,
so that both sides see byte-identical inputs.  It imports nothing else from
this package.

The paper's real inputs (ARIS screens, ATM tables, the DESHIMA 2.0 / TIFUUN
instruments, radiobear and MockSZ sources) are not available; each is replaced
by a seeded stand-in with the same shapes and magnitudes:

* zenith opacity table: tau(PWV, nu) = tau_dry(nu) + PWV kappa(nu) (1 + 0.05 PWV)
  from pressure-broadened lines at the H2O (183.31, 325.15, 380.20, 448.00,
  556.94 GHz) and O2 (118.75, 368.50, 424.76 GHz) frequencies plus a nu^2
  continuum, scaled so that exp(-tau) = 0.9 at PWV = 1 mm, 350 GHz;
  PWV rows 0..5 mm in 0.01 mm steps (501 rows);
* PWV screen: periodic Gaussian random field with a Kolmogorov k^(-11/3)
  spectrum, smoothed by a 10 m FWHM Gaussian (a 10 m dish footprint),
  0.5 m pitch, given mean and rms;
* source cubes: a beam-sized point source (single-pixel configs) or an
  isothermal-beta-like blob (IFU configs), in W/Hz, already beam-convolved;
* cascades: Table 1 style stages (spillover, Ohmic-Al, sky-coupled secondary
  spillover, warm optics, AR-coated window, cold lens).
"""
from __future__ import annotations

import math

import numpy as np

ARCSEC = math.pi / (180.0 * 3600.0)
DEG = math.pi / 180.0
GHZ = 1e9
EV = 1.602176634e-19

# Parameter values that follow the paper's DESHIMA 2.0 / ASTE model (Sect. 3.1, Table 1).
ASTE = dict(eta_taper=0.85, rho_surf=42e-6, eta_pol=0.5, T_atm=273.0, h_column=1537.0,
            T_cmb=2.725, delta_al=188e-6 * EV, eta_pb=0.4)

H2O_LINES_GHZ = (183.31, 325.15, 380.20, 448.00, 556.94)
O2_LINES_GHZ = (118.75, 368.50, 424.76)


def geometric_channels(f_lo_hz: float, f_hi_hz: float, n_ch: int) -> np.ndarray:
    """Channel centres log-spaced from f_lo to f_hi, both included."""
    if n_ch == 1:
        return np.array([math.sqrt(f_lo_hz * f_hi_hz)])
    return f_lo_hz * (f_hi_hz / f_lo_hz) ** (np.arange(n_ch) / (n_ch - 1.0))


def half_power_channels(f_lo_hz: float, f_hi_hz: float, R: float) -> np.ndarray:
    """Channel centres f_{j+1} = f_j (1 + 1/R) from f_lo while <= f_hi."""
    out = [f_lo_hz]
    while out[-1] * (1.0 + 1.0 / R) <= f_hi_hz * (1 + 1e-12):
        out.append(out[-1] * (1.0 + 1.0 / R))
    return np.array(out)


def grid_offsets(n_side: int, pitch_rad: float) -> np.ndarray:
    """n_side x n_side square spaxel grid centred on broadside, [n_pix, 2] (dphi, dtheta)."""
    c = (np.arange(n_side) - 0.5 * (n_side - 1)) * pitch_rad
    dphi, dth = np.meshgrid(c, c, indexing="xy")
    return np.stack([dphi.ravel(), dth.ravel()], axis=1)


def opacity_table(nu_hz: np.ndarray, n_pwv: int = 501, pwv_min: float = 0.0,
                  dpwv: float = 0.01) -> tuple[np.ndarray, float, float]:
    """Synthetic zenith opacity tau[n_pwv, n_freq] (float32) and its PWV grid."""
    f = nu_hz / GHZ
    gamma = 3.0

    def lines(centres, strengths):
        s = np.zeros_like(f)
        for c, a in zip(centres, strengths):
            s += a * gamma ** 2 / ((f - c) ** 2 + gamma ** 2)
        return s

    kappa = lines(H2O_LINES_GHZ, (0.8, 4.0, 6.0, 9.0, 40.0)) + 0.02 * (f / 300.0) ** 2
    tau_dry = lines(O2_LINES_GHZ, (1.5, 0.4, 0.6)) + 0.01 * (f / 300.0) ** 2
    # Scale so that exp(-tau) = 0.9 at 1 mm, 350 GHz.
    k350 = np.interp(350.0, f, kappa) if f.min() <= 350 <= f.max() else 0.1
    d350 = np.interp(350.0, f, tau_dry) if f.min() <= 350 <= f.max() else 0.0
    target = -math.log(0.9)
    scale = (target - d350) / (k350 * 1.05) if k350 > 0 else 1.0
    pwv = pwv_min + dpwv * np.arange(n_pwv)
    tab = tau_dry[None, :] + pwv[:, None] * (scale * kappa)[None, :] * (1.0 + 0.05 * pwv[:, None])
    return tab.astype(np.float32), pwv_min, dpwv


def pwv_screen(nx: int, ny: int, pitch_m: float, mean_mm: float, rms_mm: float,
               seed: int) -> np.ndarray:
    """Periodic Kolmogorov Gaussian random field [ny, nx] (float32, mm)."""
    rng = np.random.default_rng(seed)
    kx = np.fft.fftfreq(nx, d=pitch_m)
    ky = np.fft.fftfreq(ny, d=pitch_m)
    KX, KY = np.meshgrid(kx, ky, indexing="xy")
    k2 = KX ** 2 + KY ** 2
    k2[0, 0] = np.inf
    amp = k2 ** (-11.0 / 12.0)                       # sqrt of k^(-11/3)
    fwhm = 10.0
    s = fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    amp *= np.exp(-2.0 * math.pi ** 2 * s ** 2 * np.where(np.isinf(k2), 0.0, k2))
    noise = rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))
    field = np.real(np.fft.ifft2(noise * amp))
    field -= field.mean()
    field *= rms_mm / field.std()
    return (field + mean_mm).astype(np.float32)


def point_source_cube(nu_hz, n_az, n_el, half_extent_rad, el_centre_rad, T_peak_K=2.0,
                      dish_m=10.0):
    """Beam-convolved point source: Gaussian of FWHM 1.2 lambda/D at every nu, peak k_B T_peak."""
    k_b = 1.380649e-23
    az = np.linspace(-half_extent_rad, half_extent_rad, n_az)
    el = np.linspace(-half_extent_rad, half_extent_rad, n_el)
    A, E = np.meshgrid(az, el, indexing="ij")
    r2 = A ** 2 + E ** 2
    fwhm = 1.2 * (299792458.0 / nu_hz) / dish_m
    s2 = (fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))) ** 2
    cube = k_b * T_peak_K * np.exp(-0.5 * r2[:, :, None] / s2[None, None, :])
    grid = dict(az0=-half_extent_rad, daz=2 * half_extent_rad / (n_az - 1),
                el0=el_centre_rad - half_extent_rad, d_el=2 * half_extent_rad / (n_el - 1))
    return cube.astype(np.float32), grid


def blob_source_cube(nu_hz, n_az, n_el, half_extent_rad, el_centre_rad, T_peak_K=0.05,
                     core_rad=40.71 * ARCSEC, beta=0.73):
    """Extended isothermal-beta-like blob times a smooth rising spectrum, peak ~k_B T_peak."""
    k_b = 1.380649e-23
    az = np.linspace(-half_extent_rad, half_extent_rad, n_az)
    el = np.linspace(-half_extent_rad, half_extent_rad, n_el)
    A, E = np.meshgrid(az, el, indexing="ij")
    prof = (1.0 + (A ** 2 + E ** 2) / core_rad ** 2) ** (0.5 - 1.5 * beta)
    x = nu_hz / (300.0 * GHZ)
    spec = x ** 2 / (1.0 + 0.3 * x ** 2)
    cube = (k_b * T_peak_K) * prof[:, :, None] * spec[None, None, :]
    grid = dict(az0=-half_extent_rad, daz=2 * half_extent_rad / (n_az - 1),
                el0=el_centre_rad - half_extent_rad, d_el=2 * half_extent_rad / (n_el - 1))
    return cube.astype(np.float32), grid


def table1_cascade() -> list[dict]:
    """Six stages in the style of Table 1 (T 4-290 K, eta 0.5-0.99)."""
    return [
        dict(kind="reflective", eta=0.99, T=273.0),                         # primary spillover
        dict(kind="ohmic", eps_ref=0.0025, nu_ref=840 * GHZ, T=273.0),      # Ohmic-Al
        dict(kind="reflective", eta=0.85, T="sky"),                         # secondary spillover
        dict(kind="reflective", eta=0.99, T=290.0),                         # warm optics
        dict(kind="refractive", d=4e-3, n=3.41, tan_delta=1e-4, T=290.0,    # AR-coated window
             ar=True),
        dict(kind="reflective", eta=0.7, T=4.0),                            # cold leaky lens
    ]


def three_stage_cascade() -> list[dict]:
    return [dict(kind="reflective", eta=0.99, T=273.0),
            dict(kind="reflective", eta=0.85, T="sky"),
            dict(kind="reflective", eta=0.7, T=4.0)]


def pink_levels(n_ch: int, seed: int, nep_ref=1e-17):
    """Per-channel pink level A (W^2/Hz at 1 Hz) and slope alpha ~ U[0.5, 1.5].  The scenarios give
    only the slopes: with no level the knee sits at 1 Hz (the simulator sets A to each channel's
    white noise level); explicit levels remain for tests."""
    rng = np.random.default_rng(seed)
    A = (nep_ref ** 2) * rng.uniform(0.5, 2.0, n_ch)
    alpha = rng.uniform(0.5, 1.5, n_ch)
    return A, alpha


def _base(n_freq, f_lo, f_hi, f_sample, offsets, nt_total):
    sc = dict(f_lo=f_lo, f_hi=f_hi, n_freq=n_freq, f_sample=f_sample,
              pix_offsets=np.asarray(offsets, dtype=np.float64), nt_total=int(nt_total))
    sc.update({k: ASTE[k] for k in ("T_cmb", "eta_taper", "rho_surf", "eta_pol",
                                     "delta_al", "eta_pb")})
    return sc


def scenario(name: str, nt_total: int | None = None, seed: int = 0, noise_seed: int = 1):
    """The named synthetic workloads.

    single_pixel_small : 1 spaxel, 64 filterbank channels R=300 on 512 points
                         220-440 GHz, 1000 samples at 160 Hz, 256^2 screen
                         (mean 1 mm, 10 m/s wind), 3 stages, stare at el 60 deg.
    single_pixel_wide  : 1 spaxel, 347 channels R=500 log-spaced 220-440 GHz on
                         3000 points, 10 min at 160 Hz, 6 stages, daisy scan
                         (r=65", omega=2 pi 1.54/s, Omega=omega/50) on a
                         64x64x3000 point-source cube, pink noise.
    ifu25              : 5x5 spaxels at 15", 347 channels, 3000 points, 20 min
                         raster at 160 Hz, 1024^2 screen, 128x128x3000 blob cube.
    """
    if name == "single_pixel_small":
        n_freq, f_lo, f_hi, fs = 512, 220 * GHZ, 440 * GHZ, 160.0
        nt = 1000 if nt_total is None else nt_total
        sc = _base(n_freq, f_lo, f_hi, fs, np.zeros((1, 2)), nt)
        nu = np.linspace(f_lo, f_hi, n_freq)
        tab, pmin, dp = opacity_table(nu)
        screen = pwv_screen(256, 256, 0.5, 1.0, 0.02, seed)
        cube, grid = point_source_cube(nu, 32, 32, 70 * ARCSEC, 60 * DEG)
        f_c = geometric_channels(f_lo, f_hi, 64)
        sc.update(
            atmosphere=dict(screen=screen, pitch=0.5, is_epl=False, pwv0=0.0,
                            h_column=ASTE["h_column"], wind=10.0, T_atm=ASTE["T_atm"],
                            table=tab, table_is_opacity=True, pwv_min=pmin, dpwv=dp),
            source=dict(cube=cube, az0=grid["az0"], daz=grid["daz"], el0=grid["el0"],
                        **{"del": grid["d_el"]}),
            scan=dict(kind="stare", params=(), phi0=0.0, theta0=60 * DEG),
            cascade=three_stage_cascade(),
            dispersive=dict(kind="filterbank", f_c=f_c, R=np.full(64, 300.0),
                            eta_peak=np.full(64, 0.16)),
        )
        _, alpha = pink_levels(64, seed + 7)
        sc["noise"] = dict(seed=noise_seed, pink_A=None, pink_alpha=alpha, pink_f_min=fs / nt)
        return sc
    if name in ("single_pixel_wide", "ifu25"):
        n_freq, f_lo, f_hi, fs = 3000, 220 * GHZ, 440 * GHZ, 160.0
        nu = np.linspace(f_lo, f_hi, n_freq)
        f_c = geometric_channels(f_lo, f_hi, 347)
        tab, pmin, dp = opacity_table(nu)
        _, alpha = pink_levels(347, seed + 7)
        if name == "single_pixel_wide":
            nt = 96000 if nt_total is None else nt_total
            sc = _base(n_freq, f_lo, f_hi, fs, np.zeros((1, 2)), nt)
            screen = pwv_screen(512, 512, 0.5, 1.0, 0.02, seed)
            cube, grid = point_source_cube(nu, 64, 64, 70 * ARCSEC, 47.8 * DEG)
            w = 2 * math.pi * 1.54
            scan = dict(kind="daisy", params=(65 * ARCSEC, w, w / 50.0), phi0=0.0,
                        theta0=47.8 * DEG)
            f_min = 1.0 / 600.0
        else:
            nt = 192000 if nt_total is None else nt_total
            sc = _base(n_freq, f_lo, f_hi, fs, grid_offsets(5, 15 * ARCSEC), nt)
            screen = pwv_screen(1024, 1024, 0.5, 0.9, 0.02, seed)
            cube, grid = blob_source_cube(nu, 128, 128, 210 * ARCSEC, 47.8 * DEG)
            scan = dict(kind="raster", params=(180 * ARCSEC, 30 * ARCSEC, 15 * ARCSEC, 25),
                        phi0=0.0, theta0=47.8 * DEG)
            f_min = 1.0 / 1200.0
        sc.update(
            atmosphere=dict(screen=screen, pitch=0.5, is_epl=False, pwv0=0.0,
                            h_column=ASTE["h_column"], wind=10.0, T_atm=ASTE["T_atm"],
                            table=tab, table_is_opacity=True, pwv_min=pmin, dpwv=dp),
            source=dict(cube=cube, az0=grid["az0"], daz=grid["daz"], el0=grid["el0"],
                        **{"del": grid["d_el"]}),
            scan=scan,
            cascade=table1_cascade(),
            dispersive=dict(kind="filterbank", f_c=f_c, R=np.full(347, 500.0),
                            eta_peak=np.full(347, 0.16)),
        )
        sc["noise"] = dict(seed=noise_seed, pink_A=None, pink_alpha=alpha, pink_f_min=f_min)
        return sc
    raise ValueError(f"unknown scenario {name!r}")


def detector_samples(sc: dict, nt: int | None = None) -> int:
    n = sc["nt_total"] if nt is None else nt
    return int(n) * int(np.asarray(sc["pix_offsets"]).shape[0]) * int(np.asarray(sc["dispersive"]["f_c"]).size)
