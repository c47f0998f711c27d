"""FP64 CPU oracle for the gateau time-ordered-data hot path (arXiv 2604.23305).

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain reference that the
CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
It shares no code with ``paper_2604_23305_b300`` (neither imports the other);
the only common inputs come from the seeded generators in
``paper_2604_23305_b300/workloads.py``, which hold none of the method's
arithmetic.

Every function evaluates the paper's equations literally, in SI units and
float64, stage by stage, with no algebraic collapse, blocking or fusion:

  * preprocessing (source, screen) -- Sect. 2.2, Eqs. 1-3: aperture illumination,
                                      far field |FFT(A)|^2, beam convolution of the
                                      source cube, footprint smoothing of the screen
  * scan and pointing              -- Sect. 2.4, Eq. 8 (daisy) and the text after it
  * screen coordinates + PWV       -- Sect. 2.4, Eq. 9 (frozen flow) + bilinear lookup
  * zenith transmission + airmass  -- Sect. 2.4, Eq. 10
  * source sampling                -- Sect. 2.4 (bilinear, zero outside the grid)
  * radiative-transfer cascade     -- Sect. 2.5, Eqs. 11-15 and the sky-coupled stage
  * dispersive element             -- Sect. 2.3, Eqs. 6-7 (+ the 2*Delta_Al/h cutoff)
  * KID power                      -- Sect. 2.5, Eq. 16
  * photon noise                   -- Sect. 2.6, Eqs. 17-19
  * pink noise                     -- Sect. 2.6, Eq. 20 (pole-zero IIR reading, or the
                                      exact Timmer & Koenig realisation over the whole scan)
  * total                          -- Sect. 2.7, Eq. 21
  * brightness-temperature output  -- Sect. 2.7 (simulated skydip, linear P -> T_b map)
  * common-mode reduction          -- Sect. 4.3, Eqs. 25-26 (downstream of the TOD)

Readings of points the paper leaves silent or garbled (each also listed in the
design notes of the repository):
  * Eq. 6 prints ``eta_peak / (4R^2 (nu/f-1)^2)``; the Lorentzian with
    full width f/R is ``eta_peak / (1 + 4R^2 (nu/f-1)^2)``; Eq. 7 likewise.
  * Eq. 5 prints ``exp(-(4 pi rho/lambda))^2``; Ruze's law is
    ``exp(-(4 pi rho/lambda)^2)``.
  * The single-mode Johnson-Nyquist power (Sect. 2.5) is
    ``h nu / (exp(h nu / k T) - 1)`` (no zero-point term).
  * Integrals over nu (Eqs. 16-17) are trapezoid sums on the uniform grid.
  * The zenith table is interpolated linearly in opacity ``tau = -ln eta``
    between PWV grid rows; PWV is clamped to the table range.
  * The screen is periodic; screen cell (0, 0) sits at x = -nx/2 * pitch,
    y = -ny/2 * pitch, i.e. the telescope looks at the screen centre at t=0.
  * Eq. 9 uses phi(t), theta(t) without the scan offset (literal); the
    airmass (Eq. 10) uses theta(t) + theta_0 + dtheta_i (literal).
  * The source cube is inside iff 0 <= u <= n_az-1 and 0 <= v <= n_el-1 in
    fractional grid units; the cell index is min(floor(u), n-2).
  * Sky-coupled stages use the same spaxel's and time's eta_atm.
  * Random numbers: Philox4x32-10 (Salmon et al., SC'11) keyed by the seed,
    with the counter layout of ``white_normals`` / ``pink_normals``, turned
    into normals by the Box-Muller transform.
  * Pink noise: Timmer & Koenig (1995) needs the whole scan at once, which a
    chunked simulator cannot have.  The reading used here is a causal
    pole-zero filter whose power response follows A f^-alpha: poles at
    f_min*10^(j/3) (3 per decade, up to f_s/2), zeros a factor 10^(alpha/6)
    above each pole, matched-z mapping, gain set so that the one-sided PSD at
    1 Hz equals A, zero state at the first sample of the scan (n = 0).
    The exact Timmer & Koenig realisation is also provided for a scan of known
    length N: Fourier coefficients of a real series of length M = 2^ceil(log2 N)
    (the first N samples are used) with Gaussian real and imaginary parts of
    variance M f_s S(f_j) / 4 at f_j = j f_s / M, 0 < j < M/2, a real Nyquist
    coefficient of variance M f_s S / 2, no DC term, S(f) = A f^-alpha the
    one-sided PSD, and x_n = (1/M) sum_j X_j e^{2 pi i j n / M}.  Its normals
    come from Philox with counter (q lo, q hi, i, 2^30 | ch), q = j >> 1; bin j
    takes Box-Muller pair j & 1 as (re, im).
  * Aperture illumination (Eq. 2, garbled in print): a Gaussian whose amplitude
    falls to t_edge dB at the rim, A(r) = 10^((t_edge / 20) (r / R)^2) for
    r = lambda sqrt(l^2 + m^2) < R, zero outside.  The far field (Eq. 3) is the
    2-D DFT of A sampled in wavelengths with spacing 1 / (N pitch), so that the
    pattern comes out on the angular grid of pitch `pitch` (offset q pitch at
    index q mod N), |.|^2 normalised to a peak of 1.  Eq. 1 is evaluated as the
    discrete linear convolution on the cube's grid, sum over cells of
    I cos(theta') F (phi - phi', theta - theta') dphi dtheta, times A_p = pi R^2.
    The screen is smoothed (periodically) by A(r) on the screen grid in metres,
    normalised to unit sum.
  * Skydip (Sect. 2.7): the PWV is varied over n uniformly spaced zenith values
    pwv_lo .. pwv_hi at the scan's base elevation theta_0, with no source and
    no noise (the recorded power is the noise-free P_KID, the mean of
    P_tot).  T_b of a channel is the line-of-sight brightness temperature of
    the isothermal atmosphere, T_atm (1 - eta_atm), averaged over the band
    with the channel's weights eta_filt * w.  The map T_b = a P + b is the
    ordinary least-squares line through the n points, and it is applied to
    the total power P_tot of every sample.
  * Common-mode reduction (Eqs. 25-26): the zenith PWV averaged over the
    observation is the mean of the line-of-sight-screen PWV over every row
    (n, i) of the scan; eta_atm,z of a channel is the zenith transmission at
    that PWV averaged over the band with the channel's weights eta_filt w (as
    T_b is); eta_atm,i(t) = eta_atm,z^csc(el_i(t)) with the spaxel's own
    elevation (Eq. 10); S_j uses the spaxel offsets (dphi_j, dtheta_j).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# CODATA 2018 exact SI constants.
H_PLANCK = 6.62607015e-34      # J s
K_BOLTZMANN = 1.380649e-23     # J / K
C_LIGHT = 299792458.0          # m / s
E_CHARGE = 1.602176634e-19     # J / eV

F64 = np.float64


# ---------------------------------------------------------------------------
# Preprocessing: beam far field, source convolution, screen smoothing (Sect. 2.2, Eqs. 1-3)
# ---------------------------------------------------------------------------

def aperture_illumination(r_m, R_tel_m: float, t_edge_db: float):
    """Amplitude 10^((t_edge/20) (r/R)^2) inside the rim (r < R), zero outside (Eq. 2 reading)."""
    r = np.asarray(r_m, dtype=F64)
    return np.where(r < R_tel_m, 10.0 ** ((t_edge_db / 20.0) * (r / R_tel_m) ** 2), 0.0)


def _fft_offsets(n: int) -> np.ndarray:
    """Index q of an n-point DFT <-> signed offset q for q < n/2, q - n above."""
    q = np.arange(n)
    return np.where(q < n // 2, q, q - n).astype(F64)


def beam_far_field(nu_hz: float, n_a: int, n_e: int, d_az: float, d_el: float, R_tel_m: float, t_edge_db: float):
    """F(q d_az, p d_el) at index (q mod n_a, p mod n_e), peak 1 (Eq. 3): |DFT of A(l, m)|^2 with l, m
    in wavelengths on spacings 1 / (n_a d_az), 1 / (n_e d_el)."""
    lam = C_LIGHT / nu_hz
    l = _fft_offsets(n_a) / (n_a * d_az)
    m = _fft_offsets(n_e) / (n_e * d_el)
    Lg, Mg = np.meshgrid(l, m, indexing="ij")
    A = aperture_illumination(lam * np.hypot(Lg, Mg), R_tel_m, t_edge_db)
    F = np.abs(np.fft.fft2(A)) ** 2
    return F / F.max()


def convolve_source(I_cube: np.ndarray, nu_hz: np.ndarray, el0_rad: float, d_az: float, d_el: float,
                    R_tel_m: float, t_edge_db: float) -> np.ndarray:
    """P_src[a][e][nu] = A_p sum_{a', e'} I[a'][e'][nu] cos(el_e') F_nu(a - a', e - e') d_az d_el (Eq. 1),
    the beam on the grid of offsets from beam_far_field at twice the cube size (linear convolution)."""
    I_cube = np.asarray(I_cube, dtype=F64)
    n_az, n_el, n_f = I_cube.shape
    el = el0_rad + d_el * np.arange(n_el)
    A_p = math.pi * R_tel_m ** 2
    out = np.empty_like(I_cube)
    for k in range(n_f):
        F = beam_far_field(float(nu_hz[k]), 2 * n_az, 2 * n_el, d_az, d_el, R_tel_m, t_edge_db)
        src = np.zeros((2 * n_az, 2 * n_el))
        src[:n_az, :n_el] = I_cube[:, :, k] * np.cos(el)[None, :]
        conv = np.real(np.fft.ifft2(np.fft.fft2(src) * np.fft.fft2(F)))
        out[:, :, k] = A_p * d_az * d_el * conv[:n_az, :n_el]
    return out


def smooth_screen(screen: np.ndarray, pitch_m: float, R_tel_m: float, t_edge_db: float) -> np.ndarray:
    """Periodic convolution of the screen [ny][nx] with the illumination footprint A(r), r in metres on
    the screen grid, normalised to unit sum (line-of-sight PWV, Sect. 2.2)."""
    s = np.asarray(screen, dtype=F64)
    ny, nx = s.shape
    X, Y = np.meshgrid(_fft_offsets(nx) * pitch_m, _fft_offsets(ny) * pitch_m, indexing="xy")
    K = aperture_illumination(np.hypot(X, Y), R_tel_m, t_edge_db)
    K = K / K.sum()
    return np.real(np.fft.ifft2(np.fft.fft2(s) * np.fft.fft2(K)))


# ---------------------------------------------------------------------------
# Frequency grid and integration weights (Sect. 2.5, Eq. 16)
# ---------------------------------------------------------------------------

def frequency_grid(f_lo_hz: float, f_hi_hz: float, n_freq: int) -> np.ndarray:
    """Uniform grid, both end points included."""
    return np.linspace(F64(f_lo_hz), F64(f_hi_hz), int(n_freq), dtype=F64)


def trapezoid_weights(nu: np.ndarray) -> np.ndarray:
    """Trapezoid-rule weights w_k on a uniform grid, so that sum_k w_k g_k ~ int g dnu."""
    n = nu.size
    if n < 2:
        raise ValueError("need at least two frequency points")
    dnu = (nu[-1] - nu[0]) / (n - 1)
    w = np.full(n, dnu, dtype=F64)
    w[0] = w[-1] = 0.5 * dnu
    return w


# ---------------------------------------------------------------------------
# Radiometric building blocks (Sects. 2.3 and 2.5)
# ---------------------------------------------------------------------------

def johnson_nyquist(T_K, nu_hz):
    """Single-mode Johnson-Nyquist spectral power h nu / (exp(h nu/kT) - 1), W/Hz (Sect. 2.5)."""
    T = np.asarray(T_K, dtype=F64)
    nu = np.asarray(nu_hz, dtype=F64)
    out = np.zeros(np.broadcast(T, nu).shape, dtype=F64)
    Tb, nub = np.broadcast_arrays(T, nu)
    hot = Tb > 0
    x = H_PLANCK * nub[hot] / (K_BOLTZMANN * Tb[hot])
    with np.errstate(over="ignore"):
        out[hot] = H_PLANCK * nub[hot] / np.expm1(x)
    return out


def ruze_efficiency(rho_surf_m: float, nu_hz):
    """Ruze surface efficiency exp(-(4 pi rho / lambda)^2) (Sect. 2.3, Eq. 5)."""
    lam = C_LIGHT / np.asarray(nu_hz, dtype=F64)
    return np.exp(-(4.0 * np.pi * rho_surf_m / lam) ** 2)


def ohmic_efficiency(eps_ref: float, nu_ref_hz: float, nu_hz):
    """Ohmic reflector efficiency 1 - eps_ref sqrt(nu/nu_ref) (Sect. 2.5, Eq. 13)."""
    return 1.0 - eps_ref * np.sqrt(np.asarray(nu_hz, dtype=F64) / nu_ref_hz)


def refraction_efficiency(d_m: float, n_index: float, tan_delta: float, nu_hz):
    """Dielectric bulk transmission exp(-2 pi d n tan(delta) / lambda) (Sect. 2.5, Eq. 14)."""
    lam = C_LIGHT / np.asarray(nu_hz, dtype=F64)
    return np.exp(-2.0 * np.pi * d_m * n_index * tan_delta / lam)


def reflection_efficiency(n_index: float) -> float:
    """Normal-incidence surface transmission 1 - ((1-n)/(1+n))^2 (Sect. 2.5, Eq. 15)."""
    return 1.0 - ((1.0 - n_index) / (1.0 + n_index)) ** 2


# ---------------------------------------------------------------------------
# Cascade description -> list of primitive stages (Sect. 2.5)
# ---------------------------------------------------------------------------
# A stage is a dict with "kind" in {"reflective", "ohmic", "refractive"} and
#   reflective: "eta" (scalar or array over nu), "T" (K, or "sky")
#   ohmic:      "eps_ref", "nu_ref" (Hz), "T"
#   refractive: "d" (m), "n", "tan_delta", "T" (dielectric), "T_refl"
#               (surroundings seen in reflection, default T), "ar" (bool)
# A primitive stage is (eta[nu], T) with T a float or the string "sky".

SKY = "sky"


def expand_stage(stage: dict, nu: np.ndarray) -> list[tuple[np.ndarray, object]]:
    kind = stage["kind"]
    T = stage.get("T")
    if kind == "reflective":
        eta = np.broadcast_to(np.asarray(stage["eta"], dtype=F64), nu.shape).copy()
        return [(eta, T)]
    if kind == "ohmic":
        return [(ohmic_efficiency(stage["eps_ref"], stage["nu_ref"], nu), T)]
    if kind == "refractive":
        # Eq. 15 on entry, Eq. 14 through the bulk, Eq. 15 on exit; an
        # anti-reflection coating removes the two surface passes.
        bulk = (refraction_efficiency(stage["d"], stage["n"], stage["tan_delta"], nu), T)
        if stage.get("ar", False):
            return [bulk]
        T_refl = stage.get("T_refl", T)
        surf = (np.full(nu.shape, reflection_efficiency(stage["n"]), dtype=F64), T_refl)
        return [surf, bulk, surf]
    raise ValueError(f"unknown stage kind {kind!r}")


def expand_cascade(stages: list[dict], nu: np.ndarray) -> list[tuple[np.ndarray, object]]:
    prim = []
    for st in stages:
        prim.extend(expand_stage(st, nu))
    return prim


# ---------------------------------------------------------------------------
# Dispersive element (Sect. 2.3, Eqs. 6-7)
# ---------------------------------------------------------------------------

def lorentzian_profile(f_c: float, R: float, nu: np.ndarray) -> np.ndarray:
    """1 / (1 + 4 R^2 (nu/f - 1)^2): unit-peak Lorentzian of full width f/R (Eq. 6)."""
    return 1.0 / (1.0 + 4.0 * R * R * (nu / f_c - 1.0) ** 2)


def kid_cutoff_hz(delta_al_J: float) -> float:
    """Photons below 2 Delta_Al / h break no Cooper pairs (Sect. 2.3)."""
    return 2.0 * delta_al_J / H_PLANCK


def filter_efficiency(kind: str, f_c, R, eta_peak, nu: np.ndarray,
                      delta_al_J: float, custom=None) -> np.ndarray:
    """eta_filt[ch, nu] for a grating ("lorentzian"), a filterbank or custom curves.

    filterbank (Eq. 7): channels are visited from the highest centre frequency
    down; each channel's numerator is eta_peak minus the sum of the curves of
    all channels with a higher centre frequency.
    """
    f_c = np.asarray(f_c, dtype=F64)
    n_ch = f_c.size
    R = np.broadcast_to(np.asarray(R, dtype=F64), (n_ch,))
    eta_peak = np.broadcast_to(np.asarray(eta_peak, dtype=F64), (n_ch,))
    if kind == "custom":
        eta = np.array(custom, dtype=F64).reshape(n_ch, nu.size)
    elif kind == "lorentzian":
        eta = np.empty((n_ch, nu.size), dtype=F64)
        for ch in range(n_ch):
            eta[ch] = eta_peak[ch] * lorentzian_profile(f_c[ch], R[ch], nu)
    elif kind == "filterbank":
        eta = np.empty((n_ch, nu.size), dtype=F64)
        upstream = np.zeros(nu.size, dtype=F64)     # sum of eta_filt with f_bar > f
        for ch in sorted(range(n_ch), key=lambda c: -f_c[c]):
            eta[ch] = (eta_peak[ch] - upstream) * lorentzian_profile(f_c[ch], R[ch], nu)
            upstream += eta[ch]
    else:
        raise ValueError(f"unknown dispersive element {kind!r}")
    eta[:, nu < kid_cutoff_hz(delta_al_J)] = 0.0
    return eta


# ---------------------------------------------------------------------------
# Spaxel layout (Sect. 2.3)
# ---------------------------------------------------------------------------

def hex_offsets(R_hex: int, spacing_rad: float) -> np.ndarray:
    """Packed hexagon of circumradius R_hex spaxels (excluding the centre), spacing along the radius.

    Ring k holds the 6k spaxels at hexagonal distance k: start from the corner
    (k*spacing, 0) and walk its six sides of k steps each, turning by 60 degrees.
    Spaxels are returned ring by ring, each ring ordered by polar angle in [0, 2 pi).
    """
    pts = [(0.0, 0.0, 0, 0.0)]
    for k in range(1, R_hex + 1):
        ring = []
        x, y = k * spacing_rad, 0.0
        for side in range(6):
            ang = math.radians(120 + 60 * side)            # direction of this side
            for _ in range(k):
                ring.append((x, y))
                x += spacing_rad * math.cos(ang)
                y += spacing_rad * math.sin(ang)
        for (x, y) in ring:
            a = math.atan2(y, x)
            pts.append((x, y, k, a + 2 * math.pi if a < 0 else a))
    pts.sort(key=lambda p: (p[2], p[3]))
    return np.array([[p[0], p[1]] for p in pts], dtype=F64)


# ---------------------------------------------------------------------------
# Scan patterns and pointing (Sect. 2.4, Eq. 8)
# ---------------------------------------------------------------------------

def scan_pattern(kind: str, params, t: np.ndarray, n_index=None, custom=None):
    """(phi(t), theta(t)) in rad.

    stare:  (0, 0).
    daisy:  Eq. 8 with params (r_petal, omega, Omega).
    raster: a user pattern (Sect. 2.4 allows any t -> (phi, theta)); params
            (half_width, speed, row_step, n_rows): boustrophedon rows in
            azimuth of period 2*half_width/speed, row k running +phi for even k
            and -phi for odd k; the row elevation walks the n_rows positions
            up and down (a triangle over k), centred on 0.
    custom: pointing table [n_total, 2] indexed by the sample number.
    """
    t = np.asarray(t, dtype=F64)
    if kind == "stare":
        return np.zeros_like(t), np.zeros_like(t)
    if kind == "daisy":
        r, w, W = (F64(p) for p in params)
        return r * np.cos(W * t) * np.sin(w * t), r * np.sin(W * t) * np.sin(w * t)
    if kind == "raster":
        half, speed, step, n_rows = F64(params[0]), F64(params[1]), F64(params[2]), int(params[3])
        T_row = 2.0 * half / speed
        k = np.floor(t / T_row)
        s = t - k * T_row
        phi = np.where(np.mod(k, 2) == 0, -half + speed * s, half - speed * s)
        if n_rows > 1:
            m = np.mod(k, 2 * (n_rows - 1))
            row = np.where(m < n_rows, m, 2 * (n_rows - 1) - m)
        else:
            row = np.zeros_like(k)
        theta = (row - 0.5 * (n_rows - 1)) * step
        return phi, theta
    if kind == "custom":
        tab = np.asarray(custom, dtype=F64)
        n = np.asarray(n_index, dtype=np.int64)
        return tab[n, 0].copy(), tab[n, 1].copy()
    raise ValueError(f"unknown scan kind {kind!r}")


# ---------------------------------------------------------------------------
# Atmosphere: screen lookup and transmission (Sect. 2.4, Eqs. 9-10; Sect. 2.2, Eq. 4)
# ---------------------------------------------------------------------------

def epl_to_pwv(epl, pwv0_mm: float):
    """PWV = EPL / 6.587 + PWV_0 (Sect. 2.2, Eq. 4)."""
    return np.asarray(epl, dtype=F64) / 6.587 + pwv0_mm


def screen_coordinates(phi_scan, theta_scan, dphi, dtheta, t, h_column_m, wind_mps):
    """Frozen-flow screen coordinates of Eq. 9 (m)."""
    x = h_column_m * np.tan(phi_scan + dphi) + wind_mps * t
    y = h_column_m * np.tan(theta_scan + dtheta)
    return x, y


def screen_bilinear(screen: np.ndarray, x, y, pitch_m: float):
    """Bilinear PWV on a periodic screen [ny, nx]; cell (0,0) at (-nx/2, -ny/2)*pitch."""
    ny, nx = screen.shape
    gx = np.mod(np.asarray(x, dtype=F64) / pitch_m + 0.5 * nx, nx)
    gy = np.mod(np.asarray(y, dtype=F64) / pitch_m + 0.5 * ny, ny)
    ix = np.floor(gx).astype(np.int64)
    iy = np.floor(gy).astype(np.int64)
    fx = gx - ix
    fy = gy - iy
    ix = np.mod(ix, nx)          # gx may round up to exactly nx
    iy = np.mod(iy, ny)
    ix1 = np.mod(ix + 1, nx)
    iy1 = np.mod(iy + 1, ny)
    s = screen.astype(F64)
    return ((1 - fx) * (1 - fy) * s[iy, ix] + fx * (1 - fy) * s[iy, ix1]
            + (1 - fx) * fy * s[iy1, ix] + fx * fy * s[iy1, ix1])


def zenith_opacity(tau_table: np.ndarray, pwv_min_mm: float, dpwv_mm: float, pwv):
    """tau_z(PWV, nu) by linear interpolation between PWV rows of the table [n_pwv, n_freq]."""
    n_pwv = tau_table.shape[0]
    u = (np.asarray(pwv, dtype=F64) - pwv_min_mm) / dpwv_mm
    u = np.clip(u, 0.0, n_pwv - 1)
    j = np.minimum(np.floor(u).astype(np.int64), n_pwv - 2)
    f = (u - j)[..., None]
    T = tau_table.astype(F64)
    return (1.0 - f) * T[j] + f * T[j + 1]


def eta_to_opacity(eta_table):
    """Convert a zenith transmission table to opacity, tau = -ln(eta) (eta floored at 1e-30)."""
    return -np.log(np.maximum(np.asarray(eta_table, dtype=F64), 1e-30))


def atmospheric_transmission(tau_z, elevation_rad):
    """eta_atm = eta_z^csc(el) with eta_z = exp(-tau_z) (Sect. 2.4, Eq. 10)."""
    eta_z = np.exp(-tau_z)
    csc = 1.0 / np.sin(np.asarray(elevation_rad, dtype=F64))
    return eta_z ** csc[..., None]


# ---------------------------------------------------------------------------
# Source sampling (Sect. 2.4)
# ---------------------------------------------------------------------------

def source_bilinear(cube: np.ndarray, az0, daz, el0, d_el, az, el):
    """Bilinear P_nu,src at pointings (az, el) from cube [n_az, n_el, n_freq]; zero outside."""
    n_az, n_el, n_f = cube.shape
    u = (np.asarray(az, dtype=F64) - az0) / daz
    v = (np.asarray(el, dtype=F64) - el0) / d_el
    inside = (u >= 0) & (u <= n_az - 1) & (v >= 0) & (v <= n_el - 1)
    out = np.zeros(u.shape + (n_f,), dtype=F64)
    if not np.any(inside):
        return out
    ui, vi = u[inside], v[inside]
    ia = np.minimum(np.floor(ui).astype(np.int64), n_az - 2)
    ie = np.minimum(np.floor(vi).astype(np.int64), n_el - 2)
    fa = (ui - ia)[:, None]
    fe = (vi - ie)[:, None]
    c = cube.astype(F64)
    out[inside] = ((1 - fa) * (1 - fe) * c[ia, ie] + fa * (1 - fe) * c[ia + 1, ie]
                   + (1 - fa) * fe * c[ia, ie + 1] + fa * fe * c[ia + 1, ie + 1])
    return out


# ---------------------------------------------------------------------------
# Radiative-transfer cascade, literal stage by stage (Sect. 2.5, Eqs. 11-12)
# ---------------------------------------------------------------------------

def cascade(P_src, eta_atm, nu, prim_stages, T_atm, T_cmb, eta_taper, eta_surf, eta_pol):
    """Spectral power after the last stage, P_nu (W/Hz), for rows of P_src [rows, nu].

    Eq. 11 forms P_0; stage 0 is the atmosphere (eta_0 = eta_atm, T_0 = T_atm);
    every further primitive stage applies Eq. 12 with its own temperature, or,
    for a sky-coupled stage, with (1 - eta_atm) B(T_atm) + eta_atm B(T_cmb).
    """
    B_cmb = johnson_nyquist(T_cmb, nu)
    B_atm = johnson_nyquist(T_atm, nu)
    P = eta_taper * eta_surf * eta_pol * P_src + B_cmb                       # Eq. 11
    P = eta_atm * P + (1.0 - eta_atm) * B_atm                                # Eq. 12, k = 0
    for eta_k, T_k in prim_stages:                                           # Eq. 12, k >= 1
        if isinstance(T_k, str) and T_k == SKY:
            B_k = (1.0 - eta_atm) * B_atm + eta_atm * B_cmb
        else:
            B_k = johnson_nyquist(T_k, nu)
        P = eta_k * P + (1.0 - eta_k) * B_k
    return P


# ---------------------------------------------------------------------------
# Detector power and photon noise (Sect. 2.5 Eq. 16; Sect. 2.6 Eqs. 17-18)
# ---------------------------------------------------------------------------

def kid_power(eta_filt, w, P):
    """P_KID[row, ch] = int eta_filt(f, nu) P_nu dnu as a trapezoid sum (Eq. 16)."""
    return P @ (eta_filt * w).T


def nep_squared(eta_filt, w, P, nu, delta_al_J, eta_pb):
    """NEP^2[row, ch] = 2 int eta P (h nu + eta P + 2 Delta/eta_pb) dnu (Eq. 17).

    The integrand is split into its three physical terms (Sect. 2.6), each a
    trapezoid sum: shot noise int eta P h nu, bunching int (eta P)^2 and
    generation-recombination (2 Delta_Al / eta_pb) int eta P.
    """
    shot = (P * (H_PLANCK * nu)) @ (eta_filt * w).T
    bunching = (P * P) @ (eta_filt * eta_filt * w).T
    gen_rec = (2.0 * delta_al_J / eta_pb) * (P @ (eta_filt * w).T)
    return 2.0 * (shot + bunching + gen_rec)


def photon_sigma(nep2, f_sample_hz):
    """sigma = NEP sqrt(f_sample / 2) (Eq. 18)."""
    return np.sqrt(nep2 * 0.5 * f_sample_hz)


# ---------------------------------------------------------------------------
# Counter-based random numbers: Philox4x32-10 (Salmon et al., SC'11) + Box-Muller
# ---------------------------------------------------------------------------

_PHILOX_M0 = np.uint64(0xD2511F53)
_PHILOX_M1 = np.uint64(0xCD9E8D57)
_PHILOX_W0 = np.uint64(0x9E3779B9)
_PHILOX_W1 = np.uint64(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox-4x32 rounds on counters (c0..c3) with key (k0, k1); returns 4 uint32 arrays.

    One round: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2 as 64-bit products;
    new counter = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); the key is bumped by
    the Weyl constants (W0, W1) between rounds.
    """
    x = [np.asarray(c, dtype=np.uint64) & _MASK32 for c in (c0, c1, c2, c3)]
    x = list(np.broadcast_arrays(*x))
    k0 = np.uint64(k0) & _MASK32
    k1 = np.uint64(k1) & _MASK32
    for rnd in range(10):
        p0 = _PHILOX_M0 * x[0]
        p1 = _PHILOX_M1 * x[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        x = [hi1 ^ x[1] ^ k0, lo1, hi0 ^ x[3] ^ k1, lo0]
        k0 = (k0 + _PHILOX_W0) & _MASK32
        k1 = (k1 + _PHILOX_W1) & _MASK32
    return [xi.astype(np.uint32) for xi in x]


def box_muller(xa, xb):
    """Two standard normals from two uint32 words: u = (x + 1/2) 2^-32, r = sqrt(-2 ln u_a)."""
    ua = (np.asarray(xa, dtype=F64) + 0.5) * 2.0 ** -32
    ub = (np.asarray(xb, dtype=F64) + 0.5) * 2.0 ** -32
    r = np.sqrt(-2.0 * np.log(ua))
    return r * np.cos(2.0 * np.pi * ub), r * np.sin(2.0 * np.pi * ub)


def _key(seed: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


def white_normals(seed: int, n, pix, ch):
    """z_w(n, i, ch): counter (n lo, n hi, i, ch >> 2); channel ch takes output ch & 3.

    Outputs (x0, x1) and (x2, x3) give two Box-Muller pairs (cos, sin) each.
    """
    n = np.asarray(n, dtype=np.int64)
    pix = np.asarray(pix, dtype=np.int64)
    ch = np.asarray(ch, dtype=np.int64)
    n, pix, ch = np.broadcast_arrays(n, pix, ch)
    k0, k1 = _key(seed)
    x = philox4x32_10(n & 0xFFFFFFFF, n >> 32, pix, ch >> 2, k0, k1)
    za, zb = box_muller(x[0], x[1])
    zc, zd = box_muller(x[2], x[3])
    sel = ch & 3
    return np.choose(sel, [za, zb, zc, zd])


def pink_normals(seed: int, n, pix, ch):
    """z_p(n, i, ch): counter (m lo, m hi, i, 2^31 | ch) with m = n >> 2; sample n takes output n & 3."""
    n = np.asarray(n, dtype=np.int64)
    pix = np.asarray(pix, dtype=np.int64)
    ch = np.asarray(ch, dtype=np.int64)
    n, pix, ch = np.broadcast_arrays(n, pix, ch)
    m = n >> 2
    k0, k1 = _key(seed)
    x = philox4x32_10(m & 0xFFFFFFFF, m >> 32, pix, np.int64(0x80000000) | ch, k0, k1)
    za, zb = box_muller(x[0], x[1])
    zc, zd = box_muller(x[2], x[3])
    return np.choose(n & 3, [za, zb, zc, zd])


def tk_normals(seed: int, j, pix, ch):
    """(re, im) normals of Fourier bin j of the Timmer-Koenig series of (i, ch): counter
    (q lo, q hi, i, 2^30 | ch) with q = j >> 1; bin j takes Box-Muller pair j & 1."""
    j = np.asarray(j, dtype=np.int64)
    pix = np.asarray(pix, dtype=np.int64)
    ch = np.asarray(ch, dtype=np.int64)
    j, pix, ch = np.broadcast_arrays(j, pix, ch)
    q = j >> 1
    k0, k1 = _key(seed)
    x = philox4x32_10(q & 0xFFFFFFFF, q >> 32, pix, np.int64(0x40000000) | ch, k0, k1)
    za, zb = box_muller(x[0], x[1])
    zc, zd = box_muller(x[2], x[3])
    odd = (j & 1) == 1
    return np.where(odd, zc, za), np.where(odd, zd, zb)


# ---------------------------------------------------------------------------
# Pink noise, exact: Timmer & Koenig (1995) over the whole scan (Sect. 2.6, Eq. 20)
# ---------------------------------------------------------------------------

def tk_length(n_total: int) -> int:
    """Length M = 2^ceil(log2 N) of the realisation whose first N samples are the scan."""
    return max(2, 1 << int(math.ceil(math.log2(max(int(n_total), 1)))))


def pink_tk_realisation(seed: int, A: float, alpha: float, f_sample_hz: float, n_total: int, pix: int, ch: int):
    """Whole-scan pink series x_n, n = 0 .. N-1, of spaxel pix and channel ch (W): Fourier
    coefficients drawn from the one-sided PSD S(f) = A f^-alpha, then the inverse DFT."""
    M = tk_length(n_total)
    if A <= 0.0:
        return np.zeros(int(n_total), dtype=F64)
    j = np.arange(1, M // 2 + 1, dtype=np.int64)
    f = j * (f_sample_hz / M)
    S = A * f ** (-alpha)
    re, im = tk_normals(seed, j, pix, ch)
    X = np.zeros(M // 2 + 1, dtype=np.complex128)
    X[1:M // 2] = np.sqrt(M * f_sample_hz * S[:-1] / 4.0) * (re[:-1] + 1j * im[:-1])
    X[M // 2] = np.sqrt(M * f_sample_hz * S[-1] / 2.0) * re[-1]           # real Nyquist coefficient
    x = np.fft.irfft(X, n=M)                                             # (1/M) sum over the Hermitian spectrum
    return x[:int(n_total)]


# ---------------------------------------------------------------------------
# Pink noise: pole-zero filter with power response ~ A f^-alpha (Sect. 2.6, Eq. 20)
# ---------------------------------------------------------------------------

@dataclass
class PinkFilter:
    a: np.ndarray      # discrete poles (n_pole,)
    b: np.ndarray      # discrete zeros (n_pole,)
    d: float           # direct term of the partial-fraction form
    r: np.ndarray      # residues (n_pole,)
    g: float           # gain


def pink_poles_count(f_min_hz: float, f_sample_hz: float) -> int:
    """Poles at f_min * 10^(j/3) for every j with pole <= f_sample/2."""
    return int(math.floor(3.0 * math.log10(0.5 * f_sample_hz / f_min_hz) + 1e-9)) + 1


def pink_transfer(a, b, f_hz, f_sample_hz):
    """H(f) = prod_j (1 - b_j e^{-i w}) / (1 - a_j e^{-i w}), w = 2 pi f / f_s (cascade form)."""
    zinv = np.exp(-2j * np.pi * np.asarray(f_hz, dtype=F64) / f_sample_hz)
    H = np.ones(zinv.shape, dtype=np.complex128)
    for aj, bj in zip(a, b):
        H *= (1.0 - bj * zinv) / (1.0 - aj * zinv)
    return H


def pink_design(alpha: float, A: float, f_min_hz: float, f_sample_hz: float) -> PinkFilter:
    """Design the filter for one channel (level A in W^2/Hz at 1 Hz, slope alpha)."""
    n_pole = pink_poles_count(f_min_hz, f_sample_hz)
    j = np.arange(n_pole, dtype=F64)
    p = f_min_hz * 10.0 ** (j / 3.0)
    q = p * 10.0 ** (alpha / 6.0)
    a = np.exp(-2.0 * np.pi * p / f_sample_hz)
    b = np.exp(-2.0 * np.pi * q / f_sample_hz)
    d = float(np.prod(b / a))
    r = np.empty(n_pole, dtype=F64)
    for jj in range(n_pole):
        num = np.prod(1.0 - b / a[jj])
        den = np.prod(np.delete(1.0 - a / a[jj], jj))
        r[jj] = num / den
    if A > 0:
        H1 = abs(pink_transfer(a, b, 1.0, f_sample_hz))
        g = math.sqrt(A * 0.5 * f_sample_hz) / H1
    else:
        g = 0.0
    return PinkFilter(a=a, b=b, d=d, r=r, g=g)


def pink_filter_run(design: PinkFilter, z: np.ndarray, state=None):
    """y_n = g (d z_n + sum_j r_j s_j,n), s_j,n = a_j s_j,n-1 + z_n, along axis 0 of z [nt, ...].

    ``state`` [..., n_pole] is s_j,-1 (zeros at the start of the scan); returns (y, final state).
    """
    z = np.asarray(z, dtype=F64)
    s = np.zeros(z.shape[1:] + (design.a.size,), dtype=F64) if state is None else np.array(state, dtype=F64)
    y = np.empty_like(z)
    for n in range(z.shape[0]):
        s = design.a * s + z[n][..., None]
        y[n] = design.g * (design.d * z[n] + s @ design.r)
    return y, s


# ---------------------------------------------------------------------------
# Whole path (Sect. 2.4 to Sect. 2.7, Eq. 21)
# ---------------------------------------------------------------------------

@dataclass
class Instrument:
    """Everything that does not change with time, evaluated once per scenario."""
    nu: np.ndarray
    w: np.ndarray
    eta_filt: np.ndarray
    prim: list
    eta_surf: np.ndarray
    pink: list
    pink_A: np.ndarray      # pink level per channel (W^2/Hz at 1 Hz)


def reference_nep2(sc: dict, nu, w, eta_filt, prim, eta_surf) -> np.ndarray:
    """NEP^2 per channel (W^2/Hz, Eq. 17) of the source-free sky at the screen's mean PWV and the
    scan's base elevation theta_0: the white noise level of the observation as planned.  It is
    the one-sided white PSD (Eq. 18: sigma^2 = NEP^2 f_s / 2), so a pink level A = NEP^2 puts the
    knee, where the pink PSD equals the white one, at 1 Hz."""
    atm = sc["atmosphere"]
    pwv = np.array([screen_pwv_field(sc).mean()])
    tau = zenith_opacity(opacity_table(sc), atm["pwv_min"], atm["dpwv"], pwv)
    eta = atmospheric_transmission(tau, np.array([sc["scan"]["theta0"]]))
    P = cascade(np.zeros_like(eta), eta, nu, prim, atm["T_atm"], sc["T_cmb"], sc["eta_taper"], eta_surf,
                sc["eta_pol"])
    return nep_squared(eta_filt, w, P, nu, sc["delta_al"], sc["eta_pb"])[0]


def build_instrument(sc: dict) -> Instrument:
    nu = frequency_grid(sc["f_lo"], sc["f_hi"], sc["n_freq"])
    w = trapezoid_weights(nu)
    disp = sc["dispersive"]
    eta_filt = filter_efficiency(disp["kind"], disp["f_c"], disp["R"], disp["eta_peak"], nu,
                                 sc["delta_al"], disp.get("custom"))
    prim = expand_cascade(sc["cascade"], nu)
    eta_surf = ruze_efficiency(sc["rho_surf"], nu)
    pink = []
    noise = sc.get("noise", {})
    n_ch = eta_filt.shape[0]
    if "pink_alpha" in noise and noise.get("pink_A") is None:
        # no level given: the knee at 1 Hz (Sect. 2.6 reading), A = the planned white level NEP^2
        A = reference_nep2(sc, nu, w, eta_filt, prim, eta_surf)
    else:
        A = np.asarray(noise.get("pink_A", np.zeros(n_ch)), dtype=F64)
    alpha = np.asarray(noise.get("pink_alpha", np.ones(n_ch)), dtype=F64)
    for ch in range(n_ch):
        pink.append(pink_design(float(alpha[ch]), float(A[ch]), noise.get("pink_f_min", 1e-3),
                                sc["f_sample"]))
    return Instrument(nu=nu, w=w, eta_filt=eta_filt, prim=prim, eta_surf=eta_surf, pink=pink, pink_A=A)


def screen_pwv_field(sc: dict) -> np.ndarray:
    atm = sc["atmosphere"]
    screen = np.asarray(atm["screen"], dtype=F64)
    if atm.get("is_epl", False):
        screen = epl_to_pwv(screen, atm["pwv0"])
    return screen


def opacity_table(sc: dict) -> np.ndarray:
    atm = sc["atmosphere"]
    if atm.get("table_is_opacity", True):
        return np.asarray(atm["table"], dtype=F64)
    return eta_to_opacity(atm["table"])


def row_geometry(sc: dict, n: np.ndarray, pix: np.ndarray):
    """Per-row scan, pointing, PWV and elevation for rows (n, i)."""
    t = n.astype(F64) / sc["f_sample"]
    scan = sc["scan"]
    phi_s, th_s = scan_pattern(scan["kind"], scan.get("params"), t, n, scan.get("custom"))
    off = np.asarray(sc["pix_offsets"], dtype=F64)
    dphi, dth = off[pix, 0], off[pix, 1]
    az = phi_s + scan["phi0"] + dphi                                  # spaxel pointing (Sect. 2.4)
    el = th_s + scan["theta0"] + dth
    atm = sc["atmosphere"]
    x, y = screen_coordinates(phi_s, th_s, dphi, dth, t, atm["h_column"], atm["wind"])
    pwv = screen_bilinear(screen_pwv_field(sc), x, y, atm["pitch"])
    return t, az, el, pwv


def skydip_calibration(sc: dict, inst: Instrument | None = None, pwv_lo: float = 0.5, pwv_hi: float = 2.0,
                       n_pwv: int = 16):
    """Per-channel brightness-temperature scale from a simulated skydip (Sect. 2.7).

    The zenith PWV takes n_pwv uniformly spaced values pwv_lo .. pwv_hi (mm) at the base
    elevation theta_0 of the scan, with no source; for each value the cascade gives P_nu,
    the channel powers P_KID (Eq. 16) and the band-averaged sky brightness temperature
    T_b = T_atm sum_nu eta_filt w (1 - eta_atm) / sum_nu eta_filt w.  Returns
    dict(a, b, pwv, p_kid, t_b) with the least-squares line T_b = a P_KID + b per channel.
    """
    if inst is None:
        inst = build_instrument(sc)
    atm = sc["atmosphere"]
    pwv = np.linspace(pwv_lo, pwv_hi, n_pwv, dtype=F64)
    el = np.full(n_pwv, sc["scan"]["theta0"], dtype=F64)
    tau_z = zenith_opacity(opacity_table(sc), atm["pwv_min"], atm["dpwv"], pwv)
    eta_atm = atmospheric_transmission(tau_z, el)                        # [n_pwv, nu]
    P_src = np.zeros_like(eta_atm)
    P = cascade(P_src, eta_atm, inst.nu, inst.prim, atm["T_atm"], sc["T_cmb"],
                sc["eta_taper"], inst.eta_surf, sc["eta_pol"])
    p_kid = kid_power(inst.eta_filt, inst.w, P)                          # [n_pwv, ch]
    hw = inst.eta_filt * inst.w                                           # [ch, nu]
    t_b = atm["T_atm"] * ((1.0 - eta_atm) @ hw.T) / hw.sum(axis=1)       # [n_pwv, ch]
    # ordinary least squares per channel: a = cov(P, T) / var(P), b = mean(T) - a mean(P)
    dp = p_kid - p_kid.mean(axis=0)
    dt = t_b - t_b.mean(axis=0)
    a = (dp * dt).sum(axis=0) / (dp * dp).sum(axis=0)
    b = t_b.mean(axis=0) - a * p_kid.mean(axis=0)
    return dict(a=a, b=b, pwv=pwv, p_kid=p_kid, t_b=t_b)


def mean_zenith_pwv(sc: dict, n_total: int) -> float:
    """The zenith PWV averaged over the observation: mean over rows (n, i), n < n_total."""
    n_pix = np.asarray(sc["pix_offsets"]).shape[0]
    nn, ii = np.meshgrid(np.arange(n_total, dtype=np.int64), np.arange(n_pix), indexing="ij")
    _, _, _, pwv = row_geometry(sc, nn.ravel(), ii.ravel())
    return float(pwv.mean())


def common_mode_reduction(sc: dict, t_b: np.ndarray, t0: int, pwv_mean: float, r_out: float,
                          inst: Instrument | None = None):
    """T*_a,i(t, ch) from a K TOD t_b [nt, n_pix, n_ch] of samples t0 .. t0+nt-1 (Eqs. 25-26):
    T_b,i / eta_i - (1 - eta_i) / (eta_i N_out) sum_j S_j T_b,j / (1 - eta_j), S_j = 1 for spaxels
    farther than r_out (rad) from the IFU centre, N_out = sum_j S_j."""
    if inst is None:
        inst = build_instrument(sc)
    t_b = np.asarray(t_b, dtype=F64)
    nt, n_pix, n_ch = t_b.shape
    atm = sc["atmosphere"]
    tau = zenith_opacity(opacity_table(sc), atm["pwv_min"], atm["dpwv"], np.array([pwv_mean]))[0]
    hw = inst.eta_filt * inst.w
    eta_z = (hw @ np.exp(-tau)) / hw.sum(axis=1)                                  # [n_ch]
    off = np.asarray(sc["pix_offsets"], dtype=F64).reshape(n_pix, 2)
    S = (np.hypot(off[:, 0], off[:, 1]) > r_out).astype(F64)
    n_out = S.sum()
    assert n_out > 0
    nn, ii = np.meshgrid(np.arange(t0, t0 + nt, dtype=np.int64), np.arange(n_pix), indexing="ij")
    _, _, el, _ = row_geometry(sc, nn.ravel(), ii.ravel())
    csc = (1.0 / np.sin(el)).reshape(nt, n_pix)
    eta = eta_z[None, None, :] ** csc[:, :, None]                                 # Eq. 10
    common = (S[None, :, None] * t_b / (1.0 - eta)).sum(axis=1) / n_out           # [nt, n_ch]
    return t_b / eta - (1.0 - eta) / eta * common[:, None, :]


def simulate(sc: dict, t0: int, nt: int, inst: Instrument | None = None,
             white: bool = True, pink: bool = True, pink_state=None, return_parts: bool = False,
             kelvin: dict | None = None, pink_tk: int | None = None):
    """TOD out[n - t0, i, ch] in W for samples n in [t0, t0 + nt), all spaxels (Eq. 21).

    pink_state [n_pix, n_ch, n_pole] is the filter state before sample t0 (zeros at t0 = 0).
    kelvin: the result of skydip_calibration; the TOD is then a P_tot + b in K (Sect. 2.7).
    pink_tk: scan length N; the pink term is then the Timmer-Koenig realisation over [0, N).
    """
    if inst is None:
        inst = build_instrument(sc)
    n_pix = np.asarray(sc["pix_offsets"]).shape[0]
    n_ch = inst.eta_filt.shape[0]
    n_idx = np.arange(t0, t0 + nt, dtype=np.int64)
    nn, ii = np.meshgrid(n_idx, np.arange(n_pix), indexing="ij")      # rows (n, i)
    nn, ii = nn.ravel(), ii.ravel()
    t, az, el, pwv = row_geometry(sc, nn, ii)

    atm = sc["atmosphere"]
    tau_z = zenith_opacity(opacity_table(sc), atm["pwv_min"], atm["dpwv"], pwv)
    eta_atm = atmospheric_transmission(tau_z, el)

    src = sc["source"]
    P_src = source_bilinear(np.asarray(src["cube"]), src["az0"], src["daz"], src["el0"],
                            src["del"], az, el)
    P = cascade(P_src, eta_atm, inst.nu, inst.prim, atm["T_atm"], sc["T_cmb"],
                sc["eta_taper"], inst.eta_surf, sc["eta_pol"])

    p_kid = kid_power(inst.eta_filt, inst.w, P)
    nep2 = nep_squared(inst.eta_filt, inst.w, P, inst.nu, sc["delta_al"], sc["eta_pb"])
    sigma = photon_sigma(nep2, sc["f_sample"])

    seed = sc.get("noise", {}).get("seed", 0)
    chs = np.arange(n_ch, dtype=np.int64)
    if white:
        zw = white_normals(seed, nn[:, None], ii[:, None], chs[None, :])
        p_wn = sigma * zw                                                 # Eq. 19
    else:
        p_wn = np.zeros_like(sigma)

    p_kid = p_kid.reshape(nt, n_pix, n_ch)
    p_wn = p_wn.reshape(nt, n_pix, n_ch)
    sigma = sigma.reshape(nt, n_pix, n_ch)
    p_pn = np.zeros_like(p_kid)
    new_state = None
    if pink and pink_tk is not None:
        assert t0 + nt <= pink_tk
        noise = sc.get("noise", {})
        A = inst.pink_A
        alpha = np.asarray(noise.get("pink_alpha", np.ones(n_ch)), dtype=F64)
        for i in range(n_pix):
            for ch in range(n_ch):
                x = pink_tk_realisation(seed, float(A[ch]), float(alpha[ch]), sc["f_sample"], pink_tk, i, ch)
                p_pn[:, i, ch] = x[t0:t0 + nt]
    elif pink:
        zp = pink_normals(seed, nn[:, None], ii[:, None], chs[None, :]).reshape(nt, n_pix, n_ch)
        n_pole = inst.pink[0].a.size
        new_state = np.zeros((n_pix, n_ch, n_pole), dtype=F64)
        for ch in range(n_ch):
            st = None if pink_state is None else np.asarray(pink_state, dtype=F64)[:, ch, :]
            y, s = pink_filter_run(inst.pink[ch], zp[:, :, ch], st)
            p_pn[:, :, ch] = y
            new_state[:, ch, :] = s
    total = p_kid + p_wn + p_pn                                           # Eq. 21
    if kelvin is not None:
        total = kelvin["a"] * total + kelvin["b"]                        # brightness scale (Sect. 2.7)
    if return_parts:
        return dict(total=total, p_kid=p_kid, p_wn=p_wn, p_pn=p_pn, sigma=sigma,
                    pwv=pwv.reshape(nt, n_pix), el=el.reshape(nt, n_pix), pink_state=new_state)
    return total
