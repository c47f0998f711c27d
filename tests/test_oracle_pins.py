"""Pins of the FP64 oracle against facts fixed by the paper or by mathematics.

Each test checks the oracle against something other than itself: values the
paper prints or implies, closed forms, physical invariants, special cases that
reduce to a textbook result, the published Philox known-answer vectors, or a
statistical law.  A plausible slip in the oracle (dropped term, wrong sign or
index, transposed operand) fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, signal, stats

from oracle import gateau_oracle as O
from paper_2604_23305_b300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
GHZ = 1e9
KB, H = O.K_BOLTZMANN, O.H_PLANCK


def golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                k, v = line.split()[:2]
                vals[k] = float(v)
    return vals


# ---------------------------------------------------------------- constants / stages

def test_stage_efficiency_values():
    g = golden("efficiencies.txt")
    assert O.reflection_efficiency(3.41) == pytest.approx(g["refl"], abs=6e-6)
    assert O.refraction_efficiency(4e-3, 3.41, 1e-4, 300 * GHZ) == pytest.approx(g["refr_300GHz"], abs=6e-6)
    assert O.ohmic_efficiency(0.0025, 840 * GHZ, 350 * GHZ) == pytest.approx(g["ohmic_350GHz"], abs=6e-7)
    assert O.ruze_efficiency(42e-6, 350 * GHZ) == pytest.approx(g["ruze_350GHz"], abs=6e-6)
    assert O.kid_cutoff_hz(188e-6 * O.E_CHARGE) / GHZ == pytest.approx(g["cutoff_GHz"], abs=6e-3)


def test_refractive_stage_expansion():
    nu = np.array([300 * GHZ])
    st = dict(kind="refractive", d=4e-3, n=3.41, tan_delta=1e-4, T=290.0, T_refl=100.0)
    prim = O.expand_stage(st, nu)
    assert len(prim) == 3
    assert [p[1] for p in prim] == [100.0, 290.0, 100.0]
    assert prim[0][0][0] == pytest.approx(0.70135, abs=1e-5)
    assert len(O.expand_stage(dict(st, ar=True), nu)) == 1


# ---------------------------------------------------------------- Johnson-Nyquist

def test_johnson_nyquist_limits():
    # Rayleigh-Jeans: h nu << k T gives k T (1 - x/2 + x^2/12).
    T, nu = 1e4, 1 * GHZ
    x = H * nu / (KB * T)
    assert O.johnson_nyquist(T, nu) == pytest.approx(KB * T * (1 - x / 2 + x * x / 12), rel=1e-12)
    # Wien: h nu >> k T gives h nu exp(-x).
    T, nu = 1.0, 1000 * GHZ
    x = H * nu / (KB * T)
    assert O.johnson_nyquist(T, nu) == pytest.approx(H * nu * math.exp(-x), rel=1e-12)
    assert O.johnson_nyquist(0.0, 300 * GHZ) == 0.0


def test_johnson_nyquist_total_power():
    # Single-mode blackbody: int_0^inf h nu/(e^{h nu/kT}-1) d nu = (pi^2/6) (kT)^2 / h.
    for T in (2.725, 40.0, 290.0):
        total, _ = integrate.quad(lambda v: float(O.johnson_nyquist(T, v)), 0, 60 * KB * T / H,
                                  limit=400)
        assert total == pytest.approx(math.pi ** 2 / 6 * (KB * T) ** 2 / H, rel=1e-8)


# ---------------------------------------------------------------- cascade invariants

def _mixed_stages(T):
    return [dict(kind="reflective", eta=0.93, T=T),
            dict(kind="ohmic", eps_ref=0.0025, nu_ref=840 * GHZ, T=T),
            dict(kind="reflective", eta=0.85, T="sky"),
            dict(kind="refractive", d=10e-3, n=3.4, tan_delta=1e-3, T=T, T_refl=T),
            dict(kind="refractive", d=4e-3, n=3.41, tan_delta=1e-4, T=T, ar=True),
            dict(kind="reflective", eta=np.linspace(0.5, 0.9, 64), T=T)]


def test_thermal_equilibrium_invariant():
    """All stages, the sky and the CMB at one T, no source: P_nu = B(T, nu) for any eta."""
    nu = np.linspace(90 * GHZ, 900 * GHZ, 64)
    rng = np.random.default_rng(3)
    eta_atm = rng.uniform(0.01, 0.99, (5, 64))
    for T in (4.0, 150.0, 290.0):
        prim = O.expand_cascade(_mixed_stages(T), nu)
        P = O.cascade(np.zeros((5, 64)), eta_atm, nu, prim, T, T, 0.85,
                      O.ruze_efficiency(42e-6, nu), 0.5)
        np.testing.assert_allclose(P, np.broadcast_to(O.johnson_nyquist(T, nu), P.shape), rtol=1e-12)


def test_transparent_passthrough():
    """eta == 1 everywhere and a transparent sky: P_nu = eta_t eta_surf eta_pol P_src + B(T_cmb)."""
    nu = np.linspace(220 * GHZ, 440 * GHZ, 50)
    prim = O.expand_cascade([dict(kind="reflective", eta=1.0, T=290.0),
                             dict(kind="reflective", eta=1.0, T="sky")], nu)
    P_src = np.random.default_rng(0).uniform(0, 1e-22, (3, 50))
    es = O.ruze_efficiency(42e-6, nu)
    P = O.cascade(P_src, np.ones((3, 50)), nu, prim, 273.0, 2.725, 0.85, es, 0.5)
    np.testing.assert_allclose(P, 0.85 * es * 0.5 * P_src + O.johnson_nyquist(2.725, nu), rtol=1e-14)


def test_cold_cascade_is_product_of_efficiencies():
    """With every temperature at 0 K only the source survives, scaled by the product of all etas."""
    nu = np.linspace(220 * GHZ, 440 * GHZ, 40)
    stages = _mixed_stages(0.0)[:5]
    prim = O.expand_cascade(stages, nu)
    eta_atm = np.random.default_rng(1).uniform(0.2, 0.95, (4, 40))
    P_src = np.random.default_rng(2).uniform(1e-23, 1e-22, (4, 40))
    es = O.ruze_efficiency(42e-6, nu)
    P = O.cascade(P_src, eta_atm, nu, prim, 0.0, 0.0, 0.85, es, 0.5)
    n = 3.4
    refl = 1 - ((1 - n) / (1 + n)) ** 2
    prod = (0.93 * (1 - 0.0025 * np.sqrt(nu / (840 * GHZ))) * 0.85 * refl ** 2
            * np.exp(-2 * np.pi * 10e-3 * 3.4 * 1e-3 * nu / O.C_LIGHT)
            * np.exp(-2 * np.pi * 4e-3 * 3.41 * 1e-4 * nu / O.C_LIGHT))
    np.testing.assert_allclose(P, eta_atm * prod * 0.85 * es * 0.5 * P_src, rtol=1e-13)


def test_single_stage_emission_only():
    """No source, CMB at 0 K, one stage: P = (1-eta_atm) eta_1 B(T_atm) + (1-eta_1) B(T_1)."""
    nu = np.array([150 * GHZ, 350 * GHZ])
    eta_atm = np.array([[0.8, 0.6]])
    prim = O.expand_cascade([dict(kind="reflective", eta=0.9, T=40.0)], nu)
    P = O.cascade(np.zeros((1, 2)), eta_atm, nu, prim, 273.0, 0.0, 0.85, np.ones(2), 0.5)
    # Planck values by the textbook closed form at these two points, written out separately.
    B273 = np.array([H * v / math.expm1(H * v / (KB * 273.0)) for v in nu])
    B40 = np.array([H * v / math.expm1(H * v / (KB * 40.0)) for v in nu])
    np.testing.assert_allclose(P[0], 0.9 * (1 - eta_atm[0]) * B273 + 0.1 * B40, rtol=1e-13)


def test_sky_coupled_stage_by_hand():
    """One sky-coupled stage (Sect. 2.5) with T_atm != T_cmb and eta_atm != 1/2: the stage emits
    the sky it sees, (1 - eta_atm) B(T_atm) + eta_atm B(T_cmb), so
    P = eta_k [eta_atm P_0 + (1 - eta_atm) B_atm] + (1 - eta_k) [(1 - eta_atm) B_atm + eta_atm B_cmb]
    with P_0 = eta_t eta_surf eta_pol P_src + B_cmb (Eq. 11)."""
    nu = np.array([220 * GHZ, 350 * GHZ])
    eta_atm = np.array([[0.8, 0.3], [0.95, 0.6]])
    P_src = np.array([[2e-22, 5e-23], [0.0, 1e-22]])
    es = np.array([0.97, 0.95])
    prim = O.expand_cascade([dict(kind="reflective", eta=0.9, T="sky")], nu)
    P = O.cascade(P_src, eta_atm, nu, prim, 273.0, 2.725, 0.85, es, 0.5)
    # Planck single-mode powers written out by the textbook closed form at each point.
    B_atm = np.array([H * v / math.expm1(H * v / (KB * 273.0)) for v in nu])
    B_cmb = np.array([H * v / math.expm1(H * v / (KB * 2.725)) for v in nu])
    P0 = 0.85 * es * 0.5 * P_src + B_cmb
    after_sky = eta_atm * P0 + (1 - eta_atm) * B_atm
    stage_emission = (1 - eta_atm) * B_atm + eta_atm * B_cmb
    np.testing.assert_allclose(P, 0.9 * after_sky + 0.1 * stage_emission, rtol=1e-13)


# ---------------------------------------------------------------- dispersive element

def test_lorentzian_closed_form_integral():
    """Grating channel on a flat unit PSD: trapezoid sum = eta_p (f/2R)[atan 2R(nu/f-1)]_a^b."""
    nu = O.frequency_grid(220 * GHZ, 440 * GHZ, 20001)
    w = O.trapezoid_weights(nu)
    f_c = np.array([250 * GHZ, 331.7 * GHZ, 410 * GHZ])
    R = np.array([500.0, 300.0, 50.0])
    eta = O.filter_efficiency("lorentzian", f_c, R, 0.16, nu, 188e-6 * O.E_CHARGE)
    got = O.kid_power(eta, w, np.ones((1, nu.size)))[0]
    a, b = nu[0], nu[-1]
    exact = 0.16 * f_c / (2 * R) * (np.arctan(2 * R * (b / f_c - 1)) - np.arctan(2 * R * (a / f_c - 1)))
    np.testing.assert_allclose(got, exact, rtol=2e-7)


def test_nep_closed_forms_flat_psd():
    """Eq. 17 on a flat PSD P0 for a grating channel, against the closed-form integrals of
    L, L^2 and nu L (x = 2R(nu/f - 1))."""
    nu = O.frequency_grid(200 * GHZ, 500 * GHZ, 60001)
    w = O.trapezoid_weights(nu)
    f, R, ep = 300 * GHZ, 400.0, 0.3
    dal, epb = 188e-6 * O.E_CHARGE, 0.4
    eta = O.filter_efficiency("lorentzian", [f], [R], ep, nu, dal)
    P0 = 7e-22
    got = O.nep_squared(eta, w, np.full((1, nu.size), P0), nu, dal, epb)[0, 0]
    xa, xb = 2 * R * (nu[0] / f - 1), 2 * R * (nu[-1] / f - 1)
    s = f / (2 * R)
    i_L = ep * s * (math.atan(xb) - math.atan(xa))
    prim2 = lambda x: x / (2 * (1 + x * x)) + math.atan(x) / 2
    i_L2 = ep * ep * s * (prim2(xb) - prim2(xa))
    primnu = lambda x: math.atan(x) + math.log1p(x * x) / (4 * R)
    i_nuL = ep * s * f * (primnu(xb) - primnu(xa))
    exact = 2 * (H * P0 * i_nuL + P0 * P0 * i_L2 + (2 * dal / epb) * P0 * i_L)
    assert got == pytest.approx(exact, rel=1e-7)


def test_filterbank_telescoping_identity():
    """Constant eta_peak: sum over channels of Eq. 7 = eta_p (1 - prod_ch (1 - L_ch)); all >= 0;
    the recursion order follows centre frequency, not input order."""
    nu = np.linspace(200 * GHZ, 460 * GHZ, 3001)
    f_c = W.geometric_channels(220 * GHZ, 440 * GHZ, 101)
    R = np.full(101, 300.0)
    eta = O.filter_efficiency("filterbank", f_c, R, 0.16, nu, 188e-6 * O.E_CHARGE)
    prod = np.ones_like(nu)
    for f in f_c:
        prod *= 1 - 1 / (1 + 4 * 300.0 ** 2 * (nu / f - 1) ** 2)
    np.testing.assert_allclose(eta.sum(axis=0), 0.16 * (1 - prod), rtol=1e-12, atol=1e-15)
    assert (eta >= 0).all()
    perm = np.random.default_rng(0).permutation(101)
    eta_p = O.filter_efficiency("filterbank", f_c[perm], R, 0.16, nu, 188e-6 * O.E_CHARGE)
    np.testing.assert_array_equal(eta_p, eta[perm])
    # The highest channel sees the bare Lorentzian (nothing upstream).
    top = int(np.argmax(f_c))
    np.testing.assert_allclose(eta[top], 0.16 / (1 + 4 * 300.0 ** 2 * (nu / f_c[top] - 1) ** 2), rtol=1e-15)


def test_cutoff_masks_low_frequencies():
    nu = np.linspace(80 * GHZ, 120 * GHZ, 401)
    eta = O.filter_efficiency("lorentzian", [95 * GHZ], [20.0], 1.0, nu, 188e-6 * O.E_CHARGE)
    below = nu < 90.92e9 - 1e7
    assert (eta[0, below] == 0).all() and (eta[0, nu > 90.93e9] > 0).all()


def test_half_power_channels_reproduce_paper_count():
    """R = 20 over 90-180 GHz with half-power spacing gives the 15 channels of Sect. 4.1."""
    assert W.half_power_channels(90 * GHZ, 180 * GHZ, 20.0).size == 15
    assert W.half_power_channels(220 * GHZ, 440 * GHZ, 500.0).size == 347


# ---------------------------------------------------------------- atmosphere

def test_airmass_special_elevations():
    tau = np.array([[0.3, 1.2, 0.05]])
    np.testing.assert_allclose(O.atmospheric_transmission(tau, np.array([math.pi / 2])), np.exp(-tau), rtol=1e-15)
    np.testing.assert_allclose(O.atmospheric_transmission(tau, np.array([math.pi / 6])), np.exp(-tau) ** 2, rtol=1e-14)


def test_screen_uniform_linear_and_periodic():
    nx, ny, pitch = 16, 12, 0.5
    assert np.all(O.screen_bilinear(np.full((ny, nx), 0.8), np.array([-3.1, 7.7]), np.array([2.2, -9.0]), pitch) == 0.8)
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    lin = 0.3 + 0.01 * ix + 0.02 * iy
    # Points inside the non-wrapping interior: bilinear reproduces a linear field exactly.
    gx = np.array([1.25, 5.5, 10.75, 13.0])
    gy = np.array([2.5, 0.0, 9.9, 7.25])
    x = (gx - nx / 2) * pitch
    y = (gy - ny / 2) * pitch
    np.testing.assert_allclose(O.screen_bilinear(lin, x, y, pitch), 0.3 + 0.01 * gx + 0.02 * gy, rtol=1e-14)
    rnd = np.random.default_rng(0).uniform(size=(ny, nx))
    xs = np.random.default_rng(1).uniform(-20, 20, 50)
    ys = np.random.default_rng(2).uniform(-20, 20, 50)
    np.testing.assert_allclose(O.screen_bilinear(rnd, xs + 3 * nx * pitch, ys - 2 * ny * pitch, pitch),
                               O.screen_bilinear(rnd, xs, ys, pitch), rtol=1e-12)
    # Grid nodes return the node value; cell (0,0) sits at (-nx/2, -ny/2) * pitch.
    np.testing.assert_allclose(O.screen_bilinear(rnd, np.array([-nx / 2 * pitch, 0.0]),
                                                 np.array([-ny / 2 * pitch, 0.0]), pitch),
                               [rnd[0, 0], rnd[ny // 2, nx // 2]], rtol=1e-15)


def test_frozen_flow_coordinates():
    """Eq. 9: a stare drifts with the wind along x only; y depends on elevation offset only."""
    t = np.array([0.0, 1.0, 10.0])
    x, y = O.screen_coordinates(0.0, 0.0, 0.0, 0.0, t, 1537.0, 10.0)
    np.testing.assert_allclose(x, 10.0 * t)
    np.testing.assert_allclose(y, 0.0)
    x, y = O.screen_coordinates(0.0, 0.0, 1e-3, 2e-3, t, 1000.0, 0.0)
    np.testing.assert_allclose(x, 1000 * math.tan(1e-3))
    np.testing.assert_allclose(y, 1000 * math.tan(2e-3))


def test_opacity_interpolation_and_clamp():
    nu = np.linspace(220 * GHZ, 440 * GHZ, 7)
    pw = np.arange(11) * 0.5
    tab = 0.02 + np.outer(pw, np.linspace(0.05, 0.2, 7))          # exactly linear in PWV
    got = O.zenith_opacity(tab, 0.0, 0.5, np.array([0.0, 1.3, 2.75, 5.0]))
    want = 0.02 + np.outer([0.0, 1.3, 2.75, 5.0], np.linspace(0.05, 0.2, 7))
    np.testing.assert_allclose(got, want, rtol=1e-14)
    np.testing.assert_allclose(O.zenith_opacity(tab, 0.0, 0.5, np.array([-1.0, 9.0])), tab[[0, -1]], rtol=1e-15)
    np.testing.assert_allclose(O.eta_to_opacity(np.exp(-tab)), tab, rtol=1e-12)


def test_epl_conversion():
    np.testing.assert_allclose(O.epl_to_pwv(np.array([0.0, 6.587]), 1.0), [1.0, 2.0])


# ---------------------------------------------------------------- source and scan

def test_source_bilinear_linear_cube_and_outside():
    n_az, n_el, nf = 6, 5, 3
    ia, ie = np.meshgrid(np.arange(n_az), np.arange(n_el), indexing="ij")
    cube = (1.0 + 2.0 * ia + 3.0 * ie)[:, :, None] * np.array([1.0, 0.5, 0.25])
    az0, daz, el0, de = -0.5, 0.25, 0.75, 0.125       # exactly representable grid: edges are exact
    u = np.array([0.0, 2.5, 5.0, 4.9, 3.3])
    v = np.array([0.0, 1.25, 4.0, 0.1, 3.999])
    got = O.source_bilinear(cube, az0, daz, el0, de, az0 + u * daz, el0 + v * de)
    np.testing.assert_allclose(got, (1 + 2 * u + 3 * v)[:, None] * np.array([1.0, 0.5, 0.25]), rtol=1e-13)
    out = O.source_bilinear(cube, az0, daz, el0, de, np.array([az0 - 1e-6, az0, az0 + 6 * daz]),
                            np.array([el0, el0 - 1e-6, el0]))
    assert (out == 0).all()


def test_scan_patterns():
    t = np.linspace(0, 100, 1001)
    phi, th = O.scan_pattern("daisy", (1e-4, 2 * math.pi * 1.54, 2 * math.pi * 1.54 / 50), t)
    assert phi[0] == 0 and th[0] == 0
    assert np.all(np.hypot(phi, th) <= 1e-4 + 1e-18)
    phi, th = O.scan_pattern("raster", (1e-3, 2e-4, 1e-4, 5), t)
    assert np.all(np.abs(phi) <= 1e-3 + 1e-15)
    assert set(np.round(th / 1e-4, 9)) <= {-2, -1, 0, 1, 2}
    # first row runs +phi, second row -phi, rows step by one position
    assert phi[1] > phi[0] and phi[101] < phi[100] and th[101] - th[99] == pytest.approx(1e-4)
    tab = np.random.default_rng(0).uniform(size=(20, 2))
    p, q = O.scan_pattern("custom", None, np.zeros(3), np.array([0, 7, 19]), tab)
    np.testing.assert_array_equal(np.stack([p, q], 1), tab[[0, 7, 19]])


def test_daisy_quarter_periods():
    """Eq. 8 at quarter periods of the petal and of the daisy cycle (omega = 5 Omega):
    phi = r cos(Omega t) sin(omega t), theta = r sin(Omega t) sin(omega t)."""
    r, w, Om = 1e-4, 5.0, 1.0
    t = np.array([math.pi / (2 * w), math.pi / (2 * Om), math.pi / w, 3 * math.pi / (2 * w)])
    phi, th = O.scan_pattern("daisy", (r, w, Om), t)
    # omega t = pi/2, Omega t = pi/10: petal tip, rotated by pi/10.
    # Omega t = pi/2, omega t = 5 pi/2: petal tip along +theta.
    # omega t = pi: back at the centre whatever Omega t is.
    # omega t = 3 pi/2, Omega t = 3 pi/10: tip of the opposite half-petal.
    want_phi = [r * math.cos(math.pi / 10), 0.0, 0.0, -r * math.cos(3 * math.pi / 10)]
    want_th = [r * math.sin(math.pi / 10), r, 0.0, -r * math.sin(3 * math.pi / 10)]
    np.testing.assert_allclose(phi, want_phi, rtol=0, atol=1e-18)
    np.testing.assert_allclose(th, want_th, rtol=0, atol=1e-18)


def _linear_screen_geometry(nt):
    """Two spaxels staring at (phi0, theta0) = (0.4, 0.7) rad over a screen linear in x and y."""
    sc = W.scenario("single_pixel_small", nt_total=nt)
    nx = ny = 64
    ix, iy = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    sc["atmosphere"].update(screen=1.0 + 0.01 * ix + 0.004 * iy, pitch=0.5, h_column=1000.0, wind=2.0)
    sc["f_sample"] = 4.0
    sc["pix_offsets"] = np.array([[3e-3, -2e-3], [-4e-3, 5e-3]])
    sc["scan"] = dict(kind="stare", params=(), phi0=0.4, theta0=0.7)
    sc["noise"]["pink_f_min"] = 0.01
    return sc


def _expected_linear_screen_pwv(sc, n, pix):
    """Eq. 9 without the scan offset: x = h tan(dphi_i) + u_w t, y = h tan(dtheta_i); grid
    coordinates x / pitch + nx/2 (no wrap is reached here); the screen value there."""
    atm = sc["atmosphere"]
    off = sc["pix_offsets"][pix]
    t = n / sc["f_sample"]
    gx = (atm["h_column"] * np.tan(off[:, 0]) + atm["wind"] * t) / atm["pitch"] + 32
    gy = atm["h_column"] * np.tan(off[:, 1]) / atm["pitch"] + 32
    return 1.0 + 0.01 * gx + 0.004 * gy


def test_row_geometry_offsets_follow_eqs_9_and_10():
    """The screen coordinates use the scan pattern and the spaxel offset without the scan offset
    (Eq. 9), while the pointing used for the source and for the airmass adds (phi0, theta0)
    (Sect. 2.4, Eq. 10)."""
    sc = _linear_screen_geometry(8)
    n = np.repeat(np.arange(8), 2)
    pix = np.tile(np.arange(2), 8)
    t, az, el, pwv = O.row_geometry(sc, n, pix)
    np.testing.assert_allclose(t, n / 4.0, rtol=0, atol=0)
    np.testing.assert_allclose(az, 0.4 + sc["pix_offsets"][pix, 0], rtol=1e-15)
    np.testing.assert_allclose(el, 0.7 + sc["pix_offsets"][pix, 1], rtol=1e-15)
    np.testing.assert_allclose(pwv, _expected_linear_screen_pwv(sc, n, pix), rtol=1e-13)


def test_simulate_takes_the_source_and_airmass_at_the_offset_pointing():
    """Cold optics, T_cmb = 0, a flat unit filter and a constant cube that covers spaxel 0's
    pointing (phi0 + dphi_0, theta0 + dtheta_0) but not spaxel 1's: with eta = exp(-tau_z(PWV))^csc(el)
    at el = theta0 + dtheta_i (Eq. 10), P_KID = sum_nu w [eta_t eta_surf eta_pol C eta + (1 - eta) B_atm]."""
    nt = 6
    sc = _linear_screen_geometry(nt)
    nf = sc["n_freq"]
    sc["T_cmb"] = 0.0
    sc["atmosphere"]["T_atm"] = 100.0
    sc["cascade"] = [dict(kind="reflective", eta=1.0, T=0.0)]
    C = 3e-22
    sc["source"] = dict(cube=np.full((4, 4, nf), C), az0=0.401, daz=1e-3, el0=0.697, **{"del": 1e-3})
    sc["dispersive"] = dict(kind="custom", f_c=np.array([330 * GHZ]), R=np.ones(1), eta_peak=np.ones(1),
                            custom=np.ones((1, nf)))
    parts = O.simulate(sc, 0, nt, white=False, pink=False, return_parts=True)
    nu = O.frequency_grid(sc["f_lo"], sc["f_hi"], nf)
    w = np.full(nf, nu[1] - nu[0])
    w[0] = w[-1] = 0.5 * (nu[1] - nu[0])
    es = np.exp(-(4 * math.pi * sc["rho_surf"] * nu / O.C_LIGHT) ** 2)
    B_atm = np.array([H * v / math.expm1(H * v / (KB * 100.0)) for v in nu])
    atm = sc["atmosphere"]
    for i, inside in ((0, True), (1, False)):
        n = np.arange(nt)
        pwv = _expected_linear_screen_pwv(sc, n, np.full(nt, i))
        tau = O.zenith_opacity(O.opacity_table(sc), atm["pwv_min"], atm["dpwv"], pwv)
        eta = np.exp(-tau) ** (1.0 / math.sin(0.7 + sc["pix_offsets"][i, 1]))
        P = 0.85 * es * 0.5 * (C if inside else 0.0) * eta + (1 - eta) * B_atm
        np.testing.assert_allclose(parts["p_kid"][:, i, 0], P @ w, rtol=1e-12)


# ---------------------------------------------------------------- random numbers

def test_philox_known_answers():
    """Known-answer vectors of Philox4x32-10 from the Random123 distribution (Salmon et al. 2011)."""
    cases = [
        ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
        ((0xFFFFFFFF,) * 4, (0xFFFFFFFF, 0xFFFFFFFF), (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
        ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
         (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
    ]
    for ctr, key, want in cases:
        got = O.philox4x32_10(*ctr, *key)
        assert tuple(int(g) for g in got) == want


def test_normals_are_standard_gaussian():
    n = np.arange(1 << 16)
    zw = O.white_normals(5, n[:, None], 3, np.arange(4)[None, :]).ravel()
    zp = O.pink_normals(5, n, 3, 11)
    for z in (zw, zp):
        assert abs(z.mean()) < 5 / math.sqrt(z.size)
        assert abs(z.var() - 1) < 5 * math.sqrt(2 / z.size)
        assert stats.kstest(z, "norm").pvalue > 1e-4
    # distinct streams are uncorrelated
    zw2 = O.white_normals(5, n, 3, 11)
    assert abs(np.corrcoef(zw2, zp)[0, 1]) < 5 / math.sqrt(n.size)
    assert abs(np.corrcoef(zp[:-1], zp[1:])[0, 1]) < 5 / math.sqrt(n.size)


def test_white_noise_variance_matches_sigma():
    """Eqs. 18-19: the sample variance of sigma z_w is sigma^2 within a chi^2 99.99% band,
    and the one-sided white PSD equals NEP^2."""
    sigma = 3e-17
    z = O.white_normals(9, np.arange(40000), 0, 2)
    x = sigma * z
    lo, hi = stats.chi2.ppf([5e-5, 1 - 5e-5], x.size - 1) / (x.size - 1)
    assert lo < x.var() / sigma ** 2 < hi
    fs = 160.0
    f, pxx = signal.welch(x, fs=fs, nperseg=1024)
    nep2 = sigma ** 2 / (0.5 * fs)
    assert np.mean(pxx[1:-1]) == pytest.approx(nep2, rel=0.03)


# ---------------------------------------------------------------- pink noise

def test_pink_partial_fractions_equal_product_form():
    for alpha in (0.5, 1.0, 1.5):
        d = O.pink_design(alpha, 1e-34, 1 / 1200, 160.0)
        f = np.logspace(-4, math.log10(80), 50)
        zinv = np.exp(-2j * np.pi * f / 160.0)
        H_par = d.d + np.sum(d.r[None, :] / (1 - d.a[None, :] * zinv[:, None]), axis=1)
        np.testing.assert_allclose(H_par, O.pink_transfer(d.a, d.b, f, 160.0), rtol=1e-10)


def test_pink_alpha_zero_is_white_at_level_A():
    d = O.pink_design(0.0, 4e-34, 1 / 600, 160.0)
    assert d.d == pytest.approx(1.0) and np.allclose(d.r, 0)
    z = O.pink_normals(1, np.arange(1000), 0, 0)
    y, _ = O.pink_filter_run(d, z)
    np.testing.assert_allclose(y, d.g * z, rtol=1e-12)
    assert 2 * d.g ** 2 / 160.0 == pytest.approx(4e-34)


def test_pink_design_follows_power_law():
    fs, fmin = 160.0, 1 / 1200
    for alpha in (0.5, 1.0, 1.5):
        d = O.pink_design(alpha, 1e-34, fmin, fs)
        f = np.logspace(math.log10(10 * fmin), math.log10(fs / 20), 200)
        S = 2 / fs * d.g ** 2 * np.abs(O.pink_transfer(d.a, d.b, f, fs)) ** 2
        slope = np.polyfit(np.log10(f), np.log10(S), 1)[0]
        assert slope == pytest.approx(-alpha, abs=0.05)
        # ripple around the power law A f^-alpha stays within 1.5 dB in that band
        assert np.max(np.abs(10 * np.log10(S / (1e-34 * f ** -alpha)))) < 1.5


def test_pink_output_psd_matches_transfer_function():
    """Welch PSD of the filtered pink stream against (2/f_s) g^2 |H|^2 (Eq. 20 level and slope)."""
    fs = 160.0
    d = O.pink_design(1.2, 2e-34, 0.05, fs)
    n = 1 << 17
    z = O.pink_normals(3, np.arange(n), 2, 5)
    y, _ = O.pink_filter_run(d, z)
    y = y[4096:]                      # drop the start-up transient of the zero initial state
    f, pxx = signal.welch(y, fs=fs, nperseg=4096)
    sel = (f > 0.5) & (f < 60)
    S = 2 / fs * d.g ** 2 * np.abs(O.pink_transfer(d.a, d.b, f[sel], fs)) ** 2
    ratio = pxx[sel] / S
    assert np.median(ratio) == pytest.approx(1.0, abs=0.08)
    assert np.all(np.abs(np.log(ratio)) < 0.6)


def test_pink_state_carry_equals_one_pass():
    d = O.pink_design(1.0, 1e-34, 0.01, 160.0)
    z = O.pink_normals(0, np.arange(3000), 0, 0)
    y_all, s_all = O.pink_filter_run(d, z)
    y1, s1 = O.pink_filter_run(d, z[:1234])
    y2, s2 = O.pink_filter_run(d, z[1234:], s1)
    np.testing.assert_allclose(np.concatenate([y1, y2]), y_all, rtol=1e-13)
    np.testing.assert_allclose(s2, s_all, rtol=1e-13)


# ---------------------------------------------------------------- whole path

def _uniform_stare_scenario():
    sc = W.scenario("single_pixel_small", nt_total=64)
    sc["atmosphere"]["screen"] = np.full((32, 32), 1.2, dtype=np.float32)
    sc["source"]["cube"] = np.zeros_like(sc["source"]["cube"])
    return sc


def test_uniform_sky_stare_is_constant_in_time():
    sc = _uniform_stare_scenario()
    parts = O.simulate(sc, 0, 64, white=False, pink=False, return_parts=True)
    pk = parts["p_kid"][:, 0, :]
    np.testing.assert_allclose(pk, np.broadcast_to(pk[0], pk.shape), rtol=1e-13)
    assert np.allclose(parts["pwv"], 1.2)


def test_whole_path_thermal_equilibrium_gives_filter_weighted_planck():
    """Everything at one temperature, no source: P_KID = sum_nu w eta_filt B(T) for any sky."""
    sc = W.scenario("single_pixel_small", nt_total=32)
    T = 200.0
    sc["T_cmb"] = T
    sc["atmosphere"]["T_atm"] = T
    sc["cascade"] = [dict(s, T=(T if s["T"] != "sky" else "sky")) for s in sc["cascade"]]
    sc["source"]["cube"] = np.zeros_like(sc["source"]["cube"])
    parts = O.simulate(sc, 0, 32, white=False, pink=False, return_parts=True)
    inst = O.build_instrument(sc)
    B = np.array([H * v / math.expm1(H * v / (KB * T)) for v in inst.nu])
    want = (inst.eta_filt * inst.w) @ B
    np.testing.assert_allclose(parts["p_kid"][:, 0, :], np.broadcast_to(want, (32, want.size)), rtol=1e-12)


def test_chunked_simulation_equals_single_pass():
    sc = W.scenario("single_pixel_small", nt_total=200)
    full = O.simulate(sc, 0, 200, return_parts=True)
    a = O.simulate(sc, 0, 77, return_parts=True)
    b = O.simulate(sc, 77, 123, pink_state=a["pink_state"], return_parts=True)
    np.testing.assert_allclose(np.concatenate([a["total"], b["total"]]), full["total"], rtol=1e-12)


def test_hex_layout_geometry():
    """Packed hexagon (Sect. 2.3): 1 + 3R(R+1) spaxels (37 for R = 3, Sect. 4.1), nearest
    neighbours one spacing apart, outermost ring corners at R spacings, point symmetric."""
    for R in range(0, 5):
        off = O.hex_offsets(R, 2.0)
        assert off.shape == (1 + 3 * R * (R + 1), 2)
        if R == 0:
            continue
        d = np.hypot(off[:, None, 0] - off[None, :, 0], off[:, None, 1] - off[None, :, 1])
        np.fill_diagonal(d, np.inf)
        np.testing.assert_allclose(d.min(axis=1), 2.0, rtol=1e-12)
        r = np.hypot(off[:, 0], off[:, 1])
        assert r.max() == pytest.approx(2.0 * R, rel=1e-12)
        key = lambda a: set(map(tuple, np.round(a, 9)))
        assert key(off) == key(-off)
    assert O.hex_offsets(3, 1.0).shape[0] == 37


# ---------------------------------------------------------------- skydip / brightness temperature (Sect. 2.7)

def _planck_mode(T, nu):
    """Single-mode thermal power spectral density h nu / (exp(h nu / k T) - 1), written out."""
    return np.array([H * v / math.expm1(H * v / (KB * T)) for v in np.atleast_1d(nu)])


def test_skydip_single_point_channel_closed_form():
    """A channel that sees one grid frequency nu_0 (weight H w) behind the atmosphere alone:
    P = H w [B_cmb + (1 - eta)(B_atm - B_cmb)] and T_b = T_atm (1 - eta), so the skydip line is
    exactly T_b = a P + b with a = T_atm / (H w (B_atm - B_cmb)), b = -T_atm B_cmb / (B_atm - B_cmb)."""
    sc = W.scenario("single_pixel_small", nt_total=16)
    sc["cascade"] = []
    inst = O.build_instrument(sc)
    k0 = inst.nu.size // 3
    Hk = 0.37
    eta = np.zeros((1, inst.nu.size))
    eta[0, k0] = Hk
    inst.eta_filt = eta
    cal = O.skydip_calibration(sc, inst, 0.2, 3.0, 12)
    T_atm = sc["atmosphere"]["T_atm"]
    b_atm = _planck_mode(T_atm, inst.nu[k0])[0]
    b_cmb = _planck_mode(sc["T_cmb"], inst.nu[k0])[0]
    a_want = T_atm / (Hk * inst.w[k0] * (b_atm - b_cmb))
    b_want = -T_atm * b_cmb / (b_atm - b_cmb)
    np.testing.assert_allclose(cal["a"], [a_want], rtol=1e-10)
    np.testing.assert_allclose(cal["b"], [b_want], rtol=1e-8, atol=1e-12)
    # the brightness temperatures are those of the swept PWVs at the base elevation
    tau = O.zenith_opacity(np.asarray(sc["atmosphere"]["table"], dtype=float), sc["atmosphere"]["pwv_min"],
                           sc["atmosphere"]["dpwv"], cal["pwv"])[:, k0]
    eta_atm = np.exp(-tau / math.sin(sc["scan"]["theta0"]))
    np.testing.assert_allclose(cal["t_b"][:, 0], T_atm * (1 - eta_atm), rtol=1e-12)


def test_skydip_rayleigh_jeans_band_limit():
    """At h nu << k T the sky-coupled power of any band is k_B T_b sum(eta_filt w): with the
    atmosphere alone and no CMB, the skydip gives a = 1 / (k_B sum eta_filt w), b = 0, to the
    Rayleigh-Jeans accuracy h nu / 2 k T (~2e-4 at 1-2 GHz and 273 K)."""
    sc = W.scenario("single_pixel_small", nt_total=16)
    n_f = 256
    sc.update(f_lo=1.0e9, f_hi=2.0e9, n_freq=n_f, delta_al=0.0, T_cmb=0.0, cascade=[])
    f_c = np.linspace(1.2e9, 1.8e9, 5)
    sc["dispersive"] = dict(kind="filterbank", f_c=f_c, R=np.full(5, 40.0), eta_peak=np.full(5, 0.5))
    pw = np.arange(501) * 0.01
    sc["atmosphere"].update(table=(0.05 + 0.3 * pw)[:, None] * np.linspace(0.8, 1.2, n_f)[None, :],
                            table_is_opacity=True, pwv_min=0.0, dpwv=0.01)
    inst = O.build_instrument(sc)
    cal = O.skydip_calibration(sc, inst, 0.2, 3.0, 10)
    hw = (inst.eta_filt * inst.w).sum(axis=1)
    np.testing.assert_allclose(cal["a"], 1.0 / (KB * hw), rtol=5e-4)
    assert np.all(np.abs(cal["b"]) < 5e-4 * cal["t_b"].max())


def test_skydip_fit_is_the_least_squares_line():
    """The fitted (a, b) per channel equal numpy's degree-1 polynomial fit of T_b on P_KID, and
    the standard cascade's response is affine in T_b to well under a millikelvin per kelvin."""
    sc = W.scenario("single_pixel_small", nt_total=16)
    cal = O.skydip_calibration(sc, None, 0.4, 2.4, 16)
    for ch in range(0, cal["a"].size, 7):
        x = cal["p_kid"][:, ch] / cal["p_kid"][:, ch].mean()           # scaled for a well-posed fit
        slope, icpt = np.polyfit(x, cal["t_b"][:, ch], 1)
        np.testing.assert_allclose(cal["a"][ch], slope / cal["p_kid"][:, ch].mean(), rtol=1e-9)
        np.testing.assert_allclose(cal["b"][ch], icpt, rtol=1e-9, atol=1e-9)
    resid = cal["t_b"] - (cal["a"] * cal["p_kid"] + cal["b"])
    span = cal["t_b"].max(axis=0) - cal["t_b"].min(axis=0)
    assert np.all(np.abs(resid).max(axis=0) < 1e-3 * np.maximum(span, 1.0))


def test_kelvin_output_is_the_affine_map_of_the_total_power():
    sc = W.scenario("single_pixel_small", nt_total=40)
    cal = O.skydip_calibration(sc)
    w = O.simulate(sc, 0, 40)
    k = O.simulate(sc, 0, 40, kelvin=cal)
    np.testing.assert_allclose(k, cal["a"] * w + cal["b"], rtol=1e-14)


# ---------------------------------------------------------------- exact pink noise: Timmer & Koenig (Sect. 2.6)

def test_tk_realisation_is_the_inverse_dft_of_its_spectrum():
    """Brute-force inverse DFT on a short scan (N = 50 -> M = 64): x_n = (1/M) [X_{M/2} (-1)^n +
    2 sum_{0<j<M/2} Re(X_j e^{2 pi i j n / M})], with X_j built from the bin normals and the
    one-sided PSD amplitudes."""
    seed, A, alpha, fs, N = 7, 2.0e-17, 1.3, 160.0, 50
    M = O.tk_length(N)
    assert M == 64
    x = O.pink_tk_realisation(seed, A, alpha, fs, N, 2, 5)
    j = np.arange(1, M // 2 + 1)
    re, im = O.tk_normals(seed, j, 2, 5)
    S = A * (j * fs / M) ** (-alpha)
    n = np.arange(N)
    want = np.zeros(N)
    for jj in range(1, M // 2):
        Xj = math.sqrt(M * fs * S[jj - 1] / 4) * (re[jj - 1] + 1j * im[jj - 1])
        want += 2.0 * np.real(Xj * np.exp(2j * np.pi * jj * n / M))
    want += math.sqrt(M * fs * S[-1] / 2) * re[-1] * (-1.0) ** n
    np.testing.assert_allclose(x, want / M, rtol=1e-10, atol=1e-12 * np.abs(want / M).max())


def test_tk_white_limit_variance():
    """alpha = 0 is white noise of one-sided PSD A: variance sum_j S df = A f_s (M - 1) / (2 M)
    (M - 2 interior bins of weight 1, the Nyquist bin of weight 1/2); checked over 300
    independent channel series (relative standard error ~0.3 %)."""
    A, fs, N = 3.0e-18, 100.0, 1024
    xs = np.stack([O.pink_tk_realisation(11, A, 0.0, fs, N, 0, ch) for ch in range(300)])
    want = A * fs * (N - 1) / (2 * N)
    assert abs(xs.var() / want - 1.0) < 0.015


def test_tk_psd_follows_power_law():
    """Welch PSD of a long realisation: level A at 1 Hz and slope -alpha over two decades."""
    A, alpha, fs, N = 1.0e-18, 1.5, 160.0, 1 << 17
    x = O.pink_tk_realisation(3, A, alpha, fs, N, 0, 0)
    f, P = signal.welch(x, fs=fs, nperseg=1 << 13)
    band = (f > 0.1) & (f < 10.0)
    slope, icpt = np.polyfit(np.log10(f[band]), np.log10(P[band]), 1)
    assert abs(slope + alpha) < 0.1
    assert abs(icpt - math.log10(A)) < 0.1


def test_tk_streams_are_disjoint_from_white_and_pink():
    """The Fourier-bin counters (c3 = 2^30 | ch) never meet the white (c3 = ch >> 2 < 2^30) or the
    filtered pink (c3 = 2^31 | ch) counters, and the bin normals are standard normal."""
    re, im = O.tk_normals(5, np.arange(20000), 1, 3)
    z = np.concatenate([re, im])
    assert stats.kstest(z, "norm").pvalue > 1e-3
    assert abs(z.mean()) < 0.03 and abs(z.std() - 1.0) < 0.03
    w = O.white_normals(5, np.arange(2000), 1, 3)
    assert not np.any(np.isin(re[:2000], w))


# ---------------------------------------------------------------- common-mode reduction (Sect. 4.3, Eqs. 25-26)

def _cm_case(nt=24):
    sc = W.scenario("single_pixel_small", nt_total=nt)
    sc["pix_offsets"] = O.hex_offsets(2, 30 * math.pi / (180 * 3600))          # 19 spaxels, 30" apart
    sc["scan"] = dict(sc["scan"], kind="daisy", params=(20 * math.pi / (180 * 3600), 1.0, 0.1))
    inst = O.build_instrument(sc)
    pwv = 1.1
    atm = sc["atmosphere"]
    tau = O.zenith_opacity(O.opacity_table(sc), atm["pwv_min"], atm["dpwv"], np.array([pwv]))[0]
    hw = inst.eta_filt * inst.w
    eta_z = (hw @ np.exp(-tau)) / hw.sum(axis=1)
    n_pix = sc["pix_offsets"].shape[0]
    nn, ii = np.meshgrid(np.arange(nt), np.arange(n_pix), indexing="ij")
    _, _, el, _ = O.row_geometry(sc, nn.ravel(), ii.ravel())
    eta = eta_z[None, None, :] ** (1.0 / np.sin(el)).reshape(nt, n_pix)[:, :, None]
    return sc, inst, pwv, eta


def test_common_mode_recovers_the_source_closed_form():
    """T_b,i = T_sky (1 - eta_i) + eta_i T_src,i with no source on the off-source spaxels: the
    common mode is exactly T_sky and Eq. 25 returns T_src,i on every spaxel."""
    sc, inst, pwv, eta = _cm_case()
    nt, n_pix, n_ch = eta.shape
    r_out = 45 * math.pi / (180 * 3600)
    off = sc["pix_offsets"]
    inner = np.hypot(off[:, 0], off[:, 1]) <= r_out
    rng = np.random.default_rng(4)
    T_sky = 20.0 + 5.0 * rng.random((nt, 1, n_ch))
    T_src = np.where(inner[None, :, None], rng.random((nt, n_pix, n_ch)), 0.0)
    t_b = T_sky * (1 - eta) + eta * T_src
    got = O.common_mode_reduction(sc, t_b, 0, pwv, r_out, inst)
    np.testing.assert_allclose(got, T_src, atol=1e-10 * T_sky.max())


def test_common_mode_pure_atmosphere_is_zero_and_mean_pwv():
    """A pure sky seen by all spaxels gives T*_a = 0 for any off-source radius; the mean zenith PWV of a
    uniform screen is its value."""
    sc, inst, pwv, eta = _cm_case()
    t_b = 31.0 * (1 - eta)
    for r_out in (0.0, 25 * math.pi / (180 * 3600)):
        got = O.common_mode_reduction(sc, t_b, 0, pwv, r_out, inst)
        assert np.abs(got).max() < 1e-10 * 31.0
    scu = _uniform_stare_scenario()
    assert abs(O.mean_zenith_pwv(scu, 16) - float(np.float32(1.2))) < 1e-12    # the screen holds float32


def test_mean_zenith_pwv_of_a_linear_screen_drifting_with_the_wind():
    """Two spaxels stare through a screen linear in x and y while it drifts at u_w: the mean over
    every row (n, i), n < N, is the screen value at the mean grid coordinates, gx = 32 +
    mean_i(h tan dphi_i) / pitch + u_w (N - 1) / (2 f_s pitch), gy = 32 + mean_i(h tan dtheta_i) / pitch."""
    N = 16
    sc = _linear_screen_geometry(N)
    off = sc["pix_offsets"]
    gx = 32 + (1000.0 * np.tan(off[:, 0]).mean() + 2.0 * (N - 1) / (2 * 4.0)) / 0.5
    gy = 32 + 1000.0 * np.tan(off[:, 1]).mean() / 0.5
    assert O.mean_zenith_pwv(sc, N) == pytest.approx(1.0 + 0.01 * gx + 0.004 * gy, rel=1e-13)


# ---------------------------------------------------------------- preprocessing (Sect. 2.2, Eqs. 1-3)

ARCSEC_RAD = math.pi / (180 * 3600)


def test_far_field_uniform_aperture_is_airy():
    """t_edge = 0 dB: uniform circular aperture, F(theta) = [2 J1(x) / x]^2, x = 2 pi R theta / lambda
    (the grid spans 2048" at 2": the aperture radius is ~50 samples)."""
    from scipy.special import j1
    nu, R = 300e9, 5.0
    pitch = 2 * ARCSEC_RAD
    F = O.beam_far_field(nu, 1024, 1024, pitch, pitch, R, 0.0)
    lam = O.C_LIGHT / nu
    q = np.arange(1, 20)
    x = 2 * math.pi * R * q * pitch / lam
    airy = (2 * j1(x) / x) ** 2
    np.testing.assert_allclose(F[q, 0], airy, atol=1e-2)
    np.testing.assert_allclose(F[0, q], airy, atol=1e-2)


def test_far_field_untruncated_gaussian_closed_form():
    """A taper of -120 dB at the rim (field 1e-6 there) leaves an effectively untruncated Gaussian
    A = exp(-a r^2), a = (120/20) ln 10 / R^2, whose far field is F(u) = exp(-2 pi^2 u^2 / (a lambda^2))."""
    nu, R = 220e9, 5.0
    pitch = 3 * ARCSEC_RAD
    F = O.beam_far_field(nu, 512, 256, pitch, pitch, R, -120.0)
    lam = O.C_LIGHT / nu
    a = 6.0 * math.log(10.0) / R ** 2
    u = np.arange(0, 40) * pitch
    want = np.exp(-2 * math.pi ** 2 * u ** 2 / (a * lam ** 2))
    np.testing.assert_allclose(F[:40, 0], want, atol=2e-4)
    np.testing.assert_allclose(F[0, :40], want, atol=2e-4)


def test_source_convolution_of_a_point_is_the_beam():
    """I = I0 at one cell: P = A_p I0 cos(el') F(a - a', e - e') d_az d_el with F at twice the grid."""
    n_az, n_el = 16, 8
    d = 4 * ARCSEC_RAD
    nu = np.array([250e9, 400e9])
    I = np.zeros((n_az, n_el, 2))
    a0, e0 = 5, 3
    I[a0, e0, :] = 2.5e-17
    el0 = 0.8
    P = O.convolve_source(I, nu, el0, d, d, 5.0, -12.0)
    for k in range(2):
        F = O.beam_far_field(float(nu[k]), 2 * n_az, 2 * n_el, d, d, 5.0, -12.0)
        ia = (np.arange(n_az)[:, None] - a0) % (2 * n_az)
        ie = (np.arange(n_el)[None, :] - e0) % (2 * n_el)
        want = math.pi * 25.0 * 2.5e-17 * math.cos(el0 + e0 * d) * F[ia, ie] * d * d
        np.testing.assert_allclose(P[:, :, k], want, rtol=1e-9, atol=1e-12 * want.max())


def test_screen_smoothing_conserves_and_keeps_constants():
    rng = np.random.default_rng(8)
    scr = rng.normal(1.0, 0.1, (64, 128))
    out = O.smooth_screen(scr, 0.5, 5.0, -10.0)
    assert abs(out.sum() - scr.sum()) < 1e-9 * abs(scr.sum())
    np.testing.assert_allclose(O.smooth_screen(np.full((32, 32), 0.7), 0.5, 5.0, -10.0), 0.7, rtol=1e-12)
    assert out.std() < scr.std()


def test_pink_knee_at_one_hz_is_the_white_level():
    """With no pink level given, A = the planned white level: on a source-free stare through a
    uniform screen (the sky then is the reference sky), A equals the simulated white noise's own
    one-sided PSD 2 sigma^2 / f_s (Eq. 18), so pink and white PSDs cross at 1 Hz; a screen with the
    same mean PWV gives the same A (the reference takes the screen's mean)."""
    sc = _uniform_stare_scenario()
    assert sc["noise"].get("pink_A") is None and "pink_alpha" in sc["noise"]
    inst = O.build_instrument(sc)
    parts = O.simulate(sc, 0, 4, inst=inst, white=True, pink=False, return_parts=True)
    white_psd = 2.0 * parts["sigma"][0, 0, :] ** 2 / sc["f_sample"]
    np.testing.assert_allclose(inst.pink_A, white_psd, rtol=1e-12)
    for ch in (0, 31, 63):
        des = inst.pink[ch]
        one_sided_at_1hz = des.g ** 2 * abs(O.pink_transfer(des.a, des.b, 1.0, sc["f_sample"])) ** 2 * 2.0 / sc["f_sample"]
        assert one_sided_at_1hz == pytest.approx(white_psd[ch], rel=1e-12)
    c = float(np.float32(1.2))                       # the uniform screen's value, as stored
    checker = np.where((np.indices((32, 32)).sum(axis=0) % 2) == 0, c - 0.25, c + 0.25)   # same mean, exactly
    sc2 = dict(sc, atmosphere=dict(sc["atmosphere"], screen=checker))
    np.testing.assert_allclose(O.build_instrument(sc2).pink_A, inst.pink_A, rtol=1e-12)
