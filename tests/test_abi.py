"""C-ABI library checks that need no GPU: symbols, host-built FP64 tables, validation.

The host tables (frequency grid, trapezoid weights, eta_filt, the cascade
collapse c0/c1/c2, pink-filter coefficients, hexagon offsets) are built in
FP64 by libgateau_b300.so without touching the device; they are compared with
the oracle, which evaluates the paper's equations literally and shares no
code with the library.
"""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle import gateau_oracle as O
from paper_2604_23305_b300 import Plan, hex_offsets, workloads as W
from paper_2604_23305_b300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    text = open(os.path.join(ROOT, "include", "gateau.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gateau_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib = L.lib()
    names = header_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
        assert n in L.SIGNATURES, f"{n} has no ctypes signature"
    assert set(L.SIGNATURES) == set(names)
    assert b"sm_103a" in lib.gateau_version()


def _plan(name="ifu25", nt=64, **kw):
    sc = W.scenario(name, nt_total=nt)
    return sc, Plan(sc, upload=False, **kw)


@pytest.mark.parametrize("name", ["single_pixel_small", "ifu25"])
def test_host_tables_match_oracle(name):
    sc, p = _plan(name)
    inst = O.build_instrument(sc)
    nf, nch = sc["n_freq"], p.n_ch
    np.testing.assert_allclose(p.get_vector(L.VEC_NU, nf), inst.nu, rtol=1e-15)
    np.testing.assert_allclose(p.get_vector(L.VEC_WEIGHT, nf), inst.w, rtol=1e-12)
    eta = p.get_vector(L.VEC_ETA_FILT, nch * nf).reshape(nch, nf)
    np.testing.assert_allclose(eta, inst.eta_filt, rtol=1e-12, atol=1e-16)
    # The collapse P = c0 + c1 (1 - e) + c2 e P_src equals the literal stage-by-stage cascade.
    c0, c1, c2 = (p.get_vector(w, nf) for w in (L.VEC_C0, L.VEC_C1, L.VEC_C2))
    rng = np.random.default_rng(0)
    e = rng.uniform(0.01, 0.999, (7, nf))
    ps = rng.uniform(0, 3e-22, (7, nf))
    atm = sc["atmosphere"]
    lit = O.cascade(ps, e, inst.nu, inst.prim, atm["T_atm"], sc["T_cmb"], sc["eta_taper"], inst.eta_surf, sc["eta_pol"])
    np.testing.assert_allclose(c0 + c1 * (1 - e) + c2 * e * ps, lit, rtol=1e-12)
    assert (c0 >= 0).all() and (c1 >= 0).all() and (c2 >= 0).all()


def test_collapse_of_every_stage_kind():
    sc = W.scenario("single_pixel_small", nt_total=8)
    sc["cascade"] = [
        dict(kind="reflective", eta=np.linspace(0.6, 0.95, 512), T=150.0),
        dict(kind="refractive", d=10e-3, n=3.4, tan_delta=1e-3, T=290.0, T_refl=40.0),
        dict(kind="refractive", d=4e-3, n=3.41, tan_delta=1e-4, T="sky", ar=True),
        dict(kind="ohmic", eps_ref=0.0025, nu_ref=840e9, T="sky"),
        dict(kind="reflective", eta=0.5, T=0.0),
    ]
    p = Plan(sc, upload=False)
    inst = O.build_instrument(sc)
    nf = sc["n_freq"]
    c0, c1, c2 = (p.get_vector(w, nf) for w in (L.VEC_C0, L.VEC_C1, L.VEC_C2))
    e = np.random.default_rng(4).uniform(0.0, 1.0, (5, nf))
    ps = np.random.default_rng(5).uniform(0, 3e-22, (5, nf))
    lit = O.cascade(ps, e, inst.nu, inst.prim, 273.0, sc["T_cmb"], sc["eta_taper"], inst.eta_surf, sc["eta_pol"])
    np.testing.assert_allclose(c0 + c1 * (1 - e) + c2 * e * ps, lit, rtol=1e-12)


@pytest.mark.parametrize("kind", ["lorentzian", "custom"])
def test_dispersive_kinds_match_oracle(kind):
    sc = W.scenario("single_pixel_small", nt_total=8)
    if kind == "custom":
        rng = np.random.default_rng(1)
        sc["dispersive"] = dict(kind="custom", f_c=np.ones(5), R=np.ones(5), eta_peak=np.ones(5),
                                custom=rng.uniform(0, 1, (5, 512)))
    else:
        sc["dispersive"]["kind"] = "lorentzian"
    p = Plan(sc, upload=False)
    inst = O.build_instrument(sc)
    eta = p.get_vector(L.VEC_ETA_FILT, p.n_ch * 512).reshape(p.n_ch, 512)
    np.testing.assert_allclose(eta, inst.eta_filt, rtol=1e-13, atol=1e-16)


def test_pink_coefficients_match_oracle():
    # explicit levels: the automatic level (knee at 1 Hz) needs the plan prepared on a device
    sc = W.scenario("ifu25", nt_total=100)
    sc["noise"]["pink_A"] = W.pink_levels(347, 7)[0]
    p = Plan(sc, upload=False)
    inst = O.build_instrument(sc)
    info = p.info()
    npole = info.n_pole
    assert npole == inst.pink[0].a.size
    a = p.get_vector(L.VEC_PINK_A, p.n_ch * npole).reshape(p.n_ch, npole)
    r = p.get_vector(L.VEC_PINK_R, p.n_ch * npole).reshape(p.n_ch, npole)
    d = p.get_vector(L.VEC_PINK_D, p.n_ch)
    for ch in (0, 17, 346):
        des = inst.pink[ch]
        np.testing.assert_allclose(a[ch], des.a, rtol=1e-14)
        np.testing.assert_allclose(r[ch], des.g * des.r, rtol=1e-10)
        assert d[ch] == pytest.approx(des.g * des.d, rel=1e-10)


def test_hex_offsets_match_oracle():
    for R in range(0, 5):
        np.testing.assert_allclose(hex_offsets(R, 1e-4), O.hex_offsets(R, 1e-4), atol=1e-16)
    with pytest.raises(L.GateauError):
        hex_offsets(-1, 1.0)


def test_argument_validation():
    lib = L.lib()
    sc = W.scenario("single_pixel_small", nt_total=8)
    p = Plan(sc, upload=False)
    # running before the source/screen/table/scan setters reports ESTATE, not a crash
    st = lib.gateau_run(p._h, 0, 10, C.c_void_p(1), None)
    assert st == L.ESTATE and b"source cube" in lib.gateau_last_error()
    assert lib.gateau_run(None, 0, 10, C.c_void_p(1), None) == L.EINVAL
    assert lib.gateau_set_cascade(p._h, -1, None) == L.EINVAL
    bad = (L.Stage * 1)()
    bad[0].kind = L.STAGE_REFLECTIVE
    bad[0].eta = 1.5
    bad[0].T_K = 10.0
    assert lib.gateau_set_cascade(p._h, 1, bad) == L.EINVAL
    assert lib.gateau_set_dispersive_element(p._h, 7, 3, None, None, None, None) == L.EINVAL
    assert lib.gateau_set_scan(p._h, L.SCAN_DAISY, None, 0, 0.0, 0.0, None, 0, 0) == L.EINVAL
    assert lib.gateau_plan_set_wait_budget(p._h, -1) == L.EINVAL
    assert lib.gateau_plan_set_wait_budget(None, 100) == L.EINVAL
    assert lib.gateau_plan_set_wait_budget(p._h, 0) == L.OK
    assert lib.gateau_plan_set_tiles(p._h, 0, 1) == L.EINVAL and lib.gateau_plan_set_tiles(p._h, 0, 7) == L.EINVAL
    assert lib.gateau_plan_set_tiles(p._h, 65, 0) == L.EINVAL           # 64 channels: at most 64 groups
    assert lib.gateau_plan_set_tiles(p._h, -1, 0) == L.EINVAL
    assert lib.gateau_plan_set_tiles(p._h, 2, 3) == L.OK and lib.gateau_plan_set_tiles(p._h, 0, 0) == L.OK
    assert lib.gateau_plan_autotune(p._h, 0, None, None) == L.EINVAL
    d = L.PlanDesc()
    out = L.PlanP()
    assert lib.gateau_plan_create(C.byref(d), C.byref(out)) == L.EINVAL and not out.value
    with pytest.raises(L.GateauError):
        Plan(dict(sc, noise=dict(seed=0, pink_f_min=1e-12)), upload=False)   # would need > 24 poles


def test_status_and_info_without_gpu():
    sc, p = _plan("single_pixel_small")
    info = p.info()
    assert info.n_freq == 512 and info.n_freq_padded == 512 and info.n_ch == 64 and info.n_pix == 1
    assert info.device_bytes == 0
    assert p.status() == 0
    t0, st = p.get_state()
    assert t0 == 0 and (st == 0).all()


def test_argument_validation_of_the_optional_modes_and_utilities():
    """The setters and utilities added around the hot path reject bad arguments before any device
    work (so this runs without a GPU)."""
    lib = L.lib()
    sc = W.scenario("single_pixel_small", nt_total=8)
    p = Plan(sc, upload=False)
    # brightness temperature: 2 <= n_pwv <= 64, 0 <= lo < hi; disabling always works
    assert lib.gateau_set_output_kelvin(p._h, 1, 0.5, 2.0, 1) == L.EINVAL
    assert lib.gateau_set_output_kelvin(p._h, 1, 0.5, 2.0, 65) == L.EINVAL
    assert lib.gateau_set_output_kelvin(p._h, 1, 2.0, 0.5, 16) == L.EINVAL
    assert lib.gateau_set_output_kelvin(p._h, 1, -1.0, 0.5, 16) == L.EINVAL
    assert lib.gateau_set_output_kelvin(p._h, 0, 0.0, 0.0, 0) == L.OK
    assert lib.gateau_set_output_kelvin(None, 0, 0.0, 0.0, 0) == L.EINVAL
    # the skydip's scale is only readable once the plan is prepared
    assert lib.gateau_set_output_kelvin(p._h, 1, 0.5, 2.0, 16) == L.OK
    buf = np.zeros(64)
    assert lib.gateau_plan_get_vector(p._h, L.VEC_TB_A, buf.ctypes.data_as(L.dp), 64) == L.ESTATE
    # exact pink noise: 0 <= n_total <= 2^30
    assert lib.gateau_set_pink_timmer_koenig(p._h, -1) == L.EINVAL
    assert lib.gateau_set_pink_timmer_koenig(p._h, (1 << 30) + 1) == L.EINVAL
    assert lib.gateau_set_pink_timmer_koenig(p._h, 0) == L.OK
    # common mode and mean PWV need a complete plan
    v = C.c_double(0.0)
    assert lib.gateau_mean_zenith_pwv(p._h, 10, C.byref(v)) == L.ESTATE
    assert lib.gateau_common_mode(p._h, 0, 8, C.c_void_p(1), C.c_void_p(1), 1.0, 0.0, None) == L.ESTATE
    assert lib.gateau_common_mode(p._h, 0, 8, None, C.c_void_p(1), 1.0, 0.0, None) == L.EINVAL
    # preprocessing utilities: powers of two, positive pitches / radius, no aliasing
    nu = np.array([300e9])
    nup = nu.ctypes.data_as(L.dp)
    assert lib.gateau_beam_far_field(nup, 1, 100, 64, 1e-5, 1e-5, 5.0, -10.0, C.c_void_p(1), None) == L.EINVAL
    assert lib.gateau_beam_far_field(nup, 1, 64, 64, 0.0, 1e-5, 5.0, -10.0, C.c_void_p(1), None) == L.EINVAL
    assert lib.gateau_beam_far_field(nup, 1, 64, 64, 1e-5, 1e-5, -5.0, -10.0, C.c_void_p(1), None) == L.EINVAL
    assert lib.gateau_convolve_source(C.c_void_p(1), 32, 16, 1, nup, 0.8, 1e-5, 1e-5, 5.0, -10.0, C.c_void_p(1),
                                      None) == L.EINVAL                     # dev_P aliases dev_I
    assert lib.gateau_convolve_source(C.c_void_p(1), 30, 16, 1, nup, 0.8, 1e-5, 1e-5, 5.0, -10.0, C.c_void_p(2),
                                      None) == L.EINVAL
    assert lib.gateau_smooth_screen(C.c_void_p(1), 48, 64, 0.5, 5.0, -10.0, C.c_void_p(2), None) == L.EINVAL
    assert lib.gateau_smooth_screen(None, 64, 64, 0.5, 5.0, -10.0, C.c_void_p(2), None) == L.EINVAL
