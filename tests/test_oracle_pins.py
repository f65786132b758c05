"""Pins of the FP64 oracle against facts that do not come from the oracle.

Every check here is independent of the oracle's own formulas: published
tables (tests/golden), numerical quadrature of the gamma-distribution
integrals whose closed forms the oracle uses, brute-force maximisation of the
Koehler curve, the lognormal distribution of critical supersaturations,
closed-form sedimentation cases (exact shift at Courant number 1, geometric
decay of a single level), conservation invariants (total water, liquid-ice
static energy, column mass budget) and non-negativity.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, optimize, stats

import oracle as O
from paper_2010_14823_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")
P = O.param
F = synth.FIDX


def _table(name):
    rows = []
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([float(x) for x in line.split()])
    return np.array(rows)


# ------------------------------------------------------------ c1 thermodynamics
def test_es_liquid_matches_iapws_table():
    for tc, es in _table("es_liquid_water.txt"):
        assert abs(O.es_liq(273.15 + tc) / es - 1.0) < 3e-3


def test_es_ice_matches_murphy_koop_table():
    for tc, es in _table("es_ice.txt"):
        assert abs(O.es_ice(273.15 + tc) / es - 1.0) < 3e-2


def test_es_slopes_follow_clausius_clapeyron():
    # d ln e_s / dT = L / (R_v T^2): the latent heats of the parameter set must
    # be consistent with the slopes of both saturation curves (within 6 %).
    Rv = P("Rv")
    for T in (250.0, 263.0, 283.0, 298.0):
        h = 1e-3
        sl = (math.log(O.es_liq(T + h)) - math.log(O.es_liq(T - h))) / (2 * h)
        assert abs(sl / (P("Lv") / (Rv * T * T)) - 1.0) < 0.06
        si = (math.log(O.es_ice(T + h)) - math.log(O.es_ice(T - h))) / (2 * h)
        assert abs(si / ((P("Lv") + P("Lf")) / (Rv * T * T)) - 1.0) < 0.06


def test_ice_saturation_below_liquid_below_freezing():
    for tc in (-1.0, -10.0, -30.0, -50.0):
        assert O.es_ice(273.15 + tc) < O.es_liq(273.15 + tc)


def test_qsat_is_the_specific_humidity_of_saturated_air():
    # From partial densities of the ideal-gas mixture: q = rho_v / (rho_v + rho_d).
    Rd, Rv = P("Rd"), P("Rv")
    for e, p, T in ((611.2, 1e5, 273.15), (4000.0, 9e4, 300.0), (20.0, 3e4, 230.0)):
        rho_v = e / (Rv * T)
        rho_d = (p - e) / (Rd * T)
        assert abs(O.qsat(e, p) / (rho_v / (rho_v + rho_d)) - 1.0) < 1e-14


def test_dqsat_dT_matches_finite_difference():
    for T, p in ((260.0, 6e4), (285.0, 9e4), (300.0, 1e5)):
        h = 1e-4
        fd = (O.qsat(O.es_liq(T + h), p) - O.qsat(O.es_liq(T - h), p)) / (2 * h)
        assert abs(O.dqsat_liq_dT(T, p) / fd - 1.0) < 1e-7


# ------------------------------------------------------- a2 saturation adjustment
def _qs(T, p):
    return O.qsat(O.es_liq(T), p)


@pytest.mark.parametrize("T,p,rh,qc", [
    (285.0, 9e4, 1.02, 0.0),      # condensation from clear air
    (280.0, 8e4, 1.005, 3e-4),    # condensation onto cloud
    (290.0, 9.5e4, 0.98, 1e-3),   # partial evaporation
    (275.0, 8.5e4, 0.999, 5e-5),  # partial evaporation, small cloud
])
def test_satadj_root_and_invariants(T, p, rh, qc):
    qv = rh * _qs(T, p)
    T1, qv1, qc1 = O.satadj(p, T, qv, qc)
    cp, Lv = P("cp"), P("Lv")
    # brute force: the root of cp (T' - T) = Lv (qv - qs(T')) by bisection
    root = optimize.brentq(lambda t: cp * (t - T) - Lv * (qv - _qs(t, p)), T - 20, T + 20, xtol=1e-13)
    if qc1 > 0.0:
        assert abs(T1 - root) < 1e-9
        assert abs(qv1 / _qs(T1, p) - 1.0) < 1e-12
    assert abs((qv1 + qc1) - (qv + qc)) <= 4 * np.spacing(qv + qc)
    assert abs(cp * (T1 - T) - Lv * (qc1 - qc)) < 1e-9 * Lv * max(abs(qc1 - qc), 1e-12)


def test_satadj_full_evaporation_clips_at_cloud():
    T, p = 290.0, 9e4
    qv, qc = 0.9 * _qs(T, p), 2e-5
    T1, qv1, qc1 = O.satadj(p, T, qv, qc)
    assert qc1 == 0.0
    assert abs(T1 - (T - P("Lv") / P("cp") * qc)) < 1e-12
    assert qv1 < _qs(T1, p)


def test_satadj_clear_subsaturated_untouched():
    T, p = 290.0, 9e4
    qv = 0.8 * _qs(T, p)
    assert O.satadj(p, T, qv, 0.0) == (T, qv, 0.0)


# ------------------------------------------------------------- a3 activation
def test_critical_supersaturation_is_koehler_maximum():
    # kappa-Koehler: s(r) = A/r - kappa r_d^3 / r^3; its maximum over r for
    # r_d = r_m is the mode's critical supersaturation.
    for T in (260.0, 280.0, 300.0):
        A = 2 * P("surft") * P("Mw") / (P("rho_w") * P("Rgas") * T)
        rd, kap = P("arg_rm"), P("arg_kappa")
        res = optimize.minimize_scalar(lambda lr: -(A / math.exp(lr) - kap * rd ** 3 / math.exp(3 * lr)),
                                       bounds=(math.log(rd), math.log(1e3 * rd)), method="bounded",
                                       options={"xatol": 1e-12})
        assert abs(-res.fun / O.arg_sm(T) - 1.0) < 1e-8


def test_activated_fraction_is_lognormal_cdf_of_critical_supersaturation():
    # r_d ~ lognormal(r_m, sigma) and s_c ~ r_d^(-3/2): ln s_c is normal with
    # mean ln S_m and std 1.5 ln sigma; the activated fraction is P(s_c < S_max).
    sig = P("arg_sigma")
    for N, w, T, p in ((1e8, 0.5, 285.0, 9e4), (3e8, 2.0, 275.0, 8e4), (5e7, 0.05, 295.0, 1e5)):
        smax, sm = O.arg_smax(N, w, T, p), O.arg_sm(T)
        frac = stats.norm.cdf((math.log(smax) - math.log(sm)) / (1.5 * math.log(sig)))
        assert abs(O.arg_nact(N, w, T, p) / N - frac) < 1e-12


def test_activation_limits_and_monotonicity():
    T, p, N = 283.0, 9e4, 1e8
    assert O.arg_nact(N, 0.0, T, p) == 0.0
    assert O.arg_nact(N, -1.0, T, p) == 0.0
    ws = [0.01, 0.1, 0.5, 1.0, 3.0, 10.0, 100.0]
    na = [O.arg_nact(N, w, T, p) for w in ws]
    assert all(b > a for a, b in zip(na, na[1:]))
    assert all(0.0 < x <= N for x in na)
    assert O.arg_nact(N, 1e6, T, p) / N > 0.999
    # S_max falls as the aerosol population grows (competition for vapour)
    s = [O.arg_smax(n, 1.0, T, p) for n in (1e7, 1e8, 1e9)]
    assert s[0] > s[1] > s[2]
    # typical marine/continental range: S_max of order 0.1-1 % at w ~ 1 m/s
    assert 5e-4 < O.arg_smax(1e8, 1.0, T, p) < 2e-2


def test_activation_counts_existing_droplets_and_moves_aerosol_number():
    """Activation raises the cloud-droplet number to the number the updraft
    activates (Abdul-Razzak and Ghan, pinned above) out of the whole
    population n_a + n_c, never lowers it, and takes the new droplets from
    the free aerosol: with no droplets the cloud number becomes the activated
    number; with at least that many already nothing activates; in between the
    cloud number is topped up to it.  n_a + n_c is conserved throughout."""
    T, p, rho, w = 283.0, 9.0e4, 1.1, 1.5
    base = np.zeros(16)
    base[F["T"]], base[F["p"]], base[F["rho"]], base[F["w"]] = T, p, rho, w
    base[F["qv"]] = 1.005 * O.qsat(O.es_liq(T), p)      # saturated: the adjustment makes cloud
    base[F["qc"]] = 2e-4
    pop = 1.5e8                                         # n_a + n_c per kg
    cases = []
    for nc in (0.0, 0.2 * pop, 0.6 * pop, 0.999 * pop):
        st = base.copy()
        st[F["nc"]], st[F["na"]] = nc, pop - nc
        out = O.adjust_activate(st)
        assert out[F["qc"]] > P("q_min")
        nact = O.arg_nact(rho * pop, w, out[F["T"]], p) / rho   # activated per kg
        cases.append((nc, nact, out[F["nc"]], out[F["na"]]))
        assert out[F["nc"]] + out[F["na"]] == pytest.approx(pop, rel=1e-14)
        if nc >= nact:
            assert out[F["nc"]] == nc and out[F["na"]] == pop - nc       # nothing activates
        else:
            assert out[F["nc"]] == pytest.approx(min(nact, pop), rel=1e-12)
    # the cases cover both sides of the activated number
    assert any(nc < nact for nc, nact, _, _ in cases) and any(nc >= nact for nc, nact, _, _ in cases)
    # a very strong updraft activates nearly the whole population: the free
    # aerosol is nearly used up but never negative (no droplet is created
    # beyond n_a + n_c)
    st = base.copy()
    st[F["w"]], st[F["nc"]], st[F["na"]] = 1e4, 0.0, pop
    out = O.adjust_activate(st)
    assert 0.0 <= out[F["na"]] < 1e-2 * pop and out[F["nc"]] <= pop * (1 + 1e-14)


# -------------------------------------------------- gamma-distribution algebra
def _psd_quad(sp, q, lam, rho, fn):
    """int fn(D) n(D) dD with n(D) = N0 D^mu e^(-lam D), N0 set by the mass
    content rho q = int a D^b n(D) dD (both integrals by quadrature)."""
    a, b, mu = P("a_" + sp), P("b_" + sp), P("mu_" + sp)
    shape = lambda D: D ** mu * math.exp(-lam * D)
    hi = 80.0 / lam
    mass1 = integrate.quad(lambda D: a * D ** b * shape(D), 0, hi, epsabs=0, epsrel=1e-13, limit=400)[0]
    N0 = rho * q / mass1
    return integrate.quad(lambda D: fn(D) * N0 * shape(D), 0, hi, epsabs=0, epsrel=1e-13, limit=400)[0]


@pytest.mark.parametrize("sp,q,n", [("c", 3e-4, 1e8), ("r", 1e-4, 3e3), ("i", 1e-5, 1e5),
                                    ("s", 1e-4, 1e4), ("g", 1e-3, 5e3)])
def test_lambda_reproduces_mass_and_number(sp, q, n):
    rho = 1.0
    lam = O.lam(sp, q, n)
    mu = P("mu_" + sp)
    dmean = (mu + 1) / lam
    assert P("dmin_" + sp) < dmean < P("dmax_" + sp), "case must be unclamped"
    num = _psd_quad(sp, q, lam, rho, lambda D: 1.0) / rho
    assert abs(num / n - 1.0) < 1e-10


def test_lambda_clamps_mean_diameter():
    for sp in "crisg":
        mu = P("mu_" + sp)
        big = O.lam(sp, 1e-3, 1e-6)        # too few particles -> largest allowed
        assert abs((mu + 1) / big / P("dmax_" + sp) - 1.0) < 1e-14
        small = O.lam(sp, 1e-12, 1e14)     # too many -> smallest allowed
        assert abs((mu + 1) / small / P("dmin_" + sp) - 1.0) < 1e-14
        assert O.lam(sp, 1e-4, 0.0) == big
        assert O.lam(sp, 1e-4, -5.0) == big


@pytest.mark.parametrize("sp", list("crisg"))
@pytest.mark.parametrize("k", [0.0, 1.0, 1.7, 2.37, 3.0])
def test_moments_match_quadrature(sp, k):
    rho, q = 0.9, 2e-4
    lam = 3.0 / (0.3 * P("dmax_" + sp))
    quad = _psd_quad(sp, q, lam, rho, lambda D: D ** k)
    assert abs(O.moment(sp, rho, q, lam, k) / quad - 1.0) < 1e-10


@pytest.mark.parametrize("sp", list("risg"))
def test_ventilation_integral_matches_quadrature(sp):
    rho, q = 0.8, 1e-4
    lam = (P("mu_" + sp) + 1) / (0.2 * P("dmax_" + sp))
    nu = P("mu_air") / rho
    sc = nu / P("Dv")
    cv, dv = P("cv_" + sp), P("dv_" + sp)
    V = lambda D: cv * D ** dv * (P("rho0") / rho) ** 0.4
    fv = lambda D: 0.78 + 0.31 * sc ** (1 / 3) * math.sqrt(V(D) * D / nu)
    quad = _psd_quad(sp, q, lam, rho, lambda D: D * fv(D))
    assert abs(O.vent_integral(sp, rho, q, lam) / quad - 1.0) < 1e-10


@pytest.mark.parametrize("sp", list("risg"))
def test_fall_speeds_are_weighted_means(sp):
    rho = 0.7
    lam = (P("mu_" + sp) + 1) / (0.05 * P("dmax_" + sp))   # small particles: uncapped
    a, b = P("a_" + sp), P("b_" + sp)
    V = lambda D: P("cv_" + sp) * D ** P("dv_" + sp) * (P("rho0") / rho) ** 0.4
    q = 1e-4
    vq = _psd_quad(sp, q, lam, rho, lambda D: V(D) * a * D ** b) / _psd_quad(sp, q, lam, rho, lambda D: a * D ** b)
    vn = _psd_quad(sp, q, lam, rho, lambda D: V(D)) / _psd_quad(sp, q, lam, rho, lambda D: 1.0)
    assert vq < P("vmax_" + sp)
    assert abs(O.vq(sp, rho, lam) / vq - 1.0) < 1e-10
    assert abs(O.vn(sp, rho, lam) / vn - 1.0) < 1e-10
    assert O.vn(sp, rho, lam) < O.vq(sp, rho, lam)
    # large particles hit the cap
    lam_big = (P("mu_" + sp) + 1) / P("dmax_" + sp)
    if V(P("dmax_" + sp)) > 2 * P("vmax_" + sp):
        assert O.vq(sp, rho, lam_big * 1e-3) == P("vmax_" + sp)


# ----------------------------------------------------------------- rates
def _state(**kw):
    st = np.zeros(16)
    base = dict(T=280.0, qv=5e-3, p=8.5e4, rho=1.05, na=1e8, w=0.0)
    base.update(kw)
    for k, v in base.items():
        st[F[k]] = v
    return st


def test_rain_evaporation_is_growth_law_integrated_over_psd():
    T, p, rho = 288.0, 9e4, 1.08
    qv = 0.7 * _qs(T, p)
    qr, nr = 2e-4, 2e3
    st = _state(T=T, qv=qv, qr=qr, nr=nr, p=p, rho=rho)
    R = O.rates(st, 1.0)
    lam = O.lam("r", qr, nr)
    es = O.es_liq(T)
    Rv = P("Rv")
    A = P("Lv") ** 2 / (P("Ka") * Rv * T * T)
    B = Rv * T / (es * P("Dv"))
    S = qv / _qs(T, p)
    nu = P("mu_air") / rho
    V = lambda D: P("cv_r") * D ** P("dv_r") * (P("rho0") / rho) ** 0.4
    fv = lambda D: 0.78 + 0.31 * (nu / P("Dv")) ** (1 / 3) * math.sqrt(V(D) * D / nu)
    # single drop: dm/dt = 4 pi C (S - 1) f_v / (A + B) with C = D/2
    dmdt = lambda D: 4 * math.pi * (D / 2) * (S - 1) * fv(D) / (A + B)
    quad = _psd_quad("r", qr, lam, rho, dmdt) / rho
    assert R["evr"] > 0
    assert abs(-R["evr"] / quad - 1.0) < 1e-10


def test_deposition_and_melting_integrals():
    rho, p = 0.9, 7e4
    for sp, key in (("i", "depi"), ("s", "deps"), ("g", "depg")):
        T = 255.0
        qv = 1.05 * O.qsat(O.es_ice(T), p)
        q, n = 1e-4, {"i": 1e6, "s": 1e4, "g": 1e3}[sp]
        st = _state(T=T, qv=qv, p=p, rho=rho, **{"q" + sp: q, "n" + sp: n})
        R = O.rates(st, 1.0)
        lam = O.lam(sp, q, n)
        esi = O.es_ice(T)
        Ls = P("Lv") + P("Lf")
        A = Ls ** 2 / (P("Ka") * P("Rv") * T * T)
        B = P("Rv") * T / (esi * P("Dv"))
        nu = P("mu_air") / rho
        V = lambda D: P("cv_" + sp) * D ** P("dv_" + sp) * (P("rho0") / rho) ** 0.4
        fv = lambda D: 0.78 + 0.31 * (nu / P("Dv")) ** (1 / 3) * math.sqrt(V(D) * D / nu)
        Si = qv / O.qsat(esi, p)
        dmdt = lambda D: 4 * math.pi * P("ccap_" + sp) * D * (Si - 1) * fv(D) / (A + B)
        quad = _psd_quad(sp, q, lam, rho, dmdt) / rho
        assert abs(R[key] / quad - 1.0) < 1e-10
        # melting above 0 C: heat conducted in melts ice at L_f per kg
        T2 = 276.0
        st2 = _state(T=T2, qv=0.9 * _qs(T2, p), p=p, rho=rho, **{"q" + sp: q, "n" + sp: n})
        R2 = O.rates(st2, 1.0)
        melt = lambda D: 4 * math.pi * P("ccap_" + sp) * D * P("Ka") * (T2 - 273.15) * fv(D) / P("Lf")
        quad2 = _psd_quad(sp, q, lam, rho, melt) / rho
        assert abs(R2["mlt" + sp] / quad2 - 1.0) < 1e-10
        assert R2[key] == 0.0 and R[("mlt" + sp)] == 0.0


def test_riming_is_swept_volume_integral():
    rho, p, T = 0.95, 8e4, 265.0
    qc = 2e-4
    for sp, key in (("s", "rims"), ("g", "rimg")):
        q, n = 3e-4, {"s": 1e4, "g": 2e3}[sp]
        st = _state(T=T, qv=0.99 * _qs(T, p), qc=qc, nc=1e8, p=p, rho=rho, **{"q" + sp: q, "n" + sp: n})
        R = O.rates(st, 1.0)
        lam = O.lam(sp, q, n)
        V = lambda D: P("cv_" + sp) * D ** P("dv_" + sp) * (P("rho0") / rho) ** 0.4
        # collected cloud mass per kg air: (pi/4) D^2 V(D) E (rho q_c) / rho
        swept = lambda D: math.pi / 4 * D * D * V(D) * P("e_rim") * qc
        quad = _psd_quad(sp, q, lam, rho, swept)
        assert abs(R[key] / quad - 1.0) < 1e-10


def test_rate_regimes():
    p = 8e4
    # nothing present, subsaturated, warm: every rate zero
    st = _state(T=285.0, qv=0.5 * _qs(285.0, p), p=p)
    assert all(v == 0.0 for v in O.rates(st, 1.0).values())
    # nucleation only below T_nuc and only when ice-supersaturated
    T = P("T_nuc") + 0.5
    st = _state(T=T, qv=1.2 * O.qsat(O.es_ice(T), p), p=p)
    assert O.rates(st, 1.0)["nuc"] == 0.0
    T = P("T_nuc") - 0.5
    st = _state(T=T, qv=1.2 * O.qsat(O.es_ice(T), p), p=p)
    assert O.rates(st, 1.0)["nuc"] > 0.0
    st = _state(T=T, qv=0.99 * O.qsat(O.es_ice(T), p), p=p)
    assert O.rates(st, 1.0)["nuc"] == 0.0
    # KK2000 scaling with cloud water and with droplet concentration in cm^-3
    rho = 1.1
    s1 = _state(qc=1e-4, nc=1e8 / rho, rho=rho)
    s2 = _state(qc=2e-4, nc=1e8 / rho, rho=rho)
    s3 = _state(qc=1e-4, nc=2e8 / rho, rho=rho)
    r1, r2, r3 = (O.rates(s, 1.0)["aut"] for s in (s1, s2, s3))
    assert abs(r2 / r1 - 2 ** P("kk_aut_qc")) < 1e-12
    assert abs(r3 / r1 - 2 ** P("kk_aut_nc")) < 1e-12


def test_kk2000_point_values_worked_by_hand():
    """Khairoutdinov & Kogan (2000) in their own units (q in kg/kg, N_c in
    cm^-3, rates in kg kg^-1 s^-1), evaluated by hand in logarithms (seven
    digits each) at q_c = 0.5 g/kg, N_c = 100 cm^-3, q_r = 0.1 g/kg:
      autoconversion 1350 q_c^2.47 N_c^-1.79:
        ln 1350 = 7.2078599, ln 5e-4 = -7.6009025, ln 100 = 4.6051702
        7.2078599 + 2.47 (-7.6009025) - 1.79 (4.6051702)
          = 7.2078599 - 18.7742292 - 8.2432547 = -19.8096240
        exp(-19.8096240) = e^-20 e^0.1903760 = 2.0611536e-9 x 1.2097 = 2.4934e-9
      accretion 67 (q_c q_r)^1.15:
        ln 67 = 4.2046926, ln 5e-8 = -16.8112428
        4.2046926 + 1.15 (-16.8112428) = 4.2046926 - 19.3329292 = -15.1282366
        exp(-15.1282366) = e^-15 e^-0.1282366 = 3.0590232e-7 x 0.879646 = 2.6909e-7
    The droplet number is given per kg of air: 100 cm^-3 at rho = 1.1 kg m^-3
    is 1e8 / 1.1 per kg."""
    rho = 1.1
    R = O.rates(_state(qc=5e-4, nc=1e8 / rho, qr=1e-4, nr=1e4, rho=rho), 1.0)
    assert abs(R["aut"] / 2.4934e-9 - 1.0) < 5e-5
    assert abs(R["acc"] / 2.6909e-7 - 1.0) < 5e-5


def test_kk2000_droplet_number_floor():
    """The droplet concentration entering the KK2000 autoconversion is held
    at 1 cm^-3 from below: any smaller concentration gives the rate at
    1 cm^-3, and the -1.79 power law runs from exactly 1 cm^-3 upward (at
    2 cm^-3 the rate is 2^-1.79 times the rate at 1 cm^-3, and at 1.05 cm^-3
    already below it)."""
    rho = 1.1
    aut = lambda ncm3: O.rates(_state(qc=3e-4, nc=ncm3 * 1e6 / rho, rho=rho), 1.0)["aut"]
    a1 = aut(1.0)
    assert a1 > 0.0
    for low in (0.99, 0.5, 1e-3, 0.0):
        assert abs(aut(low) / a1 - 1.0) < 1e-14, low
    assert abs(aut(2.0) / a1 - 2.0 ** -1.79) < 1e-13
    assert aut(1.05) < a1 * (1.0 - 0.08)        # 1.05^-1.79 = 0.9164


def test_self_collection_point_values_worked_by_hand():
    """Seifert & Beheng self-collection in SI units with the cloud droplet
    shape nu = 1, evaluated by hand at rho = 1.1 kg m^-3:
      cloud: per m^3 of air the number falls at k_c (nu+2)/(nu+1) L_c^2 with
        L_c = rho q_c; per kg of air (divided by rho) at
        k_c (nu+2)/(nu+1) rho q_c^2 = 9.44e9 x (3/2) x 1.1 x (1e-4)^2
                                    = 1.416e10 x 1.1e-8 = 155.76 kg^-1 s^-1
      rain: per m^3 at k_r N_r L_r with N_r = rho n_r, L_r = rho q_r; per kg at
        k_r rho n_r q_r = 5.78 x 1.1 x 1e3 x 1e-4 = 0.6358 kg^-1 s^-1"""
    rho = 1.1
    R = O.rates(_state(qc=1e-4, nc=1e8 / rho, qr=1e-4, nr=1e3, rho=rho), 1.0)
    assert abs(R["scc"] / 155.76 - 1.0) < 1e-13
    assert abs(R["scr"] / 0.6358 - 1.0) < 1e-13


def test_rain_does_not_grow_in_supersaturated_air():
    """Rain exchanges vapour only by evaporating in subsaturated air: at
    S_w = 1.05, 1.0 and 1 + 1e-12 its evaporation rate is zero, at
    S_w = 0.95 positive."""
    T, p, rho = 285.0, 9.0e4, 1.1
    qs = O.qsat(O.es_liq(T), p)
    evr = lambda sw: O.rates(_state(T=T, p=p, rho=rho, qv=sw * qs, qr=2e-4, nr=1e3), 1.0)["evr"]
    for sw in (1.05, 1.0, 1.0 + 1e-12):
        assert evr(sw) == 0.0, sw
    assert evr(0.95) > 0.0


def test_accretion_scaling_and_presence():
    """KK2000 accretion is a power of the product q_c q_r: doubling either
    water content multiplies it by 2^1.15 (a law with the exponent on one
    factor only would give 2 for the other), it does not depend on either
    number concentration or on the air density, and it is zero unless both
    cloud and rain are present (above q_min)."""
    rho = 1.1
    base = dict(qc=3e-4, nc=1.5e8, qr=2e-4, nr=5e3, rho=rho)
    acc = lambda **kw: O.rates(_state(**{**base, **kw}), 1.0)["acc"]
    a0 = acc()
    assert a0 > 0.0
    assert abs(acc(qc=6e-4) / a0 - 2.0 ** 1.15) < 1e-13
    assert abs(acc(qr=4e-4) / a0 - 2.0 ** 1.15) < 1e-13
    assert abs(acc(qc=6e-4, qr=1e-4) / a0 - 1.0) < 1e-13
    assert acc(nc=4e8) == a0 and acc(nr=9e4) == a0
    assert acc(rho=0.6) == a0
    q_min = P("q_min")
    assert acc(qc=q_min) == 0.0 and acc(qr=q_min) == 0.0
    assert acc(qc=0.5 * q_min) == 0.0 and acc(qr=0.5 * q_min) == 0.0
    assert acc(qc=2 * q_min) > 0.0 and acc(qr=2 * q_min) > 0.0


def test_self_collection_scaling_and_number_only():
    """Seifert-Beheng self-collection: the cloud-number loss goes as the
    square of the cloud water and does not depend on the droplet number, the
    rain-number loss as n_r q_r, both linearly with the air density, and
    neither exists without its species.  The process moves no mass: in
    saturated warm air holding only rain (no adjustment, no evaporation, no
    cloud processes), a point update changes the rain number alone, by dt
    times the rate."""
    rho = 1.1
    cloud = dict(qc=1e-4, nc=1e8 / rho, rho=rho)
    scc = lambda **kw: O.rates(_state(**{**cloud, **kw}), 1.0)["scc"]
    c0 = scc()
    assert c0 > 0.0
    assert abs(scc(qc=2e-4) / c0 - 4.0) < 1e-13
    assert scc(nc=3e8 / rho) == c0
    assert abs(scc(rho=2 * rho) / c0 - 2.0) < 1e-13
    assert scc(qc=0.5 * P("q_min")) == 0.0
    rain = dict(qr=1e-4, nr=1e3, rho=rho)
    scr = lambda **kw: O.rates(_state(**{**rain, **kw}), 1.0)["scr"]
    r0 = scr()
    assert r0 > 0.0
    assert abs(scr(nr=2e3) / r0 - 2.0) < 1e-13
    assert abs(scr(qr=3e-4) / r0 - 3.0) < 1e-13
    assert abs(scr(rho=2 * rho) / r0 - 2.0) < 1e-13
    assert scr(qr=0.5 * P("q_min")) == 0.0
    T, p, dt = 285.0, 9e4, 1.0
    st = _state(T=T, p=p, rho=rho, qv=O.qsat(O.es_liq(T), p), qr=1e-4, nr=1e3)
    R = O.rates(st, dt)
    assert R["evr"] == 0.0 and R["aut"] == 0.0 and R["acc"] == 0.0
    out = O.point(st, dt)
    for name in ("T", "qv", "qc", "qr", "qi", "qs", "qg", "nc", "ni", "ns", "ng"):
        assert out[F[name]] == st[F[name]], name
    assert abs(out[F["nr"]] - (st[F["nr"]] - dt * R["scr"])) <= 4 * np.spacing(st[F["nr"]])
    assert out[F["nr"]] < st[F["nr"]]


def test_ice_nucleation_closed_form_and_bookkeeping():
    """Meyers et al. (1992) ice nucleation below T_nuc: the crystal number
    grows as exp(c (S_i - 1)) with the ice supersaturation, the crystals
    already present are subtracted, the difference is made within the step
    (rate ~ 1/dt) and counted per kg of air (~ 1/rho); each new crystal has
    mass m_i0, taken from the vapour, with the heat of sublimation."""
    T, p, rho = P("T_nuc") - 5.0, 6e4, 0.8
    qsi = O.qsat(O.es_ice(T), p)
    assert qsi < O.qsat(O.es_liq(T), p)
    nuc = lambda Si, ni=0.0, dt=1.0, r=rho: O.rates(_state(T=T, p=p, rho=r, qv=Si * qsi, ni=ni), dt)["nuc"]
    r1, r2 = nuc(1.02), nuc(1.07)
    assert r1 > 0.0
    assert abs(r2 / r1 / math.exp(P("mey_c") * 0.05) - 1.0) < 1e-12
    n_in = r1 * 1.0                      # crystals per kg made in a 1 s step from none
    assert abs(nuc(1.02, ni=0.25 * n_in) / r1 - 0.75) < 1e-12
    assert nuc(1.02, ni=n_in * (1 + 1e-9)) == 0.0
    assert abs(nuc(1.02, dt=4.0) / r1 - 0.25) < 1e-12
    assert abs(nuc(1.02, r=2 * rho) / r1 - 0.5) < 1e-12
    # point update: vapour -> ice only through nucleation (no ice to grow on,
    # liquid subsaturated, no cloud or rain)
    dt = 1.0
    st = _state(T=T, p=p, rho=rho, qv=1.05 * qsi)
    R = O.rates(st, dt)
    out = O.point(st, dt)
    dn = out[F["ni"]] - st[F["ni"]]
    dq = out[F["qi"]] - st[F["qi"]]
    assert abs(dn / (dt * R["nuc"]) - 1.0) < 1e-12
    assert abs(dq / (P("m_i0") * dn) - 1.0) < 1e-12
    assert abs((out[F["qv"]] - st[F["qv"]]) + dq) <= 8 * np.spacing(st[F["qv"]])
    # cp dT = (Lv + Lf) dq up to the rounding of the new temperature (dT is ~1e-6 K)
    assert abs(P("cp") * (out[F["T"]] - T) - (P("Lv") + P("Lf")) * dq) <= 4 * P("cp") * np.spacing(T)


def test_meyers_nucleation_worked_by_hand():
    """Meyers et al. (1992) at S_i = 1.1 (ice supersaturation 10 %), by hand:
      N_in = 1e3 exp(-0.639 + 12.96 x 0.1) m^-3 = 1e3 exp(0.657)
           = 1e3 x e^0.6 x e^0.057 = 1e3 x 1.8221188 x 1.0586558 = 1928.9967 m^-3
    made from none within a 1 s step and counted per kg of air at
    rho = 0.8 kg m^-3: 1928.9967 / 0.8 = 2411.2458 kg^-1 s^-1."""
    T, p = P("T_nuc") - 5.0, 6e4
    qsi = O.qsat(O.es_ice(T), p)
    nuc = O.rates(_state(T=T, p=p, rho=0.8, qv=1.1 * qsi), 1.0)["nuc"]
    assert abs(nuc / 2411.2458 - 1.0) < 5e-8


@pytest.mark.parametrize("sp", ["i", "s", "g"])
def test_melting_moves_mass_number_and_heat(sp):
    """Melting above 0 C, isolated (saturated air holding one ice species and
    nothing else: no evaporation, deposition or collection): the melted mass
    goes to rain, the species' number moves to rain in proportion to its mass
    (the mean mass is kept), and the heat of fusion comes from the air."""
    T, p, rho, dt = 275.0, 9e4, 1.1, 1.0
    q, n = 1e-4, 1e4
    st = _state(T=T, p=p, rho=rho, qv=O.qsat(O.es_liq(T), p), **{"q" + sp: q, "n" + sp: n})
    R = O.rates(st, dt)
    assert {k for k, v in R.items() if v != 0.0} == {"mlt" + sp}
    out = O.point(st, dt)
    dq = out[F["q" + sp]] - q
    dn = out[F["n" + sp]] - n
    assert abs(dq / (-dt * R["mlt" + sp]) - 1.0) < 1e-12
    assert abs(out[F["qr"]] + dq) <= 4 * np.spacing(q)
    assert abs(dn / (dq * n / q) - 1.0) < 1e-12
    assert abs(out[F["nr"]] + dn) <= 4 * np.spacing(n)
    assert out[F["qv"]] == st[F["qv"]]
    assert abs(P("cp") * (out[F["T"]] - T) - P("Lf") * dq) <= 4 * P("cp") * np.spacing(T)


def test_rain_evaporation_moves_mass_number_and_heat():
    """Rain evaporating in subsaturated warm air with no cloud: the vapour
    gains the evaporated mass, the rain number falls in proportion to the
    mass (plus rain self-collection, the one other process acting), and the
    heat of vaporisation comes from the air."""
    T, p, rho, dt = 288.0, 9e4, 1.08, 1.0
    q, n = 2e-4, 2e3
    st = _state(T=T, p=p, rho=rho, qv=0.7 * O.qsat(O.es_liq(T), p), qr=q, nr=n)
    R = O.rates(st, dt)
    assert {k for k, v in R.items() if v != 0.0} == {"evr", "scr"}
    out = O.point(st, dt)
    dq = out[F["qr"]] - q
    assert abs(dq / (-dt * R["evr"]) - 1.0) < 1e-12
    assert abs(out[F["qv"]] - st[F["qv"]] + dq) <= 4 * np.spacing(st[F["qv"]])
    assert abs((out[F["nr"]] - n) / (dq * n / q - dt * R["scr"]) - 1.0) < 1e-12
    assert abs(P("cp") * (out[F["T"]] - T) - P("Lv") * dq) <= 4 * P("cp") * np.spacing(T)


@pytest.mark.parametrize("sp", ["i", "s", "g"])
@pytest.mark.parametrize("regime", ["growth", "sublimation"])
def test_deposition_moves_mass_number_and_heat(sp, regime):
    """Vapour deposition on one ice species, isolated (270 K: below 0 C,
    above the nucleation threshold; no liquid): growth keeps the crystal
    number; sublimation removes crystals in proportion to the mass; the
    vapour balances the ice mass and the heat of sublimation the air."""
    T, p, rho, dt = 270.0, 8e4, 1.0, 1.0
    q, n = 1e-4, 1e4
    qsi, qsl = O.qsat(O.es_ice(T), p), O.qsat(O.es_liq(T), p)
    assert T > P("T_nuc") and qsi < qsl
    qv = 0.5 * (qsi + qsl) if regime == "growth" else 0.8 * qsi
    st = _state(T=T, p=p, rho=rho, qv=qv, **{"q" + sp: q, "n" + sp: n})
    R = O.rates(st, dt)
    assert {k for k, v in R.items() if v != 0.0} == {"dep" + sp}
    assert (R["dep" + sp] > 0.0) == (regime == "growth")
    out = O.point(st, dt)
    dq = out[F["q" + sp]] - q
    assert abs(dq / (dt * R["dep" + sp]) - 1.0) < 1e-12
    assert abs(out[F["qv"]] - qv + dq) <= 4 * np.spacing(qv)
    if regime == "growth":
        assert out[F["n" + sp]] == n
    else:
        assert abs((out[F["n" + sp]] - n) / (dq * n / q) - 1.0) < 1e-12
    assert abs(P("cp") * (out[F["T"]] - T) - (P("Lv") + P("Lf")) * dq) <= 4 * P("cp") * np.spacing(T)


# ------------------------------------------------------------ a10 limiter
def _liq(s):
    return s[F["qc"]] + s[F["qr"]]


def _ice(s):
    return s[F["qi"]] + s[F["qs"]] + s[F["qg"]]


def _mixed_cases():
    rng = np.random.default_rng(7)
    fld = synth.make_state("deep_convective", 64, 60, synth.dz_stretched(60), seed=3)
    pts = fld[:, :, :64].reshape(16, -1).T
    return pts[rng.choice(pts.shape[0], 200, replace=False)]


@pytest.mark.parametrize("dt", [1.0, 30.0, 3600.0])
def test_point_update_conserves_water_and_static_energy(dt):
    cp, Lv, Ls = P("cp"), P("Lv"), P("Lv") + P("Lf")
    for st in _mixed_cases():
        out = O.point(st, dt)
        qt0 = st[F["qv"]] + _liq(st) + _ice(st)
        qt1 = out[F["qv"]] + _liq(out) + _ice(out)
        assert abs(qt1 - qt0) <= 16 * np.spacing(qt0)
        # liquid-ice static energy cp T - Lv q_liq - Ls q_ice is unchanged
        h0 = cp * st[F["T"]] - Lv * _liq(st) - Ls * _ice(st)
        h1 = cp * out[F["T"]] - Lv * _liq(out) - Ls * _ice(out)
        assert abs(h1 - h0) <= 1e-10 * cp * st[F["T"]]
        # aerosol + cloud droplets: activation only moves number between them
        assert out[F["na"]] >= 0.0
        for name in ("qv", "qc", "qr", "qi", "qs", "qg", "nc", "nr", "ni", "ns", "ng"):
            assert out[F[name]] >= -8 * np.spacing(max(abs(st[F[name]]), 1e-300)), name


def test_limiter_inactive_is_forward_euler():
    # With a short step no pool runs dry: the update is X + dt * (sources - sinks).
    T, p, rho = 262.0, 7e4, 0.9
    st = _state(T=T, qv=0.98 * _qs(T, p), qc=2e-4, nc=1e8, qr=1e-4, nr=5e3, qi=1e-5, ni=1e5,
                qs=1e-4, ns=1e4, qg=1e-4, ng=1e3, p=p, rho=rho)
    dt = 1e-3
    out = O.point(st, dt)
    # the rates act on the state after saturation adjustment (w = 0: no activation)
    st[F["T"]], st[F["qv"]], st[F["qc"]] = O.satadj(p, st[F["T"]], st[F["qv"]], st[F["qc"]])
    R = O.rates(st, dt)
    rc = st[F["nc"]] / st[F["qc"]]
    exp_qc = st[F["qc"]] - dt * (R["aut"] + R["acc"] + R["rims"] + R["rimg"])
    exp_qg = st[F["qg"]] + dt * (R["rims"] + R["rimg"] + R["depg"])
    exp_nc = st[F["nc"]] - dt * ((R["aut"] + R["acc"] + R["rims"] + R["rimg"]) * rc + R["scc"])
    mr0 = 4 / 3 * math.pi * 1000.0 * 25e-6 ** 3
    exp_nr = st[F["nr"]] + dt * (R["aut"] / mr0 - R["scr"])
    assert abs(out[F["qc"]] / exp_qc - 1) < 1e-13
    assert abs(out[F["qg"]] / exp_qg - 1) < 1e-13
    assert abs(out[F["nc"]] / exp_nc - 1) < 1e-13
    assert abs(out[F["nr"]] / exp_nr - 1) < 1e-13


def test_limiter_exhausts_pool_without_going_negative():
    # A very long step: accretion + autoconversion would remove far more cloud
    # than exists, so the cloud pool must end at (almost exactly) zero.
    T, p, rho = 285.0, 9e4, 1.1
    st = _state(T=T, qv=0.95 * _qs(T, p), qc=1e-4, nc=5e7, qr=1e-3, nr=1e3, p=p, rho=rho)
    out = O.point(st, 1e5)
    assert 0.0 <= out[F["qc"]] < 1e-18 or abs(out[F["qc"]]) <= 4 * np.spacing(1e-4)
    assert out[F["nc"]] >= -4 * np.spacing(5e7)


def test_inactive_point_is_bitwise_unchanged():
    p = 9e4
    st = _state(T=290.0, qv=0.9 * _qs(290.0, p), p=p, w=1.5)
    out = O.point(st, 1.0)
    assert np.array_equal(out, st[:13])


@pytest.mark.parametrize("bad", [float("nan"), float("inf"), -float("inf")])
def test_a_non_finite_value_in_any_field_is_reported(bad):
    """The step reports a non-finite value (error bit) wherever it sits: in
    each of the 13 prognostic fields of the standard state, and in each field
    a configuration adds after the inputs (aerosol masses, sixth moments),
    planted one at a time at an inactive point (clear, dry air) of an
    otherwise clean domain, at an inner point and at the edges of the level
    and column ranges; the clean domain reports nothing."""
    nlev, ncols = 12, 4
    dz = np.full(nlev, 100.0)
    T, p = 290.0, 9e4

    def clean(nf):
        fld = np.zeros((nf, nlev, ncols))
        fld[F["T"]], fld[F["p"]], fld[F["rho"]] = T, p, 1.08
        fld[F["qv"]] = 0.5 * O.qsat(O.es_liq(T), p)
        fld[F["na"]] = 1e8
        return fld

    steps = [(O.NFIELDS, lambda f: O.step(f, ncols, dz, 1.0)[2], list(range(13))),
             (O.NFIELDS_AERO, lambda f: O.step_aero(f, ncols, dz, 1.0)[1], [16, 17, 18]),
             (O.NFIELDS_AEROC, lambda f: O.step_aero_cold(f, ncols, dz, 1.0)[1], list(range(16, 22))),
             (O.NFIELDS_3M, lambda f: O.step_3m(f, ncols, dz, 1.0)[1], [16]),
             (O.NFIELDS_3MC, lambda f: O.step_3m_cold(f, ncols, dz, 1.0)[1], list(range(16, 20)))]
    # an inner point, the last level of an inner column and the first level of the last column
    where = [(7, 2), (nlev - 1, 1), (0, ncols - 1)]
    for nf, run, fields in steps:
        assert run(clean(nf)) == 0
        for f in fields:
            for k, c in where:
                fld = clean(nf)
                fld[f, k, c] = bad
                assert run(fld) & O.ERR_NONFINITE, (nf, f, k, c)


# ---------------------------------------------------------- a12 sedimentation
def test_sedimentation_courant_one_is_exact_shift():
    # Large rain drops fall at the cap; with dz = vmax dt every level's
    # content moves down exactly one level per step.
    nlev = 6
    vmax = P("vmax_r")
    dt = 2.0
    dz = np.full(nlev, vmax * dt)
    rho = np.ones(nlev)
    q = np.zeros((4, nlev))
    n = np.zeros((4, nlev))
    q[0] = [1e-4, 2e-4, 3e-4, 4e-4, 5e-4, 6e-4]
    n[0] = q[0] / (math.pi / 6 * 1000 * (4e-3) ** 3) * 1e-2   # very large drops
    lam = O.lam("r", q[0, 2], n[0, 2])
    assert O.vq("r", 1.0, lam) == vmax            # mass-weighted speed is capped
    q1, n1, pr, ns, err = O.sediment_column(q, n, rho, dz, dt)
    assert err == 0 and ns[0] == 1
    np.testing.assert_allclose(q1[0, :-1], q[0, 1:], rtol=1e-15, atol=0)
    assert q1[0, -1] == 0.0
    assert abs(pr[0] - q[0, 0] * vmax * dt) < 1e-18
    # number falls slower than mass (V_n < V_q): the number budget still closes
    assert np.all(n1[0] >= 0.0) and np.sum(n1[0]) < np.sum(n[0])


def test_sedimentation_single_level_geometric_decay():
    # One level, constant (capped) mass-weighted speed, Courant number C = 2.5
    # -> 3 substeps, each removing C/3 of the content: q (1 - C/3)^3.
    vmax = P("vmax_r")
    dz = np.array([40.0])
    dt = 2.5 * 40.0 / vmax
    rho = np.array([0.8])
    q = np.zeros((4, 1)); n = np.zeros((4, 1))
    q[0, 0] = 5e-3
    n[0, 0] = 1.0     # few, huge drops: capped mass-weighted speed
    q1, n1, pr, ns, err = O.sediment_column(q, n, rho, dz, dt)
    assert ns[0] == 3 and err == 0
    assert abs(q1[0, 0] / (5e-3 * (1 - 2.5 / 3) ** 3) - 1) < 1e-13
    assert abs(pr[0] - 0.8 * 40.0 * (5e-3 - q1[0, 0])) < 1e-16


def test_sedimentation_budget_positivity_and_substeps():
    rng = np.random.default_rng(11)
    nlev = 40
    dz = synth.dz_stretched(nlev, 5.0, 50.0)
    rho = np.linspace(1.2, 0.5, nlev)
    for dt in (1.0, 10.0, 30.0):
        q = np.where(rng.random((4, nlev)) < 0.6, 10 ** rng.uniform(-6, -3, (4, nlev)), 0.0)
        n = q / (math.pi / 6 * 500 * (10 ** rng.uniform(-4, -2.5, (4, nlev))) ** 3)
        q1, n1, pr, ns, err = O.sediment_column(q, n, rho, dz, dt)
        assert err == 0
        for m in range(4):
            before = np.sum(rho * dz * q[m])
            after = np.sum(rho * dz * q1[m])
            assert abs(after + pr[m] - before) <= 1e-13 * before
            assert np.all(q1[m] >= -1e-25) and np.all(n1[m] >= -1e-10)
        if dt >= 10.0:
            assert ns.max() > 1


def test_substep_count_is_ceil_of_courant():
    vmax = P("vmax_r")
    for C, expect in ((0.4, 1), (1.0, 1), (1.5, 2), (3.2, 4)):
        dz = np.array([100.0, 100.0])
        dt = C * 100.0 / vmax
        q = np.zeros((4, 2)); n = np.zeros((4, 2))
        q[0, 1] = 1e-3; n[0, 1] = 1.0
        _, _, _, ns, _ = O.sediment_column(q, n, np.ones(2), dz, dt)
        assert ns[0] == expect


def test_cfl_cap_sets_error_bit():
    dz = np.array([1.0])
    q = np.zeros((4, 1)); n = np.zeros((4, 1))
    q[0, 0] = 1e-3; n[0, 0] = 1.0
    _, _, _, ns, err = O.sediment_column(q, n, np.ones(1), dz, 1000.0)
    assert err & O.ERR_CFL and ns[0] == O.NSUB_MAX


# ------------------------------------------------------------- whole step
def test_step_column_budgets_and_independence():
    fld, dz, nc, nl, dt, _ = synth.workload("stratus_16x16x50", ncols=48)
    f0 = fld.copy()
    pr, nsub, err = O.step(fld, nc, dz, dt, want_nsub=True)
    assert err == 0
    rho = f0[F["rho"]]
    names = ("qv", "qc", "qr", "qi", "qs", "qg")
    w0 = sum((f0[F[x]] * rho * dz[:, None]).sum(0) for x in names)[:nc]
    w1 = sum((fld[F[x]] * rho * dz[:, None]).sum(0) for x in names)[:nc]
    assert np.max(np.abs(w1 + pr[:, :nc].sum(0) - w0) / w0) < 1e-14
    # columns are independent: a permuted domain gives permuted results, bitwise
    perm = np.random.default_rng(5).permutation(nc)
    g = f0.copy()
    g[:, :, :nc] = f0[:, :, perm]
    pr2, _, _ = O.step(g, nc, dz, dt)
    assert np.array_equal(g[:, :, :nc], fld[:, :, perm])
    assert np.array_equal(pr2[:, :nc], pr[:, perm])
    # inputs p, rho, w are never written
    assert np.array_equal(fld[13:], f0[13:])


def test_each_species_precipitation_is_its_own_column_loss():
    """Ice, snow and graupel (no cloud, no rain) falling through air
    saturated over ice below the nucleation temperature, so that no process
    moves water between them: each species' surface precipitation row
    (r, i, s, g) is that species' column loss, and the rain row stays zero."""
    nlev, ncols, dt = 10, 3, 10.0
    dz = np.full(nlev, 100.0)
    T, p = 250.0, 7.0e4
    fld = np.zeros((O.NFIELDS, nlev, ncols))
    fld[F["T"]], fld[F["p"]], fld[F["rho"]] = T, p, p / (P("Rd") * T)
    fld[F["qv"]] = O.qsat(O.es_ice(T), p)
    fld[F["na"]] = 1e8
    for sp, q, n in (("i", 1e-5, 1e5), ("s", 1e-4, 1e4), ("g", 3e-4, 2e3)):
        fld[F["q" + sp]], fld[F["n" + sp]] = q, n
    f0 = fld.copy()
    pr, _, err = O.step(fld, ncols, dz, dt)
    assert err == 0
    m = f0[F["rho"]] * dz[:, None]
    assert np.all(pr[0] == 0.0)
    for row, sp in ((1, "qi"), (2, "qs"), (3, "qg")):
        loss = ((f0[F[sp]] - fld[F[sp]]) * m).sum(0)
        assert np.all(pr[row] > 0.0), sp
        np.testing.assert_allclose(pr[row], loss, rtol=1e-9, atol=0)


def test_step_threads_do_not_change_results():
    fld, dz, nc, nl, dt, _ = synth.workload("stratus_256x256x100", ncols=64, nlev=100)
    a, b = fld.copy(), fld.copy()
    O.step(a, nc, dz, dt, nthreads=1)
    O.step(b, nc, dz, dt, nthreads=4)
    assert np.array_equal(a, b)


def test_gas_constants_follow_from_the_molar_masses():
    """The specific gas constants of dry air and of water vapour are the
    universal gas constant over the molar masses (to the digits given), and
    their ratio is the familiar 0.622."""
    R, Ma, Mw = P("Rgas"), P("Ma"), P("Mw")
    assert R == 8.314 and Ma == 0.028965 and Mw == 0.018015
    assert abs(P("Rd") * Ma / R - 1.0) < 1e-4
    assert abs(P("Rv") * Mw / R - 1.0) < 1e-4
    assert abs(P("Rd") / P("Rv") - 0.622) < 5e-4


def test_parameters_are_the_cited_values():
    assert P("kk_aut") == 1350.0 and P("kk_aut_qc") == 2.47 and P("kk_aut_nc") == -1.79
    assert P("kk_acc") == 67.0 and P("kk_acc_exp") == 1.15
    assert P("kc_sb") == 9.44e9 and P("kr_sb") == 5.78
    assert P("mey_a") == 1e3 and P("mey_b") == -0.639 and P("mey_c") == 12.96
    assert P("es_l0") == 611.2 and P("es_la") == 17.67 and P("es_lb") == 243.5
    assert P("nc_min_cm3") == 1.0 and P("nu_c") == 1.0
    # thermodynamic and transport constants (standard values), the fall-speed
    # reference density, the ice nucleation threshold and crystal mass, the
    # new-raindrop radius, the presence threshold, the riming efficiency and
    # the Courant limit per substep
    assert P("T0") == 273.15 and P("cp") == 1005.0 and P("Lv") == 2.5e6 and P("Lf") == 3.34e5
    assert P("g") == 9.81 and P("rho_w") == 1000.0 and P("rho0") == 1.2
    assert P("Ka") == 2.4e-2 and P("Dv") == 2.26e-5 and P("mu_air") == 1.72e-5
    assert P("T_nuc") == 268.15 and P("m_i0") == 1e-12 and P("r_r0") == 25e-6
    assert P("q_min") == 1e-14 and P("e_rim") == 1.0 and P("c_max") == 1.0
    # the aerosol mode: an accumulation mode of ammonium sulphate (kappa of
    # Petters & Kreidenweis 2007) and the surface tension of water
    assert P("arg_rm") == 0.05e-6 and P("arg_sigma") == 1.5 and P("arg_kappa") == 0.61
    assert P("surft") == 0.0761
    assert math.isnan(P("no_such_parameter"))
