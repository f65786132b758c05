"""Pins of the oracle's triple-moment warm rain.

The shape parameter is recovered from the three moments it was built from;
the gamma-distribution algebra at any shape matches numerical quadrature;
where nothing can change the rain's shape (no autoconversion) the step is the
two-moment warm step; autoconversion makes monodisperse rain (G = 1);
accretion-free rain keeps its shape through evaporation and self-collection;
the sixth moment shifts exactly one level at Courant number 1; water is
conserved.
"""
import numpy as np
import pytest

import oracle as O
from paper_2010_14823_gb300 import synth

scipy = pytest.importorskip("scipy")
from scipy.integrate import quad  # noqa: E402

F = synth.FIDX
ZR = 16
A_R = O.param("a_r")
D0 = 2.0 * O.param("r_r0")


def G(mu):
    """z n / M3^2 of a gamma distribution of shape mu (its definition)."""
    return (mu + 4) * (mu + 5) * (mu + 6) / ((mu + 1) * (mu + 2) * (mu + 3))


def z_of(q, n, mu):
    return G(mu) * (q / A_R) ** 2 / n


@pytest.mark.parametrize("mu", [0.0, 0.3, 1.0, 2.5, 7.0, 13.0, 20.0])
def test_shape_is_recovered_from_the_moments(mu):
    for q, n in ((1e-4, 1e3), (2e-3, 5e4), (5e-6, 10.0)):
        assert abs(O.rain_mu(q, n, z_of(q, n, mu)) - mu) < 1e-9


def test_the_shape_solver_converges_across_the_whole_range():
    """Four Newton steps from the closed-form start reach the shape to
    rounding anywhere in [0, 20] (201 shapes, two orders of magnitude of q
    and n)."""
    for mu in np.linspace(0.0, 20.0, 201):
        for q, n in ((1e-3, 1e3), (4e-5, 70.0)):
            assert abs(O.rain_mu(q, n, z_of(q, n, mu)) - mu) < 1e-12, mu


def test_shape_clamps_and_absent_rain():
    q, n = 1e-3, 1e4
    assert O.rain_mu(q, n, 1.5 * z_of(q, n, 0.0)) == 0.0          # broader than mu = 0
    assert O.rain_mu(q, n, 0.999 * z_of(q, n, 20.0)) == 20.0      # narrower than mu = 20
    assert O.rain_mu(0.0, n, 1e-12) == O.param("mu_r")
    assert O.rain_mu(q, 0.0, 1e-12) == O.param("mu_r")


@pytest.mark.parametrize("mu", [0.7, 4.0, 11.0])
def test_gamma_algebra_at_any_shape_matches_quadrature(mu):
    rho, q, n = 1.1, 1e-3, 3e3
    lam = O.lam_mu("r", q, n, mu)
    a, b = A_R, 3.0
    # N0 fixed by the mass: rho q = a N0 Gamma(mu+b+1) / lam^(mu+b+1)
    from math import gamma
    N0 = rho * q * lam ** (mu + b + 1) / (a * gamma(mu + b + 1))
    nd = lambda D: N0 * D ** mu * np.exp(-lam * D)   # noqa: E731
    up = 60.0 / lam
    M = lambda k: quad(lambda D: D ** k * nd(D), 0, up, limit=400, epsabs=0)[0]   # noqa: E731
    assert np.isclose(a * M(3.0), rho * q, rtol=1e-8, atol=0.0)
    assert np.isclose(M(0.0), rho * n, rtol=1e-8, atol=0.0)
    for k in (1.0, 1.75, 6.0):
        assert np.isclose(O.moment_mu("r", rho, q, lam, k, mu), M(k), rtol=1e-8, atol=0.0)
    cv, dv, rho0 = O.param("cv_r"), O.param("dv_r"), O.param("rho0")
    fac = cv * (rho0 / rho) ** 0.4
    for k, fn in ((3.0, O.vq_mu), (0.0, O.vn_mu), (6.0, O.vz_mu)):
        w = quad(lambda D: fac * D ** dv * D ** k * nd(D), 0, up, limit=400, epsabs=0)[0] / M(k)
        assert np.isclose(fn("r", rho, lam, mu), min(w, O.param("vmax_r")), rtol=1e-8, atol=0.0)
    nu = O.param("mu_air") / rho
    sc = nu / O.param("Dv")
    vent = quad(lambda D: D * (0.78 + 0.31 * sc ** (1 / 3) * np.sqrt(fac * D ** dv * D / nu)) * nd(D), 0, up,
                limit=400, epsabs=0)[0]
    assert np.isclose(O.vent_integral_mu("r", rho, q, lam, mu), vent, rtol=1e-8, atol=0.0)


def _rain_state(ncols, nlev, seed, mu=None):
    """Deep-convective state, rain's z consistent with shape mu (default: random shapes)."""
    dz = synth.dz_stretched(nlev)
    base = synth.make_state("deep_convective", ncols, nlev, dz, seed=seed)
    fld = np.zeros((17,) + base.shape[1:])
    fld[:16] = base
    rng = np.random.default_rng(seed)
    qr, nr = base[F["qr"]], base[F["nr"]]
    shape = np.full(qr.shape, mu) if mu is not None else rng.uniform(0.0, 8.0, qr.shape)
    ok = (qr > 1e-14) & (nr > 0)
    fld[ZR][ok] = G(shape[ok]) * (qr[ok] / A_R) ** 2 / nr[ok]
    return np.ascontiguousarray(fld), dz


def _subsaturate_and_clear(fld):
    for k in range(fld.shape[1]):
        for c in range(fld.shape[2]):
            qs = O.qsat(O.es_liq(fld[F["T"], k, c]), fld[F["p"], k, c])
            fld[F["qv"], k, c] = min(fld[F["qv"], k, c], 0.97 * qs)
    fld[F["qc"]] = 0.0
    fld[F["nc"]] = 0.0


def test_reduces_to_two_moment_where_the_shape_cannot_change():
    """No cloud and subsaturated air: no autoconversion, the only source of a
    shape change, so with z at shape 0 (the two-moment rain's) the step is the
    two-moment warm step."""
    fld, dz = _rain_state(40, 150, seed=81, mu=0.0)
    _subsaturate_and_clear(fld)
    a = fld.copy()
    pa, ea = O.step_3m(a, 40, dz, 1.0)
    b = np.ascontiguousarray(fld[:16].copy())
    pb, _, eb = O.step(b, 40, dz, 1.0, warm=True)
    assert ea == 0 and eb == 0
    assert not np.array_equal(a[F["qr"]], fld[F["qr"]])
    for f in range(13):
        assert np.allclose(a[f, :, :40], b[f, :, :40], rtol=1e-12, atol=1e-30), synth.FIELDS[f]
    assert np.allclose(pa[:, :40], pb[:, :40], rtol=1e-12, atol=0)


@pytest.mark.parametrize("dt", [1.0, 3.0])
def test_autoconversion_makes_monodisperse_rain(dt):
    st = np.zeros(17)
    T, p = 285.0, 9.0e4
    qs = O.qsat(O.es_liq(T), p)
    st[F["T"]], st[F["p"]], st[F["rho"]] = T, p, p / (287.04 * T)
    st[F["qv"]], st[F["qc"]], st[F["nc"]], st[F["na"]] = qs, 1e-3, 5e7, 1e8
    out = O.point_3m(st, dt)
    q, n, z = out[F["qr"]], out[F["nr"]], out[13]
    assert q > 0 and n > 0
    assert np.isclose(z, n * D0 ** 6, rtol=1e-12, atol=0.0)
    assert np.isclose(z * n / (q / A_R) ** 2, 1.0, rtol=1e-9, atol=0.0)


def test_rain_keeps_its_shape_through_evaporation_and_self_collection():
    for mu in (0.0, 2.0, 9.0):
        st = np.zeros(17)
        T, p = 290.0, 9.5e4
        qs = O.qsat(O.es_liq(T), p)
        st[F["T"]], st[F["p"]], st[F["rho"]] = T, p, p / (287.04 * T)
        st[F["qv"]], st[F["qr"]], st[F["nr"]] = 0.8 * qs, 1e-3, 2e3
        st[ZR] = z_of(1e-3, 2e3, mu)
        out = O.point_3m(st, 5.0)
        q, n, z = out[F["qr"]], out[F["nr"]], out[13]
        assert q < 1e-3 and n < 2e3
        assert abs(O.rain_mu(q, n, z) - mu) < 1e-9


def test_sixth_moment_shifts_one_level_at_courant_one():
    nlev = 8
    vmax = O.param("vmax_r")
    dz = np.full(nlev, 100.0)
    dt = dz[0] / vmax
    rho = np.full(nlev, 1.0)
    q = np.zeros(nlev)
    n = np.zeros(nlev)
    q[5], n[5] = 4e-3, 10.0                       # few, large drops: the mass and z speeds capped at vmax
    z = np.zeros(nlev)
    z[5] = z_of(q[5], n[5], 1.0)
    rho_k = 1.0
    lam = O.lam_mu("r", q[5], n[5], 1.0)
    assert O.vq_mu("r", rho_k, lam, 1.0) == vmax and O.vz_mu("r", rho_k, lam, 1.0) == vmax
    q1, n1, z1, pr, ns, err = O.sediment_rain_3m(q, n, z, rho, dz, dt)
    assert err == 0 and ns == 1
    assert np.array_equal(q1, np.roll(q, -1))
    assert np.allclose(z1, np.roll(z, -1), rtol=1e-15, atol=1e-15 * z[5])   # to one rounding
    assert 0.0 < n1[5] < n[5] and np.isclose(n1.sum(), n.sum(), rtol=1e-12, atol=0.0)   # the number falls slower


def test_column_water_budget_with_random_shapes():
    fld, dz = _rain_state(32, 150, seed=82)
    out = fld.copy()
    pr, err = O.step_3m(out, 32, dz, 1.0)
    assert err == 0
    rho = fld[F["rho"], :, :32]
    liq = ("qv", "qc", "qr")
    w0 = sum((fld[F[x], :, :32] * rho * dz[:, None]).sum(0) for x in liq)
    w1 = sum((out[F[x], :, :32] * rho * dz[:, None]).sum(0) for x in liq)
    assert np.allclose(w1 + pr[0, :32], w0, rtol=1e-12, atol=0)
    assert (out[ZR, :, :32] >= 0).all()


# ------------------------------------------------ cold configuration: r, i, s, g
ZC = {"r": 16, "i": 17, "s": 18, "g": 19}
QF = {"r": F["qr"], "i": F["qi"], "s": F["qs"], "g": F["qg"]}
NF = {"r": F["nr"], "i": F["ni"], "s": F["ns"], "g": F["ng"]}


def _z_at(sp, q, n, mu):
    return G(mu) * (q / O.param(f"a_{sp}")) ** 2 / n


def _cold_state(ncols, nlev, seed, fixed_shape=False):
    dz = synth.dz_stretched(nlev)
    base = synth.make_state("deep_convective", ncols, nlev, dz, seed=seed)
    fld = np.zeros((20,) + base.shape[1:])
    fld[:16] = base
    rng = np.random.default_rng(seed)
    for sp in "risg":
        q, n = base[QF[sp]], base[NF[sp]]
        mu = np.full(q.shape, O.param(f"mu_{sp}")) if fixed_shape else rng.uniform(0.0, 8.0, q.shape)
        ok = (q > 1e-14) & (n > 0)
        fld[ZC[sp]][ok] = _z_at(sp, q[ok], n[ok], mu[ok])
    return np.ascontiguousarray(fld), dz


def _point(T, p, **kw):
    st = np.zeros(20)
    st[F["T"]], st[F["p"]], st[F["rho"]] = T, p, p / (287.04 * T)
    for k, v in kw.items():
        st[ZC[k[1]] if k.startswith("z") else F[k]] = v
    return st


def test_melting_gives_rain_the_melting_species_shape():
    """Snow melting into no rain: the rain made is the melted part of the
    snow's population, so its shape (G = z n / (q/a)^2) is the snow's; the
    snow loses mass and number in proportion and keeps its shape."""
    T, p = 276.0, 9.0e4
    qs = O.qsat(O.es_liq(T), p)
    for mu in (0.5, 3.0, 9.0):
        q, n = 2e-4, 5e3
        st = _point(T, p, qv=0.9 * qs, qs=q, ns=n, zs=_z_at("s", q, n, mu), na=1e8)
        out = O.point_3m_cold(st, 5.0)
        assert 0.0 < out[F["qr"]] < q and out[F["nr"]] > 0
        assert abs(O.shape_mu("r", out[F["qr"]], out[F["nr"]], out[13]) - mu) < 1e-9
        assert abs(O.shape_mu("s", out[F["qs"]], out[F["ns"]], out[15]) - mu) < 1e-9
        # the sixth moment is conserved in particle-mass units: (m / a_r)^2 summed
        a_r, a_s = O.param("a_r"), O.param("a_s")
        assert np.isclose(out[13] + (a_s / a_r) ** 2 * out[15], (a_s / a_r) ** 2 * st[ZC["s"]], rtol=1e-12, atol=0.0)


def test_melting_snow_adds_its_sixth_moment_to_existing_rain():
    """Snow melting into rain already present, in air saturated over water
    (no evaporation, no cloud): the rain after the step is the superposition
    of its own population, whose shape (G) self-collection does not change,
    and the melted part of the snow, one drop per melted particle carrying
    (a_s / a_r)^2 times the melted fraction of the snow's sixth moment.
    Masses and numbers of the two parts come from the snow's losses; moments
    of superposed populations add."""
    T, p = 276.0, 9.0e4
    qsl = O.qsat(O.es_liq(T), p)
    a_r, a_s = O.param("a_r"), O.param("a_s")
    for dt in (1.0, 5.0):
        for mu_r, mu_s in ((1.0, 4.0), (6.0, 0.5)):
            qr0, nr0, qs0, ns0 = 3e-4, 2e3, 2e-4, 5e3
            st = _point(T, p, qv=qsl, qr=qr0, nr=nr0, zr=_z_at("r", qr0, nr0, mu_r),
                        qs=qs0, ns=ns0, zs=_z_at("s", qs0, ns0, mu_s), na=1e8)
            out = O.point_3m_cold(st, dt)
            q_m, n_m = qs0 - out[F["qs"]], ns0 - out[F["ns"]]      # the melted part
            assert 0.0 < q_m < qs0 and 0.0 < n_m < ns0
            assert np.isclose(out[F["qr"]], qr0 + q_m, rtol=1e-13, atol=0.0)
            q_own, n_own = out[F["qr"]] - q_m, out[F["nr"]] - n_m  # rain's own population
            assert n_own < nr0                                      # self-collection acted
            z_own = G(mu_r) * (q_own / a_r) ** 2 / n_own
            z_melt = (a_s / a_r) ** 2 * (q_m / qs0) * st[ZC["s"]]
            assert np.isclose(out[13], z_own + z_melt, rtol=1e-10, atol=0.0), (dt, mu_r, mu_s)


@pytest.mark.parametrize("dt", [1.0, 4.0])
def test_nucleation_makes_monodisperse_ice(dt):
    T, p = 255.0, 5.0e4
    qsi, qsl = O.qsat(O.es_ice(T), p), O.qsat(O.es_liq(T), p)
    st = _point(T, p, qv=0.5 * (qsi + qsl), na=1e8)
    out = O.point_3m_cold(st, dt)
    q, n, z = out[F["qi"]], out[F["ni"]], out[14]
    assert q > 0 and n > 0
    assert np.isclose(z * n / (q / O.param("a_i")) ** 2, 1.0, rtol=1e-9, atol=0.0)
    assert np.isclose(z, n * (O.param("m_i0") / O.param("a_i")) ** 2, rtol=1e-12, atol=0.0)


@pytest.mark.parametrize("si", [1.005, 1.05])
def test_nucleation_just_above_ice_saturation(si):
    """A point holding no hydrometeor, subsaturated over water but
    supersaturated over ice below the nucleation temperature, is active:
    ice nucleates there exactly as in the two-moment cold step (the
    activity rule's ice-supersaturation clause, however small the excess)."""
    T, p = 255.0, 5.0e4
    qsi, qsl = O.qsat(O.es_ice(T), p), O.qsat(O.es_liq(T), p)
    assert si * qsi < qsl
    st = _point(T, p, qv=si * qsi, na=1e8)
    out = O.point_3m_cold(st, 1.0)
    assert out[F["qi"]] > 0.0 and out[F["ni"]] > 0.0
    assert np.array_equal(out[:13], O.point(st[:16], 1.0))


def test_deposition_keeps_every_ice_species_shape():
    T, p = 270.0, 7.0e4                      # warmer than nucleation, supersaturated over ice only
    qsi, qsl = O.qsat(O.es_ice(T), p), O.qsat(O.es_liq(T), p)
    kw = {"qv": 0.5 * (qsi + qsl), "na": 1e8}
    mus = {"i": 1.5, "s": 4.0, "g": 7.0}
    for sp, (q, n) in {"i": (1e-5, 1e5), "s": (1e-4, 1e4), "g": (3e-4, 2e3)}.items():
        kw["q" + sp], kw["n" + sp], kw["z" + sp] = q, n, _z_at(sp, q, n, mus[sp])
    st = _point(T, p, **kw)
    out = O.point_3m_cold(st, 2.0)
    for sp, off in (("i", 14), ("s", 15), ("g", 16)):
        assert out[QF[sp]] > st[QF[sp]]                      # grew
        assert abs(O.shape_mu(sp, out[QF[sp]], out[NF[sp]], out[off]) - mus[sp]) < 1e-9


def test_cold_reduces_to_two_moment_where_no_shape_can_change():
    """No cloud (no autoconversion, no riming), subsaturated over ice and over
    water (no nucleation, no deposition growth that matters), no ice species
    where T > T0 (no melting): with z at the species' fixed shapes the 16
    fields are those of the two-moment cold step."""
    fld, dz = _cold_state(40, 150, seed=83, fixed_shape=True)
    T0 = O.param("T0")
    for k in range(fld.shape[1]):
        for c in range(40):
            T, p = fld[F["T"], k, c], fld[F["p"], k, c]
            qs = min(O.qsat(O.es_liq(T), p), O.qsat(O.es_ice(T), p))
            fld[F["qv"], k, c] = min(fld[F["qv"], k, c], 0.97 * qs)
            if T > T0:
                for sp in "isg":
                    fld[QF[sp], k, c] = fld[NF[sp], k, c] = fld[ZC[sp], k, c] = 0.0
    fld[F["qc"]] = 0.0
    fld[F["nc"]] = 0.0
    a = fld.copy()
    pa, ea = O.step_3m_cold(a, 40, dz, 1.0)
    b = np.ascontiguousarray(fld[:16].copy())
    pb, _, eb = O.step(b, 40, dz, 1.0)
    assert ea == 0 and eb == 0
    assert not np.array_equal(a[F["qg"]], fld[F["qg"]])
    for f in range(13):
        assert np.allclose(a[f, :, :40], b[f, :, :40], rtol=1e-11, atol=1e-30), synth.FIELDS[f]
    assert np.allclose(pa[:, :40], pb[:, :40], rtol=1e-11, atol=0)


def test_cold_equals_warm_on_an_ice_free_warm_state():
    """No ice anywhere and warmer than the nucleation threshold: the cold
    triple-moment step is the warm one bit for bit (rain fields and z_r)."""
    fld, dz, ncols, nlev, dt, _ = synth.workload("stratus_16x16x50")
    top = int(np.argmax(fld[F["T"], :, :ncols].min(axis=1) < O.param("T_nuc") + 1.0))
    sub = np.ascontiguousarray(fld[:, :top, :])
    for sp in "isg":
        sub[QF[sp]] = sub[NF[sp]] = 0.0
    rng = np.random.default_rng(84)
    qr, nr = sub[F["qr"]], sub[F["nr"]]
    zr = np.zeros(qr.shape)
    ok = (qr > 1e-14) & (nr > 0)
    zr[ok] = G(rng.uniform(0.0, 6.0, qr.shape)[ok]) * (qr[ok] / A_R) ** 2 / nr[ok]
    warm = np.zeros((17,) + sub.shape[1:])
    warm[:16], warm[16] = sub, zr
    cold = np.zeros((20,) + sub.shape[1:])
    cold[:16], cold[16] = sub, zr
    warm, cold = np.ascontiguousarray(warm), np.ascontiguousarray(cold)
    dzs = np.ascontiguousarray(dz[:top])
    pw, ew = O.step_3m(warm, ncols, dzs, dt)
    pc, ec = O.step_3m_cold(cold, ncols, dzs, dt)
    assert ew == 0 and ec == 0
    assert not np.array_equal(warm[F["qr"]], sub[F["qr"]])
    assert np.array_equal(warm, cold[:17]) and np.array_equal(pw, pc)
    assert np.all(cold[17:] == 0.0)


def test_every_species_sixth_moment_falls_with_its_own_speed():
    """One substep from a single occupied level, Courant number 1/2: the level
    keeps 1 - v dt/dz of its mass and of its sixth moment, with v the
    mass- and the sixth-moment-weighted speeds at the diagnosed shape (each
    pinned by quadrature); the sixth moment falls faster (size sorting)."""
    nlev = 8
    for x, sp in enumerate("risg"):
        dz = np.full(nlev, 50.0)
        rho = np.full(nlev, 1.0)
        q, n, z = np.zeros((4, nlev)), np.zeros((4, nlev)), np.zeros((4, nlev))
        q[x, 5], n[x, 5] = 2e-4, 2e3
        z[x, 5] = _z_at(sp, q[x, 5], n[x, 5], 2.5)
        mu = O.shape_mu(sp, q[x, 5], n[x, 5], z[x, 5])
        lam = O.lam_mu(sp, q[x, 5], n[x, 5], mu)
        vq, vz = O.vq_mu(sp, 1.0, lam, mu), O.vz_mu(sp, 1.0, lam, mu)
        assert vz > vq, sp
        dt = 0.5 * dz[0] / vq
        q1, n1, z1, pr, ns, err = O.sediment_3m(q, n, z, rho, dz, dt)
        assert err == 0 and ns[x] == 1
        cq, cz = vq * dt / dz[0], min(vz, dz[0] / dt) * dt / dz[0]
        assert np.isclose(q1[x, 5], q[x, 5] * (1 - cq), rtol=1e-12, atol=0.0) and np.isclose(q1[x, 4], q[x, 5] * cq, rtol=1e-12, atol=0.0)
        assert np.isclose(z1[x, 5], z[x, 5] * (1 - cz), rtol=1e-12, atol=0.0) and np.isclose(z1[x, 4], z[x, 5] * cz, rtol=1e-12, atol=0.0)
        others = [y for y in range(4) if y != x]
        assert not q1[others].any() and not z1[others].any()


def test_cold_column_water_budget_with_random_shapes():
    fld, dz = _cold_state(32, 150, seed=85)
    out = fld.copy()
    pr, err = O.step_3m_cold(out, 32, dz, 1.0)
    assert err == 0
    rho = fld[F["rho"], :, :32]
    names = ("qv", "qc", "qr", "qi", "qs", "qg")
    w0 = sum((fld[F[x], :, :32] * rho * dz[:, None]).sum(0) for x in names)
    w1 = sum((out[F[x], :, :32] * rho * dz[:, None]).sum(0) for x in names)
    assert np.allclose(w1 + pr[:, :32].sum(0), w0, rtol=1e-12, atol=0)
    assert (out[16:, :, :32] >= 0).all()
    assert (out[16:, :, :32] > 0).any(axis=(1, 2)).all()


def test_an_inactive_point_keeps_its_sixth_moments():
    """A point the chain leaves unchanged (no hydrometeor, subsaturated over
    liquid and, when cold, over ice or warmer than T_nuc) keeps every field,
    its sixth moments included, even where they describe no species; an
    active point with rain absent has none left (the fixed-shape rule)."""
    p = 9e4
    for T in (290.0, 260.0):
        es = O.es_liq(T) if T > 273.15 else min(O.es_liq(T), O.es_ice(T))
        qv = 0.8 * O.qsat(es, p)
        warm = np.zeros(17)
        warm[F["T"]], warm[F["p"]], warm[F["rho"]], warm[F["qv"]], warm[F["na"]] = T, p, 1.1, qv, 1e8
        warm[ZR] = 3e-12
        out = O.point_3m(warm, 1.0)
        assert np.array_equal(out[:13], warm[:13]) and out[13] == warm[ZR]
        cold = np.zeros(20)
        cold[:16] = warm[:16]
        cold[16:20] = [3e-12, 1e-14, 2e-13, 5e-12]
        out = O.point_3m_cold(cold, 1.0)
        assert np.array_equal(out[:13], cold[:13]) and np.array_equal(out[13:], cold[16:20])
    # the same warm point made active by a little cloud: the absent rain's z is dropped
    act = np.zeros(17)
    act[F["T"]], act[F["p"]], act[F["rho"]], act[F["na"]] = 290.0, p, 1.1, 1e8
    act[F["qv"]] = 0.8 * O.qsat(O.es_liq(290.0), p)
    act[F["qc"]], act[F["nc"]], act[ZR] = 1e-5, 5e7, 3e-12
    out = O.point_3m(act, 1.0)
    assert out[13] == 0.0
