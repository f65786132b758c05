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
    assert np.isclose(a * M(3.0), rho * q, rtol=1e-8)
    assert np.isclose(M(0.0), rho * n, rtol=1e-8)
    for k in (1.0, 1.75, 6.0):
        assert np.isclose(O.moment_mu("r", rho, q, lam, k, mu), M(k), rtol=1e-8)
    cv, dv, rho0 = O.param("cv_r"), O.param("dv_r"), O.param("rho0")
    fac = cv * (rho0 / rho) ** 0.4
    for k, fn in ((3.0, O.vq_mu), (0.0, O.vn_mu), (6.0, O.vz_mu)):
        w = quad(lambda D: fac * D ** dv * D ** k * nd(D), 0, up, limit=400, epsabs=0)[0] / M(k)
        assert np.isclose(fn("r", rho, lam, mu), min(w, O.param("vmax_r")), rtol=1e-8)
    nu = O.param("mu_air") / rho
    sc = nu / O.param("Dv")
    vent = quad(lambda D: D * (0.78 + 0.31 * sc ** (1 / 3) * np.sqrt(fac * D ** dv * D / nu)) * nd(D), 0, up,
                limit=400, epsabs=0)[0]
    assert np.isclose(O.vent_integral_mu("r", rho, q, lam, mu), vent, rtol=1e-8)


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


def test_autoconversion_makes_monodisperse_rain():
    st = np.zeros(17)
    T, p = 285.0, 9.0e4
    qs = O.qsat(O.es_liq(T), p)
    st[F["T"]], st[F["p"]], st[F["rho"]] = T, p, p / (287.04 * T)
    st[F["qv"]], st[F["qc"]], st[F["nc"]], st[F["na"]] = qs, 1e-3, 5e7, 1e8
    out = O.point_3m(st, 1.0)
    q, n, z = out[F["qr"]], out[F["nr"]], out[13]
    assert q > 0 and n > 0
    assert np.isclose(z, n * D0 ** 6, rtol=1e-12)
    assert np.isclose(z * n / (q / A_R) ** 2, 1.0, rtol=1e-9)


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
    assert 0.0 < n1[5] < n[5] and np.isclose(n1.sum(), n.sum())   # the number falls slower


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
