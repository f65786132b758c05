"""Pins of the oracle's activated-aerosol mass (warm configuration).

Aerosol mass moves with the water: it is an addition to the warm step, so the
16 standard fields are exactly the warm step's; it is conserved per column
(free + in cloud + in rain + deposited); without activation the aerosol per
unit water in cloud and in rain cannot change in subsaturated air, through
evaporation, autoconversion, accretion or sedimentation alike; activation
takes the free aerosol's mean particle mass; cloud that evaporates returns all
of its aerosol.  In the cold configuration (aerosol also in ice, snow and
graupel) the 16 standard fields are the cold step's, total aerosol is
conserved with the deposition row, an ice-free warm state gives the warm
result bit for bit, melting and sublimation move exactly the melted and
sublimated shares, and each species' aerosol falls with its mass.
"""
import numpy as np

import oracle as O
from paper_2010_14823_gb300 import synth

F = synth.FIDX
MA, MAC, MAR = 16, 17, 18


def _aero_state(ncols, nlev, seed, ratio=None, w=None):
    dz = synth.dz_stretched(nlev)
    base = synth.make_state("deep_convective", ncols, nlev, dz, seed=seed)
    fld = np.zeros((19,) + base.shape[1:])
    fld[:16] = base
    rng = np.random.default_rng(seed)
    fld[MA] = rng.uniform(1e-9, 5e-9, base.shape[1:])         # ~100 cm^-3 of 0.05 um particles
    if ratio is None:
        fld[MAC] = fld[F["qc"]] * rng.uniform(1e-5, 1e-4, base.shape[1:])
        fld[MAR] = fld[F["qr"]] * rng.uniform(1e-5, 1e-4, base.shape[1:])
    else:
        fld[MAC] = ratio * fld[F["qc"]]
        fld[MAR] = ratio * fld[F["qr"]]
    if w is not None:
        fld[F["w"]] = w
    return np.ascontiguousarray(fld), dz


def test_standard_fields_are_the_warm_steps():
    fld, dz = _aero_state(48, 150, seed=1)
    a = fld.copy()
    pa, ea = O.step_aero(a, 48, dz, 1.0)
    b = np.ascontiguousarray(fld[:16].copy())
    pb, _, eb = O.step(b, 48, dz, 1.0, warm=True)
    assert ea == 0 and eb == 0
    assert np.array_equal(a[:16], b) and np.array_equal(pa[:4], pb)
    assert not np.array_equal(a[MAR], fld[MAR])


def test_column_aerosol_budget():
    for dt in (1.0, 30.0):
        fld, dz = _aero_state(48, 150, seed=2)
        a = fld.copy()
        pr, err = O.step_aero(a, 48, dz, dt)
        assert err == 0
        rho = fld[F["rho"], :, :48]
        m0 = ((fld[MA] + fld[MAC] + fld[MAR])[:, :48] * rho * dz[:, None]).sum(0)
        m1 = ((a[MA] + a[MAC] + a[MAR])[:, :48] * rho * dz[:, None]).sum(0)
        assert pr[4, :48].max() > 0.0
        assert np.allclose(m1 + pr[4, :48], m0, rtol=1e-12, atol=0)


def test_aerosol_per_water_is_invariant_without_activation_or_condensation():
    """Subsaturated air (the adjustment can only evaporate) and w < 0 (no
    activation): every remaining process moves aerosol in proportion to the
    water it moves, so aerosol per unit water in cloud and rain stays r."""
    r = 3.7e-5
    fld, dz = _aero_state(48, 150, seed=3, ratio=r, w=-1.0)
    for k in range(150):
        for c in range(48):
            qs = O.qsat(O.es_liq(fld[F["T"], k, c]), fld[F["p"], k, c])
            fld[F["qv"], k, c] = min(fld[F["qv"], k, c], 0.97 * qs)
    a = fld.copy()
    _, err = O.step_aero(a, 48, dz, 5.0)
    assert err == 0
    for q, m in ((F["qc"], MAC), (F["qr"], MAR)):
        qn, mn = a[q, :, :48], a[m, :, :48]
        assert not np.array_equal(qn, fld[q, :, :48])         # the water did move
        assert np.allclose(mn, r * qn, rtol=1e-11, atol=1e-30)
    assert np.array_equal(a[MA], fld[MA]) or np.all(a[MA] >= fld[MA])   # only returns to the free aerosol


def test_activation_takes_the_mean_particle_mass():
    st = np.zeros(19)
    T, p = 285.0, 9.0e4
    qs = O.qsat(O.es_liq(T), p)
    st[F["T"]], st[F["p"]], st[F["rho"]], st[F["w"]] = T, p, p / (287.04 * T), 2.0
    st[F["qv"]], st[F["qc"]], st[F["nc"]], st[F["na"]] = qs, 1e-4, 1e6, 1e8
    st[MA], st[MAC] = 4e-9, 0.0
    out = O.point_aero(st, 1e-9)                 # dt -> 0: activation only
    dn = st[F["na"]] - out[F["na"]]
    assert dn > 0
    assert np.isclose(out[14], st[MA] * dn / st[F["na"]], rtol=1e-9, atol=0.0)
    assert np.isclose(out[13] + out[14] + out[15], st[MA], rtol=1e-15, atol=0.0)


def test_evaporated_cloud_returns_all_its_aerosol():
    st = np.zeros(19)
    T, p = 290.0, 9.5e4
    qs = O.qsat(O.es_liq(T), p)
    st[F["T"]], st[F["p"]], st[F["rho"]] = T, p, p / (287.04 * T)
    st[F["qv"]], st[F["qc"]], st[F["nc"]], st[F["na"]] = 0.5 * qs, 1e-6, 1e7, 1e8
    st[MA], st[MAC] = 2e-9, 3e-10
    out = O.point_aero(st, 1.0)
    assert out[F["qc"]] == 0.0
    assert out[14] == 0.0 and out[13] == st[MA] + st[MAC]


def test_partly_evaporated_cloud_returns_its_share_of_aerosol():
    """Cloud that the adjustment evaporates in part (subsaturated air, more
    cloud water than the deficit) returns the evaporated share of its aerosol
    to the free aerosol and keeps its aerosol per unit water."""
    T, p = 285.0, 9.0e4
    qs = O.qsat(O.es_liq(T), p)
    for frac in (0.96, 0.99):
        st = np.zeros(19)
        st[F["T"]], st[F["p"]], st[F["rho"]] = T, p, p / (287.04 * T)
        st[F["qv"]], st[F["qc"]], st[F["nc"]], st[F["na"]] = frac * qs, 1e-3, 1e8, 1e8
        st[MA], st[MAC] = 2e-9, 3e-9
        out = O.point_aero(st, 1.0)
        assert 0.0 < out[F["qc"]] < 0.98 * st[F["qc"]]
        assert np.isclose(out[14] / out[F["qc"]], st[MAC] / st[F["qc"]], rtol=1e-9, atol=0.0)
        assert np.isclose(out[13] - st[MA], st[MAC] - out[14] - out[15], rtol=1e-12, atol=0.0)
        assert out[13] > st[MA]


# ------------------------------------------------ cold configuration (aerosol in ice too)
MAI, MAS, MAG = 19, 20, 21
QX = {MAR: F["qr"], MAI: F["qi"], MAS: F["qs"], MAG: F["qg"], MAC: F["qc"]}


def _aero_cold_state(ncols, nlev, seed):
    dz = synth.dz_stretched(nlev)
    base = synth.make_state("deep_convective", ncols, nlev, dz, seed=seed)
    fld = np.zeros((22,) + base.shape[1:])
    fld[:16] = base
    rng = np.random.default_rng(seed)
    fld[MA] = rng.uniform(1e-9, 5e-9, base.shape[1:])
    for f, q in QX.items():
        fld[f] = base[q] * rng.uniform(1e-5, 1e-4, base.shape[1:])
    return np.ascontiguousarray(fld), dz


def _cold_point(T, p, **kw):
    st = np.zeros(22)
    st[F["T"]], st[F["p"]], st[F["rho"]] = T, p, p / (287.04 * T)
    names = {"ma": MA, "mac": MAC, "mar": MAR, "mai": MAI, "mas": MAS, "mag": MAG}
    for k, v in kw.items():
        st[names[k] if k in names else F[k]] = v
    return st


def test_cold_standard_fields_are_the_cold_steps():
    fld, dz = _aero_cold_state(48, 150, seed=11)
    a = fld.copy()
    pa, ea = O.step_aero_cold(a, 48, dz, 1.0)
    b = np.ascontiguousarray(fld[:16].copy())
    pb, _, eb = O.step(b, 48, dz, 1.0)
    assert ea == 0 and eb == 0
    assert np.array_equal(a[:16], b) and np.array_equal(pa[:4], pb)
    for f in (MAI, MAS, MAG):
        assert not np.array_equal(a[f], fld[f])


def test_cold_total_aerosol_is_conserved():
    fld, dz = _aero_cold_state(40, 150, seed=12)
    out = fld.copy()
    pr, err = O.step_aero_cold(out, 40, dz, 1.0)
    assert err == 0
    w = fld[F["rho"], :, :40] * dz[:, None]
    m0 = (fld[MA:MAG + 1, :, :40] * w).sum(axis=(0, 1))
    m1 = (out[MA:MAG + 1, :, :40] * w).sum(axis=(0, 1))
    assert np.allclose(m1 + pr[4, :40], m0, rtol=1e-12, atol=0)
    assert pr[4, :40].max() > 0.0
    assert (out[MA:MAG + 1, :, :40] >= 0).all()


def test_cold_equals_warm_on_an_ice_free_warm_state():
    fld, dz, ncols, nlev, dt, _ = synth.workload("stratus_16x16x50")
    top = int(np.argmax(fld[F["T"], :, :ncols].min(axis=1) < O.param("T_nuc") + 1.0))
    sub = np.ascontiguousarray(fld[:, :top, :])
    for q in ("qi", "qs", "qg", "ni", "ns", "ng"):
        sub[F[q]] = 0.0
    rng = np.random.default_rng(13)
    warm = np.zeros((19,) + sub.shape[1:])
    warm[:16] = sub
    warm[MA] = rng.uniform(1e-9, 5e-9, sub.shape[1:])
    warm[MAC] = sub[F["qc"]] * 3e-5
    warm[MAR] = sub[F["qr"]] * 5e-5
    cold = np.zeros((22,) + sub.shape[1:])
    cold[:19] = warm
    warm, cold = np.ascontiguousarray(warm), np.ascontiguousarray(cold)
    dzs = np.ascontiguousarray(dz[:top])
    pw, ew = O.step_aero(warm, ncols, dzs, dt)
    pc, ec = O.step_aero_cold(cold, ncols, dzs, dt)
    assert ew == 0 and ec == 0
    assert np.array_equal(warm, cold[:19]) and np.array_equal(pw, pc)
    assert np.all(cold[MAI:] == 0.0)


def test_melting_gives_rain_the_melted_share_of_snow_aerosol():
    T, p = 276.0, 9.0e4
    qsl = O.qsat(O.es_liq(T), p)
    qs0, mas0 = 2e-4, 3e-9
    st = _cold_point(T, p, qv=0.9 * qsl, qs=qs0, ns=5e3, na=1e8, mas=mas0)
    out = O.point_aero_cold(st, 5.0)
    qs1 = out[F["qs"]]
    assert 0.0 < qs1 < qs0 and out[F["qr"]] > 0.0
    assert np.isclose(out[13 + 4], mas0 * qs1 / qs0, rtol=1e-12, atol=0.0)           # snow keeps its share
    assert np.isclose(out[13 + 2], mas0 * (1 - qs1 / qs0), rtol=1e-12, atol=0.0)     # the rest is in rain


def test_sublimation_returns_the_sublimated_share_of_ice_aerosol():
    T, p = 260.0, 6.0e4
    qsi = O.qsat(O.es_ice(T), p)
    qi0, mai0, ma0 = 5e-5, 2e-9, 1e-9
    st = _cold_point(T, p, qv=0.8 * qsi, qi=qi0, ni=1e5, na=1e8, mai=mai0, ma=ma0)
    out = O.point_aero_cold(st, 5.0)
    qi1 = out[F["qi"]]
    assert 0.0 < qi1 < qi0
    assert np.isclose(out[13 + 3], mai0 * qi1 / qi0, rtol=1e-12, atol=0.0)
    assert np.isclose(out[13 + 0], ma0 + mai0 * (1 - qi1 / qi0), rtol=1e-12, atol=0.0)


def test_collected_cloud_takes_its_share_of_cloud_aerosol_to_rain_and_graupel():
    """Cloud water collected at once by rain (accretion) and by graupel
    (riming), in air saturated over water with no updraft (no adjustment, no
    activation): the cloud keeps its aerosol per unit water, the rain gains
    the accreted share and the graupel the rimed share, each in proportion to
    the water it took, and the total is conserved."""
    T, p = 263.0, 7.0e4
    qsl = O.qsat(O.es_liq(T), p)
    qc0, mac0, mar0, mag0 = 5e-4, 4e-9, 1e-9, 2e-9
    st = _cold_point(T, p, qv=qsl, qc=qc0, nc=1e8, qr=2e-4, nr=1e3, qg=1e-3, ng=1e3,
                     na=1e8, ma=1e-9, mac=mac0, mar=mar0, mag=mag0)
    R = O.rates(st[:16], 2.0)
    assert R["acc"] > 0.0 and R["rimg"] > 0.0
    out = O.point_aero_cold(st, 2.0)
    qc1 = out[F["qc"]]
    assert 0.0 < qc1 < qc0
    assert np.isclose(out[13 + 1] / qc1, mac0 / qc0, rtol=1e-9, atol=0.0)
    to_rain, to_graupel = out[13 + 2] - mar0, out[13 + 5] - mag0
    assert to_rain > 0.0 and to_graupel > 0.0
    assert np.isclose(to_rain + to_graupel, mac0 * (1.0 - qc1 / qc0), rtol=1e-9, atol=0.0)
    assert np.isclose(to_graupel / to_rain, R["rimg"] / (R["aut"] + R["acc"]), rtol=1e-9, atol=0.0)
    assert np.isclose(out[13:19].sum(), st[16:22].sum(), rtol=1e-14, atol=0.0)


def test_cold_partly_evaporated_cloud_returns_its_share_of_aerosol():
    """The cold configuration's aerosol bookkeeping on the same partial
    evaporation (warm air, no ice): the cloud keeps its aerosol per unit
    water and the free aerosol gains the rest."""
    T, p = 285.0, 9.0e4
    qsl = O.qsat(O.es_liq(T), p)
    for frac in (0.96, 0.99):
        st = _cold_point(T, p, qv=frac * qsl, qc=1e-3, nc=1e8, na=1e8, ma=2e-9, mac=3e-9)
        out = O.point_aero_cold(st, 1.0)
        qc1 = out[F["qc"]]
        assert 0.0 < qc1 < 0.98 * st[F["qc"]]
        assert np.isclose(out[13 + 1] / qc1, st[MAC] / st[F["qc"]], rtol=1e-9, atol=0.0)
        assert np.isclose(out[13:19].sum(), st[16:22].sum(), rtol=1e-14, atol=0.0)
        assert out[13 + 0] > st[MA]


def test_each_species_aerosol_falls_with_its_mass():
    """A cold column exactly at ice saturation, without cloud or rain: the
    ice species only sediment (no deposition, nucleation, riming or
    melting), so aerosol held in fixed proportion to each species' mass
    keeps that proportion (it falls with the mass-weighted speed), and the
    column's aerosol loss is the deposited row."""
    ncols, nlev = 8, 40
    dz = np.full(nlev, 100.0)
    fld = np.zeros((22, nlev, 32))
    rng = np.random.default_rng(15)
    for k in range(nlev):
        T, p = 250.0 - 0.2 * k, 7.0e4 - 800.0 * k
        fld[F["T"], k, :ncols], fld[F["p"], k, :ncols], fld[F["rho"], k, :ncols] = T, p, p / (287.04 * T)
        fld[F["qv"], k, :ncols] = O.qsat(O.es_ice(T), p)
    for q, n, med in (("qi", "ni", 2e-5), ("qs", "ns", 1e-4), ("qg", "ng", 5e-4)):
        lev = slice(10, 30)
        fld[F[q], lev, :ncols] = med * rng.lognormal(0.0, 0.5, (20, ncols))
        fld[F[n], lev, :ncols] = fld[F[q], lev, :ncols] / (med / 1e3)
    fld[F["na"], :, :ncols] = 1e8
    for f, q in ((MAI, "qi"), (MAS, "qs"), (MAG, "qg")):
        fld[f] = 2e-5 * fld[F[q]]
    fld = np.ascontiguousarray(fld)
    out = fld.copy()
    pr, err = O.step_aero_cold(out, ncols, dz, 10.0)
    assert err == 0
    for f, q in ((MAI, "qi"), (MAS, "qs"), (MAG, "qg")):
        qq = out[F[q], :, :ncols]
        assert not np.array_equal(qq, fld[F[q], :, :ncols]), q
        assert np.allclose(out[f, :, :ncols], 2e-5 * qq, rtol=1e-10, atol=0), q
    w = fld[F["rho"], :, :ncols] * dz[:, None]
    total = (fld[MAI:MAG + 1, :, :ncols] * w).sum(axis=(0, 1))
    lost = ((fld[MAI:MAG + 1] - out[MAI:MAG + 1])[:, :, :ncols] * w).sum(axis=(0, 1))
    assert (np.abs(lost - pr[4, :ncols]) <= 1e-12 * total).all()
