"""Pins of the oracle's activated-aerosol mass (warm configuration).

Aerosol mass moves with the water: it is an addition to the warm step, so the
16 standard fields are exactly the warm step's; it is conserved per column
(free + in cloud + in rain + deposited); without activation the aerosol per
unit water in cloud and in rain cannot change in subsaturated air, through
evaporation, autoconversion, accretion or sedimentation alike; activation
takes the free aerosol's mean particle mass; cloud that evaporates returns all
of its aerosol.
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
    assert np.isclose(out[14], st[MA] * dn / st[F["na"]], rtol=1e-9)
    assert np.isclose(out[13] + out[14] + out[15], st[MA], rtol=1e-15)


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
