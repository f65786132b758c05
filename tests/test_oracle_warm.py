"""Pins of the oracle's warm configuration (liquid water only; ice fields
treated as absent and passed through unchanged).

The warm chain is the cold chain restricted to liquid water, so: on a state
without ice, and warm enough that no ice can nucleate, both configurations
give the same result bit for bit; with ice present the warm step leaves every
ice field untouched and sediments rain only; where the cold chain would
nucleate ice the warm one does nothing; water in vapour, cloud, rain and
rain precipitation is conserved.
"""
import numpy as np

import oracle as O
from paper_2010_14823_gb300 import synth

F = synth.FIDX
ICE = [F[x] for x in ("qi", "qs", "qg", "ni", "ns", "ng")]
TNUC = O.param("T_nuc")


def _ice_free_warm_state():
    fld, dz, ncols, nlev, dt, _ = synth.workload("stratus_16x16x50")
    # keep the levels where every column is warmer than the nucleation threshold
    top = int(np.argmax(fld[F["T"], :, :ncols].min(axis=1) < TNUC + 1.0))
    assert 10 < top < nlev
    sub = np.ascontiguousarray(fld[:, :top, :])
    sub[ICE] = 0.0
    return sub, np.ascontiguousarray(dz[:top]), ncols, dt


def test_warm_equals_cold_without_ice():
    fld, dz, ncols, dt = _ice_free_warm_state()
    assert (fld[F["qc"]] > 0).any() and (fld[F["qr"]] > 0).any()
    cold, warm = fld.copy(), fld.copy()
    pc, nc_, ec = O.step(cold, ncols, dz, dt, want_nsub=True)
    pw, nw, ew = O.step(warm, ncols, dz, dt, want_nsub=True, warm=True)
    assert ec == 0 and ew == 0
    assert not np.array_equal(cold, fld)          # the step did something
    assert np.array_equal(cold, warm)
    assert np.array_equal(pc, pw)
    assert np.array_equal(nc_[0], nw[0])


def test_warm_leaves_ice_untouched_and_sediments_rain_only():
    nlev = 150
    dz = synth.dz_stretched(nlev)
    fld = synth.make_state("deep_convective", 24, nlev, dz, seed=5)
    assert (fld[F["qi"]] > 0).any() and (fld[F["qg"]] > 0).any()
    out = fld.copy()
    pr, ns, err = O.step(out, 24, dz, 1.0, want_nsub=True, warm=True)
    assert err == 0
    for f in ICE:
        assert np.array_equal(out[f], fld[f])
    assert np.all(pr[1:] == 0.0) and np.all(ns[1:, :24] == 1)
    assert pr[0, :24].max() > 0.0
    # the liquid species did change
    assert not np.array_equal(out[F["qr"]], fld[F["qr"]])


def test_warm_does_not_nucleate_where_cold_does():
    st = np.zeros(O.NFIELDS)
    T, p = 250.0, 5.0e4
    qsi = O.qsat(O.es_ice(T), p)
    qsl = O.qsat(O.es_liq(T), p)
    st[F["T"]], st[F["p"]], st[F["rho"]] = T, p, p / (287.04 * T)
    st[F["qv"]] = 0.5 * (qsi + qsl)               # supersaturated over ice only
    st[F["na"]] = 1e8
    cold = O.point(st, 1.0)
    warm = O.point(st, 1.0, warm=True)
    assert cold[F["ni"]] > 0.0 and cold[F["qi"]] > 0.0
    assert np.array_equal(warm, st[:O.NPROG])
    rc, rw = O.rates(st, 1.0), O.rates(st, 1.0, warm=True)
    assert rc["nuc"] > 0.0 and all(v == 0.0 for v in rw.values())


def test_warm_rates_are_the_cold_chains_liquid_rates():
    nlev = 150
    dz = synth.dz_stretched(nlev)
    fld = synth.make_state("deep_convective", 64, nlev, dz, seed=6)
    n = 0
    for c in range(64):
        for k in range(0, nlev, 3):
            st = fld[:, k, c].copy()
            if not (st[F["qc"]] > 1e-14 or st[F["qr"]] > 1e-14):
                continue
            rc = O.rates(st, 1.0)
            st_w = st.copy()
            st_w[ICE] = 0.0
            rw = O.rates(st_w, 1.0, warm=True)
            for name in ("aut", "acc", "scc", "scr", "evr"):
                assert rw[name] == rc[name]
            for name in ("nuc", "depi", "deps", "depg", "rims", "rimg", "mlti", "mlts", "mltg"):
                assert rw[name] == 0.0
            n += 1
    assert n > 100


def test_warm_column_water_budget():
    nlev = 150
    dz = synth.dz_stretched(nlev)
    fld = synth.make_state("deep_convective", 32, nlev, dz, seed=7)
    out = fld.copy()
    pr, _, err = O.step(out, 32, dz, 1.0, warm=True)
    assert err == 0
    rho = fld[F["rho"], :, :32]
    liq = ("qv", "qc", "qr")
    w0 = sum((fld[F[x], :, :32] * rho * dz[:, None]).sum(0) for x in liq)
    w1 = sum((out[F[x], :, :32] * rho * dz[:, None]).sum(0) for x in liq)
    assert np.allclose(w1 + pr[0, :32], w0, rtol=1e-12, atol=0)
