"""The index-checked build and the per-step statistics, through the C ABI.

Debug build (libcasim_debug.so, compiled with CASIM_DEBUG): on valid inputs
it must give bit for bit what the normal library gives, and leave the error
word clear (no index check fails).  No kernel is given an invalid index on
purpose: invalid sizes are refused on the host before any launch.

Statistics (CASIM_STATS): the counts are checked where they are known
exactly (cloud planted at chosen points of dry subsaturated air: those points
and only those are active, and each changes), the substep histogram against
the oracle's substep counts, and the step's results are those of a context
without statistics, bit for bit.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_2010_14823_gb300 import build, casim, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F = synth.FIDX


@pytest.fixture(scope="module")
def D():
    build.build()
    return casim.bind(ctypes.CDLL(build.LIB_DEBUG))


def _run(L, fld, dz, ncols, dt, precision, nsteps=1, flags=0):
    ctx = ctypes.c_void_p()
    assert L.casim_init(ctypes.byref(ctx), None, precision, flags) == 0
    try:
        d = casim.Domain(fld, dz, ncols)
        for _ in range(nsteps):
            assert L.casim_step(ctx, ctypes.byref(d.state), ncols, d.nlev, dt, None) == 0
        f = ctypes.c_uint(0)
        rc = L.casim_get_error(ctx, ctypes.byref(f), None)
        return d.numpy(), rc, f.value
    finally:
        L.casim_free(ctx)


@pytest.mark.parametrize("dt", [1.0, 30.0])
@pytest.mark.parametrize("precision", [casim.CASIM_FP64, casim.CASIM_MIXED])
def test_debug_build_equals_normal_build(D, precision, dt):
    ncols, nlev = 300, 150
    dz = synth.dz_stretched(nlev)
    fld = synth.make_state("deep_convective", ncols, nlev, dz, seed=81)
    (a, pa), rc_a, fl_a = _run(casim.lib(), fld, dz, ncols, dt, precision, nsteps=2)
    (b, pb), rc_b, fl_b = _run(D, fld, dz, ncols, dt, precision, nsteps=2)
    assert rc_a == 0 and fl_a == 0
    assert rc_b == 0 and fl_b == 0, (rc_b, fl_b)      # no index check failed
    assert np.array_equal(a, b) and np.array_equal(pa, pb)


def test_debug_build_batched_and_allocation_free_steps(D):
    """The batched launch (active-column list, persistent grid) and the
    allocation-free step of the debug build: equal to the normal build's
    per-domain steps, error word clear."""
    doms = []
    for i, (nc, nl) in enumerate([(333, 150), (97, 60), (1000, 40)]):
        dz = synth.dz_stretched(nl)
        doms.append((synth.make_state("deep_convective", nc, nl, dz, seed=90 + i), dz, nc, nl))
    ref = [_run(casim.lib(), f, dz, nc, 1.0, casim.CASIM_MIXED)[0] for f, dz, nc, nl in doms]
    ctx = ctypes.c_void_p()
    assert D.casim_init(ctypes.byref(ctx), None, casim.CASIM_MIXED, 0) == 0
    try:
        dev = [casim.Domain(f, dz, nc) for f, dz, nc, nl in doms]
        n = len(dev)
        arr = (casim.casim_state * n)(*[d.state for d in dev])
        nc = (ctypes.c_int * n)(*[d.ncols for d in dev])
        nl = (ctypes.c_int * n)(*[d.nlev for d in dev])
        assert D.casim_step_batched(ctx, arr, nc, nl, n, 1.0, None) == 0
        f = ctypes.c_uint(0)
        assert D.casim_get_error(ctx, ctypes.byref(f), None) == 0 and f.value == 0
        for d, (ra, rpa) in zip(dev, ref):
            a, pa = d.numpy()
            assert np.array_equal(a, ra) and np.array_equal(pa, rpa)
    finally:
        D.casim_free(ctx)
    f0, dz0, nc0, nl0 = doms[0]
    d = casim.Domain(f0, dz0, nc0)
    fl = ctypes.c_uint(0)
    assert D.casim_step_noalloc(None, casim.CASIM_MIXED, ctypes.byref(d.state), nc0, nl0, 1.0, None,
                                ctypes.byref(fl)) == 0 and fl.value == 0
    a, pa = d.numpy()
    assert np.array_equal(a, ref[0][0]) and np.array_equal(pa, ref[0][1])


def _dry_state(ncols, nlev, seed):
    """Warm (290 K), subsaturated (70 % RH), no hydrometeors, still air: no
    point is active; cloud is planted at chosen points."""
    rng = np.random.default_rng(seed)
    pitch = (ncols + 31) // 32 * 32
    fld = np.zeros((16, nlev, pitch))
    T, p, rho = 290.0, 9.0e4, 1.08
    es = O.es_liq(T)
    fld[F["T"]] = T
    fld[F["p"]] = p
    fld[F["rho"]] = rho
    fld[F["qv"]] = 0.7 * O.qsat(es, p)
    fld[F["na"]] = 1e8
    k = rng.integers(0, nlev, 37)
    c = rng.integers(0, ncols, 37)
    pts = sorted(set(zip(k.tolist(), c.tolist())))
    for kk, cc in pts:
        fld[F["qc"], kk, cc] = 2e-5
        fld[F["nc"], kk, cc] = 5e7
    return fld, pts


@pytest.mark.parametrize("precision", [casim.CASIM_FP64, casim.CASIM_MIXED])
def test_stats_count_planted_cloud_exactly(precision):
    ncols, nlev = 200, 60
    dz = np.full(nlev, 50.0)
    fld, pts = _dry_state(ncols, nlev, seed=7)
    ctx = casim.casim_init(precision=precision, flags=casim.CASIM_STATS)
    try:
        d = casim.Domain(fld, dz, ncols)
        casim.casim_step(ctx, d.state, ncols, nlev, 1.0)
        st = casim.casim_get_stats(ctx, reset=True)
        assert casim.casim_get_error(ctx)[0] == 0
        out = d.numpy()[0]
        changed = int((out[:13, :, :ncols] != fld[:13, :, :ncols]).any(axis=0).sum())
        assert st["steps"] == 1 and st["points"] == ncols * nlev
        assert st["active_points"] == len(pts)
        assert st["changed_points"] == len(pts) == changed
        assert st["active_columns"] == len({c for _, c in pts})
        # single-substep path: every column's every species took one substep
        assert np.array_equal(st["nsub"][:, 1], np.full(4, ncols)) and st["nsub"].sum() == 4 * ncols
        # the reset took effect
        z = casim.casim_get_stats(ctx)
        assert z["steps"] == 0 and z["active_points"] == 0 and z["nsub"].sum() == 0
    finally:
        casim.casim_free(ctx)


def test_stats_host_step_on_pinned_state():
    """A statistics context's host step on pinned host state (stepped in
    place by the statistics kernel over the host link): the planted cloud
    counted exactly, one step of every point, results equal to the device
    step's bit for bit."""
    import torch
    ncols, nlev = 200, 60
    dz = np.full(nlev, 50.0)
    fld, pts = _dry_state(ncols, nlev, seed=9)
    ctx = casim.casim_init(precision=casim.CASIM_MIXED, flags=casim.CASIM_STATS)
    try:
        d = casim.Domain(fld, dz, ncols)
        casim.casim_step(ctx, d.state, ncols, nlev, 1.0)
        out, pr = d.numpy()
        casim.casim_get_stats(ctx, reset=True)
        th = torch.from_numpy(fld.copy()).pin_memory()
        tpr = torch.zeros((4, fld.shape[2]), dtype=torch.float64).pin_memory()
        h, hpr = th.numpy(), tpr.numpy()
        casim.casim_step_host(ctx, casim.make_state(h, fld.shape[2], np.ascontiguousarray(dz), hpr), ncols, nlev, 1.0)
        st = casim.casim_get_stats(ctx)
        assert casim.casim_get_error(ctx)[0] == 0
        assert np.array_equal(h, out) and np.array_equal(hpr, pr)
        assert st["steps"] == 1 and st["points"] == ncols * nlev
        assert st["active_points"] == len(pts) and st["changed_points"] == len(pts)
    finally:
        casim.casim_free(ctx)


@pytest.mark.parametrize("dt", [1.0, 30.0])
def test_stats_substep_histogram_matches_oracle_and_results_unchanged(dt):
    """FP64 form on a deep-convective state; dt = 30 s takes the multi-substep
    path: per species, the histogram of the columns' substep counts equals the
    oracle's; the changed points are those whose state differs (no fewer);
    the results equal those of a context without statistics, bit for bit."""
    ncols, nlev = 160, 100
    dz = synth.dz_stretched(nlev)
    fld = synth.make_state("deep_convective", ncols, nlev, dz, seed=int(dt) + 5)
    ctx = casim.casim_init(precision=casim.CASIM_FP64, flags=casim.CASIM_STATS)
    try:
        d = casim.Domain(fld, dz, ncols)
        casim.casim_step(ctx, d.state, ncols, nlev, dt)
        st = casim.casim_get_stats(ctx)
        assert casim.casim_get_error(ctx)[0] == 0
        out, pr = d.numpy()
    finally:
        casim.casim_free(ctx)
    ref = fld.copy()
    _, nsub, err = O.step(ref, ncols, dz, dt, want_nsub=True)
    assert err == 0
    for x in range(4):
        hist = np.bincount(nsub[x, :ncols], minlength=65)[:65]
        assert np.array_equal(st["nsub"][x], hist), (x, np.nonzero(st["nsub"][x])[0], np.nonzero(hist)[0])
    if dt == 30.0:
        assert st["nsub"][:, 2:].sum() > 0          # some columns took several substeps
    differ = int((out[:13, :, :ncols] != fld[:13, :, :ncols]).any(axis=0).sum())
    assert differ <= st["changed_points"] <= ncols * nlev
    assert st["active_points"] > 0 and st["active_columns"] <= ncols
    # the same step without statistics
    plain = casim.casim_init(precision=casim.CASIM_FP64)
    try:
        d2 = casim.Domain(fld, dz, ncols)
        casim.casim_step(plain, d2.state, ncols, nlev, dt)
        b, pb = d2.numpy()
    finally:
        casim.casim_free(plain)
    assert np.array_equal(out, b) and np.array_equal(pr, pb)


def test_stats_needs_the_standard_configuration():
    for flags in (casim.CASIM_WARM, casim.CASIM_AEROSOL, casim.CASIM_THREE_MOMENT):
        with pytest.raises(casim.CasimError):
            casim.casim_init(precision=casim.CASIM_MIXED, flags=flags | casim.CASIM_STATS)
    ctx = casim.casim_init(precision=casim.CASIM_MIXED)
    try:
        with pytest.raises(casim.CasimError):
            casim.casim_get_stats(ctx)
    finally:
        casim.casim_free(ctx)
