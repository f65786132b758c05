"""Batched step (many uneven domains per launch): bitwise equal to per-domain
steps for every launch configuration, with and without the active-column
list, replayed from a CUDA graph, after autotuning; FP64 form against the
oracle on sampled columns."""
import numpy as np
import pytest

import oracle as O
from paper_2010_14823_gb300 import casim, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def domains(seed=5):
    """Uneven domains: ragged column counts, 1..150 levels, cloudy, clear, empty."""
    specs = [("deep_convective", 333, 150), ("stratus_broken", 1000, 60), ("stratus", 64, 17),
             (synth.Recipe(cloud_frac=0.0, T_sfc=300.0, rh_clear=(0.5, 0.8)), 200, 40),
             ("stratus_broken", 97, 1), ("deep_convective", 0, 30), ("stratus", 2500, 50)]
    out = []
    for i, (rc, nc, nl) in enumerate(specs):
        dz = synth.dz_stretched(nl) if nl > 1 else np.array([50.0])
        out.append((synth.make_state(rc, nc, nl, dz, seed=seed + i), dz, nc, nl))
    return out


def to_device(doms):
    return [casim.Domain(f, dz, nc) for f, dz, nc, nl in doms]


def reference(doms, precision, nsteps, dt=1.0):
    """Each domain stepped on its own with casim_step."""
    dev = to_device(doms)
    ctx = casim.casim_init(precision=precision)
    try:
        for _ in range(nsteps):
            for d in dev:
                casim.casim_step(ctx, d.state, d.ncols, d.nlev, dt)
        assert casim.casim_get_error(ctx)[0] == 0
        return [d.numpy() for d in dev]
    finally:
        casim.casim_free(ctx)


def run_batch(doms, precision, nsteps, config=None, graph=None, tune=False, dt=1.0):
    dev = to_device(doms)
    ctx = casim.casim_init(precision=precision)
    try:
        b = casim.casim_batch_create(ctx, [d.state for d in dev], [d.ncols for d in dev], [d.nlev for d in dev])
        try:
            done = 0
            if tune:
                table = casim.casim_batch_tune(ctx, b, dt, steps=1)
                assert all(t["ms_per_step"] > 0 for t in table)
                done += casim.casim_batch_tune_steps(1)
            if config:
                casim.casim_batch_config(b, *config)
            if graph:
                casim.casim_batch_graph(ctx, b, dt, graph)
                while done + graph <= nsteps:
                    casim.casim_batch_graph_launch(b)
                    done += graph
            while done < nsteps:
                casim.casim_batch_step(ctx, b, dt)
                done += 1
            assert casim.casim_get_error(ctx)[0] == 0
            cfg = casim.casim_batch_get_config(b)
        finally:
            casim.casim_batch_free(b)
        return [d.numpy() for d in dev], cfg
    finally:
        casim.casim_free(ctx)


def same(a, b):
    for (fa, pa), (fb, pb) in zip(a, b):
        assert np.array_equal(fa, fb) and np.array_equal(pa, pb)


@pytest.mark.parametrize("precision", [casim.CASIM_MIXED, casim.CASIM_FP64])
@pytest.mark.parametrize("config", [(64, 0, 0), (128, 1, 1), (256, 1, 0), (256, 0, 1)])
def test_batch_equals_per_domain_steps(precision, config):
    doms = domains()
    ref = reference(doms, precision, 2)
    got, cfg = run_batch(doms, precision, 2, config=config)
    assert cfg == config
    same(got, ref)


def test_graph_replay_equals_eager():
    doms = domains(seed=9)
    ref = reference(doms, casim.CASIM_MIXED, 6)
    got, _ = run_batch(doms, casim.CASIM_MIXED, 6, config=(128, 1, 1), graph=3)
    same(got, ref)


def test_autotuned_run_equals_eager():
    doms = domains(seed=13)
    n = casim.casim_batch_tune_steps(1) + 2
    ref = reference(doms, casim.CASIM_MIXED, n)
    got, cfg = run_batch(doms, casim.CASIM_MIXED, n, tune=True)
    assert cfg[0] in (64, 128, 256)
    same(got, ref)


def test_clear_domain_untouched_and_oracle_parity():
    doms = domains(seed=21)
    got, _ = run_batch(doms, casim.CASIM_FP64, 1, config=(128, 1, 1))
    f, dz, nc, nl = doms[3]             # cloud-free, dry domain: nothing to do
    assert np.array_equal(got[3][0], f)
    for (fo, po), (f, dz, nc, nl) in zip(got, doms):
        if nc == 0:
            continue
        cols = np.unique(np.linspace(0, nc - 1, min(nc, 24)).astype(int))
        sub = np.zeros((16, nl, 32))
        sub[:, :, :len(cols)] = f[:, :, cols]
        pr = np.zeros((4, 32))
        O.step(sub, len(cols), dz, 1.0, precip=pr)
        a, b = fo[:13, :, cols], sub[:13, :, :len(cols)]
        tol = 1e-12 * np.abs(b) + np.array([1e-10] + [1e-20] * 6 + [1e-6] * 6)[:, None, None]
        assert (np.abs(a - b) <= tol).all()


def test_batch_argument_errors():
    ctx = casim.casim_init()
    try:
        with pytest.raises(casim.CasimError):
            casim.casim_batch_create(ctx, [], [], [])
        d = casim.Domain(*domains()[2][:2], 64)
        with pytest.raises(casim.CasimError):
            casim.casim_batch_create(ctx, [d.state], [64], [5000])
        b = casim.casim_batch_create(ctx, [d.state], [64], [17])
        with pytest.raises(casim.CasimError):
            casim.casim_batch_config(b, 96, 1, 1)
        with pytest.raises(casim.CasimError):
            casim.casim_batch_graph_launch(b)          # nothing captured yet
        casim.casim_batch_free(b)
    finally:
        casim.casim_free(ctx)


@pytest.mark.parametrize("precision", [casim.CASIM_MIXED, casim.CASIM_FP64])
def test_step_batched_equals_batch_step_and_follows_the_domain_list(precision):
    """casim_step_batched (one call per step for a list of domains) gives, bit
    for bit, what casim_batch_step gives on a batch of the same domains; when
    the list changes (another subset, in another order) the context's batch
    is rebuilt and the result is again that of per-domain steps."""
    doms = domains(seed=29)
    ref, _ = run_batch(doms, precision, 3)
    dev = to_device(doms)
    ctx = casim.casim_init(precision=precision)
    try:
        st, nc, nl = [d.state for d in dev], [d.ncols for d in dev], [d.nlev for d in dev]
        for _ in range(3):
            casim.casim_step_batched(ctx, st, nc, nl, 1.0)
        assert casim.casim_get_error(ctx)[0] == 0
        same([d.numpy() for d in dev], ref)
        # another list: three of the domains, reversed, one step from fresh states
        pick = [6, 2, 0]
        sub = [doms[i] for i in pick]
        dev2 = to_device(sub)
        casim.casim_step_batched(ctx, [d.state for d in dev2], [d.ncols for d in dev2], [d.nlev for d in dev2], 1.0)
        assert casim.casim_get_error(ctx)[0] == 0
        same([d.numpy() for d in dev2], reference(sub, precision, 1))
    finally:
        casim.casim_free(ctx)


def test_step_batched_argument_errors():
    ctx = casim.casim_init()
    try:
        d = casim.Domain(*domains()[2][:2], 64)
        with pytest.raises(casim.CasimError):
            casim.casim_step_batched(ctx, [], [], [], 1.0)
        with pytest.raises(casim.CasimError):
            casim.casim_step_batched(ctx, [d.state], [64], [17], 0.0)
        with pytest.raises(casim.CasimError):
            casim.casim_step_batched(ctx, [d.state], [64], [5000], 1.0)
    finally:
        casim.casim_free(ctx)
    warm = casim.casim_init(flags=casim.CASIM_WARM)
    try:
        with pytest.raises(casim.CasimError):
            casim.casim_step_batched(warm, [d.state], [64], [17], 1.0)
    finally:
        casim.casim_free(warm)
