"""casim_step_noalloc: the step for callers that cannot allocate device memory.

It must give what the context-based casim_step gives, bit for bit, call after
call, using only the library's fixed scratch array.  Two calls in a row are
checked, for both precision forms and for both sedimentation paths (dt = 1 s
takes the fused single-substep path, dt = 30 s the multi-substep path, which
this entry point chooses from the smallest layer thickness it finds on the
device), against two casim_step calls on an identical copy.  A smaller call
after a larger one shows that what the larger call left in the shared array
(tiles, list entries, the domain table) is not read.
"""
import numpy as np
import pytest

from paper_2010_14823_gb300 import casim, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _reference(fld, dz, ncols, nlev, dt, precision, nsteps):
    ref = casim.Domain(fld, dz, ncols)
    ctx = casim.casim_init(precision=precision)
    try:
        for _ in range(nsteps):
            casim.casim_step(ctx, ref.state, ncols, nlev, dt)
        assert casim.casim_get_error(ctx)[0] == 0
    finally:
        casim.casim_free(ctx)
    return ref.numpy()


def _noalloc(fld, dz, ncols, nlev, dt, precision, nsteps):
    got = casim.Domain(fld, dz, ncols)
    for _ in range(nsteps):
        rc, flags = casim.casim_step_noalloc(None, precision, got.state, ncols, nlev, dt)
        assert rc == 0 and flags == 0
    return got.numpy()


def _assert_same(got, ref):
    (a, pa), (b, pb) = got, ref
    for f in range(a.shape[0]):
        assert np.array_equal(a[f], b[f]), synth.FIELDS[f] if f < len(synth.FIELDS) else f
    assert np.array_equal(pa, pb)


@pytest.mark.parametrize("dt", [1.0, 30.0])
@pytest.mark.parametrize("precision", [casim.CASIM_FP64, casim.CASIM_MIXED])
def test_noalloc_matches_step_on_two_calls(precision, dt):
    nlev, ncols = 150, 300
    dz = synth.dz_stretched(nlev)
    fld = synth.make_state("deep_convective", ncols, nlev, dz, seed=31)
    ref = _reference(fld, dz, ncols, nlev, dt, precision, 2)
    got = _noalloc(fld, dz, ncols, nlev, dt, precision, 2)
    _assert_same(got, ref)
    # the step changed the state (the comparison is not of two copies of the input)
    assert not np.array_equal(got[0][:13], fld[:13])
    # a smaller domain next: fewer tiles, a shorter list and other levels
    n2, l2 = 70, 60
    dz2 = synth.dz_stretched(l2)
    fld2 = synth.make_state("deep_convective", n2, l2, dz2, seed=32)
    _assert_same(_noalloc(fld2, dz2, n2, l2, dt, precision, 1), _reference(fld2, dz2, n2, l2, dt, precision, 1))


def test_noalloc_rejects_more_columns_than_its_scratch():
    n = casim.NOALLOC_MAX_COLS + 32
    # rejected on the host before any device work: the pointers are never used
    st = casim.casim_state(256, n, 256, 256)
    with pytest.raises(casim.CasimError):
        casim.casim_step_noalloc(None, casim.CASIM_MIXED, st, n, 10, 1.0)
    assert b"scratch" in casim.lib().casim_last_cuda_error()
