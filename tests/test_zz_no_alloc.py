"""casim_step_noalloc: the step for callers that cannot allocate device memory.

It must give what the context-based casim_step gives, call after call, using
only the library's fixed scratch array.  Two calls in a row are checked, for
both precision forms, against two casim_step calls on an identical copy.
"""
import numpy as np
import pytest

from paper_2010_14823_gb300 import casim, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ATOL = np.array([1e-10] + [1e-20] * 6 + [1e-6] * 6)


def _close(a, b, ncols):
    for f in range(13):
        err = np.abs(a[f, :, :ncols] - b[f, :, :ncols])
        assert (err <= 1e-12 * np.abs(b[f, :, :ncols]) + ATOL[f]).all(), synth.FIELDS[f]


@pytest.mark.parametrize("precision", [casim.CASIM_FP64, casim.CASIM_MIXED])
def test_noalloc_matches_step_on_two_calls(precision):
    nlev, ncols = 150, 300
    dz = synth.dz_stretched(nlev)
    fld = synth.make_state("deep_convective", ncols, nlev, dz, seed=31)
    ref = casim.Domain(fld, dz, ncols)
    ctx = casim.casim_init(precision=precision)
    try:
        for _ in range(2):
            casim.casim_step(ctx, ref.state, ncols, nlev, 1.0)
        assert casim.casim_get_error(ctx)[0] == 0
    finally:
        casim.casim_free(ctx)
    got = casim.Domain(fld, dz, ncols)
    for _ in range(2):
        rc, flags = casim.casim_step_noalloc(None, precision, got.state, ncols, nlev, 1.0)
        assert rc == 0 and flags == 0
    (a, pa), (b, pb) = got.numpy(), ref.numpy()
    _close(a, b, ncols)
    assert np.allclose(pa, pb, rtol=1e-12, atol=1e-20)


def test_noalloc_rejects_more_columns_than_its_scratch():
    n = casim.NOALLOC_MAX_COLS + 32
    # rejected on the host before any device work: the pointers are never used
    st = casim.casim_state(256, n, 256, 256)
    with pytest.raises(casim.CasimError):
        casim.casim_step_noalloc(None, casim.CASIM_MIXED, st, n, 10, 1.0)
    assert b"scratch" in casim.lib().casim_last_cuda_error()
