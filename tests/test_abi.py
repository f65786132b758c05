"""The C-ABI library builds, loads and exports every declared entry point (no GPU needed)."""
import ctypes
import os

import pytest

from paper_2010_14823_gb300 import build, casim

import oracle as O


@pytest.fixture(scope="module")
def L():
    build.build()
    return casim.lib()


def test_every_declared_symbol_is_exported(L):
    names = casim.declared_functions("casim.h")
    assert len(names) >= 10
    for n in names:
        assert hasattr(L, n), n
    # the index-checked build exports the same entry points
    D = ctypes.CDLL(build.LIB_DEBUG)
    for n in names:
        assert hasattr(D, n), n
    from paper_2010_14823_gb300 import peaks
    pn = casim.declared_functions("casim_peaks.h")
    assert pn == ["casim_peak_rate"]
    for n in pn:
        assert hasattr(peaks.lib(), n), n
    headers = sorted(f for f in os.listdir(casim.INCLUDE) if f.endswith(".h"))
    assert headers == ["casim.h", "casim_peaks.h"]


def test_peak_probe_argument_errors(L):
    from paper_2010_14823_gb300 import peaks
    r = ctypes.c_double(0.0)
    assert peaks.lib().casim_peak_rate(99, 10, None, ctypes.byref(r)) == -1
    assert peaks.lib().casim_peak_rate(0, 0, None, ctypes.byref(r)) == -1
    assert peaks.lib().casim_peak_rate(0, 10, None, None) == -1


def test_abi_version(L):
    assert casim.casim_abi_version() == 1


def test_default_params_match_the_oracle(L):
    p = casim.casim_default_params().as_dict()
    for k, v in p.items():
        if isinstance(v, list):
            for s, x in zip("crisg", v):
                assert x == O.param(f"{k}_{s}"), (k, s)
        else:
            assert v == O.param(k), k


def test_argument_errors_without_touching_the_device(L):
    ctx = ctypes.c_void_p()
    assert L.casim_init(ctypes.byref(ctx), None, 7, 0) == -1          # bad precision
    assert L.casim_init(ctypes.byref(ctx), None, 0, 16) == -1         # unknown flag
    assert L.casim_init(ctypes.byref(ctx), None, 0, 8 | 1) == -1      # statistics need the standard configuration
    assert L.casim_init(ctypes.byref(ctx), None, 0, 2 | 4) == -1      # aerosol mass with triple moment
    assert not ctx.value
    st = casim.casim_state(None, 32, None, None)
    assert L.casim_step(None, ctypes.byref(st), 1, 1, 1.0, None) == -1
    assert L.casim_get_error(None, None, None) == -1
    assert L.casim_launch_count(None) == -1
    el = ctypes.c_longlong(0)
    assert L.casim_wait_selftest(None, 1000, ctypes.byref(el), None) == -1
    L.casim_free(None)
    bad = casim.casim_default_params()
    bad.q_min = -1.0
    assert L.casim_init(ctypes.byref(ctx), ctypes.byref(bad), 0, 0) == -1
    assert L.casim_default_params(None) == -1


def test_a_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the built library the binding raises at first use, naming the
    missing file; there is no fallback path."""
    from paper_2010_14823_gb300 import casim
    monkeypatch.setattr(casim, "_lib", None)
    monkeypatch.setattr(casim, "LIB", str(tmp_path / "libcasim.so"))
    monkeypatch.delenv("CASIM_LIBRARY", raising=False)
    with pytest.raises(RuntimeError, match="libcasim.so is missing"):
        casim.lib()
    with pytest.raises(RuntimeError, match="is missing"):
        casim.casim_init()
