"""GPU step vs the FP64 oracle, element by element, through the C ABI.

FP64 form: every prognostic field within 1e-12 relative of the oracle, with
absolute floors of 1e-20 kg/kg (masses), 1e-6 per kg (numbers), 1e-10 K (T),
after one step and after several (the discrepancy does not grow from step to
step: test_multistep_deep_convective_fp64 checks it after each one).
Mixed form: the bound derived from its FP32 arithmetic (see mixed_bound).
"""
import numpy as np
import pytest

import oracle as O
from paper_2010_14823_gb300 import casim, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F = synth.FIDX
RTOL64 = 1e-12


def needed_rtol(a, b, atol):
    """Smallest relative tolerance that a comparison with floor atol passes."""
    excess = np.maximum(np.abs(a - b) - atol, 0.0)
    nz = excess > 0
    return float((excess[nz] / np.abs(b[nz])).max()) if nz.any() else 0.0
ATOL = np.array([1e-10] + [1e-20] * 6 + [1e-6] * 6)   # T, 6 masses, 6 numbers (incl. n_a)
QMIN = casim.casim_default_params().q_min              # a species is present above this


def run_gpu(fld, dz, ncols, dt, nsteps=1, precision=casim.CASIM_FP64, check_err=True, flags=0):
    ctx = casim.casim_init(precision=precision, flags=flags)
    try:
        d = casim.Domain(fld, dz, ncols)
        for _ in range(nsteps):
            casim.casim_step(ctx, d.state, ncols, d.nlev, dt)
        rc, flags = casim.casim_get_error(ctx)
        if check_err:
            assert rc == 0, (rc, flags)
        out, pr = d.numpy()
        return out, pr, (rc, flags)
    finally:
        casim.casim_free(ctx)


def run_oracle(fld, dz, ncols, dt, nsteps=1, warm=False):
    ref = fld.copy()
    pr = np.zeros((4, fld.shape[2]))
    for _ in range(nsteps):
        _, _, err = O.step(ref, ncols, dz, dt, precip=pr, warm=warm)
        assert err == 0
    return ref, pr


def assert_fp64_close(out, pr, ref, pr_ref, ncols, rtol=RTOL64):
    need = max(needed_rtol(out[f, :, :ncols], ref[f, :, :ncols], ATOL[f]) for f in range(13))
    print(f"FP64 vs oracle: needed rtol {need:.3g} (allowed {rtol:.3g})")
    for f in range(13):
        a, b = out[f, :, :ncols], ref[f, :, :ncols]
        err = np.abs(a - b)
        bad = err > rtol * np.abs(b) + ATOL[f]
        assert not bad.any(), (synth.FIELDS[f], int(bad.sum()), float(err.max()),
                               np.argwhere(bad)[:3].tolist())
    e = np.abs(pr[:, :ncols] - pr_ref[:, :ncols])
    assert np.all(e <= rtol * np.abs(pr_ref[:, :ncols]) + 1e-20), float(e.max())
    # branch flips: presence decisions (q > q_min) taken differently by the
    # GPU and the oracle, per hydrometeor mass
    flips = {synth.FIELDS[f]: int(((out[f, :, :ncols] > QMIN) != (ref[f, :, :ncols] > QMIN)).sum())
             for f in range(2, 7)}
    print("presence-decision flips, GPU FP64 vs oracle:", flips)
    assert not any(flips.values()), flips


def test_stratus_16x16x50_fp64():
    fld, dz, ncols, nlev, dt, nsteps = synth.workload("stratus_16x16x50")
    out, pr, _ = run_gpu(fld, dz, ncols, dt)
    ref, pr_ref = run_oracle(fld, dz, ncols, dt)
    assert_fp64_close(out, pr, ref, pr_ref, ncols)
    # inputs untouched, padding untouched
    assert np.array_equal(out[13:], fld[13:])


@pytest.mark.parametrize("ncols,nlev", [(1, 50), (33, 17), (200, 1), (97, 150)])
def test_ragged_sizes_fp64(ncols, nlev):
    dz = synth.dz_stretched(nlev)
    fld = synth.make_state("deep_convective", ncols, nlev, dz, seed=100 + ncols)
    out, pr, _ = run_gpu(fld, dz, ncols, 1.0)
    ref, pr_ref = run_oracle(fld, dz, ncols, 1.0)
    assert_fp64_close(out, pr, ref, pr_ref, ncols)
    assert np.array_equal(out[:, :, ncols:], fld[:, :, ncols:])


def test_multistep_deep_convective_fp64():
    """Five steps, compared after each one: the GPU state stays within 1e-12
    of the oracle's after every step (the rounding differences of a step do
    not accumulate into the next beyond that bound)."""
    ncols, nlev = 256, 150
    dz = synth.dz_stretched(nlev)
    fld = synth.make_state("deep_convective", ncols, nlev, dz, seed=7)
    ctx = casim.casim_init(precision=casim.CASIM_FP64)
    try:
        d = casim.Domain(fld, dz, ncols)
        ref = fld.copy()
        pr_ref = np.zeros((4, fld.shape[2]))
        for k in range(1, 6):
            casim.casim_step(ctx, d.state, ncols, nlev, 1.0)
            _, _, err = O.step(ref, ncols, dz, 1.0, precip=pr_ref)
            assert err == 0
            assert casim.casim_get_error(ctx)[0] == 0
            out, pr = d.numpy()
            print(f"after step {k}:", end=" ")
            assert_fp64_close(out, pr, ref, pr_ref, ncols, rtol=RTOL64)
    finally:
        casim.casim_free(ctx)


@pytest.mark.parametrize("dt", [5.0, 30.0])
def test_substepped_sedimentation_fp64(dt):
    # dz down to 20 m with dt >= 5 s: capped speeds exceed one level per step,
    # so columns take the multi-substep path
    dz = synth.dz_stretched(100)
    fld = synth.make_state("deep_convective", 160, 100, dz, seed=int(dt))
    out, pr, _ = run_gpu(fld, dz, 160, dt)
    ref, pr_ref = run_oracle(fld, dz, 160, dt)
    assert_fp64_close(out, pr, ref, pr_ref, 160)


def test_stratus_256x256x100_sampled_columns_fp64():
    # full-size GPU run (10 steps); the oracle follows 32 sampled columns
    fld, dz, ncols, nlev, dt, nsteps = synth.workload("stratus_256x256x100")
    out, pr, _ = run_gpu(fld, dz, ncols, dt, nsteps=nsteps)
    cols = np.sort(np.random.default_rng(0).choice(ncols, 32, replace=False))
    sub = np.zeros((16, nlev, 32))
    sub[:] = fld[:, :, cols]
    ref, pr_ref = run_oracle(sub, dz, 32, dt, nsteps=nsteps)
    assert_fp64_close(out[:, :, cols], pr[:, cols], ref, pr_ref, 32, rtol=RTOL64)


@pytest.fixture(scope="module")
def deep_full():
    """The benchmark's workload: deep convection 512x512 columns x 150 levels."""
    return synth.workload("deep_512x512x150")


@pytest.mark.parametrize("precision", [casim.CASIM_FP64, casim.CASIM_MIXED])
def test_deep_512x512x150_sampled_columns(deep_full, precision):
    """The benchmark's full-size workload in its launch configuration (one
    casim_step over all 262 144 columns): 64 seeded random columns and the
    last column against the oracle, FP64 within 1e-12, mixed within the
    derived bound."""
    fld, dz, ncols, nlev, dt, _ = deep_full
    out, pr, _ = run_gpu(fld, dz, ncols, dt, precision=precision)
    cols = np.concatenate([np.sort(np.random.default_rng(77).choice(ncols - 1, 64, replace=False)), [ncols - 1]])
    sub = np.zeros((fld.shape[0], nlev, 96))
    sub[:, :, :cols.size] = fld[:, :, cols]
    ref, pr_ref = run_oracle(sub, dz, cols.size, dt)
    got = np.zeros_like(sub)
    got[:, :, :cols.size] = out[:, :, cols]
    gpr = np.zeros((4, 96))
    gpr[:, :cols.size] = pr[:, cols]
    if precision == casim.CASIM_FP64:
        assert_fp64_close(got, gpr, ref, pr_ref, cols.size)
    else:
        n = cols.size
        for f in range(13):
            a_, b_, i_ = got[f, :, :n], ref[f, :, :n], sub[f, :, :n]
            bound = mixed_bound(b_, i_, f, ref[1, :, :n])
            assert (np.abs(a_ - b_) <= bound).all(), (synth.FIELDS[f], float((np.abs(a_ - b_) / bound).max()))


def test_maximum_level_count():
    """1024 levels (the largest column the step takes) against the oracle;
    1025 is refused before any launch."""
    ncols, nlev = 40, 1024
    dz = np.full(nlev, 20.0)
    fld = synth.make_state("deep_convective", ncols, nlev, dz, seed=21)
    out, pr, _ = run_gpu(fld, dz, ncols, 1.0)
    ref, pr_ref = run_oracle(fld, dz, ncols, 1.0)
    assert_fp64_close(out, pr, ref, pr_ref, ncols)
    ctx = casim.casim_init(precision=casim.CASIM_MIXED)
    try:
        dz2 = np.full(nlev + 1, 20.0)
        d = casim.Domain(np.zeros((16, nlev + 1, 64)), dz2, ncols)
        with pytest.raises(RuntimeError):
            casim.casim_step(ctx, d.state, ncols, nlev + 1, 1.0)
    finally:
        casim.casim_free(ctx)


def test_clear_columns_are_bitwise_unchanged():
    dz = synth.dz_uniform(40)
    rc = synth.Recipe(cloud_frac=0.0, T_sfc=300.0, rh_clear=(0.5, 0.8))
    fld = synth.make_state(rc, 64, 40, dz, seed=3)
    for prec in (casim.CASIM_FP64, casim.CASIM_MIXED):
        out, pr, _ = run_gpu(fld, dz, 64, 1.0, precision=prec)
        assert np.array_equal(out, fld)
        assert np.all(pr == 0.0)


def test_zero_columns_is_a_noop():
    dz = synth.dz_uniform(10)
    fld = synth.make_state("stratus", 32, 10, dz, seed=1)
    ctx = casim.casim_init()
    try:
        d = casim.Domain(fld, dz, 32)
        n0 = casim.casim_launch_count(ctx)
        casim.casim_step(ctx, d.state, 0, 10, 1.0)
        assert casim.casim_launch_count(ctx) == n0
        assert np.array_equal(d.numpy()[0], fld)
        with pytest.raises(casim.CasimError):
            casim.casim_step(ctx, d.state, 33, 10, 1.0)      # pitch 32 < ncols
        with pytest.raises(casim.CasimError):
            casim.casim_step(ctx, d.state, 32, 10, -1.0)
        with pytest.raises(casim.CasimError):
            casim.casim_step(ctx, d.state, 32, 2000, 1.0)    # more levels than supported
    finally:
        casim.casim_free(ctx)


def test_nonfinite_input_sets_error_flag():
    dz = synth.dz_uniform(10)
    fld = synth.make_state("stratus", 32, 10, dz, seed=2)
    fld[F["qc"], 5, 7] = np.nan
    for prec in (casim.CASIM_FP64, casim.CASIM_MIXED):
        _, _, (rc, flags) = run_gpu(fld, dz, 32, 1.0, precision=prec, check_err=False)
        assert rc == -4 and flags & casim.EFLAG_NONFINITE


def test_cfl_cap_sets_error_flag():
    dz = np.full(20, 1.0)
    fld = synth.make_state("deep_convective", 32, 20, dz, seed=4)
    fld[F["qr"], 10, :32] = 1e-3
    fld[F["nr"], 10, :32] = 1.0       # huge drops at the speed cap: 1000 m in 100 s on 1-m levels
    _, _, (rc, flags) = run_gpu(fld, dz, 32, 100.0, check_err=False)
    assert rc == -5 and flags & casim.EFLAG_CFL


def _host_buffers(fld, npr, pinned):
    """Host copies of a state for casim_step_host: numpy (pageable: the copy
    path) or pinned torch tensors viewed as numpy (mapped: the in-place path)."""
    import torch
    h = np.ascontiguousarray(fld.copy())
    hpr = np.zeros((npr, fld.shape[2]))
    if pinned:
        th, tpr = torch.from_numpy(h).pin_memory(), torch.from_numpy(hpr).pin_memory()
        return th.numpy(), tpr.numpy(), (th, tpr)
    return h, hpr, None


@pytest.mark.parametrize("pinned", [False, True], ids=["pageable", "pinned"])
@pytest.mark.parametrize("case", ["stratus_16x16x50", "deep_1000_of_1056", "deep_mixed_140000_of_140032x6"])
def test_host_entry_point_matches_device_entry_point(case, pinned):
    """The host-buffer step gives the device step's result bit for bit.
    Pageable host memory: one chunk copied whole (pitch = ncols, and pitch >
    ncols); three column chunks of 65 536, 65 536 and 8 928 pipelined over the
    internal streams, pitch > ncols, mixed form.  Pinned host memory: the step
    kernel loads and stores the host state in place."""
    precision = casim.CASIM_FP64
    if case == "stratus_16x16x50":
        fld, dz, ncols, nlev, dt, _ = synth.workload(case)
    else:
        ncols, pitch, nlev = (1000, 1056, 150) if case.startswith("deep_1000") else (140000, 140032, 6)
        dz = synth.dz_stretched(nlev)
        fld = synth.make_state("deep_convective", ncols, nlev, dz, seed=21, pitch=pitch)
        dt = 1.0
        if "mixed" in case:
            precision = casim.CASIM_MIXED
    out, pr, _ = run_gpu(fld, dz, ncols, dt, precision=precision)
    ctx = casim.casim_init(precision=precision)
    try:
        h, hpr, _keep = _host_buffers(fld, 4, pinned)
        hdz = np.ascontiguousarray(dz)
        st = casim.make_state(h, fld.shape[2], hdz, hpr)
        n0 = casim.casim_launch_count(ctx)
        casim.casim_step_host(ctx, st, ncols, nlev, dt, stream=0)
        rc, flags = casim.casim_get_error(ctx)
        assert rc == 0, (rc, flags)
        if ncols > 65536 and _readonly_host_registration() == 0:
            # in place: one launch; copies: one per 65 536-column chunk
            assert casim.casim_launch_count(ctx) - n0 == (1 if pinned else 3)
        assert np.array_equal(h, out)
        assert np.array_equal(hpr, pr)
    finally:
        casim.casim_free(ctx)


def _readonly_host_registration():
    """cudaDevAttrHostRegisterReadOnlySupported of device 0, from the CUDA
    runtime library (None if it cannot be loaded)."""
    import ctypes
    for name in ("libcudart.so.13", "/usr/local/cuda/lib64/libcudart.so"):
        try:
            rt = ctypes.CDLL(name)
        except OSError:
            continue
        v = ctypes.c_int(-1)
        if rt.cudaDeviceGetAttribute(ctypes.byref(v), 113, 0) == 0:
            return v.value
    return None


def test_registered_host_memory():
    """Host memory pinned by cudaHostRegister: stepped in place (one launch
    for 140 000 columns) on a device that cannot register host memory
    read-only, as GB300, else moved by the copies (three chunk launches);
    bit for bit the device step's result either way."""
    import torch
    ncols, pitch, nlev = 140000, 140032, 6
    dz = synth.dz_stretched(nlev)
    fld = synth.make_state("deep_convective", ncols, nlev, dz, seed=21, pitch=pitch)
    out, pr, _ = run_gpu(fld, dz, ncols, 1.0, precision=casim.CASIM_MIXED)
    nf, npr = fld.size, 4 * pitch
    raw = np.zeros(nf + npr + 64)
    off = (-raw.ctypes.data % 256) // 8
    buf = raw[off:off + nf + npr]   # the fields 256-byte aligned, then precip
    h = buf[:nf].reshape(fld.shape)
    h[...] = fld
    hpr = buf[nf:].reshape(4, pitch)
    cr = torch.cuda.cudart()
    assert int(cr.cudaHostRegister(buf.ctypes.data, buf.nbytes, 0)) == 0
    ctx = casim.casim_init(precision=casim.CASIM_MIXED)
    try:
        n0 = casim.casim_launch_count(ctx)
        casim.casim_step_host(ctx, casim.make_state(h, pitch, np.ascontiguousarray(dz), hpr), ncols, nlev, 1.0)
        ro = _readonly_host_registration()
        if ro is not None:
            assert casim.casim_launch_count(ctx) - n0 == (3 if ro else 1)
        assert casim.casim_get_error(ctx)[0] == 0
        assert np.array_equal(h, out) and np.array_equal(hpr, pr)
    finally:
        casim.casim_free(ctx)
        cr.cudaHostUnregister(buf.ctypes.data)


@pytest.mark.parametrize("precision", [casim.CASIM_FP64, casim.CASIM_MIXED])
def test_pinned_host_state_in_place_and_misaligned(precision):
    """Pinned host state stepped in place over the host link: dt = 30 s (the
    multi-substep sedimentation sweeps re-read the host state) and three steps
    in a row equal three device steps bit for bit; a pinned state whose fields
    start off the 256-byte alignment goes through the copies and agrees too."""
    import torch
    nlev, ncols, pitch, dt = 150, 1000, 1024, 30.0
    dz = synth.dz_stretched(nlev)
    fld = synth.make_state("deep_convective", ncols, nlev, dz, seed=23, pitch=pitch)
    d = casim.Domain(fld, dz, ncols)
    ctx = casim.casim_init(precision=precision)
    try:
        for _ in range(3):
            casim.casim_step(ctx, d.state, ncols, nlev, dt)
        assert casim.casim_get_error(ctx)[0] == 0
        out, pr = d.numpy()
        h, hpr, _keep = _host_buffers(fld, 4, True)
        st = casim.make_state(h, pitch, np.ascontiguousarray(dz), hpr)
        for _ in range(3):
            casim.casim_step_host(ctx, st, ncols, nlev, dt)
        assert casim.casim_get_error(ctx)[0] == 0
        assert np.array_equal(h, out) and np.array_equal(hpr, pr)
        # the same state 8 bytes into a pinned buffer
        big = torch.zeros(fld.size + 1, dtype=torch.float64).pin_memory()
        hb = big.numpy()[1:].reshape(fld.shape)
        hb[...] = fld
        assert hb.ctypes.data % 256 == 8
        hpr[...] = 0.0
        out1, pr1, _ = run_gpu(fld, dz, ncols, dt, precision=precision)
        casim.casim_step_host(ctx, casim.make_state(hb, pitch, np.ascontiguousarray(dz), hpr), ncols, nlev, dt)
        assert casim.casim_get_error(ctx)[0] == 0
        assert np.array_equal(hb, out1) and np.array_equal(hpr, pr1)
    finally:
        casim.casim_free(ctx)


@pytest.mark.parametrize("precision", [casim.CASIM_FP64, casim.CASIM_MIXED])
@pytest.mark.parametrize("dt", [0.1, 1.0 / 3.0, 2.0, 7.3, 0.25, 11.0])
def test_tendency_division_by_dt_is_correctly_rounded(precision, dt):
    """The source terms divide by dt through one reciprocal per launch (exact
    for a power-of-two dt, Markstein's correction otherwise): on every point
    of a deep-convective state, at time steps that are and are not powers of
    two, tend equals numpy's correctly rounded (x_after - x_before) / dt bit
    for bit."""
    import torch
    nlev = 120
    dz = synth.dz_stretched(nlev)
    ncols, pitch = 256, 256
    fld = synth.make_state("deep_convective", ncols, nlev, dz, seed=41, pitch=pitch)
    out, _, _ = run_gpu(fld, dz, ncols, dt, precision=precision)
    ctx = casim.casim_init(precision=precision)
    try:
        d = casim.Domain(fld, dz, ncols)
        tend = torch.full((13, nlev, pitch), float("nan"), dtype=torch.float64, device="cuda")
        casim.casim_step_tendency(ctx, d.state, ncols, nlev, dt, tend)
        assert casim.casim_get_error(ctx)[0] == 0
        diff = out[:13, :, :ncols] - fld[:13, :, :ncols]
        t = tend.cpu().numpy()[:, :, :ncols]
        assert np.count_nonzero(diff) > 10000   # many quotients that are not zero
        assert np.array_equal(t, diff / dt)
        assert np.array_equal(np.signbit(t), np.signbit(diff / dt))
    finally:
        casim.casim_free(ctx)


@pytest.mark.parametrize("precision", [casim.CASIM_FP64, casim.CASIM_MIXED])
@pytest.mark.parametrize("dt", [1.0, 30.0])
def test_tendency_mode_equals_in_place_step(precision, dt):
    """Source-term mode: the state is untouched and tend is (x_after - x_before)
    / dt of the in-place step, bit for bit, at every point (also where nothing
    changes: zero); dt = 30 s takes the multi-substep sedimentation path."""
    import torch
    nlev = 150
    dz = synth.dz_stretched(nlev)
    ncols, pitch = 333, 352
    fld = synth.make_state("deep_convective", ncols, nlev, dz, seed=31, pitch=pitch)
    out, pr, _ = run_gpu(fld, dz, ncols, dt, precision=precision)
    ctx = casim.casim_init(precision=precision)
    try:
        d = casim.Domain(fld, dz, ncols)
        tend = torch.full((13, nlev, pitch), float("nan"), dtype=torch.float64, device="cuda")
        casim.casim_step_tendency(ctx, d.state, ncols, nlev, dt, tend)
        rc, flags = casim.casim_get_error(ctx)
        assert rc == 0, (rc, flags)
        f2, p2 = d.numpy()
        assert np.array_equal(f2, fld)                      # state unchanged
        assert np.array_equal(p2, pr)                       # precipitation accumulated as in place
        t = tend.cpu().numpy()[:, :, :ncols]
        expect = (out[:13, :, :ncols] - fld[:13, :, :ncols]) / dt
        assert np.array_equal(t, expect)
        assert np.isnan(tend.cpu().numpy()[:, :, ncols:]).all()   # padding columns not written
        with pytest.raises(RuntimeError):                   # tend overlapping the state
            casim.casim_step_tendency(ctx, d.state, ncols, nlev, dt, d.fld)
    finally:
        casim.casim_free(ctx)


@pytest.mark.parametrize("precision", [casim.CASIM_FP64, casim.CASIM_MIXED])
def test_column_ranges_on_streams_equal_one_launch(precision):
    """The sharded path on one GPU: the domain split into three 32-aligned
    column ranges, each stepped on its own stream at the same time, gives the
    single launch's result bit for bit (columns are independent)."""
    import torch
    from paper_2010_14823_gb300 import shard
    nlev, ncols = 150, 1000
    dz = synth.dz_stretched(nlev)
    fld = synth.make_state("deep_convective", ncols, nlev, dz, seed=61)
    out, pr, _ = run_gpu(fld, dz, ncols, 1.0, precision=precision)
    ctx = casim.casim_init(precision=precision)
    try:
        d = casim.Domain(fld, dz, ncols)
        streams = [torch.cuda.Stream() for _ in range(3)]
        torch.cuda.synchronize()
        for r, st in enumerate(streams):
            c0, c1 = shard.column_range_aligned(ncols, r, 3)
            view = casim.make_state(d.fld.data_ptr() + 8 * c0, d.pitch, d.dz, d.precip.data_ptr() + 8 * c0)
            casim.casim_step(ctx, view, c1 - c0, nlev, 1.0, st)
        torch.cuda.synchronize()
        assert casim.casim_get_error(ctx)[0] == 0
        f2, p2 = d.numpy()
        assert np.array_equal(f2, out) and np.array_equal(p2, pr)
    finally:
        casim.casim_free(ctx)


def test_budget_sums():
    fld, dz, ncols, nlev, dt, _ = synth.workload("stratus_16x16x50")
    ctx = casim.casim_init()
    try:
        d = casim.Domain(fld, dz, ncols)
        out = torch.zeros((2, ncols), dtype=torch.float64, device="cuda")
        casim.casim_budget(ctx, d.state, ncols, nlev, out)
        got = out.cpu().numpy()
    finally:
        casim.casim_free(ctx)
    m = fld[F["rho"], :, :ncols] * dz[:, None]
    w = (m * sum(fld[F[x], :, :ncols] for x in ("qv", "qc", "qr", "qi", "qs", "qg"))).sum(0)
    n = (m * (fld[F["nc"], :, :ncols] + fld[F["na"], :, :ncols])).sum(0)
    assert np.allclose(got[0], w, rtol=1e-13, atol=0.0) and np.allclose(got[1], n, rtol=1e-13, atol=0.0)


# ------------------------------------------------------------------ mixed
def mixed_bound(ref, inp, f, qv_ref):
    """Bound of the mixed form's error against the FP64 oracle for field f.

    Rates and fall speeds run in FP32 with MUFU ex2/lg2 (relative error about
    2^-22 per call, up to ~10 chained calls) and truncating conversions
    (2^-23): each increment carries a relative error below ~1e-5.  Saturation
    adjustment evaluates q_s in FP32 (relative ~1e-6 of q_s), which moves
    ~1e-6 q_v of vapour between q_v and q_c, and Lv/cp times that in T.  The
    bound gives a factor of 10-100 over these estimates.
    """
    inc = np.abs(ref - inp)
    if f == 0:
        return 1e-3 * inc + 2.5e3 * 1e-5 * qv_ref + 1e-6
    if f in (1, 2):
        return 1e-3 * inc + 1e-5 * qv_ref + 1e-14
    if f <= 6:
        return 1e-3 * inc + 1e-5 * np.abs(ref) + 1e-14
    # numbers: ice nucleation sets n_i to exp(12.96 (S_i - 1)) scaled; S_i in
    # FP32 carries ~4e-7 relative error, i.e. ~1e-5 relative in n_i
    return 1e-3 * inc + 1e-4 * np.abs(ref) + 1e-3


@pytest.mark.parametrize("name", ["stratus_16x16x50", "deep"])
def test_mixed_within_derived_bound(name):
    if name == "deep":
        dz = synth.dz_stretched(150)
        fld = synth.make_state("deep_convective", 512, 150, dz, seed=11)
        ncols, dt = 512, 1.0
    else:
        fld, dz, ncols, nlev, dt, _ = synth.workload(name)
    out, pr, _ = run_gpu(fld, dz, ncols, dt, precision=casim.CASIM_MIXED)
    ref, pr_ref = run_oracle(fld, dz, ncols, dt)
    worst = {}
    for f in range(13):
        a, b, i = out[f, :, :ncols], ref[f, :, :ncols], fld[f, :, :ncols]
        err = np.abs(a - b)
        bound = mixed_bound(b, i, f, ref[1, :, :ncols])
        worst[synth.FIELDS[f]] = float((err / np.maximum(bound, 1e-300)).max())
        assert (err <= bound).all(), (synth.FIELDS[f], float(err.max()), np.argwhere(err > bound)[:3].tolist())
    print("mixed worst error / bound:", worst)


def test_mixed_conserves_water():
    dz = synth.dz_stretched(150)
    fld = synth.make_state("deep_convective", 512, 150, dz, seed=12)
    out, pr, _ = run_gpu(fld, dz, 512, 1.0, nsteps=3, precision=casim.CASIM_MIXED)
    rho = fld[F["rho"], :, :512]
    names = ("qv", "qc", "qr", "qi", "qs", "qg")
    w0 = sum((fld[F[x], :, :512] * rho * dz[:, None]).sum(0) for x in names)
    w1 = sum((out[F[x], :, :512] * rho * dz[:, None]).sum(0) for x in names)
    drift = np.abs(w1 + pr[:, :512].sum(0) - w0) / w0
    # each field's net increment at a point (process transfers and sedimentation,
    # summed in FP32) carries FP32 rounding of the water moved there, a small
    # fraction of the column's water per step; the FP64 additions add 1e-16
    print("mixed water drift over 3 steps:", float(drift.max()))
    assert drift.max() < 1e-9, drift.max()


# ------------------------------------------------------------------ warm configuration
ICE = [F[x] for x in ("qi", "qs", "qg", "ni", "ns", "ng")]


@pytest.mark.parametrize("dt", [1.0, 30.0])
def test_warm_fp64_matches_oracle_and_leaves_ice(dt):
    """The warm configuration on a deep-convective state that carries ice:
    liquid fields within 1e-12 of the oracle's warm mode, ice fields bitwise
    untouched, no ice, snow or graupel precipitation.  dt = 1 s over three
    steps; dt = 30 s (the multi-substep path) over one: in its first step the
    limiter exhausts some cloud-droplet pools, leaving numbers that are the
    rounding residue of n - n (e.g. 7e-9 /kg from 3.4e8), which FMA rounds
    differently, and later steps branch on that residue."""
    nlev = 150
    dz = synth.dz_stretched(nlev)
    ncols = 97
    nsteps = 3 if dt == 1.0 else 1
    fld = synth.make_state("deep_convective", ncols, nlev, dz, seed=41)
    out, pr, _ = run_gpu(fld, dz, ncols, dt, nsteps=nsteps, flags=casim.CASIM_WARM)
    ref, pr_ref = run_oracle(fld, dz, ncols, dt, nsteps=nsteps, warm=True)
    assert_fp64_close(out, pr, ref, pr_ref, ncols, rtol=RTOL64)
    for f in ICE:
        assert np.array_equal(out[f], fld[f])
    assert np.all(pr[1:] == 0.0)


def test_warm_mixed_within_derived_bound():
    nlev = 150
    dz = synth.dz_stretched(nlev)
    fld = synth.make_state("deep_convective", 512, nlev, dz, seed=42)
    out, pr, _ = run_gpu(fld, dz, 512, 1.0, precision=casim.CASIM_MIXED, flags=casim.CASIM_WARM)
    ref, pr_ref = run_oracle(fld, dz, 512, 1.0, warm=True)
    for f in range(13):
        a, b, i = out[f, :, :512], ref[f, :, :512], fld[f, :, :512]
        bound = mixed_bound(b, i, f, ref[1, :, :512])
        assert (np.abs(a - b) <= bound).all(), synth.FIELDS[f]
    for f in ICE:
        assert np.array_equal(out[f], fld[f])


def test_warm_equals_cold_on_an_ice_free_warm_state():
    """Both configurations against the oracle on a state without ice and
    warmer than the nucleation threshold, where the two chains coincide."""
    fld, dz, ncols, nlev, dt, _ = synth.workload("stratus_16x16x50")
    top = int(np.argmax(fld[F["T"], :, :ncols].min(axis=1) < O.param("T_nuc") + 1.0))
    sub = np.ascontiguousarray(fld[:, :top, :])
    sub[ICE] = 0.0
    dzs = np.ascontiguousarray(dz[:top])
    cold, pc, _ = run_gpu(sub, dzs, ncols, dt)
    warm, pw, _ = run_gpu(sub, dzs, ncols, dt, flags=casim.CASIM_WARM)
    ref, pr_ref = run_oracle(sub, dzs, ncols, dt)
    assert_fp64_close(cold, pc, ref, pr_ref, ncols)
    assert_fp64_close(warm, pw, ref, pr_ref, ncols)


@pytest.mark.parametrize("dt", [1.0, 30.0])
def test_warm_tendency_and_host_entry_points(dt):
    import torch
    nlev = 150
    dz = synth.dz_stretched(nlev)
    ncols, pitch = 200, 224
    fld = synth.make_state("deep_convective", ncols, nlev, dz, seed=43, pitch=pitch)
    out, pr, _ = run_gpu(fld, dz, ncols, dt, precision=casim.CASIM_MIXED, flags=casim.CASIM_WARM)
    ctx = casim.casim_init(precision=casim.CASIM_MIXED, flags=casim.CASIM_WARM)
    try:
        d = casim.Domain(fld, dz, ncols)
        tend = torch.full((13, nlev, pitch), float("nan"), dtype=torch.float64, device="cuda")
        casim.casim_step_tendency(ctx, d.state, ncols, nlev, dt, tend)
        assert casim.casim_get_error(ctx)[0] == 0
        t = tend.cpu().numpy()[:, :, :ncols]
        assert np.array_equal(t, (out[:13, :, :ncols] - fld[:13, :, :ncols]) / dt)
        assert np.all(t[ICE] == 0.0)
        for pinned in (False, True):   # the copies; the in-place step over the host link
            h, hpr, _keep = _host_buffers(fld, 4, pinned)
            casim.casim_step_host(ctx, casim.make_state(h, pitch, np.ascontiguousarray(dz), hpr), ncols, nlev, dt)
            assert np.array_equal(h, out) and np.array_equal(hpr, pr), pinned
        # entry points without a warm variant refuse a warm context
        with pytest.raises(RuntimeError):
            casim.casim_batch_create(ctx, [d.state], [ncols], [nlev])
    finally:
        casim.casim_free(ctx)


# ------------------------------------------------------------------ activated-aerosol mass (warm)
MA, MAC, MAR = 16, 17, 18


def _aero_state(ncols, nlev, seed, pitch=None):
    dz = synth.dz_stretched(nlev)
    base = synth.make_state("deep_convective", ncols, nlev, dz, seed=seed, pitch=pitch)
    fld = np.zeros((19,) + base.shape[1:])
    fld[:16] = base
    rng = np.random.default_rng(seed)
    fld[MA] = rng.uniform(1e-9, 5e-9, base.shape[1:])
    fld[MAC] = fld[F["qc"]] * rng.uniform(1e-5, 1e-4, base.shape[1:])
    fld[MAR] = fld[F["qr"]] * rng.uniform(1e-5, 1e-4, base.shape[1:])
    return np.ascontiguousarray(fld), dz


def _run_gpu_aero(fld, dz, ncols, dt, nsteps, precision):
    ctx = casim.casim_init(precision=precision, flags=casim.CASIM_WARM | casim.CASIM_AEROSOL)
    try:
        d = casim.Domain(fld, dz, ncols)
        for _ in range(nsteps):
            casim.casim_step(ctx, d.state, ncols, d.nlev, dt)
        rc, flags = casim.casim_get_error(ctx)
        assert rc == 0, (rc, flags)
        return d.numpy()
    finally:
        casim.casim_free(ctx)


@pytest.mark.parametrize("dt", [1.0, 30.0])
def test_aerosol_fp64_matches_oracle(dt):
    """FP64 form with activated-aerosol mass: all 16 updated fields and the 5
    precipitation rows within 1e-12 of the oracle; the standard fields equal
    the warm step's without aerosol, bit for bit (the extension is
    additive)."""
    ncols, nlev = 97, 150
    nsteps = 3 if dt == 1.0 else 1
    fld, dz = _aero_state(ncols, nlev, seed=51)
    out, pr = _run_gpu_aero(fld, dz, ncols, dt, nsteps, casim.CASIM_FP64)
    ref = fld.copy()
    pref = np.zeros((5, fld.shape[2]))
    for _ in range(nsteps):
        _, err = O.step_aero(ref, ncols, dz, dt, precip=pref)
        assert err == 0
    rt = RTOL64
    assert_fp64_close(out, pr[:4], ref, pref[:4], ncols, rtol=rt)
    # aerosol masses: relative to the point's total aerosol mass -- a pool
    # that gives most of itself away (e.g. free aerosol almost all
    # activated) ends as a small difference of large moves, so its error
    # scales with the aerosol moved, not with what is left
    scale = (fld[MA] + fld[MAC] + fld[MAR])[:, :ncols]
    for f in (MA, MAC, MAR):
        a, b = out[f, :, :ncols], ref[f, :, :ncols]
        assert (np.abs(a - b) <= rt * np.maximum(np.abs(b), scale) + 1e-26).all(), \
            (f, float(np.abs(a - b).max()))
    assert np.allclose(pr[4, :ncols], pref[4, :ncols], rtol=rt, atol=1e-26)
    assert pref[4, :ncols].max() > 0.0
    std, pstd, _ = run_gpu(np.ascontiguousarray(fld[:16]), dz, ncols, dt, nsteps=nsteps, flags=casim.CASIM_WARM)
    assert np.array_equal(out[:16], std) and np.array_equal(pr[:4], pstd)


def test_aerosol_mixed_within_bound_and_budget():
    ncols, nlev = 512, 150
    fld, dz = _aero_state(ncols, nlev, seed=52)
    out, pr = _run_gpu_aero(fld, dz, ncols, 1.0, 1, casim.CASIM_MIXED)
    ref = fld.copy()
    pref = np.zeros((5, fld.shape[2]))
    O.step_aero(ref, ncols, dz, 1.0, precip=pref)
    for f in range(13):
        a, b, i = out[f, :, :ncols], ref[f, :, :ncols], fld[f, :, :ncols]
        assert (np.abs(a - b) <= mixed_bound(b, i, f, ref[1, :, :ncols])).all(), synth.FIELDS[f]
    # aerosol moved in FP32: each amount is an FP32 product of a pool and a
    # fraction derived from FP32 rates (relative error ~1e-5, see
    # mixed_bound), and no move exceeds the point's total aerosol, so the
    # error is below ~1e-5 of that total; the bound gives a factor of 10
    scale = (fld[MA] + fld[MAC] + fld[MAR])[:, :ncols]
    for f in (MA, MAC, MAR):
        a, b = out[f, :, :ncols], ref[f, :, :ncols]
        bound = 1e-4 * scale + 1e-22
        assert (np.abs(a - b) <= bound).all(), (f, float((np.abs(a - b) / bound).max()))
    assert (out[[MA, MAC, MAR], :, :ncols] >= 0).all()
    # column budget: process moves are exact FP64 pairs; each level's
    # sedimentation increment of rain aerosol is one FP32 amount (relative
    # rounding <= 2^-23), so the drift is below 2^-22 of the summed
    # |change of mar| (an upper proxy for those increments)
    rho = fld[F["rho"], :, :ncols]
    w = rho * dz[:, None]
    m0 = ((fld[MA] + fld[MAC] + fld[MAR])[:, :ncols] * w).sum(0)
    m1 = ((out[MA] + out[MAC] + out[MAR])[:, :ncols] * w).sum(0)
    moved = (np.abs(out[MAR] - fld[MAR])[:, :ncols] * w).sum(0) + pr[4, :ncols]
    assert (np.abs(m1 + pr[4, :ncols] - m0) <= 2.0 ** -22 * moved + 1e-15 * m0).all()


def test_aerosol_context_rules():
    import torch
    for flags in (casim.CASIM_AEROSOL | casim.CASIM_THREE_MOMENT,
                  casim.CASIM_WARM | casim.CASIM_AEROSOL | casim.CASIM_THREE_MOMENT):
        with pytest.raises(RuntimeError):
            casim.casim_init(precision=casim.CASIM_MIXED, flags=flags)
    fld, dz = _aero_state(64, 40, seed=53)
    ctx = casim.casim_init(precision=casim.CASIM_MIXED, flags=casim.CASIM_WARM | casim.CASIM_AEROSOL)
    try:
        d = casim.Domain(fld, dz, 64)
        with pytest.raises(RuntimeError):                 # the batched entry points have no aerosol variant
            casim.casim_batch_create(ctx, [d.state], [64], [40])
        with pytest.raises(RuntimeError):                 # tend overlapping the state
            casim.casim_step_tendency(ctx, d.state, 64, 40, 1.0, d.fld[1:])
    finally:
        casim.casim_free(ctx)



# ------------------------------------- activated-aerosol mass, cold configuration
MAI, MAS, MAG = 19, 20, 21


def _aero_cold_state(ncols, nlev, seed):
    dz = synth.dz_stretched(nlev)
    base = synth.make_state("deep_convective", ncols, nlev, dz, seed=seed)
    fld = np.zeros((22,) + base.shape[1:])
    fld[:16] = base
    rng = np.random.default_rng(seed)
    fld[MA] = rng.uniform(1e-9, 5e-9, base.shape[1:])
    for f, q in ((MAC, "qc"), (MAR, "qr"), (MAI, "qi"), (MAS, "qs"), (MAG, "qg")):
        fld[f] = fld[F[q]] * rng.uniform(1e-5, 1e-4, base.shape[1:])
    return np.ascontiguousarray(fld), dz


def _run_oracle_aero_cold(fld, dz, ncols, dt, nsteps):
    ref = fld.copy()
    pref = np.zeros((5, fld.shape[2]))
    for _ in range(nsteps):
        _, err = O.step_aero_cold(ref, ncols, dz, dt, precip=pref)
        assert err == 0
    return ref, pref


@pytest.mark.parametrize("dt", [1.0, 30.0])
def test_aerosol_cold_fp64_matches_oracle(dt):
    """FP64 form, aerosol mass in cloud, rain and the ice species: the 13
    prognostic fields and 4 precipitation rows within 1e-12 of the oracle,
    the six aerosol masses within 1e-12 of the point's total aerosol, the
    deposited row likewise; the standard fields are the cold step's bit for
    bit (the extension is additive)."""
    ncols, nlev = 97, 150
    nsteps = 3 if dt == 1.0 else 1
    fld, dz = _aero_cold_state(ncols, nlev, seed=54)
    out, pr, _ = run_gpu(fld, dz, ncols, dt, nsteps=nsteps, flags=casim.CASIM_AEROSOL)
    ref, pref = _run_oracle_aero_cold(fld, dz, ncols, dt, nsteps)
    rt = RTOL64
    assert_fp64_close(out, pr[:4], ref, pref[:4], ncols, rtol=rt)
    scale = fld[MA:MAG + 1, :, :ncols].sum(axis=0)
    for f in range(MA, MAG + 1):
        a, b = out[f, :, :ncols], ref[f, :, :ncols]
        assert (np.abs(a - b) <= rt * np.maximum(np.abs(b), scale) + 1e-26).all(), (f, float(np.abs(a - b).max()))
    assert np.allclose(pr[4, :ncols], pref[4, :ncols], rtol=rt, atol=1e-26)
    assert pref[4, :ncols].max() > 0.0
    std, pstd, _ = run_gpu(np.ascontiguousarray(fld[:16]), dz, ncols, dt, nsteps=nsteps)
    assert np.array_equal(out[:16], std) and np.array_equal(pr[:4], pstd)


def test_aerosol_cold_mixed_within_bound_and_budget():
    """Mixed form: the 13 fields within the mixed bound; each aerosol mass
    within 1e-4 of the point's total aerosol (every amount moved is one FP32
    product of a pool and a fraction of FP32 rates, ~1e-5 relative, and no
    move exceeds the total); the column's total aerosol plus the deposited row
    conserved to 2^-22 of the aerosol moved by sedimentation (one FP32 amount
    per level and species) plus FP64 rounding."""
    ncols, nlev = 512, 150
    fld, dz = _aero_cold_state(ncols, nlev, seed=55)
    out, pr, _ = run_gpu(fld, dz, ncols, 1.0, precision=casim.CASIM_MIXED, flags=casim.CASIM_AEROSOL)
    ref, pref = _run_oracle_aero_cold(fld, dz, ncols, 1.0, 1)
    for f in range(13):
        a, b, i = out[f, :, :ncols], ref[f, :, :ncols], fld[f, :, :ncols]
        assert (np.abs(a - b) <= mixed_bound(b, i, f, ref[1, :, :ncols])).all(), synth.FIELDS[f]
    scale = fld[MA:MAG + 1, :, :ncols].sum(axis=0)
    for f in range(MA, MAG + 1):
        a, b = out[f, :, :ncols], ref[f, :, :ncols]
        bound = 1e-4 * scale + 1e-22
        assert (np.abs(a - b) <= bound).all(), (f, float((np.abs(a - b) / bound).max()))
    assert (out[MA:MAG + 1, :, :ncols] >= 0).all()
    w = fld[F["rho"], :, :ncols] * dz[:, None]
    m0 = (fld[MA:MAG + 1, :, :ncols] * w).sum(axis=(0, 1))
    m1 = (out[MA:MAG + 1, :, :ncols] * w).sum(axis=(0, 1))
    moved = (np.abs(out[MAR:MAG + 1] - fld[MAR:MAG + 1])[:, :, :ncols] * w).sum(axis=(0, 1)) + pr[4, :ncols]
    assert (np.abs(m1 + pr[4, :ncols] - m0) <= 2.0 ** -22 * moved + 1e-15 * m0).all()


# ------------------------------------------------------------------ triple-moment rain (warm)
ZR = 16


def _gamma_g(mu):
    """z n / (q/a)^2 of a gamma distribution of shape mu."""
    return (mu + 4) * (mu + 5) * (mu + 6) / ((mu + 1) * (mu + 2) * (mu + 3))


def _tri_state(ncols, nlev, seed, mu=None, pitch=None):
    """Deep-convective state with the rain's sixth moment of a gamma
    distribution of shape mu (default: shapes uniform in [0, 8])."""
    dz = synth.dz_stretched(nlev)
    base = synth.make_state("deep_convective", ncols, nlev, dz, seed=seed, pitch=pitch)
    fld = np.zeros((17,) + base.shape[1:])
    fld[:16] = base
    rng = np.random.default_rng(seed)
    qr, nr = base[F["qr"]], base[F["nr"]]
    shape = np.full(qr.shape, mu) if mu is not None else rng.uniform(0.0, 8.0, qr.shape)
    ok = (qr > 1e-14) & (nr > 0)
    fld[ZR][ok] = _gamma_g(shape[ok]) * (qr[ok] / O.param("a_r")) ** 2 / nr[ok]
    return np.ascontiguousarray(fld), dz


def _run_oracle_3m(fld, dz, ncols, dt, nsteps):
    ref = fld.copy()
    pref = np.zeros((4, fld.shape[2]))
    for _ in range(nsteps):
        _, err = O.step_3m(ref, ncols, dz, dt, precip=pref)
        assert err == 0
    return ref, pref


@pytest.mark.parametrize("dt", [1.0, 30.0])
def test_three_moment_fp64_matches_oracle(dt):
    """FP64 form with triple-moment rain: the 13 prognostic fields, z and the
    precipitation within 1e-12 of the oracle (z with an absolute floor of
    1e-16 of the domain's largest z, the floor the masses have relative to
    their typical size); ice fields untouched."""
    ncols, nlev = 97, 150
    nsteps = 3 if dt == 1.0 else 1
    fld, dz = _tri_state(ncols, nlev, seed=61)
    out, pr, _ = run_gpu(fld, dz, ncols, dt, nsteps=nsteps, flags=casim.CASIM_WARM | casim.CASIM_THREE_MOMENT)
    ref, pref = _run_oracle_3m(fld, dz, ncols, dt, nsteps)
    rt = RTOL64
    assert_fp64_close(out, pr, ref, pref, ncols, rtol=rt)
    a, b = out[ZR, :, :ncols], ref[ZR, :, :ncols]
    floor = 1e-16 * fld[ZR].max()
    assert (np.abs(a - b) <= rt * np.abs(b) + floor).all(), float(np.abs(a - b).max())
    assert not np.array_equal(out[ZR], fld[ZR])
    for f in ICE:
        assert np.array_equal(out[f], fld[f])
    assert np.all(pr[1:] == 0.0) and pr[0, :ncols].max() > 0.0


def test_three_moment_reduces_to_warm_at_the_two_moment_shape():
    """Cloud-free, subsaturated air (no autoconversion, the only source of a
    shape change) with z at the two-moment rain's shape: the 16 fields agree
    with the two-moment warm step's to rounding."""
    ncols, nlev = 64, 150
    fld, dz = _tri_state(ncols, nlev, seed=62, mu=O.param("mu_r"))
    for k in range(nlev):
        for c in range(ncols):
            qs = O.qsat(O.es_liq(fld[F["T"], k, c]), fld[F["p"], k, c])
            fld[F["qv"], k, c] = min(fld[F["qv"], k, c], 0.97 * qs)
    fld[F["qc"]] = 0.0
    fld[F["nc"]] = 0.0
    out, pr, _ = run_gpu(fld, dz, ncols, 1.0, flags=casim.CASIM_WARM | casim.CASIM_THREE_MOMENT)
    two, p2, _ = run_gpu(np.ascontiguousarray(fld[:16]), dz, ncols, 1.0, flags=casim.CASIM_WARM)
    assert_fp64_close(out, pr, two, p2, ncols, rtol=1e-12)


def test_three_moment_mixed_within_derived_bound():
    """Mixed form: the 13 fields within the mixed bound; z within
    1e-3 |its change| + 1e-4 |z| of the oracle.  Derivation: the shape comes
    from an FP32 log of G (relative error ~3e-7), and dG/dmu falls to
    |d ln G / d mu| ~ 0.016 at mu = 20, so mu carries up to ~2e-5; the
    speeds depend on mu through FP32 log-gamma differences (~1e-5), so the
    fluxes of z (each at most z itself at Courant number <= 1) carry ~1e-5
    relative; the process factor (q'/q)^2 (n/n') is formed in FP32 from
    FP32 increments (~1e-5 of the change), which is a relative error of the
    change of z."""
    ncols, nlev = 512, 150
    fld, dz = _tri_state(ncols, nlev, seed=63)
    out, pr, _ = run_gpu(fld, dz, ncols, 1.0, precision=casim.CASIM_MIXED,
                         flags=casim.CASIM_WARM | casim.CASIM_THREE_MOMENT)
    ref, pref = _run_oracle_3m(fld, dz, ncols, 1.0, 1)
    for f in range(13):
        a, b, i = out[f, :, :ncols], ref[f, :, :ncols], fld[f, :, :ncols]
        bound = mixed_bound(b, i, f, ref[1, :, :ncols])
        assert (np.abs(a - b) <= bound).all(), (synth.FIELDS[f], float((np.abs(a - b) / bound).max()))
    a, b, i = out[ZR, :, :ncols], ref[ZR, :, :ncols], fld[ZR, :, :ncols]
    bound = 1e-3 * np.abs(b - i) + 1e-4 * np.abs(b) + 1e-16 * fld[ZR].max()
    assert (np.abs(a - b) <= bound).all(), float((np.abs(a - b) / bound).max())
    assert (out[ZR, :, :ncols] >= 0).all()
    for f in ICE:
        assert np.array_equal(out[f], fld[f])


def test_three_moment_context_rules():
    import torch
    for flags in (casim.CASIM_THREE_MOMENT | casim.CASIM_AEROSOL,
                  casim.CASIM_WARM | casim.CASIM_THREE_MOMENT | casim.CASIM_AEROSOL):
        with pytest.raises(RuntimeError):
            casim.casim_init(precision=casim.CASIM_MIXED, flags=flags)
    p = casim.casim_default_params()
    p.b[3] = 2.9                                        # snow: carries z only in the cold configuration
    casim.casim_free(casim.casim_init(params=p, precision=casim.CASIM_MIXED,
                                      flags=casim.CASIM_WARM | casim.CASIM_THREE_MOMENT))
    with pytest.raises(RuntimeError):
        casim.casim_init(params=p, precision=casim.CASIM_MIXED, flags=casim.CASIM_THREE_MOMENT)
    p = casim.casim_default_params()
    p.b[1] = 2.9
    with pytest.raises(RuntimeError):                   # the shape algebra needs b = 3
        casim.casim_init(params=p, precision=casim.CASIM_MIXED, flags=casim.CASIM_WARM | casim.CASIM_THREE_MOMENT)
    fld, dz = _tri_state(64, 40, seed=64)
    ctx = casim.casim_init(precision=casim.CASIM_MIXED, flags=casim.CASIM_WARM | casim.CASIM_THREE_MOMENT)
    try:
        d = casim.Domain(fld, dz, 64)
        with pytest.raises(RuntimeError):                 # the batched entry points have no triple-moment variant
            casim.casim_batch_create(ctx, [d.state], [64], [40])
    finally:
        casim.casim_free(ctx)


# ---------------------------------------------- triple-moment r, i, s, g (cold configuration)
ZC = {"r": 16, "i": 17, "s": 18, "g": 19}
QF = {"r": F["qr"], "i": F["qi"], "s": F["qs"], "g": F["qg"]}
NF = {"r": F["nr"], "i": F["ni"], "s": F["ns"], "g": F["ng"]}


def _tri_cold_state(ncols, nlev, seed):
    """Deep-convective state with each species' sixth moment of a gamma
    distribution of shape uniform in [0, 8]."""
    dz = synth.dz_stretched(nlev)
    base = synth.make_state("deep_convective", ncols, nlev, dz, seed=seed)
    fld = np.zeros((20,) + base.shape[1:])
    fld[:16] = base
    rng = np.random.default_rng(seed)
    for sp in "risg":
        q, n = base[QF[sp]], base[NF[sp]]
        shape = rng.uniform(0.0, 8.0, q.shape)
        ok = (q > 1e-14) & (n > 0)
        fld[ZC[sp]][ok] = _gamma_g(shape[ok]) * (q[ok] / O.param(f"a_{sp}")) ** 2 / n[ok]
    return np.ascontiguousarray(fld), dz


def _run_oracle_3m_cold(fld, dz, ncols, dt, nsteps):
    ref = fld.copy()
    pref = np.zeros((4, fld.shape[2]))
    for _ in range(nsteps):
        _, err = O.step_3m_cold(ref, ncols, dz, dt, precip=pref)
        assert err == 0
    return ref, pref


@pytest.mark.parametrize("dt", [1.0, 30.0])
def test_three_moment_cold_fp64_matches_oracle(dt):
    """FP64 form, triple-moment r, i, s, g: the 13 prognostic fields, the four
    sixth moments and the precipitation within 1e-12 of the oracle (each z
    with an absolute floor of 1e-16 of the domain's largest z of the species)."""
    ncols, nlev = 97, 150
    nsteps = 3 if dt == 1.0 else 1
    fld, dz = _tri_cold_state(ncols, nlev, seed=65)
    out, pr, _ = run_gpu(fld, dz, ncols, dt, nsteps=nsteps, flags=casim.CASIM_THREE_MOMENT)
    ref, pref = _run_oracle_3m_cold(fld, dz, ncols, dt, nsteps)
    rt = RTOL64
    assert_fp64_close(out, pr, ref, pref, ncols, rtol=rt)
    for sp, f in ZC.items():
        a, b = out[f, :, :ncols], ref[f, :, :ncols]
        floor = 1e-16 * fld[f].max()
        assert (np.abs(a - b) <= rt * np.abs(b) + floor).all(), (sp, float(np.abs(a - b).max()))
        assert not np.array_equal(out[f], fld[f]), sp


def test_three_moment_cold_mixed_within_derived_bound():
    """Mixed form, triple-moment r, i, s, g: the 13 fields within the mixed
    bound; each z within 1e-3 |its change| + 1e-4 |z| (the derivation of the
    rain case holds for every species: FP32 shapes, FP32 log-gamma-free
    coefficients, FP32 process factors and sources)."""
    ncols, nlev = 512, 150
    fld, dz = _tri_cold_state(ncols, nlev, seed=66)
    out, pr, _ = run_gpu(fld, dz, ncols, 1.0, precision=casim.CASIM_MIXED, flags=casim.CASIM_THREE_MOMENT)
    ref, pref = _run_oracle_3m_cold(fld, dz, ncols, 1.0, 1)
    for f in range(13):
        a, b, i = out[f, :, :ncols], ref[f, :, :ncols], fld[f, :, :ncols]
        bound = mixed_bound(b, i, f, ref[1, :, :ncols])
        assert (np.abs(a - b) <= bound).all(), (synth.FIELDS[f], float((np.abs(a - b) / bound).max()))
    for sp, f in ZC.items():
        a, b, i = out[f, :, :ncols], ref[f, :, :ncols], fld[f, :, :ncols]
        bound = 1e-3 * np.abs(b - i) + 1e-4 * np.abs(b) + 1e-16 * fld[f].max()
        assert (np.abs(a - b) <= bound).all(), (sp, float((np.abs(a - b) / bound).max()))
        assert (a >= 0).all(), sp


# ------------------------------------- the warm/cold benchmark's state at full size
@pytest.fixture(scope="module")
def stratus_full():
    """The configurations' benchmark state: stratus 512x512 columns x 150 levels."""
    return synth.workload("stratus_512x512x150")


@pytest.mark.parametrize("config", ["warm", "cold_three_moment", "cold_aerosol"])
def test_stratus_512x512x150_sampled_columns(stratus_full, config):
    """Full size, one launch over all 262 144 columns, mixed form: 64 seeded
    random columns and the last one against the oracle (warm configuration;
    cold configuration with triple-moment r, i, s, g; cold configuration
    with aerosol mass)."""
    fld16, dz, ncols, nlev, dt, _ = stratus_full
    cols = np.concatenate([np.sort(np.random.default_rng(78).choice(ncols - 1, 64, replace=False)), [ncols - 1]])
    n = cols.size
    if config == "warm":
        fld, flags = fld16, casim.CASIM_WARM
    elif config == "cold_aerosol":
        fld = np.zeros((22,) + fld16.shape[1:])
        fld[:16] = fld16
        fld[MA] = 3e-9
        for f, q in ((MAC, "qc"), (MAR, "qr"), (MAI, "qi"), (MAS, "qs"), (MAG, "qg")):
            fld[f] = 1e-5 * fld16[F[q]]
        flags = casim.CASIM_AEROSOL
    else:
        fld = np.zeros((20,) + fld16.shape[1:])
        fld[:16] = fld16
        rng = np.random.default_rng(79)
        for sp in "risg":
            q, nn = fld16[QF[sp]], fld16[NF[sp]]
            ok = (q > 1e-14) & (nn > 0)
            shape = rng.uniform(0.0, 8.0, int(ok.sum()))
            fld[ZC[sp]][ok] = _gamma_g(shape) * (q[ok] / O.param(f"a_{sp}")) ** 2 / nn[ok]
        flags = casim.CASIM_THREE_MOMENT
    out, pr, _ = run_gpu(fld, dz, ncols, dt, precision=casim.CASIM_MIXED, flags=flags)
    sub = np.zeros((fld.shape[0], nlev, 96))
    sub[:, :, :n] = fld[:, :, cols]
    if config == "warm":
        ref, _ = run_oracle(sub, dz, n, dt, warm=True)
    elif config == "cold_aerosol":
        ref, _ = _run_oracle_aero_cold(sub, dz, n, dt, 1)
    else:
        ref, _ = _run_oracle_3m_cold(sub, dz, n, dt, 1)
    got = out[:, :, cols]
    for f in range(13):
        a_, b_, i_ = got[f], ref[f, :, :n], sub[f, :, :n]
        bound = mixed_bound(b_, i_, f, ref[1, :, :n])
        assert (np.abs(a_ - b_) <= bound).all(), (synth.FIELDS[f], float((np.abs(a_ - b_) / bound).max()))
    if config == "cold_aerosol":
        scale = sub[MA:MAG + 1, :, :n].sum(axis=0)
        for f in range(MA, MAG + 1):
            assert (np.abs(got[f] - ref[f, :, :n]) <= 1e-4 * scale + 1e-22).all(), f
    elif config != "warm":
        for sp, f in ZC.items():
            a_, b_, i_ = got[f], ref[f, :, :n], sub[f, :, :n]
            bound = 1e-3 * np.abs(b_ - i_) + 1e-4 * np.abs(b_) + 1e-16 * fld[f].max()
            assert (np.abs(a_ - b_) <= bound).all(), (sp, float((np.abs(a_ - b_) / bound).max()))


# ------------------------- source-term and host entry points, every configuration
EXT_CONFIGS = {
    "warm_aerosol": (lambda n, l, seed: _aero_state(n, l, seed), lambda: casim.CASIM_WARM | casim.CASIM_AEROSOL),
    "cold_aerosol": (lambda n, l, seed: _aero_cold_state(n, l, seed), lambda: casim.CASIM_AEROSOL),
    "warm_three_moment": (lambda n, l, seed: _tri_state(n, l, seed),
                          lambda: casim.CASIM_WARM | casim.CASIM_THREE_MOMENT),
    "cold_three_moment": (lambda n, l, seed: _tri_cold_state(n, l, seed), lambda: casim.CASIM_THREE_MOMENT),
}


@pytest.mark.parametrize("config", list(EXT_CONFIGS))
@pytest.mark.parametrize("precision", [casim.CASIM_FP64, casim.CASIM_MIXED])
@pytest.mark.parametrize("dt", [1.0, 30.0])
def test_extended_tendency_and_host_entry_points(config, precision, dt):
    """The aerosol-mass and triple-moment configurations through the
    source-term mode (state untouched; tend rows 0..12 and 13.. for the fields
    after the inputs, each (x_after - x_before) / dt of the in-place step, bit
    for bit) and the host-buffer entry point (whole-domain and chunked paths,
    bit for bit); dt = 30 s takes the multi-substep sedimentation path."""
    import torch
    make, flags = EXT_CONFIGS[config]
    ncols, nlev = 200, 60
    fld, dz = make(ncols, nlev, 91)
    nf, pitch = fld.shape[0], fld.shape[2]
    out, pr, _ = run_gpu(fld, dz, ncols, dt, precision=precision, flags=flags())
    ctx = casim.casim_init(precision=precision, flags=flags())
    try:
        d = casim.Domain(fld, dz, ncols)
        tend = torch.full((nf - 3, nlev, pitch), float("nan"), dtype=torch.float64, device="cuda")
        casim.casim_step_tendency(ctx, d.state, ncols, nlev, dt, tend)
        rc, fl = casim.casim_get_error(ctx)
        assert rc == 0, (rc, fl)
        f2, p2 = d.numpy()
        assert np.array_equal(f2, fld) and np.array_equal(p2, pr)
        rows = list(range(13)) + list(range(16, nf))
        t = tend.cpu().numpy()[:, :, :ncols]
        assert np.array_equal(t, (out[rows, :, :ncols] - fld[rows, :, :ncols]) / dt)
        # host entry point: pageable (copied whole) and pinned (stepped in place)
        for pinned in (False, True):
            h, hpr, _keep = _host_buffers(fld, pr.shape[0], pinned)
            casim.casim_step_host(ctx, casim.make_state(h, pitch, np.ascontiguousarray(dz), hpr), ncols, nlev, dt)
            assert np.array_equal(h, out) and np.array_equal(hpr, pr), pinned
    finally:
        casim.casim_free(ctx)


EXT_ORACLE = {
    "warm_aerosol": (19, lambda f, n, dz: O.step_aero(f, n, dz, 1.0)[1]),
    "cold_aerosol": (22, lambda f, n, dz: O.step_aero_cold(f, n, dz, 1.0)[1]),
    "warm_three_moment": (17, lambda f, n, dz: O.step_3m(f, n, dz, 1.0)[1]),
    "cold_three_moment": (20, lambda f, n, dz: O.step_3m_cold(f, n, dz, 1.0)[1]),
}


def _clear_ext_state(nf, ncols, nlev, seed):
    """Dry, subsaturated air with no hydrometeor (every point inactive),
    carrying nonzero aerosol masses or sixth moments that describe nothing."""
    rng = np.random.default_rng(seed)
    fld = np.zeros((nf, nlev, ncols))
    T, p = 285.0, 9e4
    fld[F["T"]] = T + rng.uniform(-1, 1, (nlev, ncols))
    fld[F["p"]], fld[F["rho"]] = p, 1.1
    fld[F["qv"]] = 0.6 * O.qsat(O.es_liq(T - 1), p)
    fld[F["na"]] = 1e8
    fld[16:] = 10.0 ** rng.uniform(-14, -9, (nf - 16, nlev, ncols))
    return fld


@pytest.mark.parametrize("config", list(EXT_ORACLE))
@pytest.mark.parametrize("precision", [casim.CASIM_FP64, casim.CASIM_MIXED])
def test_extended_fields_at_inactive_points(config, precision):
    """Inactive points keep every field, the aerosol masses and sixth moments
    included, as the oracle has them; a non-finite value in any of those
    fields at an inactive point sets the non-finite error bit."""
    nf, ostep = EXT_ORACLE[config]
    _, flags = EXT_CONFIGS[config]
    ncols, nlev = 64, 20
    dz = np.full(nlev, 100.0)
    fld = _clear_ext_state(nf, ncols, nlev, seed=7)
    out, pr, _ = run_gpu(fld, dz, ncols, 1.0, precision=precision, flags=flags())
    ref = fld.copy()
    assert ostep(ref, ncols, dz) == 0
    assert np.array_equal(ref, fld)          # the oracle leaves the clear domain as it is
    assert np.array_equal(out, ref) and not pr.any()
    for f in range(16, nf):
        bad = fld.copy()
        bad[f, 11, 37] = float("nan")
        _, _, (rc, fl) = run_gpu(bad, dz, ncols, 1.0, precision=precision, flags=flags(), check_err=False)
        assert rc == -4 and fl & casim.EFLAG_NONFINITE, (config, f)


def test_extended_host_entry_point_in_chunks():
    """More columns than one host chunk (65 536): the chunked pipeline moves
    every field of the extended state, bit for bit against the device step."""
    for config in ("cold_aerosol", "cold_three_moment"):
        make, flags = EXT_CONFIGS[config]
        ncols, nlev = 70_000, 12
        fld, dz = make(ncols, nlev, 92)
        out, pr, _ = run_gpu(fld, dz, ncols, 1.0, precision=casim.CASIM_MIXED, flags=flags())
        ctx = casim.casim_init(precision=casim.CASIM_MIXED, flags=flags())
        try:
            h = np.ascontiguousarray(fld.copy())
            hpr = np.zeros(pr.shape)
            casim.casim_step_host(ctx, casim.make_state(h, fld.shape[2], np.ascontiguousarray(dz), hpr),
                                  ncols, nlev, 1.0)
            assert np.array_equal(h, out) and np.array_equal(hpr, pr), config
        finally:
            casim.casim_free(ctx)


# ------------------------------------------------------------------ checkpoint / resume
@pytest.mark.parametrize("state", ["standard", "aerosol", "three_moment", "three_moment_cold", "aerosol_cold"])
def test_checkpoint_resume_is_bitwise(tmp_path, state):
    """N steps equal k steps, save, load into fresh device memory, N - k steps,
    bit for bit; a checkpoint of other sizes or parameters is refused."""
    ncols, nlev = 97, 150
    if state == "aerosol":
        fld, dz = _aero_state(ncols, nlev, seed=71)
        flags, nf = casim.CASIM_WARM | casim.CASIM_AEROSOL, 19
    elif state == "three_moment":
        fld, dz = _tri_state(ncols, nlev, seed=71)
        flags, nf = casim.CASIM_WARM | casim.CASIM_THREE_MOMENT, 17
    elif state == "three_moment_cold":
        fld, dz = _tri_cold_state(ncols, nlev, seed=71)
        flags, nf = casim.CASIM_THREE_MOMENT, 20
    elif state == "aerosol_cold":
        fld, dz = _aero_cold_state(ncols, nlev, seed=71)
        flags, nf = casim.CASIM_AEROSOL, 22
    else:
        dz = synth.dz_stretched(nlev)
        fld = synth.make_state("deep_convective", ncols, nlev, dz, seed=71)
        flags, nf = 0, 16
    ctx = casim.casim_init(precision=casim.CASIM_MIXED, flags=flags)
    try:
        ref = casim.Domain(fld, dz, ncols)
        for _ in range(6):
            casim.casim_step(ctx, ref.state, ncols, nlev, 1.0)
        a = casim.Domain(fld, dz, ncols)
        for _ in range(3):
            casim.casim_step(ctx, a.state, ncols, nlev, 1.0)
        path = str(tmp_path / "state.ckpt")
        casim.casim_state_save(path, a.state, ncols, nlev, nf)
        b = casim.Domain(np.zeros_like(fld), np.ones_like(dz), ncols)
        casim.casim_state_load(path, b.state, ncols, nlev, nf)
        for _ in range(3):
            casim.casim_step(ctx, b.state, ncols, nlev, 1.0)
        assert casim.casim_get_error(ctx)[0] == 0
        (f1, p1), (f2, p2) = ref.numpy(), b.numpy()
        assert np.array_equal(f1, f2) and np.array_equal(p1, p2)
        assert np.array_equal(b.dz.cpu().numpy(), dz)
        with pytest.raises(RuntimeError):                 # other column count
            casim.casim_state_load(path, b.state, ncols - 1, nlev, nf)
        other = casim.casim_default_params()
        other.c_max = 0.5
        with pytest.raises(RuntimeError):                 # other parameters
            casim.casim_state_load(path, b.state, ncols, nlev, nf, params=other)
        with pytest.raises(RuntimeError):                 # no such file
            casim.casim_state_load(str(tmp_path / "missing"), b.state, ncols, nlev, nf)
    finally:
        casim.casim_free(ctx)


# ------------------------------------------------------------------ failure detection
def test_bounded_wait_gives_up_and_the_context_stays_usable():
    """The tensor-core kernels' bounded wait, run on a barrier nothing
    completes, gives up after its limit and reports it through the error
    word (no fault, no hang); the same context then steps normally."""
    fld, dz, ncols, nlev, dt, _ = synth.workload("stratus_16x16x50")
    ctx = casim.casim_init(precision=casim.CASIM_MIXED)
    try:
        el = casim.casim_wait_selftest(ctx, 20_000_000)
        assert 20_000_000 <= el < 1_000_000_000, el
        rc, flags = casim.casim_get_error(ctx)
        assert rc == -6 and flags & casim.EFLAG_TIMEOUT, (rc, flags)
        assert casim.casim_get_error(ctx)[0] == 0                 # read and cleared
        d = casim.Domain(fld, dz, ncols)
        casim.casim_step(ctx, d.state, ncols, nlev, dt)
        assert casim.casim_get_error(ctx)[0] == 0
        out, pr = d.numpy()
    finally:
        casim.casim_free(ctx)
    ref, pref, _ = run_gpu(fld, dz, ncols, dt, precision=casim.CASIM_MIXED)
    assert np.array_equal(out, ref) and np.array_equal(pr, pref)
    with pytest.raises(RuntimeError):
        ctx = casim.casim_init(precision=casim.CASIM_MIXED)
        try:
            casim.casim_wait_selftest(ctx, 3_000_000_000)            # beyond the kernels' own limit
        finally:
            casim.casim_free(ctx)


# ---------------------------------------- hand-made regimes, one per column
def _regime_domain(nf, regimes, nlev=12, reps=3):
    """A domain whose columns hold the given point states at every level
    (each regime in `reps` neighbouring columns, the temperature nudged by
    0.01 K per copy), pitch a multiple of 32."""
    ncols = reps * len(regimes)
    pitch = (ncols + 31) // 32 * 32
    fld = np.zeros((nf, nlev, pitch))
    for i, reg in enumerate(regimes):
        for r in range(reps):
            c = reps * i + r
            for k, v in reg.items():
                fld[k, :, c] = v
            fld[F["T"], :, c] += 0.01 * r
    # padding columns: clear, subsaturated air
    fld[F["T"], :, ncols:], fld[F["p"], :, ncols:], fld[F["rho"], :, ncols:] = 280.0, 8e4, 1.0
    return np.ascontiguousarray(fld), np.full(nlev, 100.0), ncols


def _pt(T, p, extra=None, **kw):
    """One point state: T, p, rho = p / (R_d T), the named fields of the
    standard layout, and `extra` {field index: value} for the fields after
    the inputs."""
    st = {F["T"]: T, F["p"]: p, F["rho"]: p / (287.04 * T), F["na"]: 1e8}
    for k, v in kw.items():
        st[F[k]] = v
    st.update(extra or {})
    return st


def _qsl(T, p):
    return O.qsat(O.es_liq(T), p)


def _qsi(T, p):
    return O.qsat(O.es_ice(T), p)


@pytest.mark.parametrize("precision", [casim.CASIM_FP64, casim.CASIM_MIXED])
@pytest.mark.parametrize("dt", [1.0, 5.0])
def test_hand_made_regimes(dt, precision):
    """The regimes the oracle's hand-made pins single out, each in its own
    columns, against the oracle.  FP64 form: 13 fields and the precipitation
    rows within 1e-12, aerosol masses within 1e-12 of the point's total
    aerosol, sixth moments within 1e-12 of the largest.  Mixed form: the 13
    fields within the derived mixed bound, aerosol masses within 1e-4 of the
    point's total aerosol, sixth moments within 1e-3 of their change plus 1e-4
    of their value (the bounds of the configurations' own mixed tests).
    The regimes:
    snow, ice and graupel falling at ice saturation (each species' own
    precipitation row); Meyers nucleation at S_i = 1.1; rain in air
    supersaturated over water; partial evaporation of cloud holding aerosol;
    cloud collected at once by rain and graupel, with aerosol; nucleation just
    above ice saturation and snow melting into existing rain with
    triple-moment species."""
    std = [_pt(250.0, 7e4, qv=_qsi(250.0, 7e4), qi=1e-5, ni=1e5, qs=1e-4, ns=1e4, qg=3e-4, ng=2e3),
           _pt(263.15, 6e4, qv=1.1 * _qsi(263.15, 6e4)),
           _pt(285.0, 9e4, qv=1.05 * _qsl(285.0, 9e4), qr=2e-4, nr=1e3)]
    aero_warm = [_pt(285.0, 9e4, qv=0.96 * _qsl(285.0, 9e4), qc=1e-3, nc=1e8, extra={MA: 2e-9, MAC: 3e-9}),
                 _pt(285.0, 9e4, qv=0.99 * _qsl(285.0, 9e4), qc=1e-3, nc=1e8, qr=2e-4, nr=1e3,
                     extra={MA: 2e-9, MAC: 3e-9, MAR: 1e-9})]
    aero_cold = [_pt(263.0, 7e4, qv=_qsl(263.0, 7e4), qc=5e-4, nc=1e8, qr=2e-4, nr=1e3, qg=1e-3, ng=1e3,
                     extra={MA: 1e-9, MAC: 4e-9, MAR: 1e-9, 21: 2e-9})]
    a = casim.casim_default_params().a

    def z_at(x, q, n, mu):
        return _gamma_g(mu) * (q / a[1 + x]) ** 2 / n
    tri_cold = [_pt(255.0, 5e4, qv=1.005 * _qsi(255.0, 5e4)),
                _pt(276.0, 9e4, qv=_qsl(276.0, 9e4), qr=3e-4, nr=2e3, qs=2e-4, ns=5e3,
                    extra={ZC["r"]: z_at(0, 3e-4, 2e3, 1.0), ZC["s"]: z_at(2, 2e-4, 5e3, 4.0)})]
    cases = [(16, std, 0, lambda f, n, dz: O.step(f, n, dz, dt)),
             (19, aero_warm, casim.CASIM_WARM | casim.CASIM_AEROSOL, lambda f, n, dz: O.step_aero(f, n, dz, dt)),
             (22, aero_cold, casim.CASIM_AEROSOL, lambda f, n, dz: O.step_aero_cold(f, n, dz, dt)),
             (20, tri_cold, casim.CASIM_THREE_MOMENT, lambda f, n, dz: O.step_3m_cold(f, n, dz, dt))]
    for nf, regimes, flags, ostep in cases:
        fld, dz, ncols = _regime_domain(nf, regimes)
        out, pr, _ = run_gpu(fld, dz, ncols, dt, precision=precision, flags=flags)
        ref = fld.copy()
        res = ostep(ref, ncols, dz)
        assert res[-1] == 0
        pref = res[0]
        assert not np.array_equal(ref[:13, :, :ncols], fld[:13, :, :ncols])     # the regimes do act
        if precision == casim.CASIM_MIXED:
            for f in range(13):
                a_, b_, i_ = out[f, :, :ncols], ref[f, :, :ncols], fld[f, :, :ncols]
                bound = mixed_bound(b_, i_, f, ref[1, :, :ncols])
                assert (np.abs(a_ - b_) <= bound).all(), (nf, synth.FIELDS[f], float((np.abs(a_ - b_) / bound).max()))
            if nf in (19, 22):
                scale = fld[MA:nf, :, :ncols].sum(axis=0)
                assert (np.abs(out[MA:nf, :, :ncols] - ref[MA:nf, :, :ncols]) <= 1e-4 * scale + 1e-22).all(), nf
            if nf == 20:
                a_, b_, i_ = out[16:20, :, :ncols], ref[16:20, :, :ncols], fld[16:20, :, :ncols]
                bound = 1e-3 * np.abs(b_ - i_) + 1e-4 * np.abs(b_) + 1e-16 * np.abs(fld[16:20]).max()
                assert (np.abs(a_ - b_) <= bound).all(), float((np.abs(a_ - b_) / bound).max())
            continue
        assert_fp64_close(out, pr[:4], ref, pref[:4], ncols)
        if nf in (19, 22):
            hi = 19 if nf == 19 else 22
            scale = fld[MA:hi, :, :ncols].sum(axis=0)
            for f in range(MA, hi):
                d = np.abs(out[f, :, :ncols] - ref[f, :, :ncols])
                assert (d <= RTOL64 * np.maximum(np.abs(ref[f, :, :ncols]), scale)).all(), (nf, f, float(d.max()))
            assert np.all(np.abs(pr[4, :ncols] - pref[4, :ncols]) <= RTOL64 * np.abs(pref[4, :ncols]) + 1e-26)
        if nf == 20:
            zmax = np.abs(ref[16:20, :, :ncols]).max()
            d = np.abs(out[16:20, :, :ncols] - ref[16:20, :, :ncols])
            assert (d <= RTOL64 * np.abs(ref[16:20, :, :ncols]) + 1e-12 * zmax).all(), float(d.max())
