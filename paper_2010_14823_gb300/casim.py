"""Python binding of the C ABI in include/casim.h (ctypes; marshalling only).

Each function has the C entry point's name and forwards its arguments: torch
CUDA tensors are passed as device pointers, torch streams as cudaStream_t.
Every step of the computation runs in libcasim.so; there is no fallback.  If
the library has not been built, loading fails with an error naming the
build command.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from .build import LIB, LIB_DEBUG, INCLUDE

CASIM_FP64 = 0
CASIM_MIXED = 1
CASIM_WARM = 1          # casim_init flag: the warm configuration
CASIM_AEROSOL = 2       # casim_init flag: activated-aerosol mass (with CASIM_WARM 19 fields, else 22), 5 precip rows
CASIM_THREE_MOMENT = 4  # casim_init flag: triple-moment rain (with CASIM_WARM, 17 fields) or r, i, s, g (20 fields)
NFIELDS_AERO = 19
NFIELDS_3MOM = 17
NFIELDS_3MOM_COLD = 20
NFIELDS_AERO_COLD = 22
CASIM_MAX_LEV = 1024   # largest level count of a column
NFIELDS = 16
NPROG = 13
NPRECIP = 4
NSUB_MAX = 64
EFLAG_NONFINITE = 1
EFLAG_CFL = 2
EFLAG_TIMEOUT = 4
EFLAG_INDEX = 8         # the debug build (libcasim_debug.so): an index check failed
CASIM_STATS = 8         # casim_init flag: per-step statistics (casim_get_stats)
NOALLOC_MAX_COLS = 1 << 20
_ERRORS = {-1: "CASIM_ERR_ARG", -2: "CASIM_ERR_OOM", -3: "CASIM_ERR_CUDA",
           -4: "CASIM_ERR_NONFINITE", -5: "CASIM_ERR_CFL", -6: "CASIM_ERR_TIMEOUT", -7: "CASIM_ERR_IO",
           -8: "CASIM_ERR_INDEX"}


class CasimError(RuntimeError):
    def __init__(self, code: int, where: str, detail: str = ""):
        self.code = code
        super().__init__(f"{where}: {_ERRORS.get(code, code)}{(' (' + detail + ')') if detail else ''}")


_D = ctypes.c_double
_SCALARS = ("T0 cp Lv Lf Rd Rv g rho_w rho0 Ka Dv mu_air q_min T_nuc m_i0 r_r0 kk_aut kk_aut_qc kk_aut_nc "
            "nc_min_cm3 kk_acc kk_acc_exp kc_sb nu_c kr_sb mey_a mey_b mey_c arg_rm arg_sigma arg_kappa surft "
            "Mw Ma Rgas e_rim c_max es_l0 es_la es_lb es_i0 es_ia es_it es_ib").split()
_ARRAYS = "a b mu cv dv vmax dmin dmax ccap".split()


class casim_params(ctypes.Structure):
    _fields_ = [(n, _D) for n in _SCALARS] + [(n, _D * 5) for n in _ARRAYS]

    def as_dict(self) -> dict:
        d = {n: getattr(self, n) for n in _SCALARS}
        for n in _ARRAYS:
            d[n] = list(getattr(self, n))
        return d


class casim_state(ctypes.Structure):
    _fields_ = [("fld", ctypes.c_void_p), ("pitch", ctypes.c_longlong),
                ("dz", ctypes.c_void_p), ("precip", ctypes.c_void_p)]


class casim_stats(ctypes.Structure):
    _fields_ = [("steps", ctypes.c_longlong), ("points", ctypes.c_longlong), ("active_points", ctypes.c_longlong),
                ("changed_points", ctypes.c_longlong), ("active_columns", ctypes.c_longlong),
                ("nsub", (ctypes.c_longlong * 65) * 4)]


class casim_tune_entry(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int), ("compact", ctypes.c_int), ("persistent", ctypes.c_int),
                ("ms_per_step", ctypes.c_float)]


_lib = None


def library_path() -> str:
    """The library this process uses: libcasim.so, or its index-checked build
    libcasim_debug.so when the environment sets CASIM_LIBRARY=debug."""
    return LIB_DEBUG if os.environ.get("CASIM_LIBRARY", "") == "debug" else LIB


def lib():
    """Load the library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        L = bind(ctypes.CDLL(path))
        _lib = L
    return _lib


def bind(L):
    """Declare the argument and result types of a loaded library's entry points."""
    vp, i, d, u = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_uint
    ps = ctypes.POINTER(casim_state)
    L.casim_default_params.argtypes = [ctypes.POINTER(casim_params)]
    L.casim_default_params.restype = i
    L.casim_init.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(casim_params), i, i]
    L.casim_init.restype = i
    L.casim_step.argtypes = [vp, ps, i, i, d, vp]
    L.casim_step.restype = i
    L.casim_step_tendency.argtypes = [vp, ps, i, i, d, vp, vp]
    L.casim_step_tendency.restype = i
    L.casim_step_host.argtypes = [vp, ps, i, i, d, vp]
    L.casim_step_host.restype = i
    L.casim_budget.argtypes = [vp, ps, i, i, vp, vp]
    for name in ("casim_state_save", "casim_state_load"):
        getattr(L, name).argtypes = [ctypes.c_char_p, ctypes.c_void_p, ps, i, i, i, vp]
        getattr(L, name).restype = i
    L.casim_budget.restype = i
    L.casim_get_error.argtypes = [vp, ctypes.POINTER(u), vp]
    L.casim_wait_selftest.argtypes = [vp, ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong), vp]
    L.casim_wait_selftest.restype = i
    L.casim_get_error.restype = i
    L.casim_launch_count.argtypes = [vp]
    L.casim_launch_count.restype = ctypes.c_longlong
    L.casim_last_cuda_error.argtypes = []
    L.casim_last_cuda_error.restype = ctypes.c_char_p
    L.casim_free.argtypes = [vp]
    L.casim_free.restype = None
    L.casim_abi_version.argtypes = []
    L.casim_abi_version.restype = i
    pi = ctypes.POINTER(i)
    L.casim_batch_create.argtypes = [vp, ps, pi, pi, i, ctypes.POINTER(vp)]
    L.casim_batch_create.restype = i
    L.casim_batch_step.argtypes = [vp, vp, d, vp]
    L.casim_batch_step.restype = i
    L.casim_step_batched.argtypes = [vp, ps, pi, pi, i, d, vp]
    L.casim_step_batched.restype = i
    L.casim_batch_config.argtypes = [vp, i, i, i]
    L.casim_batch_config.restype = i
    L.casim_batch_get_config.argtypes = [vp, pi, pi, pi]
    L.casim_batch_get_config.restype = i
    L.casim_batch_tune.argtypes = [vp, vp, d, i, vp, ctypes.POINTER(casim_tune_entry), i]
    L.casim_batch_tune.restype = i
    L.casim_batch_tune_steps.argtypes = [i]
    L.casim_batch_tune_steps.restype = i
    L.casim_batch_graph.argtypes = [vp, vp, d, i, vp]
    L.casim_batch_graph.restype = i
    L.casim_batch_graph_launch.argtypes = [vp, vp]
    L.casim_batch_graph_launch.restype = i
    L.casim_batch_columns.argtypes = [vp]
    L.casim_batch_columns.restype = ctypes.c_longlong
    L.casim_batch_free.argtypes = [vp]
    L.casim_batch_free.restype = None
    L.casim_step_noalloc.argtypes = [ctypes.POINTER(casim_params), i, ps, i, i, d, vp, ctypes.POINTER(u)]
    L.casim_step_noalloc.restype = i
    pf = ctypes.POINTER(ctypes.c_float)
    ll = ctypes.c_longlong
    L.casim_mlp_create.argtypes = [ctypes.POINTER(vp), ctypes.c_ulonglong]
    L.casim_mlp_create.restype = i
    L.casim_mlp_param_count.argtypes = []
    L.casim_mlp_param_count.restype = ll
    L.casim_mlp_set_params.argtypes = [vp, pf, ll]
    L.casim_mlp_set_params.restype = i
    L.casim_mlp_get_params.argtypes = [vp, pf, ll]
    L.casim_mlp_get_params.restype = i
    L.casim_mlp_forward_host.argtypes = [vp, pf, i, pf]
    L.casim_mlp_forward_host.restype = i
    L.casim_mlp_forward.argtypes = [vp, vp, ctypes.c_longlong, vp, vp]
    L.casim_mlp_forward.restype = i
    L.casim_mlp_loss_grad_host.argtypes = [vp, pf, pf, pf, i, ctypes.POINTER(d), pf]
    L.casim_mlp_loss_grad_host.restype = i
    L.casim_mlp_data.argtypes = [vp, ps, i, i, d, vp, vp, vp, vp, ll, ctypes.POINTER(ll), vp]
    L.casim_mlp_data.restype = i
    L.casim_mlp_fit.argtypes = [vp, vp, vp, vp, ll, i, i, ctypes.c_float, ctypes.c_ulonglong, pf, vp]
    L.casim_mlp_fit.restype = i
    L.casim_mlp_get_norm.argtypes = [vp, pf]
    L.casim_mlp_get_norm.restype = i
    L.casim_mlp_set_norm.argtypes = [vp, pf]
    L.casim_mlp_set_norm.restype = i
    L.casim_step_surrogate.argtypes = [vp, vp, ps, i, i, d, vp, ctypes.POINTER(ll)]
    L.casim_step_surrogate.restype = i
    L.casim_batch_step_surrogate.argtypes = [vp, vp, vp, d, vp, ctypes.POINTER(ll)]
    L.casim_batch_step_surrogate.restype = i
    L.casim_mlp_set_engine.argtypes = [vp, i]
    L.casim_mlp_set_engine.restype = i
    L.casim_mlp_free.argtypes = [vp]
    L.casim_mlp_free.restype = None
    L.casim_get_stats.argtypes = [vp, ctypes.POINTER(casim_stats), i, vp]
    L.casim_get_stats.restype = i
    return L


def declared_functions(header: str | None = None) -> list[str]:
    """Names of the functions declared in include/*.h (or in one header)."""
    names = []
    for f in sorted(os.listdir(INCLUDE)):
        if f.endswith(".h") and (header is None or f == header):
            text = open(os.path.join(INCLUDE, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^[A-Za-z_][\w \*]*?\b(casim_\w+)\s*\(", text, flags=re.M)
    return names


def _check(rc: int, where: str):
    if rc != 0:
        detail = lib().casim_last_cuda_error().decode() if rc == -3 else ""
        raise CasimError(rc, where, detail)


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return x.data_ptr()   # torch tensor


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def casim_default_params() -> casim_params:
    p = casim_params()
    _check(lib().casim_default_params(ctypes.byref(p)), "casim_default_params")
    return p


def casim_init(params: casim_params | None = None, precision: int = CASIM_FP64, flags: int = 0):
    ctx = ctypes.c_void_p()
    _check(lib().casim_init(ctypes.byref(ctx), ctypes.byref(params) if params is not None else None,
                            precision, flags), "casim_init")
    return ctx


def make_state(fld, pitch: int, dz, precip) -> casim_state:
    return casim_state(_ptr(fld), int(pitch), _ptr(dz), _ptr(precip))


def casim_step(ctx, state: casim_state, ncols: int, nlev: int, dt: float, stream=None):
    _check(lib().casim_step(ctx, ctypes.byref(state), ncols, nlev, dt, _stream(stream)), "casim_step")


def casim_step_tendency(ctx, state: casim_state, ncols: int, nlev: int, dt: float, tend, stream=None):
    """Source-term mode: state unchanged, tend [13][nlev][pitch] (device) = (x_after - x_before) / dt."""
    _check(lib().casim_step_tendency(ctx, ctypes.byref(state), ncols, nlev, dt, _ptr(tend), _stream(stream)),
           "casim_step_tendency")


def casim_wait_selftest(ctx, limit_ns: int, stream=None) -> int:
    """Run the kernels' bounded wait on a barrier nothing completes; returns
    how long it waited (ns).  The give-up is left in the error word."""
    el = ctypes.c_longlong(0)
    _check(lib().casim_wait_selftest(ctx, limit_ns, ctypes.byref(el), _stream(stream)), "casim_wait_selftest")
    return el.value


def casim_step_host(ctx, state: casim_state, ncols: int, nlev: int, dt: float, stream=None):
    _check(lib().casim_step_host(ctx, ctypes.byref(state), ncols, nlev, dt, _stream(stream)), "casim_step_host")


def casim_budget(ctx, state: casim_state, ncols: int, nlev: int, out, stream=None):
    _check(lib().casim_budget(ctx, ctypes.byref(state), ncols, nlev, _ptr(out), _stream(stream)), "casim_budget")


def casim_state_save(path: str, state: casim_state, ncols: int, nlev: int, nfields: int = NFIELDS, params=None,
                     stream=None):
    """Checkpoint a domain's device state (dz, fields, precip) to a file."""
    _check(lib().casim_state_save(path.encode(), ctypes.byref(params) if params is not None else None,
                                  ctypes.byref(state), ncols, nlev, nfields, _stream(stream)), "casim_state_save")


def casim_state_load(path: str, state: casim_state, ncols: int, nlev: int, nfields: int = NFIELDS, params=None,
                     stream=None):
    """Restore a checkpoint into a domain's device arrays (same sizes and parameters)."""
    _check(lib().casim_state_load(path.encode(), ctypes.byref(params) if params is not None else None,
                                  ctypes.byref(state), ncols, nlev, nfields, _stream(stream)), "casim_state_load")


def casim_get_error(ctx, stream=None) -> tuple[int, int]:
    """Returns (status, flags); status is 0 or a negative CASIM_ERR_* code."""
    f = ctypes.c_uint(0)
    rc = lib().casim_get_error(ctx, ctypes.byref(f), _stream(stream))
    if rc == -3:
        _check(rc, "casim_get_error")
    return rc, f.value


def casim_get_stats(ctx, reset: bool = False, stream=None) -> dict:
    """Statistics of a CASIM_STATS context (waits for the stream)."""
    st = casim_stats()
    _check(lib().casim_get_stats(ctx, ctypes.byref(st), int(reset), _stream(stream)), "casim_get_stats")
    return {"steps": st.steps, "points": st.points, "active_points": st.active_points,
            "changed_points": st.changed_points, "active_columns": st.active_columns,
            "nsub": np.array([[st.nsub[x][n] for n in range(65)] for x in range(4)], dtype=np.int64)}


def casim_launch_count(ctx) -> int:
    return lib().casim_launch_count(ctx)


def casim_free(ctx):
    lib().casim_free(ctx)


def casim_abi_version() -> int:
    return lib().casim_abi_version()


def casim_batch_create(ctx, states, ncols, nlev):
    """states: list of casim_state (device); ncols, nlev: lists of ints."""
    n = len(states)
    arr = (casim_state * n)(*states)
    nc = (ctypes.c_int * n)(*ncols)
    nl = (ctypes.c_int * n)(*nlev)
    b = ctypes.c_void_p()
    _check(lib().casim_batch_create(ctx, arr, nc, nl, n, ctypes.byref(b)), "casim_batch_create")
    return b


def casim_batch_step(ctx, batch, dt: float, stream=None):
    _check(lib().casim_batch_step(ctx, batch, dt, _stream(stream)), "casim_batch_step")


def casim_step_batched(ctx, states, ncols, nlev, dt: float, stream=None):
    """One step of many domains (the context keeps the batch of the last list)."""
    n = len(states)
    arr = (casim_state * n)(*states)
    nc = (ctypes.c_int * n)(*ncols)
    nl = (ctypes.c_int * n)(*nlev)
    _check(lib().casim_step_batched(ctx, arr, nc, nl, n, dt, _stream(stream)), "casim_step_batched")


def casim_batch_config(batch, block: int, compact: int, persistent: int):
    _check(lib().casim_batch_config(batch, block, compact, persistent), "casim_batch_config")


def casim_batch_get_config(batch) -> tuple[int, int, int]:
    b, c, p = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().casim_batch_get_config(batch, ctypes.byref(b), ctypes.byref(c), ctypes.byref(p)),
           "casim_batch_get_config")
    return b.value, c.value, p.value


def casim_batch_tune(ctx, batch, dt: float, steps: int = 2, stream=None) -> list[dict]:
    table = (casim_tune_entry * 12)()
    _check(lib().casim_batch_tune(ctx, batch, dt, steps, _stream(stream), table, 12), "casim_batch_tune")
    return [{"block": e.block, "compact": e.compact, "persistent": e.persistent, "ms_per_step": e.ms_per_step}
            for e in table]


def casim_batch_tune_steps(steps: int) -> int:
    return lib().casim_batch_tune_steps(steps)


def casim_batch_graph(ctx, batch, dt: float, nsteps: int, stream=None):
    _check(lib().casim_batch_graph(ctx, batch, dt, nsteps, _stream(stream)), "casim_batch_graph")


def casim_batch_graph_launch(batch, stream=None):
    _check(lib().casim_batch_graph_launch(batch, _stream(stream)), "casim_batch_graph_launch")


def casim_batch_columns(batch) -> int:
    return lib().casim_batch_columns(batch)


def casim_batch_free(batch):
    lib().casim_batch_free(batch)


class Domain:
    """A domain's device state as torch tensors, in the layout of include/casim.h."""

    def __init__(self, fld, dz: np.ndarray, ncols: int, device="cuda"):
        """fld: host array [16][nlev][pitch] (copied to the device) or a device
        tensor of that shape (cloned); 19 fields for the activated-aerosol
        state, whose precip then has 5 rows."""
        import torch
        nf, nlev, pitch = fld.shape
        assert nf in (NFIELDS, NFIELDS_3MOM, NFIELDS_AERO, NFIELDS_3MOM_COLD, NFIELDS_AERO_COLD)
        assert pitch % 32 == 0 and pitch >= ncols
        self.ncols, self.nlev, self.pitch = ncols, nlev, pitch
        if isinstance(fld, torch.Tensor):
            assert fld.dtype == torch.float64
            self.fld = fld.detach().clone().contiguous()
        else:
            self.fld = torch.from_numpy(np.ascontiguousarray(fld)).to(device)
        assert self.fld.data_ptr() % 256 == 0
        self.dz = torch.from_numpy(np.ascontiguousarray(dz, dtype=np.float64)).to(device)
        nrows = NPRECIP + (nf in (NFIELDS_AERO, NFIELDS_AERO_COLD))
        self.precip = torch.zeros((nrows, pitch), dtype=torch.float64, device=device)
        self.state = make_state(self.fld, pitch, self.dz, self.precip)

    def numpy(self):
        return self.fld.cpu().numpy(), self.precip.cpu().numpy()


def casim_step_noalloc(params, precision: int, state: casim_state, ncols: int, nlev: int, dt: float,
                       stream=None, want_flags: bool = True) -> tuple[int, int]:
    """One step without any device allocation (scratch is a fixed array in the
    library).  Returns (status, flags); with want_flags the call waits for the
    stream and reports this step's error bits."""
    f = ctypes.c_uint(0)
    rc = lib().casim_step_noalloc(ctypes.byref(params) if params is not None else None, precision,
                                  ctypes.byref(state), ncols, nlev, dt, _stream(stream),
                                  ctypes.byref(f) if want_flags else None)
    if rc in (-1, -3):
        _check(rc, "casim_step_noalloc")
    return rc, f.value


MLP_NIN = 12
MLP_NOUT = 4
MLP_NSTATS = 2 * 12 + 2 * 4 + 2 * 12


def _fp(a: np.ndarray):
    assert a.dtype == np.float32 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def casim_mlp_create(seed: int = 0):
    m = ctypes.c_void_p()
    _check(lib().casim_mlp_create(ctypes.byref(m), seed), "casim_mlp_create")
    return m


def casim_mlp_param_count() -> int:
    return lib().casim_mlp_param_count()


def casim_mlp_set_params(mlp, theta: np.ndarray):
    t = np.ascontiguousarray(theta, dtype=np.float32)
    _check(lib().casim_mlp_set_params(mlp, _fp(t), t.size), "casim_mlp_set_params")


def casim_mlp_get_params(mlp) -> np.ndarray:
    t = np.zeros(casim_mlp_param_count(), dtype=np.float32)
    _check(lib().casim_mlp_get_params(mlp, _fp(t), t.size), "casim_mlp_get_params")
    return t


def casim_mlp_forward_host(mlp, Xn: np.ndarray) -> np.ndarray:
    X = np.ascontiguousarray(Xn, dtype=np.float32)
    Y = np.zeros((X.shape[0], MLP_NOUT), dtype=np.float32)
    _check(lib().casim_mlp_forward_host(mlp, _fp(X), X.shape[0], _fp(Y)), "casim_mlp_forward_host")
    return Y


def casim_mlp_forward(mlp, Xn, Y, stream=None):
    """Xn: device float32 tensor [n][12] (standardised inputs); Y: device
    float32 tensor [n][4], written.  Synchronises the stream."""
    import torch
    assert Xn.is_cuda and Y.is_cuda and Xn.dtype == torch.float32 and Y.dtype == torch.float32
    assert Xn.is_contiguous() and Y.is_contiguous() and Xn.shape[1] == MLP_NIN and Y.shape == (Xn.shape[0], MLP_NOUT)
    _check(lib().casim_mlp_forward(mlp, Xn.data_ptr(), Xn.shape[0], Y.data_ptr(), _stream(stream)),
           "casim_mlp_forward")


def casim_mlp_loss_grad_host(mlp, Xn, Tn, M):
    X = np.ascontiguousarray(Xn, dtype=np.float32)
    T = np.ascontiguousarray(Tn, dtype=np.float32)
    Mk = np.ascontiguousarray(M, dtype=np.float32)
    g = np.zeros(casim_mlp_param_count(), dtype=np.float32)
    loss = ctypes.c_double(0.0)
    _check(lib().casim_mlp_loss_grad_host(mlp, _fp(X), _fp(T), _fp(Mk), X.shape[0], ctypes.byref(loss), _fp(g)),
           "casim_mlp_loss_grad_host")
    return loss.value, g


def casim_mlp_data(ctx, state: casim_state, ncols: int, nlev: int, dt: float, X, Y, M, cap: int, pts=None,
                   stream=None) -> int:
    rows = ctypes.c_longlong(0)
    _check(lib().casim_mlp_data(ctx, ctypes.byref(state), ncols, nlev, dt, _ptr(X), _ptr(Y), _ptr(M), _ptr(pts),
                                cap, ctypes.byref(rows), _stream(stream)), "casim_mlp_data")
    return rows.value


def casim_mlp_fit(mlp, X, Y, M, n: int, steps: int, batch: int, lr: float, seed: int = 0, stream=None,
                  history: bool = True) -> np.ndarray | None:
    hist = np.zeros(max(steps, 1), dtype=np.float32) if history else None
    _check(lib().casim_mlp_fit(mlp, _ptr(X), _ptr(Y), _ptr(M), n, steps, batch, lr, seed,
                               _fp(hist) if history else None, _stream(stream)), "casim_mlp_fit")
    return hist[:steps] if history else None


def casim_mlp_get_norm(mlp) -> np.ndarray:
    st = np.zeros(MLP_NSTATS, dtype=np.float32)
    _check(lib().casim_mlp_get_norm(mlp, _fp(st)), "casim_mlp_get_norm")
    return st


def casim_mlp_set_norm(mlp, stats: np.ndarray):
    st = np.ascontiguousarray(stats, dtype=np.float32)
    assert st.size == MLP_NSTATS
    _check(lib().casim_mlp_set_norm(mlp, _fp(st)), "casim_mlp_set_norm")


def casim_step_surrogate(ctx, mlp, state: casim_state, ncols: int, nlev: int, dt: float, stream=None) -> int:
    served = ctypes.c_longlong(0)
    _check(lib().casim_step_surrogate(ctx, mlp, ctypes.byref(state), ncols, nlev, dt, _stream(stream),
                                      ctypes.byref(served)), "casim_step_surrogate")
    return served.value


def casim_batch_step_surrogate(ctx, batch, mlp, dt: float, stream=None, want_served: bool = False) -> int | None:
    """One surrogate step of every domain of a batch; with want_served the call
    waits for the stream and returns the points that took the network's rates."""
    served = ctypes.c_longlong(0)
    _check(lib().casim_batch_step_surrogate(ctx, batch, mlp, dt, _stream(stream),
                                            ctypes.byref(served) if want_served else None),
           "casim_batch_step_surrogate")
    return served.value if want_served else None


def casim_mlp_free(mlp):
    lib().casim_mlp_free(mlp)


def casim_mlp_set_engine(mlp, engine: int):
    """1: tcgen05 inference kernel (default), 0: mma.sync GEMMs."""
    _check(lib().casim_mlp_set_engine(mlp, engine), "casim_mlp_set_engine")
