"""FP64 CPU oracle of the column microphysics step -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  It wraps ``casim_oracle.c`` (plain C, compiled
with ``-ffp-contract=off``) through ctypes and shares no code with the CUDA
path.  See ``casim_oracle.c`` for the scheme and the parameterisation each
function follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "casim_oracle.c")
_LIB = os.path.join(_HERE, "libcasim_oracle.so")

NFIELDS = 16
NPROG = 13
NFIELDS_AERO = 19      # + free aerosol mass, aerosol mass in cloud, in rain
NPROG_AERO = 16
NFIELDS_3M = 17        # + the rain's sixth moment
NPROG_3M = 14
NFIELDS_3MC = 20       # cold configuration: + the sixth moments of r, i, s, g
NFIELDS_AEROC = 22     # cold configuration: + aerosol mass free, in c, r, i, s, g
NPROG_AEROC = 19
NPROG_3MC = 17
NPROC = 14
SPECIES = {"c": 0, "r": 1, "i": 2, "s": 3, "g": 4}
PROCS = ("aut", "acc", "scc", "scr", "evr", "nuc", "depi", "deps", "depg",
         "rims", "rimg", "mlti", "mlts", "mltg")
ERR_NONFINITE = 1
ERR_CFL = 2
NSUB_MAX = 64


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "casim_oracle.h"))):
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
               "-shared", "-std=c11", "-o", _LIB, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        d, pd, i, u = ctypes.c_double, ctypes.POINTER(ctypes.c_double), ctypes.c_int, ctypes.c_uint
        for name in ("orc_es_liq", "orc_es_ice", "orc_arg_sm"):
            getattr(L, name).restype = d
            getattr(L, name).argtypes = [d]
        L.orc_qsat.restype = d
        L.orc_qsat.argtypes = [d, d]
        L.orc_dqsat_liq_dT.restype = d
        L.orc_dqsat_liq_dT.argtypes = [d, d]
        L.orc_satadj.restype = None
        L.orc_satadj.argtypes = [d, pd, pd, pd]
        for name in ("orc_arg_smax", "orc_arg_nact"):
            getattr(L, name).restype = d
            getattr(L, name).argtypes = [d, d, d, d]
        L.orc_lambda.restype = d
        L.orc_lambda.argtypes = [i, d, d]
        L.orc_moment.restype = d
        L.orc_moment.argtypes = [i, d, d, d, d]
        L.orc_vent_integral.restype = d
        L.orc_vent_integral.argtypes = [i, d, d, d]
        for name in ("orc_vq", "orc_vn"):
            getattr(L, name).restype = d
            getattr(L, name).argtypes = [i, d, d]
        L.orc_rates.restype = None
        L.orc_rates.argtypes = [pd, d, pd]
        L.orc_point.restype = None
        L.orc_adjust_activate.restype = None
        L.orc_adjust_activate.argtypes = [pd, pd]
        L.orc_point.argtypes = [pd, d, pd]
        L.orc_sediment_column.restype = u
        L.orc_sediment_column.argtypes = [pd, pd, pd, pd, i, d, pd, ctypes.POINTER(ctypes.c_int)]
        L.orc_step.restype = u
        L.orc_step.argtypes = [pd, ctypes.c_long, i, i, pd, pd, ctypes.POINTER(ctypes.c_int), d, i]
        L.orc_step_cfg.restype = u
        L.orc_step_cfg.argtypes = [pd, ctypes.c_long, i, i, pd, pd, ctypes.POINTER(ctypes.c_int), d, i, i]
        L.orc_point_cfg.restype = None
        L.orc_point_cfg.argtypes = [pd, d, pd, i]
        L.orc_rates_cfg.restype = None
        L.orc_rates_cfg.argtypes = [pd, d, pd, i]
        for name in ("orc_lambda_mu",):
            getattr(L, name).restype = d
            getattr(L, name).argtypes = [i, d, d, d]
        L.orc_moment_mu.restype = d
        L.orc_moment_mu.argtypes = [i, d, d, d, d, d]
        L.orc_vent_integral_mu.restype = d
        L.orc_vent_integral_mu.argtypes = [i, d, d, d, d]
        for name in ("orc_vq_mu", "orc_vn_mu", "orc_vz_mu"):
            getattr(L, name).restype = d
            getattr(L, name).argtypes = [i, d, d, d]
        L.orc_rain_mu.restype = d
        L.orc_rain_mu.argtypes = [d, d, d]
        L.orc_point_3m.restype = None
        L.orc_point_3m.argtypes = [pd, d, pd]
        L.orc_sediment_rain_3m.restype = u
        L.orc_sediment_rain_3m.argtypes = [pd, pd, pd, pd, pd, i, d, pd, ctypes.POINTER(ctypes.c_int)]
        L.orc_step_3m.restype = u
        L.orc_step_3m.argtypes = [pd, ctypes.c_long, i, i, pd, pd, d, i]
        L.orc_shape_mu.restype = d
        L.orc_shape_mu.argtypes = [i, d, d, d]
        L.orc_point_3m_cold.restype = None
        L.orc_point_3m_cold.argtypes = [pd, d, pd]
        L.orc_sediment_3m.restype = u
        L.orc_sediment_3m.argtypes = [pd, pd, pd, pd, pd, i, d, pd, ctypes.POINTER(ctypes.c_int)]
        L.orc_point_aero_cold.restype = None
        L.orc_point_aero_cold.argtypes = [pd, d, pd]
        L.orc_step_aero_cold.restype = u
        L.orc_step_aero_cold.argtypes = [pd, ctypes.c_long, i, i, pd, pd, d, i]
        L.orc_step_3m_cold.restype = u
        L.orc_step_3m_cold.argtypes = [pd, ctypes.c_long, i, i, pd, pd, d, i]
        L.orc_point_aero.restype = None
        L.orc_point_aero.argtypes = [pd, d, pd]
        L.orc_step_aero.restype = u
        L.orc_step_aero.argtypes = [pd, ctypes.c_long, i, i, pd, pd, d, i]
        L.orc_param.restype = d
        L.orc_param.argtypes = [ctypes.c_char_p]
        L.orc_max_threads.restype = i
        L.orc_max_threads.argtypes = []
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def param(name: str) -> float:
    return lib().orc_param(name.encode())


def es_liq(T: float) -> float:
    return lib().orc_es_liq(T)


def es_ice(T: float) -> float:
    return lib().orc_es_ice(T)


def qsat(es: float, p: float) -> float:
    return lib().orc_qsat(es, p)


def dqsat_liq_dT(T: float, p: float) -> float:
    return lib().orc_dqsat_liq_dT(T, p)


def satadj(p: float, T: float, qv: float, qc: float):
    t, v, c = ctypes.c_double(T), ctypes.c_double(qv), ctypes.c_double(qc)
    lib().orc_satadj(p, ctypes.byref(t), ctypes.byref(v), ctypes.byref(c))
    return t.value, v.value, c.value


def arg_sm(T: float) -> float:
    return lib().orc_arg_sm(T)


def arg_smax(N: float, w: float, T: float, p: float) -> float:
    return lib().orc_arg_smax(N, w, T, p)


def arg_nact(N: float, w: float, T: float, p: float) -> float:
    return lib().orc_arg_nact(N, w, T, p)


def lam(sp: str, q: float, n: float) -> float:
    return lib().orc_lambda(SPECIES[sp], q, n)


def moment(sp: str, rho: float, q: float, lam_: float, k: float) -> float:
    return lib().orc_moment(SPECIES[sp], rho, q, lam_, k)


def vent_integral(sp: str, rho: float, q: float, lam_: float) -> float:
    return lib().orc_vent_integral(SPECIES[sp], rho, q, lam_)


def vq(sp: str, rho: float, lam_: float) -> float:
    return lib().orc_vq(SPECIES[sp], rho, lam_)


def vn(sp: str, rho: float, lam_: float) -> float:
    return lib().orc_vn(SPECIES[sp], rho, lam_)


def rates(state: np.ndarray, dt: float, warm: bool = False) -> dict:
    st = np.ascontiguousarray(state, dtype=np.float64)
    assert st.shape == (NFIELDS,)
    out = np.zeros(NPROC)
    lib().orc_rates_cfg(_dp(st), dt, _dp(out), int(warm))
    return dict(zip(PROCS, out.tolist()))


def point(state: np.ndarray, dt: float, warm: bool = False) -> np.ndarray:
    st = np.ascontiguousarray(state, dtype=np.float64)
    assert st.shape == (NFIELDS,)
    out = np.zeros(NPROG)
    lib().orc_point_cfg(_dp(st), dt, _dp(out), int(warm))
    return out


def sediment_column(q: np.ndarray, n: np.ndarray, rho: np.ndarray, dz: np.ndarray, dt: float):
    """q, n: [4][nlev] for r, i, s, g (copied); returns (q, n, precip[4], nsub[4], err)."""
    q = np.array(q, dtype=np.float64, order="C")
    n = np.array(n, dtype=np.float64, order="C")
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    dz = np.ascontiguousarray(dz, dtype=np.float64)
    nlev = rho.shape[0]
    assert q.shape == (4, nlev) and n.shape == (4, nlev) and dz.shape == (nlev,)
    pr = np.zeros(4)
    ns = np.zeros(4, dtype=np.int32)
    err = lib().orc_sediment_column(_dp(q), _dp(n), _dp(rho), _dp(dz), nlev, dt, _dp(pr),
                                    ns.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return q, n, pr, ns, err


def step(fld: np.ndarray, ncols: int, dz: np.ndarray, dt: float, precip: np.ndarray | None = None,
         nthreads: int = 0, want_nsub: bool = False, warm: bool = False):
    """One step over a domain, in place on ``fld`` [16][nlev][pitch].

    Returns (precip [4][pitch] accumulated, nsub [4][pitch] or None, err bits).
    warm: the warm configuration (liquid water only; ice fields untouched).
    """
    assert fld.dtype == np.float64 and fld.flags["C_CONTIGUOUS"] and fld.shape[0] == NFIELDS
    nlev, pitch = fld.shape[1], fld.shape[2]
    assert ncols <= pitch
    dz = np.ascontiguousarray(dz, dtype=np.float64)
    assert dz.shape == (nlev,)
    if precip is None:
        precip = np.zeros((4, pitch))
    assert precip.shape == (4, pitch) and precip.dtype == np.float64 and precip.flags["C_CONTIGUOUS"]
    nsub = np.zeros((4, pitch), dtype=np.int32) if want_nsub else None
    nsp = nsub.ctypes.data_as(ctypes.POINTER(ctypes.c_int)) if want_nsub else None
    err = lib().orc_step_cfg(_dp(fld), pitch, ncols, nlev, _dp(dz), _dp(precip), nsp, dt, nthreads, int(warm))
    return precip, nsub, err


def max_threads() -> int:
    return lib().orc_max_threads()


def adjust_activate(state: np.ndarray) -> np.ndarray:
    """The state after saturation adjustment and activation (what the rates see)."""
    st = np.ascontiguousarray(state, dtype=np.float64)
    assert st.shape == (NFIELDS,)
    out = np.zeros(NFIELDS)
    lib().orc_adjust_activate(_dp(st), _dp(out))
    return out


def point_aero(state: np.ndarray, dt: float) -> np.ndarray:
    """Warm point with activated-aerosol mass: state[19] -> [13 prognostic, ma, mac, mar]."""
    st = np.ascontiguousarray(state, dtype=np.float64)
    assert st.shape == (NFIELDS_AERO,)
    out = np.zeros(NPROG_AERO)
    lib().orc_point_aero(_dp(st), dt, _dp(out))
    return out


def step_aero(fld: np.ndarray, ncols: int, dz: np.ndarray, dt: float, precip: np.ndarray | None = None,
              nthreads: int = 0):
    """Warm step with activated-aerosol mass, in place on fld [19][nlev][pitch];
    precip [5][pitch] (r, i, s, g, aerosol) accumulated.  Returns (precip, err)."""
    assert fld.dtype == np.float64 and fld.flags["C_CONTIGUOUS"] and fld.shape[0] == NFIELDS_AERO
    nlev, pitch = fld.shape[1], fld.shape[2]
    dz = np.ascontiguousarray(dz, dtype=np.float64)
    if precip is None:
        precip = np.zeros((5, pitch))
    assert precip.shape == (5, pitch) and precip.dtype == np.float64 and precip.flags["C_CONTIGUOUS"]
    err = lib().orc_step_aero(_dp(fld), pitch, ncols, nlev, _dp(dz), _dp(precip), dt, nthreads)
    return precip, err


# ------------------------------------------------------- triple-moment rain
def lam_mu(sp: str, q: float, n: float, mu: float) -> float:
    return lib().orc_lambda_mu(SPECIES[sp], q, n, mu)


def moment_mu(sp: str, rho: float, q: float, lam_: float, k: float, mu: float) -> float:
    return lib().orc_moment_mu(SPECIES[sp], rho, q, lam_, k, mu)


def vent_integral_mu(sp: str, rho: float, q: float, lam_: float, mu: float) -> float:
    return lib().orc_vent_integral_mu(SPECIES[sp], rho, q, lam_, mu)


def vq_mu(sp: str, rho: float, lam_: float, mu: float) -> float:
    return lib().orc_vq_mu(SPECIES[sp], rho, lam_, mu)


def vn_mu(sp: str, rho: float, lam_: float, mu: float) -> float:
    return lib().orc_vn_mu(SPECIES[sp], rho, lam_, mu)


def vz_mu(sp: str, rho: float, lam_: float, mu: float) -> float:
    return lib().orc_vz_mu(SPECIES[sp], rho, lam_, mu)


def rain_mu(q: float, n: float, z: float) -> float:
    """The rain shape parameter diagnosed from its mass, number and sixth moment."""
    return lib().orc_rain_mu(q, n, z)


def point_3m(state: np.ndarray, dt: float) -> np.ndarray:
    """Warm point with triple-moment rain: state[17] -> [13 prognostic, z]."""
    st = np.ascontiguousarray(state, dtype=np.float64)
    assert st.shape == (NFIELDS_3M,)
    out = np.zeros(NPROG_3M)
    lib().orc_point_3m(_dp(st), dt, _dp(out))
    return out


def sediment_rain_3m(q, n, z, rho, dz, dt: float):
    """Rain sedimentation of q, n, z [nlev] (copied); returns (q, n, z, precip, nsub, err)."""
    q, n, z = (np.array(x, dtype=np.float64, order="C") for x in (q, n, z))
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    dz = np.ascontiguousarray(dz, dtype=np.float64)
    pr = np.zeros(1)
    ns = np.zeros(1, dtype=np.int32)
    err = lib().orc_sediment_rain_3m(_dp(q), _dp(n), _dp(z), _dp(rho), _dp(dz), rho.shape[0], dt, _dp(pr),
                                      ns.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return q, n, z, pr[0], int(ns[0]), err


def step_3m(fld: np.ndarray, ncols: int, dz: np.ndarray, dt: float, precip: np.ndarray | None = None,
            nthreads: int = 0):
    """Warm step with triple-moment rain, in place on fld [17][nlev][pitch];
    precip [4][pitch] accumulated.  Returns (precip, err)."""
    assert fld.dtype == np.float64 and fld.flags["C_CONTIGUOUS"] and fld.shape[0] == NFIELDS_3M
    nlev, pitch = fld.shape[1], fld.shape[2]
    dz = np.ascontiguousarray(dz, dtype=np.float64)
    if precip is None:
        precip = np.zeros((4, pitch))
    err = lib().orc_step_3m(_dp(fld), pitch, ncols, nlev, _dp(dz), _dp(precip), dt, nthreads)
    return precip, err


# --------------------------------------- triple-moment, cold configuration
def shape_mu(sp: str, q: float, n: float, z: float) -> float:
    """Shape parameter of species sp diagnosed from q, n and its sixth moment z."""
    return lib().orc_shape_mu(SPECIES[sp], q, n, z)


def point_3m_cold(state: np.ndarray, dt: float) -> np.ndarray:
    """Cold point with triple-moment r, i, s, g: state[20] -> [13 prognostic, z_r, z_i, z_s, z_g]."""
    st = np.ascontiguousarray(state, dtype=np.float64)
    assert st.shape == (NFIELDS_3MC,)
    out = np.zeros(NPROG_3MC)
    lib().orc_point_3m_cold(_dp(st), dt, _dp(out))
    return out


def sediment_3m(q, n, z, rho, dz, dt: float):
    """Sedimentation of q, n, z [4][nlev] (r, i, s, g; copied); returns (q, n, z, precip[4], nsub[4], err)."""
    q, n, z = (np.array(x, dtype=np.float64, order="C") for x in (q, n, z))
    assert q.shape[0] == 4 and n.shape == q.shape and z.shape == q.shape
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    dz = np.ascontiguousarray(dz, dtype=np.float64)
    pr = np.zeros(4)
    ns = np.zeros(4, dtype=np.int32)
    err = lib().orc_sediment_3m(_dp(q), _dp(n), _dp(z), _dp(rho), _dp(dz), rho.shape[0], dt, _dp(pr),
                                ns.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return q, n, z, pr, ns, err


def step_3m_cold(fld: np.ndarray, ncols: int, dz: np.ndarray, dt: float, precip: np.ndarray | None = None,
                 nthreads: int = 0):
    """Cold step with triple-moment r, i, s, g, in place on fld [20][nlev][pitch];
    precip [4][pitch] accumulated.  Returns (precip, err)."""
    assert fld.dtype == np.float64 and fld.flags["C_CONTIGUOUS"] and fld.shape[0] == NFIELDS_3MC
    nlev, pitch = fld.shape[1], fld.shape[2]
    dz = np.ascontiguousarray(dz, dtype=np.float64)
    if precip is None:
        precip = np.zeros((4, pitch))
    err = lib().orc_step_3m_cold(_dp(fld), pitch, ncols, nlev, _dp(dz), _dp(precip), dt, nthreads)
    return precip, err


# ------------------------------------- activated-aerosol mass, cold configuration
def point_aero_cold(state: np.ndarray, dt: float) -> np.ndarray:
    """Cold point with aerosol mass: state[22] -> [13 prognostic, ma, mac, mar, mai, mas, mag]."""
    st = np.ascontiguousarray(state, dtype=np.float64)
    assert st.shape == (NFIELDS_AEROC,)
    out = np.zeros(NPROG_AEROC)
    lib().orc_point_aero_cold(_dp(st), dt, _dp(out))
    return out


def step_aero_cold(fld: np.ndarray, ncols: int, dz: np.ndarray, dt: float, precip: np.ndarray | None = None,
                   nthreads: int = 0):
    """Cold step with aerosol mass, in place on fld [22][nlev][pitch]; precip
    [5][pitch] (r, i, s, g, aerosol) accumulated.  Returns (precip, err)."""
    assert fld.dtype == np.float64 and fld.flags["C_CONTIGUOUS"] and fld.shape[0] == NFIELDS_AEROC
    nlev, pitch = fld.shape[1], fld.shape[2]
    dz = np.ascontiguousarray(dz, dtype=np.float64)
    if precip is None:
        precip = np.zeros((5, pitch))
    assert precip.shape == (5, pitch) and precip.dtype == np.float64 and precip.flags["C_CONTIGUOUS"]
    err = lib().orc_step_aero_cold(_dp(fld), pitch, ncols, nlev, _dp(dz), _dp(precip), dt, nthreads)
    return precip, err
