"""Seeded synthetic MONC-shaped column profiles.

The paper's benchmark is MONC's stratus case (Section 3.3: columns of 60 levels,
warm and cold configurations); neither MONC nor that case ships with it, so
these generators stand in for it.  They build atmospheric states in the
level-major structure-of-arrays layout the step consumes,
``fld[field][level][column]``.

This module is shared by the product, the tests and the oracle's callers.  It
holds none of the microphysics method's arithmetic: saturation here uses the
Tetens (1930) formula purely to place the humidity profile, mean particle
masses use spheres of a nominal density, and pressure is integrated
hydrostatically.  None of these formulas is used by the step itself.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# Field order of the state array (13 prognostic fields updated in place,
# then 3 read-only inputs).  Units: K, kg/kg, 1/kg, Pa, kg/m^3, m/s.
FIELDS = ("T", "qv", "qc", "qr", "qi", "qs", "qg",
          "nc", "nr", "ni", "ns", "ng", "na",
          "p", "rho", "w")
NFIELDS = len(FIELDS)
NPROG = 13
FIDX = {name: i for i, name in enumerate(FIELDS)}
# Surface precipitation accumulators, one per sedimenting species.
PRECIP = ("r", "i", "s", "g")

_RD = 287.04
_G = 9.81


def pad_columns(ncols: int, multiple: int = 32) -> int:
    """Column pitch: ncols rounded up to a multiple of ``multiple``."""
    return max(multiple, ((ncols + multiple - 1) // multiple) * multiple)


def dz_uniform(nlev: int, dz: float = 100.0) -> np.ndarray:
    return np.full(nlev, dz, dtype=np.float64)


def dz_stretched(nlev: int, dz_bottom: float = 20.0, dz_top: float = 200.0) -> np.ndarray:
    """Geometric stretching from dz_bottom at the surface to dz_top aloft."""
    if nlev == 1:
        return np.array([dz_bottom], dtype=np.float64)
    r = (dz_top / dz_bottom) ** (1.0 / (nlev - 1))
    return dz_bottom * r ** np.arange(nlev, dtype=np.float64)


def _tetens_qsat(T: np.ndarray, p: np.ndarray) -> np.ndarray:
    # Tetens (1930) over liquid; only used to place relative humidity.
    tc = T - 273.15
    es = 610.78 * np.exp(17.27 * tc / (tc + 237.3))
    return 0.622 * es / (p - 0.378 * es)


@dataclass(frozen=True)
class Recipe:
    """Parameters of one synthetic workload (all lengths in m)."""
    T_sfc: float = 290.0            # surface temperature, K
    lapse: float = 6.5e-3           # K/m
    T_noise: float = 0.5            # K, std of additive noise
    cloud_frac: float = 1.0         # fraction of columns that carry cloud
    base_range: tuple = (1000.0, 1000.0)
    top_range: tuple = (3000.0, 3000.0)
    w_max: float = 2.0              # w ~ U(-w_max, w_max)
    medians: tuple = (1e-4, 1e-5, 1e-5, 1e-5, 1e-6)   # c, r, i, s, g (kg/kg)
    sigma_ln: float = 1.0           # lognormal spread of masses
    q_cap: tuple = (2e-3, 5e-3, 1e-3, 2e-3, 5e-3)
    rh_clear: tuple = (0.90, 0.99)
    rh_cloud: tuple = (1.002, 1.02)
    na_cm3: float = 100.0           # aerosol number concentration, cm^-3


# Nominal sphere densities and mass-mean diameter ranges used to turn a mass
# into a number (kg/m^3; m).  Profile construction only.
_GEN_DENS = (1000.0, 1000.0, 500.0, 100.0, 400.0)
_GEN_DIAM = ((10e-6, 20e-6), (0.3e-3, 1.5e-3), (30e-6, 100e-6), (0.3e-3, 2e-3), (0.5e-3, 3e-3))

RECIPES = {
    # 16x16 x 50 levels, dz = 100 m, one cloud layer at 1-3 km everywhere.
    "stratus": Recipe(),
    # 256x256 x 100 levels stretched; 30% cloudy columns, base/top in 0.5-4 km.
    "stratus_broken": Recipe(cloud_frac=0.30, base_range=(500.0, 2000.0), top_range=(2000.0, 4000.0)),
    # 512x512 x 150: deep convection, freezing level at 3 km, graupel up to 5e-3.
    "deep_convective": Recipe(T_sfc=273.15 + 6.5 * 3.0, cloud_frac=0.6,
                              base_range=(500.0, 1500.0), top_range=(6000.0, 10000.0),
                              w_max=10.0, medians=(3e-4, 1e-4, 2e-5, 1e-4, 3e-4)),
}


def make_state(recipe: str | Recipe, ncols: int, nlev: int, dz: np.ndarray, seed: int,
               pitch: int | None = None) -> np.ndarray:
    """Return fld[NFIELDS][nlev][pitch] (float64); columns >= ncols are zero-padded.

    Level k = 0 is the surface.  Columns are independent draws.
    """
    rc = RECIPES[recipe] if isinstance(recipe, str) else recipe
    pitch = pad_columns(ncols) if pitch is None else pitch
    if pitch < ncols:
        raise ValueError("pitch < ncols")
    dz = np.asarray(dz, dtype=np.float64)
    assert dz.shape == (nlev,)
    rng = np.random.default_rng(seed)
    fld = np.zeros((NFIELDS, nlev, pitch), dtype=np.float64)
    if ncols == 0 or nlev == 0:
        return fld
    z = np.cumsum(dz) - 0.5 * dz                       # level centres
    T_mean = rc.T_sfc - rc.lapse * z
    # Hydrostatic pressure from 1000 hPa using the noise-free temperature.
    lnp = np.empty(nlev)
    lnp[0] = math.log(1e5) - _G * z[0] / (_RD * rc.T_sfc)
    for k in range(1, nlev):
        Tm = 0.5 * (T_mean[k] + T_mean[k - 1])
        lnp[k] = lnp[k - 1] - _G * (z[k] - z[k - 1]) / (_RD * Tm)
    p = np.exp(lnp)[:, None] * np.ones((1, ncols))
    T = T_mean[:, None] + rng.normal(0.0, rc.T_noise, size=(nlev, ncols))
    rho = p / (_RD * T)

    cloudy = rng.random(ncols) < rc.cloud_frac
    zb = rng.uniform(*rc.base_range, size=ncols)
    zt = np.maximum(rng.uniform(*rc.top_range, size=ncols), zb + 200.0)
    zz = z[:, None]
    in_cloud = cloudy[None, :] & (zz >= zb[None, :]) & (zz <= zt[None, :])

    rh = np.where(in_cloud, rng.uniform(*rc.rh_cloud, size=(nlev, ncols)),
                  rng.uniform(*rc.rh_clear, size=(nlev, ncols)))
    qv = rh * _tetens_qsat(T, p)

    T0 = 273.15
    masks = (
        in_cloud,                                                                  # cloud
        cloudy[None, :] & (zz <= zt[None, :]) & (T > T0 - 5.0),                   # rain
        cloudy[None, :] & (zz >= zb[None, :]) & (zz <= zt[None, :] + 2000.0) & (T < T0 - 5.0),  # ice
        cloudy[None, :] & (zz >= zb[None, :]) & (zz <= zt[None, :] + 1000.0) & (T < T0),       # snow
        cloudy[None, :] & (zz >= zb[None, :]) & (zz <= zt[None, :]) & (T < T0 + 2.0),           # graupel
    )
    q = []
    nums = []
    for s in range(5):
        m = rc.medians[s] * np.exp(rc.sigma_ln * rng.normal(size=(nlev, ncols)))
        m = np.minimum(m, rc.q_cap[s])
        m = np.where(masks[s], m, 0.0)
        d = rng.uniform(*_GEN_DIAM[s], size=(nlev, ncols))
        mass1 = math.pi / 6.0 * _GEN_DENS[s] * d ** 3
        n = np.where(m > 0.0, m / mass1, 0.0)
        q.append(m)
        nums.append(n)
    na = rc.na_cm3 * 1e6 / rho
    w = rng.uniform(-rc.w_max, rc.w_max, size=(nlev, ncols))

    cols = slice(0, ncols)
    fld[FIDX["T"], :, cols] = T
    fld[FIDX["qv"], :, cols] = qv
    for s, name in enumerate(("qc", "qr", "qi", "qs", "qg")):
        fld[FIDX[name], :, cols] = q[s]
    for s, name in enumerate(("nc", "nr", "ni", "ns", "ng")):
        fld[FIDX[name], :, cols] = nums[s]
    fld[FIDX["na"], :, cols] = na
    fld[FIDX["p"], :, cols] = p
    fld[FIDX["rho"], :, cols] = rho
    fld[FIDX["w"], :, cols] = w
    return fld


def workload(name: str, ncols: int | None = None, nlev: int | None = None, seed: int | None = None):
    """Named workloads: (fld, dz, ncols, nlev, dt, nsteps).

    stratus_16x16x50        16x16 columns x 50 levels, dz = 100 m, dt = 1 s, 1 step
    stratus_256x256x100     256x256 x 100 stretched 20-200 m, 30% cloudy, 10 steps
    deep_512x512x150        512x512 x 150 stretched, deep convection, 100 steps
    stratus_512x512x150     512x512 x 150 stretched, 30% cloudy stratus (warm vs cold configuration)
    ``ncols`` / ``nlev`` override the sizes (same recipe) for sub-sampled runs.
    """
    table = {
        "stratus_16x16x50": ("stratus", 256, 50, "uniform", 1.0, 1, 1234),
        "stratus_256x256x100": ("stratus_broken", 65536, 100, "stretched", 1.0, 10, 1235),
        "deep_512x512x150": ("deep_convective", 262144, 150, "stretched", 1.0, 100, 1236),
        "stratus_512x512x150": ("stratus_broken", 262144, 150, "stretched", 1.0, 100, 1238),
    }
    recipe, nc, nl, dzk, dt, nsteps, sd = table[name]
    nc = nc if ncols is None else ncols
    nl = nl if nlev is None else nlev
    sd = sd if seed is None else seed
    dz = dz_uniform(nl) if dzk == "uniform" else dz_stretched(nl)
    fld = make_state(recipe, nc, nl, dz, sd)
    return fld, dz, nc, nl, dt, nsteps


def batch_workload(ndom: int = 64, seed: int = 1237, ncols_range=(1_000, 100_000), nlev_range=(40, 150),
                   cloud_range=(0.05, 0.60), scale: float = 1.0):
    """Many independent domains of uneven size (config of the batched step):
    column counts log-uniform in ncols_range (times `scale`), level counts
    uniform in nlev_range, stretched dz 20-200 m, stratus-type profiles with a
    cloud fraction uniform in cloud_range.  Returns a list of (fld, dz, ncols,
    nlev) and dt = 1 s."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(ndom):
        nc = int(round(math.exp(rng.uniform(math.log(ncols_range[0]), math.log(ncols_range[1]))) * scale))
        nc = max(nc, 1)
        nl = int(rng.integers(nlev_range[0], nlev_range[1] + 1))
        cf = float(rng.uniform(*cloud_range))
        rc = Recipe(cloud_frac=cf, base_range=(500.0, 2000.0), top_range=(2000.0, 4000.0))
        dz = dz_stretched(nl)
        out.append((make_state(rc, nc, nl, dz, seed=int(rng.integers(1 << 30))), dz, nc, nl))
    return out, 1.0
