"""Pin of the activation parameterisation against the equations it approximates.

Abdul-Razzak & Ghan (2000) give a closed-form approximation to the maximum
supersaturation of an air parcel rising at constant w through one lognormal
aerosol mode: dS/dt = alpha w - gamma dW/dt, with droplets growing by
dr/dt = (G / r) (S - A / r + B r_d^3 / r^3) and W = (4 pi rho_w / 3) sum N r^3
per unit volume.  Here those equations are integrated numerically (stiff
solver, the mode split into 120 bins, droplets starting at their equilibrium
radius at S = 0) with the oracle's constants, and the oracle's closed form is
required to agree within the parameterisation's stated accuracy: 20 % for
S_max (the published comparison is within about 10 %), 10 % for the number
activated (the bins whose wet radius has passed the critical radius).  A
wrong exponent or a dropped term in the closed form moves S_max by tens of
per cent or more.
"""
import numpy as np
import pytest

import oracle as O

scipy = pytest.importorskip("scipy")
from scipy.integrate import solve_ivp  # noqa: E402
from scipy.stats import norm  # noqa: E402


def parcel(N, w, T, p, nb=120):
    g, cp, Lv = O.param("g"), O.param("cp"), O.param("Lv")
    rhow, Dv, Ka = O.param("rho_w"), O.param("Dv"), O.param("Ka")
    Mw, Ma, R = O.param("Mw"), O.param("Ma"), O.param("Rgas")
    sig, rm, kap, sg = O.param("surft"), O.param("arg_rm"), O.param("arg_kappa"), O.param("arg_sigma")
    es = O.es_liq(T)
    # the parcel balance and growth law with their standard coefficients
    alpha = g * Mw * Lv / (cp * R * T * T) - g * Ma / (R * T)
    gam = R * T / (es * Mw) + Mw * Lv * Lv / (cp * p * Ma * T)
    G = 1.0 / (rhow * R * T / (es * Dv * Mw) + Lv * rhow / (Ka * T) * (Lv * Mw / (R * T) - 1.0))
    A = 2.0 * sig * Mw / (rhow * R * T)
    z = np.linspace(-5.0, 5.0, nb + 1)
    Ni = N * np.diff(norm.cdf(z))
    rd = rm * sg ** (0.5 * (z[1:] + z[:-1]))
    B = kap * rd ** 3

    def f(t, y):
        S, r = y[0], y[1:]
        drdt = G / r * (S - A / r + B / r ** 3)
        return np.concatenate(([alpha * w - gam * 4.0 * np.pi * rhow * np.sum(Ni * r * r * drdt)], drdt))

    t_end = 4.0 * 0.01 / (alpha * w)
    sol = solve_ivp(f, (0.0, t_end), np.concatenate(([0.0], np.sqrt(B / A))), method="BDF", rtol=1e-7,
                    atol=np.concatenate(([1e-10], np.full(nb, 1e-12))), max_step=t_end / 400)
    assert sol.success
    k = int(np.argmax(sol.y[0]))
    assert 0 < k < sol.y.shape[1] - 1          # the maximum lies inside the integration
    activated = Ni[sol.y[1:, -1] > np.sqrt(3.0 * B / A)].sum()
    return sol.y[0, k], activated


@pytest.mark.parametrize("N,w,T,p", [(1e8, 0.5, 283.0, 9.0e4), (1e8, 2.0, 283.0, 9.0e4), (1e9, 1.0, 283.0, 9.0e4),
                                     (3e8, 5.0, 283.0, 9.0e4), (5e7, 0.2, 283.0, 9.0e4), (3e8, 1.0, 275.0, 7.5e4)])
def test_arg_smax_and_activation_against_a_parcel_integration(N, w, T, p):
    smax, act = parcel(N, w, T, p)
    assert abs(O.arg_smax(N, w, T, p) / smax - 1.0) < 0.20
    assert abs(O.arg_nact(N, w, T, p) / act - 1.0) < 0.10


def test_arg_closed_form_worked_by_hand():
    """The closed form evaluated by hand, term by term, at T = 283 K,
    p = 900 hPa, w = 0.5 m/s and N = 1e9 m^-3 (about half the mode activates,
    so both S_max and the activated number are sensitive to every term):
      e_s (Bolton, t = 9.85 C) = 611.2 exp(17.67 t / (t + 243.5))   = 1214.8994 Pa
      alpha = g M_w L_v / (c_p R T^2) - g M_a / (R T)               = 5.3946220e-4 m^-1
      gamma = R T / (e_s M_w) + M_w L_v^2 / (c_p p M_a T)           = 259.36414 m^3 kg^-1
      F_d = rho_w R T / (e_s D_v M_w)                              = 4.7567841e9
      F_k = L_v rho_w / (K_a T) (L_v M_w / (R T) - 1)              = 6.6775551e9
      G = 1 / (F_d + F_k)                                          = 8.7455863e-11 m^2 s^-1
      A = 2 sigma_w M_w / (rho_w R T)                              = 1.1653395e-9 m
      S_m = (2 / sqrt(kappa)) (A / (3 r_m))^1.5                     = 1.7535045e-3
      alpha w / G                                                  = 3.0841969e6 m^-2
      zeta = (2 A / 3) (alpha w / G)^0.5                           = 1.3643703e-6
      eta = (alpha w / G)^1.5 / (2 pi rho_w gamma N)               = 3.3237117e-6
      f_1 = 0.5 exp(2.5 ln^2 sigma), f_2 = 1 + 0.25 ln sigma       = 0.75416636, 1.1013663
      f_1 (zeta / eta)^1.5 = 0.19834923, f_2 (S_m^2 / (eta + 3 zeta))^0.75 = 0.56902151
      S_max = S_m / sqrt(0.19834923 + 0.56902151)                  = 2.0017243e-3
      u = 2 ln(S_m / S_max) / (3 sqrt(2) ln sigma)                 = -0.15392318
      N_act = (N / 2) erfc(u)                                      = 5.8616087e8 m^-3"""
    N, w, T, p = 1e9, 0.5, 283.0, 9.0e4
    assert abs(O.arg_sm(T) / 1.7535045e-3 - 1.0) < 1e-7
    assert abs(O.arg_smax(N, w, T, p) / 2.0017243e-3 - 1.0) < 1e-7
    assert abs(O.arg_nact(N, w, T, p) / 5.8616087e8 - 1.0) < 1e-7
