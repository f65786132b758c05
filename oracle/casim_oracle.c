/*
 * FP64 CPU oracle of the column microphysics step -- TEST INFRASTRUCTURE.
 *
 * Plain, slow, sequential-per-column C, compiled with -ffp-contract=off so
 * every product and sum is rounded as written.  Only the tests, the smoke
 * check and the benchmark's CPU-baseline leg load it.  Nothing here is shared
 * with the CUDA path.
 *
 * The paper (Section 2) describes CASIM as a bulk scheme in which each
 * species carries a gamma-type size distribution described by a diameter D,
 * a shape mu, a slope lambda and an intercept N0, with columns independent
 * and processes (accretion, autoconversion, sedimentation, activation)
 * acting in the vertical only.  It prints no rate laws, so each process
 * below follows a named published parameterisation:
 *   saturation vapour pressure   Bolton (1980) over liquid; Murray (1967)
 *                                Tetens form over ice
 *   saturation adjustment        Newton iteration on the isobaric enthalpy
 *                                balance, 4 fixed iterations
 *   activation                   Abdul-Razzak & Ghan (2000), one lognormal mode
 *   autoconversion, accretion    Khairoutdinov & Kogan (2000)
 *   self-collection              Seifert & Beheng (2001) cloud, (2006) rain
 *   evaporation, deposition,     ventilated diffusional growth integrated
 *   melting                      over the gamma distribution (Pruppacher &
 *                                Klett ventilation 0.78 + 0.31 Sc^1/3 Re^1/2)
 *   ice nucleation               Meyers, DeMott & Cotton (1992)
 *   riming                       continuous collection, E = 1
 *   sedimentation                mass/number-weighted fall speeds, upwind
 *                                flux form, CFL substeps
 * Parity of the whole step with CASIM itself is unpinned: CASIM's source is
 * not available; this file defines the scheme the GPU path must reproduce.
 */
#include "casim_oracle.h"

#include <math.h>
#include <string.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- constants */
static const double T0 = 273.15;       /* melting point, K */
static const double CP = 1005.0;       /* J kg^-1 K^-1 */
static const double LV = 2.5e6;        /* J kg^-1 */
static const double LF = 3.34e5;       /* J kg^-1 */
#define LS (LV + LF)
static const double RD = 287.04;
static const double RV = 461.5;
#define EPS (RD / RV)
static const double GRAV = 9.81;
static const double RHOW = 1000.0;
static const double RHO0 = 1.2;        /* fall-speed reference density */
static const double KA = 2.4e-2;       /* thermal conductivity of air */
static const double DV = 2.26e-5;      /* vapour diffusivity */
static const double MUAIR = 1.72e-5;   /* dynamic viscosity of air */
static const double QMIN = 1e-14;      /* species present iff q > QMIN */
static const double TNUC = 268.15;     /* ice nucleation below this, K */
static const double MI0 = 1e-12;       /* mass of a nucleated crystal, kg */
static const double RR0 = 25e-6;       /* radius of a new raindrop, m */
static const double KK_AUT = 1350.0, KK_AUT_QC = 2.47, KK_AUT_NC = -1.79;
static const double NC_MIN_CM3 = 1.0;  /* floor on N_c in the KK formula */
static const double KK_ACC = 67.0, KK_ACC_EXP = 1.15;
static const double KC_SB = 9.44e9, NU_C = 1.0;   /* cloud self-collection */
static const double KR_SB = 5.78;                 /* rain self-collection */
static const double MEY_A = 1e3, MEY_B = -0.639, MEY_C = 12.96;
static const double ARG_RM = 0.05e-6, ARG_SIGMA = 1.5, ARG_KAPPA = 0.61;
static const double MU3_MAX = 20.0;     /* largest rain shape parameter of the triple-moment scheme */
static const double SURFT = 0.0761, MW = 0.018015, MA = 0.028965, RGAS = 8.314;
static const double E_RIM = 1.0;
static const double CMAX = 1.0;        /* Courant limit per substep */
static const double ES_L0 = 611.2, ES_LA = 17.67, ES_LB = 243.5;      /* Bolton */
static const double ES_I0 = 610.78, ES_IA = 21.875, ES_IT = 273.16, ES_IB = 7.66;

typedef struct {
  double a, b;        /* m(D) = a D^b */
  double mu;          /* gamma shape */
  double cv, dv;      /* V(D) = cv D^dv (rho0/rho)^0.4 */
  double vmax;        /* fall-speed cap, m/s */
  double dmin, dmax;  /* bounds on the mean diameter (mu+1)/lambda */
  double ccap;        /* capacitance C = ccap * D */
} orc_species;

#define PI 3.14159265358979323846
static const orc_species SP[ORC_NSPECIES] = {
  /* cloud   */ {PI / 6.0 * 1000.0, 3.0, 2.0, 0.0, 0.0, 0.0, 1e-6, 1e-4, 0.5},
  /* rain    */ {PI / 6.0 * 1000.0, 3.0, 0.0, 130.0, 0.5, 10.0, 50e-6, 5e-3, 0.5},
  /* ice     */ {PI / 6.0 * 500.0, 3.0, 0.0, 700.0, 1.0, 2.0, 1e-6, 500e-6, 0.5},
  /* snow    */ {PI / 6.0 * 100.0, 3.0, 0.0, 11.72, 0.41, 4.0, 10e-6, 5e-3, 1.0 / PI},
  /* graupel */ {PI / 6.0 * 400.0, 3.0, 0.5, 19.3, 0.37, 10.0, 10e-6, 5e-3, 0.5},
};

/* ------------------------------------------------------ c1 thermodynamics */
double orc_es_liq(double T) {
  /* Bolton (1980): e_s = 611.2 exp(17.67 Tc / (Tc + 243.5)), Tc in deg C */
  double tc = T - T0;
  return ES_L0 * exp(ES_LA * tc / (tc + ES_LB));
}

double orc_es_ice(double T) {
  /* Murray (1967) Tetens form over ice */
  return ES_I0 * exp(ES_IA * (T - ES_IT) / (T - ES_IB));
}

double orc_qsat(double es, double p) {
  /* saturation mixing ratio of vapour over the given saturation pressure */
  return EPS * es / (p - (1.0 - EPS) * es);
}

double orc_dqsat_liq_dT(double T, double p) {
  double tc = T - T0;
  double es = orc_es_liq(T);
  double des = es * ES_LA * ES_LB / ((tc + ES_LB) * (tc + ES_LB));
  double den = p - (1.0 - EPS) * es;
  return EPS * p / (den * den) * des;
}

/* ------------------------------------------------ a2 saturation adjustment */
void orc_satadj(double p, double *T, double *qv, double *qc) {
  /* Isobaric adjustment to liquid saturation: find T* with
       cp (T* - T) = Lv (qv - qs(T*))
     by Newton's method, 4 fixed iterations from T (no convergence test, so
     every implementation takes the same path).  The condensed amount
     dq = (cp/Lv)(T* - T) is limited below by -qc (evaporation cannot exceed
     the cloud present); T then follows from dq so that cp dT = Lv dq. */
  double T0v = *T, qv0 = *qv, qc0 = *qc;
  double qs0 = orc_qsat(orc_es_liq(T0v), p);
  if (!(qv0 > qs0 || qc0 > QMIN)) return;
  double Tn = T0v;
  for (int it = 0; it < 4; ++it) {
    double qs = orc_qsat(orc_es_liq(Tn), p);
    double f = (Tn - T0v) - (LV / CP) * (qv0 - qs);
    double fp = 1.0 + (LV / CP) * orc_dqsat_liq_dT(Tn, p);
    Tn = Tn - f / fp;
  }
  double dq = (CP / LV) * (Tn - T0v);
  if (dq < -qc0) dq = -qc0;
  *T = T0v + (LV / CP) * dq;
  *qv = qv0 - dq;
  *qc = qc0 + dq;
}

/* ---------------------------------------------------------- a3 activation */
double orc_arg_sm(double T) {
  /* Critical supersaturation of a particle at the mode radius (Koehler
     theory, kappa form): S_m = (2/sqrt(B)) (A / (3 r_m))^(3/2),
     A = 2 sigma_w M_w / (rho_w R T). */
  double A = 2.0 * SURFT * MW / (RHOW * RGAS * T);
  return 2.0 / sqrt(ARG_KAPPA) * pow(A / (3.0 * ARG_RM), 1.5);
}

double orc_arg_smax(double N, double w, double T, double p) {
  /* Abdul-Razzak & Ghan (2000) maximum supersaturation of a parcel rising at
     w through one lognormal mode of N particles per m^3. */
  double es = orc_es_liq(T);
  double alpha = GRAV * MW * LV / (CP * RGAS * T * T) - GRAV * MA / (RGAS * T);
  double gam = RGAS * T / (es * MW) + MW * LV * LV / (CP * p * MA * T);
  double G = 1.0 / (RHOW * RGAS * T / (es * DV * MW) +
                    LV * RHOW / (KA * T) * (LV * MW / (RGAS * T) - 1.0));
  double A = 2.0 * SURFT * MW / (RHOW * RGAS * T);
  double sm = orc_arg_sm(T);
  double awg = alpha * w / G;
  double zeta = 2.0 * A / 3.0 * sqrt(awg);
  double eta = pow(awg, 1.5) / (2.0 * PI * RHOW * gam * N);
  double lns = log(ARG_SIGMA);
  double f1 = 0.5 * exp(2.5 * lns * lns);
  double f2 = 1.0 + 0.25 * lns;
  double sum = (1.0 / (sm * sm)) * (f1 * pow(zeta / eta, 1.5) + f2 * pow(sm * sm / (eta + 3.0 * zeta), 0.75));
  return 1.0 / sqrt(sum);
}

double orc_arg_nact(double N, double w, double T, double p) {
  /* Number activated (per m^3): the part of the lognormal mode whose
     critical supersaturation lies below S_max. */
  if (!(w > 0.0) || !(N > 0.0)) return 0.0;
  double smax = orc_arg_smax(N, w, T, p);
  double sm = orc_arg_sm(T);
  double u = 2.0 * log(sm / smax) / (3.0 * sqrt(2.0) * log(ARG_SIGMA));
  return 0.5 * N * erfc(u);
}

/* ------------------------------------------------ gamma-distribution algebra */
/* The functions below take the shape parameter mu explicitly; the exported
   ones without _mu use the species' fixed mu (double-moment scheme). */
double orc_lambda_mu(int sp, double q, double n, double mu) {
  /* n(D) = N0 D^mu exp(-lambda D) with m(D) = a D^b:
       q / n = a Gamma(mu+b+1) / (Gamma(mu+1) lambda^b)
     lambda is clamped so the mean diameter (mu+1)/lambda stays inside
     [dmin, dmax]; a non-positive number gives the largest particles. */
  const orc_species *s = &SP[sp];
  double nn = n > 0.0 ? n : 0.0;
  double lam = pow(s->a * tgamma(mu + s->b + 1.0) / tgamma(mu + 1.0) * nn / q, 1.0 / s->b);
  double lo = (mu + 1.0) / s->dmax, hi = (mu + 1.0) / s->dmin;
  if (lam < lo) lam = lo;
  if (lam > hi) lam = hi;
  return lam;
}

double orc_moment_mu(int sp, double rho, double q, double lam, double k, double mu) {
  /* M_k = int D^k n(D) dD per m^3, with N0 fixed by the mass content
     rho q = a N0 Gamma(mu+b+1) / lambda^(mu+b+1):
       M_k = (rho q / a) Gamma(mu+k+1) / Gamma(mu+b+1) * lambda^(b-k) */
  const orc_species *s = &SP[sp];
  return rho * q / s->a * tgamma(mu + k + 1.0) / tgamma(mu + s->b + 1.0) * pow(lam, s->b - k);
}

double orc_vent_integral_mu(int sp, double rho, double q, double lam, double mu) {
  /* int D f_v(D) n(D) dD with f_v = 0.78 + 0.31 Sc^(1/3) Re^(1/2),
     Re = V(D) D / nu, V(D) = cv D^dv (rho0/rho)^0.4, Sc = nu / Dv. */
  const orc_species *s = &SP[sp];
  double nu = MUAIR / rho;
  double sc = nu / DV;
  double vfac = s->cv * pow(RHO0 / rho, 0.4);
  return 0.78 * orc_moment_mu(sp, rho, q, lam, 1.0, mu) +
         0.31 * cbrt(sc) * sqrt(vfac / nu) * orc_moment_mu(sp, rho, q, lam, 0.5 * (s->dv + 3.0), mu);
}

/* fall speed weighted by the k-th moment, int D^k V n dD / int D^k n dD, capped */
static double vk_mu(int sp, double rho, double lam, double mu, double k) {
  const orc_species *s = &SP[sp];
  double v = s->cv * pow(RHO0 / rho, 0.4) * tgamma(mu + k + s->dv + 1.0) / tgamma(mu + k + 1.0) * pow(lam, -s->dv);
  return v < s->vmax ? v : s->vmax;
}

double orc_vq_mu(int sp, double rho, double lam, double mu) { return vk_mu(sp, rho, lam, mu, SP[sp].b); }
double orc_vn_mu(int sp, double rho, double lam, double mu) { return vk_mu(sp, rho, lam, mu, 0.0); }
double orc_vz_mu(int sp, double rho, double lam, double mu) { return vk_mu(sp, rho, lam, mu, 2.0 * SP[sp].b); }

double orc_lambda(int sp, double q, double n) { return orc_lambda_mu(sp, q, n, SP[sp].mu); }
double orc_moment(int sp, double rho, double q, double lam, double k) {
  return orc_moment_mu(sp, rho, q, lam, k, SP[sp].mu);
}
double orc_vent_integral(int sp, double rho, double q, double lam) {
  return orc_vent_integral_mu(sp, rho, q, lam, SP[sp].mu);
}
double orc_vq(int sp, double rho, double lam) { return orc_vq_mu(sp, rho, lam, SP[sp].mu); }
double orc_vn(int sp, double rho, double lam) { return orc_vn_mu(sp, rho, lam, SP[sp].mu); }

/* Triple-moment species: the shape parameter from q, n and the sixth moment
   z (m^6 per kg of air).  With m = a D^3 (every species here has b = 3),
   M3 = q / a per kg and
     G = z n / M3^2 = (mu+4)(mu+5)(mu+6) / ((mu+1)(mu+2)(mu+3)),
   decreasing from 20 at mu = 0 to 1 as mu -> inf.  Start from the root of
   G^(1/3) = (mu+5)/(mu+2), then four Newton steps on ln G(mu) - ln G_obs,
   every iterate clamped to [0, MU3_MAX].  Species absent, or n or z not
   positive: the species' fixed mu. */
double orc_shape_mu(int sp, double q, double n, double z) {
  if (!(q > QMIN) || !(n > 0.0) || !(z > 0.0)) return SP[sp].mu;
  double m3 = q / SP[sp].a;
  double lg = log(z * n / (m3 * m3));
  double g = cbrt(z * n / (m3 * m3));
  double mu = g > 1.0 ? (5.0 - 2.0 * g) / (g - 1.0) : MU3_MAX;
  if (mu < 0.0) mu = 0.0;
  if (mu > MU3_MAX) mu = MU3_MAX;
  for (int it = 0; it < 4; ++it) {
    double f = log((mu + 4.0) * (mu + 5.0) * (mu + 6.0) / ((mu + 1.0) * (mu + 2.0) * (mu + 3.0))) - lg;
    double fp = 1.0 / (mu + 4.0) + 1.0 / (mu + 5.0) + 1.0 / (mu + 6.0) - 1.0 / (mu + 1.0) - 1.0 / (mu + 2.0) -
                1.0 / (mu + 3.0);
    mu -= f / fp;
    if (mu < 0.0) mu = 0.0;
    if (mu > MU3_MAX) mu = MU3_MAX;
  }
  return mu;
}

double orc_rain_mu(double q, double n, double z) { return orc_shape_mu(ORC_R, q, n, z); }

/* --------------------------------------------------------- a4..a9 rates */
static void rates_core(const double *st, double dt, double *R, int warm, const double *mu4);

void orc_rates_cfg(const double *st, double dt, double *R, int warm) { rates_core(st, dt, R, warm, NULL); }

/* mu4: the shape parameters of r, i, s, g (the triple-moment scheme's
   diagnosed ones), or NULL for the species' own */
static void rates_core(const double *st, double dt, double *R, int warm, const double *mu4) {
  const double mu_r = mu4 ? mu4[0] : SP[ORC_R].mu;
  /* Rates in kg kg^-1 s^-1 (masses) except SCC, SCR (number kg^-1 s^-1) and
     NUC (new crystals kg^-1 s^-1).  All are >= 0 except DEPx, which is
     positive for deposition and negative for sublimation.  MLTx is the
     melted mass rate.  warm != 0: the warm configuration, which considers
     liquid water only (Section 2.1): a4 and a5; no ice process. */
  double T = st[ORC_T], qv = st[ORC_QV], qc = st[ORC_QC], qr = st[ORC_QR];
  double nc = st[ORC_NC], nr = st[ORC_NR], ni = st[ORC_NI];
  double p = st[ORC_P], rho = st[ORC_RHO];
  for (int j = 0; j < ORC_NPROC; ++j) R[j] = 0.0;

  double esl = orc_es_liq(T), esi = orc_es_ice(T);
  double qsl = orc_qsat(esl, p), qsi = orc_qsat(esi, p);
  double Sw = qv / qsl, Si = qv / qsi;
  double Aw = LV * LV / (KA * RV * T * T), Bw = RV * T / (esl * DV);
  double Ai = LS * LS / (KA * RV * T * T), Bi = RV * T / (esi * DV);

  int hc = qc > QMIN, hr = qr > QMIN;

  /* a4 warm rain: Khairoutdinov & Kogan (2000), N_c in cm^-3 */
  if (hc) {
    double ncc = rho * nc * 1e-6;
    if (ncc < NC_MIN_CM3) ncc = NC_MIN_CM3;
    R[ORC_AUT] = KK_AUT * pow(qc, KK_AUT_QC) * pow(ncc, KK_AUT_NC);
    /* Seifert & Beheng (2001) cloud self-collection, number only:
       dN/dt = -k_c (nu+2)/(nu+1) L_c^2, L_c = rho q_c */
    R[ORC_SCC] = KC_SB * (NU_C + 2.0) / (NU_C + 1.0) * rho * qc * qc;
  }
  if (hc && hr) R[ORC_ACC] = KK_ACC * pow(qc * qr, KK_ACC_EXP);
  if (hr) {
    /* Seifert & Beheng (2006) rain self-collection: dN/dt = -k_r N_r L_r */
    R[ORC_SCR] = KR_SB * rho * (nr > 0.0 ? nr : 0.0) * qr;
    /* a5 rain evaporation in subsaturated air: capacitance D/2 */
    if (Sw < 1.0) {
      double lam = orc_lambda_mu(ORC_R, qr, nr, mu_r);
      R[ORC_EVR] = 2.0 * PI * (1.0 - Sw) * orc_vent_integral_mu(ORC_R, rho, qr, lam, mu_r) / (rho * (Aw + Bw));
    }
  }
  if (warm) return;
  /* a6 ice nucleation: Meyers et al. (1992), N_in in m^-3 */
  if (T < TNUC && Si > 1.0) {
    double nin = MEY_A * exp(MEY_B + MEY_C * (Si - 1.0));
    double dn = nin / rho - ni;
    if (dn > 0.0) R[ORC_NUC] = dn / dt;
  }
  /* a7 deposition / sublimation, a8 riming, a9 melting for i, s, g */
  static const int spx[3] = {ORC_I, ORC_S, ORC_G};
  static const int qx[3] = {ORC_QI, ORC_QS, ORC_QG};
  static const int nx[3] = {ORC_NI, ORC_NS, ORC_NG};
  static const int depj[3] = {ORC_DEPI, ORC_DEPS, ORC_DEPG};
  static const int mltj[3] = {ORC_MLTI, ORC_MLTS, ORC_MLTG};
  for (int m = 0; m < 3; ++m) {
    int sp = spx[m];
    double q = st[qx[m]];
    if (!(q > QMIN)) continue;
    const double mu = mu4 ? mu4[1 + m] : SP[sp].mu;
    double lam = orc_lambda_mu(sp, q, st[nx[m]], mu);
    if (T < T0) {
      double iv = orc_vent_integral_mu(sp, rho, q, lam, mu);
      R[depj[m]] = 4.0 * PI * SP[sp].ccap * (Si - 1.0) * iv / (rho * (Ai + Bi));
      if (sp != ORC_I && hc) {
        /* collection of cloud: (pi/4) E q_c int D^2 V(D) n(D) dD */
        double vfac = SP[sp].cv * pow(RHO0 / rho, 0.4);
        double r = 0.25 * PI * E_RIM * qc * vfac * orc_moment_mu(sp, rho, q, lam, 2.0 + SP[sp].dv, mu);
        R[sp == ORC_S ? ORC_RIMS : ORC_RIMG] = r;
      }
    } else if (T > T0) {
      double iv = orc_vent_integral_mu(sp, rho, q, lam, mu);
      R[mltj[m]] = 4.0 * PI * SP[sp].ccap * KA * (T - T0) * iv / (rho * LF);
    }
  }
}

/* --------------------------------------------- a10 limiter and update */
typedef struct {
  double rate;    /* mass moved per second (kg/kg/s), >= 0 */
  int msrc, mdst; /* mass pools (state index) or -1 */
  int nsrc;       /* number pool drawn from, or -1 */
  double nsink;   /* number removed per second */
  int ndst;       /* number pool fed, or -1 */
  double nsource; /* number added per second */
  double heat;    /* latent heat released per kg moved (J/kg) */
} orc_transfer;

static double ratio(double n, double q) { return (n > 0.0 ? n : 0.0) / q; }

void orc_adjust_activate(const double *in, double *st) {
  memcpy(st, in, ORC_NFIELDS * sizeof(double));
  double p = st[ORC_P], rho = st[ORC_RHO], w = st[ORC_W];

  /* a2 */
  orc_satadj(p, &st[ORC_T], &st[ORC_QV], &st[ORC_QC]);

  /* a3: aerosol activated from the population carried as n_a + n_c; the
     cloud number is raised to N_act, taking the difference from n_a. */
  if (w > 0.0 && st[ORC_QC] > QMIN) {
    double N = rho * (st[ORC_NA] + st[ORC_NC]);
    double nact = orc_arg_nact(N, w, st[ORC_T], p);
    double dn = nact / rho - st[ORC_NC];
    if (dn < 0.0) dn = 0.0;
    if (dn > st[ORC_NA]) dn = st[ORC_NA];
    st[ORC_NC] += dn;
    st[ORC_NA] -= dn;
  }
}

static const int ICE_FIELDS[6] = {ORC_QI, ORC_QS, ORC_QG, ORC_NI, ORC_NS, ORC_NG};

/* what the aerosol-mass bookkeeping needs from one point's step */
typedef struct {
  double qc0, evap;         /* cloud before adjustment; cloud evaporated by it (>= 0) */
  double na0, dn_act;       /* free aerosol number before activation; droplets activated */
  double qc_post, qr_post;  /* cloud and rain after activation (what the rates see) */
  double tau_cr, tau_rv;    /* cloud -> rain (autoconversion + accretion), rain -> vapour */
  double tau_aut, nr_aut;   /* autoconversion: rain mass, new drops */
  double nuc_q, nuc_n;      /* ice nucleation: mass and crystals made */
  double tau_rim;           /* cloud -> graupel by riming (snow and graupel collecting cloud) */
  double sub_q[3];          /* sublimation of i, s, g: mass returned to vapour */
  double melt_q[3], melt_n[3];  /* melting of i, s, g into rain: mass and particles */
} orc_record;

static void point_core(const double *in0, double dt, double *out, int warm, orc_record *rec, const double *mu4) {
  /* warm: the ice fields are not part of the warm state; they are treated as
     absent and passed through unchanged */
  double in[ORC_NFIELDS];
  memcpy(in, in0, sizeof in);
  if (warm)
    for (int i = 0; i < 6; ++i) in[ICE_FIELDS[i]] = 0.0;
  double st[ORC_NFIELDS];
  orc_adjust_activate(in, st);
  if (rec) {
    /* the adjustment changes T, qv, qc only; activation nc and na only */
    double T = in[ORC_T], qv = in[ORC_QV], qc = in[ORC_QC];
    orc_satadj(in[ORC_P], &T, &qv, &qc);
    rec->qc0 = in[ORC_QC];
    rec->evap = in[ORC_QC] > qc ? in[ORC_QC] - qc : 0.0;
    rec->na0 = in[ORC_NA];
    rec->dn_act = in[ORC_NA] - st[ORC_NA];
    rec->qc_post = st[ORC_QC];
    rec->qr_post = st[ORC_QR];
    rec->tau_cr = rec->tau_rv = rec->tau_aut = rec->nr_aut = 0.0;
    rec->nuc_q = rec->nuc_n = rec->tau_rim = 0.0;
    for (int m = 0; m < 3; ++m) rec->melt_q[m] = rec->melt_n[m] = rec->sub_q[m] = 0.0;
  }

  /* a4..a9 from the post-activation state */
  double R[ORC_NPROC];
  rates_core(st, dt, R, warm, mu4);

  double qc = st[ORC_QC], qr = st[ORC_QR];
  orc_transfer tr[ORC_NPROC];
  int nt = 0;
#define ADD(rt, ms, md, ns, nsk, nd, nso, ht) \
  do { tr[nt].rate = (rt); tr[nt].msrc = (ms); tr[nt].mdst = (md); tr[nt].nsrc = (ns); \
       tr[nt].nsink = (nsk); tr[nt].ndst = (nd); tr[nt].nsource = (nso); tr[nt].heat = (ht); ++nt; } while (0)
  double rc = qc > QMIN ? ratio(st[ORC_NC], qc) : 0.0;
  double rr = qr > QMIN ? ratio(st[ORC_NR], qr) : 0.0;
  double mr0 = 4.0 / 3.0 * PI * RHOW * RR0 * RR0 * RR0;
  ADD(R[ORC_AUT], ORC_QC, ORC_QR, ORC_NC, R[ORC_AUT] * rc, ORC_NR, R[ORC_AUT] / mr0, 0.0);
  ADD(R[ORC_ACC], ORC_QC, ORC_QR, ORC_NC, R[ORC_ACC] * rc, -1, 0.0, 0.0);
  ADD(0.0, -1, -1, ORC_NC, R[ORC_SCC], -1, 0.0, 0.0);
  ADD(0.0, -1, -1, ORC_NR, R[ORC_SCR], -1, 0.0, 0.0);
  ADD(R[ORC_EVR], ORC_QR, ORC_QV, ORC_NR, R[ORC_EVR] * rr, -1, 0.0, -LV);
  ADD(R[ORC_NUC] * MI0, ORC_QV, ORC_QI, -1, 0.0, ORC_NI, R[ORC_NUC], LS);
  static const int qx[3] = {ORC_QI, ORC_QS, ORC_QG};
  static const int nx[3] = {ORC_NI, ORC_NS, ORC_NG};
  for (int m = 0; m < 3; ++m) {
    double d = R[ORC_DEPI + m];
    if (d >= 0.0) {
      ADD(d, ORC_QV, qx[m], -1, 0.0, -1, 0.0, LS);
    } else {
      double q = st[qx[m]];
      ADD(-d, qx[m], ORC_QV, nx[m], -d * ratio(st[nx[m]], q), -1, 0.0, -LS);
    }
  }
  ADD(R[ORC_RIMS], ORC_QC, ORC_QG, ORC_NC, R[ORC_RIMS] * rc, -1, 0.0, LF);
  ADD(R[ORC_RIMG], ORC_QC, ORC_QG, ORC_NC, R[ORC_RIMG] * rc, -1, 0.0, LF);
  for (int m = 0; m < 3; ++m) {
    double r = R[ORC_MLTI + m];
    double q = st[qx[m]];
    double nq = r > 0.0 ? r * ratio(st[nx[m]], q) : 0.0;
    ADD(r, qx[m], ORC_QR, nx[m], nq, ORC_NR, nq, -LF);
  }
#undef ADD

  /* Sinks per pool; f_X = min(1, X / (S_X dt)); each transfer is scaled by
     the smallest f over the pools it draws from, then applied once: taken
     from its source and given to its destination. */
  double S[ORC_NPROG], f[ORC_NPROG];
  for (int x = 0; x < ORC_NPROG; ++x) S[x] = 0.0;
  for (int j = 0; j < nt; ++j) {
    if (tr[j].rate > 0.0) S[tr[j].msrc] += tr[j].rate;
    if (tr[j].nsink > 0.0) S[tr[j].nsrc] += tr[j].nsink;
  }
  for (int x = 0; x < ORC_NPROG; ++x) {
    double X = st[x];
    f[x] = 1.0;
    if (S[x] * dt > X) f[x] = (X > 0.0 ? X : 0.0) / (S[x] * dt);
  }
  for (int j = 0; j < nt; ++j) {
    double g = 1.0;
    if (tr[j].rate > 0.0 && f[tr[j].msrc] < g) g = f[tr[j].msrc];
    if (tr[j].nsink > 0.0 && f[tr[j].nsrc] < g) g = f[tr[j].nsrc];
    if (tr[j].rate > 0.0) {
      double tau = g * tr[j].rate * dt;
      st[tr[j].msrc] -= tau;
      st[tr[j].mdst] += tau;
      st[ORC_T] += tau * tr[j].heat / CP;
      if (rec && (j == 0 || j == 1)) rec->tau_cr += tau;   /* autoconversion, accretion */
      if (rec && j == 0) rec->tau_aut = tau;
      if (rec && j == 4) rec->tau_rv += tau;               /* rain evaporation */
      if (rec && j == 5) rec->nuc_q = tau;                 /* nucleation */
      if (rec && j >= 6 && j <= 8 && tr[j].mdst == ORC_QV) rec->sub_q[j - 6] = tau;   /* sublimation */
      if (rec && (j == 9 || j == 10)) rec->tau_rim += tau; /* riming by snow and graupel */
      if (rec && j >= nt - 3) rec->melt_q[j - (nt - 3)] = tau;   /* melting of i, s, g */
    }
    if (tr[j].nsink > 0.0) st[tr[j].nsrc] -= g * tr[j].nsink * dt;
    if (tr[j].ndst >= 0 && tr[j].nsource > 0.0) {
      st[tr[j].ndst] += g * tr[j].nsource * dt;
      if (rec && j == 0) rec->nr_aut = g * tr[j].nsource * dt;
      if (rec && j == 5) rec->nuc_n = g * tr[j].nsource * dt;
      if (rec && j >= nt - 3) rec->melt_n[j - (nt - 3)] = g * tr[j].nsource * dt;
    }
  }
  if (warm)
    for (int i = 0; i < 6; ++i) st[ICE_FIELDS[i]] = in0[ICE_FIELDS[i]];
  memcpy(out, st, ORC_NPROG * sizeof(double));
}

void orc_point_cfg(const double *in, double dt, double *out, int warm) {
  point_core(in, dt, out, warm, NULL, NULL);
}

/* Triple-moment rain in the warm configuration (Section 2: CASIM is a
   three-moment scheme): the rain's sixth moment z (m^6 per kg of air) is the
   third prognostic moment.  The step's rates see the shape parameter
   diagnosed from the input (orc_rain_mu); z then changes as
     - accretion, self-collection and evaporation act at that fixed shape:
       z' = z (q'/q)^2 (n/n'), q', n' the rain without the autoconversion
       part (the shape measure G = z n / M3^2 unchanged);
     - autoconversion adds drops of one size D0 = 2 r0: + n_aut D0^6.
   in[ORC_NFIELDS_3M] -> out[ORC_NPROG_3M] (13 prognostic fields, then z). */
/* a1, the activity flag: a point is active when it holds a hydrometeor
   (q > q_min), is supersaturated over liquid, or (cold configuration) is
   colder than T_nuc and supersaturated over ice; the chain leaves every
   other point unchanged.  The fixed-shape rule for a sixth moment (z_kept:
   none left where the species is absent) acts at active points only, so an
   inactive point keeps its sixth moments too. */
static int point_active(const double *in, int warm) {
  if (in[ORC_QC] > QMIN || in[ORC_QR] > QMIN) return 1;
  if (in[ORC_QV] > orc_qsat(orc_es_liq(in[ORC_T]), in[ORC_P])) return 1;
  if (warm) return 0;
  if (in[ORC_QI] > QMIN || in[ORC_QS] > QMIN || in[ORC_QG] > QMIN) return 1;
  return in[ORC_T] < TNUC && in[ORC_QV] / orc_qsat(orc_es_ice(in[ORC_T]), in[ORC_P]) > 1.0;
}

void orc_point_3m(const double *in, double dt, double *out) {
  if (!point_active(in, 1)) {
    memcpy(out, in, ORC_NPROG * sizeof(double));
    out[ORC_NPROG] = in[ORC_ZR];
    return;
  }
  double mu4[4] = {orc_rain_mu(in[ORC_QR], in[ORC_NR], in[ORC_ZR]), SP[ORC_I].mu, SP[ORC_S].mu, SP[ORC_G].mu};
  orc_record r;
  double o[ORC_NPROG];
  point_core(in, dt, o, 1, &r, mu4);
  memcpy(out, o, sizeof o);
  double q0 = in[ORC_QR], n0 = in[ORC_NR], z0 = in[ORC_ZR];
  double q1 = o[ORC_QR] - r.tau_aut, n1 = o[ORC_NR] - r.nr_aut;
  double z = 0.0;
  if (q0 > QMIN && n0 > 0.0 && q1 > 0.0 && n1 > 0.0) z = z0 * (q1 / q0) * (q1 / q0) * (n0 / n1);
  double d0 = 2.0 * RR0, d3 = d0 * d0 * d0;
  out[ORC_NPROG] = z + r.nr_aut * (d3 * d3);
}

/* the fixed-shape part of a sixth moment after the processes: z (q1/q0)^2
   (n0/n1), q0, n0 what the rates saw, q1, n1 the result without the source
   terms (zero where any of them is not positive) */
static double z_kept(double z0, double q0, double n0, double q1, double n1) {
  if (q0 > QMIN && n0 > 0.0 && q1 > 0.0 && n1 > 0.0) return z0 * (q1 / q0) * (q1 / q0) * (n0 / n1);
  return 0.0;
}

/* Triple-moment scheme in the cold configuration: every sedimenting species
   x in r, i, s, g carries its sixth moment z_x (fields ORC_ZR..ORC_ZG), each
   rate sees the shape diagnosed per species from the input, and
     - processes that keep a species' shape (accretion, self-collection,
       evaporation, deposition, sublimation, riming, loss by melting) scale
       its z as z (q'/q)^2 (n/n');
     - sources add the sixth moment of what they add (moments of superposed
       populations add): autoconversion n_aut (2 r0)^6 to rain; nucleation
       n_nuc (m_i0 / a_i)^2 to ice; melting of species m gives rain the
       melted fraction of its sixth moment in rain diameters, (a_m / a_r)^2
       (tau_m / q_m) z_m, a particle of mass m having (m / a_r)^2.
   in[ORC_NFIELDS_3MC] -> out[ORC_NPROG_3MC] (13 prognostic fields, then
   z_r, z_i, z_s, z_g). */
void orc_point_3m_cold(const double *in, double dt, double *out) {
  if (!point_active(in, 0)) {
    memcpy(out, in, ORC_NPROG * sizeof(double));
    for (int x = 0; x < 4; ++x) out[ORC_NPROG + x] = in[ORC_ZR + x];
    return;
  }
  static const int sp[4] = {ORC_R, ORC_I, ORC_S, ORC_G};
  static const int qf[4] = {ORC_QR, ORC_QI, ORC_QS, ORC_QG};
  static const int nf[4] = {ORC_NR, ORC_NI, ORC_NS, ORC_NG};
  double mu4[4];
  for (int x = 0; x < 4; ++x) mu4[x] = orc_shape_mu(sp[x], in[qf[x]], in[nf[x]], in[ORC_ZR + x]);
  orc_record r;
  double o[ORC_NPROG];
  point_core(in, dt, o, 0, &r, mu4);
  memcpy(out, o, sizeof o);
  /* rain: the adjustment and activation leave it unchanged, so the rates saw the input */
  double q1 = o[ORC_QR] - r.tau_aut, n1 = o[ORC_NR] - r.nr_aut, zsrc = 0.0;
  for (int m = 0; m < 3; ++m) {
    q1 -= r.melt_q[m];
    n1 -= r.melt_n[m];
    const double q0m = in[qf[1 + m]];
    if (r.melt_q[m] > 0.0 && q0m > QMIN) {
      const double ar = SP[sp[1 + m]].a / SP[ORC_R].a;
      zsrc += ar * ar * (r.melt_q[m] / q0m) * in[ORC_ZR + 1 + m];
    }
  }
  const double d0 = 2.0 * RR0, d3 = d0 * d0 * d0;
  out[ORC_NPROG] = z_kept(in[ORC_ZR], in[ORC_QR], in[ORC_NR], q1, n1) + r.nr_aut * (d3 * d3) + zsrc;
  /* ice species */
  for (int m = 0; m < 3; ++m) {
    double q1m = o[qf[1 + m]], n1m = o[nf[1 + m]], src = 0.0;
    if (m == 0) {
      q1m -= r.nuc_q;
      n1m -= r.nuc_n;
      const double di = MI0 / SP[ORC_I].a;
      src = r.nuc_n * di * di;
    }
    out[ORC_NPROG + 1 + m] = z_kept(in[ORC_ZR + 1 + m], in[qf[1 + m]], in[nf[1 + m]], q1m, n1m) + src;
  }
}

void orc_rates(const double *st, double dt, double *R) { orc_rates_cfg(st, dt, R, 0); }

void orc_point(const double *in, double dt, double *out) { orc_point_cfg(in, dt, out, 0); }

/* Activated-aerosol mass (Section 2: once activated, aerosol mass is carried
   in the cloud and returned to the air when the water evaporates).  Three
   mass mixing ratios -- free aerosol ma, aerosol in cloud droplets mac, in
   rain mac -- move with the water in the warm configuration:
     a2 the cloud the adjustment evaporates returns its share of mac to ma;
     a3 activated droplets take the free aerosol's mean particle mass,
        ma dn / na (na before activation);
     a4 autoconversion and accretion carry mac into rain in proportion to the
        cloud water they move (fraction of the post-activation cloud);
     a5 rain evaporation returns mar to ma in proportion to the rain it
        evaporates;
     a12 mar sediments with the rain's mass-weighted fall speed.
   Water, numbers and temperature are those of the warm step, unchanged.
   in[ORC_NFIELDS_AERO] -> out[ORC_NPROG_AERO]. */
void orc_point_aero(const double *in, double dt, double *out) {
  orc_record r;
  double o[ORC_NPROG];
  point_core(in, dt, o, 1, &r, NULL);
  memcpy(out, o, sizeof o);
  double ma = in[ORC_MA], mac = in[ORC_MAC], mar = in[ORC_MAR], d;
  if (r.evap > 0.0 && r.qc0 > 0.0) {
    d = r.evap >= r.qc0 ? mac : mac * (r.evap / r.qc0);
    mac -= d;
    ma += d;
  }
  if (r.dn_act > 0.0 && r.na0 > 0.0) {
    d = ma * (r.dn_act / r.na0);
    ma -= d;
    mac += d;
  }
  if (r.tau_cr > 0.0 && r.qc_post > 0.0) {
    d = r.tau_cr >= r.qc_post ? mac : mac * (r.tau_cr / r.qc_post);
    mac -= d;
    mar += d;
  }
  if (r.tau_rv > 0.0 && r.qr_post > 0.0) {
    d = r.tau_rv >= r.qr_post ? mar : mar * (r.tau_rv / r.qr_post);
    mar -= d;
    ma += d;
  }
  out[ORC_NPROG + 0] = ma;
  out[ORC_NPROG + 1] = mac;
  out[ORC_NPROG + 2] = mar;
}

/* Activated-aerosol mass in the cold configuration: six mass mixing ratios,
   free aerosol ma and aerosol in cloud mac, rain mar, ice mai, snow mas,
   graupel mag.  Beyond the warm configuration's moves (the adjustment returns
   evaporated cloud's share to ma; activation takes ma dn/na; rain
   evaporation returns mar in proportion):
     cloud sinks: autoconversion and accretion carry mac to rain, riming by
        snow and graupel carries it to graupel (rimed mass goes to graupel),
        together as the fraction (tau_cr + tau_rim) / q_c of the
        post-activation cloud, split in proportion to the water;
     ice species m: sublimation returns its aerosol to ma, melting gives it
        to rain, together as the fraction (sub_m + melt_m) / q_m, split in
        proportion (after rain evaporation, so aerosol melted into rain this
        step is not evaporated with it);
     nucleated crystals carry no aerosol mass (the ice nuclei are not a
        tracked population); deposition and self-collection move none.
   Each species' aerosol sediments with that species' mass-weighted speed.
   in[ORC_NFIELDS_AEROC] -> out[ORC_NPROG_AEROC]. */
void orc_point_aero_cold(const double *in, double dt, double *out) {
  static const int qf[3] = {ORC_QI, ORC_QS, ORC_QG};
  orc_record r;
  double o[ORC_NPROG];
  point_core(in, dt, o, 0, &r, NULL);
  memcpy(out, o, sizeof o);
  double ma = in[ORC_MA], mac = in[ORC_MAC], mar = in[ORC_MAR], d;
  double mx[3] = {in[ORC_MAI], in[ORC_MAS], in[ORC_MAG]};
  if (r.evap > 0.0 && r.qc0 > 0.0) {
    d = r.evap >= r.qc0 ? mac : mac * (r.evap / r.qc0);
    mac -= d;
    ma += d;
  }
  if (r.dn_act > 0.0 && r.na0 > 0.0) {
    d = ma * (r.dn_act / r.na0);
    ma -= d;
    mac += d;
  }
  const double cs = r.tau_cr + r.tau_rim;
  if (cs > 0.0 && r.qc_post > 0.0) {
    d = cs >= r.qc_post ? mac : mac * (cs / r.qc_post);
    mac -= d;
    const double dg = d * (r.tau_rim / cs);
    mx[2] += dg;
    mar += d - dg;
  }
  if (r.tau_rv > 0.0 && r.qr_post > 0.0) {
    d = r.tau_rv >= r.qr_post ? mar : mar * (r.tau_rv / r.qr_post);
    mar -= d;
    ma += d;
  }
  for (int m = 0; m < 3; ++m) {
    const double q0 = in[qf[m]], sk = r.sub_q[m] + r.melt_q[m];
    if (sk > 0.0 && q0 > 0.0) {
      d = sk >= q0 ? mx[m] : mx[m] * (sk / q0);
      mx[m] -= d;
      const double dm = d * (r.melt_q[m] / sk);
      mar += dm;
      ma += d - dm;
    }
  }
  out[ORC_NPROG + 0] = ma;
  out[ORC_NPROG + 1] = mac;
  out[ORC_NPROG + 2] = mar;
  for (int m = 0; m < 3; ++m) out[ORC_NPROG + 3 + m] = mx[m];
}

/* ------------------------------------------------------ a12 sedimentation */
static unsigned sediment_species(double *q, double *n, const double *rho, const double *dz, int nlev, double dt,
                                 double *precip, int *nsub, int nspecies, double *aer, double *aprecip,
                                 double *zr);

unsigned orc_sediment_column(double *q, double *n, const double *rho, const double *dz,
                             int nlev, double dt, double *precip, int *nsub) {
  return sediment_species(q, n, rho, dz, nlev, dt, precip, nsub, 4, NULL, NULL, NULL);
}

unsigned orc_sediment_rain_3m(double *q, double *n, double *z, const double *rho, const double *dz, int nlev,
                              double dt, double *precip, int *nsub) {
  return sediment_species(q, n, rho, dz, nlev, dt, precip, nsub, 1, NULL, NULL, z);
}

unsigned orc_sediment_3m(double *q, double *n, double *z, const double *rho, const double *dz, int nlev, double dt,
                         double *precip, int *nsub) {
  return sediment_species(q, n, rho, dz, nlev, dt, precip, nsub, 4, NULL, NULL, z);
}

/* the first nspecies of r, i, s, g (warm configuration: rain only); aer (may
   be NULL): aerosol mass in the species (nspecies arrays of nlev), each moved
   with its species' mass-weighted speed, the surface fluxes accumulated in
   *aprecip; zr (may be NULL): the species'
   sixth moments (triple-moment scheme; nspecies arrays of nlev), each moved
   with its sixth-moment-weighted speed, every speed of the species then
   taken at the shape diagnosed per level and substep */
static unsigned sediment_species(double *q, double *n, const double *rho, const double *dz, int nlev, double dt,
                                 double *precip, int *nsub, int nspecies, double *aer, double *aprecip,
                                 double *zr) {
  /* For x in r, i, s, g: F_k = rho_k q_k Vq_k (mass), G_k = rho_k n_k Vn_k
     (number), fluxes downward.  Per substep of length dt/n_sub, with all
     fluxes taken from the substep's starting state:
        X_k += dts (F_{k+1} - F_k) / (rho_k dz_k),  F_nlev = 0,
        precip += F_0 dts.
     n_sub = max(1, ceil(max_k Vq_k dt / dz_k / C_max)) from the state
     entering sedimentation; capped at ORC_NSUB_MAX (error bit).  Speeds are
     recomputed from the updated q, n at every substep, and limited to
     dz_k / dts so that no level can be emptied below zero. */
  static const int spx[4] = {ORC_R, ORC_I, ORC_S, ORC_G};
  unsigned err = 0;
  double *F = (double *)malloc(sizeof(double) * (size_t)(nlev + 1));
  double *G = (double *)malloc(sizeof(double) * (size_t)(nlev + 1));
  double *A = (double *)malloc(sizeof(double) * (size_t)(nlev + 1));
  double *H = (double *)malloc(sizeof(double) * (size_t)(nlev + 1));
  for (int m = 0; m < nspecies; ++m) {
    int sp = spx[m];
    double *qq = q + (size_t)m * nlev, *nn = n + (size_t)m * nlev;
    const int tri = zr != NULL;
    double *zz = tri ? zr + (size_t)m * nlev : NULL;
    double cmax = 0.0;
    for (int k = 0; k < nlev; ++k) {
      if (!(qq[k] > QMIN)) continue;
      double mu = tri ? orc_shape_mu(sp, qq[k], nn[k], zz[k]) : SP[sp].mu;
      double lam = orc_lambda_mu(sp, qq[k], nn[k], mu);
      double c = orc_vq_mu(sp, rho[k], lam, mu) * dt / dz[k];
      if (c > cmax) cmax = c;
    }
    int ns = (int)ceil(cmax / CMAX);
    if (ns < 1) ns = 1;
    if (ns > ORC_NSUB_MAX) { ns = ORC_NSUB_MAX; err |= ORC_ERR_CFL; }
    if (nsub) nsub[m] = ns;
    double dts = dt / ns;
    for (int s = 0; s < ns; ++s) {
      const int with_aer = aer != NULL;
      double *am = with_aer ? aer + (size_t)m * nlev : NULL;
      for (int k = 0; k < nlev; ++k) {
        F[k] = 0.0;
        G[k] = 0.0;
        A[k] = 0.0;
        H[k] = 0.0;
        if (qq[k] > QMIN) {
          double mu = tri ? orc_shape_mu(sp, qq[k], nn[k], zz[k]) : SP[sp].mu;
          double lam = orc_lambda_mu(sp, qq[k], nn[k], mu);
          /* a level never loses more than it holds within one substep: the
             speed is limited to dz_k / dts (binds only when a later substep's
             speeds exceed the maximum that set n_sub) */
          double vlim = dz[k] / dts;
          double vq = orc_vq_mu(sp, rho[k], lam, mu), vn = orc_vn_mu(sp, rho[k], lam, mu);
          if (vq > vlim) vq = vlim;
          if (vn > vlim) vn = vlim;
          F[k] = rho[k] * qq[k] * vq;
          G[k] = rho[k] * (nn[k] > 0.0 ? nn[k] : 0.0) * vn;
          if (with_aer) A[k] = rho[k] * am[k] * vq;
          if (tri) {
            double vz = orc_vz_mu(sp, rho[k], lam, mu);
            if (vz > vlim) vz = vlim;
            H[k] = rho[k] * (zz[k] > 0.0 ? zz[k] : 0.0) * vz;
          }
        }
      }
      F[nlev] = 0.0;
      G[nlev] = 0.0;
      A[nlev] = 0.0;
      H[nlev] = 0.0;
      for (int k = 0; k < nlev; ++k) {
        qq[k] += dts * (F[k + 1] - F[k]) / (rho[k] * dz[k]);
        nn[k] += dts * (G[k + 1] - G[k]) / (rho[k] * dz[k]);
        if (with_aer) am[k] += dts * (A[k + 1] - A[k]) / (rho[k] * dz[k]);
        if (tri) zz[k] += dts * (H[k + 1] - H[k]) / (rho[k] * dz[k]);
      }
      precip[m] += F[0] * dts;
      if (with_aer) *aprecip += A[0] * dts;
    }
  }
  free(F);
  free(G);
  free(A);
  free(H);
  return err;
}

/* ----------------------------------------------------------- full step */
/* aero: the state has ORC_NFIELDS_AERO (warm) or ORC_NFIELDS_AEROC (cold)
   fields and precip 5 rows;
   tri: the state has ORC_NFIELDS_3M fields (warm) or ORC_NFIELDS_3MC (cold) */
static unsigned step_column(double *fld, long pitch, int nlev, int c, const double *dz,
                            double *precip, int *nsub, double dt, int warm, int aero, int tri) {
  unsigned err = 0;
  long fs = (long)nlev * pitch; /* field stride */
  const int nfields = aero ? (warm ? ORC_NFIELDS_AERO : ORC_NFIELDS_AEROC)
                            : tri ? (warm ? ORC_NFIELDS_3M : ORC_NFIELDS_3MC) : ORC_NFIELDS;
  const int nz = tri ? (warm ? 1 : 4) : 0;        /* sixth moments carried */
  const int na = aero ? (warm ? 1 : 4) : 0;       /* species carrying aerosol mass */
  double in[ORC_NFIELDS_AEROC], out[ORC_NPROG_AEROC];
  const int map[ORC_NPROG_AEROC] = {0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12,
                                    ORC_MA, ORC_MAC, ORC_MAR, ORC_MAI, ORC_MAS, ORC_MAG};
  for (int k = 0; k < nlev; ++k) {
    for (int f = 0; f < nfields; ++f) in[f] = fld[f * fs + (long)k * pitch + c];
    if (aero) {
      if (warm) orc_point_aero(in, dt, out);
      else orc_point_aero_cold(in, dt, out);
      const int nout = warm ? ORC_NPROG_AERO : ORC_NPROG_AEROC;
      for (int f = 0; f < nout; ++f) fld[map[f] * fs + (long)k * pitch + c] = out[f];
    } else if (tri) {
      if (warm) orc_point_3m(in, dt, out);
      else orc_point_3m_cold(in, dt, out);
      for (int f = 0; f < ORC_NPROG; ++f) fld[f * fs + (long)k * pitch + c] = out[f];
      for (int x = 0; x < nz; ++x) fld[(ORC_ZR + x) * fs + (long)k * pitch + c] = out[ORC_NPROG + x];
    } else {
      orc_point_cfg(in, dt, out, warm);
      for (int f = 0; f < ORC_NPROG; ++f) fld[f * fs + (long)k * pitch + c] = out[f];
    }
  }
  double *buf = (double *)malloc(sizeof(double) * (size_t)(17 * nlev));
  double *q = buf, *n = buf + 4 * nlev, *rho = buf + 8 * nlev, *aer = buf + 9 * nlev, *zr = buf + 13 * nlev;
  static const int qf[4] = {ORC_QR, ORC_QI, ORC_QS, ORC_QG};
  static const int nf[4] = {ORC_NR, ORC_NI, ORC_NS, ORC_NG};
  for (int k = 0; k < nlev; ++k) {
    rho[k] = fld[ORC_RHO * fs + (long)k * pitch + c];
    for (int x = 0; x < na; ++x) aer[x * nlev + k] = fld[(ORC_MAR + x) * fs + (long)k * pitch + c];
    for (int x = 0; x < nz; ++x) zr[x * nlev + k] = fld[(ORC_ZR + x) * fs + (long)k * pitch + c];
    for (int m = 0; m < 4; ++m) {
      q[m * nlev + k] = fld[qf[m] * fs + (long)k * pitch + c];
      n[m * nlev + k] = fld[nf[m] * fs + (long)k * pitch + c];
    }
  }
  double pr[4] = {0.0, 0.0, 0.0, 0.0};
  int ns[4] = {1, 1, 1, 1};
  const int nsp = warm ? 1 : 4;
  double apr = 0.0;
  err |= sediment_species(q, n, rho, dz, nlev, dt, pr, ns, nsp, aero ? aer : NULL, &apr, tri ? zr : NULL);
  for (int x = 0; x < nz; ++x)
    for (int k = 0; k < nlev; ++k) fld[(ORC_ZR + x) * fs + (long)k * pitch + c] = zr[x * nlev + k];
  if (aero) {
    for (int x = 0; x < na; ++x)
      for (int k = 0; k < nlev; ++k) fld[(ORC_MAR + x) * fs + (long)k * pitch + c] = aer[x * nlev + k];
    precip[4 * pitch + c] += apr;
  }
  for (int k = 0; k < nlev; ++k)
    for (int m = 0; m < nsp; ++m) {
      fld[qf[m] * fs + (long)k * pitch + c] = q[m * nlev + k];
      fld[nf[m] * fs + (long)k * pitch + c] = n[m * nlev + k];
    }
  for (int m = 0; m < 4; ++m) {
    precip[m * pitch + c] += pr[m];
    if (nsub) nsub[m * pitch + c] = ns[m];
  }
  free(buf);
  for (int k = 0; k < nlev; ++k) {
    for (int f = 0; f < ORC_NPROG; ++f)
      if (!isfinite(fld[f * fs + (long)k * pitch + c])) err |= ORC_ERR_NONFINITE;
    if (aero)
      for (int f = ORC_MA; f < ORC_MAR + na; ++f)
        if (!isfinite(fld[f * fs + (long)k * pitch + c])) err |= ORC_ERR_NONFINITE;
    for (int x = 0; x < nz; ++x)
      if (!isfinite(fld[(ORC_ZR + x) * fs + (long)k * pitch + c])) err |= ORC_ERR_NONFINITE;
  }
  return err;
}

unsigned orc_step_cfg(double *fld, long pitch, int ncols, int nlev, const double *dz,
                      double *precip, int *nsub, double dt, int nthreads, int warm) {
  unsigned err = 0;
  if (nlev <= 0 || ncols <= 0) return 0;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(guided) num_threads(nthreads) reduction(| : err)
#endif
  for (int c = 0; c < ncols; ++c) err |= step_column(fld, pitch, nlev, c, dz, precip, nsub, dt, warm, 0, 0);
  (void)nthreads;
  return err;
}

unsigned orc_step_aero(double *fld, long pitch, int ncols, int nlev, const double *dz,
                       double *precip, double dt, int nthreads) {
  unsigned err = 0;
  if (nlev <= 0 || ncols <= 0) return 0;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(guided) num_threads(nthreads) reduction(| : err)
#endif
  for (int c = 0; c < ncols; ++c) err |= step_column(fld, pitch, nlev, c, dz, precip, NULL, dt, 1, 1, 0);
  (void)nthreads;
  return err;
}

unsigned orc_step_3m(double *fld, long pitch, int ncols, int nlev, const double *dz, double *precip, double dt,
                     int nthreads) {
  unsigned err = 0;
  if (nlev <= 0 || ncols <= 0) return 0;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(guided) num_threads(nthreads) reduction(| : err)
#endif
  for (int c = 0; c < ncols; ++c) err |= step_column(fld, pitch, nlev, c, dz, precip, NULL, dt, 1, 0, 1);
  (void)nthreads;
  return err;
}

unsigned orc_step_aero_cold(double *fld, long pitch, int ncols, int nlev, const double *dz, double *precip,
                            double dt, int nthreads) {
  unsigned err = 0;
  if (nlev <= 0 || ncols <= 0) return 0;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(guided) num_threads(nthreads) reduction(| : err)
#endif
  for (int c = 0; c < ncols; ++c) err |= step_column(fld, pitch, nlev, c, dz, precip, NULL, dt, 0, 1, 0);
  (void)nthreads;
  return err;
}

unsigned orc_step_3m_cold(double *fld, long pitch, int ncols, int nlev, const double *dz, double *precip,
                          double dt, int nthreads) {
  unsigned err = 0;
  if (nlev <= 0 || ncols <= 0) return 0;
#ifdef _OPENMP
  if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(guided) num_threads(nthreads) reduction(| : err)
#endif
  for (int c = 0; c < ncols; ++c) err |= step_column(fld, pitch, nlev, c, dz, precip, NULL, dt, 0, 0, 1);
  (void)nthreads;
  return err;
}

unsigned orc_step(double *fld, long pitch, int ncols, int nlev, const double *dz,
                  double *precip, int *nsub, double dt, int nthreads) {
  return orc_step_cfg(fld, pitch, ncols, nlev, dz, precip, nsub, dt, nthreads, 0);
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* -------------------------------------------------------- parameter table */
double orc_param(const char *name) {
  const struct { const char *n; double v; } tab[] = {
    {"T0", T0}, {"cp", CP}, {"Lv", LV}, {"Lf", LF}, {"Rd", RD}, {"Rv", RV},
    {"g", GRAV}, {"rho_w", RHOW}, {"rho0", RHO0}, {"Ka", KA}, {"Dv", DV},
    {"mu_air", MUAIR}, {"q_min", QMIN}, {"T_nuc", TNUC}, {"m_i0", MI0}, {"r_r0", RR0},
    {"kk_aut", KK_AUT}, {"kk_aut_qc", KK_AUT_QC}, {"kk_aut_nc", KK_AUT_NC}, {"nc_min_cm3", NC_MIN_CM3},
    {"kk_acc", KK_ACC}, {"kk_acc_exp", KK_ACC_EXP}, {"kc_sb", KC_SB}, {"nu_c", NU_C}, {"kr_sb", KR_SB},
    {"mey_a", MEY_A}, {"mey_b", MEY_B}, {"mey_c", MEY_C}, {"arg_rm", ARG_RM},
    {"arg_sigma", ARG_SIGMA}, {"arg_kappa", ARG_KAPPA}, {"surft", SURFT}, {"Mw", MW},
    {"Ma", MA}, {"Rgas", RGAS}, {"e_rim", E_RIM}, {"c_max", CMAX},
    {"es_l0", ES_L0}, {"es_la", ES_LA}, {"es_lb", ES_LB},
    {"es_i0", ES_I0}, {"es_ia", ES_IA}, {"es_it", ES_IT}, {"es_ib", ES_IB},
  };

  for (size_t i = 0; i < sizeof(tab) / sizeof(tab[0]); ++i)
    if (strcmp(tab[i].n, name) == 0) return tab[i].v;
  /* species parameters: "<field>_<c|r|i|s|g>" */
  static const char *fn[] = {"a", "b", "mu", "cv", "dv", "vmax", "dmin", "dmax", "ccap"};
  static const char sc[] = "crisg";
  for (int s = 0; s < ORC_NSPECIES; ++s)
    for (int f = 0; f < 9; ++f) {
      char buf[16];
      size_t l = strlen(fn[f]);
      memcpy(buf, fn[f], l);
      buf[l] = '_';
      buf[l + 1] = sc[s];
      buf[l + 2] = 0;
      if (strcmp(buf, name) == 0) {
        const double *v = &SP[s].a;
        return v[f];
      }
    }
  return NAN;
}
