/*
 * FP64 CPU oracle of the column microphysics step -- TEST INFRASTRUCTURE.
 *
 * Only the tests, the package's smoke check and the benchmark's CPU-baseline
 * leg may load this library.  It shares no code with the CUDA path: it has
 * its own constants, its own formulas and its own layout handling.
 *
 * The step it defines (Section 2: independent columns, processes limited to
 * the vertical; Section 3.2: one column handled sequentially per call):
 *   a2 saturation adjustment -> a3 aerosol activation -> a4..a9 process rates
 *   -> a10 positivity/conservation limiter and forward-Euler update
 *   -> a12 CFL-substepped flux-form sedimentation.
 * The paper names these processes but prints no equations; every rate law
 * below follows a named published parameterisation, listed in casim_oracle.c.
 */
#ifndef CASIM_ORACLE_H
#define CASIM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Field order of the state (identical meaning to the product's state). */
enum {
  ORC_T = 0, ORC_QV, ORC_QC, ORC_QR, ORC_QI, ORC_QS, ORC_QG,
  ORC_NC, ORC_NR, ORC_NI, ORC_NS, ORC_NG, ORC_NA,
  ORC_P, ORC_RHO, ORC_W, ORC_NFIELDS
};
#define ORC_NPROG 13
/* Activated-aerosol mass extension (warm configuration): three more fields
   after the 16 above -- free aerosol mass ma, aerosol mass in cloud mac and in
   rain mar (kg/kg) -- and a fifth precipitation row (aerosol deposited). */
enum { ORC_MA = ORC_NFIELDS, ORC_MAC, ORC_MAR, ORC_NFIELDS_AERO };
#define ORC_NPROG_AERO (ORC_NPROG + 3)
/* Cold configuration: three more after those -- aerosol mass in ice mai,
   snow mas and graupel mag (the aerosol of r, i, s, g is fields 18..21). */
enum { ORC_MAI = ORC_NFIELDS_AERO, ORC_MAS, ORC_MAG, ORC_NFIELDS_AEROC };
#define ORC_NPROG_AEROC (ORC_NPROG + 6)
/* Triple-moment extension: the sixth moments z (m^6 per kg of air) after the
   16 fields above -- rain only in the warm configuration (17 fields), rain,
   ice, snow and graupel in the cold one (20 fields). */
enum { ORC_ZR = ORC_NFIELDS, ORC_NFIELDS_3M };
enum { ORC_ZI = ORC_NFIELDS_3M, ORC_ZS, ORC_ZG, ORC_NFIELDS_3MC };
#define ORC_NPROG_3M (ORC_NPROG + 1)
#define ORC_NPROG_3MC (ORC_NPROG + 4)

/* Hydrometeor species index. */
enum { ORC_C = 0, ORC_R, ORC_I, ORC_S, ORC_G, ORC_NSPECIES };

/* Process index (a4..a9). */
enum {
  ORC_AUT = 0, ORC_ACC, ORC_SCC, ORC_SCR, ORC_EVR, ORC_NUC,
  ORC_DEPI, ORC_DEPS, ORC_DEPG, ORC_RIMS, ORC_RIMG,
  ORC_MLTI, ORC_MLTS, ORC_MLTG, ORC_NPROC
};

/* Error bits returned by orc_step. */
#define ORC_ERR_NONFINITE 1u
#define ORC_ERR_CFL 2u
#define ORC_NSUB_MAX 64

double orc_es_liq(double T);
double orc_es_ice(double T);
double orc_qsat(double es, double p);
double orc_dqsat_liq_dT(double T, double p);
void   orc_satadj(double p, double *T, double *qv, double *qc);
double orc_arg_sm(double T);
double orc_arg_smax(double N, double w, double T, double p);
double orc_arg_nact(double N, double w, double T, double p);
double orc_lambda(int sp, double q, double n);
double orc_moment(int sp, double rho, double q, double lam, double k);
double orc_vent_integral(int sp, double rho, double q, double lam);
double orc_vq(int sp, double rho, double lam);
double orc_vn(int sp, double rho, double lam);
/* Raw process rates (before the limiter) at one point, from its state after
   adjustment and activation.  rates[ORC_NPROC]; see casim_oracle.c for signs. */
void   orc_rates(const double *st, double dt, double *rates);
/* a2 and a3 at one point: the state the process rates see, st[ORC_NFIELDS]. */
void   orc_adjust_activate(const double *in, double *st);
/* a2..a10 at one point: in[ORC_NFIELDS] -> out[ORC_NPROG]. */
void   orc_point(const double *in, double dt, double *out);
/* a12 for one column: q,n are [4][nlev] (r,i,s,g), updated in place;
   precip[4] accumulates (kg m^-2); nsub[4] receives the substep counts. */
unsigned orc_sediment_column(double *q, double *n, const double *rho, const double *dz,
                             int nlev, double dt, double *precip, int *nsub);
/* One full step over a domain.  fld is [ORC_NFIELDS][nlev][pitch] (column
   fastest), updated in place; precip is [4][pitch], accumulated; nsub (may be
   NULL) is [4][pitch].  nthreads <= 0 uses the OpenMP default. */
unsigned orc_step(double *fld, long pitch, int ncols, int nlev, const double *dz,
                  double *precip, int *nsub, double dt, int nthreads);
/* The warm configuration (warm != 0; Section 2.1: liquid water only): the
   ice fields are treated as absent and passed through unchanged; no
   nucleation, deposition, riming or melting; only rain sediments (ice, snow
   and graupel precipitation stay zero).  warm = 0 is the functions above. */
void   orc_rates_cfg(const double *st, double dt, double *rates, int warm);
void   orc_point_cfg(const double *in, double dt, double *out, int warm);
unsigned orc_step_cfg(double *fld, long pitch, int ncols, int nlev, const double *dz,
                      double *precip, int *nsub, double dt, int nthreads, int warm);
/* The warm configuration with activated-aerosol mass: in[ORC_NFIELDS_AERO]
   -> out[ORC_NPROG_AERO] (the 13 prognostic fields, then ma, mac, mar); and a
   step over fld[ORC_NFIELDS_AERO][nlev][pitch] with precip[5][pitch] (r, i,
   s, g, aerosol).  The first 16 fields and 4 precipitation rows are exactly
   those of orc_step_cfg(..., warm = 1). */
void   orc_point_aero(const double *in, double dt, double *out);
/* Gamma-distribution algebra with an explicit shape parameter mu (the
   functions without _mu use the species' fixed mu); the k-th-moment-weighted
   fall speeds for k = b (mass), 0 (number), 2b (sixth moment). */
double orc_lambda_mu(int sp, double q, double n, double mu);
double orc_moment_mu(int sp, double rho, double q, double lam, double k, double mu);
double orc_vent_integral_mu(int sp, double rho, double q, double lam, double mu);
double orc_vq_mu(int sp, double rho, double lam, double mu);
double orc_vn_mu(int sp, double rho, double lam, double mu);
double orc_vz_mu(int sp, double rho, double lam, double mu);
/* Triple-moment warm rain: the shape parameter diagnosed from q, n, z; a
   point in[ORC_NFIELDS_3M] -> out[ORC_NPROG_3M]; rain sedimentation of q, n,
   z (all [nlev]) with the per-level shape; a step over
   fld[ORC_NFIELDS_3M][nlev][pitch] with precip[4][pitch].  The first 16
   fields evolve as in the warm configuration, except that rain evaporation
   and the rain fall speeds use the diagnosed shape. */
double orc_rain_mu(double q, double n, double z);
/* the same for any species (all have mass exponent b = 3) */
double orc_shape_mu(int sp, double q, double n, double z);
/* The cold configuration with triple-moment r, i, s, g: a point
   in[ORC_NFIELDS_3MC] -> out[ORC_NPROG_3MC]; sedimentation of q, n, z for the
   four species ([4][nlev] each); a step over fld[ORC_NFIELDS_3MC][nlev][pitch]
   with precip[4][pitch].  Every rate and fall speed of a species takes its
   diagnosed shape. */
void   orc_point_3m_cold(const double *in, double dt, double *out);
unsigned orc_sediment_3m(double *q, double *n, double *z, const double *rho, const double *dz, int nlev, double dt,
                         double *precip, int *nsub);
unsigned orc_step_3m_cold(double *fld, long pitch, int ncols, int nlev, const double *dz, double *precip,
                          double dt, int nthreads);
void   orc_point_3m(const double *in, double dt, double *out);
unsigned orc_sediment_rain_3m(double *q, double *n, double *z, const double *rho, const double *dz, int nlev,
                              double dt, double *precip, int *nsub);
unsigned orc_step_3m(double *fld, long pitch, int ncols, int nlev, const double *dz, double *precip, double dt,
                     int nthreads);
unsigned orc_step_aero(double *fld, long pitch, int ncols, int nlev, const double *dz,
                       double *precip, double dt, int nthreads);
/* The cold configuration with activated-aerosol mass in cloud, rain and the
   ice species: in[ORC_NFIELDS_AEROC] -> out[ORC_NPROG_AEROC] (13 prognostic
   fields, then ma, mac, mar, mai, mas, mag); a step over
   fld[ORC_NFIELDS_AEROC][nlev][pitch] with precip[5][pitch].  The first 16
   fields and 4 precipitation rows are exactly those of orc_step. */
void   orc_point_aero_cold(const double *in, double dt, double *out);
unsigned orc_step_aero_cold(double *fld, long pitch, int ncols, int nlev, const double *dz,
                            double *precip, double dt, int nthreads);
/* Parameter lookup by name for the tests (returns NaN for an unknown name). */
double orc_param(const char *name);
int    orc_max_threads(void);

#ifdef __cplusplus
}
#endif
#endif
