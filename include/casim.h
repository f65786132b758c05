/*
 * casim.h -- C ABI of the GB300 column-microphysics step.
 *
 * The step advances independent atmospheric columns through one model
 * timestep of a bulk, double-moment cloud-microphysics scheme: saturation
 * adjustment, aerosol activation, warm-rain and ice process rates, a
 * positivity/conservation limiter, and CFL-substepped flux-form
 * sedimentation.  The paper (Brown et al., "Porting the microphysics model
 * CASIM to GPU and KNL Cray machines", Section 2) defines the structure:
 * columns are independent, every process acts in the vertical only, and each
 * hydrometeor carries a gamma-type size distribution.  Its Section 3.2 gives
 * the host protocol mirrored here: set-up once (initialise_micromain), one
 * call per timestep that runs the whole scheme for every column
 * (shipway_microphysics around CASIM()), tear-down (finalise_micromain).
 *
 * Conventions for every entry point:
 *  - All functions return CASIM_OK (0) or a negative CASIM_ERR_* code; they
 *    never abort the process and no kernel traps.  Device-side problems
 *    (non-finite results, substep cap reached) set bits in an error word kept
 *    by the context and read with casim_get_error().
 *  - Device pointers are plain CUDA device addresses (e.g. from a PyTorch
 *    tensor); the caller owns them.  `stream` is a cudaStream_t passed as
 *    void* (NULL = the legacy default stream).  Work is enqueued
 *    asynchronously on that stream.
 *  - State layout (level-major structure of arrays, column fastest):
 *      fld[f * nlev * pitch + k * pitch + c]
 *    f in [0, CASIM_NFIELDS) in the order of enum casim_field, k = 0 is the
 *    lowest level, c in [0, ncols).  pitch >= ncols and a multiple of 32;
 *    fld must be 256-byte aligned.  Columns ncols..pitch-1 are padding: they
 *    are never written and their contents are ignored.
 *  - Units: T in K; q* specific contents in kg/kg of moist air; n* numbers
 *    per kg of air; p in Pa; rho in kg/m^3; w in m/s; dz in m; dt in s;
 *    precipitation in kg/m^2.
 */
#ifndef CASIM_H
#define CASIM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CASIM_ABI_VERSION 1

enum casim_field {
  CASIM_T = 0, CASIM_QV, CASIM_QC, CASIM_QR, CASIM_QI, CASIM_QS, CASIM_QG,
  CASIM_NC, CASIM_NR, CASIM_NI, CASIM_NS, CASIM_NG, CASIM_NA,
  CASIM_P, CASIM_RHO, CASIM_W,
  CASIM_NFIELDS
};
#define CASIM_NPROG 13      /* fields T..NA are updated in place; p, rho, w are read only */
#define CASIM_NPRECIP 4     /* surface accumulators: rain, ice, snow, graupel */
#define CASIM_NSUB_MAX 64   /* sedimentation substep cap per column and species */

/* precision forms */
enum casim_precision {
  CASIM_FP64 = 0,   /* every operation in FP64 */
  CASIM_MIXED = 1   /* rates, fall speeds, special functions in FP32; FP64 for the
                       state, the vapour difference of saturation adjustment and
                       every mass transfer applied by the limiter */
};

/* return codes */
enum casim_status {
  CASIM_OK = 0,
  CASIM_ERR_ARG = -1,        /* invalid argument (null pointer, size, alignment) */
  CASIM_ERR_OOM = -2,        /* device allocation failed */
  CASIM_ERR_CUDA = -3,       /* a CUDA call failed (see casim_last_cuda_error) */
  CASIM_ERR_NONFINITE = -4,  /* casim_get_error: a non-finite value was produced */
  CASIM_ERR_CFL = -5,        /* casim_get_error: substep cap reached in sedimentation */
  CASIM_ERR_TIMEOUT = -6,    /* casim_get_error: a bounded wait inside the surrogate network's
                                kernel gave up; its rows were left to the scheme's rates */
  CASIM_ERR_IO = -7,         /* a checkpoint file could not be opened, read or written */
  CASIM_ERR_INDEX = -8       /* casim_get_error: the debug build (libcasim_debug.so) found an
                                index outside its array and skipped the access */
};

/* device error-word bits (casim_get_error) */
#define CASIM_EFLAG_NONFINITE 1u
#define CASIM_EFLAG_CFL 2u
#define CASIM_EFLAG_TIMEOUT 4u
#define CASIM_EFLAG_INDEX 8u   /* debug build only: an index check failed */

/* Scheme parameters.  casim_default_params() fills the published values the
   scheme is defined with; callers may change them before casim_init(). */
typedef struct {
  double T0, cp, Lv, Lf, Rd, Rv, g, rho_w, rho0, Ka, Dv, mu_air;
  double q_min;              /* species present iff q > q_min */
  double T_nuc, m_i0, r_r0;  /* nucleation threshold (K), crystal mass (kg), new-drop radius (m) */
  double kk_aut, kk_aut_qc, kk_aut_nc, nc_min_cm3, kk_acc, kk_acc_exp;
  double kc_sb, nu_c, kr_sb;
  double mey_a, mey_b, mey_c;
  double arg_rm, arg_sigma, arg_kappa, surft, Mw, Ma, Rgas;
  double e_rim, c_max;
  double es_l0, es_la, es_lb, es_i0, es_ia, es_it, es_ib;
  /* per species c, r, i, s, g: m(D) = a D^b; gamma shape mu; V(D) = cv D^dv
     (rho0/rho)^0.4 capped at vmax; mean diameter kept in [dmin, dmax];
     capacitance ccap * D */
  double a[5], b[5], mu[5], cv[5], dv[5], vmax[5], dmin[5], dmax[5], ccap[5];
} casim_params;

/* Caller-owned device state of one domain. */
typedef struct {
  double *fld;          /* [CASIM_NFIELDS][nlev][pitch], 256-byte aligned */
  long long pitch;      /* >= ncols, multiple of 32 */
  const double *dz;     /* [nlev] layer thickness, k = 0 lowest */
  double *precip;       /* [CASIM_NPRECIP][pitch] accumulated surface precipitation */
} casim_state;

typedef struct casim_ctx casim_ctx;

/* Fill *p with the default scheme parameters.  Returns CASIM_ERR_ARG if p is NULL. */
int casim_default_params(casim_params *p);

/* casim_init flag: the warm configuration (Section 2.1: liquid water only,
   5 moisture fields instead of the cold configuration's 18).  Steps read and
   write only T, qv, qc, qr, nc, nr, na (and read p, rho, w); the ice fields
   qi, qs, qg, ni, ns, ng are neither read nor written; no nucleation,
   deposition, riming or melting; only rain sediments.  On a state without
   ice and warmer than the nucleation threshold it gives the cold
   configuration's result.  Supported by casim_step, casim_step_host and
   casim_step_tendency (whose ice source terms are zero); the batched and
   surrogate entry points reject a warm context (CASIM_ERR_ARG). */
#define CASIM_WARM 1

/* casim_init flag (not with CASIM_THREE_MOMENT): activated-aerosol mass
   (Section 2: CASIM carries the mass of activated aerosol in the cloud and
   returns it to the air when the water evaporates).  With CASIM_WARM the
   state has 19 fields -- the 16 above, then ma (free aerosol mass), mac
   (aerosol mass in cloud droplets), mar (aerosol mass in rain), kg/kg;
   without it 22 fields -- then also mai, mas, mag (aerosol mass in ice,
   snow, graupel).  precip then has 5 rows, the fifth the aerosol mass
   deposited at the surface (kg m^-2).  Aerosol mass moves with the water:
   the cloud the adjustment evaporates returns its share of mac to ma;
   activated droplets take the free aerosol's mean particle mass
   ma * dn / na; autoconversion and accretion carry mac to rain, and (cold)
   riming by snow and graupel carries it to graupel, in proportion to the
   cloud water they move; rain evaporation returns mar to ma in proportion;
   (cold) sublimation returns, and melting passes on to rain, an ice
   species' aerosol in proportion to the mass it loses; nucleated crystals
   carry none; each species' aerosol sediments with its mass-weighted fall
   speed.  The other 16 fields and 4 precipitation rows evolve exactly as
   without aerosol mass.  Supported by casim_step, casim_step_tendency,
   casim_step_host (both precisions) and the checkpoint calls; the batched and
   surrogate entry points reject such a context (CASIM_ERR_ARG). */
#define CASIM_AEROSOL 2

/* casim_init flag (not with CASIM_AEROSOL): the triple-moment scheme
   (Section 2: CASIM is a three-moment bulk scheme).  Each sedimenting species
   x carries its sixth moment z_x (m^6 per kg of air; for rain the radar
   reflectivity factor per unit mass): with CASIM_WARM rain only, a 17-field
   state (the 16 above, then zr); without it r, i, s, g, a 20-field state
   (then zr, zi, zs, zg).  A species' shape parameter mu is diagnosed at every
   point from
     G = z n / (q/a)^2 = (mu+4)(mu+5)(mu+6) / ((mu+1)(mu+2)(mu+3))
   (mu in [0, 20]; the species' fixed mu where it is absent); its rates
   (evaporation, deposition, riming, melting) and fall speeds use that shape,
   and z sediments with the sixth-moment-weighted speed.  Processes that keep
   a species' shape change z as z (q'/q)^2 (n/n'); sources add the sixth
   moment of what they bring: autoconversion (2 r_r0)^6 per new drop,
   nucleation (m_i0 / a_i)^2 per new crystal, and melting of species m the
   melted fraction of z_m in rain diameters, (a_m / a_r)^2 (melted / q_m) z_m.
   Requires mass exponent b = 3 for those species.  Supported by casim_step
   (both precisions), casim_step_tendency, casim_step_host and the
   checkpoint calls; the batched and surrogate entry points reject such a
   context. */
#define CASIM_THREE_MOMENT 4

/* casim_init flag (standard configuration only: not with CASIM_WARM,
   CASIM_AEROSOL or CASIM_THREE_MOMENT): casim_step and casim_step_host also
   count per-step statistics, read by casim_get_stats.  The step then runs a
   statistics build of its kernel (one warp-aggregated atomic per counter and
   warp).  No paper counterpart: diagnostics of where the scheme acts. */
#define CASIM_STATS 8

/* Largest level count of a column (the step keeps a column's dz in shared
   memory). */
#define CASIM_MAX_LEV 1024

/* Create a context on the current CUDA device (Section 3.2: the one-off
   set-up that copies constants and allocates device memory).  `params` may be
   NULL for the defaults; `precision` is a casim_precision; `flags` is 0 or
   CASIM_WARM, optionally with one of CASIM_AEROSOL or CASIM_THREE_MOMENT
   (CASIM_ERR_ARG otherwise).  Allocates a small device error word.  On
   failure *ctx is set to NULL. */
int casim_init(casim_ctx **ctx, const casim_params *params, int precision, int flags);

/* Advance every column of one domain by one timestep dt, in place
   (Section 3.2: the per-timestep call running the whole scheme on the GPU).
   ncols >= 0 (0 is a no-op), 1 <= nlev <= CASIM_MAX_LEV, dt > 0 (else
   CASIM_ERR_ARG before any launch; the same limits hold for every entry point
   that takes ncols and nlev).  Updates the 13 prognostic
   fields and adds the step's surface precipitation to s->precip.  Reads
   s->dz on the device.  Asynchronous on `stream`. */
int casim_step(casim_ctx *ctx, const casim_state *s, int ncols, int nlev, double dt, void *stream);

/* Source-term mode: CASIM itself does not update the state but writes a
   source term per field for the parent model to add (Section 3.2: results go
   into source-term arguments for each q field; Section 3.1: source terms are
   copied back and integrated on the host).  The same step as casim_step, but
   s->fld is left unchanged and tend (device, [nfields - 3][nlev][s->pitch]
   for the context's state of nfields fields -- 13 rows for the standard
   state -- owned by the caller, not overlapping s->fld) receives
   (x_after - x_before) / dt of the 13 prognostic fields (rows 0..12) and of
   the configuration's fields after the inputs p, rho, w (field 16 + i in
   row 13 + i) at every point of the first ncols columns, where
   x_after is what casim_step would store (so x_before + tend * dt reproduces
   it to the rounding of the subtraction and division).  s->precip
   accumulates the step's surface precipitation as in casim_step.
   Asynchronous on `stream`; errors as casim_step, and CASIM_ERR_ARG for a
   NULL, misaligned or overlapping tend. */
int casim_step_tendency(casim_ctx *ctx, const casim_state *s, int ncols, int nlev, double dt, double *tend,
                        void *stream);

/* Same step for a domain held in HOST memory (the paper's per-step
   transfers, Section 3.3).  The state layout is the device one, with host
   pointers.  Two paths, chosen per call:
   - fields and precip each in pinned host memory mapped into the device's
     address space (cudaHostAlloc / cudaMallocHost, as torch's pin_memory()
     allocates, or a cudaHostRegister range) and host->fld 256-byte aligned,
     on a device that cannot register host memory read-only
     (cudaDevAttrHostRegisterReadOnlySupported = 0, as on GB300; where it can,
     a registered range cannot be told apart from a writable one and this path
     is not taken): the step kernel loads and stores the host state in
     place over the host link on `stream` (each input crosses once; written
     back are only the rows of 32 columns of the fields the step changed
     somewhere in them; dz is copied to the device);
   - otherwise (pageable or misaligned memory): copies.  A domain of more than
     65 536 columns is processed in column chunks of 65 536 (fewer if the
     state's fields x nlev of them exceed 2 GB) on three internal streams of
     the context, so one chunk's copy in (every field of the context's state,
     and precip), another's step and a third's copy out (the prognostic fields
     -- all but p, rho, w -- and precip) run at once; a smaller domain is
     copied whole on `stream`.
   Starts after the work already queued on `stream` and returns when the host
   state holds the result.  Results equal casim_step's on the same state, bit
   for bit, on either path.  Device buffers grow to the largest size seen and
   are freed by casim_free. */
int casim_step_host(casim_ctx *ctx, const casim_state *host, int ncols, int nlev, double dt,
                    void *stream);

/* Per-column FP64 budget sums, written to out[2][ncols] (device):
   out[0][c] = sum_k rho dz (qv+qc+qr+qi+qs+qg)   (kg/m^2)
   out[1][c] = sum_k rho dz (nc + na)              (aerosol + droplets, m^-2)
   Asynchronous on `stream`. */
int casim_budget(casim_ctx *ctx, const casim_state *s, int ncols, int nlev, double *out, void *stream);

/* Failure detection without a fault: run the bounded wait every
   tensor-core kernel uses on a barrier that nothing completes, with a limit
   of limit_ns (1 ns .. 2 s, the kernels' own limit; CASIM_ERR_ARG outside),
   so that it gives up; the kernel records that in the context's error word
   (casim_get_error then returns CASIM_ERR_TIMEOUT with CASIM_EFLAG_TIMEOUT)
   and the context stays usable.  Synchronises `stream`; *elapsed_ns
   receives how long the wait lasted on the device. */
int casim_wait_selftest(casim_ctx *ctx, long long limit_ns, long long *elapsed_ns, void *stream);

/* Wait for `stream`, read and clear the device error word.  *flags receives the
   CASIM_EFLAG_* bits (may be NULL).  Returns CASIM_OK, CASIM_ERR_NONFINITE or
   CASIM_ERR_CFL (the first set, in that order of precedence, after CASIM_ERR_INDEX
   and CASIM_ERR_TIMEOUT), or CASIM_ERR_CUDA. */
int casim_get_error(casim_ctx *ctx, unsigned *flags, void *stream);

/* Statistics counted by a CASIM_STATS context since casim_init or the last
   reset, over casim_step and casim_step_host calls. */
typedef struct {
  long long steps;            /* calls counted */
  long long points;           /* grid points stepped (sum of ncols x nlev) */
  long long active_points;    /* points the activity flag (any hydrometeor above q_min, or
                                 supersaturation over liquid, or over ice below T_nuc) sent
                                 through the processes */
  long long changed_points;   /* points the step changed (processes or sedimentation) */
  long long active_columns;   /* columns with at least one active point, summed over steps */
  long long nsub[4][65];      /* per sedimenting species r, i, s, g: columns whose sweep took
                                 n substeps, n = 1..64 (1 in the single-substep path and for a
                                 species absent from the column, as max(1, ceil(Courant))) */
} casim_stats;

/* Wait for `stream` and copy the statistics into *out; reset != 0 then sets
   them to zero.  CASIM_ERR_ARG if the context was not created with
   CASIM_STATS or out is NULL. */
int casim_get_stats(casim_ctx *ctx, casim_stats *out, int reset, void *stream);

/* ----------------------------------------------------------------------------
 * Batches: many independent domains advanced by one launch per step.
 * (Section 2: columns are independent, so domains of different sizes can share
 * one launch; Section 3.4: the best launch configuration depends on the
 * column count and must be found by experiment -- casim_batch_tune does so.)
 * ------------------------------------------------------------------------- */
typedef struct casim_batch casim_batch;

/* One measured candidate of casim_batch_tune. */
typedef struct {
  int block;          /* threads (columns) per block: 64, 128 or 256 */
  int compact;        /* 1: flag pass + active-column list, 0: every column */
  int persistent;     /* 1: one resident wave taking items from a counter, 0: one item per block */
  float ms_per_step;
} casim_tune_entry;

/* Describe ndom domains (device states as for casim_step; ncols[i] >= 0,
   1 <= nlev[i] <= 1024).  Reads every domain's dz once (they must not change
   afterwards), orders work by descending level count and allocates the
   batch's device scratch: a domain table, an active-column list of
   sum(ncols) ints, per-domain counts, a work counter.  The default launch
   configuration is block 128, compaction on, persistent grid. */
int casim_batch_create(casim_ctx *ctx, const casim_state *domains, const int *ncols, const int *nlev, int ndom,
                       casim_batch **batch);

/* Advance every domain of the batch by dt (asynchronous on `stream`): an
   optional flag/compaction launch and one step launch. Results are identical,
   bit for bit, to casim_step on each domain, for every launch configuration. */
int casim_batch_step(casim_ctx *ctx, casim_batch *batch, double dt, void *stream);

/* Set / read the launch configuration (invalidates a captured graph). */
int casim_batch_config(casim_batch *batch, int block, int compact, int persistent);
int casim_batch_get_config(const casim_batch *batch, int *block, int *compact, int *persistent);

/* Autotuner: times the 12 configurations (block 64/128/256 x compaction x
   persistent), each for 1 warm-up and `steps` timed steps, and keeps the
   fastest.  These are REAL timesteps of the batch: the state advances by
   casim_batch_tune_steps(steps) = 12 (steps + 1) steps.  Fills up to
   table_len entries of `table` (may be NULL when table_len is 0).
   Synchronises `stream`. */
int casim_batch_tune(casim_ctx *ctx, casim_batch *batch, double dt, int steps, void *stream,
                     casim_tune_entry *table, int table_len);
int casim_batch_tune_steps(int steps);

/* Capture nsteps steps of the batch (current configuration, this dt) into a
   CUDA graph held by the batch; casim_batch_graph_launch replays it on
   `stream`.  A new capture or configuration replaces the graph. */
int casim_batch_graph(casim_ctx *ctx, casim_batch *batch, double dt, int nsteps, void *stream);
int casim_batch_graph_launch(casim_batch *batch, void *stream);

/* One call per timestep for many domains (Section 3.2: the host makes one
   call per timestep, which runs the whole scheme for every column; here the
   columns of ndom domains of different sizes go in one launch).  Arguments
   as for casim_batch_create, plus dt (> 0, s) and `stream`.  Results are,
   bit for bit, those of casim_step on each domain.
   The context keeps the batch object of the last domain list it was given
   and reuses it while the same list comes back (same state pointers, pitches,
   ncols, nlev); a different list replaces it.  Building a batch reads every
   domain's dz and synchronises the device, so the first call with a list is
   not asynchronous; later calls with that list are (one or two launches on
   `stream`).  As for casim_batch_create, dz must not change while its list
   is in use; the launch configuration is the batch default (block 128,
   compaction, persistent grid); tune a batch object with casim_batch_tune
   where that matters.  The cached batch is released by casim_free.
   Errors: CASIM_ERR_ARG for invalid arguments or a context with CASIM_WARM,
   CASIM_AEROSOL or CASIM_THREE_MOMENT; CASIM_ERR_OOM; CASIM_ERR_CUDA. */
int casim_step_batched(casim_ctx *ctx, const casim_state *domains, const int *ncols, const int *nlev, int ndom,
                       double dt, void *stream);

/* Total columns of the batch (sum of ncols). */
long long casim_batch_columns(const casim_batch *batch);

/* Release the batch (waits for the device). NULL is a no-op. */
void casim_batch_free(casim_batch *batch);

/* ----------------------------------------------------------------------------
 * Warm-rain surrogate: a network 12 -> 256 -> 256 -> 256 -> 4 (tanh hidden
 * layers) that predicts the natural logarithms of autoconversion, accretion,
 * cloud and rain self-collection from 12 features of a point's state after
 * adjustment and activation.  Weights and every GEMM operand are BF16, sums
 * FP32 (tensor cores).  The paper has no learned component; the network, its
 * training and its guard follow the mixed form of the step.
 *
 * Features (in order): ln qc, ln qr (floored at q_min), ln nc (floored at 1),
 * ln nr (floored at 1e-3), ln rho, T - T0, ln p, ln qv (floored at 1e-10), w,
 * ln na (floored at 1), [qc > q_min], [qr > q_min].
 * Flat parameter order: W1[12][256], b1[256], W2[256][256], b2, W3[256][256],
 * b3, W4[256][4], b4[4]; W[k][n] multiplies input k into unit n.
 * ------------------------------------------------------------------------- */
typedef struct casim_mlp casim_mlp;
#define CASIM_MLP_NIN 12
#define CASIM_MLP_NOUT 4
#define CASIM_MLP_NSTATS (2 * CASIM_MLP_NIN + 2 * CASIM_MLP_NOUT + 2 * CASIM_MLP_NIN)

/* New network on the current device: Xavier-uniform weights from `seed`, zero biases. */
int casim_mlp_create(casim_mlp **mlp, unsigned long long seed);
long long casim_mlp_param_count(void);
/* FP32 master parameters, host arrays of casim_mlp_param_count() floats. */
int casim_mlp_set_params(casim_mlp *mlp, const float *host, long long n);
int casim_mlp_get_params(const casim_mlp *mlp, float *host, long long n);
/* Engine: 1 (default) = the tensor-core (tcgen05/TMEM) kernels -- inference
   and the training GEMMs (forward, data and weight gradients); 0 = the
   mma.sync GEMMs for both.  casim_mlp_fit and casim_mlp_loss_grad_host
   return CASIM_ERR_TIMEOUT if a bounded wait of a tensor-core kernel gave
   up (the error is cleared). */
int casim_mlp_set_engine(casim_mlp *mlp, int engine);
/* Standardised inputs Xn[n][12] -> outputs Y[n][4] (host arrays; synchronous;
   runs the selected engine). */
int casim_mlp_forward_host(casim_mlp *mlp, const float *Xn, int n, float *Y);
/* The same on DEVICE arrays: Xn[n][12] and Y[n][4], FP32 row-major, caller-
   owned; 1 <= n <= 2^27.  Launches on `stream` (the engine's input
   conversion, then the network), then synchronises that stream to read the
   kernel's bounded-wait flag: returns CASIM_ERR_CUDA if a wait gave up
   (outputs then undefined).  The tcgen05 engine keeps a BF16 input buffer of
   n x 32 bytes, grown on demand and freed by casim_mlp_free; the mma.sync
   engine uses the training workspace.  Y must not overlap Xn. */
int casim_mlp_forward(casim_mlp *mlp, const float *Xn, long long n, float *Y, void *stream);
/* Loss sum_i sum_j M (Y - Tn)^2 / sum M and its gradient (host arrays of
   n x 12, n x 4, n x 4, and param_count floats; synchronous). */
int casim_mlp_loss_grad_host(casim_mlp *mlp, const float *Xn, const float *Tn, const float *M, int n, double *loss,
                             float *grad);
/* Training data from one state (mixed form): for every point with cloud or
   rain after adjustment and activation, raw features X[row][12], the scheme's
   log-rates Y[row][4] and masks M[row][4] (1 where the scheme defines the
   rate), and (if pts is not NULL) the point index k * pitch + c of each row.
   Device buffers of `cap` rows; *rows receives the number of such points
   (rows beyond cap are not written).  Synchronises `stream`. */
int casim_mlp_data(casim_ctx *ctx, const casim_state *s, int ncols, int nlev, double dt, float *X, float *Y,
                   float *M, long long *pts, long long cap, long long *rows, void *stream);
/* Fit the standardisation and the input box to n rows of device data, then
   train with Adam (lr, betas 0.9/0.999) for `steps` mini-batches of `batch`
   rows drawn with a counter-based hash of (seed, step, row).  loss_hist
   (host, may be NULL) receives the loss of every step.  Synchronises `stream`. */
int casim_mlp_fit(casim_mlp *mlp, const float *X, const float *Y, const float *M, long long n, int steps, int batch,
                  float lr, unsigned long long seed, float *loss_hist, void *stream);
/* Standardisation and box: [12 mean][12 sd][4 mean][4 sd][12 lo][12 hi]. */
int casim_mlp_get_norm(const casim_mlp *mlp, float *stats);
int casim_mlp_set_norm(casim_mlp *mlp, const float *stats);
/* One mixed-form step in which the four warm-rain rates come from the network
   at every point whose features lie inside the training box, and from the
   scheme elsewhere (the out-of-distribution guard).  The context must be
   CASIM_MIXED.  Allocates the network's scratch on first use for a domain
   size (features, row map, per-point rates).  Synchronises `stream` once
   (to size the network's pass); *served (may be NULL) receives the number of
   points that took the network's rates. */
int casim_step_surrogate(casim_ctx *ctx, casim_mlp *mlp, const casim_state *s, int ncols, int nlev, double dt,
                         void *stream, long long *served);

/* Every domain of a batch advanced by dt with the surrogate's warm-rain
   rates where its guard admits the point (as casim_step_surrogate for each
   domain; the results are, bit for bit, those per-domain calls').  One
   feature pass over all the batch's points, one network launch over their
   rows, then the batch's step launch(es) in its configuration.  The
   context must be CASIM_MIXED and the batch's; the network fitted.
   Allocates the network's scratch on first use for the batch's point count
   (sum of nlev * pitch).  On the tensor-core engine (the default) the
   network reads the row count on the device, so the call only enqueues
   work; if `served` is non-NULL it waits for `stream` and stores the number
   of points that took the network's rates.  (No paper counterpart: the
   paper has no learned part.) */
int casim_batch_step_surrogate(casim_ctx *ctx, casim_batch *batch, casim_mlp *mlp, double dt, void *stream,
                               long long *served);
void casim_mlp_free(casim_mlp *mlp);

/* ----------------------------------------------------------------------------
 * Allocation-free step.  The paper has no counterpart; this entry point exists
 * for callers that cannot allocate device memory: a host model whose memory
 * pool already owns the GPU, a plug-in called while its framework forbids
 * allocation, or a real-time loop that must never meet a failed allocation.
 * It needs no context and calls no cudaMalloc or cudaFree (nor any routine
 * that allocates): its scratch -- the error word, a work counter, the domain
 * table and the active-column list -- is one fixed array of device memory
 * that the library holds on every GPU it is loaded on, until the process
 * exits (about 4.2 MB for the limit below).
 *  - Runs the compacted step (flag pass, then the step over the active
 *    columns); results are bit-for-bit those of casim_step with the same
 *    parameters and precision.
 *  - ncols above CASIM_NOALLOC_MAX_COLS is rejected with CASIM_ERR_ARG and a
 *    message in casim_last_cuda_error(); other arguments as for casim_step.
 *  - The first call on each device looks up the array's device address (with
 *    that device current); make that first call before any stream capture.
 *  - Every call on a device shares the one array and leaves its contents
 *    behind; the call clears what must start at zero.  Two calls whose work
 *    overlaps on the GPU (different streams, no ordering) race on the array
 *    and give wrong results: order them on one stream.
 *  - params may be NULL (defaults).  If flags is non-NULL the call waits for
 *    `stream`, stores the CASIM_EFLAG_* bits of this step in *flags and
 *    returns CASIM_ERR_NONFINITE / CASIM_ERR_CFL when they are set; if NULL it
 *    returns after enqueuing, and the step's error bits are never reported:
 *    the next call clears them before it runs.  A caller that must learn of
 *    non-finite values or the substep cap passes flags.
 *  - Host threads may make their first call on a device concurrently (the
 *    address lookup is thread-safe); their GPU work must still be ordered. */
#define CASIM_NOALLOC_MAX_COLS (1 << 20)
int casim_step_noalloc(const casim_params *params, int precision, const casim_state *s, int ncols, int nlev,
                       double dt, void *stream, unsigned *flags);

/* Number of kernel launches this context has enqueued since casim_init. */
long long casim_launch_count(const casim_ctx *ctx);

/* The last CUDA error string seen by this library (static storage). */
const char *casim_last_cuda_error(void);

/* ----------------------------------------------------------------------------
 * Checkpoint / resume.  The state is plain arrays, so a checkpoint is a
 * header (format tag, ABI version, nfields, precipitation rows, nlev, pitch,
 * ncols and a hash of the scheme parameters) followed by dz, the fields and
 * the precipitation rows as raw FP64 values in host byte order.  A run of N
 * steps equals, bit for bit, k steps, save, load, N - k steps.
 * nfields is CASIM_NFIELDS, CASIM_NFIELDS_3MOM or CASIM_NFIELDS_3MOM_COLD for
 * the triple-moment states (warm, cold), CASIM_NFIELDS_AEROSOL_COLD for the
 * cold activated-aerosol state (whose precip has CASIM_NPRECIP + 1 rows),
 * or CASIM_NFIELDS_AEROSOL for the activated-aerosol state (whose precip has
 * CASIM_NPRECIP + 1 rows).  Device pointers;
 * both calls wait for `stream`.  params may be NULL (the defaults).
 * casim_state_load rejects (CASIM_ERR_ARG) a file whose dimensions or
 * parameter hash differ from the arguments; file errors give CASIM_ERR_IO. */
#define CASIM_NFIELDS_AEROSOL 19
#define CASIM_NFIELDS_3MOM 17
#define CASIM_NFIELDS_3MOM_COLD 20
#define CASIM_NFIELDS_AEROSOL_COLD 22
int casim_state_save(const char *path, const casim_params *params, const casim_state *s, int ncols, int nlev,
                     int nfields, void *stream);
int casim_state_load(const char *path, const casim_params *params, const casim_state *s, int ncols, int nlev,
                     int nfields, void *stream);

/* Release the context and its device memory (waits for the device). NULL is a no-op. */
void casim_free(casim_ctx *ctx);

int casim_abi_version(void);

#ifdef __cplusplus
}
#endif
#endif
