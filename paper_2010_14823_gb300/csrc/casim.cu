// Host side of the C ABI declared in include/casim.h.
//
// The library owns no state memory: the caller passes device pointers (for
// instance PyTorch tensors) and a stream.  A context carries the derived
// scheme constants, the precision form, a device error word and, for
// casim_step_host only, staging buffers (its copy path for pageable host
// memory; pinned host state is stepped in place).  Mirrors the paper's host protocol
// (Section 3.2): one-off set-up, one asynchronous call per timestep running
// the whole scheme for every column, tear-down.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdint>

#include <algorithm>
#include <atomic>
#include <type_traits>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "casim.h"
#include "casim_device.cuh"
#include "casim_batch.cuh"
#include "casim_mlp.cuh"

#include <random>

using namespace casim_dev;

// An NVTX range named after an entry point (or a phase of one) for the
// duration of the host call: the enqueue of asynchronous work, or the whole
// work of a synchronous call.  Costs nothing unless a profiler is attached.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

struct casim_ctx {
  int precision = CASIM_FP64;
  bool warm = false;   // CASIM_WARM: the warm configuration (liquid water only)
  bool aero = false;   // CASIM_AEROSOL: with activated-aerosol mass (19-field state, 5 precip rows)
  bool tri = false;    // CASIM_THREE_MOMENT: triple-moment rain (17-field state)
  int device = 0;
  int nsm = 1;
  int host_ro = 1;   // the device supports read-only registration of host memory (assumed until queried)
  KParams kp;
  unsigned *d_err = nullptr;
  long long launches = 0;
  // staging for casim_step_host: per pipeline stage a chunk of the state and
  // of precip, its own stream (the copy path); dz once (both paths)
  static constexpr int kStages = 3;
  double *h2d_fld[kStages] = {}, *h2d_precip[kStages] = {}, *h2d_dz = nullptr;
  size_t cap_fld[kStages] = {}, cap_precip[kStages] = {}, cap_dz = 0;
  cudaStream_t hst[kStages] = {};
  cudaEvent_t hev_start = nullptr, hev_dz = nullptr;
  // casim_step_batched: the batch of the last domain list it was given, and
  // that list (a different list replaces the batch)
  casim_batch *sb = nullptr;
  std::vector<casim_state> sb_dom;
  std::vector<int> sb_ncols, sb_nlev;
  // CASIM_STATS: the device counters (ColStats words) and the host's
  bool stats = false;
  unsigned long long *d_stats = nullptr;
  long long stat_steps = 0, stat_points = 0;
};

static thread_local char g_last_error[256] = "";

static int cuda_fail(cudaError_t e, const char *what) {
  std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s", what, cudaGetErrorString(e));
  return CASIM_ERR_CUDA;
}
#define CUDA_TRY(x)                                   \
  do {                                                \
    cudaError_t e_ = (x);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #x);  \
  } while (0)

extern "C" int casim_abi_version(void) { return CASIM_ABI_VERSION; }

extern "C" const char *casim_last_cuda_error(void) { return g_last_error; }

extern "C" int casim_default_params(casim_params *p) {
  if (!p) return CASIM_ERR_ARG;
  std::memset(p, 0, sizeof(*p));
  // thermodynamic constants
  p->T0 = 273.15; p->cp = 1005.0; p->Lv = 2.5e6; p->Lf = 3.34e5; p->Rd = 287.04; p->Rv = 461.5;
  p->g = 9.81; p->rho_w = 1000.0; p->rho0 = 1.2; p->Ka = 2.4e-2; p->Dv = 2.26e-5; p->mu_air = 1.72e-5;
  p->q_min = 1e-14; p->T_nuc = 268.15; p->m_i0 = 1e-12; p->r_r0 = 25e-6;
  // Khairoutdinov & Kogan (2000)
  p->kk_aut = 1350.0; p->kk_aut_qc = 2.47; p->kk_aut_nc = -1.79; p->nc_min_cm3 = 1.0;
  p->kk_acc = 67.0; p->kk_acc_exp = 1.15;
  // Seifert & Beheng (2001, 2006)
  p->kc_sb = 9.44e9; p->nu_c = 1.0; p->kr_sb = 5.78;
  // Meyers et al. (1992)
  p->mey_a = 1e3; p->mey_b = -0.639; p->mey_c = 12.96;
  // Abdul-Razzak & Ghan (2000), one ammonium-sulphate-like mode
  p->arg_rm = 0.05e-6; p->arg_sigma = 1.5; p->arg_kappa = 0.61; p->surft = 0.0761;
  p->Mw = 0.018015; p->Ma = 0.028965; p->Rgas = 8.314;
  p->e_rim = 1.0; p->c_max = 1.0;
  // Bolton (1980) over liquid, Murray (1967) over ice
  p->es_l0 = 611.2; p->es_la = 17.67; p->es_lb = 243.5;
  p->es_i0 = 610.78; p->es_ia = 21.875; p->es_it = 273.16; p->es_ib = 7.66;
  const double pi = 3.14159265358979323846;
  //                  cloud             rain              ice              snow             graupel
  const double a[5] = {pi / 6 * 1000.0, pi / 6 * 1000.0, pi / 6 * 500.0, pi / 6 * 100.0, pi / 6 * 400.0};
  const double mu[5] = {2.0, 0.0, 0.0, 0.0, 0.5};
  const double cv[5] = {0.0, 130.0, 700.0, 11.72, 19.3};
  const double dv[5] = {0.0, 0.5, 1.0, 0.41, 0.37};
  const double vmax[5] = {0.0, 10.0, 2.0, 4.0, 10.0};
  const double dmin[5] = {1e-6, 50e-6, 1e-6, 10e-6, 10e-6};
  const double dmax[5] = {1e-4, 5e-3, 500e-6, 5e-3, 5e-3};
  const double ccap[5] = {0.5, 0.5, 0.5, 1.0 / pi, 0.5};
  for (int x = 0; x < 5; ++x) {
    p->a[x] = a[x]; p->b[x] = 3.0; p->mu[x] = mu[x]; p->cv[x] = cv[x]; p->dv[x] = dv[x];
    p->vmax[x] = vmax[x]; p->dmin[x] = dmin[x]; p->dmax[x] = dmax[x]; p->ccap[x] = ccap[x];
  }
  return CASIM_OK;
}

// Derived constants.  `l` is the logarithm the policy works in (natural log
// for FP64, log2 for the mixed form, whose special functions run on ex2/lg2).
template <class R>
static void derive(const casim_params &p, ConstK<R> &K, double (*l)(double)) {
  const double pi = 3.14159265358979323846;
  const double Ls = p.Lv + p.Lf;
  const double eps = p.Rd / p.Rv;
  K.T0 = (R)p.T0; K.Tnuc = (R)p.T_nuc; K.qmin = (R)p.q_min; K.tnuc0 = (R)(p.T_nuc - p.T0);
  K.t0_esit = (R)(p.T0 - p.es_it); K.t0_esib = (R)(p.T0 - p.es_ib);
  K.lv_cp = (R)(p.Lv / p.cp); K.cp_lv = (R)(p.cp / p.Lv); K.cp = (R)p.cp; K.inv_cp = (R)(1.0 / p.cp);
  K.lv = (R)p.Lv; K.ls = (R)Ls; K.lf = (R)p.Lf;
  K.eps = (R)eps; K.ome = (R)(1.0 - eps);
  K.esl0 = (R)p.es_l0; K.esla = (R)p.es_la; K.eslb = (R)p.es_lb; K.eslab = (R)(p.es_la * p.es_lb);
  K.esi0 = (R)p.es_i0; K.esia = (R)p.es_ia; K.esit = (R)p.es_it; K.esib = (R)p.es_ib;
  K.awc = (R)(p.Lv * p.Lv / (p.Ka * p.Rv));
  K.aic = (R)(Ls * Ls / (p.Ka * p.Rv));
  K.rv_dv = (R)(p.Rv / p.Dv);
  K.akel = (R)(2.0 * p.surft * p.Mw / (p.rho_w * p.Rgas));
  K.smc = (R)(2.0 / std::sqrt(p.arg_kappa) * std::pow(1.0 / (3.0 * p.arg_rm), 1.5));
  K.al1 = (R)(p.g * p.Mw * p.Lv / (p.cp * p.Rgas));
  K.al2 = (R)(p.g * p.Ma / p.Rgas);
  K.ga1 = (R)(p.Rgas / p.Mw);
  K.ga2 = (R)(p.Mw * p.Lv * p.Lv / (p.cp * p.Ma));
  K.gg1 = (R)(p.rho_w * p.Rgas / (p.Dv * p.Mw));
  K.gg2 = (R)(p.Lv * p.rho_w / p.Ka);
  K.gg3 = (R)(p.Lv * p.Mw / p.Rgas);
  const double lns = std::log(p.arg_sigma);
  K.twopirhow = (R)(2.0 * pi * p.rho_w);
  K.f1 = (R)(0.5 * std::exp(2.5 * lns * lns));
  K.f2 = (R)(1.0 + 0.25 * lns);
  K.uc = (R)(2.0 / (3.0 * std::sqrt(2.0) * lns));
  K.kk_aut = (R)p.kk_aut; K.kk_aut_qc = (R)p.kk_aut_qc; K.kk_aut_nc = (R)p.kk_aut_nc;
  K.nc_min = (R)p.nc_min_cm3; K.kk_acc = (R)p.kk_acc; K.kk_acc_exp = (R)p.kk_acc_exp;
  K.kcf = (R)(p.kc_sb * (p.nu_c + 2.0) / (p.nu_c + 1.0));
  K.kr = (R)p.kr_sb;
  K.inv_mr0 = (R)(1.0 / (4.0 / 3.0 * pi * p.rho_w * p.r_r0 * p.r_r0 * p.r_r0));
  K.mey_a = (R)p.mey_a; K.mey_b = (R)p.mey_b; K.mey_c = (R)p.mey_c; K.mi0 = (R)p.m_i0;
  K.mu_air = (R)p.mu_air; K.inv_dv = (R)(1.0 / p.Dv); K.lgrho0 = (R)l(p.rho0); K.twopi = (R)(2.0 * pi);
  for (int x = 0; x < 5; ++x) {
    const double a = p.a[x], b = p.b[x], mu = p.mu[x], cv = p.cv[x], dv = p.dv[x];
    const double gb = std::tgamma(mu + b + 1.0);
    SpeciesK<R> &S = K.sp[x];
    S.lglamfac = (R)l(a * gb / std::tgamma(mu + 1.0));
    S.invb = (R)(1.0 / b);
    S.lglo = (R)l((mu + 1.0) / p.dmax[x]);
    S.lghi = (R)l((mu + 1.0) / p.dmin[x]);
    S.ev1 = (R)(0.78 * std::tgamma(mu + 2.0) / gb / a);
    S.ex1 = (R)(b - 1.0);
    const double k2 = 0.5 * (dv + 3.0);
    S.ev2 = (R)(0.31 * std::sqrt(cv) * std::tgamma(mu + k2 + 1.0) / gb / a);
    S.ex2 = (R)(b - k2);
    S.rim = (R)(0.25 * pi * p.e_rim * cv * std::tgamma(mu + dv + 3.0) / gb / a);
    S.exr = (R)(b - 2.0 - dv);
    S.vq = (R)(cv * std::tgamma(mu + b + dv + 1.0) / gb);
    S.vn = (R)(cv * std::tgamma(mu + dv + 1.0) / std::tgamma(mu + 1.0));
    S.exv = (R)(-dv);
    S.vmax = (R)p.vmax[x];
    S.dep = (R)(4.0 * pi * p.ccap[x]);
    S.mlt = (R)(4.0 * pi * p.ccap[x] * p.Ka / p.Lf);
  }
  // triple-moment species r, i, s, g (species 1..4)
  for (int x = 0; x < 4; ++x) {
    const int sp = 1 + x;
    K.s3_a[x] = (R)p.a[sp];
    K.s3_dv[x] = (R)p.dv[sp];
    K.s3_mu0[x] = (R)p.mu[sp];
    K.s3_lgdmax[x] = (R)l(p.dmax[sp]);
    K.s3_lgdmin[x] = (R)l(p.dmin[sp]);
    K.s3_ev1c[x] = (R)(0.78 / p.a[sp]);
    K.s3_ev2c[x] = (R)(0.31 * std::sqrt(p.cv[sp]) / p.a[sp]);
    K.s3_cv[x] = (R)p.cv[sp];
    K.s3_rimc[x] = (R)(0.25 * pi * p.e_rim * p.cv[sp] / p.a[sp]);
    const double ar = p.a[sp] / p.a[1];
    K.s3_ar2[x] = (R)(ar * ar);
  }
  K.s3_mumax = (R)20.0;
  const double d0 = 2.0 * p.r_r0, d3 = d0 * d0 * d0;
  K.s3_d0_6 = (R)(d3 * d3);
  const double di = p.m_i0 / p.a[2];
  K.s3_di_6 = (R)(di * di);
}

static double ln_(double x) { return std::log(x); }
static double log2_(double x) { return std::log2(x); }

static bool params_ok(const casim_params &p) {
  if (!(p.cp > 0 && p.Lv > 0 && p.Lf >= 0 && p.Rd > 0 && p.Rv > 0 && p.rho0 > 0 && p.Ka > 0 && p.Dv > 0 &&
        p.mu_air > 0 && p.q_min > 0 && p.m_i0 > 0 && p.r_r0 > 0 && p.c_max > 0 && p.arg_sigma > 1 &&
        p.arg_kappa > 0 && p.arg_rm > 0))
    return false;
  for (int x = 0; x < 5; ++x)
    if (!(p.a[x] > 0 && p.b[x] > 0 && p.mu[x] > -1 && p.dmin[x] > 0 && p.dmax[x] > p.dmin[x] && p.cv[x] >= 0 &&
          p.vmax[x] >= 0))
      return false;
  return true;
}

// a staged step kernel (in place, its whole-line-store form, source-term
// mode) may use the dynamic shared memory of a column of the largest level count
template <class M>
static cudaError_t allow_step_smem() {
  cudaError_t e = cudaFuncSetAttribute(k_step<M, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)step_smem_bytes<M, false>(kMaxLev));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_step<M, false, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)step_smem_bytes<M, false>(kMaxLev));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_step<M, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)step_smem_bytes<M, true>(kMaxLev));
  return e;
}

extern "C" int casim_init(casim_ctx **out, const casim_params *params, int precision, int flags) {
  if (!out) return CASIM_ERR_ARG;
  *out = nullptr;
  if (precision != CASIM_FP64 && precision != CASIM_MIXED) return CASIM_ERR_ARG;
  if ((flags & ~(CASIM_WARM | CASIM_AEROSOL | CASIM_THREE_MOMENT | CASIM_STATS)) != 0) return CASIM_ERR_ARG;
  if ((flags & CASIM_STATS) && (flags & (CASIM_WARM | CASIM_AEROSOL | CASIM_THREE_MOMENT))) return CASIM_ERR_ARG;
  if ((flags & CASIM_AEROSOL) && (flags & CASIM_THREE_MOMENT)) return CASIM_ERR_ARG;
  if ((flags & CASIM_THREE_MOMENT) && params) {
    // the shape identity needs b = 3 for every species that carries z
    const int last = (flags & CASIM_WARM) ? 1 : 4;
    for (int x = 1; x <= last; ++x)
      if (params->b[x] != 3.0) return CASIM_ERR_ARG;
  }
  casim_params p;
  if (params) p = *params;
  else casim_default_params(&p);
  if (!params_ok(p)) return CASIM_ERR_ARG;
  casim_ctx *ctx = new casim_ctx();
  ctx->precision = precision;
  ctx->warm = (flags & CASIM_WARM) != 0;
  ctx->aero = (flags & CASIM_AEROSOL) != 0;
  ctx->tri = (flags & CASIM_THREE_MOMENT) != 0;
  derive<double>(p, ctx->kp.d, ln_);
  derive<float>(p, ctx->kp.f, log2_);
  ctx->kp.c_max = p.c_max;
  ctx->kp.T0 = p.T0;
  for (int x = 0; x < 5; ++x) ctx->kp.vmax[x] = p.vmax[x];
  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->nsm, cudaDevAttrMultiProcessorCount, ctx->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->host_ro, cudaDevAttrHostRegisterReadOnlySupported, ctx->device);
  // the staged mixed steps' dynamic shared memory (prefetch stage and level
  // tables) exceeds the default 48 KB for long columns
  if (e == cudaSuccess) e = allow_step_smem<PolicyMix>();
  if (e == cudaSuccess) e = allow_step_smem<PolicyMixWarm>();
  if (e == cudaSuccess) e = allow_step_smem<PolicyMixWarmAero>();
  if (e == cudaSuccess) e = allow_step_smem<PolicyMixWarm3>();
  if (e == cudaSuccess) e = allow_step_smem<PolicyMixAero>();
  if (e == cudaSuccess) e = allow_step_smem<PolicyMix3>();
  // and the batched step's (256-thread blocks: a 64 KB stage)
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_step_batch<PolicyMix, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)batch_smem_bytes<PolicyMix>(kBatchNarrowBlock, kMaxLev));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_step_batch<PolicyMix, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)batch_smem_bytes<PolicyMix>(kBatchMaxBlock, kMaxLev));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_step<PolicyMix, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)step_smem_bytes<PolicyMix, false>(kMaxLev));
  ctx->stats = (flags & CASIM_STATS) != 0;
  if (e == cudaSuccess && ctx->stats) e = cudaMalloc(&ctx->d_stats, kStatsWords * sizeof(unsigned long long));
  if (e == cudaSuccess && ctx->stats) e = cudaMemset(ctx->d_stats, 0, kStatsWords * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&ctx->d_err, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(ctx->d_err, 0, sizeof(unsigned));
  if (e != cudaSuccess) {
    int rc = e == cudaErrorMemoryAllocation ? CASIM_ERR_OOM : cuda_fail(e, "casim_init");
    if (ctx->d_err) cudaFree(ctx->d_err);
    delete ctx;
    return rc;
  }
  *out = ctx;
  return CASIM_OK;
}

static_assert(kMaxLev == CASIM_MAX_LEV, "the header's level limit is the kernels' shared dz array");
static_assert(kEflagIndex == CASIM_EFLAG_INDEX, "the debug build's error bit");
static_assert(kStatsWords == 3 + 4 * 65 && sizeof(((casim_stats *)0)->nsub) == 4 * 65 * sizeof(long long),
              "the statistics buffer's layout");

static int check_state(const casim_state *s, int ncols, int nlev, double dt) {
  if (!s || ncols < 0 || nlev < 1 || nlev > kMaxLev || !(dt > 0.0) || !std::isfinite(dt)) return CASIM_ERR_ARG;
  if (ncols == 0) return CASIM_OK;
  if (!s->fld || !s->dz || !s->precip) return CASIM_ERR_ARG;
  if (s->pitch < ncols || s->pitch % 32 != 0) return CASIM_ERR_ARG;
  if (((uintptr_t)s->fld) % 256 != 0) return CASIM_ERR_ARG;
  return CASIM_OK;
}

static KArgs make_args(const casim_ctx *ctx, const casim_state *s, int ncols, int nlev, double dt) {
  KArgs a;
  a.fld = s->fld;
  a.pitch = s->pitch;
  a.dz = s->dz;
  a.precip = s->precip;
  a.err = ctx->d_err;
  a.ncols = ncols;
  a.nlev = nlev;
  a.dt = dt;
  a.surr = nullptr;
  a.stats = ctx->stats ? ctx->d_stats : nullptr;
  return a;
}

// tend null: the in-place step; else the source-term mode
// fields and precipitation rows of a context's state
static int ctx_nfields(const casim_ctx *ctx) {
  if (ctx->aero) return ctx->warm ? CASIM_NFIELDS_AEROSOL : CASIM_NFIELDS_AEROSOL_COLD;
  if (ctx->tri) return ctx->warm ? CASIM_NFIELDS_3MOM : CASIM_NFIELDS_3MOM_COLD;
  return CASIM_NFIELDS;
}
static int ctx_nprecip(const casim_ctx *ctx) { return CASIM_NPRECIP + (ctx->aero ? 1 : 0); }

// one configuration's kernels: the in-place step, or (tend) the source-term
// mode; line: the state is mapped host memory (the mixed step's whole-line
// stores)
template <class PMix, class PF64>
static void launch_pair(const casim_ctx *ctx, dim3 grid, cudaStream_t st, const KArgs &a, double *tend, bool line) {
  const KParams &kp = ctx->kp;
  if constexpr (std::is_same<PMix, PolicyMix>::value) {
    // the statistics build (a CASIM_STATS context: standard configuration)
    if (a.stats && !tend) {
      if (ctx->precision == CASIM_MIXED)
        k_step<PMix, false, true><<<grid, kBlock, step_smem_bytes<PMix, false>(a.nlev), st>>>(a, kp, nullptr);
      else
        k_step<PF64, false, true><<<grid, kBlock, step_smem_bytes<PF64, false>(a.nlev), st>>>(a, kp, nullptr);
      return;
    }
  }
  if (ctx->precision == CASIM_MIXED) {
    if (tend) k_step<PMix, true><<<grid, kBlock, step_smem_bytes<PMix, true>(a.nlev), st>>>(a, kp, tend);
    else if (line)
      k_step<PMix, false, false, true><<<grid, kBlock, step_smem_bytes<PMix, false>(a.nlev), st>>>(a, kp, nullptr);
    else k_step<PMix, false><<<grid, kBlock, step_smem_bytes<PMix, false>(a.nlev), st>>>(a, kp, nullptr);
  } else {
    if (tend) k_step<PF64, true><<<grid, kBlock, step_smem_bytes<PF64, true>(a.nlev), st>>>(a, kp, tend);
    else k_step<PF64, false><<<grid, kBlock, step_smem_bytes<PF64, false>(a.nlev), st>>>(a, kp, nullptr);
  }
}

static int launch_step(casim_ctx *ctx, const KArgs &a, int ncols, double *tend, void *stream, bool line = false) {
  const dim3 grid((unsigned)((ncols + kBlock - 1) / kBlock));
  cudaStream_t st = (cudaStream_t)stream;
  if (ctx->aero && ctx->warm) launch_pair<PolicyMixWarmAero, PolicyF64WarmAero>(ctx, grid, st, a, tend, line);
  else if (ctx->aero) launch_pair<PolicyMixAero, PolicyF64Aero>(ctx, grid, st, a, tend, line);
  else if (ctx->tri && ctx->warm) launch_pair<PolicyMixWarm3, PolicyF64Warm3>(ctx, grid, st, a, tend, line);
  else if (ctx->tri) launch_pair<PolicyMix3, PolicyF643>(ctx, grid, st, a, tend, line);
  else if (ctx->warm) launch_pair<PolicyMixWarm, PolicyF64Warm>(ctx, grid, st, a, tend, line);
  else launch_pair<PolicyMix, PolicyF64>(ctx, grid, st, a, tend, line);
  ctx->launches++;
  CUDA_TRY(cudaGetLastError());
  return CASIM_OK;
}

extern "C" int casim_step_tendency(casim_ctx *ctx, const casim_state *s, int ncols, int nlev, double dt, double *tend,
                                   void *stream) {
  NvtxRange nvtx_range_("casim_step_tendency");
  if (!ctx || !tend) return CASIM_ERR_ARG;
  int rc = check_state(s, ncols, nlev, dt);
  if (rc != CASIM_OK || ncols == 0) return rc;
  const int NF = ctx_nfields(ctx);
  const size_t span = (size_t)NF * nlev * s->pitch;
  const size_t tspan = (size_t)(NF - 3) * nlev * s->pitch;   // no rows for the inputs p, rho, w
  if (reinterpret_cast<uintptr_t>(tend) % alignof(double) != 0 ||
      (tend < s->fld + span && s->fld < tend + tspan))   // must not overlap the state
    return CASIM_ERR_ARG;
  const KArgs a = make_args(ctx, s, ncols, nlev, dt);
  return launch_step(ctx, a, ncols, tend, stream);
}

// line: the state is mapped host memory
static int step_device(casim_ctx *ctx, const casim_state *s, int ncols, int nlev, double dt, void *stream,
                       bool line = false) {
  int rc = check_state(s, ncols, nlev, dt);
  if (rc != CASIM_OK || ncols == 0) return rc;
  const KArgs a = make_args(ctx, s, ncols, nlev, dt);
  return launch_step(ctx, a, ncols, nullptr, stream, line);
}

// a CASIM_STATS context counts the step and its points on the host
static void count_step(casim_ctx *ctx, int ncols, int nlev) {
  if (!ctx->stats) return;
  ++ctx->stat_steps;
  ctx->stat_points += (long long)ncols * nlev;
}

extern "C" int casim_step(casim_ctx *ctx, const casim_state *s, int ncols, int nlev, double dt, void *stream) {
  NvtxRange nvtx_range_("casim_step");
  if (!ctx) return CASIM_ERR_ARG;
  const int rc = step_device(ctx, s, ncols, nlev, dt, stream);
  if (rc == CASIM_OK) count_step(ctx, ncols, nlev);
  return rc;
}

static int grow(double **buf, size_t *cap, size_t n) {
  if (*cap >= n) return CASIM_OK;
  if (*buf) cudaFree(*buf);
  *buf = nullptr;
  *cap = 0;
  cudaError_t e = cudaMalloc(buf, n * sizeof(double));
  if (e != cudaSuccess) {
    *buf = nullptr;
    return e == cudaErrorMemoryAllocation ? CASIM_ERR_OOM : cuda_fail(e, "cudaMalloc");
  }
  *cap = n;
  return CASIM_OK;
}

// Host pipeline chunks: strided host<->device copies run at full speed only
// with contiguous runs of about 512 KB (measured on GB300: 512 KB rows 205
// GB/s, 128 KB rows 100 GB/s), so a chunk is at least 65 536 columns wide;
// at most 2 GB of device state per stage.
constexpr size_t kHostMinRowBytes = 512ull << 10;
constexpr size_t kHostChunkBytes = 2ull << 30;

// one column chunk [c0, c0 + wc) of a host state: fields (3-D strided copy:
// wc columns x nlev levels x nfields) and precip (2-D copy)
// fields [f0, f0 + nf) of one column chunk between the host state and a
// device chunk of width W (one 3-D copy)
static cudaError_t copy_fields(double *dev_fld, int W, const casim_state *h, int c0, int wc, int nlev, int f0,
                               int nf, cudaMemcpyKind kind, cudaStream_t st) {
  cudaMemcpy3DParms p = {};
  const bool up = kind == cudaMemcpyHostToDevice;
  const size_t hs = (size_t)nlev * h->pitch, ds = (size_t)nlev * W;   // field strides
  cudaPitchedPtr hp = make_cudaPitchedPtr(h->fld + f0 * hs + c0, (size_t)h->pitch * sizeof(double), (size_t)wc,
                                          (size_t)nlev);
  cudaPitchedPtr dp = make_cudaPitchedPtr(dev_fld + f0 * ds, (size_t)W * sizeof(double), (size_t)wc, (size_t)nlev);
  p.srcPtr = up ? hp : dp;
  p.dstPtr = up ? dp : hp;
  p.extent = make_cudaExtent((size_t)wc * sizeof(double), (size_t)nlev, (size_t)nf);
  p.kind = kind;
  return cudaMemcpy3DAsync(&p, st);
}

// one column chunk: up, every field; down, the prognostic ones (0..12 and
// the configuration's fields after the inputs p, rho, w); and the precip rows
static cudaError_t copy_chunk(double *dev_fld, double *dev_precip, int W, const casim_state *h, int c0, int wc,
                              int nlev, int nfields, int nprecip, cudaMemcpyKind kind, cudaStream_t st) {
  const bool up = kind == cudaMemcpyHostToDevice;
  cudaError_t e = copy_fields(dev_fld, W, h, c0, wc, nlev, 0, up ? nfields : CASIM_NPROG, kind, st);
  if (e == cudaSuccess && !up && nfields > CASIM_NFIELDS)
    e = copy_fields(dev_fld, W, h, c0, wc, nlev, CASIM_NFIELDS, nfields - CASIM_NFIELDS, kind, st);
  if (e != cudaSuccess) return e;
  double *hpr = h->precip + c0;
  const size_t hpitch = (size_t)h->pitch * sizeof(double), dpitch = (size_t)W * sizeof(double);
  return up ? cudaMemcpy2DAsync(dev_precip, dpitch, hpr, hpitch, (size_t)wc * sizeof(double), nprecip, kind, st)
            : cudaMemcpy2DAsync(hpr, hpitch, dev_precip, dpitch, (size_t)wc * sizeof(double), nprecip, kind, st);
}



// The device address of the host range [p, p + bytes) when the whole range
// is pinned host memory mapped into the device's address space (a
// cudaHostAlloc / cudaMallocHost allocation or a cudaHostRegister range),
// which this device reaches over the host link: both ends are host memory
// with device addresses the same distance apart as the host ones.  nullptr
// for pageable memory.  (Whether the device may also store to it is the
// caller's concern: see host_ro.)
static void *mapped_host(const void *p, size_t bytes) {
  if (!p || bytes == 0) return nullptr;
  const char *b = static_cast<const char *>(p);
  cudaPointerAttributes a0, a1;
  if (cudaPointerGetAttributes(&a0, b) != cudaSuccess || cudaPointerGetAttributes(&a1, b + bytes - 1) != cudaSuccess) {
    (void)cudaGetLastError();   // the query's own error, not a sticky one
    return nullptr;
  }
  if (a0.type != cudaMemoryTypeHost || a1.type != cudaMemoryTypeHost || !a0.devicePointer || !a1.devicePointer)
    return nullptr;
  if (static_cast<const char *>(a1.devicePointer) - static_cast<const char *>(a0.devicePointer) !=
      static_cast<ptrdiff_t>(bytes - 1))
    return nullptr;
  return a0.devicePointer;
}

extern "C" int casim_step_host(casim_ctx *ctx, const casim_state *h, int ncols, int nlev, double dt,
                               void *stream) {
  NvtxRange nvtx_range_("casim_step_host");
  if (!ctx) return CASIM_ERR_ARG;
  if (!h || ncols < 0 || nlev < 1 || nlev > kMaxLev || !(dt > 0.0) || !std::isfinite(dt)) return CASIM_ERR_ARG;
  if (ncols == 0) return CASIM_OK;
  if (!h->fld || !h->dz || !h->precip || h->pitch < ncols || h->pitch % 32 != 0) return CASIM_ERR_ARG;
  const int NF = ctx_nfields(ctx), NP = ctx_nprecip(ctx);
  int rc;
  // mapped pinned state: the step kernel loads and stores it in place over the
  // host link (every input crosses once; back come only the 32-column rows of
  // the fields the step changed somewhere in them; its prefetch keeps a level
  // of loads in flight), no staging copies
  // (the device state's 256-byte alignment; otherwise the copies below).  On
  // a device that can register host memory read-only, a registered range
  // cannot be told apart from a writable one, so there only the copies run.
  void *mfld = ctx->host_ro == 0 ? mapped_host(h->fld, (size_t)NF * nlev * h->pitch * sizeof(double)) : nullptr;
  if (reinterpret_cast<uintptr_t>(mfld) % 256 != 0) mfld = nullptr;
  void *mpr = mfld ? mapped_host(h->precip, (size_t)NP * h->pitch * sizeof(double)) : nullptr;
  if (mfld && mpr) {
    cudaStream_t st = (cudaStream_t)stream;
    if ((rc = grow(&ctx->h2d_dz, &ctx->cap_dz, (size_t)nlev)) != CASIM_OK) return rc;
    CUDA_TRY(cudaMemcpyAsync(ctx->h2d_dz, h->dz, (size_t)nlev * sizeof(double), cudaMemcpyHostToDevice, st));
    casim_state d;
    d.fld = static_cast<double *>(mfld);
    d.pitch = h->pitch;
    d.dz = ctx->h2d_dz;
    d.precip = static_cast<double *>(mpr);
    if ((rc = step_device(ctx, &d, ncols, nlev, dt, stream, true)) != CASIM_OK) return rc;
    CUDA_TRY(cudaStreamSynchronize(st));
    count_step(ctx, ncols, nlev);
    return CASIM_OK;
  }
  // chunk width: a multiple of 32 columns with long contiguous rows, within the byte cap
  const size_t col_bytes = (size_t)NF * nlev * sizeof(double);
  const int wcap = (int)std::max<size_t>(32, kHostChunkBytes / col_bytes / 32 * 32);
  const int W = (int)std::min<size_t>(kHostMinRowBytes / sizeof(double), (size_t)wcap);
  const int nchunk = (ncols + W - 1) / W;
  if (nchunk == 1) {
    // one chunk: contiguous copies of the whole state at the host pitch
    const size_t nf = (size_t)NF * nlev * h->pitch, np = (size_t)NP * h->pitch;
    if ((rc = grow(&ctx->h2d_fld[0], &ctx->cap_fld[0], nf)) != CASIM_OK) return rc;
    if ((rc = grow(&ctx->h2d_precip[0], &ctx->cap_precip[0], np)) != CASIM_OK) return rc;
    if ((rc = grow(&ctx->h2d_dz, &ctx->cap_dz, (size_t)nlev)) != CASIM_OK) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    CUDA_TRY(cudaMemcpyAsync(ctx->h2d_fld[0], h->fld, nf * sizeof(double), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(ctx->h2d_dz, h->dz, (size_t)nlev * sizeof(double), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(ctx->h2d_precip[0], h->precip, np * sizeof(double), cudaMemcpyHostToDevice, st));
    casim_state d;
    d.fld = ctx->h2d_fld[0];
    d.pitch = h->pitch;
    d.dz = ctx->h2d_dz;
    d.precip = ctx->h2d_precip[0];
    if ((rc = step_device(ctx, &d, ncols, nlev, dt, stream)) != CASIM_OK) return rc;
    const size_t fsz = (size_t)nlev * h->pitch, nprog = (size_t)CASIM_NPROG * fsz;
    CUDA_TRY(cudaMemcpyAsync(h->fld, ctx->h2d_fld[0], nprog * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (NF > CASIM_NFIELDS)   // the configuration's prognostic fields after the inputs
      CUDA_TRY(cudaMemcpyAsync(h->fld + CASIM_NFIELDS * fsz, ctx->h2d_fld[0] + CASIM_NFIELDS * fsz,
                               (size_t)(NF - CASIM_NFIELDS) * fsz * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(h->precip, ctx->h2d_precip[0], np * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    count_step(ctx, ncols, nlev);
    return CASIM_OK;
  }
  const int S = std::min(casim_ctx::kStages, nchunk);
  for (int s = 0; s < S; ++s) {
    if ((rc = grow(&ctx->h2d_fld[s], &ctx->cap_fld[s], (size_t)NF * nlev * W)) != CASIM_OK) return rc;
    if ((rc = grow(&ctx->h2d_precip[s], &ctx->cap_precip[s], (size_t)NP * W)) != CASIM_OK) return rc;
    if (!ctx->hst[s]) CUDA_TRY(cudaStreamCreateWithFlags(&ctx->hst[s], cudaStreamNonBlocking));
  }
  if ((rc = grow(&ctx->h2d_dz, &ctx->cap_dz, (size_t)nlev)) != CASIM_OK) return rc;
  if (!ctx->hev_start) CUDA_TRY(cudaEventCreateWithFlags(&ctx->hev_start, cudaEventDisableTiming));
  if (!ctx->hev_dz) CUDA_TRY(cudaEventCreateWithFlags(&ctx->hev_dz, cudaEventDisableTiming));
  // the stages start after the caller's earlier work on `stream`; dz goes up once
  CUDA_TRY(cudaEventRecord(ctx->hev_start, (cudaStream_t)stream));
  CUDA_TRY(cudaStreamWaitEvent(ctx->hst[0], ctx->hev_start, 0));
  CUDA_TRY(cudaMemcpyAsync(ctx->h2d_dz, h->dz, (size_t)nlev * sizeof(double), cudaMemcpyHostToDevice, ctx->hst[0]));
  CUDA_TRY(cudaEventRecord(ctx->hev_dz, ctx->hst[0]));
  for (int s = 1; s < S; ++s) CUDA_TRY(cudaStreamWaitEvent(ctx->hst[s], ctx->hev_dz, 0));
  // chunk i on stage i % S: copy in, step, copy out; the stages overlap
  // one chunk's copies in, another's step and a third's copies out
  cudaError_t e = cudaSuccess;
  rc = CASIM_OK;
  for (int i = 0; i < nchunk && e == cudaSuccess && rc == CASIM_OK; ++i) {
    const int s = i % S;
    const int c0 = i * W, wc = std::min(W, ncols - c0);
    e = copy_chunk(ctx->h2d_fld[s], ctx->h2d_precip[s], W, h, c0, wc, nlev, NF, NP, cudaMemcpyHostToDevice,
                   ctx->hst[s]);
    if (e != cudaSuccess) break;
    casim_state d;
    d.fld = ctx->h2d_fld[s];
    d.pitch = W;
    d.dz = ctx->h2d_dz;
    d.precip = ctx->h2d_precip[s];
    rc = step_device(ctx, &d, wc, nlev, dt, ctx->hst[s]);
    if (rc != CASIM_OK) break;
    e = copy_chunk(ctx->h2d_fld[s], ctx->h2d_precip[s], W, h, c0, wc, nlev, NF, NP, cudaMemcpyDeviceToHost,
                   ctx->hst[s]);
  }
  for (int s = 0; s < S; ++s) {
    const cudaError_t es = cudaStreamSynchronize(ctx->hst[s]);
    if (e == cudaSuccess) e = es;
  }
  if (e != cudaSuccess) return cuda_fail(e, "casim_step_host");
  if (rc == CASIM_OK) count_step(ctx, ncols, nlev);
  return rc;
}

extern "C" int casim_budget(casim_ctx *ctx, const casim_state *s, int ncols, int nlev, double *out, void *stream) {
  NvtxRange nvtx_range_("casim_budget");
  if (!ctx || !out) return CASIM_ERR_ARG;
  int rc = check_state(s, ncols, nlev, 1.0);
  if (rc != CASIM_OK || ncols == 0) return rc;
  const KArgs a = make_args(ctx, s, ncols, nlev, 1.0);
  k_budget<<<(unsigned)((ncols + 255) / 256), 256, 0, (cudaStream_t)stream>>>(a, out);
  ctx->launches++;
  CUDA_TRY(cudaGetLastError());
  return CASIM_OK;
}

extern "C" int casim_get_error(casim_ctx *ctx, unsigned *flags, void *stream) {
  if (!ctx) return CASIM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned h = 0;
  CUDA_TRY(cudaStreamSynchronize(st));
  CUDA_TRY(cudaMemcpy(&h, ctx->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemset(ctx->d_err, 0, sizeof(unsigned)));
  if (flags) *flags = h;
  if (h & CASIM_EFLAG_INDEX) return CASIM_ERR_INDEX;
  if (h & CASIM_EFLAG_TIMEOUT) return CASIM_ERR_TIMEOUT;
  if (h & CASIM_EFLAG_NONFINITE) return CASIM_ERR_NONFINITE;
  if (h & CASIM_EFLAG_CFL) return CASIM_ERR_CFL;
  return CASIM_OK;
}


extern "C" int casim_wait_selftest(casim_ctx *ctx, long long limit_ns, long long *elapsed_ns, void *stream) {
  NvtxRange nvtx_range_("casim_wait_selftest");
  if (!ctx || limit_ns < 1 || limit_ns > (long long)kWaitLimitNs || !elapsed_ns) return CASIM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long *d_el = nullptr;
  CUDA_TRY(cudaMalloc(&d_el, sizeof(unsigned long long)));
  k_wait_selftest<<<1, 32, 0, st>>>((uint64_t)limit_ns, ctx->d_err, d_el);
  ctx->launches++;
  cudaError_t e = cudaGetLastError();
  unsigned long long h = 0;
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaMemcpy(&h, d_el, sizeof h, cudaMemcpyDeviceToHost);
  cudaFree(d_el);
  if (e != cudaSuccess) return cuda_fail(e, "casim_wait_selftest");
  *elapsed_ns = (long long)h;
  return CASIM_OK;
}

// ------------------------------------------------------------------ batches
struct casim_batch {
  casim_ctx *ctx = nullptr;
  int ndom = 0;
  std::vector<DomDesc> dom;       // host copy of the device table
  std::vector<int> order;         // domains by descending level count
  DomDesc *d_dom = nullptr;
  int *d_list = nullptr, *d_count = nullptr, *d_counter = nullptr;
  Item *d_tiles = nullptr;
  int ntiles = 0;
  Item *d_items = nullptr;
  int nitems = 0, items_block = 0, items_cap = 0;
  long long total_cols = 0;
  long long total_pts = 0;        // sum of nlev pitch over the non-empty domains (per-point arrays)
  int maxlev = 1;                 // most levels of any domain
  int block = 128, compact = 1, persistent = 1;
  cudaGraphExec_t gexec = nullptr;
  int graph_steps = 0;
};

static std::vector<Item> make_items(const casim_batch &b, int width) {
  std::vector<Item> v;
  for (int d : b.order) {
    const int n = (b.dom[d].ncols + width - 1) / width;
    for (int ch = 0; ch < n; ++ch) v.push_back(Item{d, ch});
  }
  return v;
}

static int set_items(casim_batch *b, int block) {
  if (b->items_block == block) return CASIM_OK;
  std::vector<Item> v = make_items(*b, block);
  if ((int)v.size() > b->items_cap) {
    if (b->d_items) cudaFree(b->d_items);
    b->d_items = nullptr;
    b->items_cap = 0;
    cudaError_t e = cudaMalloc(&b->d_items, std::max<size_t>(1, v.size()) * sizeof(Item));
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? CASIM_ERR_OOM : cuda_fail(e, "cudaMalloc");
    b->items_cap = (int)v.size();
  }
  if (!v.empty()) CUDA_TRY(cudaMemcpy(b->d_items, v.data(), v.size() * sizeof(Item), cudaMemcpyHostToDevice));
  b->nitems = (int)v.size();
  b->items_block = block;
  return CASIM_OK;
}

extern "C" void casim_batch_free(casim_batch *b) {
  if (!b) return;
  cudaDeviceSynchronize();
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  cudaFree(b->d_dom);
  cudaFree(b->d_list);
  cudaFree(b->d_count);
  cudaFree(b->d_counter);
  cudaFree(b->d_tiles);
  cudaFree(b->d_items);
  delete b;
}

extern "C" int casim_batch_create(casim_ctx *ctx, const casim_state *domains, const int *ncols, const int *nlev,
                                  int ndom, casim_batch **out) {
  if (!out) return CASIM_ERR_ARG;
  *out = nullptr;
  if (!ctx || ctx->warm || ctx->tri || ctx->aero || ndom < 1 || !domains || !ncols || !nlev) return CASIM_ERR_ARG;
  casim_batch *b = new casim_batch();
  b->ctx = ctx;
  b->ndom = ndom;
  b->dom.resize(ndom);
  long long off = 0, pts = 0;
  std::vector<double> hdz;
  for (int i = 0; i < ndom; ++i) {
    const casim_state &s = domains[i];
    if (ncols[i] < 0 || nlev[i] < 1 || nlev[i] > kMaxLev) { delete b; return CASIM_ERR_ARG; }
    if (ncols[i] > 0 && (check_state(&s, ncols[i], nlev[i], 1.0) != CASIM_OK)) { delete b; return CASIM_ERR_ARG; }
    DomDesc &d = b->dom[i];
    d.fld = s.fld;
    d.pitch = s.pitch;
    d.dz = s.dz;
    d.precip = s.precip;
    d.ncols = ncols[i];
    d.nlev = nlev[i];
    d.list_off = off;
    d.pt_off = pts;
    d.dzmin = 1e300;
    if (ncols[i] > 0) {
      pts += (long long)nlev[i] * s.pitch;
      hdz.resize(nlev[i]);
      cudaError_t e = cudaMemcpy(hdz.data(), s.dz, nlev[i] * sizeof(double), cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) { delete b; return cuda_fail(e, "casim_batch_create: dz"); }
      for (double v : hdz) {
        if (!(v > 0.0)) { delete b; return CASIM_ERR_ARG; }
        d.dzmin = std::min(d.dzmin, v);
      }
    }
    off += ncols[i];
  }
  b->total_cols = off;
  b->total_pts = pts;
  for (int i = 0; i < ndom; ++i) b->maxlev = std::max(b->maxlev, nlev[i]);
  b->order.resize(ndom);
  for (int i = 0; i < ndom; ++i) b->order[i] = i;
  std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) { return b->dom[x].nlev > b->dom[y].nlev; });
  std::vector<Item> tiles = make_items(*b, kTile);
  b->ntiles = (int)tiles.size();
  cudaError_t e = cudaMalloc(&b->d_dom, ndom * sizeof(DomDesc));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_list, std::max<long long>(1, off) * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_count, ndom * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_tiles, std::max<size_t>(1, tiles.size()) * sizeof(Item));
  if (e == cudaSuccess) e = cudaMemcpy(b->d_dom, b->dom.data(), ndom * sizeof(DomDesc), cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !tiles.empty())
    e = cudaMemcpy(b->d_tiles, tiles.data(), tiles.size() * sizeof(Item), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    int rc = e == cudaErrorMemoryAllocation ? CASIM_ERR_OOM : cuda_fail(e, "casim_batch_create");
    casim_batch_free(b);
    return rc;
  }
  int rc = set_items(b, b->block);
  if (rc != CASIM_OK) { casim_batch_free(b); return rc; }
  *out = b;
  return CASIM_OK;
}

static BatchArgs batch_args(const casim_batch *b, double dt) {
  BatchArgs a;
  a.dom = b->d_dom;
  a.items = b->d_items;
  a.nitems = b->nitems;
  a.list = b->d_list;
  a.count = b->d_count;
  a.counter = b->d_counter;
  a.err = b->ctx->d_err;
  a.dt = dt;
  a.compact = b->compact;
  a.persistent = b->persistent;
  a.surr = nullptr;
  a.maxlev = b->maxlev;
  a.ndom = b->ndom;
  return a;
}

// the batch kernel for a block size: blocks of up to 128 threads take the
// instantiation with the single-domain step's register budget (mixed: 5
// blocks of 128 per SM, FP64: 3), wider blocks the one built for 256
template <class M>
static auto batch_kernel(int block) {
  return block <= kBatchNarrowBlock ? k_step_batch<M, true> : k_step_batch<M, false>;
}

template <class M>
static int persistent_grid(const casim_batch *b) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<M>(b->block), b->block,
                                                batch_smem_bytes<M>(b->block, b->maxlev));
  return std::max(1, per_sm) * b->ctx->nsm;
}

// enqueue one step of every domain (no validation; used by step and capture);
// surr: the surrogate's per-point rates of the batch (mixed form), or null
static int enqueue_batch_step(casim_batch *b, double dt, cudaStream_t st, const float4 *surr = nullptr) {
  casim_ctx *ctx = b->ctx;
  if (b->nitems == 0) return CASIM_OK;
  BatchArgs a = batch_args(b, dt);
  a.surr = surr;
  if (b->compact) {
    CUDA_TRY(cudaMemsetAsync(b->d_count, 0, b->ndom * sizeof(int), st));
    if (ctx->precision == CASIM_MIXED)
      k_compact<PolicyMix><<<b->ntiles, kTile, 0, st>>>(a, b->d_tiles, b->ntiles, ctx->kp);
    else
      k_compact<PolicyF64><<<b->ntiles, kTile, 0, st>>>(a, b->d_tiles, b->ntiles, ctx->kp);
    ctx->launches++;
    CUDA_TRY(cudaGetLastError());
  }
  if (b->persistent) CUDA_TRY(cudaMemsetAsync(b->d_counter, 0, sizeof(int), st));
  if (ctx->precision == CASIM_MIXED) {
    const int grid = b->persistent ? std::min(b->nitems, persistent_grid<PolicyMix>(b)) : b->nitems;
    batch_kernel<PolicyMix>(b->block)<<<grid, b->block, batch_smem_bytes<PolicyMix>(b->block, b->maxlev), st>>>(a, ctx->kp);
  } else {
    const int grid = b->persistent ? std::min(b->nitems, persistent_grid<PolicyF64>(b)) : b->nitems;
    batch_kernel<PolicyF64>(b->block)<<<grid, b->block, batch_smem_bytes<PolicyF64>(b->block, b->maxlev), st>>>(a, ctx->kp);
  }
  ctx->launches++;
  CUDA_TRY(cudaGetLastError());
  return CASIM_OK;
}

extern "C" int casim_batch_step(casim_ctx *ctx, casim_batch *b, double dt, void *stream) {
  NvtxRange nvtx_range_("casim_batch_step");
  if (!ctx || !b || b->ctx != ctx || !(dt > 0.0) || !std::isfinite(dt)) return CASIM_ERR_ARG;
  return enqueue_batch_step(b, dt, (cudaStream_t)stream);
}

extern "C" int casim_batch_config(casim_batch *b, int block, int compact, int persistent) {
  if (!b || (block != 64 && block != 128 && block != 256) || (compact != 0 && compact != 1) ||
      (persistent != 0 && persistent != 1))
    return CASIM_ERR_ARG;
  int rc = set_items(b, block);
  if (rc != CASIM_OK) return rc;
  b->block = block;
  b->compact = compact;
  b->persistent = persistent;
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    b->graph_steps = 0;
  }
  return CASIM_OK;
}

extern "C" int casim_batch_get_config(const casim_batch *b, int *block, int *compact, int *persistent) {
  if (!b) return CASIM_ERR_ARG;
  if (block) *block = b->block;
  if (compact) *compact = b->compact;
  if (persistent) *persistent = b->persistent;
  return CASIM_OK;
}

extern "C" int casim_batch_tune(casim_ctx *ctx, casim_batch *b, double dt, int steps, void *stream,
                                casim_tune_entry *table, int table_len) {
  NvtxRange nvtx_range_("casim_batch_tune");
  if (!ctx || !b || b->ctx != ctx || steps < 1 || !(dt > 0.0) || table_len < 0 || (table_len && !table))
    return CASIM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  static const int blocks[3] = {64, 128, 256};
  float best = 1e30f;
  int bb = b->block, bc = b->compact, bp = b->persistent;
  int n = 0;
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  int rc = CASIM_OK;
  for (int bi = 0; bi < 3 && rc == CASIM_OK; ++bi)
    for (int comp = 0; comp < 2 && rc == CASIM_OK; ++comp)
      for (int pers = 0; pers < 2 && rc == CASIM_OK; ++pers) {
        if ((rc = casim_batch_config(b, blocks[bi], comp, pers)) != CASIM_OK) break;
        if ((rc = enqueue_batch_step(b, dt, st)) != CASIM_OK) break;   // warm-up (a real step)
        cudaEventRecord(e0, st);
        for (int s = 0; s < steps && rc == CASIM_OK; ++s) rc = enqueue_batch_step(b, dt, st);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = cuda_fail(cudaGetLastError(), "casim_batch_tune"); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= steps;
        if (n < table_len) {
          table[n].block = blocks[bi];
          table[n].compact = comp;
          table[n].persistent = pers;
          table[n].ms_per_step = ms;
        }
        ++n;
        if (ms < best) { best = ms; bb = blocks[bi]; bc = comp; bp = pers; }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != CASIM_OK) return rc;
  return casim_batch_config(b, bb, bc, bp);
}

extern "C" int casim_batch_tune_steps(int steps) { return 12 * (steps + 1); }

extern "C" int casim_batch_graph(casim_ctx *ctx, casim_batch *b, double dt, int nsteps, void *stream) {
  NvtxRange nvtx_range_("casim_batch_graph");
  if (!ctx || !b || b->ctx != ctx || nsteps < 1 || !(dt > 0.0) || !std::isfinite(dt)) return CASIM_ERR_ARG;
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
    b->graph_steps = 0;
  }
  // capture on a private stream (the legacy default stream cannot capture)
  cudaStream_t cs;
  CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  const long long l0 = ctx->launches;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  int rc = CASIM_OK;
  if (e == cudaSuccess) {
    for (int s = 0; s < nsteps && rc == CASIM_OK; ++s) rc = enqueue_batch_step(b, dt, cs);
    cudaError_t e2 = cudaStreamEndCapture(cs, &g);
    if (rc == CASIM_OK && e2 != cudaSuccess) rc = cuda_fail(e2, "cudaStreamEndCapture");
  } else {
    rc = cuda_fail(e, "cudaStreamBeginCapture");
  }
  ctx->launches = l0;   // captured, not launched
  if (rc == CASIM_OK) {
    e = cudaGraphInstantiate(&b->gexec, g, 0);
    if (e != cudaSuccess) rc = cuda_fail(e, "cudaGraphInstantiate");
  }
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  if (rc == CASIM_OK) b->graph_steps = nsteps;
  (void)stream;
  return rc;
}

extern "C" int casim_batch_graph_launch(casim_batch *b, void *stream) {
  NvtxRange nvtx_range_("casim_batch_graph_launch");
  if (!b || !b->gexec) return CASIM_ERR_ARG;
  CUDA_TRY(cudaGraphLaunch(b->gexec, (cudaStream_t)stream));
  b->ctx->launches += (long long)b->graph_steps * (b->compact ? 2 : 1);
  return CASIM_OK;
}

extern "C" long long casim_batch_columns(const casim_batch *b) { return b ? b->total_cols : -1; }

// One call per timestep for many domains (the paper's one call per step that
// runs the whole scheme over every column, Section 3.2, with several domains
// in one launch).  The batch object is built on the first call and kept in
// the context while the same domain list comes back.
extern "C" int casim_step_batched(casim_ctx *ctx, const casim_state *domains, const int *ncols, const int *nlev,
                                  int ndom, double dt, void *stream) {
  NvtxRange nvtx_range_("casim_step_batched");
  if (!ctx || ndom < 1 || !domains || !ncols || !nlev || !(dt > 0.0) || !std::isfinite(dt)) return CASIM_ERR_ARG;
  bool same = ctx->sb && (int)ctx->sb_dom.size() == ndom;
  for (int i = 0; same && i < ndom; ++i) {
    const casim_state &a = ctx->sb_dom[i], &b = domains[i];
    same = a.fld == b.fld && a.pitch == b.pitch && a.dz == b.dz && a.precip == b.precip &&
           ctx->sb_ncols[i] == ncols[i] && ctx->sb_nlev[i] == nlev[i];
  }
  if (!same) {
    casim_batch_free(ctx->sb);
    ctx->sb = nullptr;
    ctx->sb_dom.clear();
    ctx->sb_ncols.clear();
    ctx->sb_nlev.clear();
    casim_batch *b = nullptr;
    const int rc = casim_batch_create(ctx, domains, ncols, nlev, ndom, &b);
    if (rc != CASIM_OK) return rc;
    ctx->sb = b;
    ctx->sb_dom.assign(domains, domains + ndom);
    ctx->sb_ncols.assign(ncols, ncols + ndom);
    ctx->sb_nlev.assign(nlev, nlev + ndom);
  }
  return casim_batch_step(ctx, ctx->sb, dt, stream);
}


// ------------------------------------------------------- allocation-free step
// Some callers cannot allocate device memory at all: code embedded in a host
// model whose memory pool owns the whole GPU, a plug-in running under a
// framework that forbids allocation while it is capturing or replaying work,
// or a real-time loop that must not risk an allocation failing mid-run.  For
// them casim_step_noalloc runs the compacted step (flag pass + step over the
// active-column list) with every piece of scratch memory taken from the
// fixed array below, which exists once per GPU for as long as the library is
// loaded.
constexpr int kNoallocMaxCols = CASIM_NOALLOC_MAX_COLS;
constexpr int kNoallocMaxTiles = (kNoallocMaxCols + kTile - 1) / kTile;

struct NoallocScratch {
  unsigned err;          // device error word of the call
  int counter;           // work counter of the persistent grid
  int count;             // active columns found by the flag pass
  int pad;
  DomDesc dom;           // the one domain
  Item tiles[kNoallocMaxTiles];
  int list[kNoallocMaxCols];
};

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

// Writes the call's domain table and tiles and clears the words that must
// start at zero; the column list needs no clearing (the flag pass fills it).
__global__ void k_noalloc_setup(NoallocScratch *sc, DomDesc d, int ntiles) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) {
    sc->err = 0u;
    sc->counter = 0;
    sc->count = 0;
    sc->dom = d;
  }
  if (i < ntiles) sc->tiles[i] = Item{0, i};
}


// smallest layer thickness of the no-alloc call's domain, into its table
__global__ void k_noalloc_dzmin(NoallocScratch *sc) {
  __shared__ double red[8];
  double m = 1e300;
  for (int k = threadIdx.x; k < sc->dom.nlev; k += blockDim.x) m = fmin(m, sc->dom.dz[k]);
  for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) m = fmin(m, red[i]);
    sc->dom.dzmin = fmin(m, red[0]);
  }
}

static NoallocScratch *noalloc_scratch_ptr(int dev, int *rc) {
  // set-up once per device, with that device current; host code must not
  // take the address of the __device__ array directly (that would be the
  // host-side stand-in, not device memory).  Host threads making their first
  // call on one device at the same time may both look the address up; they
  // find the same value, and the atomic entries make the concurrent stores
  // and loads well defined.
  static std::atomic<NoallocScratch *> ptrs[64];
  if (dev < 0 || dev >= 64) { *rc = CASIM_ERR_ARG; return nullptr; }
  NoallocScratch *cached = ptrs[dev].load(std::memory_order_acquire);
  if (!cached) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) { *rc = cuda_fail(e, "cudaGetSymbolAddress"); return nullptr; }
    cached = static_cast<NoallocScratch *>(p);
    ptrs[dev].store(cached, std::memory_order_release);
  }
  *rc = CASIM_OK;
  return cached;
}

extern "C" int casim_step_noalloc(const casim_params *params, int precision, const casim_state *s, int ncols,
                                  int nlev, double dt, void *stream, unsigned *flags) {
  NvtxRange nvtx_range_("casim_step_noalloc");
  if (precision != CASIM_FP64 && precision != CASIM_MIXED) return CASIM_ERR_ARG;
  int rc = check_state(s, ncols, nlev, dt);
  if (rc != CASIM_OK) return rc;
  if (ncols > kNoallocMaxCols) {
    std::snprintf(g_last_error, sizeof(g_last_error),
                  "casim_step_noalloc: %d columns exceed the fixed scratch of %d columns", ncols, kNoallocMaxCols);
    return CASIM_ERR_ARG;
  }
  if (flags) *flags = 0u;
  if (ncols == 0) return CASIM_OK;
  casim_params p;
  if (params) p = *params;
  else casim_default_params(&p);
  if (!params_ok(p)) return CASIM_ERR_ARG;
  KParams kp;
  derive<double>(p, kp.d, ln_);
  derive<float>(p, kp.f, log2_);
  kp.c_max = p.c_max;
  kp.T0 = p.T0;
  for (int x = 0; x < 5; ++x) kp.vmax[x] = p.vmax[x];

  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  NoallocScratch *sc = noalloc_scratch_ptr(dev, &rc);
  if (!sc) return rc;
  int nsm = 1;
  CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));

  // the domain's smallest layer thickness (which decides the fused
  // sedimentation path) is found on the device, without a host copy
  DomDesc d;
  d.fld = s->fld;
  d.pitch = s->pitch;
  d.dz = s->dz;
  d.precip = s->precip;
  d.ncols = ncols;
  d.nlev = nlev;
  d.dzmin = 0.0;   // replaced on the device by k_noalloc_dzmin
  d.list_off = 0;
  d.pt_off = 0;
  const int ntiles = (ncols + kTile - 1) / kTile;
  cudaStream_t st = (cudaStream_t)stream;
  k_noalloc_setup<<<(ntiles + 255) / 256, 256, 0, st>>>(sc, d, ntiles);
  k_noalloc_dzmin<<<1, 256, 0, st>>>(sc);
  CUDA_TRY(cudaGetLastError());

  BatchArgs a;
  a.dom = &sc->dom;
  a.items = sc->tiles;
  a.nitems = ntiles;
  a.list = sc->list;
  a.count = &sc->count;
  a.counter = &sc->counter;
  a.err = &sc->err;
  a.dt = dt;
  a.compact = 1;
  a.persistent = 1;
  a.surr = nullptr;
  a.maxlev = nlev;
  a.ndom = 1;
  int per_sm = 1;
  if (precision == CASIM_MIXED) {
    k_compact<PolicyMix><<<ntiles, kTile, 0, st>>>(a, sc->tiles, ntiles, kp);
    const size_t smem = batch_smem_bytes<PolicyMix>(kTile, nlev);
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<PolicyMix>(kTile), kTile, smem));
    batch_kernel<PolicyMix>(kTile)<<<std::min(ntiles, std::max(1, per_sm) * nsm), kTile, smem, st>>>(a, kp);
  } else {
    k_compact<PolicyF64><<<ntiles, kTile, 0, st>>>(a, sc->tiles, ntiles, kp);
    const size_t smem = batch_smem_bytes<PolicyF64>(kTile, nlev);
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<PolicyF64>(kTile), kTile, smem));
    batch_kernel<PolicyF64>(kTile)<<<std::min(ntiles, std::max(1, per_sm) * nsm), kTile, smem, st>>>(a, kp);
  }
  CUDA_TRY(cudaGetLastError());
  if (flags) {
    unsigned h = 0;
    CUDA_TRY(cudaMemcpyAsync(&h, &sc->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    *flags = h;
    if (h & CASIM_EFLAG_NONFINITE) return CASIM_ERR_NONFINITE;
    if (h & CASIM_EFLAG_CFL) return CASIM_ERR_CFL;
  }
  return CASIM_OK;
}


// ------------------------------------------------------------ surrogate network
struct casim_mlp {
  float *theta = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr;   // FP32 [kNParam]
  MlpBf16 wb{};
  __nv_bfloat16 *wbuf = nullptr;
  unsigned char *img = nullptr;   // weight images for the tcgen05 kernel
  float *wsplit = nullptr;        // split-K partial weight gradients [kSplitMax][256][256]
  unsigned *d_err = nullptr;
  int engine = 1;                 // 1: tcgen05 inference, 0: mma.sync
  float *norm = nullptr;   // [12 mean][12 sd][4 mean][4 sd]
  float *box = nullptr;    // [12 lo][12 hi]
  bool fitted = false;
  long long adam_t = 0;
  // batch workspace
  int cap_b = 0;
  __nv_bfloat16 *h0 = nullptr, *h1 = nullptr, *h2 = nullptr, *h3 = nullptr;
  __nv_bfloat16 *dzb4 = nullptr, *dzb3 = nullptr, *dzb2 = nullptr, *dzb1 = nullptr;
  float *a1 = nullptr, *a2 = nullptr, *a3 = nullptr, *y = nullptr;
  float *dz4 = nullptr, *dz3 = nullptr, *dz2 = nullptr, *dz1 = nullptr;
  float *Xn = nullptr, *Tn = nullptr, *Mb = nullptr, *cnt = nullptr;
  double *loss = nullptr;
  // surrogate-step scratch
  long long cap_rows = 0, cap_pts = 0;
  __nv_bfloat16 *xb = nullptr;
  long long *rowpt = nullptr;
  float4 *surr = nullptr;
  unsigned long long *rowctr = nullptr;
  // device-array inference: BF16 inputs [cap_f][16]
  long long cap_f = 0;
  __nv_bfloat16 *fxb = nullptr;
};

template <class T>
static cudaError_t dalloc(T **p, size_t n) {
  return cudaMalloc(reinterpret_cast<void **>(p), std::max<size_t>(n, 1) * sizeof(T));
}

static void mlp_free_batch(casim_mlp *m) {
  void *ps[] = {m->h0, m->h1, m->h2, m->h3, m->dzb4, m->dzb3, m->dzb2, m->dzb1, m->a1, m->a2, m->a3, m->y,
                m->dz4, m->dz3, m->dz2, m->dz1, m->Xn, m->Tn, m->Mb};
  for (void *p : ps) cudaFree(p);
  m->h0 = m->h1 = m->h2 = m->h3 = m->dzb4 = m->dzb3 = m->dzb2 = m->dzb1 = nullptr;
  m->a1 = m->a2 = m->a3 = m->y = m->dz4 = m->dz3 = m->dz2 = m->dz1 = m->Xn = m->Tn = m->Mb = nullptr;
  m->cap_b = 0;
}

static int mlp_batch_ws(casim_mlp *m, int n) {
  if (n <= m->cap_b) return CASIM_OK;
  mlp_free_batch(m);
  const size_t H = (size_t)n * kNh;
  cudaError_t e = dalloc(&m->h0, (size_t)n * kNinPad);
  if (e == cudaSuccess) e = dalloc(&m->h1, H);
  if (e == cudaSuccess) e = dalloc(&m->h2, H);
  if (e == cudaSuccess) e = dalloc(&m->h3, H);
  if (e == cudaSuccess) e = dalloc(&m->dzb4, (size_t)n * kNoutPad);
  if (e == cudaSuccess) e = dalloc(&m->dzb3, H);
  if (e == cudaSuccess) e = dalloc(&m->dzb2, H);
  if (e == cudaSuccess) e = dalloc(&m->dzb1, H);
  if (e == cudaSuccess) e = dalloc(&m->a1, H);
  if (e == cudaSuccess) e = dalloc(&m->a2, H);
  if (e == cudaSuccess) e = dalloc(&m->a3, H);
  if (e == cudaSuccess) e = dalloc(&m->y, (size_t)n * kNout);
  if (e == cudaSuccess) e = dalloc(&m->dz4, (size_t)n * kNout);
  if (e == cudaSuccess) e = dalloc(&m->dz3, H);
  if (e == cudaSuccess) e = dalloc(&m->dz2, H);
  if (e == cudaSuccess) e = dalloc(&m->dz1, H);
  if (e == cudaSuccess) e = dalloc(&m->Xn, (size_t)n * kNin);
  if (e == cudaSuccess) e = dalloc(&m->Tn, (size_t)n * kNout);
  if (e == cudaSuccess) e = dalloc(&m->Mb, (size_t)n * kNout);
  if (e != cudaSuccess) {
    mlp_free_batch(m);
    return e == cudaErrorMemoryAllocation ? CASIM_ERR_OOM : cuda_fail(e, "cudaMalloc");
  }
  m->cap_b = n;
  return CASIM_OK;
}

// the tcgen05 GEMM takes operands that are K-major or MN-major with
// 16-byte aligned rows (strides in multiples of 8 elements)
static bool tc_operands_ok(long long sr, long long sk) {
  return (sk == 1 && sr % 8 == 0) || (sr == 1 && sk % 8 == 0);
}

// one training GEMM: on the tensor-core engine (engine 1) the tcgen05 kernel,
// else (or for operands it does not take) the mma.sync kernel
template <class Epi>
static void launch_gemm(const casim_mlp *m, const GemmArgs &g, const Epi &epi, int nsplit, cudaStream_t st);

template <class Epi>
static void gemm(const casim_mlp *m, const __nv_bfloat16 *A, long long sam, long long sak, const __nv_bfloat16 *B,
                 long long sbn, long long sbk, int M, int N, int K, const Epi &epi, cudaStream_t st) {
  GemmArgs g{A, sam, sak, B, sbn, sbk, M, N, K, K};
  launch_gemm(m, g, epi, 1, st);
}

// weight gradient out[m][n] (ld N) = sum_k A(m, k) B(n, k) over a long K (the
// batch): K split into chunks (kSplitK rows on the mma.sync engine; on the
// tensor-core engine 256, enough chunks to give every SM a tile), partial
// tiles summed in order
constexpr int kSplitK = 512, kSplitKTc = 256, kSplitMax = 64;
static void gemm_wgrad(casim_mlp *m, const __nv_bfloat16 *A, long long sam, long long sak, const __nv_bfloat16 *B,
                       long long sbn, long long sbk, int M, int N, int K, float *out, cudaStream_t st) {
  const int split = m->engine == 1 ? kSplitKTc : kSplitK;
  const int kchunk = std::max(split, (K + kSplitMax - 1) / kSplitMax + kGBK - 1) / kGBK * kGBK;
  const int nsplit = (K + kchunk - 1) / kchunk;
  GemmArgs g{A, sam, sak, B, sbn, sbk, M, N, K, kchunk};
  const long long len = (long long)M * N;
  launch_gemm(m, g, EpiPartial{m->wsplit, N, len}, nsplit, st);
  k_splitk_sum<<<(unsigned)((len + 255) / 256), 256, 0, st>>>(m->wsplit, nsplit, len, out);
}

template <class Epi>
static void launch_gemm(const casim_mlp *m, const GemmArgs &g, const Epi &epi, int nsplit, cudaStream_t st) {
  if (m->engine == 1 && tc_operands_ok(g.sam, g.sak) && tc_operands_ok(g.sbn, g.sbk)) {
    const dim3 grid((g.N + kTcBN - 1) / kTcBN, (g.M + kTcBM - 1) / kTcBM, nsplit);
    k_gemm_tc<Epi><<<grid, 128, kTcSmem, st>>>(g, epi, m->d_err);
  } else {
    const dim3 grid((g.N + kGBN - 1) / kGBN, (g.M + kGBM - 1) / kGBM, nsplit);
    k_gemm<Epi><<<grid, 128, 0, st>>>(g, epi);
  }
}

// forward pass of n rows whose BF16 inputs are in m->h0; keep_act stores the
// FP32 activations the backward pass needs
static void mlp_forward(casim_mlp *m, int n, bool keep_act, cudaStream_t st) {
  gemm(m, m->h0, kNinPad, 1, m->wb.w1t, kNinPad, 1, n, kNh, kNinPad,
       EpiHidden{m->theta + kOffB1, keep_act ? m->a1 : nullptr, m->h1, kNh}, st);
  gemm(m, m->h1, kNh, 1, m->wb.w2t, kNh, 1, n, kNh, kNh, EpiHidden{m->theta + kOffB2, keep_act ? m->a2 : nullptr, m->h2, kNh}, st);
  gemm(m, m->h2, kNh, 1, m->wb.w3t, kNh, 1, n, kNh, kNh, EpiHidden{m->theta + kOffB3, keep_act ? m->a3 : nullptr, m->h3, kNh}, st);
  gemm(m, m->h3, kNh, 1, m->wb.w4t, kNh, 1, n, kNout, kNh, EpiOut{m->theta + kOffB4, m->y, kNout}, st);
}

// loss and gradient of n rows (inputs in h0, targets Tn, masks Mb)
static void mlp_backward(casim_mlp *m, int n, cudaStream_t st) {
  cudaMemsetAsync(m->cnt, 0, sizeof(float), st);
  cudaMemsetAsync(m->loss, 0, sizeof(double), st);
  k_sum<<<64, 256, 0, st>>>(m->Mb, (long long)n * kNout, m->cnt);
  const long long tot = (long long)n * kNoutPad;
  k_mlp_loss<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(m->y, m->Tn, m->Mb, n, m->cnt, m->loss, m->dz4, m->dzb4);
  const dim3 cs(32, kColsumY);
  // bias gradients: column sums over row chunks (into wsplit's tail), then in order
  float *cpart = m->wsplit + (size_t)(kSplitMax - 1) * kNh * kNh;
  auto colsum = [&](const float *dz, int cols, float *g) {
    k_colsum<<<dim3((cols + 31) / 32, kColsumChunks), cs, 0, st>>>(dz, n, cols, cols, cpart);
    k_colsum_fin<<<1, 256, 0, st>>>(cpart, kColsumChunks, cols, g);
  };
  // layer 4
  gemm_wgrad(m, m->h3, 1, kNh, m->dzb4, 1, kNoutPad, kNh, kNout, n, m->grad + kOffW4, st);
  colsum(m->dz4, kNout, m->grad + kOffB4);
  gemm(m, m->dzb4, kNoutPad, 1, m->wb.w4k, kNoutPad, 1, n, kNh, kNoutPad, EpiBackTanh{m->a3, m->dz3, m->dzb3, kNh}, st);
  // layer 3
  gemm_wgrad(m, m->h2, 1, kNh, m->dzb3, 1, kNh, kNh, kNh, n, m->grad + kOffW3, st);
  colsum(m->dz3, kNh, m->grad + kOffB3);
  gemm(m, m->dzb3, kNh, 1, m->wb.w3k, kNh, 1, n, kNh, kNh, EpiBackTanh{m->a2, m->dz2, m->dzb2, kNh}, st);
  // layer 2
  gemm_wgrad(m, m->h1, 1, kNh, m->dzb2, 1, kNh, kNh, kNh, n, m->grad + kOffW2, st);
  colsum(m->dz2, kNh, m->grad + kOffB2);
  gemm(m, m->dzb2, kNh, 1, m->wb.w2k, kNh, 1, n, kNh, kNh, EpiBackTanh{m->a1, m->dz1, m->dzb1, kNh}, st);
  // layer 1
  gemm_wgrad(m, m->h0, 1, kNinPad, m->dzb1, 1, kNh, kNin, kNh, n, m->grad + kOffW1, st);
  colsum(m->dz1, kNh, m->grad + kOffB1);
}

static void mlp_cast(casim_mlp *m, cudaStream_t st) {
  k_mlp_cast<<<(kNh * kNh + 255) / 256, 256, 0, st>>>(m->theta, m->wb);
  k_mlp_images<<<(kNh * kNh + 255) / 256, 256, 0, st>>>(m->theta, m->img);
}

// forward pass of n rows of BF16 inputs on the tcgen05 kernel: rates at the
// rows' points (rowpt) or standardised outputs in m->y (rowpt null)
// rows_dev: if set, the row count is read on the device (written by the
// feature pass before it on the stream) and n is its upper bound
static cudaError_t mlp_forward_umma(casim_mlp *m, const __nv_bfloat16 *xb, long long n, const long long *rowpt,
                                    float4 *surr, unsigned *err, int nsm, cudaStream_t st, float *y = nullptr,
                                    const unsigned long long *rows_dev = nullptr, long long npts = 0) {
  UmmaArgs u;
  u.npts = npts;
  u.xb = xb;
  u.rows = n;
  u.rows_dev = rows_dev;
  u.rowpt = rowpt;
  u.img = m->img;
  u.theta = m->theta;
  u.norm = m->norm;
  u.surr = surr;
  u.y = y ? y : m->y;
  u.err = err;
  const long long tiles = (n + 127) / 128;
  if (tiles == 0) return cudaSuccess;
  const int grid = (int)std::min<long long>(tiles, nsm);
  k_mlp_umma<<<grid, kUmmaThreads, kUmmaSmem, st>>>(u);
  return cudaGetLastError();
}

extern "C" void casim_mlp_free(casim_mlp *m) {
  if (!m) return;
  cudaDeviceSynchronize();
  mlp_free_batch(m);
  void *ps[] = {m->theta, m->grad, m->m1, m->m2, m->wbuf, m->norm, m->box, m->cnt, m->loss,
                m->xb, m->rowpt, m->surr, m->rowctr, m->img, m->wsplit, m->d_err, m->fxb};
  for (void *p : ps) cudaFree(p);
  delete m;
}

extern "C" int casim_mlp_create(casim_mlp **out, unsigned long long seed) {
  if (!out) return CASIM_ERR_ARG;
  *out = nullptr;
  casim_mlp *m = new casim_mlp();
  // Xavier-uniform weights, zero biases
  std::vector<float> th(kNParam, 0.f);
  std::mt19937_64 rng(seed);
  const int sz[5] = {kNin, kNh, kNh, kNh, kNout};
  const int offw[4] = {kOffW1, kOffW2, kOffW3, kOffW4};
  for (int l = 0; l < 4; ++l) {
    const double lim = std::sqrt(6.0 / (sz[l] + sz[l + 1]));
    std::uniform_real_distribution<double> u(-lim, lim);
    for (int i = 0; i < sz[l] * sz[l + 1]; ++i) th[offw[l] + i] = (float)u(rng);
  }
  const size_t nw = (size_t)kNh * kNinPad + 2 * (size_t)kNh * kNh + (size_t)kNoutPad * kNh +
                    2 * (size_t)kNh * kNh + (size_t)kNh * kNoutPad;
  cudaError_t e = dalloc(&m->theta, kNParam);
  if (e == cudaSuccess) e = dalloc(&m->grad, kNParam);
  if (e == cudaSuccess) e = dalloc(&m->m1, kNParam);
  if (e == cudaSuccess) e = dalloc(&m->m2, kNParam);
  if (e == cudaSuccess) e = dalloc(&m->wbuf, nw);
  if (e == cudaSuccess) e = dalloc(&m->norm, 2 * kNin + 2 * kNout);
  if (e == cudaSuccess) e = dalloc(&m->box, 2 * kNin);
  if (e == cudaSuccess) e = dalloc(&m->cnt, 1);
  if (e == cudaSuccess) e = dalloc(&m->loss, 1);
  if (e == cudaSuccess) e = dalloc(&m->rowctr, 1);
  if (e == cudaSuccess) e = dalloc(&m->img, kImgBytes);
  if (e == cudaSuccess) e = dalloc(&m->wsplit, (size_t)kSplitMax * kNh * kNh);
  if (e == cudaSuccess) e = dalloc(&m->d_err, 1);
  if (e == cudaSuccess) e = cudaMemset(m->d_err, 0, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mlp_umma, cudaFuncAttributeMaxDynamicSharedMemorySize, kUmmaSmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm_tc<EpiHidden>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm_tc<EpiOut>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm_tc<EpiBackTanh>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_gemm_tc<EpiPartial>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
  if (e == cudaSuccess) e = cudaMemcpy(m->theta, th.data(), kNParam * sizeof(float), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m->m1, 0, kNParam * sizeof(float));
  if (e == cudaSuccess) e = cudaMemset(m->m2, 0, kNParam * sizeof(float));
  if (e != cudaSuccess) {
    int rc = e == cudaErrorMemoryAllocation ? CASIM_ERR_OOM : cuda_fail(e, "casim_mlp_create");
    casim_mlp_free(m);
    return rc;
  }
  __nv_bfloat16 *w = m->wbuf;
  m->wb.w1t = w; w += (size_t)kNh * kNinPad;
  m->wb.w2t = w; w += (size_t)kNh * kNh;
  m->wb.w3t = w; w += (size_t)kNh * kNh;
  m->wb.w4t = w; w += (size_t)kNoutPad * kNh;
  m->wb.w2k = w; w += (size_t)kNh * kNh;
  m->wb.w3k = w; w += (size_t)kNh * kNh;
  m->wb.w4k = w;
  mlp_cast(m, 0);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaDeviceSynchronize());
  *out = m;
  return CASIM_OK;
}

extern "C" long long casim_mlp_param_count(void) { return kNParam; }

extern "C" int casim_mlp_set_params(casim_mlp *m, const float *host, long long n) {
  if (!m || !host || n != kNParam) return CASIM_ERR_ARG;
  CUDA_TRY(cudaMemcpy(m->theta, host, kNParam * sizeof(float), cudaMemcpyHostToDevice));
  mlp_cast(m, 0);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaDeviceSynchronize());
  return CASIM_OK;
}

extern "C" int casim_mlp_get_params(const casim_mlp *m, float *host, long long n) {
  if (!m || !host || n != kNParam) return CASIM_ERR_ARG;
  CUDA_TRY(cudaMemcpy(host, m->theta, kNParam * sizeof(float), cudaMemcpyDeviceToHost));
  return CASIM_OK;
}

// after the device has finished the network's work: a bounded wait of a
// tensor-core kernel that gave up (error bit 4) is reported, and cleared
static int mlp_wait_report(casim_mlp *m, const char *where) {
  unsigned herr = 0;
  CUDA_TRY(cudaMemcpy(&herr, m->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (herr) {
    cudaMemset(m->d_err, 0, sizeof(unsigned));
    std::snprintf(g_last_error, sizeof(g_last_error), "%s: a bounded wait of a tensor-core kernel gave up", where);
    return CASIM_ERR_TIMEOUT;
  }
  return CASIM_OK;
}

extern "C" int casim_mlp_set_engine(casim_mlp *m, int engine) {
  if (!m || (engine != 0 && engine != 1)) return CASIM_ERR_ARG;
  m->engine = engine;
  return CASIM_OK;
}

// largest row count of one casim_mlp_forward call (its BF16 input buffer is
// n x 32 bytes; the input kernel's grid stays below 2^31 threads)
constexpr long long kMlpForwardMaxRows = 1LL << 27;

extern "C" int casim_mlp_forward_host(casim_mlp *m, const float *Xn, int n, float *Y) {
  NvtxRange nvtx_range_("casim_mlp_forward_host");
  if (!m || !Xn || !Y || n < 1) return CASIM_ERR_ARG;
  int rc = mlp_batch_ws(m, n);
  if (rc != CASIM_OK) return rc;
  CUDA_TRY(cudaMemcpy(m->Xn, Xn, (size_t)n * kNin * sizeof(float), cudaMemcpyHostToDevice));
  k_mlp_inputs<<<(unsigned)(((long long)n * kNinPad + 255) / 256), 256>>>(m->Xn, n, m->h0);
  if (m->engine == 1) {
    int dev = 0, nsm = 1;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    CUDA_TRY(mlp_forward_umma(m, m->h0, n, nullptr, nullptr, m->d_err, nsm, 0));
  } else {
    mlp_forward(m, n, false, 0);
  }
  CUDA_TRY(cudaGetLastError());
  unsigned herr = 0;
  CUDA_TRY(cudaMemcpy(&herr, m->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (herr) {
    cudaMemset(m->d_err, 0, sizeof(unsigned));
    std::snprintf(g_last_error, sizeof(g_last_error), "casim_mlp_forward_host: a bounded wait gave up");
    return CASIM_ERR_CUDA;
  }
  CUDA_TRY(cudaMemcpy(Y, m->y, (size_t)n * kNout * sizeof(float), cudaMemcpyDeviceToHost));
  return CASIM_OK;
}

extern "C" int casim_mlp_forward(casim_mlp *m, const float *Xn, long long n, float *Y, void *stream) {
  NvtxRange nvtx_range_("casim_mlp_forward");
  if (!m || !Xn || !Y || n < 1 || n > kMlpForwardMaxRows) return CASIM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const unsigned gin = (unsigned)((n * kNinPad + 255) / 256);
  if (m->engine == 1) {
    if (n > m->cap_f) {
      cudaFree(m->fxb);
      m->fxb = nullptr;
      m->cap_f = 0;
      cudaError_t e = dalloc(&m->fxb, (size_t)n * kNinPad);
      if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? CASIM_ERR_OOM : cuda_fail(e, "cudaMalloc");
      m->cap_f = n;
    }
    k_mlp_inputs<<<gin, 256, 0, st>>>(Xn, (int)n, m->fxb);
    int dev = 0, nsm = 1;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    CUDA_TRY(mlp_forward_umma(m, m->fxb, n, nullptr, nullptr, m->d_err, nsm, st, Y));
  } else {
    int rc = mlp_batch_ws(m, (int)n);
    if (rc != CASIM_OK) return rc;
    k_mlp_inputs<<<gin, 256, 0, st>>>(Xn, (int)n, m->h0);
    mlp_forward(m, (int)n, false, st);
    CUDA_TRY(cudaMemcpyAsync(Y, m->y, (size_t)n * kNout * sizeof(float), cudaMemcpyDeviceToDevice, st));
  }
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(st));
  unsigned herr = 0;
  CUDA_TRY(cudaMemcpy(&herr, m->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (herr) {
    cudaMemset(m->d_err, 0, sizeof(unsigned));
    std::snprintf(g_last_error, sizeof(g_last_error), "casim_mlp_forward: a bounded wait gave up");
    return CASIM_ERR_CUDA;
  }
  return CASIM_OK;
}

extern "C" int casim_mlp_loss_grad_host(casim_mlp *m, const float *Xn, const float *Tn, const float *M, int n,
                                        double *loss, float *grad) {
  if (!m || !Xn || !Tn || !M || n < 1) return CASIM_ERR_ARG;
  int rc = mlp_batch_ws(m, n);
  if (rc != CASIM_OK) return rc;
  CUDA_TRY(cudaMemcpy(m->Xn, Xn, (size_t)n * kNin * sizeof(float), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(m->Tn, Tn, (size_t)n * kNout * sizeof(float), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(m->Mb, M, (size_t)n * kNout * sizeof(float), cudaMemcpyHostToDevice));
  k_mlp_inputs<<<(unsigned)(((long long)n * kNinPad + 255) / 256), 256>>>(m->Xn, n, m->h0);
  mlp_forward(m, n, true, 0);
  mlp_backward(m, n, 0);
  CUDA_TRY(cudaGetLastError());
  if (loss) CUDA_TRY(cudaMemcpy(loss, m->loss, sizeof(double), cudaMemcpyDeviceToHost));
  if (grad) CUDA_TRY(cudaMemcpy(grad, m->grad, kNParam * sizeof(float), cudaMemcpyDeviceToHost));
  return mlp_wait_report(m, "casim_mlp_loss_grad_host");
}

extern "C" int casim_mlp_data(casim_ctx *ctx, const casim_state *s, int ncols, int nlev, double dt, float *X,
                              float *Y, float *M, long long *pts, long long cap, long long *rows, void *stream) {
  NvtxRange nvtx_range_("casim_mlp_data");
  if (!ctx || ctx->warm || ctx->tri || ctx->aero || !X || !Y || !M || cap < 0 || !rows) return CASIM_ERR_ARG;
  int rc = check_state(s, ncols, nlev, dt);
  if (rc != CASIM_OK) return rc;
  *rows = 0;
  if (ncols == 0) return CASIM_OK;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long *ctr = nullptr;
  CUDA_TRY(cudaMalloc(&ctr, sizeof(unsigned long long)));
  cudaMemsetAsync(ctr, 0, sizeof(unsigned long long), st);
  FeatArgs fa{};
  fa.mode = 0;
  fa.cap = cap;
  fa.rows = ctr;
  fa.X = X;
  fa.Y = Y;
  fa.M = M;
  fa.rowpt = pts;
  const KArgs a = make_args(ctx, s, ncols, nlev, dt);
  const long long np = (long long)nlev * s->pitch;
  k_mlp_features<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(a, ctx->kp, fa);
  ctx->launches++;
  unsigned long long h = 0;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, ctr, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(ctr);
  if (e != cudaSuccess) return cuda_fail(e, "casim_mlp_data");
  *rows = (long long)h;   // may exceed cap: only cap rows were written
  return CASIM_OK;
}

extern "C" int casim_mlp_fit(casim_mlp *m, const float *X, const float *Y, const float *M, long long n, int steps,
                             int batch, float lr, unsigned long long seed, float *loss_hist, void *stream) {
  NvtxRange nvtx_range_("casim_mlp_fit");
  if (!m || !X || !Y || !M || n < 2 || steps < 0 || batch < 1) return CASIM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  // normalisation and the out-of-distribution box from the data
  double *acc = nullptr;
  int *lh = nullptr;
  CUDA_TRY(cudaMalloc(&acc, (2 * kNin + 3 * kNout) * sizeof(double)));
  CUDA_TRY(cudaMalloc(&lh, 2 * kNin * sizeof(int)));
  std::vector<int> init(2 * kNin);
  for (int k = 0; k < kNin; ++k) { init[k] = 0x7fffffff; init[kNin + k] = -0x7fffffff; }
  cudaMemsetAsync(acc, 0, (2 * kNin + 3 * kNout) * sizeof(double), st);
  cudaMemcpyAsync(lh, init.data(), 2 * kNin * sizeof(int), cudaMemcpyHostToDevice, st);
  k_mlp_stats<<<256, 256, 0, st>>>(X, Y, M, n, acc);
  k_mlp_box<<<256, 256, 0, st>>>(X, n, lh, lh + kNin);
  std::vector<double> ha(2 * kNin + 3 * kNout);
  std::vector<int> hl(2 * kNin);
  cudaMemcpyAsync(ha.data(), acc, ha.size() * sizeof(double), cudaMemcpyDeviceToHost, st);
  cudaMemcpyAsync(hl.data(), lh, hl.size() * sizeof(int), cudaMemcpyDeviceToHost, st);
  cudaError_t e = cudaStreamSynchronize(st);
  cudaFree(acc);
  cudaFree(lh);
  if (e != cudaSuccess) return cuda_fail(e, "casim_mlp_fit: statistics");
  float norm[2 * kNin + 2 * kNout], box[2 * kNin];
  for (int k = 0; k < kNin; ++k) {
    const double mu = ha[k] / n, var = ha[kNin + k] / n - mu * mu;
    norm[k] = (float)mu;
    norm[kNin + k] = (float)std::sqrt(std::max(var, 1e-12));
    auto ordf = [](int i) { const int b = i >= 0 ? i : i ^ 0x7fffffff; float f; std::memcpy(&f, &b, 4); return f; };
    box[k] = ordf(hl[k]);
    box[kNin + k] = ordf(hl[kNin + k]);
  }
  for (int c = 0; c < kNout; ++c) {
    const double cnt = std::max(ha[2 * kNin + 2 * kNout + c], 1.0);
    const double mu = ha[2 * kNin + c] / cnt, var = ha[2 * kNin + kNout + c] / cnt - mu * mu;
    norm[2 * kNin + c] = (float)mu;
    norm[2 * kNin + kNout + c] = (float)std::sqrt(std::max(var, 1e-12));
  }
  CUDA_TRY(cudaMemcpyAsync(m->norm, norm, sizeof(norm), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(m->box, box, sizeof(box), cudaMemcpyHostToDevice, st));
  m->fitted = true;
  int rc = mlp_batch_ws(m, batch);
  if (rc != CASIM_OK) return rc;
  for (int s = 0; s < steps; ++s) {
    k_mlp_batch<<<(batch + 255) / 256, 256, 0, st>>>(X, Y, M, n, seed, s, batch, m->norm, m->Xn, m->Tn, m->Mb);
    k_mlp_inputs<<<(unsigned)(((long long)batch * kNinPad + 255) / 256), 256, 0, st>>>(m->Xn, batch, m->h0);
    mlp_forward(m, batch, true, st);
    mlp_backward(m, batch, st);
    ++m->adam_t;
    const float c1 = 1.f - (float)std::pow(0.9, (double)m->adam_t), c2 = 1.f - (float)std::pow(0.999, (double)m->adam_t);
    k_adam<<<(kNParam + 255) / 256, 256, 0, st>>>(m->theta, m->grad, m->m1, m->m2, kNParam, lr, 0.9f, 0.999f, 1e-8f, c1, c2);
    mlp_cast(m, st);
    if (loss_hist) {
      double l = 0.0;
      CUDA_TRY(cudaMemcpyAsync(&l, m->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
      CUDA_TRY(cudaStreamSynchronize(st));
      loss_hist[s] = (float)l;
    }
  }
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaStreamSynchronize(st));
  return mlp_wait_report(m, "casim_mlp_fit");
}

extern "C" int casim_mlp_get_norm(const casim_mlp *m, float *stats) {
  if (!m || !stats || !m->fitted) return CASIM_ERR_ARG;
  CUDA_TRY(cudaMemcpy(stats, m->norm, (2 * kNin + 2 * kNout) * sizeof(float), cudaMemcpyDeviceToHost));
  CUDA_TRY(cudaMemcpy(stats + 2 * kNin + 2 * kNout, m->box, 2 * kNin * sizeof(float), cudaMemcpyDeviceToHost));
  return CASIM_OK;
}

extern "C" int casim_mlp_set_norm(casim_mlp *m, const float *stats) {
  if (!m || !stats) return CASIM_ERR_ARG;
  CUDA_TRY(cudaMemcpy(m->norm, stats, (2 * kNin + 2 * kNout) * sizeof(float), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMemcpy(m->box, stats + 2 * kNin + 2 * kNout, 2 * kNin * sizeof(float), cudaMemcpyHostToDevice));
  m->fitted = true;
  return CASIM_OK;
}

// the surrogate step's scratch for np points: BF16 features and the point
// of each row (a row per point at most), the rates at every point
static int surrogate_scratch(casim_mlp *m, long long np) {
  if (np <= m->cap_pts) return CASIM_OK;
  cudaFree(m->xb);
  cudaFree(m->rowpt);
  cudaFree(m->surr);
  m->xb = nullptr;
  m->rowpt = nullptr;
  m->surr = nullptr;
  m->cap_pts = m->cap_rows = 0;
  cudaError_t e = dalloc(&m->xb, (size_t)np * kNinPad);
  if (e == cudaSuccess) e = dalloc(&m->rowpt, (size_t)np);
  if (e == cudaSuccess) e = dalloc(&m->surr, (size_t)np);
  if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? CASIM_ERR_OOM : cuda_fail(e, "cudaMalloc");
  m->cap_pts = m->cap_rows = np;
  return CASIM_OK;
}

extern "C" int casim_step_surrogate(casim_ctx *ctx, casim_mlp *m, const casim_state *s, int ncols, int nlev,
                                    double dt, void *stream, long long *served) {
  NvtxRange nvtx_range_("casim_step_surrogate");
  if (!ctx || ctx->warm || ctx->tri || ctx->aero || !m || !m->fitted || ctx->precision != CASIM_MIXED) return CASIM_ERR_ARG;
  int rc = check_state(s, ncols, nlev, dt);
  if (rc != CASIM_OK || ncols == 0) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const long long np = (long long)nlev * s->pitch;
  if ((rc = surrogate_scratch(m, np)) != CASIM_OK) return rc;
  // 1. features of every warm point inside the box; NaN rates outside it
  CUDA_TRY(cudaMemsetAsync(m->rowctr, 0, sizeof(unsigned long long), st));
  FeatArgs fa{};
  fa.mode = 1;
  fa.cap = m->cap_rows;
  fa.rows = m->rowctr;
  fa.xb = m->xb;
  fa.rowpt = m->rowpt;
  fa.surr = m->surr;
  fa.norm = m->norm;
  fa.box = m->box;
  KArgs a = make_args(ctx, s, ncols, nlev, dt);
  k_mlp_features<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(a, ctx->kp, fa);
  ctx->launches++;
  unsigned long long hrows = 0;
  CUDA_TRY(cudaMemcpyAsync(&hrows, m->rowctr, sizeof(hrows), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  const long long rows = std::min((long long)hrows, m->cap_rows);
  // 2. the network on the rows
  if (m->engine == 1) {
    CUDA_TRY(mlp_forward_umma(m, m->xb, rows, m->rowpt, m->surr, ctx->d_err, ctx->nsm, st, nullptr, nullptr, np));
    ctx->launches++;
  } else {
    const int chunk = 1 << 17;
    if ((rc = mlp_batch_ws(m, (int)std::min<long long>(chunk, std::max<long long>(rows, 1)))) != CASIM_OK) return rc;
    for (long long r0 = 0; r0 < rows; r0 += m->cap_b) {
      const int n = (int)std::min<long long>(m->cap_b, rows - r0);
      __nv_bfloat16 *save = m->h0;
      m->h0 = m->xb + r0 * kNinPad;
      mlp_forward(m, n, false, st);
      m->h0 = save;
      k_mlp_scatter<<<(n + 255) / 256, 256, 0, st>>>(m->y, n, m->rowpt + r0, m->norm, m->surr, np, ctx->d_err);
      ctx->launches += 5;
    }
  }
  // 3. the step, taking the network's rates where given
  a.surr = m->surr;
  const dim3 grid((unsigned)((ncols + kBlock - 1) / kBlock));
  k_step<PolicyMix, false><<<grid, kBlock, step_smem_bytes<PolicyMix, false>(nlev), st>>>(a, ctx->kp, nullptr);
  ctx->launches++;
  CUDA_TRY(cudaGetLastError());
  if (served) *served = rows;
  return CASIM_OK;
}

// Every domain of a batch with the surrogate's warm-rain rates: one feature
// pass over all the batch's points, one network launch over their rows and
// the batch's step launch(es) reading the network's rates where it gave them.
// On the tensor-core engine the network reads the row count on the device,
// so nothing waits for the host unless `served` is asked for.
extern "C" int casim_batch_step_surrogate(casim_ctx *ctx, casim_batch *b, casim_mlp *m, double dt, void *stream,
                                          long long *served) {
  NvtxRange nvtx_range_("casim_batch_step_surrogate");
  if (!ctx || !b || b->ctx != ctx || ctx->precision != CASIM_MIXED || !m || !m->fitted || !(dt > 0.0) ||
      !std::isfinite(dt))
    return CASIM_ERR_ARG;
  if (served) *served = 0;
  if (b->total_pts == 0) return CASIM_OK;
  int rc = surrogate_scratch(m, b->total_pts);
  if (rc != CASIM_OK) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  // 1. features of every warm point inside the box, in one pass over all domains
  CUDA_TRY(cudaMemsetAsync(m->rowctr, 0, sizeof(unsigned long long), st));
  FeatArgs fa{};
  fa.mode = 1;
  fa.cap = m->cap_rows;
  fa.rows = m->rowctr;
  fa.xb = m->xb;
  fa.rowpt = m->rowpt;
  fa.surr = m->surr;
  fa.norm = m->norm;
  fa.box = m->box;
  k_mlp_features_batch<<<(unsigned)((b->total_pts + 255) / 256), 256, 0, st>>>(b->d_dom, b->ndom, b->total_pts, dt,
                                                                               ctx->kp, fa);
  ctx->launches++;
  CUDA_TRY(cudaGetLastError());
  // 2. the network on the rows
  long long rows = -1;
  if (m->engine == 1) {
    CUDA_TRY(mlp_forward_umma(m, m->xb, m->cap_rows, m->rowpt, m->surr, ctx->d_err, ctx->nsm, st, nullptr,
                              m->rowctr, b->total_pts));
    ctx->launches++;
  } else {
    unsigned long long hrows = 0;
    CUDA_TRY(cudaMemcpyAsync(&hrows, m->rowctr, sizeof(hrows), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    rows = std::min((long long)hrows, m->cap_rows);
    const int chunk = 1 << 17;
    if ((rc = mlp_batch_ws(m, (int)std::min<long long>(chunk, std::max<long long>(rows, 1)))) != CASIM_OK) return rc;
    for (long long r0 = 0; r0 < rows; r0 += m->cap_b) {
      const int n = (int)std::min<long long>(m->cap_b, rows - r0);
      __nv_bfloat16 *save = m->h0;
      m->h0 = m->xb + r0 * kNinPad;
      mlp_forward(m, n, false, st);
      m->h0 = save;
      k_mlp_scatter<<<(n + 255) / 256, 256, 0, st>>>(m->y, n, m->rowpt + r0, m->norm, m->surr, b->total_pts,
                                                     ctx->d_err);
      ctx->launches += 5;
    }
  }
  // 3. the batch's step, taking the network's rates where given
  if ((rc = enqueue_batch_step(b, dt, st, m->surr)) != CASIM_OK) return rc;
  if (served) {
    if (rows < 0) {
      unsigned long long hrows = 0;
      CUDA_TRY(cudaMemcpyAsync(&hrows, m->rowctr, sizeof(hrows), cudaMemcpyDeviceToHost, st));
      CUDA_TRY(cudaStreamSynchronize(st));
      rows = std::min((long long)hrows, m->cap_rows);
    }
    *served = rows;
  }
  return CASIM_OK;
}

extern "C" long long casim_launch_count(const casim_ctx *ctx) { return ctx ? ctx->launches : -1; }

// ---------------------------------------------------------------- checkpoints
namespace {
struct CkptHeader {
  char tag[8];                 // "CASIMSV1"
  int32_t abi, nfields, nprecip, nlev, pitch, ncols;
  uint64_t params_hash;        // FNV-1a of the parameter block
};

uint64_t params_hash(const casim_params *params) {
  casim_params p;
  if (params) p = *params;
  else casim_default_params(&p);
  const unsigned char *b = reinterpret_cast<const unsigned char *>(&p);
  uint64_t h = 1469598103934665603ull;
  for (size_t i = 0; i < sizeof(p); ++i) h = (h ^ b[i]) * 1099511628211ull;
  return h;
}

int ckpt_check(const casim_state *s, int ncols, int nlev, int nfields) {
  if (!s || !s->fld || !s->dz || !s->precip || ncols < 0 || nlev < 1 || nlev > kMaxLev) return CASIM_ERR_ARG;
  if (s->pitch < ncols || s->pitch % 32 != 0) return CASIM_ERR_ARG;
  if (nfields != CASIM_NFIELDS && nfields != CASIM_NFIELDS_AEROSOL && nfields != CASIM_NFIELDS_3MOM &&
      nfields != CASIM_NFIELDS_3MOM_COLD && nfields != CASIM_NFIELDS_AEROSOL_COLD)
    return CASIM_ERR_ARG;
  return CASIM_OK;
}
}  // namespace

extern "C" int casim_state_save(const char *path, const casim_params *params, const casim_state *s, int ncols,
                                int nlev, int nfields, void *stream) {
  NvtxRange nvtx_range_("casim_state_save");
  if (!path) return CASIM_ERR_ARG;
  int rc = ckpt_check(s, ncols, nlev, nfields);
  if (rc != CASIM_OK) return rc;
  CkptHeader h{};
  std::memcpy(h.tag, "CASIMSV1", 8);
  h.abi = CASIM_ABI_VERSION;
  h.nfields = nfields;
  h.nprecip = CASIM_NPRECIP + (nfields == CASIM_NFIELDS_AEROSOL || nfields == CASIM_NFIELDS_AEROSOL_COLD);
  h.nlev = nlev;
  h.pitch = s->pitch;
  h.ncols = ncols;
  h.params_hash = params_hash(params);
  const size_t nf = (size_t)nfields * nlev * s->pitch, np = (size_t)h.nprecip * s->pitch;
  std::vector<double> buf(nlev + nf + np);
  cudaStream_t st = (cudaStream_t)stream;
  CUDA_TRY(cudaMemcpyAsync(buf.data(), s->dz, (size_t)nlev * sizeof(double), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(buf.data() + nlev, s->fld, nf * sizeof(double), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(buf.data() + nlev + nf, s->precip, np * sizeof(double), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  FILE *f = std::fopen(path, "wb");
  if (!f) return CASIM_ERR_IO;
  const bool ok = std::fwrite(&h, sizeof h, 1, f) == 1 && std::fwrite(buf.data(), sizeof(double), buf.size(), f) == buf.size();
  return (std::fclose(f) == 0 && ok) ? CASIM_OK : CASIM_ERR_IO;
}

extern "C" int casim_state_load(const char *path, const casim_params *params, const casim_state *s, int ncols,
                                int nlev, int nfields, void *stream) {
  NvtxRange nvtx_range_("casim_state_load");
  if (!path) return CASIM_ERR_ARG;
  int rc = ckpt_check(s, ncols, nlev, nfields);
  if (rc != CASIM_OK) return rc;
  FILE *f = std::fopen(path, "rb");
  if (!f) return CASIM_ERR_IO;
  CkptHeader h{};
  if (std::fread(&h, sizeof h, 1, f) != 1) {
    std::fclose(f);
    return CASIM_ERR_IO;
  }
  if (std::memcmp(h.tag, "CASIMSV1", 8) != 0 || h.abi != CASIM_ABI_VERSION || h.nfields != nfields ||
      h.nprecip != CASIM_NPRECIP + (nfields == CASIM_NFIELDS_AEROSOL || nfields == CASIM_NFIELDS_AEROSOL_COLD) ||
      h.nlev != nlev || h.pitch != s->pitch ||
      h.ncols != ncols || h.params_hash != params_hash(params)) {
    std::fclose(f);
    return CASIM_ERR_ARG;
  }
  const size_t nf = (size_t)nfields * nlev * s->pitch, np = (size_t)h.nprecip * s->pitch;
  std::vector<double> buf(nlev + nf + np);
  const bool ok = std::fread(buf.data(), sizeof(double), buf.size(), f) == buf.size();
  std::fclose(f);
  if (!ok) return CASIM_ERR_IO;
  cudaStream_t st = (cudaStream_t)stream;
  CUDA_TRY(cudaMemcpyAsync(const_cast<double *>(s->dz), buf.data(), (size_t)nlev * sizeof(double),
                           cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(s->fld, buf.data() + nlev, nf * sizeof(double), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(s->precip, buf.data() + nlev + nf, np * sizeof(double), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  return CASIM_OK;
}

extern "C" int casim_get_stats(casim_ctx *ctx, casim_stats *out, int reset, void *stream) {
  if (!ctx || !ctx->stats || !out) return CASIM_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned long long h[kStatsWords];
  CUDA_TRY(cudaMemcpyAsync(h, ctx->d_stats, sizeof(h), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  out->steps = ctx->stat_steps;
  out->points = ctx->stat_points;
  out->active_points = (long long)h[0];
  out->changed_points = (long long)h[1];
  out->active_columns = (long long)h[2];
  for (int x = 0; x < 4; ++x)
    for (int n = 0; n < 65; ++n) out->nsub[x][n] = (long long)h[3 + 65 * x + n];
  if (reset) {
    CUDA_TRY(cudaMemsetAsync(ctx->d_stats, 0, sizeof(h), st));
    CUDA_TRY(cudaStreamSynchronize(st));
    ctx->stat_steps = ctx->stat_points = 0;
  }
  return CASIM_OK;
}

extern "C" void casim_free(casim_ctx *ctx) {
  if (!ctx) return;
  cudaDeviceSynchronize();
  casim_batch_free(ctx->sb);
  if (ctx->d_stats) cudaFree(ctx->d_stats);
  if (ctx->d_err) cudaFree(ctx->d_err);
  for (int s = 0; s < casim_ctx::kStages; ++s) {
    if (ctx->h2d_fld[s]) cudaFree(ctx->h2d_fld[s]);
    if (ctx->h2d_precip[s]) cudaFree(ctx->h2d_precip[s]);
    if (ctx->hst[s]) cudaStreamDestroy(ctx->hst[s]);
  }
  if (ctx->h2d_dz) cudaFree(ctx->h2d_dz);
  if (ctx->hev_start) cudaEventDestroy(ctx->hev_start);
  if (ctx->hev_dz) cudaEventDestroy(ctx->hev_dz);
  delete ctx;
}
