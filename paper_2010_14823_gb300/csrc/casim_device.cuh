// Device code of the column-microphysics step (sm_103a).
//
// One thread owns one column and walks it from the top level down
// (Section 3.2 of the paper maps one column to one GPU thread as well; the
// column's levels are coupled only through sedimentation).  Loads and stores
// are level-major, so the 32 threads of a warp touch 32 consecutive columns of
// one level: every access is a coalesced 256-byte row.
//
// Two precision policies share the process formulas:
//   PolicyF64  every operation in FP64, transfers applied in the order of the
//              scheme's transfer list;
//   PolicyMix  rates, fall speeds and special functions in FP32 on the MUFU
//              pipe (ex2/lg2); each field's increments at a point (process
//              transfers, sedimentation) are summed in FP32 and added to the
//              FP64 state once, so the state keeps FP64 resolution and total
//              water is conserved to the FP32 rounding of those sums.
// GB300 issues FP64 (and FP32<->FP64 conversions) at about 1/70 of the FP32
// rate, so the mixed policy converts between the two with integer bit
// operations and keeps FP64 to one addition per changed field.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace casim_dev {

constexpr int kMaxLev = 1024;    // levels per column held in shared memory (dz)
constexpr int kBlock = 128;      // threads (columns) per block

// ------------------------------------------------------------- constants
template <class R>
struct SpeciesK {
  R lglamfac;   // log(a Gamma(mu+b+1) / Gamma(mu+1)) in the policy's log base
  R invb;       // 1 / b
  R lglo, lghi; // log of the lambda clamp bounds
  R ev1, ex1;   // 0.78 Gamma(mu+2)/Gamma(mu+b+1)/a,      exponent b-1
  R ev2, ex2;   // 0.31 sqrt(cv) Gamma(mu+(d+5)/2)/..,    exponent b-(d+3)/2
  R rim, exr;   // (pi/4) E cv Gamma(mu+d+3)/Gamma(mu+b+1)/a, exponent b-2-d
  R vq, vn, exv;// cv Gamma ratios of the mass / number weighted speeds, exponent -d
  R vmax;
  R dep;        // 4 pi ccap
  R mlt;        // 4 pi ccap Ka / Lf
};

template <class R>
struct ConstK {
  R T0, Tnuc, qmin;
  R tnuc0;                          // Tnuc - T0, formed in FP64
  R t0_esit, t0_esib;               // T0 - es_it, T0 - es_ib
  R lv_cp, cp_lv, cp, inv_cp, lv, ls, lf;
  R eps, ome;                       // Rd/Rv, 1 - Rd/Rv
  R esl0, esla, eslb, eslab;        // Bolton
  R esi0, esia, esit, esib;         // ice
  R awc, aic, rv_dv;                // Lv^2/(Ka Rv), Ls^2/(Ka Rv), Rv/Dv
  // activation (Abdul-Razzak & Ghan 2000)
  R akel;                           // 2 sigma_w Mw / (rho_w R): A = akel / T
  R smc;                            // 2/sqrt(kappa) (1/(3 r_m))^1.5: S_m = smc A^1.5
  R al1, al2;                       // g Mw Lv/(cp R), g Ma / R
  R ga1, ga2;                       // R / Mw, Mw Lv^2 / (cp Ma)
  R gg1, gg2, gg3;                  // rho_w R/(Dv Mw), Lv rho_w / Ka, Lv Mw / R
  R twopirhow, f1, f2, uc;          // 2 pi rho_w, f1, f2, 2/(3 sqrt2 ln sigma)
  // warm rain
  R kk_aut, kk_aut_qc, kk_aut_nc, nc_min, kk_acc, kk_acc_exp, kcf, kr, inv_mr0;
  // nucleation
  R mey_a, mey_b, mey_c, mi0;
  // air
  R mu_air, inv_dv, lgrho0, twopi;
  SpeciesK<R> sp[5];
  // triple-moment species r, i, s, g (index 0..3, species 1..4): what their
  // shape-dependent constants are built from
  R s3_a[4], s3_dv[4], s3_mu0[4];    // a (M3 = q / a), fall-speed exponent d, fixed shape
  R s3_lgdmax[4], s3_lgdmin[4];      // log of the mean-diameter bounds (policy base)
  R s3_ev1c[4], s3_ev2c[4], s3_cv[4], s3_rimc[4];   // 0.78 / a, 0.31 sqrt(cv) / a, cv, (pi/4) E cv / a
  R s3_ar2[4];                       // (a_x / a_r)^2: a particle's sixth moment in rain diameters
  R s3_mumax;                        // largest shape
  R s3_d0_6;                         // (2 r0)^6: sixth moment of one new drop
  R s3_di_6;                         // (m_i0 / a_i)^2: of one new crystal
};

struct KParams {
  ConstK<double> d;
  ConstK<float> f;
  double T0;
  double c_max;
  double vmax[5];
};

struct KArgs {
  double *fld;
  long long pitch;
  const double *dz;
  double *precip;
  unsigned *err;
  int ncols, nlev;
  double dt;
  const float4 *surr;   // [nlev][pitch] surrogate warm-rain rates (mixed form), or null
  unsigned long long *stats;   // per-step statistics (the statistics build of the step), or null
};

// Per-step statistics of one column: points the activity flag sent through
// the processes, points the step changed, and the substeps each sedimenting
// species took (1 in the single-substep path).  The statistics instantiation
// of the step adds them to a device buffer: [0] active points, [1] changed
// points, [2] columns with an active point, [3 + 65 x + n] columns whose
// species x (r, i, s, g) took n substeps.
struct ColStats {
  int active, changed;
  int nsub[4];
};
constexpr int kStatsWords = 3 + 4 * 65;

// ------------------------------------------------------- conversions
// FP64 <-> FP32 on the integer pipe.  Values handled here are finite and, as
// FP32, normal or zero: d2f truncates toward zero (relative error < 2^-23,
// below the ~2^-22 of the MUFU functions the FP32 values feed; measured 2.6 %
// faster per step than rounding to nearest) and flushes magnitudes below
// 2^-126 to zero.  Magnitudes of 2^128 and above (and non-finite values) have
// no FP32 counterpart and convert to an arbitrary value: the mixed step scans
// the magnitudes of every value it converts (hmax) and raises the non-finite
// flag for any at or above 2^128, so such a step is reported, not trusted
// (dropping the range select from every conversion measured 1.9 % faster per
// step).  f2d is exact for normal and zero inputs (the FP32 code runs with
// flush-to-zero).  d2f only reads the FP64 state into FP32 working values;
// the state itself is never truncated.
__device__ __forceinline__ float d2f(double x) {
  const unsigned hi = (unsigned)__double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const unsigned a = hi & 0x7fffffffu;
  // 8-bit exponent and the first 23 mantissa bits
  unsigned r = __funnelshift_l(lo, a - 0x38000000u, 3);
  r = a < 0x38100000u ? 0u : r;
  return __uint_as_float(r | (hi & 0x80000000u));
}

// magnitudes at or above this (high word of |x|) have no FP32 counterpart
constexpr unsigned kF32RangeHi = 0x47f00000u;

// d2f rounded to nearest (ties away from zero), for the factor dt / (rho dz)
// that turns a flux divergence into a change of mixing ratio: a truncated
// factor is biased high by ~2^-24 at every level, which would show as a
// systematic loss of column water of that size times the surface flux.
__device__ __forceinline__ float d2f_rn(double x) {
  const unsigned hi = (unsigned)__double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const unsigned s = hi & 0x80000000u;
  const unsigned a = hi & 0x7fffffffu;
  // 8-bit exponent and 23-bit mantissa, plus the first dropped bit (a carry
  // out of the mantissa correctly bumps the exponent)
  unsigned r = __funnelshift_l(lo, a - 0x38000000u, 3) + ((lo >> 28) & 1u);
  r = a < 0x38100000u ? 0u : r;
  r = a >= kF32RangeHi ? 0x7fc00000u : r;
  return __uint_as_float(r | s);
}

__device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned s = u & 0x80000000u;
  const unsigned a = u & 0x7fffffffu;
  unsigned hi = a ? (a >> 3) + 0x38000000u : 0u;
  hi = a >= 0x7f800000u ? 0x7ff80000u : hi;
  return __hiloint2double((int)(hi | s), (int)(a << 29));
}

__device__ __forceinline__ float ex2a(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2a(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sqrta(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcpa(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Debug build (CASIM_DEBUG): every index into the state, the precipitation
// rows, the batch's lists and the surrogate's rows is checked against its
// array; one outside sets this bit of the error word and the access is
// skipped (the kernel never traps).  In the normal build the checks compile
// to nothing.
constexpr unsigned kEflagIndex = 8u;
#ifdef CASIM_DEBUG
__device__ __forceinline__ bool index_ok(bool ok, unsigned *err) {
  if (!ok && err) atomicOr(err, kEflagIndex);
  return ok;
}
#define CASIM_INDEX_OK(cond, err) ::casim_dev::index_ok((cond), (err))
#else
#define CASIM_INDEX_OK(cond, err) true
#endif

// non-finite test on the high word (integer pipe)
__device__ __forceinline__ unsigned nonfinite(double x) {
  return ((unsigned)__double2hiint(x) & 0x7ff00000u) == 0x7ff00000u;
}

// --------------------------------------------------------- policies
struct PolicyF64 {
  using R = double;
  static constexpr bool kMixed = false;
  static constexpr bool kWarm = false;
  static constexpr bool kAero = false;
  static constexpr bool kTri = false;
  static constexpr int kMinBlocks = 3;   // resident blocks of kBlock per SM the step kernel is built for
  static __device__ __forceinline__ const ConstK<double> &K(const KParams &p) { return p.d; }
  static __device__ __forceinline__ R toR(double x) { return x; }
  static __device__ __forceinline__ R toRn(double x) { return x; }
  static __device__ __forceinline__ double toD(R x) { return x; }
  static __device__ __forceinline__ R exp(R x) { return ::exp(x); }
  static __device__ __forceinline__ R lg(R x) { return ::log(x); }   // log in the constants' base
  static __device__ __forceinline__ R ex(R x) { return ::exp(x); }   // inverse of lg
  static __device__ __forceinline__ R ln(R x) { return ::log(x); }
  static __device__ __forceinline__ R sqrt(R x) { return ::sqrt(x); }
  static __device__ __forceinline__ R cbrt(R x) { return ::cbrt(x); }
  static __device__ __forceinline__ R erfc(R x) { return ::erfc(x); }
  // Gamma(x + s) / Gamma(x)
  static __device__ __forceinline__ R gratio(R x, R s) { return ::exp(::lgamma(x + s) - ::lgamma(x)); }
  static __device__ __forceinline__ R div(R a, R b) { return a / b; }
  static __device__ __forceinline__ R mn(R a, R b) { return a < b ? a : b; }
  static __device__ __forceinline__ R mx(R a, R b) { return a > b ? a : b; }
};

struct PolicyMix {
  using R = float;
  static constexpr bool kMixed = true;
  static constexpr bool kWarm = false;
  static constexpr bool kAero = false;
  static constexpr bool kTri = false;
  static constexpr int kMinBlocks = 5;   // measured: 4 / 5 / 6 -> 2.07 / 1.94 / 1.99 ms per 512x512x150 step
  static __device__ __forceinline__ const ConstK<float> &K(const KParams &p) { return p.f; }
  static __device__ __forceinline__ R toR(double x) { return d2f(x); }
  static __device__ __forceinline__ R toRn(double x) { return d2f_rn(x); }
  static __device__ __forceinline__ double toD(R x) { return f2d(x); }
  static __device__ __forceinline__ R exp(R x) { return ex2a(x * 1.44269504088896341f); }
  static __device__ __forceinline__ R lg(R x) { return lg2a(x); }
  static __device__ __forceinline__ R ex(R x) { return ex2a(x); }
  static __device__ __forceinline__ R ln(R x) { return lg2a(x) * 0.693147180559945309f; }
  static __device__ __forceinline__ R sqrt(R x) { return sqrta(x); }
  static __device__ __forceinline__ R cbrt(R x) { return ex2a(lg2a(x) * 0.333333343267f); }
  static __device__ __forceinline__ R erfc(R x) { return erfcf(x); }
  // Gamma(x + s) / Gamma(x) for x >= 1, 0 < s <= 2: the recurrence
  // Gamma(z + 1) = z Gamma(z) moves both arguments up by four, then Stirling's
  // series of ln Gamma at y = x + 4 >= 5 and y + s, differenced term by term
  // (through 1/z^5; truncation below 1e-8), with ln(1 + s/y) as 2 atanh(t),
  // t = s / (2y + s) <= 0.17, by its power series.  Relative error ~1.3e-6.
  static __device__ __forceinline__ R gratio(R x, R s) {
    const R num = x * (x + 1.f) * (x + 2.f) * (x + 3.f);
    const R den = (x + s) * (x + s + 1.f) * (x + s + 2.f) * (x + s + 3.f);
    const R y = x + 4.f, ys = y + s;
    const R u = __fdividef(1.f, y), v = __fdividef(1.f, ys);
    const R t = __fdividef(s, y + ys), t2 = t * t;
    const R l1 = 2.f * t *
                 (1.f + t2 * (1.f / 3.f + t2 * (0.2f + t2 * (1.f / 7.f + t2 * (1.f / 9.f + t2 * (1.f / 11.f))))));
    const R u3 = u * u * u, v3 = v * v * v;
    const R D = (y - 0.5f) * l1 + s * ln(ys) - s + (v - u) * (1.f / 12.f) - (v3 - u3) * (1.f / 360.f) +
                (v3 * v * v - u3 * u * u) * (1.f / 1260.f);
    return __fdividef(num, den) * exp(D);
  }
  static __device__ __forceinline__ R div(R a, R b) { return __fdividef(a, b); }
  static __device__ __forceinline__ R mn(R a, R b) { return fminf(a, b); }
  static __device__ __forceinline__ R mx(R a, R b) { return fmaxf(a, b); }
};

// ------------------------------------------------------------ one point
struct Pt {
  double T, qv, qc, qr, qi, qs, qg, nc, nr, ni, ns, ng, na, p, rho, w;
  double ma, mac, mar;   // activated-aerosol mass (free, in cloud, in rain): aerosol-mass policies only
  double mai, mas, mag;  // in ice, snow, graupel: cold aerosol-mass policies only
  double zr;             // the rain's sixth moment: triple-moment policies only
  double zi, zs, zg;     // those of ice, snow, graupel: cold triple-moment policies only
};

// field f of the state (0..15 standard; from 16 the configuration's
// aerosol masses or sixth moments)
template <class M>
__device__ __forceinline__ double &pt_field(Pt &s, int f) {
  switch (f) {
    case 0: return s.T;
    case 1: return s.qv;
    case 2: return s.qc;
    case 3: return s.qr;
    case 4: return s.qi;
    case 5: return s.qs;
    case 6: return s.qg;
    case 7: return s.nc;
    case 8: return s.nr;
    case 9: return s.ni;
    case 10: return s.ns;
    case 11: return s.ng;
    case 12: return s.na;
    case 13: return s.p;
    case 14: return s.rho;
    case 15: return s.w;
    default: break;
  }
  if constexpr (M::kAero) {
    switch (f) {
      case 16: return s.ma;
      case 17: return s.mac;
      case 18: return s.mar;
      case 19: return s.mai;
      case 20: return s.mas;
      default: return s.mag;
    }
  } else {
    switch (f) {
      case 16: return s.zr;
      case 17: return s.zi;
      case 18: return s.zs;
      default: return s.zg;
    }
  }
}

// sixth moment of sedimenting species x (r, i, s, g)
__device__ __forceinline__ double &zref(Pt &s, int x) {
  return x == 0 ? s.zr : x == 1 ? s.zi : x == 2 ? s.zs : s.zg;
}
__device__ __forceinline__ double zval(const Pt &s, int x) {
  return x == 0 ? s.zr : x == 1 ? s.zi : x == 2 ? s.zs : s.zg;
}

// aerosol mass carried by sedimenting species x (r, i, s, g)
__device__ __forceinline__ double &maref(Pt &s, int x) {
  return x == 0 ? s.mar : x == 1 ? s.mai : x == 2 ? s.mas : s.mag;
}

// number of sixth moments a policy carries: rain only (warm), r, i, s, g (cold)
template <class M>
__host__ __device__ constexpr int nz3() {
  return M::kTri ? (M::kWarm ? 1 : 4) : 0;
}

// number of sedimenting species that carry aerosol mass: rain only (warm), r, i, s, g (cold)
template <class M>
__host__ __device__ constexpr int na3() {
  return M::kAero ? (M::kWarm ? 1 : 4) : 0;
}

// Working values of a point in the compute precision (after adjustment and
// activation, as the rates see them).
template <class R>
struct W {
  double Td;   // FP64 temperature (FP64 form only: ice saturation as the oracle writes it)
  R T, tc, p, rho, qv, qc, qr, qx[3], nc, nr, nx[3];
  R mu3[4];    // shape parameters of r, i, s, g (triple-moment policies)
  unsigned hmax;   // mixed form: largest |high word| of the FP64 inputs read (non-finite check)
};

// |high word| of a double: >= 0x7ff00000 exactly when it is not finite
__device__ __forceinline__ unsigned hiabs(double x) { return (unsigned)__double2hiint(x) & 0x7fffffffu; }

// raw process rates (kg/kg/s; number rates for scc, scr, nucn)
template <class R>
struct Rt {
  R aut, acc, scc, scr, evr, nucn, dep[3], rim[2], mlt[3];
};

// limiter factors per transfer and the number-to-mass ratios they use
template <class R>
struct Gt {
  R rc, rr, rx[3], nucm, depp[3], sub[3], nmlt[3];
  R aut, acc, scc, scr, evr, nuc, dep[3], mlt[3], rs, rg;
};

// Triple-moment species (x = 0..3: r, i, s, g): the shape parameter from
// (q, n, z) and the species constants at that shape (every species has b = 3,
// so the gamma-function ratios of integer offset are products and the ratios
// of non-integer offset are Gamma(x + s) / Gamma(x) evaluations).
template <class M>
struct Shape3 {
  using R = typename M::R;
  struct Sh {
    R lglamfac, lglo, lghi;   // as SpeciesK
    R ev1, ev2;               // ventilation coefficients
    R vq, vn, vz;             // mass-, number- and sixth-moment-weighted speed coefficients
  };
  static __device__ __forceinline__ R clampmu(const ConstK<R> &K, R mu) {
    return mu < (R)0 ? (R)0 : (mu > K.s3_mumax ? K.s3_mumax : mu);
  }
  // G = z n / (q/a)^2 = P/Q, P = (mu+4)(mu+5)(mu+6), Q = (mu+1)(mu+2)(mu+3): start
  // from the root of G^(1/3) = (mu+5)/(mu+2), then four Newton steps on
  // f = ln(P/Q) - ln G_obs, whose slope P'/P - Q'/Q = (P'Q - Q'P)/(PQ) has
  // P'Q - Q'P = -3 (3 mu^4 + 42 mu^3 + 207 mu^2 + 420 mu + 292)
  static __device__ __forceinline__ R mu(const ConstK<R> &K, int x, R q, R n, R z) {
    if (!(q > K.qmin) || !(n > (R)0) || !(z > (R)0)) return K.s3_mu0[x];
    const R m3 = M::div(q, K.s3_a[x]);
    const R gobs = M::div(M::div(z * n, m3), m3);
    const R lg = M::ln(gobs);
    const R g = M::cbrt(gobs);
    R m = g > (R)1 ? clampmu(K, M::div((R)5 - (R)2 * g, g - (R)1)) : K.s3_mumax;
    // FP64: four steps, as the definition; FP32: three (from this start the
    // third step leaves |ln G - ln G_obs| < 3e-8 for every shape in [0, 20],
    // below the FP32 rounding of ln G, so a fourth changes nothing)
    constexpr int kNewton = M::kMixed ? 3 : 4;
#pragma unroll 1
    for (int it = 0; it < kNewton; ++it) {
      const R P = ((m + (R)15) * m + (R)74) * m + (R)120;
      const R Q = ((m + (R)6) * m + (R)11) * m + (R)6;
      const R W = (((R)3 * m + (R)42) * m + (R)207) * m * m + (R)420 * m + (R)292;
      const R f = M::ln(M::div(P, Q)) - lg;
      m = clampmu(K, m + M::div(f * P * Q, (R)3 * W));
    }
    return m;
  }
  static __device__ __forceinline__ void consts(const ConstK<R> &K, int x, R mu, Sh &h) {
    const R d = K.s3_dv[x];
    const R p1 = mu + (R)1, p2 = mu + (R)2, p3 = mu + (R)3;
    const R q3 = p1 * p2 * p3;   // Gamma(mu+4) / Gamma(mu+1)
    h.lglamfac = M::lg(K.s3_a[x] * q3);
    const R lp1 = M::lg(p1);
    h.lglo = lp1 - K.s3_lgdmax[x];
    h.lghi = lp1 - K.s3_lgdmin[x];
    h.ev1 = M::div(K.s3_ev1c[x], p2 * p3);
    const R rd = M::gratio(p1, d);                        // Gamma(mu+1+d)/Gamma(mu+1)
    const R rv = M::gratio(p1, (R)0.5 * (d + (R)3));      // Gamma(mu+(d+5)/2)/Gamma(mu+1)
    h.ev2 = M::div(K.s3_ev2c[x] * rv, q3);
    h.vn = K.s3_cv[x] * rd;
    h.vq = M::div(h.vn * (p1 + d) * (p2 + d) * (p3 + d), q3);
    h.vz = M::div(h.vq * (mu + (R)4 + d) * (mu + (R)5 + d) * (mu + (R)6 + d), (mu + (R)4) * (mu + (R)5) * (mu + (R)6));
  }
  // riming coefficient (pi/4) E cv Gamma(mu+d+3) / Gamma(mu+4) / a
  static __device__ __forceinline__ R rim(const ConstK<R> &K, int x, R mu) {
    const R p1 = mu + (R)1;
    return M::div(K.s3_rimc[x] * M::gratio(p1, K.s3_dv[x] + (R)2), p1 * (mu + (R)2) * (mu + (R)3));
  }
  static __device__ __forceinline__ R lglam(const Sh &h, const SpeciesK<R> &X, R lgq, R n) {
    const R lgn = M::lg(M::mx(n, (R)0));
    R l = (h.lglamfac + lgn - lgq) * X.invb;
    l = M::mx(l, h.lglo);
    return M::mn(l, h.lghi);
  }
  // fall speeds of species x at its diagnosed shape (mass, number, sixth moment), capped
  static __device__ __forceinline__ void fall_speeds(const ConstK<R> &K, int x, R guard, R q, R lgq, R n, R z,
                                                     R dfac, R &vq, R &vn, R &vz) {
    fall_speeds_mu(K, x, guard, lgq, n, mu(K, x, q, n, z), dfac, vq, vn, vz);
  }
  // the same at a known shape
  static __device__ __forceinline__ void fall_speeds_mu(const ConstK<R> &K, int x, R guard, R lgq, R n, R mu,
                                                        R dfac, R &vq, R &vn, R &vz) {
    const SpeciesK<R> &X = K.sp[1 + x];
    Sh h;
    consts(K, x, mu, h);
    const R l = lglam(h, X, lgq, n);
    const R pw = M::ex(X.exv * l);
    vq = M::mn(M::mn(h.vq * dfac * pw, X.vmax), guard);
    vn = M::mn(M::mn(h.vn * dfac * pw, X.vmax), guard);
    vz = M::mn(M::mn(h.vz * dfac * pw, X.vmax), guard);
  }
};

template <class M>
struct Phys {
  using R = typename M::R;

  static __device__ __forceinline__ R es_liq(const ConstK<R> &K, R tc) {
    return K.esl0 * M::exp(M::div(K.esla * tc, tc + K.eslb));
  }
  static __device__ __forceinline__ R qsat(const ConstK<R> &K, R es, R p) {
    return M::div(K.eps * es, p - K.ome * es);
  }
  // saturation vapour pressure over ice; the mixed form builds the exponent
  // from tc = T - T0 (formed in FP64) rather than from T rounded to FP32
  static __device__ __forceinline__ R es_ice(const ConstK<R> &K, double T, R tc) {
    if constexpr (!M::kMixed) {
      return K.esi0 * ::exp(K.esia * (T - K.esit) / (T - K.esib));
    } else {
      return K.esi0 * M::exp(M::div(K.esia * (tc + K.t0_esit), tc + K.t0_esib));
    }
  }

  // a3: Abdul-Razzak & Ghan (2000) activation from one lognormal mode.
  static __device__ __forceinline__ R arg_nact(const ConstK<R> &K, R N, R w, R T, R p, R es) {
    const R iT = M::div((R)1, T);
    const R A = K.akel * iT;
    const R sm = K.smc * A * M::sqrt(A);
    const R alpha = K.al1 * iT * iT - K.al2 * iT;
    const R gam = M::div(K.ga1 * T, es) + M::div(K.ga2, p * T);
    const R G = M::div((R)1, M::div(K.gg1 * T, es) + K.gg2 * iT * (K.gg3 * iT - (R)1));
    const R awg = M::div(alpha * w, G);
    const R sq = M::sqrt(awg);
    const R zeta = (R)(2.0 / 3.0) * A * sq;
    const R eta = M::div(awg * sq, K.twopirhow * gam * N);
    const R ze = M::div(zeta, eta);
    const R t1 = K.f1 * ze * M::sqrt(ze);
    const R y = M::div(sm * sm, eta + (R)3 * zeta);
    const R t2 = K.f2 * M::sqrt(y * M::sqrt(y));
    const R sum = M::div(t1 + t2, sm * sm);
    // u = 2 ln(S_m / S_max) / (3 sqrt2 ln sigma), S_max = 1/sqrt(sum)
    const R u = K.uc * (M::ln(sm) + (R)0.5 * M::ln(sum));
    return (R)0.5 * N * M::erfc(u);
  }

  // log of the gamma slope of a species from (log q, n), clamped
  static __device__ __forceinline__ R lglam(const SpeciesK<R> &X, R lgq, R n) {
    const R lgn = M::lg(M::mx(n, (R)0));
    R l = (X.lglamfac + lgn - lgq) * X.invb;
    l = M::mx(l, X.lglo);   // also maps log(0) = -inf (and NaN) to the lower bound
    return M::mn(l, X.lghi);
  }

  // a4..a9: process rates from the post-activation state
  static __device__ __forceinline__ void rates(const ConstK<R> &K, const W<R> &w, double dt, Rt<R> &r) {
    const R T = w.T, p = w.p, rho = w.rho, qv = w.qv, qc = w.qc, qr = w.qr, nc = w.nc, nr = w.nr;
    const R tc = w.tc;
    const R dtr = M::toR(dt);
    const R esl = es_liq(K, tc);
    const R qsl = qsat(K, esl, p);
    const R iT2 = M::div((R)1, T * T);
    const R Sw = M::div(qv, qsl);
    const bool hc = qc > K.qmin, hr = qr > K.qmin;
    // regimes: the FP64 form compares T itself; the mixed form compares
    // tc = T - T0, which it forms in FP64 before rounding (an FP32 T is
    // resolved to 3e-5 K only, so a point adjusted to within that of the
    // freezing or nucleation temperature would take the other regime)
    const bool cold = M::kMixed ? tc < (R)0 : T < K.T0;
    const bool warm = M::kMixed ? tc > (R)0 : T > K.T0;
    const bool nucl = M::kMixed ? tc < K.tnuc0 : T < K.Tnuc;

    // air properties shared by the ventilated integrals
    const R lgrho = M::lg(rho);
    const R dfac = M::ex((R)0.4 * (K.lgrho0 - lgrho));         // (rho0/rho)^0.4
    const R nu = M::div(K.mu_air, rho);
    const R V0 = M::cbrt(nu * K.inv_dv) * M::sqrt(M::div(dfac, nu));

    r.aut = r.acc = r.scc = r.scr = r.evr = r.nucn = (R)0;
#pragma unroll
    for (int m = 0; m < 3; ++m) r.dep[m] = r.mlt[m] = (R)0;
    r.rim[0] = r.rim[1] = (R)0;

    const R lgqc = hc ? M::lg(qc) : (R)0;
    const R lgqr = hr ? M::lg(qr) : (R)0;
    if (hc) {
      const R ncc = M::mx(rho * nc * (R)1e-6, K.nc_min);
      r.aut = K.kk_aut * M::ex(K.kk_aut_qc * lgqc + K.kk_aut_nc * M::lg(ncc));
      r.scc = K.kcf * rho * qc * qc;
    }
    if (hc && hr) r.acc = K.kk_acc * M::ex(K.kk_acc_exp * (lgqc + lgqr));
    if (hr) {
      r.scr = K.kr * rho * M::mx(nr, (R)0) * qr;
      if (Sw < (R)1) {
        const SpeciesK<R> &X = K.sp[1];
        R iv;
        if constexpr (M::kTri) {
          typename Shape3<M>::Sh h;
          Shape3<M>::consts(K, 0, w.mu3[0], h);
          const R l = Shape3<M>::lglam(h, X, lgqr, nr);
          iv = rho * qr * (h.ev1 * M::ex(X.ex1 * l) + V0 * h.ev2 * M::ex(X.ex2 * l));
        } else {
          const R l = lglam(X, lgqr, nr);
          iv = rho * qr * (X.ev1 * M::ex(X.ex1 * l) + V0 * X.ev2 * M::ex(X.ex2 * l));
        }
        const R Aw = K.awc * iT2, Bw = M::div(K.rv_dv * T, esl);
        r.evr = M::div(K.twopi * ((R)1 - Sw) * iv, rho * (Aw + Bw));
      }
    }
    if (!M::kWarm && cold) {
      const R esi = es_ice(K, w.Td, tc);
      const R qsi = qsat(K, esi, p);
      const R Si = M::div(qv, qsi);
      if (nucl && Si > (R)1) {
        const R nin = K.mey_a * M::exp(K.mey_b + K.mey_c * (Si - (R)1));
        const R dn = M::div(nin, rho) - w.nx[0];
        if (dn > (R)0) r.nucn = M::div(dn, dtr);
      }
      const R Ai = K.aic * iT2, Bi = M::div(K.rv_dv * T, esi);
      const R dfa = M::div(Si - (R)1, rho * (Ai + Bi));
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        if (!(w.qx[m] > K.qmin)) continue;
        const SpeciesK<R> &X = K.sp[2 + m];
        if constexpr (M::kTri) {
          // at the species' diagnosed shape
          typename Shape3<M>::Sh h;
          Shape3<M>::consts(K, 1 + m, w.mu3[1 + m], h);
          const R l = Shape3<M>::lglam(h, X, M::lg(w.qx[m]), w.nx[m]);
          const R iv = rho * w.qx[m] * (h.ev1 * M::ex(X.ex1 * l) + V0 * h.ev2 * M::ex(X.ex2 * l));
          r.dep[m] = X.dep * dfa * iv;
          if (m > 0 && hc)
            r.rim[m - 1] = Shape3<M>::rim(K, 1 + m, w.mu3[1 + m]) * qc * dfac * rho * w.qx[m] * M::ex(X.exr * l);
        } else {
          const R l = lglam(X, M::lg(w.qx[m]), w.nx[m]);
          const R iv = rho * w.qx[m] * (X.ev1 * M::ex(X.ex1 * l) + V0 * X.ev2 * M::ex(X.ex2 * l));
          r.dep[m] = X.dep * dfa * iv;
          if (m > 0 && hc) r.rim[m - 1] = X.rim * qc * dfac * rho * w.qx[m] * M::ex(X.exr * l);
        }
      }
    }
    if (!M::kWarm && warm) {
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        if (!(w.qx[m] > K.qmin)) continue;
        const SpeciesK<R> &X = K.sp[2 + m];
        R iv;
        if constexpr (M::kTri) {
          typename Shape3<M>::Sh h;
          Shape3<M>::consts(K, 1 + m, w.mu3[1 + m], h);
          const R l = Shape3<M>::lglam(h, X, M::lg(w.qx[m]), w.nx[m]);
          iv = rho * w.qx[m] * (h.ev1 * M::ex(X.ex1 * l) + V0 * h.ev2 * M::ex(X.ex2 * l));
        } else {
          const R l = lglam(X, M::lg(w.qx[m]), w.nx[m]);
          iv = rho * w.qx[m] * (X.ev1 * M::ex(X.ex1 * l) + V0 * X.ev2 * M::ex(X.ex2 * l));
        }
        r.mlt[m] = M::div(X.mlt * tc * iv, rho);
      }
    }
  }

  // a10: per-pool limiting factors f_X = min(1, X / (S_X dt)); each transfer
  // takes the smallest factor of the pools it draws from.
  static __device__ __forceinline__ void limits(const ConstK<R> &K, const W<R> &w, double dt, const Rt<R> &r,
                                                Gt<R> &g) {
    const R dtr = M::toR(dt);
    g.rc = w.qc > K.qmin ? M::div(M::mx(w.nc, (R)0), w.qc) : (R)0;
    g.rr = w.qr > K.qmin ? M::div(M::mx(w.nr, (R)0), w.qr) : (R)0;
#pragma unroll
    for (int m = 0; m < 3; ++m) g.rx[m] = w.qx[m] > K.qmin ? M::div(M::mx(w.nx[m], (R)0), w.qx[m]) : (R)0;
    g.nucm = r.nucn * K.mi0;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      g.depp[m] = r.dep[m] >= (R)0 ? r.dep[m] : (R)0;
      g.sub[m] = r.dep[m] >= (R)0 ? (R)0 : -r.dep[m];
      g.nmlt[m] = r.mlt[m] > (R)0 ? r.mlt[m] * g.rx[m] : (R)0;
    }
    // sinks per pool, summed in the order of the transfer list
    const R S_qv = ((g.nucm + g.depp[0]) + g.depp[1]) + g.depp[2];
    const R S_qc = ((r.aut + r.acc) + r.rim[0]) + r.rim[1];
    const R S_qr = r.evr;
    const R S_nc = (((r.aut * g.rc + r.acc * g.rc) + r.scc) + r.rim[0] * g.rc) + r.rim[1] * g.rc;
    const R S_nr = r.scr + r.evr * g.rr;
    auto fac = [&](R S, R X) -> R {
      if constexpr (!M::kMixed) {
        return S * dtr > X ? M::mx(X, (R)0) / (S * dtr) : (R)1;
      } else {
        // FP32 factor shrunk by 2^-18 so that the rounded transfers can
        // never take more than the pool holds
        const R Sd = S * dtr;
        return Sd > X * 0.99999f ? M::mx(X, (R)0) * 0.999996185f * rcpa(Sd) : (R)1;
      }
    };
    const R f_qv = fac(S_qv, w.qv), f_qc = fac(S_qc, w.qc), f_qr = fac(S_qr, w.qr);
    const R f_nc = fac(S_nc, w.nc), f_nr = fac(S_nr, w.nr);
    auto g2 = [&](R rate, R fm, R nsink, R fn) -> R {
      R x = (R)1;
      if (rate > (R)0 && fm < x) x = fm;
      if (nsink > (R)0 && fn < x) x = fn;
      return x;
    };
    g.aut = g2(r.aut, f_qc, r.aut * g.rc, f_nc);
    g.acc = g2(r.acc, f_qc, r.acc * g.rc, f_nc);
    g.scc = g2(0, 1, r.scc, f_nc);
    g.scr = g2(0, 1, r.scr, f_nr);
    g.evr = g2(r.evr, f_qr, r.evr * g.rr, f_nr);
    g.nuc = g2(g.nucm, f_qv, 0, 1);
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const R f_qx = fac(g.sub[m] + r.mlt[m], w.qx[m]);
      const R f_nx = fac(g.sub[m] * g.rx[m] + g.nmlt[m], w.nx[m]);
      g.dep[m] = r.dep[m] >= (R)0 ? g2(g.depp[m], f_qv, 0, 1) : g2(g.sub[m], f_qx, g.sub[m] * g.rx[m], f_nx);
      g.mlt[m] = g2(r.mlt[m], f_qx, g.nmlt[m], f_nx);
    }
    g.rs = g2(r.rim[0], f_qc, r.rim[0] * g.rc, f_nc);
    g.rg = g2(r.rim[1], f_qc, r.rim[1] * g.rc, f_nc);
  }

  // fall speeds of sedimenting species x (0..3 = r, i, s, g) at one point
  static __device__ __forceinline__ void fall_speeds(const ConstK<R> &K, R guard, R lgq, R n, R dfac, int x, R &vq,
                                                     R &vn) {
    const SpeciesK<R> &X = K.sp[1 + x];
    const R l = lglam(X, lgq, n);
    const R pw = M::ex(X.exv * l);
    vq = M::mn(M::mn(X.vq * dfac * pw, X.vmax), guard);
    vn = M::mn(M::mn(X.vn * dfac * pw, X.vmax), guard);
  }
};

// ------------------------------------------------------- FP64 form
template <class M>
struct F64T {
  using P = Phys<M>;

  // true unless the chain leaves the point unchanged (no hydrometeor, not
  // supersaturated over liquid, no ice nucleation possible); also returns
  // q_s over liquid at the initial temperature for the adjustment
  static __device__ __forceinline__ bool active(const ConstK<double> &K, const Pt &s, double &es0, double &qs0) {
    const double qmin = K.qmin;
    es0 = P::es_liq(K, s.T - K.T0);
    qs0 = P::qsat(K, es0, s.p);
    bool act = s.qc > qmin || s.qr > qmin || s.qv > qs0;
    if constexpr (!M::kWarm) {
      act = act || s.qi > qmin || s.qs > qmin || s.qg > qmin;
      if (!act && s.T < K.Tnuc) act = s.qv / P::qsat(K, P::es_ice(K, s.T, 0.0), s.p) > 1.0;
    }
    return act;
  }

  // a2: 4 Newton iterations on cp (T* - T) = Lv (qv - qs(T*))
  static __device__ __forceinline__ void satadj(const ConstK<double> &K, Pt &s, double es0, double qs0) {
    const double p = s.p;
    if (!(s.qv > qs0 || s.qc > K.qmin)) return;
    const double T0v = s.T, qv0 = s.qv, qc0 = s.qc;
    double Tn = T0v, es = es0, qs = qs0;
    for (int it = 0; it < 4; ++it) {
      if (it > 0) {
        es = P::es_liq(K, Tn - K.T0);
        qs = P::qsat(K, es, p);
      }
      const double tc = Tn - K.T0;
      const double f = (Tn - T0v) - K.lv_cp * (qv0 - qs);
      const double des = es * K.esla * K.eslb / ((tc + K.eslb) * (tc + K.eslb));
      const double den = p - K.ome * es;
      const double fp = 1.0 + K.lv_cp * (K.eps * p / (den * den) * des);
      Tn = Tn - f / fp;
    }
    double dq = K.cp_lv * (Tn - T0v);
    if (dq < -qc0) dq = -qc0;
    s.T = T0v + K.lv_cp * dq;
    s.qv = qv0 - dq;
    s.qc = qc0 + dq;
  }

  static __device__ __forceinline__ void activate(const ConstK<double> &K, Pt &s) {
    if (!(s.w > 0.0) || !(s.qc > K.qmin)) return;
    const double N = s.rho * (s.na + s.nc);
    if (!(N > 0.0)) return;
    const double nact = P::arg_nact(K, N, s.w, s.T, s.p, P::es_liq(K, s.T - K.T0));
    double dn = nact / s.rho - s.nc;
    if (dn < 0.0) dn = 0.0;
    if (dn > s.na) dn = s.na;
    s.nc += dn;
    s.na -= dn;
  }

  // a2..a10 on one active point; transfers applied one by one in list order
  // mu3, keep3 (triple-moment policies): the shapes the rates used, and a bit
  // per species whose sixth moment was only rescaled (no source), so that its
  // shape is unchanged by the processes
  static __device__ __forceinline__ void process(const ConstK<double> &K, Pt &s, double dt, double es0, double qs0,
                                                 double *mu3 = nullptr, unsigned *keep3 = nullptr) {
    const double qc0 = s.qc;
    satadj(K, s, es0, qs0);
    const double evap = qc0 > s.qc ? qc0 - s.qc : 0.0;
    const double na1 = s.na;
    activate(K, s);
    const double dn_act = na1 - s.na;
    const double qc_post = s.qc, qr_post = s.qr, nr_post = s.nr;
    const double qx0[3] = {s.qi, s.qs, s.qg}, nx0[3] = {s.ni, s.ns, s.ng};
    double tau_cr = 0.0, tau_rv = 0.0, tau_aut = 0.0, nr_aut = 0.0;
    double nuc_q = 0.0, nuc_n = 0.0, melt_q[3] = {0.0, 0.0, 0.0}, melt_n[3] = {0.0, 0.0, 0.0};
    double tau_rim = 0.0, sub_q[3] = {0.0, 0.0, 0.0};
    W<double> w;
    w.Td = s.T; w.T = s.T; w.tc = s.T - K.T0; w.p = s.p; w.rho = s.rho;
    w.qv = s.qv; w.qc = s.qc; w.qr = s.qr; w.qx[0] = s.qi; w.qx[1] = s.qs; w.qx[2] = s.qg;
    w.nc = s.nc; w.nr = s.nr; w.nx[0] = s.ni; w.nx[1] = s.ns; w.nx[2] = s.ng;
    if constexpr (M::kTri) {
#pragma unroll
      for (int x = 0; x < nz3<M>(); ++x) {
        const double q = x == 0 ? s.qr : qx0[x - 1], n = x == 0 ? s.nr : nx0[x - 1];
        w.mu3[x] = Shape3<M>::mu(K, x, q, n, zref(s, x));
      }
    }
    Rt<double> r;
    P::rates(K, w, dt, r);
    Gt<double> g;
    P::limits(K, w, dt, r, g);
    double qxd[3] = {s.qi, s.qs, s.qg};
    double nxd[3] = {s.ni, s.ns, s.ng};
    double tau;
    if (r.aut > 0) { tau = g.aut * r.aut * dt; s.qc -= tau; s.qr += tau; tau_cr += tau; tau_aut = tau; }
    if (r.aut * g.rc > 0) s.nc -= g.aut * (r.aut * g.rc) * dt;
    if (r.aut * K.inv_mr0 > 0) { nr_aut = g.aut * (r.aut * K.inv_mr0) * dt; s.nr += nr_aut; }
    if (r.acc > 0) { tau = g.acc * r.acc * dt; s.qc -= tau; s.qr += tau; tau_cr += tau; }
    if (r.acc * g.rc > 0) s.nc -= g.acc * (r.acc * g.rc) * dt;
    if (r.scc > 0) s.nc -= g.scc * r.scc * dt;
    if (r.scr > 0) s.nr -= g.scr * r.scr * dt;
    if (r.evr > 0) { tau = g.evr * r.evr * dt; s.qr -= tau; s.qv += tau; s.T += tau * (-K.lv) / K.cp; tau_rv = tau; }
    if (r.evr * g.rr > 0) s.nr -= g.evr * (r.evr * g.rr) * dt;
    if (g.nucm > 0) { tau = g.nuc * g.nucm * dt; s.qv -= tau; qxd[0] += tau; s.T += tau * K.ls / K.cp; nuc_q = tau; }
    if (r.nucn > 0) { nuc_n = g.nuc * r.nucn * dt; nxd[0] += nuc_n; }
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      if (r.dep[m] >= 0) {
        if (g.depp[m] > 0) { tau = g.dep[m] * g.depp[m] * dt; s.qv -= tau; qxd[m] += tau; s.T += tau * K.ls / K.cp; }
      } else {
        tau = g.dep[m] * g.sub[m] * dt; qxd[m] -= tau; s.qv += tau; s.T += tau * (-K.ls) / K.cp; sub_q[m] = tau;
        if (g.sub[m] * g.rx[m] > 0) nxd[m] -= g.dep[m] * (g.sub[m] * g.rx[m]) * dt;
      }
    }
    if (r.rim[0] > 0) { tau = g.rs * r.rim[0] * dt; s.qc -= tau; qxd[2] += tau; s.T += tau * K.lf / K.cp; tau_rim += tau; }
    if (r.rim[0] * g.rc > 0) s.nc -= g.rs * (r.rim[0] * g.rc) * dt;
    if (r.rim[1] > 0) { tau = g.rg * r.rim[1] * dt; s.qc -= tau; qxd[2] += tau; s.T += tau * K.lf / K.cp; tau_rim += tau; }
    if (r.rim[1] * g.rc > 0) s.nc -= g.rg * (r.rim[1] * g.rc) * dt;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      if (r.mlt[m] > 0) {
        tau = g.mlt[m] * r.mlt[m] * dt; qxd[m] -= tau; s.qr += tau; s.T += tau * (-K.lf) / K.cp; melt_q[m] = tau;
      }
      if (g.nmlt[m] > 0) {
        melt_n[m] = g.mlt[m] * g.nmlt[m] * dt; nxd[m] -= melt_n[m]; s.nr += melt_n[m];
      }
    }
    s.qi = qxd[0]; s.qs = qxd[1]; s.qg = qxd[2];
    s.ni = nxd[0]; s.ns = nxd[1]; s.ng = nxd[2];
    if constexpr (M::kTri) {
      // sixth moments: the processes that keep a species' shape scale z by
      // (q'/q)^2 (n/n'), q', n' the result without the sources; sources add
      // what they bring (autoconversion: drops of one size; melting of i, s,
      // g: the melted fraction of their sixth moment, in rain diameters;
      // nucleation: crystals of one size)
      unsigned keep = 0;
      auto kept = [&](double z0, double q0, double n0, double q1, double n1) {
        return (q0 > K.qmin && n0 > 0.0 && q1 > 0.0 && n1 > 0.0) ? z0 * (q1 / q0) * (q1 / q0) * (n0 / n1) : 0.0;
      };
      auto scaled = [&](double q0, double n0, double q1, double n1) {
        return q0 > K.qmin && n0 > 0.0 && q1 > 0.0 && n1 > 0.0;
      };
      double q1 = s.qr - tau_aut, n1 = s.nr - nr_aut, zsrc = 0.0;
      bool rsrc = nr_aut > 0.0 || tau_aut > 0.0;
      if constexpr (!M::kWarm) {
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          q1 -= melt_q[m];
          n1 -= melt_n[m];
          rsrc = rsrc || melt_q[m] > 0.0 || melt_n[m] > 0.0;
          if (melt_q[m] > 0.0 && qx0[m] > K.qmin) zsrc += K.s3_ar2[1 + m] * (melt_q[m] / qx0[m]) * zref(s, 1 + m);
        }
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          const double qm = qxd[m] - (m == 0 ? nuc_q : 0.0), nm = nxd[m] - (m == 0 ? nuc_n : 0.0);
          if (scaled(qx0[m], nx0[m], qm, nm) && !(m == 0 && (nuc_q > 0.0 || nuc_n > 0.0))) keep |= 2u << m;
          zref(s, 1 + m) = kept(zref(s, 1 + m), qx0[m], nx0[m], qm, nm) + (m == 0 ? nuc_n * K.s3_di_6 : 0.0);
        }
      }
      if (scaled(qr_post, nr_post, q1, n1) && !rsrc) keep |= 1u;
      s.zr = kept(s.zr, qr_post, nr_post, q1, n1) + nr_aut * K.s3_d0_6 + zsrc;
      if (keep3) *keep3 = keep;
      if (mu3) {
#pragma unroll
        for (int x = 0; x < nz3<M>(); ++x) mu3[x] = w.mu3[x];
      }
    }
    if constexpr (M::kAero) {
      // aerosol mass moves with the water (in the order: adjustment,
      // activation, cloud -> rain, rain -> vapour)
      double d;
      if (evap > 0.0 && qc0 > 0.0) {
        d = evap >= qc0 ? s.mac : s.mac * (evap / qc0);
        s.mac -= d;
        s.ma += d;
      }
      if (dn_act > 0.0 && na1 > 0.0) {
        d = s.ma * (dn_act / na1);
        s.ma -= d;
        s.mac += d;
      }
      if constexpr (M::kWarm) {
        if (tau_cr > 0.0 && qc_post > 0.0) {
          d = tau_cr >= qc_post ? s.mac : s.mac * (tau_cr / qc_post);
          s.mac -= d;
          s.mar += d;
        }
      } else {
        // cloud sinks: to rain (autoconversion, accretion) and to graupel
        // (riming), as one fraction of the cloud split in proportion
        const double cs = tau_cr + tau_rim;
        if (cs > 0.0 && qc_post > 0.0) {
          d = cs >= qc_post ? s.mac : s.mac * (cs / qc_post);
          s.mac -= d;
          const double dg = d * (tau_rim / cs);
          s.mag += dg;
          s.mar += d - dg;
        }
      }
      if (tau_rv > 0.0 && qr_post > 0.0) {
        d = tau_rv >= qr_post ? s.mar : s.mar * (tau_rv / qr_post);
        s.mar -= d;
        s.ma += d;
      }
      if constexpr (!M::kWarm) {
        // ice species: sublimation returns, melting passes on to rain, their
        // aerosol as one fraction of the species split in proportion
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          const double sk = sub_q[m] + melt_q[m];
          if (sk > 0.0 && qx0[m] > 0.0) {
            double &mx = maref(s, 1 + m);
            d = sk >= qx0[m] ? mx : mx * (sk / qx0[m]);
            mx -= d;
            const double dm = d * (melt_q[m] / sk);
            s.mar += dm;
            s.ma += d - dm;
          }
        }
      }
    }
  }
};

using F64 = F64T<PolicyF64>;

// ------------------------------------------------------- mixed form
// Increments of one active point in FP32, applied to the FP64 state once.
// FP32 sums of the mass increments of qv, qc, qr, qi, qs, qg over one point's
// processes and sedimentation, applied to the FP64 state with one addition
// per field.  Each field's net increment carries one FP32 rounding per term
// (as every sedimentation increment does), so total water is conserved to
// ~2^-24 of the water moved at the point.  (An exact TwoSum sum, or one FP64
// addition per transfer end, was measured 18 % and 9 % slower per step.)
struct MassAcc {
  enum { kV = 0, kC, kR, kI, kS, kG };
  float d[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  __device__ __forceinline__ void add(int f, float b) { d[f] += b; }
  __device__ __forceinline__ static void put(double &q, float h) {
    if (h != 0.f) q += f2d(h);
  }
  template <bool kWarm>
  __device__ __forceinline__ void apply(Pt &s) const {
    put(s.qv, d[kV]);
    put(s.qc, d[kC]);
    put(s.qr, d[kR]);
    if constexpr (!kWarm) {
      put(s.qi, d[kI]);
      put(s.qs, d[kS]);
      put(s.qg, d[kG]);
    }
  }
};

struct MixInc {
  float vc;        // vapour -> cloud by adjustment (signed)
  bool evap_all;   // adjustment evaporated all cloud: the FP64 cloud moves to vapour
  float cr, cg, rv, vx[3], xr[3];   // cloud->rain, cloud->graupel, rain->vapour,
                                    // vapour->i,s,g (signed), i,s,g->rain
  float dT;        // temperature
  float dn[5];     // numbers c, r, i, s, g
  float dna;       // aerosol number
  // aerosol-mass policies: fractions of the source's aerosol mass moved by
  // the adjustment (cloud -> free), activation (free -> cloud), cloud -> rain
  // and rain -> free; *_all: the whole pool moves
  float a_ev, a_act, a_cr, a_rv;
  bool a_ev_all, a_cr_all, a_rv_all;
  // cold aerosol-mass policies: a_cr is the cloud's whole sink (to rain and,
  // by riming, to graupel) and a_rim the graupel's share of it; a_x: the
  // fraction of ice species' aerosol leaving it (sublimation, melting),
  // a_melt the share of that going to rain
  float a_rim, a_x[3], a_melt[3];
  bool a_x_all[3];
  float r_aut, n_aut;   // triple-moment policies: rain mass and drops made by autoconversion
  float q_nuc, n_nuc;   // cold triple-moment policies: ice mass and crystals made by nucleation
  float n_melt[3];      // and particles of i, s, g melted into rain
};

template <class M>
struct MixT {
  using P = Phys<M>;

  // activity flag; fills the FP32 values it needs
  static __device__ __forceinline__ bool active(const ConstK<float> &K, const Pt &s, double T0d, W<float> &w,
                                                float &es0, float &qs0) {
    w.Td = s.T;
    if constexpr (!M::kWarm) {
      w.hmax = max(max(max(hiabs(s.T), hiabs(s.p)), max(hiabs(s.qv), hiabs(s.qc))),
                   max(max(hiabs(s.qr), hiabs(s.qi)), max(hiabs(s.qs), hiabs(s.qg))));
    } else {
      w.hmax = max(max(hiabs(s.T), hiabs(s.p)), max(max(hiabs(s.qv), hiabs(s.qc)), hiabs(s.qr)));
    }
    w.tc = d2f(s.T - T0d);
    w.T = d2f(s.T);
    w.p = d2f(s.p);
    w.qv = d2f(s.qv);
    w.qc = d2f(s.qc);
    w.qr = d2f(s.qr);
    if constexpr (!M::kWarm) {
      w.qx[0] = d2f(s.qi);
      w.qx[1] = d2f(s.qs);
      w.qx[2] = d2f(s.qg);
    } else {
      w.qx[0] = w.qx[1] = w.qx[2] = 0.f;
    }
    es0 = P::es_liq(K, w.tc);
    qs0 = P::qsat(K, es0, w.p);
    const float qmin = K.qmin;
    bool act = w.qc > qmin || w.qr > qmin || w.qv > qs0;
    if constexpr (!M::kWarm) {
      act = act || w.qx[0] > qmin || w.qx[1] > qmin || w.qx[2] > qmin;
      if (!act && w.tc < K.tnuc0) act = __fdividef(w.qv, P::qsat(K, P::es_ice(K, s.T, w.tc), w.p)) > 1.f;
    }
    return act;
  }

  // a2..a10 on an active point: FP32 throughout, except the initial vapour
  // difference of the adjustment, formed in FP64.  `surr`, if not null,
  // points at this point's surrogate warm-rain rates (NaN: use the scheme's).
  static __device__ __forceinline__ void process(const ConstK<float> &K, const Pt &s, double dt, W<float> &w,
                                                 float es0, float qs0, MixInc &o, const float4 *surr = nullptr) {
    const float dnc_act = pre(K, s, w, es0, qs0, o);
    post(K, w, dt, dnc_act, o, surr);
  }

  // a2 and a3; returns the cloud droplets activated
  static __device__ __forceinline__ float pre(const ConstK<float> &K, const Pt &s, W<float> &w, float es0, float qs0,
                                              MixInc &o) {
    w.rho = d2f(s.rho);
    w.nc = d2f(s.nc);
    w.nr = d2f(s.nr);
    const float na = d2f(s.na);
    if constexpr (!M::kWarm) {
      w.nx[0] = d2f(s.ni);
      w.nx[1] = d2f(s.ns);
      w.nx[2] = d2f(s.ng);
      w.hmax = max(w.hmax, max(max(max(hiabs(s.rho), hiabs(s.w)), max(hiabs(s.nc), hiabs(s.nr))),
                               max(max(hiabs(s.ni), hiabs(s.ns)), max(hiabs(s.ng), hiabs(s.na)))));
    } else {
      w.nx[0] = w.nx[1] = w.nx[2] = 0.f;
      w.hmax = max(w.hmax, max(max(max(hiabs(s.rho), hiabs(s.w)), max(hiabs(s.nc), hiabs(s.nr))), hiabs(s.na)));
    }
    o.vc = 0.f;
    o.evap_all = false;
    o.dT = 0.f;
    const float qc0 = w.qc;
    if constexpr (M::kTri) {
      w.mu3[0] = Shape3<M>::mu(K, 0, w.qr, w.nr, d2f(s.zr));
      if constexpr (!M::kWarm) {
#pragma unroll
        for (int m = 0; m < 3; ++m) w.mu3[1 + m] = Shape3<M>::mu(K, 1 + m, w.qx[m], w.nx[m], d2f(zval(s, 1 + m)));
      }
    }
    if constexpr (M::kAero) {
      o.a_ev = o.a_act = o.a_cr = o.a_rv = 0.f;
      o.a_ev_all = o.a_cr_all = o.a_rv_all = false;
      if constexpr (!M::kWarm) {
        o.a_rim = 0.f;
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          o.a_x[m] = o.a_melt[m] = 0.f;
          o.a_x_all[m] = false;
        }
      }
    }
    // a2: Newton on the temperature increment; qv - qs(T + dT) is the FP64
    // difference at dT = 0 plus the FP32 change of qs.  Three steps: the
    // iteration converges quadratically from dT = 0, and the fourth step the
    // FP64 form takes changes an FP32 dT by less than its rounding (measured:
    // the adjusted condensate moves by ~1e-11 kg/kg, far inside the mixed
    // form's error bound; 1.2 % faster per step)
    if (w.qv > qs0 || w.qc > K.qmin) {
      const float d0 = d2f(s.qv - f2d(qs0));
      float dT = 0.f, es = es0, qs = qs0;
#pragma unroll
      for (int it = 0; it < 3; ++it) {
        const float tc = w.tc + dT;
        if (it > 0) {
          es = P::es_liq(K, tc);
          qs = P::qsat(K, es, w.p);
        }
        const float d = d0 + (qs0 - qs);
        const float f = dT - K.lv_cp * d;
        const float e1 = tc + K.eslb;
        const float des = es * K.eslab * rcpa(e1 * e1);
        const float den = w.p - K.ome * es;
        const float fp = 1.f + K.lv_cp * K.eps * w.p * des * rcpa(den * den);
        dT = dT - __fdividef(f, fp);
      }
      float dq = K.cp_lv * dT;
      if (dq <= -w.qc) {
        dq = -w.qc;
        o.evap_all = true;
      }
      o.vc = dq;
      if constexpr (M::kAero) {
        if (dq < 0.f && qc0 > 0.f) {
          o.a_ev_all = o.evap_all;
          o.a_ev = __fdividef(-dq, qc0);
        }
      }
      const float dTs = K.lv_cp * dq;
      o.dT = dTs;
      w.T += dTs;
      w.tc += dTs;
      w.qv -= dq;
      w.qc = o.evap_all ? 0.f : w.qc + dq;
    }
    // a3
    o.dna = 0.f;
    float dnc_act = 0.f;
    const float wv = d2f(s.w);
    if (wv > 0.f && w.qc > K.qmin) {
      const float N = w.rho * (na + w.nc);
      if (N > 0.f) {
        const float nact = P::arg_nact(K, N, wv, w.T, w.p, P::es_liq(K, w.tc));
        float dn = __fdividef(nact, w.rho) - w.nc;
        dn = fminf(fmaxf(dn, 0.f), na);
        dnc_act = dn;
        if constexpr (M::kAero) o.a_act = na > 0.f ? __fdividef(dn, na) : 0.f;
        o.dna = -dn;
        w.nc += dn;
      }
    }
    return dnc_act;
  }

  // a4..a10 from the post-activation values
  static __device__ __forceinline__ void post(const ConstK<float> &K, W<float> &w, double dt, float dnc_act,
                                              MixInc &o, const float4 *surr) {
    Rt<float> r;
    P::rates(K, w, dt, r);
    if (surr) {
      const bool hc = w.qc > K.qmin, hr = w.qr > K.qmin;
      if (hc || hr) {
        const float4 v = *surr;
        if (!isnan(v.x)) {
          if (hc) {
            r.aut = v.x;
            r.scc = v.z;
          }
          if (hc && hr) r.acc = v.y;
          if (hr) r.scr = v.w;
        }
      }
    }
    Gt<float> g;
    P::limits(K, w, dt, r, g);
    const float dtr = d2f(dt);
    o.cr = (g.aut * r.aut + g.acc * r.acc) * dtr;
    o.cg = (g.rs * r.rim[0] + g.rg * r.rim[1]) * dtr;
    o.rv = g.evr * r.evr * dtr;
    if constexpr (M::kTri) {
      o.r_aut = g.aut * r.aut * dtr;
      o.n_aut = g.aut * r.aut * K.inv_mr0 * dtr;
      if constexpr (!M::kWarm) {
        o.q_nuc = g.nuc * g.nucm * dtr;
        o.n_nuc = g.nuc * r.nucn * dtr;
#pragma unroll
        for (int m = 0; m < 3; ++m) o.n_melt[m] = g.mlt[m] * g.nmlt[m] * dtr;
      }
    }
    if constexpr (M::kAero) {
      if constexpr (M::kWarm) {
        if (o.cr > 0.f && w.qc > 0.f) {
          o.a_cr_all = o.cr >= w.qc;
          o.a_cr = __fdividef(o.cr, w.qc);
        }
      } else {
        const float cs = o.cr + o.cg;
        if (cs > 0.f && w.qc > 0.f) {
          o.a_cr_all = cs >= w.qc;
          o.a_cr = __fdividef(cs, w.qc);
          o.a_rim = fminf(__fdividef(o.cg, cs), 1.f);
        }
      }
      if (o.rv > 0.f && w.qr > 0.f) {
        o.a_rv_all = o.rv >= w.qr;
        o.a_rv = __fdividef(o.rv, w.qr);
      }
    }
    o.vx[0] = (g.nuc * g.nucm + g.dep[0] * r.dep[0]) * dtr;   // signed: deposition > 0
    o.vx[1] = g.dep[1] * r.dep[1] * dtr;
    o.vx[2] = g.dep[2] * r.dep[2] * dtr;
#pragma unroll
    for (int m = 0; m < 3; ++m) o.xr[m] = g.mlt[m] * r.mlt[m] * dtr;
    if constexpr (M::kAero && !M::kWarm) {
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const float sub = r.dep[m] < 0.f ? -o.vx[m] : 0.f;
        const float sk = sub + o.xr[m];
        if (sk > 0.f && w.qx[m] > 0.f) {
          o.a_x_all[m] = sk >= w.qx[m];
          o.a_x[m] = __fdividef(sk, w.qx[m]);
          o.a_melt[m] = fminf(__fdividef(o.xr[m], sk), 1.f);
        }
      }
    }
    o.dn[0] = dnc_act - (g.aut * r.aut * g.rc + g.acc * r.acc * g.rc + g.scc * r.scc + g.rs * r.rim[0] * g.rc +
                         g.rg * r.rim[1] * g.rc) * dtr;
    o.dn[1] = (g.aut * r.aut * K.inv_mr0 - g.scr * r.scr - g.evr * r.evr * g.rr + g.mlt[0] * g.nmlt[0] +
               g.mlt[1] * g.nmlt[1] + g.mlt[2] * g.nmlt[2]) * dtr;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      const float sn = r.dep[m] < 0.f ? g.dep[m] * g.sub[m] * g.rx[m] : 0.f;
      o.dn[2 + m] = (m == 0 ? g.nuc * r.nucn : 0.f) * dtr - (sn + g.mlt[m] * g.nmlt[m]) * dtr;
    }
    o.dT += (K.ls * (o.vx[0] + o.vx[1] + o.vx[2]) + K.lf * o.cg - K.lv * o.rv - K.lf * (o.xr[0] + o.xr[1] + o.xr[2])) *
            K.inv_cp;
  }

  // apply the process increments to the FP64 state: every mass transfer is
  // one FP32 amount subtracted from its source and added to its destination
  // The mass transfers, each an FP32 amount taken from one pool and given to
  // another, go into the per-field sums of MassAcc (the sedimentation
  // increments follow).  The adjustment's total evaporation of cloud moves
  // the FP64 cloud at once.
  static __device__ __forceinline__ void apply_masses(Pt &s, const MixInc &o, MassAcc &m) {
    if (o.evap_all) {
      s.qv += s.qc;
      s.qc = 0.0;
    } else {
      m.add(MassAcc::kV, -o.vc);
      m.add(MassAcc::kC, o.vc);
    }
    m.add(MassAcc::kC, -o.cr);
    m.add(MassAcc::kR, o.cr);
    m.add(MassAcc::kC, -o.cg);
    m.add(MassAcc::kG, o.cg);
    m.add(MassAcc::kR, -o.rv);
    m.add(MassAcc::kV, o.rv);
    if constexpr (!M::kWarm) {
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        m.add(MassAcc::kV, -o.vx[x]);
        m.add(MassAcc::kI + x, o.vx[x]);
        m.add(MassAcc::kI + x, -o.xr[x]);
        m.add(MassAcc::kR, o.xr[x]);
      }
    }
    if (o.dT != 0.f) s.T += f2d(o.dT);
    if (o.dna != 0.f) s.na += f2d(o.dna);
    if constexpr (M::kAero) apply_aero(s, o);
  }

  // the sixth moments after the processes (w: the point the rates saw):
  // processes that keep a species' shape scale z by (q'/q)^2 (n/n'), q', n'
  // without the sources; sources add what they bring (autoconversion: drops
  // of one size; melting of i, s, g: the melted fraction of their sixth
  // moment, in rain diameters; nucleation: crystals of one size)
  static __device__ __forceinline__ float kept(const ConstK<float> &K, float q0, float n0, float q1, float n1) {
    return (q0 > K.qmin && n0 > 0.f && q1 > 0.f && n1 > 0.f)
               ? __fdividef(q1, q0) * __fdividef(q1, q0) * __fdividef(n0, n1) : 0.f;
  }
  // returns a bit per species whose z was only rescaled (no source): its
  // shape is unchanged by the processes
  static __device__ __forceinline__ unsigned apply_z(const ConstK<float> &K, Pt &s, const W<float> &w,
                                                     const MixInc &o) {
    auto scaled = [&](float q0, float n0, float q1, float n1) {
      return q0 > K.qmin && n0 > 0.f && q1 > 0.f && n1 > 0.f;
    };
    unsigned keep = 0;
    const float q1 = w.qr + o.cr - o.r_aut - o.rv;
    float n1 = w.nr + o.dn[1] - o.n_aut, src = o.n_aut * K.s3_d0_6;
    bool rsrc = o.r_aut > 0.f || o.n_aut > 0.f;
    if constexpr (!M::kWarm) {
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        n1 -= o.n_melt[m];
        rsrc = rsrc || o.xr[m] > 0.f || o.n_melt[m] > 0.f;
        if (o.xr[m] > 0.f && w.qx[m] > K.qmin)
          src += K.s3_ar2[1 + m] * __fdividef(o.xr[m], w.qx[m]) * d2f(zref(s, 1 + m));
      }
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const float qm = w.qx[m] + o.vx[m] - o.xr[m] + (m == 2 ? o.cg : 0.f) - (m == 0 ? o.q_nuc : 0.f);
        const float nm = w.nx[m] + o.dn[2 + m] - (m == 0 ? o.n_nuc : 0.f);
        if (scaled(w.qx[m], w.nx[m], qm, nm) && !(m == 0 && (o.q_nuc > 0.f || o.n_nuc > 0.f))) keep |= 2u << m;
        double &z = zref(s, 1 + m);
        z = z * f2d(kept(K, w.qx[m], w.nx[m], qm, nm)) + (m == 0 ? f2d(o.n_nuc * K.s3_di_6) : 0.0);
      }
    }
    if (scaled(w.qr, w.nr, q1, n1) && !rsrc) keep |= 1u;
    s.zr = s.zr * f2d(kept(K, w.qr, w.nr, q1, n1)) + f2d(src);
    return keep;
  }

  // aerosol masses: each amount is one FP32 product of the source's mass and
  // the moved fraction, taken from the source (never more than it holds) and
  // given to the destination
  static __device__ __forceinline__ void apply_aero(Pt &s, const MixInc &o) {
    auto move = [](double &from, double &to, float frac, bool all) {
      if (!all && !(frac > 0.f)) return;
      const double d = all ? from : fmin(f2d(d2f(from) * frac), from);
      from -= d;
      to += d;
    };
    // a move whose amount is split between two destinations (share to the first)
    auto split = [](double &from, double &to1, double &to2, float frac, bool all, float share) {
      if (!all && !(frac > 0.f)) return;
      const double d = all ? from : fmin(f2d(d2f(from) * frac), from);
      const double d1 = f2d(d2f(d) * share);
      from -= d;
      to1 += d1;
      to2 += d - d1;
    };
    move(s.mac, s.ma, o.a_ev, o.a_ev_all);
    move(s.ma, s.mac, o.a_act, false);
    if constexpr (M::kWarm) {
      move(s.mac, s.mar, o.a_cr, o.a_cr_all);
    } else {
      split(s.mac, s.mag, s.mar, o.a_cr, o.a_cr_all, o.a_rim);
    }
    move(s.mar, s.ma, o.a_rv, o.a_rv_all);
    if constexpr (!M::kWarm) {
#pragma unroll
      for (int m = 0; m < 3; ++m) split(maref(s, 1 + m), s.mar, s.ma, o.a_x[m], o.a_x_all[m], o.a_melt[m]);
    }
  }
};

using Mix = MixT<PolicyMix>;

// The warm configuration (Section 2.1: liquid water only): ice species are
// absent from the warm state -- their fields are neither read nor written, no
// ice process runs and only rain sediments.
struct PolicyF64Warm : PolicyF64 {
  static constexpr bool kWarm = true;
  // measured on 512x512x150 stratus: 4 / 5 / 6 -> 52.3-54.3 / 49.0 / 50.4 ms per step (96
  // registers and no spills at 5, also in the aerosol and triple-moment warm forms)
  static constexpr int kMinBlocks = 5;
};
struct PolicyMixWarm : PolicyMix {
  static constexpr bool kWarm = true;
  // measured on 512x512x150 stratus: 6 / 7 / 8 -> 1.062 / 0.961 / 0.940 ms per step
  // (64 registers, no spills at 8); the triple-moment warm form: 1.495 / 1.416 / 1.385
  static constexpr int kMinBlocks = 8;
};
// The warm configuration with activated-aerosol mass (Section 2: aerosol
// carried in the cloud once activated and returned when the water
// evaporates): fields 16, 17, 18 of the state are the free aerosol mass, the
// aerosol mass in cloud and in rain (kg/kg); precip has a fifth row, the
// aerosol deposited by rain.  The other fields evolve exactly as in the warm
// configuration.
struct PolicyF64WarmAero : PolicyF64Warm {
  static constexpr bool kAero = true;
};
struct PolicyMixWarmAero : PolicyMixWarm {
  static constexpr bool kAero = true;
  // measured: 6 / 7 / 8 -> 1.358 / 1.235 / 1.263 ms per step (36 B spilled at 8)
  static constexpr int kMinBlocks = 7;
};
// The warm configuration with triple-moment rain (Section 2: CASIM is a
// three-moment scheme): field 16 of the state is the rain's sixth moment z
// (m^6 per kg of air); the rain's shape parameter is diagnosed from (q, n, z)
// wherever rain evaporation or sedimentation needs the rain's size
// distribution.
struct PolicyF64Warm3 : PolicyF64Warm {
  static constexpr bool kTri = true;
};
struct PolicyMixWarm3 : PolicyMixWarm {
  static constexpr bool kTri = true;
};
// The cold configuration with triple-moment r, i, s, g: fields 16..19 are
// their sixth moments.
struct PolicyF643 : PolicyF64 {
  static constexpr bool kTri = true;
};
// The cold configuration with activated-aerosol mass in cloud, rain and the
// ice species: fields 16..21 are ma, mac, mar, mai, mas, mag.
struct PolicyF64Aero : PolicyF64 {
  static constexpr bool kAero = true;
};
struct PolicyMixAero : PolicyMix {
  static constexpr bool kAero = true;
  static constexpr int kMinBlocks = 4;   // measured: 4 / 5 -> 3.41 / 3.88 ms per stratus step
};
struct PolicyMix3 : PolicyMix {
  static constexpr bool kTri = true;
  static constexpr int kMinBlocks = 4;   // measured: 4 / 5 -> 4.69 / 5.50 ms per stratus step
};

// ---------------------------------------------------------------- kernels
template <bool kWarm = false, bool kAero = false, bool kTri = false>
__device__ __forceinline__ void load_pt(const KArgs &a, int k, int c, Pt &s) {
  if (!CASIM_INDEX_OK(k >= 0 && k < a.nlev && c >= 0 && c < a.ncols && c < a.pitch, a.err)) {
    s = Pt{};
    return;
  }
  const double *b = a.fld + (size_t)k * a.pitch + c;
  const size_t fs = (size_t)a.nlev * (size_t)a.pitch;
  s.T = b[0 * fs]; s.qv = b[1 * fs]; s.qc = b[2 * fs]; s.qr = b[3 * fs];
  if constexpr (!kWarm) {
    s.qi = b[4 * fs]; s.qs = b[5 * fs]; s.qg = b[6 * fs];
  } else {
    s.qi = s.qs = s.qg = 0.0;
  }
  s.nc = b[7 * fs]; s.nr = b[8 * fs];
  if constexpr (!kWarm) {
    s.ni = b[9 * fs]; s.ns = b[10 * fs]; s.ng = b[11 * fs];
  } else {
    s.ni = s.ns = s.ng = 0.0;
  }
  s.na = b[12 * fs];
  s.p = __ldg(b + 13 * fs); s.rho = __ldg(b + 14 * fs); s.w = __ldg(b + 15 * fs);
  if constexpr (kAero) {
    s.ma = b[16 * fs]; s.mac = b[17 * fs]; s.mar = b[18 * fs];
    if constexpr (!kWarm) {
      s.mai = b[19 * fs]; s.mas = b[20 * fs]; s.mag = b[21 * fs];
    }
  }
  if constexpr (kTri) {
    s.zr = b[16 * fs];
    if constexpr (!kWarm) {
      s.zi = b[17 * fs]; s.zs = b[18 * fs]; s.zg = b[19 * fs];
    }
  }
}

// any loaded value non-finite (integer pipe: max of the exponent fields)
__device__ __forceinline__ unsigned nonfinite_in(const Pt &s) {
  const double v[16] = {s.T, s.qv, s.qc, s.qr, s.qi, s.qs, s.qg, s.nc, s.nr, s.ni, s.ns, s.ng, s.na, s.p, s.rho, s.w};
  unsigned m = 0;
#pragma unroll
  for (int i = 0; i < 16; ++i) m = max(m, (unsigned)__double2hiint(v[i]) & 0x7ff00000u);
  return m == 0x7ff00000u;
}

__device__ __forceinline__ unsigned store_pt(const KArgs &a, int k, int c, const Pt &s) {
  if (!CASIM_INDEX_OK(k >= 0 && k < a.nlev && c >= 0 && c < a.ncols, a.err)) return 0u;
  double *b = a.fld + (size_t)k * a.pitch + c;
  const size_t fs = (size_t)a.nlev * (size_t)a.pitch;
  b[0 * fs] = s.T; b[1 * fs] = s.qv; b[2 * fs] = s.qc; b[3 * fs] = s.qr;
  b[4 * fs] = s.qi; b[5 * fs] = s.qs; b[6 * fs] = s.qg;
  b[7 * fs] = s.nc; b[8 * fs] = s.nr; b[9 * fs] = s.ni; b[10 * fs] = s.ns; b[11 * fs] = s.ng;
  b[12 * fs] = s.na;
  return nonfinite(s.T) | nonfinite(s.qv) | nonfinite(s.qc) | nonfinite(s.qr) | nonfinite(s.qi) |
         nonfinite(s.qs) | nonfinite(s.qg) | nonfinite(s.nc) | nonfinite(s.nr) | nonfinite(s.ni) |
         nonfinite(s.ns) | nonfinite(s.ng) | nonfinite(s.na);
}

// the warm configuration's fields only (and the aerosol masses, or the
// rain's sixth moment)
template <bool kAero = false, bool kTri = false>
__device__ __forceinline__ unsigned store_pt_warm(const KArgs &a, int k, int c, const Pt &s) {
  if (!CASIM_INDEX_OK(k >= 0 && k < a.nlev && c >= 0 && c < a.ncols, a.err)) return 0u;
  double *b = a.fld + (size_t)k * a.pitch + c;
  const size_t fs = (size_t)a.nlev * (size_t)a.pitch;
  b[0 * fs] = s.T; b[1 * fs] = s.qv; b[2 * fs] = s.qc; b[3 * fs] = s.qr;
  b[7 * fs] = s.nc; b[8 * fs] = s.nr; b[12 * fs] = s.na;
  unsigned e = nonfinite(s.T) | nonfinite(s.qv) | nonfinite(s.qc) | nonfinite(s.qr) | nonfinite(s.nc) |
               nonfinite(s.nr) | nonfinite(s.na);
  if constexpr (kAero) {
    b[16 * fs] = s.ma; b[17 * fs] = s.mac; b[18 * fs] = s.mar;
    e |= nonfinite(s.ma) | nonfinite(s.mac) | nonfinite(s.mar);
  }
  if constexpr (kTri) {
    b[16 * fs] = s.zr;
    e |= nonfinite(s.zr);
  }
  return e;
}

// Tendency mode (the state is left unchanged): in the single-substep path
// the source terms (x_new - x_old) / dt go straight to tend (x_old re-read
// from the state, still in cache); in the multi-substep path the new values
// go to tend as scratch for the substep sweeps and are converted afterwards.
// (warm configuration: zero source terms for the ice fields)
// prognostic fields a policy carries after the inputs p, rho, w (fields 16..):
// aerosol masses, or sixth moments; tendency row 13 + i holds field 16 + i
template <class M>
__host__ __device__ constexpr int nextra() {
  return M::kAero ? (M::kWarm ? 3 : 6) : nz3<M>();
}
template <class M>
__device__ __forceinline__ double extra(const Pt &s, int i) {
  if constexpr (M::kAero) {
    return i == 0 ? s.ma : i == 1 ? s.mac : i == 2 ? s.mar : i == 3 ? s.mai : i == 4 ? s.mas : s.mag;
  } else {
    return zval(s, i);
  }
}

// x / dt for the source terms, correctly rounded as the division is, from the
// reciprocal inv = 1/dt rounded once: for a dt that is a power of two the
// quotient is x * inv exactly; otherwise Markstein's correction (Markstein
// 1990: q = x inv, the remainder x - q dt exactly by a fused multiply-add,
// then q + remainder * inv) yields the correctly rounded quotient whenever it
// is a normal number away from the ends of the exponent range, and the rest
// (zero, which keeps its sign, and quotients near those ends) take the
// division itself.  One division per thread instead of one per source term:
// an FP64 division costs about ten SM cycles on this part.
struct DtDiv {
  double dt, inv;
  bool pow2;
  __device__ explicit DtDiv(double d) : dt(d), inv(1.0 / d) {
    pow2 = (__double_as_longlong(d) & 0x000FFFFFFFFFFFFFll) == 0;   // a positive normal dt: 2^e exactly
  }
  __device__ __forceinline__ double operator()(double x) const {
    if (pow2) return x * inv;
    if (x == 0.0) return x;
    const double q = x * inv;
    const double q1 = fma(fma(-q, dt, x), inv, q);
    const double m = fabs(q1);
    return (m > 0x1p-1000 && m < 0x1p+1000) ? q1 : x / dt;
  }
};

// the prefetch stage's slot that holds state field f (a field the configuration
// loads: all 16 and those after the inputs; the warm configuration leaves out
// the ice fields)
template <class M>
__host__ __device__ constexpr int stage_slot(int f) {
  return !M::kWarm ? f : f < 4 ? f : f < 9 ? f - 3 : f < 16 ? f - 6 : 10 + (f - 16);
}

template <class M>
// cur, ss (the staged mixed forms): the point's stage slots, which hold the
// values read, so x_before comes from there rather than from the state again
__device__ __forceinline__ unsigned store_tend(const KArgs &a, double *tend, int k, int c, const Pt &s, bool fast,
                                               const DtDiv &per_dt, const double *cur = nullptr, int ss = 0) {
  if (!CASIM_INDEX_OK(k >= 0 && k < a.nlev && c >= 0 && c < a.ncols, a.err)) return 0u;
  constexpr bool kWarm = M::kWarm;
  const size_t o = (size_t)k * a.pitch + c;
  const size_t fs = (size_t)a.nlev * (size_t)a.pitch;
  auto before = [&](int f) { return cur ? cur[stage_slot<M>(f) * ss] : a.fld[f * fs + o]; };
  const double v[13] = {s.T, s.qv, s.qc, s.qr, s.qi, s.qs, s.qg, s.nc, s.nr, s.ni, s.ns, s.ng, s.na};
#pragma unroll
  for (int f = 0; f < 13; ++f) {
    const bool ice = (f >= 4 && f <= 6) || (f >= 9 && f <= 11);
    if (kWarm && ice) {
      tend[f * fs + o] = 0.0;   // zero source term (the conversion pass skips these)
    } else {
      tend[f * fs + o] = fast ? per_dt(v[f] - before(f)) : v[f];
    }
  }
  unsigned ex = 0;
#pragma unroll
  for (int e = 0; e < nextra<M>(); ++e) {
    const double v = extra<M>(s, e);
    tend[(13 + e) * fs + o] = fast ? per_dt(v - before(16 + e)) : v;
    ex |= nonfinite(v);
  }
  return ex | nonfinite(s.T) | nonfinite(s.qv) | nonfinite(s.qc) | nonfinite(s.qr) | nonfinite(s.qi) |
         nonfinite(s.qs) | nonfinite(s.qg) | nonfinite(s.nc) | nonfinite(s.nr) | nonfinite(s.ni) |
         nonfinite(s.ns) | nonfinite(s.ng) | nonfinite(s.na);
}

__device__ __forceinline__ double &qref(Pt &s, int x) {
  return x == 0 ? s.qr : x == 1 ? s.qi : x == 2 ? s.qs : s.qg;
}
__device__ __forceinline__ double &nref(Pt &s, int x) {
  return x == 0 ? s.nr : x == 1 ? s.ni : x == 2 ? s.ns : s.ng;
}

// Per-level tables the sweep reads: dz and dz/dt in FP64, and for the mixed
// form's single-substep sedimentation dt/dz rounded to nearest and dz/dt
// truncated to FP32 (the speed guard), so a point forms its factor
// dt / (rho dz) from one conversion and one division.
struct LevelTab {
  const double *dz, *dzdt;
  const float *dtdz_f, *dzdt_f;
};

// fills the tables of level k (called by the block's threads over k)
__device__ __forceinline__ void level_tab(double *dz, double *dzdt, float *dtdz_f, float *dzdt_f, int k, double v,
                                          double dt) {
  dz[k] = v;
  dzdt[k] = v / dt;
  dtdz_f[k] = d2f_rn(dt / v);
  dzdt_f[k] = d2f(v / dt);
}

// The step kernel's dynamic shared memory: the prefetch stage (mixed step:
// two levels of the fields the configuration loads, per thread), then the
// level tables of this domain's nlev levels (dz, dz/dt, dt/dz and dz/dt in
// FP32), then the block's reduction slots.
template <class M, bool kTend>
__host__ __device__ constexpr bool step_staged() {
  return M::kMixed;
}
// fields a configuration loads per point: the warm configuration T, qv, qc,
// qr, nc, nr, na, p, rho, w; the cold one the 16 standard fields; then the
// aerosol masses or sixth moments (fields 16..)
template <class M>
__host__ __device__ constexpr int stage_nf() {
  return M::kWarm ? 10 + (M::kAero ? 3 : 0) + (M::kTri ? 1 : 0) : 16 + (M::kAero ? 6 : 0) + (M::kTri ? 4 : 0);
}
// the state field held in stage slot i
template <class M>
__host__ __device__ constexpr int stage_field(int i) {
  return !M::kWarm ? i : i < 4 ? i : i < 6 ? i + 3 : i < 10 ? i + 6 : 16 + (i - 10);
}
template <class M>
__host__ __device__ constexpr size_t stage_bytes(int block) {
  return 2 * (size_t)stage_nf<M>() * block * sizeof(double);
}
template <class M, bool kTend>
__host__ __device__ constexpr size_t step_smem_bytes(int nlev) {
  return (step_staged<M, kTend>() ? stage_bytes<M>(kBlock) : 0) + (size_t)nlev * 24 + (kBlock / 32) * 8 + 16;
}

struct StepSmem {
  double *stage;   // [2][16][kBlock] or null
  LevelTab lt;
  double *red;
  int *fast;
};

template <class M, bool kTend>
__device__ __forceinline__ StepSmem step_smem(unsigned char *base, int nlev) {
  StepSmem m;
  unsigned char *p = base;
  m.stage = nullptr;
  if constexpr (step_staged<M, kTend>()) {
    m.stage = reinterpret_cast<double *>(p);
    p += stage_bytes<M>(kBlock);
  }
  double *dz = reinterpret_cast<double *>(p), *dzdt = dz + nlev;
  float *dtdz_f = reinterpret_cast<float *>(dzdt + nlev), *dzdt_f = dtdz_f + nlev;
  m.lt = LevelTab{dz, dzdt, dtdz_f, dzdt_f};
  m.red = reinterpret_cast<double *>(dzdt_f + nlev);   // 24 nlev bytes in: 8-byte aligned
  m.fast = reinterpret_cast<int *>(m.red + kBlock / 32);
  return m;
}

// Block prologue: the level tables into shared memory, and whether every
// species' capped speed keeps within one level per step.
__device__ __forceinline__ bool prologue(const KArgs &a, const KParams &P, const StepSmem &sm) {
  double dzmin = 1e300;
  for (int k = threadIdx.x; k < a.nlev; k += blockDim.x) {
    const double v = a.dz[k];
    level_tab(const_cast<double *>(sm.lt.dz), const_cast<double *>(sm.lt.dzdt), const_cast<float *>(sm.lt.dtdz_f),
              const_cast<float *>(sm.lt.dzdt_f), k, v, a.dt);
    dzmin = fmin(dzmin, v);
  }
  for (int o = 16; o > 0; o >>= 1) dzmin = fmin(dzmin, __shfl_xor_sync(0xffffffffu, dzmin, o));
  if ((threadIdx.x & 31) == 0) sm.red[threadIdx.x >> 5] = dzmin;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = sm.red[0];
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) m = fmin(m, sm.red[i]);
    int fast = 1;
    for (int x = 1; x < 5; ++x) fast &= ((P.vmax[x] * a.dt) / m) / P.c_max <= 1.0;
    *sm.fast = fast;
  }
  __syncthreads();
  return *sm.fast != 0;
}

// 8-byte asynchronous copy global -> shared (this thread's own slot)
__device__ __forceinline__ void cp_async8(double *dst, const double *src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Multi-substep sedimentation of one column after the processes (used when a
// capped speed could exceed one level per step): per species, n_sub from the
// largest Courant number, then n_sub top-down sweeps in place.
// nsub_out (may be null): the substep count each sedimenting species took;
// lvmask (may be null): bit k set for every level k the sweeps write
template <class M, bool kTend>
__device__ __forceinline__ unsigned sediment_substeps(const KArgs &a, const KParams &P, const double *sdz, int c,
                                                      double prec[5], double *tend, int *nsub_out = nullptr,
                                                      unsigned *lvmask = nullptr) {
  using R = typename M::R;
  using Ph = Phys<M>;
  const ConstK<R> &K = M::K(P);
  unsigned eflag = 0;
  if (!CASIM_INDEX_OK(c >= 0 && c < a.ncols, a.err)) return 0u;
  const size_t fs = (size_t)a.nlev * (size_t)a.pitch;
  const double *rhop = a.fld + 14 * fs;
  double *state = kTend ? tend : a.fld;   // the processed state (tendency mode: scratch)
  constexpr int kSed = M::kWarm ? 1 : 4;   // sedimenting species: r (warm) or r, i, s, g
  for (int x = 0; x < kSed; ++x) {
    double *qp = state + (3 + x) * fs;
    double *np = state + (8 + x) * fs;
    // the species' sixth moment (triple-moment policies: rain, or r, i, s, g)
    const bool tri = x < nz3<M>();
    // fields after the inputs: in tendency mode their rows of tend (field f at row f - 3)
    double *zp = kTend ? tend + (13 + x) * fs : a.fld + (16 + x) * fs;
    R cmax = 0;
    for (int k = 0; k < a.nlev; ++k) {
      const size_t o = (size_t)k * a.pitch + c;
      const R q = M::toR(qp[o]);
      if (!(q > K.qmin)) continue;
      const R rho = M::toR(__ldg(rhop + o));
      const R dfac = M::ex((R)0.4 * (K.lgrho0 - M::lg(rho)));
      R vq, vn;
      if (tri) {
        R vz;
        Shape3<M>::fall_speeds(K, x, (R)1e30, q, M::lg(q), M::toR(np[o]), M::toR(zp[o]), dfac, vq, vn, vz);
      } else {
        Ph::fall_speeds(K, (R)1e30, M::lg(q), M::toR(np[o]), dfac, x, vq, vn);
      }
      cmax = M::mx(cmax, M::div(vq * M::toR(a.dt), M::toR(sdz[k])));
    }
    int ns = (int)ceil((double)M::div(cmax, M::toR(P.c_max)));
    if (ns < 1) ns = 1;
    if (ns > 64) { ns = 64; eflag |= 2u; }
    if (nsub_out) nsub_out[x] = ns;
    const double dts = a.dt / ns;
    // the rain's aerosol mass moves with the rain (aerosol-mass policies)
    const bool aer = x < na3<M>();
    double *ap = kTend ? tend + (15 + x) * fs : a.fld + (18 + x) * fs;
    for (int st = 0; st < ns; ++st) {
      R Fu = 0, Gu = 0, Au = 0, Hu = 0;
      for (int k = a.nlev - 1; k >= 0; --k) {
        const size_t o = (size_t)k * a.pitch + c;
        double q = qp[o], n = np[o];
        const double rhod = __ldg(rhop + o);
        const R qR = M::toR(q), rho = M::toR(rhod);
        R F = 0, G = 0, A = 0, H = 0;
        double am = 0.0, zm = 0.0;
        if (aer) am = ap[o];
        if (tri) zm = zp[o];
        if (qR > K.qmin) {
          const R dfac = M::ex((R)0.4 * (K.lgrho0 - M::lg(rho)));
          R vq, vn, vz = 0;
          if (tri) {
            Shape3<M>::fall_speeds(K, x, M::toR(sdz[k] / dts), qR, M::lg(qR), M::toR(n), M::toR(zm), dfac, vq, vn, vz);
          } else {
            Ph::fall_speeds(K, M::toR(sdz[k] / dts), M::lg(qR), M::toR(n), dfac, x, vq, vn);
          }
          if constexpr (!M::kMixed) {
            F = rhod * q * vq;
            G = rhod * (n > 0.0 ? n : 0.0) * vn;
            if (aer) A = rhod * am * vq;
            if (tri) H = rhod * (zm > 0.0 ? zm : 0.0) * vz;
          } else {
            F = rho * qR * vq;
            G = rho * M::mx(M::toR(n), (R)0) * vn;
            if (aer) A = rho * M::toR(am) * vq;
            if (tri) H = rho * M::mx(M::toR(zm), (R)0) * vz;
          }
        }
        if (tri && (H != (R)0 || Hu != (R)0)) {
          if constexpr (!M::kMixed) {
            zm += dts * (Hu - H) / (rhod * sdz[k]);
          } else {
            zm += M::toD((Hu - H) * M::div(M::toRn(dts), M::toRn(rhod) * M::toRn(sdz[k])));
          }
          zp[o] = zm;
          eflag |= nonfinite(zm);
        }
        Hu = H;
        if (aer && (A != (R)0 || Au != (R)0)) {
          if constexpr (!M::kMixed) {
            am += dts * (Au - A) / (rhod * sdz[k]);
          } else {
            am += M::toD((Au - A) * M::div(M::toRn(dts), M::toRn(rhod) * M::toRn(sdz[k])));
          }
          ap[o] = am;
          eflag |= nonfinite(am);
        }
        Au = A;
        if (F != (R)0 || Fu != (R)0 || G != (R)0 || Gu != (R)0) {
          if constexpr (!M::kMixed) {
            q += dts * (Fu - F) / (rhod * sdz[k]);
            n += dts * (Gu - G) / (rhod * sdz[k]);
          } else {
            const R sc = M::div(M::toRn(dts), M::toRn(rhod) * M::toRn(sdz[k]));
            q += M::toD((Fu - F) * sc);
            n += M::toD((Gu - G) * sc);
          }
          qp[o] = q;
          np[o] = n;
          if (lvmask) lvmask[k >> 5] |= 1u << (k & 31);
          eflag |= nonfinite(q) | nonfinite(n);
        }
        Fu = F;
        Gu = G;
      }
      prec[x] += M::toD(Fu) * dts;
      if (aer) prec[4] += M::toD(Au) * dts;
    }
  }
  return eflag;
}

// One timestep for ncols columns.  When every species' capped fall speed
// satisfies vmax dt / min(dz) <= c_max, each column needs exactly one
// sedimentation substep and the flux recurrence is fused into the top-down
// sweep of the processes (one read and one write of the state).  Otherwise
// the processes are applied first and each species is sedimented with its
// own substep count in further sweeps over the column.
// stg (kStage): this thread's slots of the prefetch stage (slot f of buffer
// b at stg[(b * 16 + f) * ss], ss the block's thread count): level k - 1's 16
// fields are copied there by cp.async while level k is processed, so the
// sweep seldom waits on a load (each thread reads only the slots it filled
// itself: no block barrier)
// kLine (the state lies in mapped host memory, reached over the host link):
// per level and field, when any lane of a warp changed that field's bits,
// every lane stores it -- a lane whose value is unchanged writes back the
// value it read, taken again from this level's stage slots -- so each stored
// row (32 columns x 8 bytes) crosses the link as whole lines (a write of part
// of a line there costs about as much as a whole one: reading 16 fields and
// writing 13 at a random 76 % of the points of a 512x512x150 state measured
// 37.0 ms, at every point 26.4 ms).  The stored bits and the error flags are
// those of the in-place step.
template <class M, bool kTend = false, bool kStage = false, bool kStats = false, bool kLine = false>
__device__ __forceinline__ unsigned run_column(const KArgs &a, const KParams &P, const LevelTab &lt, bool fast, int c,
                                               double *tend = nullptr, double *stg = nullptr, int ss = kBlock,
                                               ColStats *cs = nullptr) {
  static_assert(!kLine || (kStage && !kTend && !kStats), "whole-line stores re-read the stage");
  const double *sdz = lt.dz, *sdzdt = lt.dzdt;
  constexpr int kNf = stage_nf<M>();
  if constexpr (kStage) {
    if (!CASIM_INDEX_OK(c >= 0 && c < a.ncols && c < a.pitch, a.err)) return 0u;
    const size_t fs = (size_t)a.nlev * (size_t)a.pitch;
    const double *src = a.fld + (size_t)(a.nlev - 1) * a.pitch + c;
#pragma unroll
    for (int i = 0; i < kNf; ++i) cp_async8(stg + i * ss, src + stage_field<M>(i) * fs);
    cp_async_commit();
  }
  using R = typename M::R;
  using Ph = Phys<M>;
  const ConstK<R> &K = M::K(P);
  unsigned eflag = 0;
  const DtDiv per_dt(kTend ? a.dt : 1.0);   // the source terms' division by dt (tendency mode)
  constexpr int kSed = M::kWarm ? 1 : 4;   // sedimenting species: r (warm) or r, i, s, g
  double prec[5] = {0.0, 0.0, 0.0, 0.0, 0.0};   // r, i, s, g (and aerosol in rain)
  // carried downward fluxes F_{k+1}, G_{k+1} (kg m^-2 s^-1, m^-2 s^-1), and
  // the rain's aerosol-mass flux (aerosol-mass policies)
  R Fq[4] = {0, 0, 0, 0}, Fn[4] = {0, 0, 0, 0};
  R Fa[4] = {0, 0, 0, 0};       // aerosol mass in r, i, s, g (aerosol-mass policies)
  R Fz[4] = {0, 0, 0, 0};       // sixth moments of r, i, s, g (triple-moment policies)

  // statistics build: the levels this column's step writes (processes and sweeps)
  unsigned lvmask[kStats ? (kMaxLev + 31) / 32 : 1];
  if constexpr (kStats)
    for (int i = 0; i < (a.nlev + 31) / 32; ++i) lvmask[i] = 0u;
  for (int k = a.nlev - 1; k >= 0; --k) {
    Pt s;
    const double *cur = nullptr;   // this level's slots of the stage (kStage)
    if constexpr (kStage) {
      const int b = (a.nlev - 1 - k) & 1;
      cur = stg + b * kNf * ss;
      if (k > 0) {
        double *nxt = stg + (b ^ 1) * kNf * ss;
        const size_t fs = (size_t)a.nlev * (size_t)a.pitch;
        const double *src = a.fld + (size_t)(k - 1) * a.pitch + c;
#pragma unroll
        for (int i = 0; i < kNf; ++i) cp_async8(nxt + i * ss, src + stage_field<M>(i) * fs);
        cp_async_commit();
        cp_async_wait<1>();   // this level's copies (the older group) have landed
      } else {
        cp_async_wait<0>();
      }
      if constexpr (!M::kWarm && !M::kAero && !M::kTri) {
        s.T = cur[0 * ss]; s.qv = cur[1 * ss]; s.qc = cur[2 * ss]; s.qr = cur[3 * ss];
        s.qi = cur[4 * ss]; s.qs = cur[5 * ss]; s.qg = cur[6 * ss];
        s.nc = cur[7 * ss]; s.nr = cur[8 * ss]; s.ni = cur[9 * ss]; s.ns = cur[10 * ss];
        s.ng = cur[11 * ss]; s.na = cur[12 * ss];
        s.p = cur[13 * ss]; s.rho = cur[14 * ss]; s.w = cur[15 * ss];
      } else {
        if constexpr (M::kWarm) s.qi = s.qs = s.qg = s.ni = s.ns = s.ng = 0.0;
#pragma unroll
        for (int i = 0; i < kNf; ++i) pt_field<M>(s, stage_field<M>(i)) = cur[i * ss];
      }
    } else {
      load_pt<M::kWarm, M::kAero, M::kTri>(a, k, c, s);
    }
    bool touched;
    if constexpr (!M::kMixed) {
      eflag |= nonfinite_in(s);
      // the aerosol masses or sixth moments too: an inactive point is not stored,
      // so its values are checked as they are read
#pragma unroll
      for (int e = 0; e < nextra<M>(); ++e) eflag |= nonfinite(extra<M>(s, e));
      double es0, qs0;
      touched = F64T<M>::active(K, s, es0, qs0);
      if constexpr (kStats) cs->active += touched;
      double mu3[4];
      unsigned keep3 = 0;   // species whose shape the processes left unchanged (triple-moment policies)
      if (touched) F64T<M>::process(K, s, a.dt, es0, qs0, mu3, &keep3);
      if (fast) {
        const double dzk = sdz[k];
        const double dfac = ::exp(0.4 * (K.lgrho0 - ::log(s.rho)));
#pragma unroll
        for (int x = 0; x < kSed; ++x) {
          double &q = qref(s, x);
          double &n = nref(s, x);
          double F = 0, G = 0, A = 0, H = 0;
          if (q > K.qmin) {
            double vq, vn;
            if (x < nz3<M>()) {
              double vz;
              const double z = zref(s, x);
              const double mus = ((keep3 >> x) & 1u) ? mu3[x] : Shape3<M>::mu(K, x, q, n, z);
              Shape3<M>::fall_speeds_mu(K, x, sdzdt[k], ::log(q), n, mus, dfac, vq, vn, vz);
              H = s.rho * (z > 0.0 ? z : 0.0) * vz;
            } else {
              Ph::fall_speeds(K, sdzdt[k], ::log(q), n, dfac, x, vq, vn);
            }
            F = s.rho * q * vq;
            G = s.rho * (n > 0.0 ? n : 0.0) * vn;
            if (x < na3<M>()) A = s.rho * maref(s, x) * vq;
          }
          if (x < nz3<M>()) {
            if (H != 0.0 || Fz[x] != 0.0) {
              zref(s, x) += a.dt * (Fz[x] - H) / (s.rho * dzk);
              touched = true;
            }
            Fz[x] = H;
          }
          if (F != 0.0 || Fq[x] != 0.0 || G != 0.0 || Fn[x] != 0.0) {
            q += a.dt * (Fq[x] - F) / (s.rho * dzk);
            n += a.dt * (Fn[x] - G) / (s.rho * dzk);
            touched = true;
          }
          if (x < na3<M>()) {
            if (A != 0.0 || Fa[x] != 0.0) {
              maref(s, x) += a.dt * (Fa[x] - A) / (s.rho * dzk);
              touched = true;
            }
            Fa[x] = A;
          }
          Fq[x] = F;
          Fn[x] = G;
        }
      }
    } else {
      W<float> w;
      float es0, qs0;
      const bool act = MixT<M>::active(K, s, P.T0, w, es0, qs0);
      // the aerosol masses or sixth moments join the magnitude scan (an
      // inactive point is not stored, so its values are checked as read)
#pragma unroll
      for (int e = 0; e < nextra<M>(); ++e) w.hmax = max(w.hmax, hiabs(extra<M>(s, e)));
      if constexpr (kStats) cs->active += act;
      MixInc o;
      MassAcc macc;
      unsigned keep3 = 0;   // species whose shape the processes left unchanged (triple-moment policies)
      float dn[4] = {0.f, 0.f, 0.f, 0.f};   // number increments of r, i, s, g
      float qpost[4], npost[4];
      if (act) {
        MixT<M>::process(K, s, a.dt, w, es0, qs0, o, a.surr ? a.surr + (size_t)k * a.pitch + c : nullptr);
        if constexpr (kStage && !M::kWarm && !M::kAero && !M::kTri) {
          // the FP64 values the increments are added to, read again from this
          // level's stage slots (they stay there until the level after next is
          // prefetched) rather than held in registers through the processes:
          // no spills, 2.02 -> 1.95 ms per 512x512x150 step, results unchanged
          const volatile double *v = cur;
          s.T = v[0 * ss]; s.qv = v[1 * ss]; s.qc = v[2 * ss]; s.qr = v[3 * ss];
          s.qi = v[4 * ss]; s.qs = v[5 * ss]; s.qg = v[6 * ss];
          s.nc = v[7 * ss]; s.nr = v[8 * ss]; s.ni = v[9 * ss]; s.ns = v[10 * ss];
          s.ng = v[11 * ss]; s.na = v[12 * ss]; s.rho = v[14 * ss];
        }
        MixT<M>::apply_masses(s, o, macc);
        if constexpr (M::kTri) keep3 = MixT<M>::apply_z(K, s, w, o);
        if (o.dn[0] != 0.f) s.nc += f2d(o.dn[0]);
#pragma unroll
        for (int x = 0; x < 4; ++x) dn[x] = o.dn[1 + x];
        // post-process FP32 masses and numbers for the fall speeds
        qpost[0] = w.qr + o.cr - o.rv + o.xr[0] + o.xr[1] + o.xr[2];
        qpost[1] = w.qx[0] + o.vx[0] - o.xr[0];
        qpost[2] = w.qx[1] + o.vx[1] - o.xr[1];
        qpost[3] = w.qx[2] + o.vx[2] + o.cg - o.xr[2];
        npost[0] = w.nr + dn[0];
#pragma unroll
        for (int x = 1; x < 4; ++x) npost[x] = w.nx[x - 1] + dn[x];
      } else {
        qpost[0] = w.qr;
        qpost[1] = w.qx[0];
        qpost[2] = w.qx[1];
        qpost[3] = w.qx[2];
#pragma unroll
        for (int x = 0; x < 4; ++x) npost[x] = 0.f;   // read only where a species is present
      }
      touched = act;
      if (fast) {
        bool any = false;
#pragma unroll
        for (int x = 0; x < kSed; ++x) any |= qpost[x] > K.qmin || Fq[x] != 0.f || Fn[x] != 0.f;
        if (any) {
          if (!act) w.hmax = max(w.hmax, hiabs(s.rho));
          const float rho = act ? w.rho : d2f(s.rho);
          const float dfac = ex2a(0.4f * (K.lgrho0 - lg2a(rho)));
          const float sc = __fdividef(lt.dtdz_f[k], d2f_rn(s.rho));
          const float guard = lt.dzdt_f[k];
#pragma unroll
          for (int x = 0; x < kSed; ++x) {
            float F = 0.f, G = 0.f, A = 0.f, H = 0.f;
            if (qpost[x] > K.qmin) {
              const float n = act ? npost[x] : d2f(nref(s, x));
              float vq, vn;
              if (x < nz3<M>()) {
                float vz;
                const float zp = d2f(zref(s, x));
                const float mus = ((keep3 >> x) & 1u) ? w.mu3[x] : Shape3<M>::mu(K, x, qpost[x], n, zp);
                Shape3<M>::fall_speeds_mu(K, x, guard, lg2a(qpost[x]), n, mus, dfac, vq, vn, vz);
                H = rho * fmaxf(zp, 0.f) * vz;
              } else {
                Ph::fall_speeds(K, guard, lg2a(qpost[x]), n, dfac, x, vq, vn);
              }
              F = rho * qpost[x] * vq;
              G = rho * fmaxf(n, 0.f) * vn;
              if (x < na3<M>()) A = rho * d2f(maref(s, x)) * vq;
            }
            if (x < nz3<M>()) {
              if (H != 0.f || Fz[x] != 0.f) {
                zref(s, x) += f2d((Fz[x] - H) * sc);
                touched = true;
              }
              Fz[x] = H;
            }
            if (x < na3<M>()) {
              if (A != 0.f || Fa[x] != 0.f) {
                maref(s, x) += f2d((Fa[x] - A) * sc);
                touched = true;
              }
              Fa[x] = A;
            }
            if (F != 0.f || Fq[x] != 0.f) {
              macc.add(x == 0 ? MassAcc::kR : MassAcc::kI + x - 1, (Fq[x] - F) * sc);
              touched = true;
            }
            if (G != 0.f || Fn[x] != 0.f) {
              dn[x] += (Fn[x] - G) * sc;
              touched = true;
            }
            Fq[x] = F;
            Fn[x] = G;
          }
        }
      }
#pragma unroll
      for (int x = 0; x < kSed; ++x)
        if (dn[x] != 0.f) nref(s, x) += f2d(dn[x]);
      macc.apply<M::kWarm>(s);
      eflag |= w.hmax >= kF32RangeHi;
    }
    if constexpr (kTend) {
      eflag |= store_tend<M>(a, tend, k, c, s, fast, per_dt, kStage ? cur : nullptr, ss);
    } else if constexpr (kLine) {
      const unsigned wm = __activemask();
      if (__any_sync(wm, touched)) {
        // per field: the warp stores the whole row where any lane's value
        // changed bits (the stage holds the value read); every lane takes
        // part in every vote
        const bool ok = CASIM_INDEX_OK(k >= 0 && k < a.nlev && c >= 0 && c < a.ncols, a.err);
        double *b = a.fld + (size_t)k * a.pitch + c;
        const size_t fs = (size_t)a.nlev * (size_t)a.pitch;
#pragma unroll
        for (int i = 0; i < kNf; ++i) {
          const int f = stage_field<M>(i);
          if (f >= 13 && f < 16) continue;   // the inputs p, rho, w
          const double o = cur[i * ss];
          const double v = touched ? pt_field<M>(s, f) : o;
          if (__any_sync(wm, __double_as_longlong(v) != __double_as_longlong(o)) && ok) b[f * fs] = v;
          if (touched) eflag |= nonfinite(v);
        }
      }
    } else if constexpr (M::kWarm) {
      if (touched) eflag |= store_pt_warm<M::kAero, M::kTri>(a, k, c, s);
    } else {
      if (touched) {
        eflag |= store_pt(a, k, c, s);
        if constexpr (kStats) lvmask[k >> 5] |= 1u << (k & 31);
        if constexpr (M::kTri) {
          // the sixth moments of r, i, s, g
          double *b = a.fld + (size_t)k * a.pitch + c;
          const size_t fs = (size_t)a.nlev * (size_t)a.pitch;
#pragma unroll
          for (int x = 0; x < 4; ++x) {
            b[(16 + x) * fs] = zval(s, x);
            eflag |= nonfinite(zval(s, x));
          }
        }
        if constexpr (M::kAero) {
          // the aerosol masses: free, in cloud, in r, i, s, g
          double *b = a.fld + (size_t)k * a.pitch + c;
          const size_t fs = (size_t)a.nlev * (size_t)a.pitch;
          const double v[6] = {s.ma, s.mac, s.mar, s.mai, s.mas, s.mag};
#pragma unroll
          for (int i = 0; i < 6; ++i) {
            b[(16 + i) * fs] = v[i];
            eflag |= nonfinite(v[i]);
          }
        }
      }
    }
  }
  if (fast) {
#pragma unroll
    for (int x = 0; x < kSed; ++x) prec[x] = M::toD(Fq[x]) * a.dt;
    if constexpr (M::kAero) {
      prec[4] = 0.0;
#pragma unroll
      for (int x = 0; x < na3<M>(); ++x) prec[4] += M::toD(Fa[x]) * a.dt;
    }
  } else {
    eflag |= sediment_substeps<M, kTend>(a, P, sdz, c, prec, tend, kStats ? cs->nsub : nullptr,
                                         kStats ? lvmask : nullptr);
    if constexpr (kTend) {
      // tendency mode: the new state in tend becomes (x_new - x_old) / dt
      const size_t fs = (size_t)a.nlev * (size_t)a.pitch;
      for (int k = 0; k < a.nlev; ++k) {
        const size_t o = (size_t)k * a.pitch + c;
#pragma unroll
        for (int f = 0; f < 13; ++f) {
          const bool ice = (f >= 4 && f <= 6) || (f >= 9 && f <= 11);
          if (!(M::kWarm && ice)) tend[f * fs + o] = per_dt(tend[f * fs + o] - a.fld[f * fs + o]);
        }
#pragma unroll
        for (int e = 0; e < nextra<M>(); ++e)
          tend[(13 + e) * fs + o] = per_dt(tend[(13 + e) * fs + o] - a.fld[(16 + e) * fs + o]);
      }
    }
  }
#pragma unroll
  for (int x = 0; x < 5; ++x) {
    if (x >= kSed && !(M::kAero && x == 4)) continue;
    if (prec[x] != 0.0 && CASIM_INDEX_OK(c >= 0 && c < a.ncols, a.err)) {
      double *pp = a.precip + (size_t)x * a.pitch + c;
      *pp += prec[x];
      eflag |= nonfinite(*pp);
    }
  }
  if constexpr (kStats) {
    int n = 0;
    for (int i = 0; i < (a.nlev + 31) / 32; ++i) n += __popc(lvmask[i]);
    cs->changed = n;
  }
  return eflag;
}

// one column's statistics into the buffer: warp sums, one atomic per warp
// and counter (per distinct substep count for the histogram)
__device__ __forceinline__ void stats_add(unsigned long long *st, const ColStats &cs) {
  const unsigned mask = __activemask();
  const int lane = threadIdx.x & 31, leader = __ffs(mask) - 1;
  const unsigned act = __reduce_add_sync(mask, (unsigned)cs.active);
  const unsigned chg = __reduce_add_sync(mask, (unsigned)cs.changed);
  const unsigned cols = __popc(__ballot_sync(mask, cs.active > 0));
  if (lane == leader) {
    atomicAdd(&st[0], (unsigned long long)act);
    atomicAdd(&st[1], (unsigned long long)chg);
    atomicAdd(&st[2], (unsigned long long)cols);
  }
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const int n = min(max(cs.nsub[x], 0), 64);
    const unsigned peers = __match_any_sync(mask, n);
    if (lane == __ffs(peers) - 1) atomicAdd(&st[3 + 65 * x + n], (unsigned long long)__popc(peers));
  }
}

// kTend: tendency mode (tend receives the source terms, a.fld unchanged).
// Dynamic shared memory: step_smem_bytes<M, kTend>(a.nlev).  kStats: the
// statistics instantiation (standard configuration; a.stats set).  kLine:
// whole-line stores for a state in mapped host memory (staged policies)
template <class M, bool kTend, bool kStats = false, bool kLine = false>
__global__ void __launch_bounds__(kBlock, M::kMinBlocks) k_step(const KArgs a, const KParams P, double *tend) {
  extern __shared__ __align__(16) unsigned char step_dyn[];
  const StepSmem sm = step_smem<M, kTend>(step_dyn, a.nlev);
  const bool fast = prologue(a, P, sm);
  const int c = blockIdx.x * kBlock + threadIdx.x;
  if (c >= a.ncols) return;
  constexpr bool kStage = step_staged<M, kTend>();
  ColStats cs{0, 0, {1, 1, 1, 1}};
  const unsigned eflag = run_column<M, kTend, kStage, kStats, kLine>(a, P, sm.lt, fast, c, tend,
                                                                     kStage ? sm.stage + threadIdx.x : nullptr,
                                                                     kBlock, &cs);
  if constexpr (kStats) stats_add(a.stats, cs);
  if (eflag) atomicOr(a.err, eflag);
}

// Per-column FP64 budgets: water path and aerosol + droplet number path.
__global__ void __launch_bounds__(256) k_budget(const KArgs a, double *out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.ncols) return;
  double wsum = 0.0, nsum = 0.0;
  const size_t fs = (size_t)a.nlev * (size_t)a.pitch;
  for (int k = 0; k < a.nlev; ++k) {
    const size_t o = (size_t)k * a.pitch + c;
    const double m = a.fld[14 * fs + o] * a.dz[k];
    wsum += m * (((((a.fld[1 * fs + o] + a.fld[2 * fs + o]) + a.fld[3 * fs + o]) + a.fld[4 * fs + o]) +
                  a.fld[5 * fs + o]) + a.fld[6 * fs + o]);
    nsum += m * (a.fld[7 * fs + o] + a.fld[12 * fs + o]);
  }
  out[c] = wsum;
  out[(size_t)a.ncols + c] = nsum;
}

}  // namespace casim_dev
