// Device code of the column-microphysics step (sm_103a).
//
// One thread owns one column and walks it from the top level down
// (Section 3.2 of the paper maps one column to one GPU thread as well; the
// column's levels are coupled only through sedimentation).  Loads and stores
// are level-major, so the 32 threads of a warp touch 32 consecutive columns of
// one level: every access is a coalesced 256-byte row.
//
// Two precision policies share the code:
//   PolicyF64  every operation in FP64;
//   PolicyMix  rates, fall speeds and special functions in FP32 on the MUFU
//              pipe (ex2/lg2), state and every applied transfer in FP64.
// GB300 issues FP64 (and FP32<->FP64 conversions) at about 1/70 of the FP32
// rate, so the mixed policy converts between the two with integer bit
// operations and keeps FP64 to the additions that carry conservation.
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
};

struct KParams {
  ConstK<double> d;
  ConstK<float> f;
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
};

// ------------------------------------------------------- conversions
// FP64 <-> FP32 on the integer pipe.  Values handled here are finite and, as
// FP32, normal or zero: d2f rounds to nearest (ties away from zero) and
// flushes magnitudes below 2^-126 to zero; out-of-range or non-finite inputs
// map to NaN so they still raise the non-finite flag downstream.  f2d is
// exact for normal and zero inputs (the FP32 code runs with flush-to-zero).
__device__ __forceinline__ float d2f(double x) {
  const unsigned hi = (unsigned)__double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const unsigned s = hi & 0x80000000u;
  const unsigned a = hi & 0x7fffffffu;
  // 8-bit exponent and 23-bit mantissa, plus the first dropped bit (a carry
  // out of the mantissa correctly bumps the exponent)
  unsigned r = __funnelshift_l(lo, a - 0x38000000u, 3) + ((lo >> 28) & 1u);
  r = a < 0x38100000u ? 0u : r;
  r = a >= 0x47f00000u ? 0x7fc00000u : r;
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

// non-finite test on the high word (integer pipe)
__device__ __forceinline__ unsigned nonfinite(double x) {
  return ((unsigned)__double2hiint(x) & 0x7ff00000u) == 0x7ff00000u;
}

// --------------------------------------------------------- policies
struct PolicyF64 {
  using R = double;
  static constexpr bool kMixed = false;
  static __device__ __forceinline__ const ConstK<double> &K(const KParams &p) { return p.d; }
  static __device__ __forceinline__ R toR(double x) { return x; }
  static __device__ __forceinline__ double toD(R x) { return x; }
  static __device__ __forceinline__ R exp(R x) { return ::exp(x); }
  static __device__ __forceinline__ R lg(R x) { return ::log(x); }   // log in the constants' base
  static __device__ __forceinline__ R ex(R x) { return ::exp(x); }   // inverse of lg
  static __device__ __forceinline__ R ln(R x) { return ::log(x); }
  static __device__ __forceinline__ R sqrt(R x) { return ::sqrt(x); }
  static __device__ __forceinline__ R cbrt(R x) { return ::cbrt(x); }
  static __device__ __forceinline__ R erfc(R x) { return ::erfc(x); }
  static __device__ __forceinline__ R div(R a, R b) { return a / b; }
  static __device__ __forceinline__ R mn(R a, R b) { return a < b ? a : b; }
  static __device__ __forceinline__ R mx(R a, R b) { return a > b ? a : b; }
};

struct PolicyMix {
  using R = float;
  static constexpr bool kMixed = true;
  static __device__ __forceinline__ const ConstK<float> &K(const KParams &p) { return p.f; }
  static __device__ __forceinline__ R toR(double x) { return d2f(x); }
  static __device__ __forceinline__ double toD(R x) { return f2d(x); }
  static __device__ __forceinline__ R exp(R x) { return ex2a(x * 1.44269504088896341f); }
  static __device__ __forceinline__ R lg(R x) { return lg2a(x); }
  static __device__ __forceinline__ R ex(R x) { return ex2a(x); }
  static __device__ __forceinline__ R ln(R x) { return lg2a(x) * 0.693147180559945309f; }
  static __device__ __forceinline__ R sqrt(R x) { return sqrta(x); }
  static __device__ __forceinline__ R cbrt(R x) { return ex2a(lg2a(x) * 0.333333343267f); }
  static __device__ __forceinline__ R erfc(R x) { return erfcf(x); }
  static __device__ __forceinline__ R div(R a, R b) { return __fdividef(a, b); }
  static __device__ __forceinline__ R mn(R a, R b) { return fminf(a, b); }
  static __device__ __forceinline__ R mx(R a, R b) { return fmaxf(a, b); }
};

// ------------------------------------------------------------ one point
struct Pt {
  double T, qv, qc, qr, qi, qs, qg, nc, nr, ni, ns, ng, na, p, rho, w;
};

enum { F_T = 0, F_QV, F_QC, F_QR, F_QI, F_QS, F_QG, F_NC, F_NR, F_NI, F_NS, F_NG, F_NA, F_P, F_RHO, F_W };

template <class M>
struct Chain {
  using R = typename M::R;

  // saturation specific humidity over liquid and its temperature derivative
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

  // Activity test: true unless the whole chain would leave the point
  // unchanged (no hydrometeor present, not supersaturated over liquid, no
  // ice nucleation possible).  Also returns qs over liquid at the initial
  // temperature, which saturation adjustment reuses.
  static __device__ __forceinline__ bool active(const ConstK<R> &K, const Pt &s, R &tc0, R &es0, R &qs0) {
    tc0 = M::toR(s.T - (double)K.T0);
    const R p = M::toR(s.p);
    es0 = es_liq(K, tc0);
    qs0 = qsat(K, es0, p);
    const R qmin = K.qmin;
    bool act = M::toR(s.qc) > qmin || M::toR(s.qr) > qmin || M::toR(s.qi) > qmin ||
               M::toR(s.qs) > qmin || M::toR(s.qg) > qmin || M::toR(s.qv) > qs0;
    if (!act && M::toR(s.T) < K.Tnuc) act = M::div(M::toR(s.qv), qsat(K, es_ice(K, s.T, tc0), p)) > (R)1;
    return act;
  }

  // a2: isobaric saturation adjustment, 4 Newton iterations on
  // cp (T* - T) = Lv (qv - qs(T*)), condensate limited by the cloud present.
  static __device__ __forceinline__ void satadj(const ConstK<R> &K, Pt &s, R tc0, R es0, R qs0) {
    const R p = M::toR(s.p);
    if (!(M::toR(s.qv) > qs0 || M::toR(s.qc) > K.qmin)) return;
    if constexpr (!M::kMixed) {
      const double T0v = s.T, qv0 = s.qv, qc0 = s.qc;
      double Tn = T0v, es = es0, qs = qs0;
      for (int it = 0; it < 4; ++it) {
        if (it > 0) {
          es = es_liq(K, Tn - K.T0);
          qs = qsat(K, es, p);
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
    } else {
      // FP32 Newton on the temperature increment; the vapour difference
      // qv - qs is formed in FP64 each iteration.
      R dT = 0.f, es = es0, qs = qs0;
      for (int it = 0; it < 4; ++it) {
        const R tc = tc0 + dT;
        if (it > 0) {
          es = es_liq(K, tc);
          qs = qsat(K, es, p);
        }
        const R d = M::toR(s.qv - M::toD(qs));
        const R f = dT - K.lv_cp * d;
        const R e1 = tc + K.eslb;
        const R des = es * K.eslab * rcpa(e1 * e1);
        const R den = p - K.ome * es;
        const R fp = 1.f + K.lv_cp * K.eps * p * des * rcpa(den * den);
        dT = dT - M::div(f, fp);
      }
      const R dq = K.cp_lv * dT;
      const R qc0 = M::toR(s.qc);
      double dqd;
      R dqr;
      if (dq <= -qc0) {
        dqd = -s.qc;
        dqr = -qc0;
      } else {
        dqd = M::toD(dq);
        dqr = dq;
      }
      s.T += M::toD(K.lv_cp * dqr);
      s.qv -= dqd;
      s.qc += dqd;
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

  static __device__ __forceinline__ void activate(const ConstK<R> &K, Pt &s) {
    if (!(s.w > 0.0) || !(M::toR(s.qc) > K.qmin)) return;
    const R rho = M::toR(s.rho);
    const R N = rho * M::toR(s.na + s.nc);
    if (!(N > (R)0)) return;
    const R T = M::toR(s.T);
    const R es = es_liq(K, M::toR(s.T - (double)K.T0));
    const R nact = arg_nact(K, N, M::toR(s.w), T, M::toR(s.p), es);
    if constexpr (!M::kMixed) {
      double dn = nact / s.rho - s.nc;
      if (dn < 0.0) dn = 0.0;
      if (dn > s.na) dn = s.na;
      s.nc += dn;
      s.na -= dn;
    } else {
      R dn = M::div(nact, rho) - M::toR(s.nc);
      dn = M::mx(dn, (R)0);
      dn = M::mn(dn, M::toR(s.na));
      if (dn > (R)0) {
        const double dnd = M::toD(dn);
        s.nc += dnd;
        s.na -= dnd;
      }
    }
  }

  // log of the gamma slope of species x from (q, n), clamped
  static __device__ __forceinline__ R lglam(const SpeciesK<R> &X, R lgq, R n) {
    const R lgn = M::lg(M::mx(n, (R)0));
    R l = (X.lglamfac + lgn - lgq) * X.invb;
    l = M::mx(l, X.lglo);   // also maps log(0) = -inf (and NaN) to the lower bound
    return M::mn(l, X.lghi);
  }

  // a4..a10 on an adjusted, activated point
  static __device__ __forceinline__ void rates_and_limit(const ConstK<R> &K, Pt &s, double dt) {
    const R T = M::toR(s.T), p = M::toR(s.p), rho = M::toR(s.rho);
    const R qv = M::toR(s.qv), qc = M::toR(s.qc), qr = M::toR(s.qr);
    const R qx[3] = {M::toR(s.qi), M::toR(s.qs), M::toR(s.qg)};
    const R nc = M::toR(s.nc), nr = M::toR(s.nr);
    const R nx[3] = {M::toR(s.ni), M::toR(s.ns), M::toR(s.ng)};
    const R dtr = M::toR(dt);
    const R tc = M::toR(s.T - (double)K.T0);
    const R esl = es_liq(K, tc);
    const R qsl = qsat(K, esl, p);
    const R iT2 = M::div((R)1, T * T);
    const R Sw = M::div(qv, qsl);
    const bool hc = qc > K.qmin, hr = qr > K.qmin;
    const bool cold = T < K.T0, warm = T > K.T0;

    // air properties shared by the ventilated integrals
    const R lgrho = M::lg(rho);
    const R dfac = M::ex((R)0.4 * (K.lgrho0 - lgrho));         // (rho0/rho)^0.4
    const R nu = M::div(K.mu_air, rho);
    const R V0 = M::cbrt(nu * K.inv_dv) * M::sqrt(M::div(dfac, nu));

    R aut = 0, acc = 0, scc = 0, scr = 0, evr = 0, nucn = 0;
    R dep[3] = {0, 0, 0}, rim[2] = {0, 0}, mlt[3] = {0, 0, 0};

    const R lgqc = hc ? M::lg(qc) : (R)0;
    const R lgqr = hr ? M::lg(qr) : (R)0;
    if (hc) {
      const R ncc = M::mx(rho * nc * (R)1e-6, K.nc_min);
      aut = K.kk_aut * M::ex(K.kk_aut_qc * lgqc + K.kk_aut_nc * M::lg(ncc));
      scc = K.kcf * rho * qc * qc;
    }
    if (hc && hr) acc = K.kk_acc * M::ex(K.kk_acc_exp * (lgqc + lgqr));
    if (hr) {
      scr = K.kr * rho * M::mx(nr, (R)0) * qr;
      if (Sw < (R)1) {
        const SpeciesK<R> &X = K.sp[1];
        const R l = lglam(X, lgqr, nr);
        const R iv = rho * qr * (X.ev1 * M::ex(X.ex1 * l) + V0 * X.ev2 * M::ex(X.ex2 * l));
        const R Aw = K.awc * iT2, Bw = M::div(K.rv_dv * T, esl);
        evr = M::div(K.twopi * ((R)1 - Sw) * iv, rho * (Aw + Bw));
      }
    }
    if (cold || T < K.Tnuc) {
      const R esi = es_ice(K, s.T, tc);
      const R qsi = qsat(K, esi, p);
      const R Si = M::div(qv, qsi);
      if (T < K.Tnuc && Si > (R)1) {
        const R nin = K.mey_a * M::exp(K.mey_b + K.mey_c * (Si - (R)1));
        const R dn = M::div(nin, rho) - nx[0];
        if (dn > (R)0) nucn = M::div(dn, dtr);
      }
      if (cold) {
        const R Ai = K.aic * iT2, Bi = M::div(K.rv_dv * T, esi);
        const R dfa = M::div(Si - (R)1, rho * (Ai + Bi));
#pragma unroll
        for (int m = 0; m < 3; ++m) {
          if (!(qx[m] > K.qmin)) continue;
          const SpeciesK<R> &X = K.sp[2 + m];
          const R lq = M::lg(qx[m]);
          const R l = lglam(X, lq, nx[m]);
          const R iv = rho * qx[m] * (X.ev1 * M::ex(X.ex1 * l) + V0 * X.ev2 * M::ex(X.ex2 * l));
          dep[m] = X.dep * dfa * iv;
          if (m > 0 && hc) rim[m - 1] = X.rim * qc * dfac * rho * qx[m] * M::ex(X.exr * l);
        }
      }
    }
    if (warm) {
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        if (!(qx[m] > K.qmin)) continue;
        const SpeciesK<R> &X = K.sp[2 + m];
        const R lq = M::lg(qx[m]);
        const R l = lglam(X, lq, nx[m]);
        const R iv = rho * qx[m] * (X.ev1 * M::ex(X.ex1 * l) + V0 * X.ev2 * M::ex(X.ex2 * l));
        mlt[m] = M::div(X.mlt * tc * iv, rho);
      }
    }

    limit_apply(K, s, dt, qv, qc, qr, qx, nc, nr, nx, aut, acc, scc, scr, evr, nucn, dep, rim, mlt);
  }

  // a10: per-pool limiting factors, each transfer scaled by the smallest
  // factor of the pools it draws from, applied once to source and sink.
  static __device__ __forceinline__ void limit_apply(const ConstK<R> &K, Pt &s, double dt, R qv, R qc, R qr,
                                                     const R qx[3], R nc, R nr, const R nx[3], R aut, R acc,
                                                     R scc, R scr, R evr, R nucn, const R dep[3], const R rim[2],
                                                     const R mlt[3]) {
    const R dtr = M::toR(dt);
    const R rc = qc > K.qmin ? M::div(M::mx(nc, (R)0), qc) : (R)0;
    const R rr = qr > K.qmin ? M::div(M::mx(nr, (R)0), qr) : (R)0;
    R rx[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) rx[m] = qx[m] > K.qmin ? M::div(M::mx(nx[m], (R)0), qx[m]) : (R)0;
    const R nucm = nucn * K.mi0;
    R sub[3], depp[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      depp[m] = dep[m] >= (R)0 ? dep[m] : (R)0;
      sub[m] = dep[m] >= (R)0 ? (R)0 : -dep[m];
    }
    // sinks per pool (same summation order as the transfer list)
    const R S_qv = ((nucm + depp[0]) + depp[1]) + depp[2];
    const R S_qc = ((aut + acc) + rim[0]) + rim[1];
    const R S_qr = evr;
    R S_qx[3], S_nx[3], nmlt[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      S_qx[m] = sub[m] + mlt[m];
      nmlt[m] = mlt[m] > (R)0 ? mlt[m] * rx[m] : (R)0;
      S_nx[m] = sub[m] * rx[m] + nmlt[m];
    }
    const R S_nc = (((aut * rc + acc * rc) + scc) + rim[0] * rc) + rim[1] * rc;
    const R S_nr = scr + evr * rr;

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
    const R f_qv = fac(S_qv, qv), f_qc = fac(S_qc, qc), f_qr = fac(S_qr, qr);
    const R f_nc = fac(S_nc, nc), f_nr = fac(S_nr, nr);
    R f_qx[3], f_nx[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      f_qx[m] = fac(S_qx[m], qx[m]);
      f_nx[m] = fac(S_nx[m], nx[m]);
    }
    auto g2 = [&](R rate, R fm, R nsink, R fn) -> R {
      R g = (R)1;
      if (rate > (R)0 && fm < g) g = fm;
      if (nsink > (R)0 && fn < g) g = fn;
      return g;
    };
    const R g_aut = g2(aut, f_qc, aut * rc, f_nc);
    const R g_acc = g2(acc, f_qc, acc * rc, f_nc);
    const R g_scc = g2(0, 1, scc, f_nc);
    const R g_scr = g2(0, 1, scr, f_nr);
    const R g_evr = g2(evr, f_qr, evr * rr, f_nr);
    const R g_nuc = g2(nucm, f_qv, 0, 1);
    R g_dep[3], g_mlt[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) {
      g_dep[m] = dep[m] >= (R)0 ? g2(depp[m], f_qv, 0, 1) : g2(sub[m], f_qx[m], sub[m] * rx[m], f_nx[m]);
      g_mlt[m] = g2(mlt[m], f_qx[m], nmlt[m], f_nx[m]);
    }
    const R g_rs = g2(rim[0], f_qc, rim[0] * rc, f_nc);
    const R g_rg = g2(rim[1], f_qc, rim[1] * rc, f_nc);

    if constexpr (!M::kMixed) {
      // FP64: transfers applied one by one in list order
      double qxd[3] = {s.qi, s.qs, s.qg};
      double nxd[3] = {s.ni, s.ns, s.ng};
      const double mr0i = K.inv_mr0;
      double tau;
      if (aut > 0) { tau = g_aut * aut * dt; s.qc -= tau; s.qr += tau; }
      if (aut * rc > 0) s.nc -= g_aut * (aut * rc) * dt;
      if (aut * mr0i > 0) s.nr += g_aut * (aut * mr0i) * dt;
      if (acc > 0) { tau = g_acc * acc * dt; s.qc -= tau; s.qr += tau; }
      if (acc * rc > 0) s.nc -= g_acc * (acc * rc) * dt;
      if (scc > 0) s.nc -= g_scc * scc * dt;
      if (scr > 0) s.nr -= g_scr * scr * dt;
      if (evr > 0) { tau = g_evr * evr * dt; s.qr -= tau; s.qv += tau; s.T += tau * (-K.lv) / K.cp; }
      if (evr * rr > 0) s.nr -= g_evr * (evr * rr) * dt;
      if (nucm > 0) { tau = g_nuc * nucm * dt; s.qv -= tau; qxd[0] += tau; s.T += tau * K.ls / K.cp; }
      if (nucn > 0) nxd[0] += g_nuc * nucn * dt;
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        if (dep[m] >= 0) {
          if (depp[m] > 0) { tau = g_dep[m] * depp[m] * dt; s.qv -= tau; qxd[m] += tau; s.T += tau * K.ls / K.cp; }
        } else {
          tau = g_dep[m] * sub[m] * dt; qxd[m] -= tau; s.qv += tau; s.T += tau * (-K.ls) / K.cp;
          if (sub[m] * rx[m] > 0) nxd[m] -= g_dep[m] * (sub[m] * rx[m]) * dt;
        }
      }
      if (rim[0] > 0) { tau = g_rs * rim[0] * dt; s.qc -= tau; qxd[2] += tau; s.T += tau * K.lf / K.cp; }
      if (rim[0] * rc > 0) s.nc -= g_rs * (rim[0] * rc) * dt;
      if (rim[1] > 0) { tau = g_rg * rim[1] * dt; s.qc -= tau; qxd[2] += tau; s.T += tau * K.lf / K.cp; }
      if (rim[1] * rc > 0) s.nc -= g_rg * (rim[1] * rc) * dt;
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        if (mlt[m] > 0) { tau = g_mlt[m] * mlt[m] * dt; qxd[m] -= tau; s.qr += tau; s.T += tau * (-K.lf) / K.cp; }
        if (nmlt[m] > 0) { nxd[m] -= g_mlt[m] * nmlt[m] * dt; s.nr += g_mlt[m] * nmlt[m] * dt; }
      }
      s.qi = qxd[0]; s.qs = qxd[1]; s.qg = qxd[2];
      s.ni = nxd[0]; s.ns = nxd[1]; s.ng = nxd[2];
    } else {
      // Mixed: each (source, destination) pair moves one FP32 amount, added
      // to and subtracted from the FP64 state, so water is conserved to FP64
      // rounding.  Net number and heat changes are FP32 sums.
      const R t_cr = g_aut * aut * dtr + g_acc * acc * dtr;
      const R t_cg = g_rs * rim[0] * dtr + g_rg * rim[1] * dtr;
      const R t_rv = g_evr * evr * dtr;
      R t_vx[3], t_xr[3];
      t_vx[0] = g_nuc * nucm * dtr + g_dep[0] * dep[0] * dtr;  // signed: deposition > 0
      t_vx[1] = g_dep[1] * dep[1] * dtr;
      t_vx[2] = g_dep[2] * dep[2] * dtr;
#pragma unroll
      for (int m = 0; m < 3; ++m) t_xr[m] = g_mlt[m] * mlt[m] * dtr;
      if (t_cr != (R)0) { const double d = M::toD(t_cr); s.qc -= d; s.qr += d; }
      if (t_cg != (R)0) { const double d = M::toD(t_cg); s.qc -= d; s.qg += d; }
      if (t_rv != (R)0) { const double d = M::toD(t_rv); s.qr -= d; s.qv += d; }
      if (t_vx[0] != (R)0) { const double d = M::toD(t_vx[0]); s.qv -= d; s.qi += d; }
      if (t_vx[1] != (R)0) { const double d = M::toD(t_vx[1]); s.qv -= d; s.qs += d; }
      if (t_vx[2] != (R)0) { const double d = M::toD(t_vx[2]); s.qv -= d; s.qg += d; }
      if (t_xr[0] != (R)0) { const double d = M::toD(t_xr[0]); s.qi -= d; s.qr += d; }
      if (t_xr[1] != (R)0) { const double d = M::toD(t_xr[1]); s.qs -= d; s.qr += d; }
      if (t_xr[2] != (R)0) { const double d = M::toD(t_xr[2]); s.qg -= d; s.qr += d; }
      const R dnc = -(g_aut * aut * rc + g_acc * acc * rc + g_scc * scc + g_rs * rim[0] * rc + g_rg * rim[1] * rc) * dtr;
      const R dnr = (g_aut * aut * K.inv_mr0 - g_scr * scr - g_evr * evr * rr +
                     g_mlt[0] * nmlt[0] + g_mlt[1] * nmlt[1] + g_mlt[2] * nmlt[2]) * dtr;
      R dnx[3];
      dnx[0] = g_nuc * nucn * dtr;
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const R sn = dep[m] < (R)0 ? g_dep[m] * sub[m] * rx[m] : (R)0;
        dnx[m] = (m == 0 ? dnx[0] : (R)0) - (sn + g_mlt[m] * nmlt[m]) * dtr;
      }
      const R dT = (K.ls * (t_vx[0] + t_vx[1] + t_vx[2]) + K.lf * t_cg - K.lv * t_rv -
                    K.lf * (t_xr[0] + t_xr[1] + t_xr[2])) * K.inv_cp;
      if (dnc != (R)0) s.nc += M::toD(dnc);
      if (dnr != (R)0) s.nr += M::toD(dnr);
      if (dnx[0] != (R)0) s.ni += M::toD(dnx[0]);
      if (dnx[1] != (R)0) s.ns += M::toD(dnx[1]);
      if (dnx[2] != (R)0) s.ng += M::toD(dnx[2]);
      if (dT != (R)0) s.T += M::toD(dT);
    }
  }

  // sedimentation: speeds of species x (0..3 = r,i,s,g) at one point
  static __device__ __forceinline__ void fall_speeds(const ConstK<R> &K, R guard, R q, R n, R rho, int x, R &vq,
                                                     R &vn) {
    const SpeciesK<R> &X = K.sp[1 + x];
    const R l = lglam(X, M::lg(q), n);
    const R dfac = M::ex((R)0.4 * (K.lgrho0 - M::lg(rho)));
    const R pw = M::ex(X.exv * l);
    vq = M::mn(X.vq * dfac * pw, X.vmax);
    vn = M::mn(X.vn * dfac * pw, X.vmax);
    vq = M::mn(vq, guard);
    vn = M::mn(vn, guard);
  }
};

// ---------------------------------------------------------------- kernels
__device__ __forceinline__ size_t fidx(const KArgs &a, int f, int k, int c) {
  return ((size_t)f * (size_t)a.nlev + (size_t)k) * (size_t)a.pitch + (size_t)c;
}

__device__ __forceinline__ void load_pt(const KArgs &a, int k, int c, Pt &s) {
  const double *b = a.fld + (size_t)k * a.pitch + c;
  const size_t fs = (size_t)a.nlev * (size_t)a.pitch;
  s.T = b[0 * fs]; s.qv = b[1 * fs]; s.qc = b[2 * fs]; s.qr = b[3 * fs];
  s.qi = b[4 * fs]; s.qs = b[5 * fs]; s.qg = b[6 * fs];
  s.nc = b[7 * fs]; s.nr = b[8 * fs]; s.ni = b[9 * fs]; s.ns = b[10 * fs]; s.ng = b[11 * fs];
  s.na = b[12 * fs];
  s.p = __ldg(b + 13 * fs); s.rho = __ldg(b + 14 * fs); s.w = __ldg(b + 15 * fs);
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

__device__ __forceinline__ double &qref(Pt &s, int x) {
  return x == 0 ? s.qr : x == 1 ? s.qi : x == 2 ? s.qs : s.qg;
}
__device__ __forceinline__ double &nref(Pt &s, int x) {
  return x == 0 ? s.nr : x == 1 ? s.ni : x == 2 ? s.ns : s.ng;
}

// One timestep for ncols columns.  When every species' capped fall speed
// satisfies vmax dt / min(dz) <= c_max, each column needs exactly one
// sedimentation substep and the flux recurrence is fused into the top-down
// sweep of the processes (one read and one write of the state).  Otherwise
// the processes are applied first and each species is sedimented with its
// own substep count in further sweeps over the column.
template <class M>
__global__ void __launch_bounds__(kBlock) k_step(const KArgs a, const KParams P) {
  using R = typename M::R;
  using C = Chain<M>;
  __shared__ double s_dz[kMaxLev];
  __shared__ int s_fast;
  const ConstK<R> &K = M::K(P);

  double dzmin = 1e300;
  for (int k = threadIdx.x; k < a.nlev; k += blockDim.x) {
    const double v = a.dz[k];
    s_dz[k] = v;
    dzmin = fmin(dzmin, v);
  }
  // block-wide minimum of dz
  for (int o = 16; o > 0; o >>= 1) dzmin = fmin(dzmin, __shfl_xor_sync(0xffffffffu, dzmin, o));
  __shared__ double s_red[kBlock / 32];
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = dzmin;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = s_red[0];
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) m = fmin(m, s_red[i]);
    int fast = 1;
    for (int x = 1; x < 5; ++x) fast &= ((P.vmax[x] * a.dt) / m) / P.c_max <= 1.0;
    s_fast = fast;
  }
  __syncthreads();
  const bool fast = s_fast != 0;

  const int c = blockIdx.x * kBlock + threadIdx.x;
  if (c >= a.ncols) return;

  unsigned eflag = 0;
  double prec[4] = {0.0, 0.0, 0.0, 0.0};

  if (fast) {
    // carried downward fluxes F_{k+1}, G_{k+1} (kg m^-2 s^-1, m^-2 s^-1)
    R Fq[4] = {0, 0, 0, 0}, Fn[4] = {0, 0, 0, 0};
    for (int k = a.nlev - 1; k >= 0; --k) {
      Pt s;
      load_pt(a, k, c, s);
      eflag |= nonfinite_in(s);
      R tc0, es0, qs0;
      const bool act = C::active(K, s, tc0, es0, qs0);
      if (act) {
        C::satadj(K, s, tc0, es0, qs0);
        C::activate(K, s);
        C::rates_and_limit(K, s, a.dt);
      }
      const double dzk = s_dz[k];
      const R vguard = M::toR(dzk / a.dt);
      const R rho = M::toR(s.rho);
      bool touched = act;
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        double &q = qref(s, x);
        double &n = nref(s, x);
        R F = 0, G = 0;
        const R qR = M::toR(q);
        if (qR > K.qmin) {
          R vq, vn;
          C::fall_speeds(K, vguard, qR, M::toR(n), rho, x, vq, vn);
          if constexpr (!M::kMixed) {
            F = s.rho * q * vq;
            G = s.rho * (n > 0.0 ? n : 0.0) * vn;
          } else {
            F = rho * qR * vq;
            G = rho * M::mx(M::toR(n), (R)0) * vn;
          }
        }
        if (F != (R)0 || Fq[x] != (R)0 || G != (R)0 || Fn[x] != (R)0) {
          if constexpr (!M::kMixed) {
            q += a.dt * (Fq[x] - F) / (s.rho * dzk);
            n += a.dt * (Fn[x] - G) / (s.rho * dzk);
          } else {
            const R sc = M::div(M::toR(a.dt), rho * M::toR(dzk));
            q += M::toD((Fq[x] - F) * sc);
            n += M::toD((Fn[x] - G) * sc);
          }
          touched = true;
        }
        Fq[x] = F;
        Fn[x] = G;
      }
      if (touched) eflag |= store_pt(a, k, c, s);
    }
#pragma unroll
    for (int x = 0; x < 4; ++x) prec[x] = M::toD(Fq[x]) * a.dt;
  } else {
    // processes first ...
    for (int k = a.nlev - 1; k >= 0; --k) {
      Pt s;
      load_pt(a, k, c, s);
      eflag |= nonfinite_in(s);
      R tc0, es0, qs0;
      if (C::active(K, s, tc0, es0, qs0)) {
        C::satadj(K, s, tc0, es0, qs0);
        C::activate(K, s);
        C::rates_and_limit(K, s, a.dt);
        eflag |= store_pt(a, k, c, s);
      }
    }
    // ... then each species with its own substep count
    const size_t fs = (size_t)a.nlev * (size_t)a.pitch;
    const double *rhop = a.fld + 14 * fs;
    for (int x = 0; x < 4; ++x) {
      double *qp = a.fld + (3 + x) * fs;
      double *np = a.fld + (8 + x) * fs;
      R cmax = 0;
      for (int k = 0; k < a.nlev; ++k) {
        const size_t o = (size_t)k * a.pitch + c;
        const R q = M::toR(qp[o]);
        if (!(q > K.qmin)) continue;
        R vq, vn;
        C::fall_speeds(K, (R)1e30, q, M::toR(np[o]), M::toR(__ldg(rhop + o)), x, vq, vn);
        const R cr = M::div(vq * M::toR(a.dt), M::toR(s_dz[k]));
        cmax = M::mx(cmax, cr);
      }
      int ns = (int)ceil((double)M::div(cmax, M::toR(P.c_max)));
      if (ns < 1) ns = 1;
      if (ns > 64) { ns = 64; eflag |= 2u; }
      const double dts = a.dt / ns;
      for (int st = 0; st < ns; ++st) {
        R Fu = 0, Gu = 0;
        for (int k = a.nlev - 1; k >= 0; --k) {
          const size_t o = (size_t)k * a.pitch + c;
          double q = qp[o], n = np[o];
          const double rhod = __ldg(rhop + o);
          const R qR = M::toR(q), rho = M::toR(rhod);
          R F = 0, G = 0;
          if (qR > K.qmin) {
            R vq, vn;
            C::fall_speeds(K, M::toR(s_dz[k] / dts), qR, M::toR(n), rho, x, vq, vn);
            if constexpr (!M::kMixed) {
              F = rhod * q * vq;
              G = rhod * (n > 0.0 ? n : 0.0) * vn;
            } else {
              F = rho * qR * vq;
              G = rho * M::mx(M::toR(n), (R)0) * vn;
            }
          }
          if (F != (R)0 || Fu != (R)0 || G != (R)0 || Gu != (R)0) {
            if constexpr (!M::kMixed) {
              q += dts * (Fu - F) / (rhod * s_dz[k]);
              n += dts * (Gu - G) / (rhod * s_dz[k]);
            } else {
              const R sc = M::div(M::toR(dts), rho * M::toR(s_dz[k]));
              q += M::toD((Fu - F) * sc);
              n += M::toD((Gu - G) * sc);
            }
            qp[o] = q;
            np[o] = n;
            eflag |= nonfinite(q) | nonfinite(n);
          }
          Fu = F;
          Gu = G;
        }
        prec[x] += M::toD(Fu) * dts;
      }
    }
  }
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    if (prec[x] != 0.0) {
      double *pp = a.precip + (size_t)x * a.pitch + c;
      *pp += prec[x];
      eflag |= nonfinite(*pp);
    }
  }
  if (eflag) atomicOr(a.err, eflag);
}

// Per-column FP64 budgets: water path and aerosol + droplet number path.
__global__ void __launch_bounds__(256) k_budget(const KArgs a, double *out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= a.ncols) return;
  double wsum = 0.0, nsum = 0.0;
  for (int k = 0; k < a.nlev; ++k) {
    const size_t o = (size_t)k * a.pitch + c;
    const size_t fs = (size_t)a.nlev * (size_t)a.pitch;
    const double m = a.fld[14 * fs + o] * a.dz[k];
    wsum += m * (((((a.fld[1 * fs + o] + a.fld[2 * fs + o]) + a.fld[3 * fs + o]) + a.fld[4 * fs + o]) +
                  a.fld[5 * fs + o]) + a.fld[6 * fs + o]);
    nsum += m * (a.fld[7 * fs + o] + a.fld[12 * fs + o]);
  }
  out[c] = wsum;
  out[(size_t)a.ncols + c] = nsum;
}

}  // namespace casim_dev
