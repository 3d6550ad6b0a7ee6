// EES-L1 device model on the GPU with a hand-derived Jacobian.
//
// The paper evaluates BSIM4 v4.82 per device in the compute phase of every Newton iteration
// (Sec. II (i): terminal currents, charges and linearised conductances at the present bias) but
// prints no model equations. This file implements the documented BSIM-style level EES-L1:
//   (1) source/drain mode swap, (2) smooth body effect with DIBL, (3) softplus effective
//   overdrive, (4) bulk-charge factor, (5) mobility degradation, (6) velocity saturation,
//   (7) smooth min(vds, Vdsat), (8) drain current with length modulation, (9) channel current
//   into the terminals, (10) body-drain / body-source junctions with exponent limiting above
//   40 Vt, (11) charge partition with overlaps, (12) the analytic Jacobian dI_t/dV_u.
//
// The code is written once for a scalar type S: S = double for the forward kernels, and S = a
// tangent (forward-mode) type for the backward kernel, which needs derivatives of the Jacobian.
// Every division and square root goes through rcp()/rsqrt() overloads so that one reciprocal is
// shared between a quotient and its derivatives.
#pragma once

#include "eec_fastmath.cuh"
#include "eec_internal.h"

namespace eec {

// ---- scalar helpers for S = double ----
__device__ __forceinline__ double sval(double x) { return x; }
__device__ __forceinline__ double rcp(double x) { return fm_rcp(x); }
__device__ __forceinline__ double rsqrt_(double x) { return fm_rsqrt(x); }
__device__ __forceinline__ double exp_(double x) { return fm_exp(x); }
__device__ __forceinline__ double expm1_(double x) { return fm_expm1(x); }
// log(1 + e) for e in [0, 1], given inv_y = 1 / (1 + e)
__device__ __forceinline__ double log1p_(double e, double inv_y) { return fm_log1p01(e, inv_y); }
// x * (+1 or -1) as a sign-bit flip on the integer pipe (sb is 0 or the sign bit).
__device__ __forceinline__ double flip(double x, unsigned long long sb) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)sb);
}
constexpr unsigned long long kSignBit = 0x8000000000000000ull;
// 2 x and x / 2: for S = double exact exponent-field adds on the integer pipe (fm_pow2), for
// the tangent types of the backward a multiplication.
__device__ __forceinline__ double twice(double x) { return fm_pow2(x, 1); }
__device__ __forceinline__ double half(double x) { return fm_pow2(x, -1); }
template <class S>
__device__ __forceinline__ S twice(const S& x) { return 2.0 * x; }
template <class S>
__device__ __forceinline__ S half(const S& x) { return 0.5 * x; }

template <class S>
struct PrmS {
  S beta0;   // U0 Cox W / L
  S cE;      // 2 VSAT L / U0 (EsatL = cE * mobility denominator)
  S inv_cE;  // 1 / cE
  S lamL;    // LAMBDA LREF / L
  S Isat;    // JS W HDIF
  S Coxt;    // Cox W L
  S CovS;    // CGSO W
  S CovD;    // CGDO W
  S IsatVt;  // Isat / Vt   (junction conductance slope)
  S IsatVtG; // Isat / Vt + GMIN
};

// Per-device parameters from W and L (the forward stores these per position; the backward
// recomputes them in tangent arithmetic so that W and L derivatives flow through).
template <class S>
__device__ __forceinline__ PrmS<S> derive_params(const CardK& c, const S& W, const S& L) {
  PrmS<S> P;
  const S iL = rcp(L);
  P.beta0 = c.U0Cox * W * iL;
  P.cE = c.twoVSAT_U0 * L;
  P.inv_cE = iL * (1.0 / c.twoVSAT_U0);
  P.lamL = c.LAMBDA_LREF * iL;
  P.Isat = c.JS_HDIF * W;
  P.Coxt = c.Cox * W * L;
  P.CovS = c.CGSO * W;
  P.CovD = c.CGDO * W;
  P.IsatVt = P.Isat * c.inv_Vt;
  P.IsatVtG = P.IsatVt + c.GMIN;
  return P;
}

template <class S>
struct EvalOut {
  S I[4];      // current from node t into the device, t = d, g, s, b (I[1] == 0)
  S G[3][4];   // rows d, s, b of dI_t / dV_u, u = d, g, s, b (gate row is zero in DC)
  S Q[4];      // terminal charges (only when requested)
  S C[4][4];   // dQ_t / dV_u, rows d, g, s, b (transient only)
  // the parts I and G are formed from (see i_entry, g_entry): channel row of the physical
  // drain, junction currents and conductances, polarity sign bit
  S cdd, cdg, cds, cdb, gjd, gjs, Ichd, Ijd, Ijs;
  unsigned long long psb;
  // the parts C is formed from (see c_entry): mode-frame derivatives of the inversion charge,
  // of its drain share and of the depletion charge, by physical terminal; the overlap
  // capacitances; the mode
  S MQi[4], MQD[4], MQb[4], CovS, CovD;
  bool fwd;
};

// Entry (r, u) of G and entry t of I, formed from their parts. The DC stamps call these inside
// their tests for free rows and columns, so that entries of held terminals cost no FP64 issue
// slot (two thirds of a logic netlist's devices have source and body on a rail); I and G as
// stored by ees_l1 are the same expressions.
template <class S>
__device__ __forceinline__ S g_entry(const EvalOut<S>& o, int r, int u) {
  if (r == 0) return u == 0 ? o.cdd + o.gjd : u == 1 ? o.cdg : u == 2 ? o.cds : o.cdb - o.gjd;
  if (r == 1) return u == 0 ? -o.cdd : u == 1 ? -o.cdg : u == 2 ? o.gjs - o.cds : -o.cdb - o.gjs;
  return u == 0 ? -o.gjd : u == 1 ? S(0.0) : u == 2 ? -o.gjs : o.gjd + o.gjs;
}
// Entry (t, u) of C, formed from its parts: physical d carries the drain share QD in forward
// mode and QS = Qinv - QD in reverse mode; the gate row is minus the sum of the others; then the
// overlaps, q_g += CovS (Vg - Vs) + CovD (Vg - Vd), q_s -= CovS (Vg - Vs), q_d -= CovD (Vg - Vd).
template <class S>
__device__ __forceinline__ S c_entry(const EvalOut<S>& o, int t, int u) {
  if (t == 0) {
    const S base = o.fwd ? o.MQD[u] : o.MQi[u] - o.MQD[u];
    return u == 0 ? base + o.CovD : u == 1 ? base - o.CovD : base;
  }
  if (t == 1) {
    const S base = -(o.MQb[u] + o.MQi[u]);
    return u == 1 ? base + (o.CovS + o.CovD) : u == 0 ? base - o.CovD : u == 2 ? base - o.CovS : base;
  }
  if (t == 2) {
    const S base = o.fwd ? o.MQi[u] - o.MQD[u] : o.MQD[u];
    return u == 2 ? base + o.CovS : u == 1 ? base - o.CovS : base;
  }
  return o.MQb[u];
}
template <class S>
__device__ __forceinline__ S i_entry(const EvalOut<S>& o, int t) {
  if (t == 0) return o.Ichd - flip(o.Ijd, o.psb);
  if (t == 2) return -o.Ichd - flip(o.Ijs, o.psb);
  if (t == 3) return flip(o.Ijd + o.Ijs, o.psb);
  return S(0.0);
}

// Junction current and conductance: Ij(v) = Isat (explim(v/Vt) - 1) + GMIN v with
// explim(z) = exp(z) for z <= 40 and e^40 (1 + z - 40) above; gj = dIj/dv
// = (Isat/Vt) explim'(z) + GMIN, written as fma(Isat/Vt, expm1(z), Isat/Vt + GMIN). Deep in
// reverse bias (expm1 -> -1) the Isat/Vt e^z part of gj keeps an absolute error of about
// 1e-16 Isat/Vt, negligible beside GMIN (1e-12 S with the default cards).
template <class S>
__device__ __forceinline__ void junction(const CardK& c, const PrmS<S>& P, const S& v, S& Ij,
                                         S& gj) {
  const S z = v * c.inv_Vt;
  if (fm_le_pos(sval(z), kBits40)) {
    const S em1 = expm1_(z);
    Ij = P.Isat * em1 + c.GMIN * v;
    gj = P.IsatVt * em1 + P.IsatVtG;
  } else {
    const S em1 = expm1_(S(40.0));
    Ij = P.Isat * (em1 + (em1 + 1.0) * (z - 40.0)) + c.GMIN * v;
    gj = P.IsatVt * em1 + P.IsatVtG;
  }
}

// Terms that depend on vbs alone: body effect (2) and bulk-charge factor (4).
// phis = (u + R1)/2, R1 = sqrt(u^2 + 4 D1^2), u = PHI - vbs; d phis/du = phis/R1,
// d sqs/dvbs = -sqs/(2 R1). Vthb is the threshold without the DIBL term.
template <class S>
__device__ __forceinline__ void body_terms(const CardK& c, const S& vbs, S& sqs, S& Vthb,
                                           S& dVth_dvbs, S& Ab, S& dAb_dvbs) {
  const S u = c.PHI - vbs;
  const S R1sq = u * u + c.fourD1sq;
  const S inv_R1 = rsqrt_(R1sq);
  const S R1 = R1sq * inv_R1;
  S phis;
  if (fm_ge0(sval(u))) phis = half(u + R1);
  else phis = c.twoD1sq * rcp(R1 - u);
  const S inv_sqs = rsqrt_(phis);
  sqs = phis * inv_sqs;
  Vthb = c.K1 * sqs + c.Vthc;                     // VTH0 + K1 (sqs - sqrt(PHI))
  const S hK1R = c.halfK1 * inv_R1;
  dVth_dvbs = -(hK1R * sqs);
  Ab = c.halfK1 * inv_sqs + 1.0;
  dAb_dvbs = half(hK1R * inv_sqs);
}

// x-independent terms of a device whose source and body are both source-held: in forward mode
// vbs is constant, and the source junction is constant in either mode.
// Layout [kNBody][N] in this order; Qb = -Cox W L K1 sqs is the depletion charge.
struct BodyK {
  double sqs, Vthb, dVth_dvbs, Ab, dAb_dvbs, Ijs, gjs, Qb;
};

// Mode-frame channel current (steps 3, 5-8) and its gradient g = (gm, gds, gmb) with respect to
// (vgs, vds, vbs), given the vbs-dependent terms of step (2)/(4). Vg and F1 feed the charges.
template <class S>
struct Chan {
  S Ids, gm, gds, gmb, Vg, F1;
  S Vdsat, Vdseff, inv_Vdsat_parts[3];  // for the charge Jacobian: Dd, 1/EsatL, 1/Vgst2
  S sr;                                 // Vdseff / Vdsat = 2 vds / E (charge partition)
  S sig, F1_Vg, F1_Ab, F1_vds;          // for the charge Jacobian
  S Vdsat_Vg, Vdsat_Ab, Vde_Vg, Vde_Ab, Vde_vds;
};

// want_vbs = false skips the vbs (bulk-charge) derivative chain: gmb and the Ab partials come
// back zero. Callers pass false only when the S and b columns of the Jacobian are not stamped.
template <class S>
__device__ __forceinline__ void channel(const CardK& c, const PrmS<S>& P, const S& vgs,
                                        const S& vds, const S& Vthb, const S& dVth_dvbs,
                                        const S& Ab, const S& dAb_dvbs, Chan<S>& ch,
                                        bool want_vbs = true) {
  const S Vth = Vthb - c.ETA0 * vds;

  // (3) Vgsteff = nVt softplus(z), dVgsteff/dz = nVt sigmoid(z), z = (vgs - Vth) / nVt
  const S ov = vgs - Vth;
  const S z = ov * c.inv_nVt;
  const bool zpos = fm_ge0(sval(z));
  const S e = exp_(zpos ? -z : z);               // exp(-|z|)
  const S inv_1pe = rcp(1.0 + e);
  const S lg = log1p_(e, inv_1pe);
  const S Vg = c.nVt * lg + (zpos ? ov : S(0.0));  // nVt (z + lg) = ov + nVt lg for z >= 0
  const S sig = zpos ? inv_1pe : e * inv_1pe;

  // (5) mobility denominator, (6) velocity saturation
  const S den = 1.0 + Vg * (c.UA + c.UB * Vg);
  const S dden = c.twoUB * Vg + c.UA;
  const S Vgst2 = Vg + c.twoVt;
  const S EsatL = P.cE * den;
  const S Dd = Ab * EsatL + Vgst2;
  // one reciprocal for 1/den, 1/Vgst2 and 1/Dd: r = 1/(X Dd) with X = den Vgst2
  const S X = den * Vgst2;
  const S rXD = rcp(X * Dd);
  const S inv_pair = Dd * rXD;                    // 1 / (den Vgst2)
  const S inv_Dd = X * rXD;
  const S inv_den = Vgst2 * inv_pair;
  const S inv_Vgst2 = den * inv_pair;
  const S beta = P.beta0 * inv_den;
  const S inv_EsatL = P.inv_cE * inv_den;
  const S EsatL_Vg = P.cE * dden;
  const S r1 = Vgst2 * inv_Dd;
  const S r2 = EsatL * inv_Dd;
  const S Vdsat = EsatL * r1;
  const S Vdsat_Vg = r1 * r1 * EsatL_Vg + Ab * (r2 * r2);   // dVgst2/dVg = 1


  // (7) Vdseff = 2 Vdsat vds / (Vdsat + vds + DELTA + R2), R2 = sqrt(t^2 + 4 DELTA Vdsat)
  const S t = Vdsat - vds - c.DELTA;
  const S R2sq = t * t + c.fourDELTA * Vdsat;
  const S inv_R2 = rsqrt_(R2sq);
  const S R2 = R2sq * inv_R2;
  const S twoVdsat = twice(Vdsat);
  const S E = (twoVdsat - t) + R2;               // Vdsat + vds + DELTA + R2
  const S inv_E = rcp(E);
  const S twoVds = twice(vds);
  const S sr = twoVds * inv_E;                   // Vdseff / Vdsat (charge partition)
  const S Vdseff = Vdsat * sr;
  const S dE_dVdsat = 1.0 + (t + c.twoDELTA) * inv_R2;
  const S dE_dvds = 1.0 - t * inv_R2;
  const S Vde_Vdsat = (twoVds - Vdseff * dE_dVdsat) * inv_E;
  const S Vde_vds = (twoVdsat - Vdseff * dE_dvds) * inv_E;

  // (8) Ids = beta Vg Vdseff F1 F3 / F2
  const S h = half(inv_Vgst2);
  const S Abh = Ab * h;
  const S F1 = 1.0 - Abh * Vdseff;
  const S F2 = 1.0 + Vdseff * inv_EsatL;
  const S inv_F2 = rcp(F2);
  const S F3 = 1.0 + P.lamL * (vds - Vdseff);
  const S Pb = beta * Vg;
  const S F13 = F1 * F3;
  const S VF13 = Vdseff * F13;
  const S Ids = Pb * VF13 * inv_F2;

  // partial derivatives with Vg, Ab and vds as independent variables
  const S Vde_Vg = Vde_Vdsat * Vdsat_Vg;
  const S F1_Vg = -Abh * (Vde_Vg - Vdseff * inv_Vgst2);
  const S F1_vds = -Abh * Vde_vds;
  const S ddi = dden * inv_den;                  // d ln(den) / dVg
  const S F2_Vg = inv_EsatL * (Vde_Vg - Vdseff * ddi);
  const S F2_vds = inv_EsatL * Vde_vds;
  const S F3_Vg = -(P.lamL * Vde_Vg);
  const S F3_vds = P.lamL - P.lamL * Vde_vds;    // lamL (1 - dVdseff/dvds), one multiply-add
  const S Pb_Vg = beta - Pb * ddi;               // d(beta Vg)/dVg = beta (1 - Vg ddi)
  const S dV_Vg = Vde_Vg * F13 + Vdseff * (F1_Vg * F3 + F1 * F3_Vg);
  const S dV_vds = Vde_vds * F13 + Vdseff * (F1_vds * F3 + F1 * F3_vds);
  const S Ids_Vg = (Pb_Vg * VF13 + Pb * dV_Vg - Ids * F2_Vg) * inv_F2;
  const S Ids_vds = (Pb * dV_vds - Ids * F2_vds) * inv_F2;

  // chain to the mode-frame voltages: dVg/dvgs = sig, dVg/dvds = sig ETA0,
  // dVg/dvbs = -sig dVth/dvbs
  const S gm = Ids_Vg * sig;
  const S gds = gm * c.ETA0 + Ids_vds;
  // vbs chain through the bulk-charge factor, only when its columns are stamped
  S gmb = S(0.0), Vdsat_Ab = S(0.0), Vde_Ab = S(0.0), F1_Ab = S(0.0);
  if (want_vbs) {
    Vdsat_Ab = -(r2 * r2) * Vgst2;
    Vde_Ab = Vde_Vdsat * Vdsat_Ab;
    F1_Ab = -h * (Vdseff + Ab * Vde_Ab);
    const S F2_Ab = inv_EsatL * Vde_Ab;
    const S F3_Ab = -(P.lamL * Vde_Ab);
    const S dV_Ab = Vde_Ab * F13 + Vdseff * (F1_Ab * F3 + F1 * F3_Ab);
    const S Ids_Ab = (Pb * dV_Ab - Ids * F2_Ab) * inv_F2;
    gmb = Ids_Ab * dAb_dvbs - gm * dVth_dvbs;
  }

  ch.Ids = Ids;
  ch.gm = gm;
  ch.gds = gds;
  ch.gmb = gmb;
  ch.Vg = Vg;
  ch.F1 = F1;
  ch.Vdsat = Vdsat;
  ch.Vdseff = Vdseff;
  ch.inv_Vdsat_parts[0] = Dd;
  ch.inv_Vdsat_parts[1] = inv_EsatL;
  ch.inv_Vdsat_parts[2] = inv_Vgst2;
  ch.sr = sr;
  ch.sig = sig;
  ch.F1_Vg = F1_Vg;
  ch.F1_Ab = F1_Ab;
  ch.F1_vds = F1_vds;
  ch.Vdsat_Vg = Vdsat_Vg;
  ch.Vdsat_Ab = Vdsat_Ab;
  ch.Vde_Vg = Vde_Vg;
  ch.Vde_Ab = Vde_Ab;
  ch.Vde_vds = Vde_vds;
}

template <class S, bool WANT_Q, bool WANT_C = false>
__device__ __forceinline__ void ees_l1(const CardK& c, unsigned long long psb, const PrmS<S>& P,
                                       const S V[4], EvalOut<S>& o, bool sb_fixed = false,
                                       const BodyK* bk = nullptr) {
  // (1) mode
  const S vds0 = flip(V[0] - V[2], psb);
  const bool fwd = fm_ge0(sval(vds0));
  const S VD = fwd ? V[0] : V[2];
  const S VS = fwd ? V[2] : V[0];
  const S vgs = flip(V[1] - VS, psb);
  const S vds = flip(vds0, fwd ? 0ull : kSignBit);   // VD - VS in the polarity frame

  // (2) body effect, (4) bulk charge: precomputed when vbs cannot change
  S sqs, Vthb, dVth_dvbs, Ab, dAb_dvbs;
  if (sb_fixed && fwd) {
    sqs = S(bk->sqs);
    Vthb = S(bk->Vthb);
    dVth_dvbs = S(bk->dVth_dvbs);
    Ab = S(bk->Ab);
    dAb_dvbs = S(bk->dAb_dvbs);
  } else {
    body_terms<S>(c, flip(V[3] - VS, psb), sqs, Vthb, dVth_dvbs, Ab, dAb_dvbs);
  }
  Chan<S> ch;
  channel<S>(c, P, vgs, vds, Vthb, dVth_dvbs, Ab, dAb_dvbs, ch, !(sb_fixed && fwd));
  const S& Ids = ch.Ids;
  const S& gm = ch.gm;
  const S& gds = ch.gds;
  const S& gmb = ch.gmb;
  const S& Vg = ch.Vg;
  const S& F1 = ch.F1;
  const S gsum = gm + gds + gmb;

  // (9) channel current into physical d (into s is the negative), and its Jacobian row
  const S Ichd = flip(Ids, fwd ? psb : (psb ^ kSignBit));
  const S cdd = fwd ? gds : gsum;
  const S cdg = fwd ? gm : -gm;
  const S cds = fwd ? -gsum : -gds;
  const S cdb = fwd ? gmb : -gmb;

  // (10) junctions on the physical terminals
  S Ijd, gjd, Ijs, gjs;
  junction<S>(c, P, flip(V[3] - V[0], psb), Ijd, gjd);
  if (sb_fixed) {
    Ijs = S(bk->Ijs);
    gjs = S(bk->gjs);
  } else {
    junction<S>(c, P, flip(V[3] - V[2], psb), Ijs, gjs);
  }

  o.cdd = cdd;
  o.cdg = cdg;
  o.cds = cds;
  o.cdb = cdb;
  o.gjd = gjd;
  o.gjs = gjs;
  o.Ichd = Ichd;
  o.Ijd = Ijd;
  o.Ijs = Ijs;
  o.psb = psb;
#pragma unroll
  for (int t = 0; t < 4; ++t) o.I[t] = i_entry(o, t);
#pragma unroll
  for (int r = 0; r < 3; ++r)
#pragma unroll
    for (int u = 0; u < 4; ++u) o.G[r][u] = g_entry(o, r, u);

  if (WANT_Q) {
    // (11) charges: depletion, inversion partitioned to the mode drain by
    //      fD = 1/2 - (1/2 - XPART) Vdseff / Vdsat (continuous across the source/drain swap),
    //      overlaps
    const S Qb = (sb_fixed && fwd) ? S(bk->Qb) : -(P.Coxt * c.K1 * sqs);
    const S Qinv = -(P.Coxt * Vg * F1);
    const S sr = ch.sr;   // Vdseff / Vdsat
    const S fD = c.XPm * sr + 0.5;
    const S QD = fD * Qinv;
    const S QS = Qinv - QD;
    // overlaps: V1 - V2 and V1 - V0 are vgs and vgd in some order (polarity frame)
    const S vgd = flip(V[1] - VD, psb);
    const S Qovs = P.CovS * (fwd ? vgs : vgd);
    const S Qovd = P.CovD * (fwd ? vgd : vgs);
    const S Q0 = (fwd ? QD : QS) - Qovd;
    const S Q2 = (fwd ? QS : QD) - Qovs;
    o.Q[0] = flip(Q0, psb);
    o.Q[2] = flip(Q2, psb);
    o.Q[3] = flip(Qb, psb);
    o.Q[1] = flip(-(Q0 + Q2 + Qb), psb);              // the charges sum to zero
    if (WANT_C) {
      // (11') charge Jacobian. Mode-frame derivatives of Qinv = -Coxt Vg F1 and Qb, with
      // dVg/d(vgs, vds, vbs) = sig (1, ETA0, -dVth/dvbs) and the total derivatives of F1; mapped
      // to the physical terminals as for G (the polarity factors cancel). Columns sum to zero.
      const S Vg_vds = ch.sig * c.ETA0;
      const S F1_vgs = ch.F1_Vg * ch.sig;
      const S F1_vdsT = ch.F1_Vg * Vg_vds + ch.F1_vds;
      const S mC = -P.Coxt;
      const S Qi_vgs = mC * (ch.sig * F1 + Vg * F1_vgs);
      const S Qi_vds = mC * (Vg_vds * F1 + Vg * F1_vdsT);
      // partition fraction: sr = Vdseff / Vdsat with Vdsat(Vg, Ab), Vdseff(Vdsat, vds)
      // 1 / Vdsat = Dd / (EsatL Vgst2): both reciprocals are already at hand
      const S inv_Vdsat = ch.inv_Vdsat_parts[0] * ch.inv_Vdsat_parts[1] * ch.inv_Vdsat_parts[2];
      const S sr_Vg = (ch.Vde_Vg - sr * ch.Vdsat_Vg) * inv_Vdsat;
      const S sr_vds = ch.Vde_vds * inv_Vdsat;
      const double mx = c.XPm;                     // dfD / dsr
      const S fD_vgs = mx * (sr_Vg * ch.sig);
      const S fD_vds = mx * (sr_Vg * Vg_vds + sr_vds);
      const S QD_vgs = fD * Qi_vgs + Qinv * fD_vgs;
      const S QD_vds = fD * Qi_vds + Qinv * fD_vds;
      // vbs column: with source and body held, in forward mode, the body and source columns are
      // never stamped (both terminals are held), so their entries are left at zero
      S Qi_vbs = S(0.0), Qb_vbs = S(0.0), QD_vbs = S(0.0);
      if (!(sb_fixed && fwd)) {
        const S Vg_vbs = -(ch.sig * dVth_dvbs);
        const S F1_vbsT = ch.F1_Vg * Vg_vbs + ch.F1_Ab * dAb_dvbs;
        Qi_vbs = mC * (Vg_vbs * F1 + Vg * F1_vbsT);
        Qb_vbs = mC * dVth_dvbs;
        const S sr_Ab = (ch.Vde_Ab - sr * ch.Vdsat_Ab) * inv_Vdsat;
        const S fD_vbs = mx * (sr_Vg * Vg_vbs + sr_Ab * dAb_dvbs);
        QD_vbs = fD * Qi_vbs + Qinv * fD_vbs;
      }
      const int iD = fwd ? 0 : 2, iS = fwd ? 2 : 0;
      S MQi[4], MQb[4], MQD[4];
      MQi[1] = Qi_vgs;
      MQi[iD] = Qi_vds;
      MQi[3] = Qi_vbs;
      MQi[iS] = -(Qi_vgs + Qi_vds + Qi_vbs);
      MQD[1] = QD_vgs;
      MQD[iD] = QD_vds;
      MQD[3] = QD_vbs;
      MQD[iS] = -(QD_vgs + QD_vds + QD_vbs);
      MQb[1] = S(0.0);
      MQb[iD] = S(0.0);
      MQb[3] = Qb_vbs;
      MQb[iS] = -Qb_vbs;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        o.MQi[u] = MQi[u];
        o.MQD[u] = MQD[u];
        o.MQb[u] = MQb[u];
      }
      o.CovS = P.CovS;
      o.CovD = P.CovD;
      o.fwd = fwd;
#pragma unroll
      for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int u = 0; u < 4; ++u) o.C[t][u] = c_entry(o, t, u);
    }
  }
}

}  // namespace eec
