// Cancellation-free differences r(t_s, th_s) - r(t, th) of the surface kinds, with th_s real or
// complex (Section 4, Remark): closed forms by sum-to-product identities for the ellipsoid and the
// star, the straight-path line integral of the first derivatives for the other kinds.  Shared by the
// pair pipeline and the O(M) route.
#pragma once
#include "bie_internal.cuh"

namespace bie {

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------------ generic trig for real / complex
__device__ __forceinline__ void trig(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ void trig(cplx z, cplx* s, cplx* c) { ccossin(z, c, s); }
__device__ __forceinline__ double re_of(double v) { return v; }
__device__ __forceinline__ double re_of(cplx v) { return v.re; }
__device__ __forceinline__ double shift_by(double v, double s) { return v - s; }
__device__ __forceinline__ cplx shift_by(cplx v, double s) { return C(v.re - s, v.im); }
template <typename T>
__device__ __forceinline__ T mk(double v);
template <>
__device__ __forceinline__ double mk<double>(double v) { return v; }
template <>
__device__ __forceinline__ cplx mk<cplx>(double v) { return C(v); }
__device__ __forceinline__ double ipow(double x, int n) {
  double r = 1.0;
  for (int i = 0; i < n; ++i) r *= x;
  return r;
}

// r(t_s, ths) - r(t, th) by the line integral of the first derivatives along the straight parameter
// path (Section 4, Remark), 16-point Gauss-Legendre: the cancellation-free difference of the surface
// kinds without a closed form below (bean, tori); ths real or complex.
__device__ __forceinline__ void first_derivs(const SurfP& S, double t, double th, R3* rt, R3* rth) {
  Geo G;
  surf_eval(S, t, th, 1, &G);
  *rt = G.rt;
  *rth = G.rth;
}
__device__ __forceinline__ void first_derivs(const SurfP& S, double t, cplx th, C3* rt, C3* rth) {
  C3 r;
  surf_eval_c(S, t, th, &r, rt, rth);
}
__device__ __forceinline__ double wrapped_dth(double th, double ths) { return wrap_pi(th - ths); }
__device__ __forceinline__ cplx wrapped_dth(double th, cplx ths) { return C(wrap_pi(th - ths.re), -ths.im); }
template <typename T>
__device__ __noinline__ V3<T> diff_path(const SurfP& S, double ts, T ths, double t, double th) {
  const double dt = t - ts;
  const T dth = wrapped_dth(th, ths);
  V3<T> acc = {mk<T>(0.0), mk<T>(0.0), mk<T>(0.0)};
  for (int j = 0; j < 16; ++j) {
    const double lam = S.gl.x[j], w = S.gl.w[j];
    V3<T> rt, rth;
    first_derivs(S, ts + lam * dt, ths + lam * dth, &rt, &rth);
    acc.x = acc.x + w * (dt * rt.x + rth.x * dth);
    acc.y = acc.y + w * (dt * rt.y + rth.y * dth);
    acc.z = acc.z + w * (dt * rt.z + rth.z * dth);
  }
  return {-1.0 * acc.x, -1.0 * acc.y, -1.0 * acc.z};
}

// r(t_s, ths) - r(t, th) without cancellation (sum-to-product identities); ths real or complex.
template <typename T>
__device__ __noinline__ V3<T> diff_ana(const SurfP& S, double ts, T ths, double t, double th) {
  if (S.kind >= 2) return diff_path<T>(S, ts, ths, t, th);
  double s1, c1, s0, c0, smt, cmt;
  sincos(ts, &s1, &c1);
  sincos(t, &s0, &c0);
  sincos(0.5 * (ts + t), &smt, &cmt);
  const double sdt = sin(0.5 * (ts - t));
  const double dS = 2 * cmt * sdt;    // sin t_s - sin t
  const double dC = -2 * smt * sdt;   // cos t_s - cos t
  const double n2pi = kTwoPi * rint((re_of(ths) - th) / kTwoPi);
  const T del = shift_by(ths, th + n2pi);        // wrapped th_s - th
  const T mid = shift_by(0.5 * del, -th);        // th + del/2
  T sp, cp, sm, cm, sd, cdum;
  trig(ths, &sp, &cp);
  trig(mid, &sm, &cm);
  trig(0.5 * del, &sd, &cdum);
  const T dCos = -2.0 * (sm * sd);   // cos th_s - cos th
  const T dSin = 2.0 * (cm * sd);    // sin th_s - sin th
  if (S.kind == 0) {
    return {S.ax * (dS * cp + s0 * dCos), S.ay * (dS * sp + s0 * dSin), mk<T>(S.az * dC)};
  }
  // star: r = h e;  r_s - r = h_s (e_s - e) + (h_s - h) e
  const V3<T> de = {dS * cp + s0 * dCos, dS * sp + s0 * dSin, mk<T>(dC)};
  T hs = mk<T>(1.0), dh = mk<T>(0.0);
  T smm = mk<T>(0.0), cmm = mk<T>(1.0), sdm = mk<T>(0.0), cdm2 = mk<T>(1.0), smid = mk<T>(0.0), cmid = mk<T>(1.0);
  for (int i = 0; i < S.nt; ++i) {
    const int p = S.p[i], q = S.q[i];
    const double mm = S.m[i];
    double sp_sum = 0.0, cq_sum = 0.0;   // (s1^p - s0^p)/dS and (c1^q - c0^q)/dC
    for (int j = 0; j < p; ++j) sp_sum += ipow(s1, j) * ipow(s0, p - 1 - j);
    for (int j = 0; j < q; ++j) cq_sum += ipow(c1, j) * ipow(c0, q - 1 - j);
    const double g1 = ipow(s1, p) * ipow(c1, q), g0 = ipow(s0, p) * ipow(c0, q);
    const double dg = dS * sp_sum * ipow(c1, q) + ipow(s0, p) * dC * cq_sum;
    if (i == 0 || S.m[i] != S.m[i - 1]) {   // reused along a run of equal m
      trig(mm * ths, &smm, &cmm);
      trig(mm * mid, &smid, &cmid);
      trig((0.5 * mm) * del, &sdm, &cdm2);
    }
    T Ts, dT;
    if (S.s[i] == 0) {
      Ts = cmm;
      dT = -2.0 * (smid * sdm);
    } else {
      Ts = smm;
      dT = 2.0 * (cmid * sdm);
    }
    hs = hs + (S.c[i] * g1) * Ts;
    dh = dh + (S.c[i] * dg) * Ts + (S.c[i] * g0) * dT;
  }
  double st, ct;
  sincos(th, &st, &ct);
  const double ex = s0 * ct, ey = s0 * st, ez = c0;
  return {hs * de.x + ex * dh, hs * de.y + ey * dh, hs * de.z + ez * dh};
}

// ------------------------------------------------------------------ stars with a per-pair table
// The Newton iterations of one pair evaluate the star at its source ring's t_s and at its target many
// times.  The factors of each term that depend on t only, multiplied by the term's coefficient exactly
// as the evaluations above multiply them, are taken once per pair into a table in local memory; the
// evaluations below read them and perform the same remaining operations, so they return the same
// values bit for bit.  Stars with more than kStarTabTerms terms take the direct evaluations.
constexpr int kStarTabTerms = 40;
struct StarTab {
  double s0, c0, dS, dC, sth, cth;       // sin t, cos t, sin t_s - sin t, cos t_s - cos t, target theta
  double st, ct;                         // sin t_s, cos t_s
  double v[6 * kStarTabTerms];           // per term: c gg, c gt, c gtt (at t_s), c g1, c dg, c g0
};

static __device__ __noinline__ void star_tab_fill(const SurfP& S, double ts, double t, double th, StarTab* tb) {
  double s1, c1, s0, c0, smt, cmt;
  sincos(ts, &s1, &c1);
  sincos(t, &s0, &c0);
  sincos(0.5 * (ts + t), &smt, &cmt);
  const double sdt = sin(0.5 * (ts - t));
  const double dS = 2 * cmt * sdt;    // sin t_s - sin t
  const double dC = -2 * smt * sdt;   // cos t_s - cos t
  tb->s0 = s0;
  tb->c0 = c0;
  tb->dS = dS;
  tb->dC = dC;
  sincos(th, &tb->sth, &tb->cth);
  tb->st = s1;
  tb->ct = c1;
  for (int i = 0; i < S.nt; ++i) {
    double gg, gt, gtt;
    scpow_d(s1, c1, S.p[i], S.q[i], &gg, &gt, &gtt);
    const double c = S.c[i];
    tb->v[6 * i + 0] = c * gg;
    tb->v[6 * i + 1] = c * gt;
    tb->v[6 * i + 2] = c * gtt;
    const int p = S.p[i], q = S.q[i];
    double sp_sum = 0.0, cq_sum = 0.0;
    for (int j = 0; j < p; ++j) sp_sum += ipow(s1, j) * ipow(s0, p - 1 - j);
    for (int j = 0; j < q; ++j) cq_sum += ipow(c1, j) * ipow(c0, q - 1 - j);
    const double g1 = ipow(s1, p) * ipow(c1, q), g0 = ipow(s0, p) * ipow(c0, q);
    const double dg = dS * sp_sum * ipow(c1, q) + ipow(s0, p) * dC * cq_sum;
    tb->v[6 * i + 3] = S.c[i] * g1;
    tb->v[6 * i + 4] = S.c[i] * dg;
    tb->v[6 * i + 5] = S.c[i] * g0;
  }
}

// surf_eval at (t_s, th) of a star from the table
static __device__ __noinline__ void surf_eval_star_tab(const SurfP& S, const StarTab& tb, double th, int order, Geo* g) {
  const double st = tb.st, ct = tb.ct;
  double sp, cp;
  sincos(th, &sp, &cp);
  double h = 1.0, ht = 0.0, hth = 0.0, htt = 0.0, htth = 0.0, hthth = 0.0;
  double sm = 0.0, cm = 1.0;
  for (int i = 0; i < S.nt; ++i) {
    const double mm = S.m[i];
    if (i == 0 || S.m[i] != S.m[i - 1]) sincos(mm * th, &sm, &cm);
    double T, Tth, Tthth;
    if (S.s[i] == 0) {
      T = cm; Tth = -mm * sm; Tthth = -mm * mm * cm;
    } else {
      T = sm; Tth = mm * cm; Tthth = -mm * mm * sm;
    }
    const double cgg = tb.v[6 * i], cgt = tb.v[6 * i + 1], cgtt = tb.v[6 * i + 2];
    h += cgg * T;
    ht += cgt * T;
    hth += cgg * Tth;
    htt += cgtt * T;
    htth += cgt * Tth;
    hthth += cgg * Tthth;
  }
  R3 e = {st * cp, st * sp, ct};
  R3 et = {ct * cp, ct * sp, -st};
  R3 eth = {-st * sp, st * cp, 0.0};
  g->r = {h * e.x, h * e.y, h * e.z};
  if (order >= 1) {
    g->rt = {ht * e.x + h * et.x, ht * e.y + h * et.y, ht * e.z + h * et.z};
    g->rth = {hth * e.x + h * eth.x, hth * e.y + h * eth.y, hth * e.z + h * eth.z};
  }
  if (order >= 2) {
    R3 etth = {-ct * sp, ct * cp, 0.0};
    R3 ethth = {-st * cp, -st * sp, 0.0};
    g->rtt = {htt * e.x + 2 * ht * et.x - h * e.x, htt * e.y + 2 * ht * et.y - h * e.y,
              htt * e.z + 2 * ht * et.z - h * e.z};
    g->rtth = {htth * e.x + ht * eth.x + hth * et.x + h * etth.x, htth * e.y + ht * eth.y + hth * et.y + h * etth.y,
               htth * e.z + ht * eth.z + hth * et.z + h * etth.z};
    g->rthth = {hthth * e.x + 2 * hth * eth.x + h * ethth.x, hthth * e.y + 2 * hth * eth.y + h * ethth.y,
                hthth * e.z + 2 * hth * eth.z + h * ethth.z};
  }
}

// surf_eval_c at (t_s, complex th) of a star from the table
static __device__ __noinline__ void surf_eval_c_star_tab(const SurfP& S, const StarTab& tb, cplx th, C3* r, C3* rt, C3* rth) {
  const double st = tb.st, ct = tb.ct;
  cplx cp, sp;
  ccossin(th, &cp, &sp);
  cplx h = C(1.0), ht = C(0.0), hth = C(0.0);
  cplx cm = C(1.0), sm = C(0.0);
  for (int i = 0; i < S.nt; ++i) {
    const double mm = S.m[i];
    if (i == 0 || S.m[i] != S.m[i - 1]) ccossin(mm * th, &cm, &sm);
    cplx T, Tth;
    if (S.s[i] == 0) {
      T = cm; Tth = -mm * sm;
    } else {
      T = sm; Tth = mm * cm;
    }
    h = h + tb.v[6 * i] * T;
    ht = ht + tb.v[6 * i + 1] * T;
    hth = hth + tb.v[6 * i] * Tth;
  }
  C3 e = {st * cp, st * sp, C(ct)};
  C3 et = {ct * cp, ct * sp, C(-st)};
  C3 eth = {-st * sp, st * cp, C(0.0)};
  *r = {h * e.x, h * e.y, h * e.z};
  *rt = {ht * e.x + h * et.x, ht * e.y + h * et.y, ht * e.z + h * et.z};
  *rth = {hth * e.x + h * eth.x, hth * e.y + h * eth.y, hth * e.z + h * eth.z};
}

// diff_ana of a star at (t_s, ths) against the pair's target, from the table
template <typename T>
__device__ __noinline__ V3<T> diff_star_tab(const SurfP& S, const StarTab& tb, T ths, double th) {
  const double s0 = tb.s0, c0 = tb.c0, dS = tb.dS, dC = tb.dC;
  const double n2pi = kTwoPi * rint((re_of(ths) - th) / kTwoPi);
  const T del = shift_by(ths, th + n2pi);        // wrapped th_s - th
  const T mid = shift_by(0.5 * del, -th);        // th + del/2
  T sp, cp, sm, cm, sd, cdum;
  trig(ths, &sp, &cp);
  trig(mid, &sm, &cm);
  trig(0.5 * del, &sd, &cdum);
  const T dCos = -2.0 * (sm * sd);   // cos th_s - cos th
  const T dSin = 2.0 * (cm * sd);    // sin th_s - sin th
  const V3<T> de = {dS * cp + s0 * dCos, dS * sp + s0 * dSin, mk<T>(dC)};
  T hs = mk<T>(1.0), dh = mk<T>(0.0);
  T smm = mk<T>(0.0), cmm = mk<T>(1.0), sdm = mk<T>(0.0), cdm2 = mk<T>(1.0), smid = mk<T>(0.0), cmid = mk<T>(1.0);
  for (int i = 0; i < S.nt; ++i) {
    const double mm = S.m[i];
    if (i == 0 || S.m[i] != S.m[i - 1]) {
      trig(mm * ths, &smm, &cmm);
      trig(mm * mid, &smid, &cmid);
      trig((0.5 * mm) * del, &sdm, &cdm2);
    }
    T Ts, dT;
    if (S.s[i] == 0) {
      Ts = cmm;
      dT = -2.0 * (smid * sdm);
    } else {
      Ts = smm;
      dT = 2.0 * (cmid * sdm);
    }
    hs = hs + tb.v[6 * i + 3] * Ts;
    dh = dh + tb.v[6 * i + 4] * Ts + tb.v[6 * i + 5] * dT;
  }
  const double ex = s0 * tb.cth, ey = s0 * tb.sth, ez = c0;
  return {hs * de.x + ex * dh, hs * de.y + ey * dh, hs * de.z + ez * dh};
}

}  // namespace bie
