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

}  // namespace bie
