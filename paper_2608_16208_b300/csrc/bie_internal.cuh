// Internal device helpers of the B300 surface-BIE library.
//   * complex arithmetic on double2
//   * analytic surfaces r(t, th) with first and second derivatives, for real
//     theta and for complex theta (analytic continuation, Section 3.3)
//   * cancellation-free differences r(v) - r(u) by the straight-path line
//     integral of the first derivatives (Section 4, Remark), 16-point
//     Gauss-Legendre
//   * warp-cooperative mixed-radix (4, 2, 3, 5) Stockham FFT in shared memory
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/bie.h"

namespace bie {

constexpr double kPi = 3.141592653589793238462643383279502884;
constexpr double kTwoPi = 6.283185307179586476925286766559005768;
constexpr double kStableDelta = 0.06;  // |t - t_s| + |th - th_s| below which differences use the line integral
// ... or |r_s - r| below which they do: next to a pole (J ~ sin t -> 0) a whole ring of source
// angles is physically close to the target, and plain subtraction would cost tau_0 ~ kappa rho^2/2
// a relative error ~2 eps |r| / (kappa rho^2)
constexpr double kStableDist = 0.06;
constexpr double kRootTol = 1e-14;     // Newton stops when |dz| <= tol*b + 4e-16|z| (then one more step)
constexpr double kSeriesX = 0.5;       // alpha, beta by Taylor series when k rho < this
constexpr double kSmallB = 0.1;        // translated swapping for tau_3 when b < this
constexpr double kNearPhi = 0.05;      // |th_q - a| below which the translated remainder uses the stable sum
constexpr double kBCap = 4.0;          // roots farther than this from the real axis: (a0, kBCap)
constexpr double kForwardLimit = 7.0;  // A_m: forward difference recurrence when L*b <= this
constexpr double kMillerLog = 39.2;    // Miller start N = L + ceil(kMillerLog/(2b)) + 16

// ------------------------------------------------------------------ complex
struct cplx {
  double re, im;
};
__host__ __device__ __forceinline__ cplx C(double r, double i = 0.0) { return {r, i}; }
__host__ __device__ __forceinline__ cplx operator+(cplx a, cplx b) { return {a.re + b.re, a.im + b.im}; }
__host__ __device__ __forceinline__ cplx operator-(cplx a, cplx b) { return {a.re - b.re, a.im - b.im}; }
__host__ __device__ __forceinline__ cplx operator-(cplx a) { return {-a.re, -a.im}; }
__host__ __device__ __forceinline__ cplx operator*(cplx a, cplx b) {
  return {fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
}
__host__ __device__ __forceinline__ cplx operator*(double s, cplx a) { return {s * a.re, s * a.im}; }
__host__ __device__ __forceinline__ cplx operator*(cplx a, double s) { return {s * a.re, s * a.im}; }
__host__ __device__ __forceinline__ cplx conj(cplx a) { return {a.re, -a.im}; }
__host__ __device__ __forceinline__ double abs2(cplx a) { return a.re * a.re + a.im * a.im; }
__device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
  double d = 1.0 / (b.re * b.re + b.im * b.im);
  return {(a.re * b.re + a.im * b.im) * d, (a.im * b.re - a.re * b.im) * d};
}
__device__ __forceinline__ cplx cexpi(double x) {
  double s, c;
  sincos(x, &s, &c);
  return {c, s};
}
// cos and sin of a complex argument
__device__ __forceinline__ void ccossin(cplx z, cplx* c, cplx* s) {
  double sx, cx;
  sincos(z.re, &sx, &cx);
  double ch = cosh(z.im), sh = sinh(z.im);
  *c = {cx * ch, -sx * sh};
  *s = {sx * ch, cx * sh};
}
__device__ __forceinline__ cplx shfl(cplx v, int src) {
  return {__shfl_sync(0xffffffffu, v.re, src), __shfl_sync(0xffffffffu, v.im, src)};
}

// ------------------------------------------------------------------ surfaces
// 16-point Gauss-Legendre on [0, 1] (nodes and weights), filled by the host.
struct GL16 {
  double x[16], w[16];
};

struct SurfP {
  int kind;       // 0 ellipsoid, 1 star, 2 bean, 3 torus, 4 Fourier torus
  int nt;         // number of star / Fourier-torus terms
  int periodic;   // t-periodic (tori): the first and last panels are neighbours
  double L;       // parameter length of the generating curve (pi, or 2 pi for tori)
  double ax, ay, az;
  double R, eps;  // tori: R; the wiggly torus's eps and m (mm)
  int mm;
  double c[BIE_MAX_TERMS];
  int8_t p[BIE_MAX_TERMS], q[BIE_MAX_TERMS], m[BIE_MAX_TERMS], s[BIE_MAX_TERMS];   // Fourier torus: m, n in m, q
  GL16 gl;        // Gauss-Legendre on [0, 1] for the line-integral differences of kinds 2-4
};

template <typename T>
struct V3 {
  T x, y, z;
};
using R3 = V3<double>;
using C3 = V3<cplx>;

__device__ __forceinline__ double dot(const R3& a, const R3& b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ R3 cross(const R3& a, const R3& b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}

// sin^p cos^q and its first two t-derivatives
__device__ __forceinline__ double scpow(double st, double ct, int p, int q) {
  double v = 1.0;
  for (int i = 0; i < p; ++i) v *= st;
  for (int i = 0; i < q; ++i) v *= ct;
  return v;
}
__device__ __forceinline__ void scpow_d(double st, double ct, int p, int q, double* g, double* gt, double* gtt) {
  *g = scpow(st, ct, p, q);
  double d1 = 0.0, d2 = 0.0;
  if (p) d1 += p * scpow(st, ct, p - 1, q + 1);
  if (q) d1 -= q * scpow(st, ct, p + 1, q - 1);
  if (p) {
    if (p > 1) d2 += p * (p - 1) * scpow(st, ct, p - 2, q + 2);
    d2 -= p * (q + 1) * scpow(st, ct, p, q);
  }
  if (q) {
    d2 -= q * (p + 1) * scpow(st, ct, p, q);
    if (q > 1) d2 += q * (q - 1) * scpow(st, ct, p + 2, q - 2);
  }
  *gt = d1;
  *gtt = d2;
}

// Surface point and derivatives at real (t, th).  order: 0 -> r; 1 -> r, rt, rth;
// 2 -> also rtt, rtth, rthth.
struct Geo {
  R3 r, rt, rth, rtt, rtth, rthth;
};
// tsc: sin t, cos t when the caller holds them (a fixed t over many calls), else null
static __device__ __noinline__ void surf_eval(const SurfP& S, double t, double th, int order, Geo* g,
                                              const double2* tsc = nullptr) {
  double st, ct, sp, cp;
  if (tsc) {
    st = tsc->x;
    ct = tsc->y;
  } else {
    sincos(t, &st, &ct);
  }
  sincos(th, &sp, &cp);
  if (S.kind == 0) {
    g->r = {S.ax * st * cp, S.ay * st * sp, S.az * ct};
    if (order >= 1) {
      g->rt = {S.ax * ct * cp, S.ay * ct * sp, -S.az * st};
      g->rth = {-S.ax * st * sp, S.ay * st * cp, 0.0};
    }
    if (order >= 2) {
      g->rtt = {-S.ax * st * cp, -S.ay * st * sp, -S.az * ct};
      g->rtth = {-S.ax * ct * sp, S.ay * ct * cp, 0.0};
      g->rthth = {-S.ax * st * cp, -S.ay * st * sp, 0.0};
    }
    return;
  }
  if (S.kind == 2) {   // bean: r = (f_A(t) cos th, y0(t) + f_B(t) sin th, cos t)
    const double u = cos(kPi * ct), su = sin(kPi * ct);
    const double du = kPi * st * su, ddu = kPi * ct * su - (kPi * st) * (kPi * st) * u;
    double fa[3], fb[3];
    for (int which = 0; which < 2; ++which) {
      const double c0 = which ? 0.4 : 0.1;
      const double g = 1 - c0 * u, sg = sqrt(g), dg = -c0 * du, ddg = -c0 * ddu;
      const double dsg = dg / (2 * sg), ddsg = ddg / (2 * sg) - dg * dg / (4 * g * sg);
      double* f = which ? fb : fa;
      f[0] = 0.8 * sg * st;
      f[1] = 0.8 * (dsg * st + sg * ct);
      f[2] = 0.8 * (ddsg * st + 2 * dsg * ct - sg * st);
    }
    const double y0 = -0.3 * u, y0t = -0.3 * du, y0tt = -0.3 * ddu;
    g->r = {fa[0] * cp, y0 + fb[0] * sp, ct};
    if (order >= 1) {
      g->rt = {fa[1] * cp, y0t + fb[1] * sp, -st};
      g->rth = {-fa[0] * sp, fb[0] * cp, 0.0};
    }
    if (order >= 2) {
      g->rtt = {fa[2] * cp, y0tt + fb[2] * sp, -ct};
      g->rtth = {-fa[1] * sp, fb[1] * cp, 0.0};
      g->rthth = {-fa[0] * cp, -fb[0] * sp, 0.0};
    }
    return;
  }
  if (S.kind == 3) {   // torus: r = (a w cos t, b w sin t, c sin th), w = R + cos th + eps cos(m t)
    double smt, cmt;
    sincos(S.mm * t, &smt, &cmt);
    const double w = S.R + cp + S.eps * cmt, wt = -S.eps * S.mm * smt, wth = -sp;
    const double wtt = -S.eps * S.mm * S.mm * cmt, wthth = -cp;
    g->r = {S.ax * w * ct, S.ay * w * st, S.az * sp};
    if (order >= 1) {
      g->rt = {S.ax * (wt * ct - w * st), S.ay * (wt * st + w * ct), 0.0};
      g->rth = {S.ax * wth * ct, S.ay * wth * st, S.az * cp};
    }
    if (order >= 2) {
      g->rtt = {S.ax * (wtt * ct - 2 * wt * st - w * ct), S.ay * (wtt * st + 2 * wt * ct - w * st), 0.0};
      g->rtth = {-S.ax * wth * st, S.ay * wth * ct, 0.0};
      g->rthth = {S.ax * wthth * ct, S.ay * wthth * st, -S.az * sp};
    }
    return;
  }
  if (S.kind == 4) {   // Fourier torus: r = (w cos t, w sin t, zeta), w = R + sum c cos(m th + n t), zeta = sum c sin(.)
    double w = S.R, wt = 0, wth = 0, wtt = 0, wtth = 0, wthth = 0, z = 0, zt = 0, zh = 0, ztt = 0, zth = 0, zhh = 0;
    for (int i = 0; i < S.nt; ++i) {
      const double mm = S.m[i], nn = S.q[i], c = S.c[i];
      double sph, cph;
      sincos(mm * th + nn * t, &sph, &cph);
      w += c * cph; wt -= c * nn * sph; wth -= c * mm * sph;
      wtt -= c * nn * nn * cph; wtth -= c * mm * nn * cph; wthth -= c * mm * mm * cph;
      z += c * sph; zt += c * nn * cph; zh += c * mm * cph;
      ztt -= c * nn * nn * sph; zth -= c * mm * nn * sph; zhh -= c * mm * mm * sph;
    }
    g->r = {w * ct, w * st, z};
    if (order >= 1) {
      g->rt = {wt * ct - w * st, wt * st + w * ct, zt};
      g->rth = {wth * ct, wth * st, zh};
    }
    if (order >= 2) {
      g->rtt = {wtt * ct - 2 * wt * st - w * ct, wtt * st + 2 * wt * ct - w * st, ztt};
      g->rtth = {wtth * ct - wth * st, wtth * st + wth * ct, zth};
      g->rthth = {wthth * ct, wthth * st, zhh};
    }
    return;
  }
  double h = 1.0, ht = 0.0, hth = 0.0, htt = 0.0, htth = 0.0, hthth = 0.0;
  double sm = 0.0, cm = 1.0;
  for (int i = 0; i < S.nt; ++i) {
    double gg, gt, gtt;
    scpow_d(st, ct, S.p[i], S.q[i], &gg, &gt, &gtt);
    const double mm = S.m[i];
    if (i == 0 || S.m[i] != S.m[i - 1]) sincos(mm * th, &sm, &cm);   // reused along a run of equal m
    double T, Tth, Tthth;
    if (S.s[i] == 0) {
      T = cm; Tth = -mm * sm; Tthth = -mm * mm * cm;
    } else {
      T = sm; Tth = mm * cm; Tthth = -mm * mm * sm;
    }
    const double c = S.c[i];
    h += c * gg * T;
    ht += c * gt * T;
    hth += c * gg * Tth;
    htt += c * gtt * T;
    htth += c * gt * Tth;
    hthth += c * gg * Tthth;
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

// r, r_t, r_th at real t and complex th (analytic continuation in theta).
static __device__ __noinline__ void surf_eval_c(const SurfP& S, double t, cplx th, C3* r, C3* rt, C3* rth,
                                                const double2* tsc = nullptr) {
  double st, ct;
  if (tsc) {
    st = tsc->x;
    ct = tsc->y;
  } else {
    sincos(t, &st, &ct);
  }
  cplx cp, sp;
  ccossin(th, &cp, &sp);
  if (S.kind == 0) {
    *r = {S.ax * st * cp, S.ay * st * sp, C(S.az * ct)};
    *rt = {S.ax * ct * cp, S.ay * ct * sp, C(-S.az * st)};
    *rth = {-S.ax * st * sp, S.ay * st * cp, C(0.0)};
    return;
  }
  if (S.kind == 2) {   // bean (t real: every factor of t is real)
    const double u = cos(kPi * ct), su = sin(kPi * ct), du = kPi * st * su;
    double fa0, fa1, fb0, fb1;
    for (int which = 0; which < 2; ++which) {
      const double c0 = which ? 0.4 : 0.1;
      const double g = 1 - c0 * u, sg = sqrt(g), dsg = -c0 * du / (2 * sg);
      (which ? fb0 : fa0) = 0.8 * sg * st;
      (which ? fb1 : fa1) = 0.8 * (dsg * st + sg * ct);
    }
    *r = {fa0 * cp, C(-0.3 * u) + fb0 * sp, C(ct)};
    *rt = {fa1 * cp, C(-0.3 * du) + fb1 * sp, C(-st)};
    *rth = {-fa0 * sp, fb0 * cp, C(0.0)};
    return;
  }
  if (S.kind == 3) {   // torus
    double smt, cmt;
    sincos(S.mm * t, &smt, &cmt);
    const cplx w = C(S.R + S.eps * cmt) + cp;
    const double wt = -S.eps * S.mm * smt;
    const cplx wth = -sp;
    *r = {(S.ax * ct) * w, (S.ay * st) * w, S.az * sp};
    *rt = {S.ax * (C(wt * ct) - st * w), S.ay * (C(wt * st) + ct * w), C(0.0)};
    *rth = {(S.ax * ct) * wth, (S.ay * st) * wth, S.az * cp};
    return;
  }
  if (S.kind == 4) {   // Fourier torus
    cplx w = C(S.R), wt = C(0.0), wth = C(0.0), z = C(0.0), zt = C(0.0), zh = C(0.0);
    for (int i = 0; i < S.nt; ++i) {
      const double mm = S.m[i], nn = S.q[i], c = S.c[i];
      cplx cph, sph;
      ccossin(mm * th + C(nn * t), &cph, &sph);
      w = w + c * cph; wt = wt - (c * nn) * sph; wth = wth - (c * mm) * sph;
      z = z + c * sph; zt = zt + (c * nn) * cph; zh = zh + (c * mm) * cph;
    }
    *r = {ct * w, st * w, z};
    *rt = {ct * wt - st * w, st * wt + ct * w, zt};
    *rth = {ct * wth, st * wth, zh};
    return;
  }
  cplx h = C(1.0), ht = C(0.0), hth = C(0.0);
  cplx cm = C(1.0), sm = C(0.0);
  for (int i = 0; i < S.nt; ++i) {
    double gg, gt, gtt;
    scpow_d(st, ct, S.p[i], S.q[i], &gg, &gt, &gtt);
    const double mm = S.m[i];
    if (i == 0 || S.m[i] != S.m[i - 1]) ccossin(mm * th, &cm, &sm);   // reused along a run of equal m
    cplx T, Tth;
    if (S.s[i] == 0) {
      T = cm; Tth = -mm * sm;
    } else {
      T = sm; Tth = mm * cm;
    }
    h = h + (S.c[i] * gg) * T;
    ht = ht + (S.c[i] * gt) * T;
    hth = hth + (S.c[i] * gg) * Tth;
  }
  C3 e = {st * cp, st * sp, C(ct)};
  C3 et = {ct * cp, ct * sp, C(-st)};
  C3 eth = {-st * sp, st * cp, C(0.0)};
  *r = {h * e.x, h * e.y, h * e.z};
  *rt = {ht * e.x + h * et.x, ht * e.y + h * et.y, ht * e.z + h * et.z};
  *rth = {hth * e.x + h * eth.x, hth * e.y + h * eth.y, hth * e.z + h * eth.z};
}

constexpr double kInvTwoPi = 0.15915494309189533576888376337251436;
__device__ __forceinline__ double wrap_pi(double d) { return d - kTwoPi * rint(d * kInvTwoPi); }

// r(t_s, th_s) - r(t, th) for complex th_s by the line integral of the first
// derivatives along gamma(lam) = v + lam (u - v) (Section 4, Remark).
__device__ inline C3 path_difference_c(const SurfP& S, const GL16& gl, double ts, cplx ths, double t, double th) {
  const double dt = t - ts;
  cplx dth = C(wrap_pi(th - ths.re), -ths.im);
  C3 acc = {C(0), C(0), C(0)};
  for (int j = 0; j < 16; ++j) {
    C3 r, rt, rth;
    surf_eval_c(S, ts + gl.x[j] * dt, ths + gl.x[j] * dth, &r, &rt, &rth);
    const double w = gl.w[j];
    acc.x = acc.x + w * (dt * rt.x + rth.x * dth);
    acc.y = acc.y + w * (dt * rt.y + rth.y * dth);
    acc.z = acc.z + w * (dt * rt.z + rth.z * dth);
  }
  return {-acc.x, -acc.y, -acc.z};
}

// ------------------------------------------------------------------ FFT
// Twiddle table for length T (a multiple of every transform length used):
// tw[k] = e^{-2 pi i k / T}.  A length-n transform uses index k*(T/n).
struct FFTPlan {
  int n;
  int nst;
  int rad[16];
};

__host__ __device__ inline FFTPlan make_plan(int n) {
  FFTPlan p;
  p.n = n;
  p.nst = 0;
  int m = n;
  while (m % 4 == 0) { p.rad[p.nst++] = 4; m /= 4; }
  while (m % 2 == 0) { p.rad[p.nst++] = 2; m /= 2; }
  while (m % 3 == 0) { p.rad[p.nst++] = 3; m /= 3; }
  while (m % 5 == 0) { p.rad[p.nst++] = 5; m /= 5; }
  if (m != 1) p.nst = -1;
  return p;
}

// One stage per radix, each butterfly's inputs held in named registers (a runtime-indexed array
// would live in local memory); the stage index j = q Ns + jm by shift and mask when Ns is a power
// of two.  The twiddle index r jm T / (Ns R) stays below T.
__device__ __forceinline__ cplx tw64(const cplx* __restrict__ tw, int idx, int sign) {
  const double2 w2 = __ldg(reinterpret_cast<const double2*>(tw) + idx);
  return C(w2.x, sign > 0 ? -w2.y : w2.y);
}

// In-place (returns pointer to the buffer holding the result) transform of x[0..n)
// using y as scratch.  sign = -1: X_k = sum x_j e^{-2 pi i jk/n}; sign = +1: inverse
// (unnormalised).  Called by all 32 lanes of a warp.  st0 > 0: the first st0 stages are done (x
// holds their output).
static __device__ __noinline__ cplx* warp_fft(cplx* x, cplx* y, int n, const cplx* __restrict__ tw, int T, int sign,
                                              int st0 = 0) {
  const int lane = threadIdx.x & 31;
  const FFTPlan p = make_plan(n);
  cplx* src = x;
  cplx* dst = y;
  int Ns = 1;
  for (int st = 0; st < st0; ++st) Ns *= p.rad[st];
  const double s3 = 0.86602540378443864676 * sign;
  for (int st = st0; st < p.nst; ++st) {
    const int R = p.rad[st];
    const int stride = n / R;
    const int tstep = (T / n) * (n / (Ns * R));
    const int sh = (Ns & (Ns - 1)) == 0 ? __ffs(Ns) - 1 : -1;
    if (R == 4) {
      for (int j = lane; j < stride; j += 32) {
        const int jm = sh >= 0 ? (j & (Ns - 1)) : j % Ns;
        const int q = sh >= 0 ? (j >> sh) : j / Ns;
        cplx v0 = src[j], v1 = src[j + stride], v2 = src[j + 2 * stride], v3 = src[j + 3 * stride];
        if (jm) {
          v1 = v1 * tw64(tw, jm * tstep, sign);
          v2 = v2 * tw64(tw, 2 * jm * tstep, sign);
          v3 = v3 * tw64(tw, 3 * jm * tstep, sign);
        }
        const cplx s02 = v0 + v2, d02 = v0 - v2, s13 = v1 + v3, d13 = v1 - v3;
        const cplx jd = sign < 0 ? C(d13.im, -d13.re) : C(-d13.im, d13.re);   // sign i d13
        const int idx = q * Ns * 4 + jm;
        dst[idx] = s02 + s13;
        dst[idx + Ns] = d02 + jd;
        dst[idx + 2 * Ns] = s02 - s13;
        dst[idx + 3 * Ns] = d02 - jd;
      }
    } else if (R == 2) {
      for (int j = lane; j < stride; j += 32) {
        const int jm = sh >= 0 ? (j & (Ns - 1)) : j % Ns;
        const int q = sh >= 0 ? (j >> sh) : j / Ns;
        const cplx v0 = src[j];
        cplx v1 = src[j + stride];
        if (jm) v1 = v1 * tw64(tw, jm * tstep, sign);
        const int idx = q * Ns * 2 + jm;
        dst[idx] = v0 + v1;
        dst[idx + Ns] = v0 - v1;
      }
    } else if (R == 5) {
      // DFT of length 5: cos and sin of 2 pi / 5 and 4 pi / 5
      const double c1 = 0.30901699437494742, c2 = -0.80901699437494742;
      const double s1 = 0.95105651629515357 * sign, s2 = 0.58778525229247313 * sign;
      for (int j = lane; j < stride; j += 32) {
        const int jm = sh >= 0 ? (j & (Ns - 1)) : j % Ns;
        const int q = sh >= 0 ? (j >> sh) : j / Ns;
        const cplx v0 = src[j];
        cplx v1 = src[j + stride], v2 = src[j + 2 * stride], v3 = src[j + 3 * stride], v4 = src[j + 4 * stride];
        if (jm) {
          v1 = v1 * tw64(tw, jm * tstep, sign);
          v2 = v2 * tw64(tw, 2 * jm * tstep, sign);
          v3 = v3 * tw64(tw, 3 * jm * tstep, sign);
          v4 = v4 * tw64(tw, 4 * jm * tstep, sign);
        }
        const cplx t1 = v1 + v4, t2 = v2 + v3, t3 = v1 - v4, t4 = v2 - v3;
        const cplx a1 = v0 + c1 * t1 + c2 * t2, a2 = v0 + c2 * t1 + c1 * t2;
        const cplx b1 = s1 * t3 + s2 * t4, b2 = s2 * t3 - s1 * t4;   // times i below
        const int idx = q * Ns * 5 + jm;
        dst[idx] = v0 + t1 + t2;
        dst[idx + Ns] = a1 + C(-b1.im, b1.re);
        dst[idx + 4 * Ns] = a1 - C(-b1.im, b1.re);
        dst[idx + 2 * Ns] = a2 + C(-b2.im, b2.re);
        dst[idx + 3 * Ns] = a2 - C(-b2.im, b2.re);
      }
    } else {
      for (int j = lane; j < stride; j += 32) {
        const int jm = sh >= 0 ? (j & (Ns - 1)) : j % Ns;
        const int q = sh >= 0 ? (j >> sh) : j / Ns;
        const cplx v0 = src[j];
        cplx v1 = src[j + stride], v2 = src[j + 2 * stride];
        if (jm) {
          v1 = v1 * tw64(tw, jm * tstep, sign);
          v2 = v2 * tw64(tw, 2 * jm * tstep, sign);
        }
        const cplx t1 = v1 + v2, d = v1 - v2;
        const cplx t2 = C(-s3 * d.im, s3 * d.re);
        const cplx base = v0 - 0.5 * t1;
        const int idx = q * Ns * 3 + jm;
        dst[idx] = v0 + t1;
        dst[idx + Ns] = base + t2;
        dst[idx + 2 * Ns] = base - t2;
      }
    }
    __syncwarp();
    cplx* tmp = src;
    src = dst;
    dst = tmp;
    Ns *= R;
  }
  return src;
}

}  // namespace bie

// Opaque handles (host side)
// kernel families timed by the context's launch trace (bie_ctx_trace)
enum { kTracePairRoot = 0, kTracePairTransform = 1, kTracePairFused = 2, kTraceNearFill = 3, kTraceFarFill = 4,
       kTraceKinds = 5 };
struct TraceMark {
  int kind;
  cudaEvent_t e0, e1;
};
struct bie_ctx_s {
  cudaStream_t stream;
  int device;
  int sms;
  int* d_status;       // device status word (error flags from kernels)
  int trace = 0;       // record CUDA events around the pair, near-fill and far-fill launches
  int fp64_transforms = 0;   // BIE_OPT_FP64_TRANSFORMS
  std::vector<TraceMark>* marks = nullptr;
  // pair-pipeline work buffers of this context (grown on demand, freed by bie_ctx_free): the
  // per-warp recurrence scratch of the fused kernels and the per-pair records of the split launch
  double* pair_scratch = nullptr;
  size_t pair_scratch_bytes = 0;
  double* pair_records = nullptr;
  size_t pair_records_bytes = 0;
  // the O(M) route's per-warp rows of U (grown on demand)
  void* band_scratch = nullptr;
  size_t band_scratch_bytes = 0;
};

struct bie_surface_s {
  bie_ctx ctx;
  bie::SurfP sp;
  int Np, Mt;
  double L, h;
  int64_t N, n_rings;
  double* t_nodes;     // [dev] [16 Np]
  double* pts;         // [dev] [N][3]
  double* nrm;         // [dev] [N][3]
  double* jac;         // [dev] [N]
  double* ring_t;      // [dev] [n_rings]
  double* ring_r;      // [dev] [n_rings][Mt][3]
  double* ring_n;      // [dev] [n_rings][Mt][3]
  double* near_coef;   // [dev] [3][16][16][16] = w_g L_n(x_g) on the reference panel
  float2* near_coef_dw;  // [dev] the same as double words
  double* ggq_x;       // [dev] [3][16][16]
  bie::cplx* tw;       // [dev] twiddles for length 12 Mt
  float4* twf;         // [dev] the same twiddles as double words (re.h, re.l, im.h, im.l)
  double* thgrid;      // [dev] [Mt][3]: th_q = 2 pi q / Mt, sin(th_q/2), cos(th_q/2)
  int tw_len;
  double* host_t_nodes;
  double gl_x[16], gl_w[16];   // Gauss-Legendre rule on [-1, 1] from the caller's tables
  bie::GL16 gl01;              // the same rule mapped to [0, 1]
};

struct bie_net_infer_s;

namespace bie {
// launch trace: trace_begin returns an index (or -1 when tracing is off), trace_end records the end
int trace_begin(bie_ctx ctx, int kind);
void trace_end(bie_ctx ctx, int mark);
void set_error(const char* fmt, ...);
bie_status cuda_fail(cudaError_t e, const char* where);
// BIE_OK if the context's device is the current one, else BIE_EINVAL naming the call
bie_status check_device(bie_ctx ctx, const char* where);
// near fill of one target panel of s into a band buffer from weights in a ring of pair rows
bie_status near_fill_ring(bie_surface s, int jpanel, const bie::cplx* W, int64_t pbase, int64_t ring, int w_ld,
                          bie::cplx* band, cudaStream_t st);
// preconditioners (blockdiag.cu, precond_net.cu)
bie_status blockdiag_apply_dev(bie_blockdiag P, const double2* r, int nv, double2* z);
bie_status blockdiag_apply_f32(bie_blockdiag P, const float2* r, int nv, float2* z);
bie_net_infer_s* net_infer_new();
void net_infer_free(bie_net_infer_s* I);
bie_status net_precond_apply_dev(bie_net net, bie_net_infer_s* I, bie_blockdiag block, bie_surface s, double k,
                                 const double2* v, int nv, double2* z);
}  // namespace bie
