// Per-pair pipeline of the correction stage (Sections 3.2-3.4, 4): for a target
// node x = r(t_j^l, th_i) and a GGQ source ring t_s, the theta_s-Fourier modes
// of the single-layer kernel e^{ik rho}/rho (Eq. (Sphi:appr2)) and of the
// double-layer kernel alpha tau_1 - tau_3 - i beta tau_0 (Eq. (dis:K)) by
// singularity swapping, and their Parseval weights on the theta grid.
//
// A warp takes a batch of up to 32 pairs:
//   A. (warp per pair)  rho^2 on the ring, grid minimiser (near-ties to the
//      sample nearest the target angle, then the lower index).
//   B. (lane per pair)  real Newton for the minimiser a0, b0 = sqrt(2 rho^2 /
//      rho^2''), complex Newton for the root theta_+ = a + ib of rho^2
//      continued to complex theta (Section 3.3); roots beyond kBCap become
//      (a0, kBCap).  Differences r(t_s, zeta) - r(t, th) near the target are
//      written in closed form without cancellation (sum-to-product).
//   C. (lane per pair)  A_m(b), m = 0..L (Eq. (Am)): closed forms A_0, A_1 by
//      the AGM, then the difference recurrence (Eq. (diff-recurrence)) if
//      L b <= 7, else Miller's backward recurrence normalised by A_0; written
//      to the warp's global scratch slice with D_m = A_m - A_{m-1}.
//   D. (warp per pair)  smooth factors on the grid (F = (s_{a,b}/rho^2)^{1/2},
//      Eq. (F-smooth); cos(k rho); tau_0 (second-derivative line integral of
//      the Section 4 Remark near the target), alpha, beta tau_0, H3 = tau_0 F^3),
//      packed complex FFTs of length Mth, the trigonometric interpolants
//      multiplied on a grid of P points shifted by a, and the singular
//      convolutions (Eqs. (convolution), (tau1), (tau3-standard),
//      (tau3-modified)) as Toeplitz products with the circulants A_{|d|},
//      B_{|d|} (or B~_{|d|}) through shared-memory FFTs of length P
//      (P = 3 Mth for S alone, 4 Mth with K).  Modes |m| <= M are exact
//      linear-convolution values.  Parseval weights: the swapped part through
//      an inverse FFT (Nyquist split evenly), the smooth part (i sin(k rho)/rho,
//      -i beta tau_0) by the trapezoid rule (Section 3.2).
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "bie_internal.cuh"
#include "dw.cuh"
#include "pair_args.cuh"
#include "surf_diff.cuh"

namespace bie {

constexpr int kMaxWarpsPerBlock = 4;
constexpr size_t kSmemLimit = 227 * 1024;

// ------------------------------------------------------------------ AGM (DLMF 19.8.1, 19.8.6)
__device__ inline void ellipke(double m, double m1, double* K, double* E) {
  double a = 1.0, g = sqrt(m1), c2sum = 0.5 * m, scale = 0.5;
  for (int it = 0; it < 40; ++it) {
    const double an = 0.5 * (a + g), cn = 0.5 * (a - g);
    g = sqrt(a * g);
    a = an;
    scale *= 2.0;
    c2sum += scale * cn * cn;
    if (fabs(cn) <= 1e-17 * a) break;
  }
  *K = kPi / (2 * a);
  *E = *K * (1.0 - c2sum);
}

// Exponent e (|e| <= 60) with 2^e close to rms(x) / rms(y), from the warp-summed squares sx, sy; 0 when
// either part is zero.  Two real signals packed in one complex transform each come out with an error
// in proportion to the larger of the two: the smaller is multiplied by this exact power of two before
// packing and divided by it after.
__device__ __forceinline__ int pack_exponent(double sx, double sy) {
  if (!(sx > 0.0) || !(sy > 0.0)) return 0;
  const int e = (int)rint(0.5 * log2(sx / sy));
  return max(-60, min(60, e));
}

// ------------------------------------------------------------------ phase B: root (one lane)
struct PairInfo {
  int64_t row, ring;
  double t, th, ts, x, y, z;
  double a, b, a0;
  double qb, om, sha, cha;   // e^{-b}, 1 - e^{-b}, sin(a/2), cos(a/2) (set with the root)
  int valid, bi, capped, pad;
};

// the batch info lives in registers (lane p holds pair p); a pass over the batch broadcasts it
__device__ __forceinline__ PairInfo bcast(const PairInfo& p, int src) {
  PairInfo o;
  o.row = __shfl_sync(0xffffffffu, (long long)p.row, src);
  o.ring = __shfl_sync(0xffffffffu, (long long)p.ring, src);
  o.t = __shfl_sync(0xffffffffu, p.t, src);
  o.th = __shfl_sync(0xffffffffu, p.th, src);
  o.ts = __shfl_sync(0xffffffffu, p.ts, src);
  o.x = __shfl_sync(0xffffffffu, p.x, src);
  o.y = __shfl_sync(0xffffffffu, p.y, src);
  o.z = __shfl_sync(0xffffffffu, p.z, src);
  o.a = __shfl_sync(0xffffffffu, p.a, src);
  o.b = __shfl_sync(0xffffffffu, p.b, src);
  o.a0 = __shfl_sync(0xffffffffu, p.a0, src);
  o.qb = __shfl_sync(0xffffffffu, p.qb, src);
  o.om = __shfl_sync(0xffffffffu, p.om, src);
  o.sha = __shfl_sync(0xffffffffu, p.sha, src);
  o.cha = __shfl_sync(0xffffffffu, p.cha, src);
  o.valid = __shfl_sync(0xffffffffu, p.valid, src);
  o.bi = __shfl_sync(0xffffffffu, p.bi, src);
  o.capped = __shfl_sync(0xffffffffu, p.capped, src);
  o.pad = 0;
  return o;
}

// tb: the pair's star table (stars with at most kStarTabTerms terms), or null
__device__ inline void rho2_cplx(const SurfP& S, const PairInfo& P, const StarTab* tb, const double2* tsc, cplx z,
                                 cplx* f, cplx* df) {
  C3 r, rt, rth;
  if (tb) surf_eval_c_star_tab(S, *tb, z, &r, &rt, &rth);
  else surf_eval_c(S, P.ts, z, &r, &rt, &rth, tsc);
  C3 Y = {r.x - C(P.x), r.y - C(P.y), r.z - C(P.z)};
  const bool near = fabs(P.ts - P.t) + fabs(wrap_pi(z.re - P.th)) <= kStableDelta ||
                    abs2(Y.x) + abs2(Y.y) + abs2(Y.z) <= kStableDist * kStableDist;
  if (near) Y = tb ? diff_star_tab<cplx>(S, *tb, z, P.th) : diff_ana<cplx>(S, P.ts, z, P.t, P.th);
  *f = Y.x * Y.x + Y.y * Y.y + Y.z * Y.z;
  *df = 2.0 * (Y.x * rth.x + Y.y * rth.y + Y.z * rth.z);
}

__device__ __noinline__ void locate_root(const SurfP& S, int Mt, PairInfo& P) {
  const double hgrid = kTwoPi / Mt;
  double a0 = kTwoPi * P.bi / Mt;   // same value as the theta table entry
  const double start = a0;
  double g0 = 0, g1 = 0, g2 = 0;
  StarTab tbs;   // in local memory
  const StarTab* tb = nullptr;
  if (S.kind == 1 && S.nt <= kStarTabTerms) {
    star_tab_fill(S, P.ts, P.t, P.th, &tbs);
    tb = &tbs;
  }
  double2 tsc;   // sin t_s, cos t_s for every evaluation of the ring
  sincos(P.ts, &tsc.x, &tsc.y);
  auto eval_r = [&](double z) {
    Geo G;
    if (tb) surf_eval_star_tab(S, *tb, z, 2, &G);
    else surf_eval(S, P.ts, z, 2, &G, &tsc);
    const double yx = G.r.x - P.x, yy = G.r.y - P.y, yz = G.r.z - P.z;
    g0 = yx * yx + yy * yy + yz * yz;
    g1 = 2 * (yx * G.rth.x + yy * G.rth.y + yz * G.rth.z);
    g2 = 2 * (dot(G.rth, G.rth) + yx * G.rthth.x + yy * G.rthth.y + yz * G.rthth.z);
  };
  for (int it = 0; it < 40; ++it) {
    eval_r(a0);
    double step = g2 > 0 ? g1 / g2 : 0.0;
    step = fmin(fmax(step, -hgrid), hgrid);
    a0 = fmin(fmax(a0 - step, start - hgrid), start + hgrid);
    if (fabs(step) <= 1e-15 * (1 + fabs(a0))) break;
  }
  eval_r(a0);
  if (fabs(P.ts - P.t) + fabs(wrap_pi(a0 - P.th)) <= kStableDelta || g0 <= kStableDist * kStableDist) {
    // rho^2(a0) without cancellation
    const R3 Y = tb ? diff_star_tab<double>(S, *tb, a0, P.th) : diff_ana<double>(S, P.ts, a0, P.t, P.th);
    g0 = dot(Y, Y);
  }
  const double b0 = sqrt(2 * g0 / (g2 > 0 ? g2 : 0.0));
  P.a0 = a0;
  P.capped = !(b0 <= kBCap);
  cplx z = C(a0, P.capped ? kBCap : b0);
  bool done = P.capped, extra = false;
  for (int it = 0; it < 60 && !done; ++it) {
    cplx f, df;
    rho2_cplx(S, P, tb, &tsc, z, &f, &df);
    const cplx dz = cdiv(f, df);
    cplx zn = z - dz;
    if (zn.im < 0) zn = conj(zn);
    const bool over = !(zn.im <= kBCap);
    if (over) {
      P.capped = 1;
      zn = C(a0, kBCap);
    }
    z = zn;
    const bool small = sqrt(abs2(dz)) <= kRootTol * fabs(z.im) + 4e-16 * sqrt(abs2(z));
    if (over || extra) done = true;
    extra = extra || small;
  }
  P.a = z.re;
  P.b = z.im;
  if (!(P.b > 0.0) || !(P.a == P.a)) {   // no usable root (never expected): fall back to the cap
    P.a = a0;
    P.b = kBCap;
    P.capped = 1;
  }
}

// ------------------------------------------------------------------ phase C: A_m, D_m (one lane)
// rec[4m..4m+3] = (2m-1)/(2m+1), 8m/(2m+1), t_m, w_m (Miller's rescaled recurrence; recurrence_table)
__device__ __noinline__ void a_modes_lane(double b, int L, const double* __restrict__ rec, int rec_len, double* A,
                                    double* D, int stride, bool dw_out) {
  // D may be null (only A is needed for the single-layer kernel); dw_out: A is left as double words
  // (float2 in the same 8-byte slots) for the double-word phase D
  const double q = exp(-b);
  double K, E;
  ellipke(q * q, -expm1(-2 * b), &K, &E);
  const double A0 = 2 / kPi * K;
  const double sh2 = sinh(b / 2) * sinh(b / 2);
  if (L * b <= kForwardLimit) {
    auto put = [&](int m, double v) {   // A_m, as a double word where asked
      if (dw_out) reinterpret_cast<float2*>(A)[m * stride] = dw_from(v);
      else A[m * stride] = v;
    };
    double am = A0, dm = (2 / kPi) * ((K - E) / q - K);
    put(0, am);
    if (D) D[0] = -dm;
    am += dm;
    put(1, am);
    if (D) D[stride] = dm;
    for (int m = 1; m < L; ++m) {
      dm = rec[4 * m] * dm + (rec[4 * m + 1] * sh2) * am;
      am += dm;
      put(m + 1, am);
      if (D) D[(m + 1) * stride] = dm;
    }
    return;
  }
  // Miller: backward from N with B_{N+1} = 0, B_N = 1 (A~_m = w_m B_m); rescale on growth; normalise
  // by A_0.
  int N = L + (int)ceil(kMillerLog / (2 * b)) + 16;
  if (N > rec_len - 2) N = rec_len - 2;
  const double ch = cosh(b);
  double up = 0.0, cur = 1.0;   // B_{m+1}, B_m
  for (int m = N; m >= 1; --m) {
    const double prev = fma(rec[4 * m + 2] * ch, cur, -up);   // B_{m-1}
    up = cur;
    cur = prev;
    if (m - 1 <= L) A[(m - 1) * stride] = cur;
    // |B| grows by at most (4 cosh(b) + 1) a step over two steps (t_m alternates about 4/5 and 4):
    // checking every 8 steps keeps it below 1e220
    if ((m & 7) == 0 && fabs(cur) > 1e200) {
      cur *= 1e-200;
      up *= 1e-200;
      for (int j = m - 1; j <= L; ++j) A[j * stride] *= 1e-200;
    }
  }
  const double f = A0 / A[0];   // w_0 = 1
  if (dw_out) {   // normalised and split into double words in one pass
    for (int m = 0; m <= L; ++m) reinterpret_cast<float2*>(A)[m * stride] = dw_from(A[m * stride] * (rec[4 * m + 3] * f));
    return;
  }
  double prevA = 0.0;
  for (int m = 0; m <= L; ++m) {
    const double am = A[m * stride] * (rec[4 * m + 3] * f);
    A[m * stride] = am;
    if (D && m) D[m * stride] = am - prevA;
    prevA = am;
  }
  if (D) D[0] = A[0] - A[stride];
}

// ------------------------------------------------------------------ small helpers of phase D
// sin x for |x| <= 0.05 by its Taylor polynomial through x^9 (the first omitted term is below
// 2^-60 |x|): relative accuracy without the range reduction of the library sine.
__device__ __forceinline__ double sin_small(double x) {
  const double x2 = x * x;
  return x * fma(x2, fma(x2, fma(x2, fma(x2, 1.0 / 362880.0, -1.0 / 5040.0), 1.0 / 120.0), -1.0 / 6.0), 1.0);
}
__device__ __forceinline__ int wrapi(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}
// v mod n for |v| < n
__device__ __forceinline__ int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// sin(k x) - k sin(x), k >= 0, without cancellation: the Taylor series when |k x| < 1 (its term
// ratios are constants once the loop unrolls), else from skx = sin(k x) and sx = sin(x).
__device__ inline double sin_k_minus(int k, double x, double skx, double sx) {
  const double kx = k * x;
  if (fabs(kx) < 1.0) {
    const double kx2 = kx * kx, x2 = x * x;
    constexpr double r6 = 1.0 / 6.0;
    double an = kx * kx2 * r6, bn = k * x * x2 * r6, acc = 0.0, sg = -1.0;
#pragma unroll
    for (int n = 1; n <= 12; ++n) {
      acc += sg * (an - bn);
      const double rden = 1.0 / ((2.0 * n + 2) * (2.0 * n + 3));
      an *= kx2 * rden;
      bn *= x2 * rden;
      sg = -sg;
    }
    return acc;
  }
  return skx - k * sx;
}

struct Smem {
  double *sn, *tau0, *bt0, *hr, *alph, *Acal, *Bcal;
  cplx *W0, *W1, *ph, *kc, *kk;
  unsigned* nearbits;   // double layer: samples whose differences take the cancellation-free forms
};

// Per-warp shared memory of the pair pipeline, in doubles.  Single layer: sn, A~, the two
// transform buffers, the phases.  With the double layer also tau_0, beta, H3, alpha on the grid,
// B~, and one buffer of singular modes (kc for S, then kk for K: the S outputs leave first).
__host__ __device__ inline size_t smem_doubles(int Mt, int P, int L, bool withK) {
  (void)L;
  const int M = Mt / 2;
  size_t d = 0;
  d += Mt;                                   // sn
  d += withK ? 4 * Mt : 0;                   // tau0, bt0, hr, alph
  d += withK ? (Mt + 63) / 64 : 0;           // nearbits (one bit per sample)
  d += P;                                    // Acal
  d += withK ? P : 0;                        // Bcal
  d += d & 1;                                // W0, W1 start on 16 bytes: the transforms read float4
  d += 4 * P;                                // W0, W1 (complex)
  d += withK ? 2 * 2 * (2 * M + 1) : 2 * (2 * M + 1);   // ph (, kc = kk)
  return d;
}

__device__ inline Smem carve(double* base, int Mt, int P, int L, bool withK) {
  (void)L;
  const int M = Mt / 2;
  Smem s = {};
  double* p = base;
  s.sn = p; p += Mt;
  if (withK) {
    s.tau0 = p; p += Mt; s.bt0 = p; p += Mt; s.hr = p; p += Mt; s.alph = p; p += Mt;
    s.nearbits = reinterpret_cast<unsigned*>(p); p += (Mt + 63) / 64;
  }
  s.Acal = p; p += P;
  if (withK) { s.Bcal = p; p += P; }
  p += (p - base) & 1;   // 16-byte start for the double-word transforms
  s.W0 = (cplx*)p; p += 2 * P;
  s.W1 = (cplx*)p; p += 2 * P;
  s.ph = (cplx*)p; p += 2 * (2 * M + 1);
  if (withK) {
    s.kc = (cplx*)p;
    s.kk = s.kc;
    p += 2 * (2 * M + 1);
  }
  return s;
}

// Transform of complex doubles (warp_fft's contract) through the double-word FFT: convert in place,
// transform, convert the result back (integer splits, one FP64 add per component on the way back).
__device__ __noinline__ cplx* warp_fft_x(cplx* x, cplx* y, int n, const float4* __restrict__ twf, int T, int sign) {
  const int lane = threadIdx.x & 31;
  float4* xf = reinterpret_cast<float4*>(x);
  for (int i = lane; i < n; i += 32) {
    const cplx v = x[i];
    xf[i] = dwc_from(v);
  }
  __syncwarp();
  float4* r = warp_fft_dw(xf, reinterpret_cast<float4*>(y), n, twf, T, sign);
  cplx* rc = reinterpret_cast<cplx*>(r);
  for (int i = lane; i < n; i += 32) {
    const float4 v = r[i];
    rc[i] = dwc_to(v);
  }
  __syncwarp();
  return rc;
}

// e^{ija} Z_j / Mt (j = -M..M, Nyquist split evenly) placed on the P grid in X, inverse
// transform with scratch Y (in double words if dw); returns the buffer holding the result.
// The modes sit at |j| <= M of the length-P input, so where the transform's first stage is radix 4
// with stride s = P/4 > M, its butterfly j < s meets at most x_j (j <= M) and x_{j+3s} (j >= s - M):
// that stage runs here, fused with the placement and without the zeros (the same values).
__device__ __noinline__ cplx* upsample(const cplx* Z, const cplx* ph, cplx* X, cplx* Y, int Mt, int P, const cplx* tw,
                                 const float4* twf, int T, bool dw) {
  const int lane = threadIdx.x & 31;
  const int M = Mt / 2;
  auto mode_at = [&](int jv) {
    cplx z = Z[wrapi(jv, Mt)] * (1.0 / Mt);
    if (jv == M || jv == -M) z = 0.5 * z;
    return ph[jv + M] * z;
  };
  const int s4 = P / 4;
  if (P % 4 == 0 && s4 > M) {
    if (dw) {
      float4* Xf = reinterpret_cast<float4*>(X);
      for (int j = lane; j < s4; j += 32) {
        const float4 v0 = j <= M ? dwc_from(mode_at(j)) : dwc_zero();
        const float4 v3 = j >= s4 - M ? dwc_from(mode_at(j - s4)) : dwc_zero();
        const float4 jd = mul_i(dwc_sub(dwc_zero(), v3), +1);
        Xf[4 * j] = dwc_add(v0, v3);
        Xf[4 * j + 1] = dwc_add(v0, jd);
        Xf[4 * j + 2] = dwc_sub(v0, v3);
        Xf[4 * j + 3] = dwc_sub(v0, jd);
      }
      __syncwarp();
      float4* r = warp_fft_dw(Xf, reinterpret_cast<float4*>(Y), P, twf, T, +1, 1);
      cplx* rc = reinterpret_cast<cplx*>(r);
      for (int i = lane; i < P; i += 32) {
        const float4 v = r[i];
        rc[i] = dwc_to(v);
      }
      __syncwarp();
      return rc;
    }
    for (int j = lane; j < s4; j += 32) {
      const cplx v0 = j <= M ? mode_at(j) : C(0.0);
      const cplx v3 = j >= s4 - M ? mode_at(j - s4) : C(0.0);
      const cplx jd = C(v3.im, -v3.re);   // +i (x_{j+s} - x_{j+3s})
      X[4 * j] = v0 + v3;
      X[4 * j + 1] = v0 + jd;
      X[4 * j + 2] = v0 - v3;
      X[4 * j + 3] = v0 - jd;
    }
    __syncwarp();
    return warp_fft(X, Y, P, tw, T, +1, 1);
  }
  for (int pp = lane; pp < P; pp += 32) X[pp] = C(0.0);
  __syncwarp();
  for (int jj = lane; jj <= 2 * M; jj += 32) X[wrapi(jj - M, P)] = mode_at(jj - M);
  __syncwarp();
  return dw ? warp_fft_x(X, Y, P, twf, T, +1) : warp_fft(X, Y, P, tw, T, +1);
}

// ------------------------------------------------------------------ phase D, single layer alone
// Arithmetic of the single layer's transforms: double words on the FP32 pipe (ArDW, the default) or
// FP64 throughout (ArF64, a context option that measures what the narrower arithmetic buys).  Both
// hold a complex value in 16 bytes and a real one in 8, so the records and shared memory are shared.
struct ArDW {
  using C = float4;
  using R = float2;
  static __device__ __forceinline__ R rfrom(double v) { return dw_from(v); }
  static __device__ __forceinline__ double rto(R v) { return dw_to(v); }
  static __device__ __forceinline__ cplx cto(C v) { return dwc_to(v); }
  static __device__ __forceinline__ C mul(C x, C y) { return dwc_mul(x, y); }
  static __device__ __forceinline__ C mulr(C x, R r) { return dwc_mulr(x, r); }
  static __device__ __forceinline__ C conjg(C x) { return dwc_conj(x); }
  static __device__ __forceinline__ C add(C x, C y) { return dwc_add(x, y); }
  static __device__ __forceinline__ C sub(C x, C y) { return dwc_sub(x, y); }
  static __device__ __forceinline__ C jneg(C x) { return mul_i(dwc_sub(dwc_zero(), x), +1); }   // i (0 - x)
  static __device__ __forceinline__ C half(C x) { return dwc_scale2(x, 0.5f); }
  static __device__ __forceinline__ C zero() { return dwc_zero(); }
  static __device__ __forceinline__ C mk(R re, R im) { return mkc(re, im); }
  static __device__ __forceinline__ R re(C x) { return cre(x); }
  static __device__ __forceinline__ R im(C x) { return cim(x); }
  static __device__ __forceinline__ R rzero() { return make_float2(0.f, 0.f); }
  static __device__ __forceinline__ R rmul(R x, R y) { return dw_mul(x, y); }
  static __device__ __forceinline__ R radd(R x, R y) { return dw_add(x, y); }
  static __device__ __forceinline__ R rsub(R x, R y) { return dw_sub(x, y); }
  static __device__ __forceinline__ R rscale(R x, int e) { return dw_scale2(x, ldexpf(1.f, e)); }
  static __device__ __forceinline__ C imscale(C x, int e) {
    const float sc = ldexpf(1.f, e);
    return make_float4(x.x, x.y, x.z * sc, x.w * sc);
  }
  static __device__ __forceinline__ double lead(R x) { return (double)x.x; }
  static __device__ __forceinline__ void sincosr(double x, R* s, R* c) { dw_sincos(x, s, c); }
  // F = sqrt(s) / rho from s (FP64) and 1/rho (FP64 and in this form)
  static __device__ __forceinline__ R smooth_f(double s, double rinv, R ri) {
    (void)rinv;
    return dw_mul(dw_sqrt(dw_from(s)), ri);
  }
  static __device__ __forceinline__ C* fft(C* x, C* y, int n, const PairArgs& a, int sign, int st0 = 0) {
    return warp_fft_dw(x, y, n, a.twf, a.T, sign, st0);
  }
};
struct ArF64 {
  using C = cplx;
  using R = double;
  static __device__ __forceinline__ R rfrom(double v) { return v; }
  static __device__ __forceinline__ double rto(R v) { return v; }
  static __device__ __forceinline__ cplx cto(C v) { return v; }
  static __device__ __forceinline__ C mul(C x, C y) { return x * y; }
  static __device__ __forceinline__ C mulr(C x, R r) { return x * r; }
  static __device__ __forceinline__ C conjg(C x) { return conj(x); }
  static __device__ __forceinline__ C add(C x, C y) { return x + y; }
  static __device__ __forceinline__ C sub(C x, C y) { return x - y; }
  static __device__ __forceinline__ C jneg(C x) { return bie::C(x.im, -x.re); }   // i (0 - x)
  static __device__ __forceinline__ C half(C x) { return 0.5 * x; }
  static __device__ __forceinline__ C zero() { return bie::C(0.0); }
  static __device__ __forceinline__ C mk(R re, R im) { return bie::C(re, im); }
  static __device__ __forceinline__ R re(C x) { return x.re; }
  static __device__ __forceinline__ R im(C x) { return x.im; }
  static __device__ __forceinline__ R rzero() { return 0.0; }
  static __device__ __forceinline__ R rmul(R x, R y) { return x * y; }
  static __device__ __forceinline__ R radd(R x, R y) { return x + y; }
  static __device__ __forceinline__ R rsub(R x, R y) { return x - y; }
  static __device__ __forceinline__ R rscale(R x, int e) { return ldexp(x, e); }
  static __device__ __forceinline__ C imscale(C x, int e) { return bie::C(x.re, ldexp(x.im, e)); }
  static __device__ __forceinline__ double lead(R x) { return x; }
  static __device__ __forceinline__ void sincosr(double x, R* s, R* c) { sincos(x, s, c); }
  static __device__ __forceinline__ R smooth_f(double s, double rinv, R ri) {
    (void)ri;
    return sqrt(s) * rinv;
  }
  static __device__ __forceinline__ C* fft(C* x, C* y, int n, const PairArgs& a, int sign, int st0 = 0) {
    return warp_fft(x, y, n, a.tw, a.T, sign, st0);
  }
};

// The same steps as the general phase D below, with every transform, the upsampling, the products
// and the unpacking in the arithmetic Ar; FP64 for the samples and the outputs.
//   E       [pair][33] e^{i l a} (l < 32) and e^{32 i a} of the batch (phase B), in Ar's complex form
//   Ab      A_m in Ar's real form: A_m of pair j at Ab[j a_ps + m a_ms]
//   R2      rho^2 on the ring, [pair][Mt] (phase A, with the cancellation-free differences)
template <class Ar>
__device__ __forceinline__ void phase_d_single(const PairArgs& a, const Smem& sm, const typename Ar::R* Ab, int a_ps,
                                               int a_ms, const typename Ar::C* E, const double* R2,
                                               const PairInfo& mine, unsigned valid_mask, int64_t p0, int nb) {
  using Cx = typename Ar::C;
  using Rx = typename Ar::R;
  const int lane = threadIdx.x & 31;
  const int Mt = a.Mt, M = a.M, P = a.P, L = a.L;
  Cx* W0 = reinterpret_cast<Cx*>(sm.W0);
  Cx* W1 = reinterpret_cast<Cx*>(sm.W1);
  Rx* Acal = reinterpret_cast<Rx*>(sm.Acal);
  const Rx invMt = Ar::rfrom(1.0 / Mt);
  const Rx ratio = Ar::rfrom((double)Mt / P);   // e^{ija}/Mt -> e^{ija}/P
  int acal_next = -1;   // pair whose circulant transform already sits in Acal
  for (int pi = 0; pi < nb; ++pi) {
    const PairInfo pr = bcast(mine, pi);
    const int64_t p = a.out_mod ? (a.out_base + p0 + pi) % a.out_mod : p0 + pi;   // output slot
    // the next pair's records (rho^2 on the ring, e^{ila}) on their way to L2 while this pair runs:
    // one 128-byte line per lane, every line starting inside its record
    if (pi + 1 < nb) {
      const char* nr = reinterpret_cast<const char*>(R2 + (pi + 1) * Mt);
      const char* ne = reinterpret_cast<const char*>(E + (pi + 1) * 33);
      const int lr = (Mt * 8 + 127) / 128, le = (33 * 16 + 127) / 128;
      const char* pf = lane < lr ? nr + lane * 128 : (lane < lr + le ? ne + (lane - lr) * 128 : nullptr);
      if (pf && __isGlobal(pf)) asm volatile("prefetch.global.L2 [%0];" ::"l"(pf));
    }
    if (!pr.valid) {
      if (a.modes_out)
        for (int m = lane; m < 2 * (Mt + 1); m += 32) a.modes_out[p * 2 * (Mt + 1) + m] = 0.0;
      if (a.weights_out)
        for (int m = lane; m < Mt; m += 32) a.weights_out[p * a.w_ld + m] = C(0.0);
      continue;
    }
    const double* r2p = R2 + pi * Mt;
    // ---- phases e^{ija}/Mt, j = -M..M: lane l starts from e^{i l a}, steps of e^{32 i a}
    Cx* ph = reinterpret_cast<Cx*>(sm.ph);
    {
      Cx e = E[pi * 33 + lane];
      const Cx step = E[pi * 33 + 32];
      for (int j = lane; j <= M; j += 32) {
        const Cx es = Ar::mulr(e, invMt);
        ph[M + j] = es;
        ph[M - j] = Ar::conjg(es);
        e = Ar::mul(e, step);
      }
    }
    __syncwarp();
    auto phase = [&](int jj) { return ph[jj]; };   // e^{ija}/Mt, jj = j + M
    // ---- circulant transform of A_{|d|}, unless it came packed with the previous pair
    if (acal_next != pi) {
      for (int pp = lane; pp < P; pp += 32) {
        const int dd = pp <= P / 2 ? pp : P - pp;
        W1[pp] = Ar::mk(dd <= L ? Ab[pi * a_ps + dd * a_ms] : Ar::rzero(), Ar::rzero());
      }
      __syncwarp();
      const Cx* Af = Ar::fft(W1, W0, P, a, -1);
      for (int pp = lane; pp < P; pp += 32) Acal[pp] = Ar::re(Af[pp]);
    }
    __syncwarp();
    // ---- samples: F + i cos(k rho) and sin(k rho)/rho
    Rx* snw = reinterpret_cast<Rx*>(sm.sn);
    for (int q = lane; q < Mt; q += 32) {
      const double thq = a.thg[3 * q];
      const double r2 = r2p[q];
      const double rinv = rsqrt(r2);
      const double rho = r2 * rinv;
      const double dq = thq - pr.a;
      const double sp = fabs(dq) < 0.1 ? sin_small(0.5 * dq) : a.thg[3 * q + 1] * pr.cha - a.thg[3 * q + 2] * pr.sha;
      const double sv = pr.om * pr.om + 4 * pr.qb * sp * sp;
      const Rx ri = Ar::rfrom(rinv);
      Rx skr, ckr;
      Ar::sincosr(a.k * rho, &skr, &ckr);
      W0[q] = Ar::mk(Ar::smooth_f(sv, rinv, ri), ckr);
      snw[q] = Ar::rmul(skr, ri);
    }
    __syncwarp();
    // ---- modes of F and cos(k rho); upsample onto the shifted P grid.  The modes sit at |j| <= M of
    // the length-P input: where the first stage is radix 4 with stride s = P/4 > M, its butterfly
    // j < s meets at most x_j (j <= M) and x_{j+3s} (j >= s - M), and it runs here, fused with the
    // placement and without the zeros (the same values)
    Cx* Z1 = Ar::fft(W0, W1, Mt, a, -1);
    Cx* X = (Z1 == W0) ? W1 : W0;
    auto mode_at = [&](int jv) {
      Cx z = Ar::mul(phase(jv + M), Z1[wrap1(jv, Mt)]);
      if (jv == M || jv == -M) z = Ar::half(z);
      return z;
    };
    Cx* up1;   // re: F~, im: C~
    const int s4 = P / 4;
    if (P % 4 == 0 && s4 > M) {
      for (int j = lane; j < s4; j += 32) {
        const Cx v0 = j <= M ? mode_at(j) : Ar::zero();
        const Cx v3 = j >= s4 - M ? mode_at(j - s4) : Ar::zero();
        const Cx jd = Ar::jneg(v3);
        X[4 * j] = Ar::add(v0, v3);
        X[4 * j + 1] = Ar::add(v0, jd);
        X[4 * j + 2] = Ar::sub(v0, v3);
        X[4 * j + 3] = Ar::sub(v0, jd);
      }
      __syncwarp();
      up1 = Ar::fft(X, Z1, P, a, +1, 1);
    } else {
      for (int pp = lane; pp < P; pp += 32) X[pp] = Ar::zero();
      __syncwarp();
      for (int jj = lane; jj <= 2 * M; jj += 32) X[wrap1(jj - M, P)] = mode_at(jj - M);
      __syncwarp();
      up1 = Ar::fft(X, Z1, P, a, +1);
    }
    Cx* uf = (up1 == W0) ? W1 : W0;
    // ---- U = F~ C~ Acal in the real part, the next valid pair's circulant in the imaginary part.
    // Each part comes out of the shared transform with an error in proportion to the other's size
    // (the product is 10^3 times the circulant next to a pole), so the circulant is scaled by an
    // exact power of two to the product's root-mean-square size before packing.
    const unsigned later = valid_mask & ~((2u << pi) - 1u);
    const int nxt = later ? __ffs(later) - 1 : nb;
    const bool pack = nxt < nb;
    float su = 0.f, sa = 0.f;
    for (int pp = lane; pp < P; pp += 32) {
      const int dd = pp <= P / 2 ? pp : P - pp;
      const Cx u = up1[pp];
      const Rx prod = Ar::rmul(Ar::rmul(Ar::re(u), Ar::im(u)), Acal[pp]);
      const Rx an = (pack && dd <= L) ? Ab[nxt * a_ps + dd * a_ms] : Ar::rzero();
      const float pf = (float)Ar::lead(prod), af = (float)Ar::lead(an);
      su = fmaf(pf, pf, su);
      sa = fmaf(af, af, sa);
      uf[pp] = Ar::mk(prod, an);
    }
    for (int o = 16; o; o >>= 1) {
      su += __shfl_xor_sync(0xffffffffu, su, o);
      sa += __shfl_xor_sync(0xffffffffu, sa, o);
    }
    int pe = 0;   // circulant scale 2^pe
    if (pack && sa > 0.f && su > 0.f) pe = max(-60, min(60, (int)rintf(0.5f * log2f(su / sa))));
    if (pe) {
      __syncwarp();
      for (int pp = lane; pp < P; pp += 32) uf[pp] = Ar::imscale(uf[pp], pe);
    }
    __syncwarp();
    const Cx* Yf = Ar::fft(uf, up1, P, a, -1);
    // ---- kernel modes kc_m = e^{-ima} (Re-part transform)_m / P, m = -M..M, written straight to the
    // modes output and to the free buffer in the input order of the weights' inverse transform
    // (q = m mod Mt; q = M holds the mean of m = -M and m = M)
    Cx* Wi = (Yf == W0) ? W1 : W0;
    double* out = a.modes_out ? a.modes_out + p * 2 * (Mt + 1) : nullptr;
    auto kc_of = [&](int jj) {
      const int m = jj - M;
      const Cx zp = Yf[wrap1(m, P)], zm = Ar::conjg(Yf[wrap1(-m, P)]);
      return Ar::mul(Ar::mulr(Ar::conjg(phase(jj)), ratio), Ar::half(Ar::add(zp, zm)));
    };
    for (int jj = lane; jj <= 2 * M; jj += 32) {
      const Cx kv = kc_of(jj);
      if (out) {
        const cplx c = Ar::cto(kv);
        out[2 * jj] = c.re;
        out[2 * jj + 1] = c.im;
      }
      if (a.weights_out) {
        const int m = jj - M;
        if (jj == 0) Wi[M] = Ar::half(Ar::add(kv, kc_of(2 * M)));
        else if (jj < 2 * M) Wi[m < 0 ? m + Mt : m] = kv;
      }
    }
    if (pack) {
      for (int pp = lane; pp < P; pp += 32) {
        const Cx zp = Yf[pp], zm = Ar::conjg(Yf[pp == 0 ? 0 : P - pp]);
        Acal[pp] = Ar::rscale(Ar::rsub(Ar::im(zp), Ar::im(zm)), -pe - 1);
      }
      acal_next = nxt;
    }
    __syncwarp();
    // ---- Parseval weights: inverse transform of the kernel modes, plus sin(k rho)/(rho Mt)
    if (a.weights_out) {
      const Cx* Wt = Ar::fft(Wi, (Wi == W0) ? W1 : W0, Mt, a, +1);
      cplx* wout = a.weights_out + p * a.w_ld;
      if (a.weights_dw) {   // (double-word arithmetic only)
        Cx* wo = reinterpret_cast<Cx*>(wout);
        for (int q = lane; q < Mt; q += 32) {
          const Cx w = Wt[q];
          wo[q] = Ar::mk(Ar::rmul(Ar::re(w), invMt), Ar::rmul(Ar::radd(Ar::im(w), snw[q]), invMt));
        }
      } else {
        for (int q = lane; q < Mt; q += 32) {
          const cplx w = Ar::cto(Wt[q]) * (1.0 / Mt);
          wout[q] = C(w.re, w.im + Ar::rto(snw[q]) * (1.0 / Mt));
        }
      }
      __syncwarp();
    }
    // ---- modes K_m = kc_m + i <sin(k rho)/rho>_m: the smooth part added to the kernel part in out
    // (each entry by the lane that wrote it)
    if (out) {
      for (int q = lane; q < Mt; q += 32) W0[q] = Ar::mk(snw[q], Ar::rzero());
      __syncwarp();
      const Cx* Sf = Ar::fft(W0, W1, Mt, a, -1);
      for (int mm = lane; mm <= 2 * M; mm += 32) {
        const int m = mm - M;
        cplx sv = Ar::cto(Sf[wrap1(m, Mt)]) * (1.0 / Mt);
        if (m == M || m == -M) sv = 0.5 * sv;
        out[2 * mm] -= sv.im;
        out[2 * mm + 1] += sv.re;
      }
      __syncwarp();
    }
  }
  __syncwarp();
}

// ------------------------------------------------------------------ the kernel
// Decode and phases A-C of one batch of up to 32 consecutive pairs [p0, p0 + nb).  Outputs per
// pair j of the batch: rho^2 on the ring at R2 + j Mt (single layer; shared memory with the double
// layer); e^{i l a} at E + 33 j (single layer); A_m at Ab + j a_ps + m a_ms (double words for the
// single layer); D_m at scrD + j + 32 m (double layer).
// nlist: this warp's shared-memory list of kNearList near samples (single layer), or null: the
// samples of phase A that take the cancellation-free difference are then collected over the batch's
// pairs and evaluated with every lane busy (one lane per sample) instead of one pair at a time.
constexpr int kNearList = 256;
template <bool kWithK>
__device__ __forceinline__ void front_batch(const PairArgs& a, const Smem& sm, int64_t p0, int nb, double* R2,
                                            float4* E, double* Ab, int a_ps, int a_ms, double* scrD, PairInfo& mine,
                                            unsigned& valid_mask, int* nlist = nullptr) {
  const int lane = threadIdx.x & 31;
  const int Mt = a.Mt, L = a.L;
  constexpr bool wantK = kWithK;
    // ---------------- decode the batch (lane per pair)
    mine = PairInfo{};
    if (lane < nb) {
      const int64_t p = p0 + lane;
      int64_t row;
      int d, g;
      if (a.enumerate) {
        const int64_t pg = a.p0 + p;
        const int i = (int)(pg % Mt);
        int64_t rest = pg / Mt;
        g = (int)(rest % 16);
        rest /= 16;
        d = (int)(rest % 3);
        row = (rest / 3) * Mt + i;
      } else {
        row = a.rows[p];
        const int src = a.srcs[p];
        d = src / 16;
        g = src % 16;
        if (src < 0 || src >= 48) d = -1;
      }
      PairInfo pr = {};
      const int64_t tn = row / Mt;
      const int ip = (int)(tn / 16) + d - 1;   // on a torus every panel has both neighbours
      pr.valid = !(row < 0 || row >= a.N || d < 0 || (!a.S.periodic && (ip < 0 || ip >= a.Np)));
      pr.row = row;
      if (pr.valid) {
        pr.ring = (tn * 3 + d) * 16 + g;
        pr.t = a.t_nodes[tn];
        pr.th = a.thg[3 * (int)(row % Mt)];
        pr.ts = a.ring_t[pr.ring];
        pr.x = a.pts[3 * row];
        pr.y = a.pts[3 * row + 1];
        pr.z = a.pts[3 * row + 2];
      } else if (!a.enumerate) {
        atomicAdd(a.status, 1);
      }
      mine = pr;
    }
    valid_mask = __ballot_sync(0xffffffffu, lane < nb && mine.valid);
    // ---------------- A. grid minimiser (warp per pair); rho^2 kept for the single layer
    if (!wantK && nlist) {
      // A1. rho^2 by plain subtraction on every sample; the samples near the target (those that take the
      // cancellation-free difference) go to the list, or are evaluated here once the list is full
      int nn = 0;
      for (int pi = 0; pi < nb; ++pi) {
        const PairInfo pr = bcast(mine, pi);
        if (!pr.valid) continue;
        double* rho2 = R2 + pi * Mt;
        const double* rr = a.ring_r + pr.ring * 3 * Mt;
        const int i = (int)(pr.row % Mt);
        const double dts = fabs(pr.t - pr.ts);
        const int kn = dts <= kStableDelta ? (int)((kStableDelta - dts) * Mt / kTwoPi) : -1;
        for (int q0 = 0; q0 < Mt; q0 += 32) {
          const int q = q0 + lane;
          bool nr = false;
          if (q < Mt) {
            const int dq = q > i ? q - i : i - q;
            const double yx = rr[3 * q] - pr.x, yy = rr[3 * q + 1] - pr.y, yz = rr[3 * q + 2] - pr.z;
            const double r2 = yx * yx + yy * yy + yz * yz;
            nr = min(dq, Mt - dq) <= kn || r2 <= kStableDist * kStableDist;
            rho2[q] = r2;
          }
          const unsigned m = __ballot_sync(0xffffffffu, nr);
          if (nr) {
            const int slot = nn + __popc(m & ((1u << lane) - 1u));
            if (slot < kNearList) {
              nlist[slot] = (pi << 16) | q;
            } else {
              const R3 Y = diff_ana<double>(a.S, pr.ts, a.thg[3 * q], pr.t, pr.th);
              rho2[q] = dot(Y, Y);
            }
          }
          nn += __popc(m);
        }
      }
      __syncwarp();
      // A2. the listed samples, one per lane
      const int nl = min(nn, kNearList);
      for (int b0 = 0; b0 < nl; b0 += 32) {
        const int e = b0 + lane;
        const int code = e < nl ? nlist[e] : 0;
        const int pi = code >> 16, q = code & 0xffff;
        const double ts = __shfl_sync(0xffffffffu, mine.ts, pi), t = __shfl_sync(0xffffffffu, mine.t, pi);
        const double th = __shfl_sync(0xffffffffu, mine.th, pi);
        if (e < nl) {
          const R3 Y = diff_ana<double>(a.S, ts, a.thg[3 * q], t, th);
          R2[pi * Mt + q] = dot(Y, Y);
        }
      }
      __syncwarp();
      // A3. grid minimiser of each pair (near-ties to the sample nearest the target, then the lower index)
      for (int pi = 0; pi < nb; ++pi) {
        const PairInfo pr = bcast(mine, pi);
        if (!pr.valid) continue;
        const double* rho2 = R2 + pi * Mt;
        const int i = (int)(pr.row % Mt);
        double bv = INFINITY;
        for (int q = lane; q < Mt; q += 32) bv = fmin(bv, rho2[q]);
        for (int o = 16; o; o >>= 1) bv = fmin(bv, __shfl_xor_sync(0xffffffffu, bv, o));
        int bkey = 0x7fffffff;
        const double tie = bv * (1 + 1e-12);
        for (int q = lane; q < Mt; q += 32)
          if (rho2[q] <= tie) {
            const int dq = q > i ? q - i : i - q;
            bkey = min(bkey, min(dq, Mt - dq) * Mt + q);
          }
        for (int o = 16; o; o >>= 1) bkey = min(bkey, __shfl_xor_sync(0xffffffffu, bkey, o));
        if (lane == pi) mine.bi = bkey % Mt;
        __syncwarp();
      }
    } else {
      for (int pi = 0; pi < nb; ++pi) {
        const PairInfo pr = bcast(mine, pi);
        if (!pr.valid) continue;
        double* rho2 = wantK ? (double*)sm.W0 : R2 + pi * Mt;
        const double* rr = a.ring_r + pr.ring * 3 * Mt;
        const int i = (int)(pr.row % Mt);
        const double dts = fabs(pr.t - pr.ts);
        // |t - t_s| + |th_i - th_q| <= kStableDelta as a bound on the grid distance |i - q| (both
        // branches give rho^2 to rounding, so the boundary only picks the cheaper formula)
        const int kn = dts <= kStableDelta ? (int)((kStableDelta - dts) * Mt / kTwoPi) : -1;
        double bv = INFINITY;
        for (int q = lane; q < Mt; q += 32) {
          const double thq = a.thg[3 * q];
          const int dq = q > i ? q - i : i - q;
          const double yx = rr[3 * q] - pr.x, yy = rr[3 * q + 1] - pr.y, yz = rr[3 * q + 2] - pr.z;
          double r2 = yx * yx + yy * yy + yz * yz;
          if (min(dq, Mt - dq) <= kn || r2 <= kStableDist * kStableDist) {
            const R3 Y = diff_ana<double>(a.S, pr.ts, thq, pr.t, pr.th);
            r2 = dot(Y, Y);
          }
          rho2[q] = r2;
          bv = fmin(bv, r2);
        }
        for (int o = 16; o; o >>= 1) bv = fmin(bv, __shfl_xor_sync(0xffffffffu, bv, o));
        __syncwarp();
        int bkey = 0x7fffffff;
        const double tie = bv * (1 + 1e-12);
        for (int q = lane; q < Mt; q += 32)
          if (rho2[q] <= tie) {
            const int dq = q > i ? q - i : i - q;
            bkey = min(bkey, min(dq, Mt - dq) * Mt + q);
          }
        for (int o = 16; o; o >>= 1) bkey = min(bkey, __shfl_xor_sync(0xffffffffu, bkey, o));
        if (lane == pi) mine.bi = bkey % Mt;
        __syncwarp();
      }
    }
    // ---------------- B. complex root and C. A_m, D_m (lane per pair)
    if (lane < nb && mine.valid) {
      locate_root(a.S, Mt, mine);
      mine.qb = exp(-mine.b);
      mine.om = -expm1(-mine.b);
      sincos(0.5 * mine.a, &mine.sha, &mine.cha);
      if (!wantK) {
        // e^{i l a} for l = 0..31 by rotation and e^{32 i a} directly ([pair][33]), as double words or
        // (FP64 transforms) as complex doubles
        float4* El = E + lane * 33;
        const cplx e1 = C(mine.cha * mine.cha - mine.sha * mine.sha, 2 * mine.sha * mine.cha);
        cplx e = C(1.0);
        for (int l = 0; l < 32; ++l) {
          if (a.fp64_transforms) reinterpret_cast<cplx*>(El)[l] = e;
          else El[l] = dwc_from(e);
          e = e * e1;
        }
        if (a.fp64_transforms) reinterpret_cast<cplx*>(El)[32] = cexpi(32.0 * mine.a);
        else El[32] = dwc_from(cexpi(32.0 * mine.a));
      }
      // FP64 recurrences (Miller runs up to L + 20/b steps: its rounding would add up in double words);
      // the single layer keeps A_m as double words for its transforms (or FP64 with FP64 transforms)
      a_modes_lane(mine.b, L, a.rec, a.rec_len, Ab + lane * a_ps, wantK ? scrD + lane : nullptr, a_ms,
                   !wantK && !a.fp64_transforms);
    }
    __syncwarp();
}

// One batch of up to 32 consecutive pairs [p0, p0 + nb) of the argument set a (phases A-D).
template <bool kWithK>
__device__ __forceinline__ void process_batch(const PairArgs& a, const Smem& sm, double* scrA, double* scrD,
                                              int64_t p0, int nb) {
  const int lane = threadIdx.x & 31;
  const int Mt = a.Mt, M = a.M, P = a.P, L = a.L;
  const bool wantS = a.kernels & BIE_KERNEL_S;
  constexpr bool wantK = kWithK;
  const int nk = (wantS ? 1 : 0) + (wantK ? 1 : 0);
    PairInfo mine;
    unsigned valid_mask;
    double* R2 = wantK ? nullptr : scrD + 2 * 33 * 32;
    front_batch<kWithK>(a, sm, p0, nb, R2, reinterpret_cast<float4*>(scrD), scrA, 1, 32, scrD, mine, valid_mask);
    if constexpr (!kWithK) {
      phase_d_single<ArDW>(a, sm, reinterpret_cast<const float2*>(scrA), 1, 32, reinterpret_cast<const float4*>(scrD),
                           R2, mine, valid_mask, p0, nb);
    } else {
    // ---------------- D. per pair (warp)
    // The transforms this layer shares with the single layer (the samples F + i cos, their
    // upsampling, the S product, the outputs) run in double words; those of the double layer stay
    // FP64: they pack signals of very different size (tau_0 ~ curvature rho^2 beside alpha ~ k^2,
    // A beside B, V_K A~ beside V_H), and extracting the small one costs digits in proportion.
    // Shared memory per warp holds only what outlives a step: A~ and B~ are rescaled in place
    // (A~ -> F~ A~ -> alpha~ tau0~ F~ A~, B~ -> h3~ B~), A_m, D_m and B_m are read from the
    // batch's recurrence scratch, and the single-layer outputs leave before the double layer's
    // singular modes take their buffer.
    auto emit = [&](int64_t p, int kidx, bool isS, const cplx* sing) {
      if (a.modes_out) {
        for (int q = lane; q < Mt; q += 32) sm.W0[q] = C(isS ? sm.sn[q] : sm.bt0[q], 0.0);
        __syncwarp();
        const cplx* Sf = warp_fft_x(sm.W0, sm.W1, Mt, a.twf, a.T, -1);
        double* out = a.modes_out + (p * a.out_nk + a.out_k0 + kidx) * 2 * (Mt + 1);
        for (int mm = lane; mm <= 2 * M; mm += 32) {
          const int m = mm - M;
          cplx sv = Sf[wrapi(m, Mt)] * (1.0 / Mt);
          if (m == M || m == -M) sv = 0.5 * sv;
          const cplx smooth = isS ? C(-sv.im, sv.re) : C(sv.im, -sv.re);   // i <sn> or -i <beta tau0>
          out[2 * mm] = sing[mm].re + smooth.re;
          out[2 * mm + 1] = sing[mm].im + smooth.im;
        }
        __syncwarp();
      }
      if (a.weights_out) {
        for (int q = lane; q < Mt; q += 32) {
          const int m = q < M ? q : q - Mt;
          sm.W0[q] = (q == M) ? 0.5 * (sing[2 * M] + sing[0]) : sing[m + M];
        }
        __syncwarp();
        const cplx* Wt = warp_fft_x(sm.W0, sm.W1, Mt, a.twf, a.T, +1);
        cplx* wout = a.weights_out + kidx * a.weights_stride + p * a.w_ld;
        for (int q = lane; q < Mt; q += 32) {
          const cplx w = Wt[q] * (1.0 / Mt);
          const double sv = (isS ? sm.sn[q] : -sm.bt0[q]) / Mt;
          wout[q] = C(w.re, w.im + sv);
        }
        __syncwarp();
      }
    };
    for (int pi = 0; pi < nb; ++pi) {
      const PairInfo pr = bcast(mine, pi);
      const int64_t p = a.out_mod ? (a.out_base + p0 + pi) % a.out_mod : p0 + pi;   // output slot
      if (!pr.valid) {
        if (a.modes_out)
          for (int m = lane; m < 2 * nk * (Mt + 1); m += 32)
            a.modes_out[(p * a.out_nk + a.out_k0) * 2 * (Mt + 1) + m] = 0.0;
        if (a.weights_out)
          for (int kk = 0; kk < nk; ++kk)
            for (int m = lane; m < Mt; m += 32) a.weights_out[kk * a.weights_stride + p * a.w_ld + m] = C(0.0);
        continue;
      }
      const double ra = pr.a, rb = pr.b;
      const double* rr = a.ring_r + pr.ring * 3 * Mt;
      const double* rn = a.ring_n + pr.ring * 3 * Mt;
      const double dts = fabs(pr.t - pr.ts);
      const double qb = exp(-rb), om = -expm1(-rb);
      const bool translated = rb < kSmallB;
      // ---- D1. phases e^{ija}, each from its own sincos: the translated tau_3 combines
      // phase-weighted terms that cancel, so a rotation recurrence's ulp drift would be amplified;
      // e^{-ija} is the conjugate (sin odd, cos even)
      for (int j = lane; j <= M; j += 32) {
        const cplx e = cexpi(j * ra);
        sm.ph[M - j] = conj(e);
        sm.ph[M + j] = e;
      }
      // A_m and B_m(0,b) = -(m - 1/2) e^b (D_m + 2 sinh^2(b/2) A_m) / sinh^2 b from the scratch
      const double shb = sinh(rb), sh2b = sinh(0.5 * rb) * sinh(0.5 * rb);
      const double fac = exp(rb) / (shb * shb);
      auto Am = [&](int m) { return scrA[m * 32 + pi]; };
      auto Bm = [&](int m) { return -(m - 0.5) * fac * (scrD[m * 32 + pi] + 2 * sh2b * scrA[m * 32 + pi]); };
      // ---- D2. circulant transforms: A_{|d|} (|d| <= P/2) and B_{|d|} or B~_{|d|} (|d| <= 2M)
      {
        double sa = 0.0, sb = 0.0;
        for (int pp = lane; pp < P; pp += 32) {
          const int dd = pp <= P / 2 ? pp : P - pp;
          const double av = dd <= L ? Am(dd) : 0.0;
          double bv = 0.0;
          if (dd <= 2 * M) {
            bv = Bm(dd);
            if (translated) bv = (Am(dd) - om * om * bv) / (4 * qb);
          }
          sa += av * av;
          sb += bv * bv;
          sm.W1[pp] = C(av, bv);
        }
        const int eb = pack_exponent(warp_sum(sa), warp_sum(sb));   // B scaled to A's size for the packing
        const double up = ldexp(1.0, eb), down = ldexp(1.0, -eb);
        for (int pp = lane; pp < P; pp += 32) sm.W1[pp].im *= up;
        __syncwarp();
        const cplx* Af = warp_fft(sm.W1, sm.W0, P, a.tw, a.T, -1);
        for (int pp = lane; pp < P; pp += 32) {
          sm.Acal[pp] = Af[pp].re;
          sm.Bcal[pp] = Af[pp].im * down;
        }
      }
      __syncwarp();
      // ---- D3. samples
      double sha, cha;   // sin(a/2), cos(a/2)
      sincos(0.5 * ra, &sha, &cha);
      const double nux = a.kprime ? a.nrm[3 * pr.row] : 0.0, nuy = a.kprime ? a.nrm[3 * pr.row + 1] : 0.0,
                   nuz = a.kprime ? a.nrm[3 * pr.row + 2] : 0.0;
      for (int w = lane; w < (Mt + 31) / 32; w += 32) sm.nearbits[w] = 0u;
      __syncwarp();
      for (int q = lane; q < Mt; q += 32) {
        const double thq = a.thg[3 * q];
        double yx = rr[3 * q] - pr.x, yy = rr[3 * q + 1] - pr.y, yz = rr[3 * q + 2] - pr.z;
        double r2 = yx * yx + yy * yy + yz * yz;
        const bool near = dts + fabs(wrap_pi(pr.th - thq)) <= kStableDelta || r2 <= kStableDist * kStableDist;
        if (near) {
          const R3 Y = diff_ana<double>(a.S, pr.ts, thq, pr.t, pr.th);
          yx = Y.x; yy = Y.y; yz = Y.z;
          r2 = yx * yx + yy * yy + yz * yz;
          atomicOr(&sm.nearbits[q >> 5], 1u << (q & 31));
        }
        const double rinv = rsqrt(r2);
        const double rho = r2 * rinv;
        // sin((th_q - a)/2): direct where th_q - a is small (exact difference, relative accuracy),
        // angle addition from the table elsewhere
        const double dq = thq - ra;
        const double sp = fabs(dq) < 0.1 ? sin(0.5 * dq) : a.thg[3 * q + 1] * cha - a.thg[3 * q + 2] * sha;
        const double s = om * om + 4 * qb * sp * sp;
        const double F = sqrt(s) * rinv;
        double skr, ckr;
        sincos(a.k * rho, &skr, &ckr);
        sm.W0[q] = C(F, ckr);          // F + i cos(k rho)
        sm.sn[q] = skr * rinv;
        const double x = a.k * rho;
        double al, be;
        if (x < kSeriesX) {  // Taylor series of alpha/k^2 and beta/k^3
          const double x2 = x * x;
          double sa = 0.0, sb = 0.0, pw = 1.0, fa = 2.0, fb = 6.0;
          for (int n = 1; n <= 9; ++n) {
            const double sg = (n & 1) ? 1.0 : -1.0;
            sa += sg * (1 - 2 * n) / fa * pw;
            sb += sg * (2 * n) / fb * pw;
            pw *= x2;
            fa *= (2 * n + 1) * (2 * n + 2);
            fb *= (2 * n + 2) * (2 * n + 3);
          }
          al = a.k * a.k * sa;
          be = a.k * a.k * a.k * sb;
        } else {
          const double ri2 = rinv * rinv;   // 1 / rho^2 from the rsqrt already taken (no division)
          al = (1 - ckr - x * skr) * ri2;
          be = (skr - x * ckr) * (ri2 * rinv);
        }
        // tau_0 = nu(y) . (y - x) (K: the source normal) or nu(x) . (x - y) (K': the target's normal);
        // near ones are replaced below
        sm.tau0[q] = a.kprime ? -(nux * yx + nuy * yy + nuz * yz) : rn[3 * q] * yx + rn[3 * q + 1] * yy + rn[3 * q + 2] * yz;
        sm.alph[q] = al;
        sm.bt0[q] = be;
        sm.hr[q] = F;
      }
      __syncwarp();
      {
        // tau_0 of near samples: second-derivative line integral (Section 4 Remark), 16 lanes per
        // sample, two samples at a time, taken from the near bits of D3
        for (int wd = 0; wd < (Mt + 31) / 32; ++wd) {
          unsigned bits = sm.nearbits[wd];
          while (bits) {
            const int qa = __ffs(bits) - 1;
            bits &= bits - 1;
            const int qb = bits ? __ffs(bits) - 1 : -1;
            if (bits) bits &= bits - 1;
          const int qsel = (lane >> 4) ? qb : qa;
          const bool nearq = qsel >= 0;
          const int q = 32 * wd + (nearq ? qsel : 0);
          const double thq = a.thg[3 * q];
          const double dth = wrap_pi(pr.th - thq);
          double acc = 0.0;
          if (nearq) {
            // int_0^1 (lam - 1) nu(v) . D^2 r(v + lam d)[d, d] dlam from the point v whose normal enters:
            // the source (K) or the target (K')
            const int jn = lane & 15;
            const double lam = a.gl.x[jn];
            const double dt = a.kprime ? pr.ts - pr.t : pr.t - pr.ts;
            const double dd = a.kprime ? -dth : dth;
            const double tv = a.kprime ? pr.t : pr.ts, thv = a.kprime ? pr.th : thq;
            const double vx = a.kprime ? nux : rn[3 * q], vy = a.kprime ? nuy : rn[3 * q + 1],
                         vz = a.kprime ? nuz : rn[3 * q + 2];
            Geo G;
            surf_eval(a.S, tv + lam * dt, thv + lam * dd, 2, &G);
            const double qx = G.rtt.x * dt * dt + 2 * G.rtth.x * dt * dd + G.rthth.x * dd * dd;
            const double qy = G.rtt.y * dt * dt + 2 * G.rtth.y * dt * dd + G.rthth.y * dd * dd;
            const double qz = G.rtt.z * dt * dt + 2 * G.rtth.z * dt * dd + G.rthth.z * dd * dd;
            acc = a.gl.w[jn] * (lam - 1) * (vx * qx + vy * qy + vz * qz);
          }
          for (int o = 8; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
          if (nearq && (lane & 15) == 0) sm.tau0[q] = acc;
          __syncwarp();
          }
        }
        __syncwarp();
        for (int q = lane; q < Mt; q += 32) {
          const double F = sm.hr[q], t0 = sm.tau0[q];
          sm.bt0[q] *= t0;              // beta tau_0
          sm.hr[q] = t0 * F * F * F;    // H3 = tau_0 F^3
        }
        __syncwarp();
      }
      // ---- D4. FFT of F + i cos(k rho), upsample; A~ <- F~ A~; S: Toeplitz with A, then its outputs
      cplx* Z1 = warp_fft_x(sm.W0, sm.W1, Mt, a.twf, a.T, -1);
      cplx* Zf = (Z1 == sm.W0) ? sm.W1 : sm.W0;
      double dFa = 0.0;   // F'(a) from the interpolant of F (well conditioned, unlike the direct form)
      if (translated) {
        double acc = 0.0;
        for (int jj = lane; jj <= 2 * M; jj += 32) {
          const int jv = jj - M;
          const cplx zp = Z1[wrapi(jv, Mt)], zm = conj(Z1[wrapi(-jv, Mt)]);
          cplx fj = 0.5 * (zp + zm) * (1.0 / Mt);
          if (jv == M || jv == -M) fj = 0.5 * fj;
          const cplx v = fj * sm.ph[jj];
          acc += -jv * v.im;   // Re(f_j i j e^{ija})
        }
        dFa = warp_sum(acc);
      }
      cplx* up1 = upsample(Z1, sm.ph, Zf, Z1, Mt, P, a.tw, a.twf, a.T, true);   // re: F~, im: C~
      cplx* uf = (up1 == sm.W0) ? sm.W1 : sm.W0;
      for (int pp = lane; pp < P; pp += 32) {
        const double g = up1[pp].re * sm.Acal[pp];   // F~ A~ (kept for V_K)
        sm.Acal[pp] = g;
        if (wantS) uf[pp] = C(up1[pp].im * g, 0.0);
      }
      __syncwarp();
      if (wantS) {
        const cplx* Yf = warp_fft_x(uf, up1, P, a.twf, a.T, -1);
        for (int jj = lane; jj <= 2 * M; jj += 32) sm.kc[jj] = conj(sm.ph[jj]) * Yf[wrapi(jj - M, P)] * (1.0 / P);
        __syncwarp();
        emit(p, 0, true, sm.kc);
      }
      // ---- D5. A~ <- V_K A~ = alpha~ tau0~ F~ A~ on the P grid
      {
        // tau_0 (~ kappa rho^2, amplified ~50x in K) packed with alpha (~k^2/2) scaled to tau_0's size
        double st0 = 0.0, sal = 0.0;
        for (int q = lane; q < Mt; q += 32) {
          st0 += sm.tau0[q] * sm.tau0[q];
          sal += sm.alph[q] * sm.alph[q];
        }
        const int ea = pack_exponent(warp_sum(st0), warp_sum(sal));
        const double up = ldexp(1.0, ea), down = ldexp(1.0, -ea);
        for (int q = lane; q < Mt; q += 32) sm.W0[q] = C(sm.tau0[q], sm.alph[q] * up);
        __syncwarp();
        cplx* Z2 = warp_fft(sm.W0, sm.W1, Mt, a.tw, a.T, -1);
        cplx* Zf2 = (Z2 == sm.W0) ? sm.W1 : sm.W0;
        cplx* up2 = upsample(Z2, sm.ph, Zf2, Z2, Mt, P, a.tw, a.twf, a.T, false);   // re: tau0~, im: 2^ea alpha~
        for (int pp = lane; pp < P; pp += 32) sm.Acal[pp] = up2[pp].re * (up2[pp].im * down) * sm.Acal[pp];
      }
      __syncwarp();
      // ---- D6. H3 modes (symmetric) from a transform of H3 alone: their rounding is amplified in the
      // tau_3 term (and by up to k^2 in the translated remainder next to a), so nothing larger shares it
      // (kk: kc is spent)
      for (int q = lane; q < Mt; q += 32) sm.W0[q] = C(sm.hr[q], 0.0);
      __syncwarp();
      const cplx* Z3 = warp_fft(sm.W0, sm.W1, Mt, a.tw, a.T, -1);
      for (int jj = lane; jj <= 2 * M; jj += 32) {
        const int jv = jj - M;
        const cplx zp = Z3[wrapi(jv, Mt)], zm = conj(Z3[wrapi(-jv, Mt)]);
        cplx h = 0.5 * (zp + zm) * (1.0 / Mt);
        if (jv == M || jv == -M) h = 0.5 * h;
        sm.kk[jj] = h;
      }
      __syncwarp();
      double H3a = 0.0, H3pa = 0.0;
      if (translated) {
        // ---- D7. H3(a), H3'(a) directly from the geometry at th_s = a
        Geo G;
        surf_eval(a.S, pr.ts, ra, 2, &G);
        R3 Y = {G.r.x - pr.x, G.r.y - pr.y, G.r.z - pr.z};
        const bool neara = dts + fabs(wrap_pi(ra - pr.th)) <= kStableDelta || dot(Y, Y) <= kStableDist * kStableDist;
        if (neara) Y = diff_ana<double>(a.S, pr.ts, ra, pr.t, pr.th);
        const R3 n = cross(G.rt, G.rth);
        const double J = sqrt(dot(n, n));
        const R3 nu = {n.x / J, n.y / J, n.z / J};
        const R3 dn1 = cross(G.rtth, G.rth), dn2 = cross(G.rt, G.rthth);
        const R3 dn = {dn1.x + dn2.x, dn1.y + dn2.y, dn1.z + dn2.z};
        const double nd = dot(nu, dn);
        const R3 dnu = {(dn.x - nu.x * nd) / J, (dn.y - nu.y * nd) / J, (dn.z - nu.z * nd) / J};
        // K: tau_0(a) = nu(a) . Y, tau_0'(a) = nu'(a) . Y (+ nu . r_th = 0);
        // K': tau_0(a) = -nu(x) . Y, tau_0'(a) = -nu(x) . r_th(t_s, a)
        const R3 nux3 = {nux, nuy, nuz};
        double t0a = a.kprime ? -dot(nux3, Y) : dot(nu, Y);
        if (neara) {
          double acc = 0.0;
          if (lane < 16) {
            const double lam = a.gl.x[lane];
            const double dt = a.kprime ? pr.ts - pr.t : pr.t - pr.ts;
            const double dth = a.kprime ? wrap_pi(ra - pr.th) : wrap_pi(pr.th - ra);
            const double tv = a.kprime ? pr.t : pr.ts, thv = a.kprime ? pr.th : ra;
            const R3 nv = a.kprime ? nux3 : nu;
            Geo H;
            surf_eval(a.S, tv + lam * dt, thv + lam * dth, 2, &H);
            const double qx = H.rtt.x * dt * dt + 2 * H.rtth.x * dt * dth + H.rthth.x * dth * dth;
            const double qy = H.rtt.y * dt * dt + 2 * H.rtth.y * dt * dth + H.rthth.y * dth * dth;
            const double qz = H.rtt.z * dt * dt + 2 * H.rtth.z * dt * dth + H.rthth.z * dth * dth;
            acc = a.gl.w[lane] * (lam - 1) * (nv.x * qx + nv.y * qy + nv.z * qz);
          }
          t0a = warp_sum(acc);
        }
        const double r2a = dot(Y, Y);
        const double Fa = om / sqrt(r2a);
        const double dt0 = a.kprime ? -dot(nux3, G.rth) : dot(dnu, Y);
        H3a = t0a * Fa * Fa * Fa;
        H3pa = dt0 * Fa * Fa * Fa + 3 * t0a * Fa * Fa * dFa;
        // ---- D8. remainder R on the grid (stable sum within kNearPhi of a); modes d_k
        for (int q = lane; q < Mt; q += 32) {
          const double phq = wrap_pi(kTwoPi * q / Mt - ra);
          const double s2 = sin(0.5 * phq) * sin(0.5 * phq);
          sm.tau0[q] = (fabs(phq) < kNearPhi) ? 0.0 : (sm.hr[q] - H3a - H3pa * sin(phq)) / s2;
        }
        __syncwarp();
        // only the grid angles within kNearPhi of a: those next to the nearest one
        const int qc = (int)rint(ra * (Mt / kTwoPi));
        const int qr = (int)(kNearPhi * Mt / kTwoPi) + 2;
        for (int dq = -qr; dq <= qr; ++dq) {
          const int q = wrapi(qc + dq, Mt);
          const double phq = wrap_pi(kTwoPi * q / Mt - ra);
          if (!(fabs(phq) < kNearPhi)) continue;
          const double sh = sin(0.5 * phq), s2 = sh * sh, rs2 = 1.0 / s2, sph = sin(phq);
          // modes k and -k share |k|'s factors (the real one even, the imaginary one odd in k);
          // k = 0 contributes nothing
          double acc = 0.0;
          for (int ka = lane + 1; ka <= M; ka += 32) {
            const cplx hp = sm.kk[M + ka] * sm.ph[M + ka], hm = sm.kk[M - ka] * sm.ph[M - ka];   // h3_k e^{ika}
            double gre, gim;
            if (s2 == 0.0) {
              gre = -2.0 * ka * ka;
              gim = 0.0;
            } else {
              double sk, ck;   // sin, cos of k phq / 2; sin(k phq) = 2 sk ck
              sincos(0.5 * ka * phq, &sk, &ck);
              gre = -2.0 * sk * sk * rs2;
              gim = sin_k_minus(ka, phq, 2.0 * sk * ck, sph) * rs2;
            }
            acc += (hp.re + hm.re) * gre - (hp.im - hm.im) * gim;
          }
          acc = warp_sum(acc);
          if (lane == 0) sm.tau0[q] = acc;
          __syncwarp();
        }
        __syncwarp();
        for (int q = lane; q < Mt; q += 32) sm.W0[q] = C(sm.tau0[q], 0.0);
        __syncwarp();
        const cplx* Zr = warp_fft(sm.W0, sm.W1, Mt, a.tw, a.T, -1);
        for (int jj = lane; jj <= 2 * M; jj += 32) {
          const int jv = jj - M;
          cplx dv = Zr[wrapi(jv, Mt)] * (1.0 / Mt);
          if (jv == M || jv == -M) dv = 0.5 * dv;
          sm.kk[jj] = dv;        // kk now holds d_k
        }
        __syncwarp();
      }
      // ---- D9. upsample h3 (or d); B~ <- V_H = h3~ B~.  The upsampled signal is real: with
      // E_k = X_k + X_{k+P/2}, O_k = e^{2 pi i k / P} (X_k - X_{k+P/2}), the inverse transform of length
      // P/2 of E + i O holds the even samples in its real parts and the odd ones in its imaginary
      // parts, i.e. sample pp at double pp.  X_k = e^{ika} h_k sits at k <= M and P - M <= k.
      {
        const int P2 = P / 2;
        for (int pp = lane; pp < P2; pp += 32) sm.W0[pp] = C(0.0);
        __syncwarp();
        for (int jj = lane; jj <= 2 * M; jj += 32) {
          const int kv = jj - M;
          const int kz = kv >= 0 ? kv : P2 + kv;
          const cplx x = sm.ph[jj] * sm.kk[jj];
          const cplx iw = C(0.0, kv >= 0 ? 1.0 : -1.0) * tw64(a.tw, kz * (a.T / P), +1);   // +-i e^{2 pi i kz / P}
          sm.W0[kz] = x + iw * x;
        }
        __syncwarp();
        const double* up3 = reinterpret_cast<const double*>(warp_fft(sm.W0, sm.W1, P2, a.tw, a.T, +1));
        for (int pp = lane; pp < P; pp += 32) sm.Bcal[pp] = up3[pp] * sm.Bcal[pp];
        __syncwarp();
      }
      // ---- D10. transform (V_K A~) + i (V_H), unpack AT1 and the tau_3 Toeplitz part
      double y2down;
      {
        double sk = 0.0, sh = 0.0;
        for (int pp = lane; pp < P; pp += 32) {
          sk += sm.Acal[pp] * sm.Acal[pp];
          sh += sm.Bcal[pp] * sm.Bcal[pp];
        }
        const int ey = pack_exponent(warp_sum(sk), warp_sum(sh));   // V_H scaled to V_K A~'s size
        const double up = ldexp(1.0, ey);
        y2down = ldexp(1.0, -ey) / P;
        for (int pp = lane; pp < P; pp += 32) sm.W0[pp] = C(sm.Acal[pp], sm.Bcal[pp] * up);
      }
      __syncwarp();
      const cplx* Y2 = warp_fft(sm.W0, sm.W1, P, a.tw, a.T, -1);
      for (int jj = lane; jj <= 2 * M; jj += 32) {
        const int m = jj - M;
        const cplx zp = Y2[wrapi(m, P)], zm = conj(Y2[wrapi(-m, P)]);
        const cplx y1 = 0.5 * (zp + zm) * (1.0 / P);
        const cplx y2 = C(0.5 * (zp.im - zm.im), -0.5 * (zp.re - zm.re)) * y2down;
        const cplx e = conj(sm.ph[jj]);                                  // e^{-ima}
        cplx t3 = e * y2;
        if (translated) {
          // H3(a) B_n(a,b) + H3'(a)/(2i) e^{-ina} (B_{|n-1|} - B_{|n+1|}), with the exact
          // cancellation-free B_{n-1} - B_{n+1} = 2 n e^b A_{|n|}
          const int ma = m < 0 ? -m : m;
          const cplx expl = C(H3a * Bm(ma), -H3pa * m * exp(rb) * Am(ma));
          t3 = t3 + e * expl;
        }
        sm.kk[jj] = e * y1 - t3;   // swapped part of K (kk was consumed in D9)
      }
      __syncwarp();
      // ---- D11. double-layer outputs
      emit(p, nk - 1, false, sm.kk);
    }
    }
    __syncwarp();
}

template <bool kWithK>
__global__ void __launch_bounds__(32 * kMaxWarpsPerBlock, 1) pair_kernel(const __grid_constant__ PairArgs a) {
  extern __shared__ double smem[];
  const int wib = threadIdx.x >> 5;
  const size_t per_warp = smem_doubles(a.Mt, a.P, a.L, kWithK);
  const Smem sm = carve(smem + per_warp * wib, a.Mt, a.P, a.L, kWithK);
  const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double* scrA = a.scratch + gwarp * a.scratch_per_warp;
  double* scrD = scrA + (int64_t)(a.L + 1) * 32;
  for (int64_t p0 = gwarp * 32; p0 < a.n_pairs; p0 += nwarps * 32)
    process_batch<kWithK>(a, sm, scrA, scrD, p0, (int)min((int64_t)32, a.n_pairs - p0));
}

// ------------------------------------------------------------------ single layer: split launch
// The root kernel runs phases A-C (FP64; lane per pair for the root and the recurrence; no shared
// memory) and writes one record per pair; the transform kernel runs phase D on the records (double
// words, shared-memory FFTs).  Each kernel gets its own register and occupancy budget.  Both cover
// the pairs [c0, c0 + cn) of the launch; the record of pair p is p - c0.
__global__ void __launch_bounds__(128, 4) pair_root_kernel(const __grid_constant__ PairArgs a, int64_t c0, int64_t cn) {
  __shared__ int near_list[4][kNearList];   // phase A's near samples, per warp
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int Mt = a.Mt, L = a.L;
  for (int64_t p0 = c0 + gwarp * 32; p0 < c0 + cn; p0 += nwarps * 32) {
    const int nb = (int)min((int64_t)32, c0 + cn - p0);
    const int64_t r0 = p0 - c0;
    PairInfo mine;
    unsigned vm;
    front_batch<false>(a, Smem{}, p0, nb, a.rec_R2 + r0 * Mt, a.rec_E + r0 * 33, a.rec_A + r0 * (L + 1), L + 1, 1,
                       nullptr, mine, vm, near_list[threadIdx.x >> 5]);
    if (lane < nb) {
      double* h = a.rec_hdr + (r0 + lane) * 8;
      h[0] = mine.a;
      h[1] = mine.qb;
      h[2] = mine.om;
      h[3] = mine.sha;
      h[4] = mine.cha;
      h[5] = mine.valid ? 1.0 : 0.0;
    }
  }
}

template <class Ar>
__global__ void __launch_bounds__(32 * kMaxWarpsPerBlock)
    pair_transform_kernel(const __grid_constant__ PairArgs a, int64_t c0, int64_t cn) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const size_t per_warp = smem_doubles(a.Mt, a.P, a.L, false);
  const Smem sm = carve(smem + per_warp * wib, a.Mt, a.P, a.L, false);
  const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int Mt = a.Mt, L = a.L;
  for (int64_t p0 = c0 + gwarp * 32; p0 < c0 + cn; p0 += nwarps * 32) {
    const int nb = (int)min((int64_t)32, c0 + cn - p0);
    const int64_t r0 = p0 - c0;
    PairInfo mine = {};
    if (lane < nb) {
      const double* h = a.rec_hdr + (r0 + lane) * 8;
      mine.a = h[0];
      mine.qb = h[1];
      mine.om = h[2];
      mine.sha = h[3];
      mine.cha = h[4];
      mine.valid = h[5] != 0.0;
    }
    const unsigned vm = __ballot_sync(0xffffffffu, lane < nb && mine.valid);
    phase_d_single<Ar>(a, sm, reinterpret_cast<const typename Ar::R*>(a.rec_A + r0 * (L + 1)), L + 1, 1,
                       reinterpret_cast<const typename Ar::C*>(a.rec_E + r0 * 33),
                   a.rec_R2 + r0 * Mt, mine, vm, p0, nb);
  }
}

// ------------------------------------------------------------------ host side
// Columns 2, 3 serve Miller's recurrence A~_{m-1} = c_m cosh(b) A~_m - d_m A~_{m+1}, c_m = 4m/(2m-1),
// d_m = (2m+1)/(2m-1), rescaled as A~_m = w_m B_m with w_{m+1} = w_{m-1} / d_m (w_0 = w_1 = 1) so that
// B_{m-1} = t_m cosh(b) B_m - B_{m+1}, t_m = c_m w_m / w_{m-1}: one multiply and one FMA a step.
static std::vector<double> recurrence_table(int n) {
  std::vector<double> r(4 * (size_t)n, 0.0);
  std::vector<long double> w(n + 1, 1.0L);
  for (int m = 1; m < n; ++m) w[m + 1] = w[m - 1] * (2.0L * m - 1) / (2.0L * m + 1);
  r[3] = 1.0;
  for (int m = 1; m < n; ++m) {
    const long double mm = m;
    r[4 * m + 0] = (double)((2 * mm - 1) / (2 * mm + 1));
    r[4 * m + 1] = (double)((8 * mm) / (2 * mm + 1));
    r[4 * m + 2] = (double)((4 * mm) / (2 * mm - 1) * w[m] / w[m - 1]);
    r[4 * m + 3] = (double)w[m];
  }
  return r;
}

// Recurrence coefficient table, one per device, allocated once at the size the largest grid of the
// library needs (Mth <= 1024: L <= 2048) and never freed, so that plans and captured graphs holding
// its address stay valid for the life of the process.
constexpr int kMaxMtLib = 1024;
constexpr int kRecLenMax = (int)(3.8 * 2 * kMaxMtLib) + 64;   // Miller needs N < 3.8 L + 17 (it runs only when L b > 7)
static double* g_rec[64];
static std::mutex g_rec_mu;

// grow a context-owned device buffer (stream-synchronised free of the old one)
static bie_status grow(bie_ctx ctx, double** buf, size_t* have, size_t need, const char* what) {
  if (*have >= need) return BIE_OK;
  cudaStreamSynchronize(ctx->stream);
  if (*buf) cudaFree(*buf);
  *buf = nullptr;
  *have = 0;
  const cudaError_t e = cudaMalloc((void**)buf, need);
  if (e != cudaSuccess) return cuda_fail(e, what);
  *have = need;
  return BIE_OK;
}

PairArgs make_pair_args(bie_surface s, double k, unsigned kernels) {
  PairArgs a = {};
  a.S = s->sp;
  a.gl = s->gl01;
  a.Np = s->Np;
  a.Mt = s->Mt;
  a.M = s->Mt / 2;
  a.kernels = (int)kernels;
  const bool withK = kernels & (BIE_KERNEL_K | BIE_KERNEL_KP);
  a.kprime = (kernels & BIE_KERNEL_KP) ? 1 : 0;
  a.fp64_transforms = s->ctx->fp64_transforms;
  a.out_nk = ((kernels & BIE_KERNEL_S) ? 1 : 0) + (withK ? 1 : 0);
  a.out_k0 = 0;
  a.P = (withK ? 4 : 3) * s->Mt;
  a.L = (withK ? 4 : 3) * a.M;
  a.T = s->tw_len;
  a.h = s->h;
  a.k = k;
  a.N = s->N;
  a.t_nodes = s->t_nodes;
  a.pts = s->pts;
  a.nrm = s->nrm;
  a.ring_t = s->ring_t;
  a.ring_r = s->ring_r;
  a.ring_n = s->ring_n;
  a.tw = s->tw;
  a.twf = s->twf;
  a.thg = s->thgrid;
  a.w_ld = s->Mt;
  a.status = s->ctx->d_status;
  return a;
}

int pair_warps_per_block(int Mt, unsigned kernels) {
  // the CTA shape (1, 2 or 4 warps) with the most resident warps per SM
  const bool withK = kernels & (BIE_KERNEL_K | BIE_KERNEL_KP);
  const int P = (withK ? 4 : 3) * Mt, L = (withK ? 4 : 3) * (Mt / 2);
  const size_t per = smem_doubles(Mt, P, L, withK) * sizeof(double);
  auto kern = withK ? pair_kernel<true> : pair_kernel<false>;
  int best = 0, best_w = 0;
  for (int w = kMaxWarpsPerBlock; w >= 1; w /= 2) {
    if (per * w > kSmemLimit) continue;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(per * w)) != cudaSuccess) continue;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, 32 * w, per * w) != cudaSuccess) continue;
    if (nb * w > best_w) { best_w = nb * w; best = w; }
  }
  return best;
}

static bie_status ensure_rec(bie_ctx ctx, int L, const double** rec, int* rec_len) {
  if (L < 0 || L > 2 * kMaxMtLib) { set_error("recurrence table: L = %d beyond the library limit", L); return BIE_EINVAL; }
  const bie_status ds = check_device(ctx, "pair pipeline");
  if (ds != BIE_OK) return ds;
  if (ctx->device < 0 || ctx->device >= 64) { set_error("pair pipeline: device ordinal out of range"); return BIE_EINVAL; }
  std::lock_guard<std::mutex> lock(g_rec_mu);
  double*& t = g_rec[ctx->device];
  if (!t) {
    const std::vector<double> r = recurrence_table(kRecLenMax);
    double* d = nullptr;
    cudaError_t e = cudaMalloc((void**)&d, sizeof(double) * r.size());
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(recurrence table)");
    e = cudaMemcpy(d, r.data(), sizeof(double) * r.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { cudaFree(d); return cuda_fail(e, "cudaMemcpy(recurrence table)"); }
    t = d;
  }
  *rec = t;
  *rec_len = kRecLenMax;
  return BIE_OK;
}

// pairs per chunk of the split launch (records: (74 + L + 1 + Mt) doubles per pair, 3.5 GB at Mt = 128)
constexpr int64_t kSplitChunk = 1 << 20;

static bie_status launch_pairs_split(bie_surface s, PairArgs& a) {
  const cudaStream_t st = s->ctx->stream;
  bie_status rs = ensure_rec(s->ctx, a.L, &a.rec, &a.rec_len);
  if (rs != BIE_OK) return rs;
  const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(a.n_pairs, kSplitChunk));
  const int64_t per_pair = 8 + 2 * 33 + (a.L + 1) + a.Mt;
  const size_t rbytes = sizeof(double) * (size_t)(per_pair * chunk);
  cudaError_t e;
  rs = grow(s->ctx, &s->ctx->pair_records, &s->ctx->pair_records_bytes, rbytes, "cudaMalloc(pair records)");
  if (rs != BIE_OK) return rs;
  double* records = s->ctx->pair_records;
  a.rec_hdr = records;
  a.rec_E = reinterpret_cast<float4*>(records + 8 * chunk);
  a.rec_A = records + (8 + 2 * 33) * chunk;
  a.rec_R2 = a.rec_A + (a.L + 1) * chunk;
  // root kernel: register-limited occupancy, no shared memory
  int per_r = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_r, pair_root_kernel, 128, 0);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy(pair_root_kernel)");
  if (per_r < 1) per_r = 1;
  // transform kernel (double words, or FP64 when the context asks): the CTA shape (1, 2 or 4 warps) with
  // the most resident warps
  auto tkern = a.fp64_transforms ? pair_transform_kernel<ArF64> : pair_transform_kernel<ArDW>;
  const size_t per_w = smem_doubles(a.Mt, a.P, a.L, false) * sizeof(double);
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, tkern);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncGetAttributes(pair transform kernel)");
  int wpb = 0, best_w = 0, per_t = 0;
  for (int w = kMaxWarpsPerBlock; w >= 1; w /= 2) {
    if (per_w * w > kSmemLimit || 32 * w > fa.maxThreadsPerBlock) continue;
    if (cudaFuncSetAttribute(tkern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(per_w * w)) != cudaSuccess)
      continue;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, tkern, 32 * w, per_w * w) != cudaSuccess) continue;
    if (nb * w > best_w) { best_w = nb * w; wpb = w; per_t = nb; }
  }
  if (wpb < 1) { set_error("pair transform kernel: Mth = %d needs more shared memory than a CTA has", a.Mt); return BIE_EUNSUPPORTED; }
  const size_t smem = per_w * wpb;
  e = cudaFuncSetAttribute(tkern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(pair_transform_kernel)");
  for (int64_t c0 = 0; c0 < a.n_pairs; c0 += chunk) {
    const int64_t cn = std::min(chunk, a.n_pairs - c0);
    const int64_t br = std::max<int64_t>(1, std::min<int64_t>((int64_t)s->ctx->sms * per_r, (cn + 127) / 128));
    int tm = trace_begin(s->ctx, kTracePairRoot);
    pair_root_kernel<<<(unsigned)br, 128, 0, st>>>(a, c0, cn);
    trace_end(s->ctx, tm);
    const int64_t bt = std::max<int64_t>(1, std::min<int64_t>((int64_t)s->ctx->sms * per_t, (cn + 32 * wpb - 1) / (32 * wpb)));
    tm = trace_begin(s->ctx, kTracePairTransform);
    tkern<<<(unsigned)bt, 32 * wpb, smem, st>>>(a, c0, cn);
    trace_end(s->ctx, tm);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "pair kernels (split launch)");
  return BIE_OK;
}

bie_status launch_pairs(bie_surface s, PairArgs& a) {
  const bool withK = a.kernels & (BIE_KERNEL_K | BIE_KERNEL_KP);
  if (!withK) return launch_pairs_split(s, a);
  const int wpb = pair_warps_per_block(a.Mt, (unsigned)a.kernels);
  if (wpb < 1) { set_error("pair kernel: Mth = %d needs more shared memory than a CTA has", a.Mt); return BIE_EUNSUPPORTED; }
  const size_t smem = smem_doubles(a.Mt, a.P, a.L, withK) * sizeof(double) * wpb;
  auto kern = withK ? pair_kernel<true> : pair_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(pair_kernel)");
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * wpb, smem);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy(pair_kernel)");
  if (per_sm < 1) { set_error("pair kernel does not fit (shared memory %zu bytes)", smem); return BIE_EUNSUPPORTED; }
  int64_t blocks = (int64_t)s->ctx->sms * per_sm;
  const int64_t need = (a.n_pairs + 32 * wpb - 1) / (32 * wpb);
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  {
    const bie_status rs = ensure_rec(s->ctx, a.L, &a.rec, &a.rec_len);
    if (rs != BIE_OK) return rs;
  }
  a.scratch_per_warp = pair_scratch_per_warp(a.L, withK, a.Mt);
  const size_t sbytes = sizeof(double) * (size_t)a.scratch_per_warp * (size_t)blocks * wpb;
  {
    const bie_status rs = grow(s->ctx, &s->ctx->pair_scratch, &s->ctx->pair_scratch_bytes, sbytes,
                               "cudaMalloc(pair scratch)");
    if (rs != BIE_OK) return rs;
  }
  a.scratch = s->ctx->pair_scratch;
  const int tm = trace_begin(s->ctx, kTracePairFused);
  kern<<<(unsigned)blocks, 32 * wpb, smem, s->ctx->stream>>>(a);
  trace_end(s->ctx, tm);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "pair_kernel launch");
  return BIE_OK;
}

}  // namespace bie

using namespace bie;

extern "C" bie_status bie_kernel_modes(bie_ctx ctx, bie_surface s, unsigned kernels, double k,
                                       const int64_t* pair_row, const int32_t* pair_src, int64_t n_pairs,
                                       double* modes_out) {
  if (!ctx || !s || n_pairs < 0 || (n_pairs > 0 && (!pair_row || !pair_src || !modes_out))) {
    set_error("bie_kernel_modes: invalid arguments");
    return BIE_EINVAL;
  }
  if (!(k > 0) || !(k < 1e6)) { set_error("bie_kernel_modes: k must be in (0, 1e6)"); return BIE_EINVAL; }
  if (kernels == 0 || (kernels & ~(BIE_KERNEL_S | BIE_KERNEL_K | BIE_KERNEL_KP))) {
    set_error("bie_kernel_modes: bad kernel mask %u", kernels);
    return BIE_EINVAL;
  }
  if (n_pairs == 0) return BIE_OK;
  // one launch per double-layer kind: (S and) K or K' first, then K' alone when both are asked
  const int total = __builtin_popcount(kernels);
  const unsigned first = (kernels & BIE_KERNEL_S) | ((kernels & BIE_KERNEL_K) ? BIE_KERNEL_K : (kernels & BIE_KERNEL_KP));
  PairArgs a = make_pair_args(s, k, first);
  a.rows = pair_row;
  a.srcs = pair_src;
  a.n_pairs = n_pairs;
  a.modes_out = modes_out;
  a.out_nk = total;
  bie_status st = launch_pairs(s, a);
  if (st != BIE_OK || first == kernels) return st;
  PairArgs b = make_pair_args(s, k, BIE_KERNEL_KP);
  b.rows = pair_row;
  b.srcs = pair_src;
  b.n_pairs = n_pairs;
  b.modes_out = modes_out;
  b.out_nk = total;
  b.out_k0 = total - 1;
  return launch_pairs(s, b);
}

// ------------------------------------------------------------------ allocation-free variant
// For callers that must not allocate device memory.  The pair kernel's scratch (the
// A_m / D_m tables of every resident warp) and the recurrence coefficient table live in
// file-scope device arrays, sized for Mth <= kNoAllocMaxMt and a fixed grid of
// kNoAllocBlocks CTAs of kMaxWarpsPerBlock warps (the grid-stride loop covers any number
// of pairs).  Every call shares these arrays.
namespace bie {
constexpr int kNoAllocMaxMt = 128;
constexpr int kNoAllocBlocks = 32;
constexpr int kNoAllocMaxL = 2 * kNoAllocMaxMt;                 // L = 4M with the double layer
constexpr int kNoAllocRecLen = (int)(3.8 * kNoAllocMaxL) + 64;
constexpr size_t kNoAllocScratchDoubles =
    (size_t)kNoAllocBlocks * kMaxWarpsPerBlock * 2 * (kNoAllocMaxL + 1) * 32;   // 16.8 MB
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];
static __device__ __align__(256) double g_noalloc_rec[4 * kNoAllocRecLen];

struct NoAllocState {
  bool ready = false;
  double* scratch = nullptr;
  double* rec = nullptr;
};
static NoAllocState g_noalloc[64];   // per device ordinal
}  // namespace bie

extern "C" bie_status bie_kernel_modes_noalloc(bie_ctx ctx, bie_surface s, unsigned kernels, double k,
                                               const int64_t* pair_row, const int32_t* pair_src, int64_t n_pairs,
                                               double* modes_out) {
  if (!ctx || !s || n_pairs < 0 || (n_pairs > 0 && (!pair_row || !pair_src || !modes_out))) {
    set_error("bie_kernel_modes_noalloc: invalid arguments");
    return BIE_EINVAL;
  }
  if (!(k > 0) || !(k < 1e6)) { set_error("bie_kernel_modes_noalloc: k must be in (0, 1e6)"); return BIE_EINVAL; }
  if (kernels == 0 || (kernels & ~(BIE_KERNEL_S | BIE_KERNEL_K))) {
    set_error("bie_kernel_modes_noalloc: bad kernel mask %u", kernels);
    return BIE_EINVAL;
  }
  if (s->Mt > kNoAllocMaxMt) {
    set_error("bie_kernel_modes_noalloc: m_theta %d exceeds the fixed maximum %d of the static scratch", s->Mt,
              kNoAllocMaxMt);
    return BIE_EINVAL;
  }
  if (ctx->device < 0 || ctx->device >= 64) { set_error("bie_kernel_modes_noalloc: device ordinal out of range"); return BIE_EINVAL; }
  if (n_pairs == 0) return BIE_OK;
  // every call: the symbol addresses below belong to the context's device, so it must be current
  {
    const bie_status ds = check_device(ctx, "bie_kernel_modes_noalloc");
    if (ds != BIE_OK) return ds;
  }
  NoAllocState& st = g_noalloc[ctx->device];
  if (!st.ready) {
    // once per device, with that device current: device addresses of the static arrays and the
    // recurrence coefficients (a copy into the static table, no allocation)
    cudaError_t e = cudaGetSymbolAddress((void**)&st.scratch, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(scratch)");
    e = cudaGetSymbolAddress((void**)&st.rec, g_noalloc_rec);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(recurrence table)");
    const std::vector<double> r = recurrence_table(kNoAllocRecLen);
    e = cudaMemcpyToSymbol(g_noalloc_rec, r.data(), sizeof(double) * r.size());
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyToSymbol(recurrence table)");
    st.ready = true;
  }
  PairArgs a = make_pair_args(s, k, kernels);
  a.fp64_transforms = 0;   // the fused kernel's single layer runs in double words
  a.rows = pair_row;
  a.srcs = pair_src;
  a.n_pairs = n_pairs;
  a.modes_out = modes_out;
  const bool withK = kernels & BIE_KERNEL_K;
  const int wpb = pair_warps_per_block(a.Mt, kernels);   // <= kMaxWarpsPerBlock, the scratch sizing
  if (wpb < 1) { set_error("bie_kernel_modes_noalloc: shared memory does not fit"); return BIE_EUNSUPPORTED; }
  const size_t smem = smem_doubles(a.Mt, a.P, a.L, withK) * sizeof(double) * wpb;
  auto kern = withK ? pair_kernel<true> : pair_kernel<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(pair_kernel)");
  a.rec = st.rec;
  a.rec_len = kNoAllocRecLen;
  a.scratch = st.scratch;
  a.scratch_per_warp = pair_scratch_per_warp(a.L, withK, a.Mt);   // <= 2 (kNoAllocMaxL + 1) 32
  kern<<<kNoAllocBlocks, 32 * wpb, smem, ctx->stream>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "pair_kernel launch (no-alloc)");
  return BIE_OK;
}

// ------------------------------------------------------------------ batch scheduler
// Many surfaces of uneven size (panels, Mth, k) in a few launches.  The near pairs of every surface
// are cut into items of item_pairs pairs and grouped by grid size Mth into classes, largest first.
//  * Single layer alone: each class runs in chunks through the two kernels of the single-surface path
//    (the root kernel, then the transform kernel over per-pair records), each at the shared-memory
//    carve and occupancy of the class's own Mth; warps take the chunk's 32-pair batches in a fixed
//    order (the work of a batch hardly varies within a class).
//  * With a double layer: one persistent launch of the fused kernel per class, resident warps
//    claiming the class's items from an atomic counter (longest work first across classes).
// Nothing is allocated by a run, so a run can be captured in a CUDA graph.
namespace bie {
struct BatchItem {
  int surf;
  int n;
  int64_t p0;   // first enumerated pair of the item within its surface
};

// per-pair records of one chunk of a class (split path)
struct BatchRec {
  double* hdr;
  float4* E;
  double* A;
  double* R2;
  int Mt, L;
};

template <bool kWithK>
__global__ void __launch_bounds__(32 * kMaxWarpsPerBlock)
    pair_batch_kernel(const PairArgs* __restrict__ surfs, const BatchItem* __restrict__ items, int it0, int it1,
                      int* __restrict__ counter, double* __restrict__ scratch, int64_t scratch_per_warp, int Mt) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const size_t per_warp = smem_doubles(Mt, (kWithK ? 4 : 3) * Mt, (kWithK ? 4 : 3) * (Mt / 2), kWithK);
  double* wbase = smem + per_warp * wib;
  const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  double* scrA = scratch + gwarp * scratch_per_warp;
  for (int guard = 0; guard <= it1 - it0; ++guard) {   // each pass claims one item; bounded by the list length
    int it = 0;
    if (lane == 0) it = it0 + atomicAdd(counter, 1);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= it1) break;
    const BatchItem item = items[it];
    const PairArgs& a = surfs[item.surf];
    const Smem sm = carve(wbase, a.Mt, a.P, a.L, kWithK);
    double* scrD = scrA + (int64_t)(a.L + 1) * 32;
    for (int q = 0; q < item.n; q += 32) process_batch<kWithK>(a, sm, scrA, scrD, item.p0 + q, min(32, item.n - q));
  }
}

// 32-pair batch wb of a chunk of items [it0, it0 + nit): item it0 + wb / (item_pairs / 32), offset
// (wb mod (item_pairs / 32)) * 32 in it; its records start at slot 32 wb of the chunk.
__global__ void __launch_bounds__(128, 4)
    pair_root_batch_kernel(const PairArgs* __restrict__ surfs, const BatchItem* __restrict__ items, int it0, int nit,
                           int item_pairs, const BatchRec rec) {
  __shared__ int near_list[4][kNearList];   // phase A's near samples, per warp
  const int lane = threadIdx.x & 31;
  const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int wpi = item_pairs / 32;
  for (int64_t wb = gwarp; wb < (int64_t)nit * wpi; wb += nwarps) {
    const BatchItem item = items[it0 + wb / wpi];
    const int off = (int)(wb % wpi) * 32;
    if (off >= item.n) continue;
    const PairArgs& a = surfs[item.surf];
    const int nb = min(32, item.n - off);
    const int64_t r0 = wb * 32;
    PairInfo mine;
    unsigned vm;
    front_batch<false>(a, Smem{}, item.p0 + off, nb, rec.R2 + r0 * rec.Mt, rec.E + r0 * 33, rec.A + r0 * (rec.L + 1),
                       rec.L + 1, 1, nullptr, mine, vm, near_list[threadIdx.x >> 5]);
    if (lane < nb) {
      double* h = rec.hdr + (r0 + lane) * 8;
      h[0] = mine.a;
      h[1] = mine.qb;
      h[2] = mine.om;
      h[3] = mine.sha;
      h[4] = mine.cha;
      h[5] = mine.valid ? 1.0 : 0.0;
    }
  }
}

__global__ void __launch_bounds__(32 * kMaxWarpsPerBlock)
    pair_transform_batch_kernel(const PairArgs* __restrict__ surfs, const BatchItem* __restrict__ items, int it0,
                                int nit, int item_pairs, const BatchRec rec) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int Mt = rec.Mt, L = rec.L;
  const size_t per_warp = smem_doubles(Mt, 3 * Mt, L, false);
  const Smem sm = carve(smem + per_warp * wib, Mt, 3 * Mt, L, false);
  const int64_t gwarp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int wpi = item_pairs / 32;
  for (int64_t wb = gwarp; wb < (int64_t)nit * wpi; wb += nwarps) {
    const BatchItem item = items[it0 + wb / wpi];
    const int off = (int)(wb % wpi) * 32;
    if (off >= item.n) continue;
    const PairArgs& a = surfs[item.surf];
    const int nb = min(32, item.n - off);
    const int64_t r0 = wb * 32;
    PairInfo mine = {};
    if (lane < nb) {
      const double* h = rec.hdr + (r0 + lane) * 8;
      mine.a = h[0];
      mine.qb = h[1];
      mine.om = h[2];
      mine.sha = h[3];
      mine.cha = h[4];
      mine.valid = h[5] != 0.0;
    }
    const unsigned vm = __ballot_sync(0xffffffffu, lane < nb && mine.valid);
    phase_d_single<ArDW>(a, sm, reinterpret_cast<const float2*>(rec.A + r0 * (L + 1)), L + 1, 1, rec.E + r0 * 33,
                   rec.R2 + r0 * Mt, mine, vm, item.p0 + off, nb);
  }
}

constexpr int kMaxBatchClasses = 64;   // distinct grid sizes in one plan

struct BatchClass {
  int Mt;
  int it_begin, it_end;   // item range of the class (items sorted by decreasing Mth)
  // fused path
  int wpb = 0, blocks = 0;
  size_t smem = 0;
  // split path
  int root_blocks = 0, tr_wpb = 0, tr_blocks = 0;
  size_t tr_smem = 0;
};
}  // namespace bie

struct bie_batch_s {
  bie_ctx ctx;
  unsigned kernels;
  bool withK, split;
  int n_surf, maxMt, item_pairs, n_items, chunk_items;
  int64_t total_pairs, scratch_per_warp;
  std::vector<bie::PairArgs> host_args;
  std::vector<int64_t> offsets;
  std::vector<bie::BatchClass> classes;
  bie::PairArgs* d_args = nullptr;
  bie::BatchItem* d_items = nullptr;
  int* d_counter = nullptr;     // one counter per class (fused path)
  double* scratch = nullptr;    // fused path: per resident warp recurrence scratch
  double* records = nullptr;    // split path: per-pair records of one chunk
  float tuned_ms = 0.f;
  std::vector<bie_surface> surfs;
  std::vector<bie::BatchItem> h_items;   // split path: the work list, as uploaded
  int64_t slot_pairs = 0;
  // GGQ fill (single layer): each target panel, once its pairs are done, folded into a ring of
  // band_slots near-band slots of band_slot_elems complex each
  bie::cplx* band = nullptr;
  int band_slots = 0;
  int64_t band_slot_elems = 0;
  bool fill_on() const { return band != nullptr; }
};

namespace bie {
// items of every surface, ordered by decreasing Mth (stable: surfaces keep their order within a class)
static std::vector<BatchItem> make_items(const bie_batch_s& b, int item_pairs) {
  std::vector<BatchItem> items;
  for (int sidx = 0; sidx < b.n_surf; ++sidx) {
    const int64_t n = b.host_args[sidx].n_pairs;
    for (int64_t p = 0; p < n; p += item_pairs)
      items.push_back({sidx, (int)((n - p < item_pairs) ? n - p : item_pairs), p});
  }
  std::stable_sort(items.begin(), items.end(), [&](const BatchItem& x, const BatchItem& y) {
    return b.host_args[x.surf].Mt > b.host_args[y.surf].Mt;
  });
  return items;
}

static std::vector<BatchClass> make_classes(const bie_batch_s& b, const std::vector<BatchItem>& items) {
  std::vector<BatchClass> cl;
  for (int i = 0; i < (int)items.size(); ++i) {
    const int Mt = b.host_args[items[i].surf].Mt;
    if (cl.empty() || cl.back().Mt != Mt) {
      BatchClass c;
      c.Mt = Mt;
      c.it_begin = i;
      cl.push_back(c);
    }
    cl.back().it_end = i + 1;
  }
  return cl;
}

// Dynamic shared-memory limits are properties of the kernel functions, shared by every plan: they
// only grow (set when a plan is made, never during a run), so earlier plans and captured graphs keep
// launching.
static int g_batch_smem_attr[3] = {0, 0, 0};
static bie_status grow_smem_attr(int which, size_t smem) {
  int& cur = g_batch_smem_attr[which];
  if ((int)smem <= cur) return BIE_OK;
  const void* f = which == 0 ? (const void*)pair_batch_kernel<false>
                  : which == 1 ? (const void*)pair_batch_kernel<true>
                               : (const void*)pair_transform_batch_kernel;
  const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(batch kernel)");
  cur = (int)smem;
  return BIE_OK;
}

static int64_t split_record_doubles(int Mt) {
  const int L = 3 * (Mt / 2);
  return 8 + 2 * 33 + (L + 1) + Mt;
}

static BatchRec class_records(const bie_batch_s& b, const BatchClass& c) {
  const int64_t slots = (int64_t)b.chunk_items * b.item_pairs;
  BatchRec r;
  r.Mt = c.Mt;
  r.L = 3 * (c.Mt / 2);
  r.hdr = b.records;
  r.E = reinterpret_cast<float4*>(b.records + 8 * slots);
  r.A = b.records + (8 + 2 * 33) * slots;
  r.R2 = r.A + (int64_t)(r.L + 1) * slots;
  return r;
}

// configure one class: CTA shapes and grids for its kernels; false if it does not fit
static bool configure_class(bie_batch_s& b, BatchClass& c) {
  const int sms = b.ctx->sms;
  if (!b.split) {
    const bool wk = b.withK;
    const int P = (wk ? 4 : 3) * c.Mt, L = (wk ? 4 : 3) * (c.Mt / 2);
    const size_t per = smem_doubles(c.Mt, P, L, wk) * sizeof(double);
    auto kern = wk ? pair_batch_kernel<true> : pair_batch_kernel<false>;
    int best = 0;
    for (int w = kMaxWarpsPerBlock; w >= 1; w /= 2) {
      if (per * w > kSmemLimit || grow_smem_attr(wk ? 1 : 0, per * w) != BIE_OK) continue;
      int nb = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, 32 * w, per * w) != cudaSuccess) continue;
      if (nb * w > best) { best = nb * w; c.wpb = w; c.smem = per * w; c.blocks = sms * nb; }
    }
    return best > 0;
  }
  int per_r = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_r, pair_root_batch_kernel, 128, 0) != cudaSuccess) return false;
  c.root_blocks = sms * std::max(per_r, 1);
  const size_t per = smem_doubles(c.Mt, 3 * c.Mt, 3 * (c.Mt / 2), false) * sizeof(double);
  int best = 0;
  for (int w = kMaxWarpsPerBlock; w >= 1; w /= 2) {
    if (per * w > kSmemLimit || grow_smem_attr(2, per * w) != BIE_OK) continue;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pair_transform_batch_kernel, 32 * w, per * w) != cudaSuccess)
      continue;
    if (nb * w > best) { best = nb * w; c.tr_wpb = w; c.tr_smem = per * w; c.tr_blocks = sms * nb; }
  }
  return best > 0;
}

// launch every class; items at or past it_hi are left out (the autotuner times a prefix)
static bie_status batch_launch(bie_batch_s& b, int it_hi) {
  cudaStream_t st = b.ctx->stream;
  if (!b.split) {
    cudaError_t e = cudaMemsetAsync(b.d_counter, 0, sizeof(int) * b.classes.size(), st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync(batch counters)");
    for (size_t ci = 0; ci < b.classes.size(); ++ci) {
      const BatchClass& c = b.classes[ci];
      const int end = std::min(c.it_end, it_hi);
      if (end <= c.it_begin) break;
      if (b.withK)
        pair_batch_kernel<true><<<c.blocks, 32 * c.wpb, c.smem, st>>>(b.d_args, b.d_items, c.it_begin, end,
                                                                      b.d_counter + ci, b.scratch, b.scratch_per_warp, c.Mt);
      else
        pair_batch_kernel<false><<<c.blocks, 32 * c.wpb, c.smem, st>>>(b.d_args, b.d_items, c.it_begin, end,
                                                                       b.d_counter + ci, b.scratch, b.scratch_per_warp, c.Mt);
    }
  } else {
    // GGQ fill bookkeeping: pairs done per surface (its items are contiguous and in order), panels
    // already folded, and the next band slot
    std::vector<int64_t> done(b.fill_on() ? b.n_surf : 0, 0);
    std::vector<int> filled(done.size(), 0);
    int64_t slot = 0;
    for (const BatchClass& c : b.classes) {
      const int end = std::min(c.it_end, it_hi);
      if (end <= c.it_begin) break;
      const BatchRec rec = class_records(b, c);
      for (int i0 = c.it_begin; i0 < end; i0 += b.chunk_items) {
        const int nit = std::min(b.chunk_items, end - i0);
        const int64_t wbs = (int64_t)nit * (b.item_pairs / 32);
        const int br = (int)std::max<int64_t>(1, std::min<int64_t>(c.root_blocks, (wbs + 3) / 4));
        pair_root_batch_kernel<<<br, 128, 0, st>>>(b.d_args, b.d_items, i0, nit, b.item_pairs, rec);
        const int bt = (int)std::max<int64_t>(1, std::min<int64_t>(c.tr_blocks, (wbs + c.tr_wpb - 1) / c.tr_wpb));
        pair_transform_batch_kernel<<<bt, 32 * c.tr_wpb, c.tr_smem, st>>>(b.d_args, b.d_items, i0, nit, b.item_pairs,
                                                                         rec);
        if (!b.fill_on()) continue;
        for (int it = i0; it < i0 + nit; ++it) {
          const BatchItem& item = b.h_items[it];
          done[item.surf] = item.p0 + item.n;
        }
        for (int sidx = 0; sidx < b.n_surf; ++sidx) {
          const bie_surface sf = b.surfs[sidx];
          const int64_t panel_pairs = (int64_t)16 * 48 * sf->Mt;
          for (; filled[sidx] < sf->Np && (int64_t)(filled[sidx] + 1) * panel_pairs <= done[sidx]; ++filled[sidx]) {
            const bie_status fs = near_fill_ring(sf, filled[sidx], reinterpret_cast<const cplx*>(b.host_args[sidx].weights_out),
                                                 b.offsets[sidx] + (int64_t)filled[sidx] * panel_pairs, b.slot_pairs,
                                                 b.maxMt, b.band + (slot % b.band_slots) * b.band_slot_elems, st);
            if (fs != BIE_OK) return fs;
            ++slot;
          }
        }
      }
    }
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BIE_OK : cuda_fail(e, "batch kernels");
}

static bie_status upload_items(bie_batch_s& b, const std::vector<BatchItem>& items) {
  if (b.d_items) cudaFree(b.d_items);
  b.d_items = nullptr;
  cudaError_t e = cudaMalloc((void**)&b.d_items, sizeof(BatchItem) * items.size());
  if (e == cudaSuccess)
    e = cudaMemcpy(b.d_items, items.data(), sizeof(BatchItem) * items.size(), cudaMemcpyHostToDevice);
  return e == cudaSuccess ? BIE_OK : cuda_fail(e, "batch items");
}
}  // namespace bie

extern "C" bie_status bie_batch_create(bie_ctx ctx, int n_surf, const bie_surface* surfs, const double* ks,
                                       unsigned kernels, double* weights_out, int64_t slot_pairs, bie_batch* out) {
  if (!ctx || n_surf < 1 || !surfs || !ks || !weights_out || slot_pairs < 1 || !out) {
    set_error("bie_batch_create: invalid arguments");
    return BIE_EINVAL;
  }
  if (kernels == 0 || (kernels & ~(BIE_KERNEL_S | BIE_KERNEL_K | BIE_KERNEL_KP)) ||
      ((kernels & BIE_KERNEL_K) && (kernels & BIE_KERNEL_KP))) {
    set_error("bie_batch_create: bad kernel mask (S and at most one of K, KP)");
    return BIE_EINVAL;
  }
  bie_batch_s* b = new bie_batch_s();
  b->ctx = ctx;
  b->kernels = kernels;
  b->withK = kernels & (BIE_KERNEL_K | BIE_KERNEL_KP);
  b->split = !b->withK;
  b->n_surf = n_surf;
  b->maxMt = 0;
  std::vector<int> grids;
  for (int i = 0; i < n_surf; ++i) {
    if (!surfs[i] || !(ks[i] > 0) || !(ks[i] < 1e6)) { delete b; set_error("bie_batch_create: surface %d or k invalid", i); return BIE_EINVAL; }
    b->maxMt = surfs[i]->Mt > b->maxMt ? surfs[i]->Mt : b->maxMt;
    if (std::find(grids.begin(), grids.end(), surfs[i]->Mt) == grids.end()) grids.push_back(surfs[i]->Mt);
  }
  if (grids.size() > (size_t)kMaxBatchClasses) {
    delete b;
    set_error("bie_batch_create: more than %d grid sizes", kMaxBatchClasses);
    return BIE_EUNSUPPORTED;
  }
  // output rows follow the processing order (classes by decreasing Mth, surfaces in order within a
  // class), so that a bounded ring holds the most recent pairs of every surface
  std::vector<int> order(n_surf);
  for (int i = 0; i < n_surf; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return surfs[x]->Mt > surfs[y]->Mt; });
  std::vector<int64_t> start(n_surf, 0);
  {
    int64_t acc = 0;
    for (int i : order) {
      start[i] = acc;
      acc += (int64_t)16 * surfs[i]->Np * 48 * surfs[i]->Mt;
    }
  }
  b->slot_pairs = slot_pairs;
  b->surfs.assign(surfs, surfs + n_surf);
  int64_t off = 0;
  for (int i = 0; i < n_surf; ++i) {
    PairArgs a = make_pair_args(surfs[i], ks[i], kernels);
    a.fp64_transforms = 0;   // the batch kernels run the single layer in double words
    a.enumerate = 1;
    a.p0 = 0;
    a.n_pairs = (int64_t)16 * surfs[i]->Np * 48 * surfs[i]->Mt;
    a.weights_out = (cplx*)weights_out;
    a.w_ld = b->maxMt;
    a.out_base = start[i];
    a.out_mod = slot_pairs;
    a.weights_stride = slot_pairs * b->maxMt;
    b->offsets.push_back(start[i]);
    off += a.n_pairs;
    b->host_args.push_back(a);
  }
  b->total_pairs = off;
  const double* rec = nullptr;
  int rec_len = 0;
  bie_status st = ensure_rec(ctx, (b->withK ? 4 : 3) * (b->maxMt / 2), &rec, &rec_len);
  if (st != BIE_OK) { delete b; return st; }
  for (auto& a : b->host_args) {
    a.rec = rec;
    a.rec_len = rec_len;
  }
  cudaError_t e = cudaMalloc((void**)&b->d_args, sizeof(PairArgs) * n_surf);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_counter, sizeof(int) * kMaxBatchClasses);
  if (e != cudaSuccess) { bie_batch_free(b); return cuda_fail(e, "cudaMalloc(batch)"); }
  e = cudaMemcpy(b->d_args, b->host_args.data(), sizeof(PairArgs) * n_surf, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) { bie_batch_free(b); return cuda_fail(e, "cudaMemcpy(batch args)"); }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto timed = [&](int it_hi, float* ms) -> bie_status {
    cudaEventRecord(e0, ctx->stream);
    const bie_status s2 = batch_launch(*b, it_hi);
    cudaEventRecord(e1, ctx->stream);
    if (s2 != BIE_OK) return s2;
    cudaEventSynchronize(e1);
    cudaEventElapsedTime(ms, e0, e1);
    return BIE_OK;
  };
  float best = 1e30f;
  if (b->split) {
    // items of 1024 pairs; the autotuner picks the chunk (records of 2^18, 2^19 or 2^20 pairs) on the
    // first 2^20 pairs of the largest class
    b->item_pairs = 1024;
    const std::vector<BatchItem> items = make_items(*b, b->item_pairs);
    b->n_items = (int)items.size();
    b->classes = make_classes(*b, items);
    b->h_items = items;
    st = upload_items(*b, items);
    for (auto& c : b->classes)
      if (st == BIE_OK && !configure_class(*b, c)) { st = BIE_EUNSUPPORTED; set_error("bie_batch_create: a class does not fit"); }
    const int cands[3] = {256, 512, 1024};
    size_t rbytes = sizeof(double) * (size_t)split_record_doubles(b->maxMt) * 1024 * 1024;
    if (st == BIE_OK && (e = cudaMalloc((void**)&b->records, rbytes)) != cudaSuccess) st = cuda_fail(e, "cudaMalloc(batch records)");
    int best_c = 1024;
    const int probe = std::min(b->classes[0].it_end, 1024);
    for (int ci = 0; ci < 3 && st == BIE_OK; ++ci) {
      b->chunk_items = cands[ci];
      float ms = 0.f;
      st = timed(probe, &ms);
      if (st == BIE_OK && ms < best) { best = ms; best_c = cands[ci]; }
    }
    b->chunk_items = best_c;
  } else {
    // the fused kernel: the autotuner picks the item size on a prefix of the work list; each class
    // runs at the CTA shape with the most resident warps for its Mth
    const int cands[3] = {256, 1024, 4096};
    int best_item = 1024;
    b->scratch_per_warp = pair_scratch_per_warp((b->withK ? 4 : 3) * (b->maxMt / 2), b->withK, b->maxMt);
    size_t max_warps = 0;
    for (int ii = 0; ii < 3 && st == BIE_OK; ++ii) {
      b->item_pairs = cands[ii];
      const std::vector<BatchItem> items = make_items(*b, b->item_pairs);
      b->classes = make_classes(*b, items);
      for (auto& c : b->classes)
        if (!configure_class(*b, c)) { st = BIE_EUNSUPPORTED; set_error("bie_batch_create: a class does not fit"); }
      for (auto& c : b->classes) max_warps = std::max(max_warps, (size_t)c.blocks * c.wpb);
      if (st != BIE_OK) break;
      if (!b->scratch) {
        e = cudaMalloc((void**)&b->scratch, sizeof(double) * (size_t)b->scratch_per_warp * max_warps);
        if (e != cudaSuccess) { st = cuda_fail(e, "cudaMalloc(batch scratch)"); break; }
      }
      st = upload_items(*b, items);
      if (st != BIE_OK) break;
      float ms = 0.f;
      st = timed(std::max<int>(1, (int)items.size() / 16), &ms);
      if (st == BIE_OK && ms < best) { best = ms; best_item = cands[ii]; }
    }
    if (st == BIE_OK) {
      b->item_pairs = best_item;
      const std::vector<BatchItem> items = make_items(*b, b->item_pairs);
      b->n_items = (int)items.size();
      b->classes = make_classes(*b, items);
      for (auto& c : b->classes) configure_class(*b, c);
      st = upload_items(*b, items);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != BIE_OK) { bie_batch_free(b); return st; }
  b->tuned_ms = best;
  *out = b;
  return BIE_OK;
}

extern "C" bie_status bie_batch_run(bie_batch b) {
  if (!b) { set_error("bie_batch_run: NULL plan"); return BIE_EINVAL; }
  return batch_launch(*b, b->n_items);
}

extern "C" int64_t bie_batch_pairs(bie_batch b) { return b ? b->total_pairs : 0; }

extern "C" int64_t bie_batch_offset(bie_batch b, int i) {
  return (b && i >= 0 && i < b->n_surf) ? b->offsets[i] : -1;
}

extern "C" void bie_batch_config(bie_batch b, int* item_pairs, int* warps_per_block, int* blocks) {
  if (!b) return;
  if (item_pairs) *item_pairs = b->split ? b->chunk_items * b->item_pairs : b->item_pairs;
  const BatchClass* c = b->classes.empty() ? nullptr : &b->classes[0];
  if (warps_per_block) *warps_per_block = c ? (b->split ? c->tr_wpb : c->wpb) : 0;
  if (blocks) *blocks = c ? (b->split ? c->tr_blocks : c->blocks) : 0;
}

extern "C" int bie_batch_launches(bie_batch b) {
  if (!b) return 0;
  if (!b->split) return (int)b->classes.size();
  int n = 0;
  for (const BatchClass& c : b->classes) n += 2 * ((c.it_end - c.it_begin + b->chunk_items - 1) / b->chunk_items);
  if (b->fill_on())
    for (const bie_surface sf : b->surfs) n += sf->Np;   // one GGQ fill per target panel
  return n;
}

extern "C" bie_status bie_batch_set_fill(bie_batch b, double* band_ring, int band_slots) {
  if (!b || (band_ring && band_slots < 1)) { set_error("bie_batch_set_fill: invalid arguments"); return BIE_EINVAL; }
  if (!band_ring) {
    b->band = nullptr;
    b->band_slots = 0;
    return BIE_OK;
  }
  if (!b->split) {
    set_error("bie_batch_set_fill: the GGQ fill takes single-layer plans (kernels = BIE_KERNEL_S)");
    return BIE_EUNSUPPORTED;
  }
  int64_t max_panel = 0;
  for (const bie_surface sf : b->surfs) max_panel = std::max<int64_t>(max_panel, (int64_t)16 * 48 * sf->Mt);
  // a panel straddling two chunks keeps its first rows while the next chunk runs: the ring holds a
  // chunk plus a panel
  const int64_t room = (b->slot_pairs - max_panel) / b->item_pairs;
  if (room < 1) {
    set_error("bie_batch_set_fill: slot_pairs %lld holds less than a panel (%lld pairs) plus one item",
              (long long)b->slot_pairs, (long long)max_panel);
    return BIE_EINVAL;
  }
  if (b->chunk_items > room) b->chunk_items = (int)room;
  b->band = reinterpret_cast<bie::cplx*>(band_ring);
  b->band_slots = band_slots;
  b->band_slot_elems = (int64_t)16 * b->maxMt * 3 * 16 * b->maxMt;
  return BIE_OK;
}

extern "C" void bie_batch_free(bie_batch b) {
  if (!b) return;
  cudaFree(b->d_args);
  cudaFree(b->d_items);
  cudaFree(b->d_counter);
  cudaFree(b->scratch);
  cudaFree(b->records);
  delete b;
}
