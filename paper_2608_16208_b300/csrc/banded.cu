// The O(M) route to the theta_s-Fourier modes of 1/rho (Section 3.3, "An O(M) approach"), and the
// single-layer kernel modes built on it (Eq. (Sphi:appr2)).  For a target x = r(t, th) and a source
// ring t_s != t, rho^2(theta_s) = |r(t_s, theta_s) - x|^2 is a trigonometric polynomial in theta_s,
// and the modes of 1/rho obey the (2 m0 + 1)-term difference equation Eq. (lin:diff) with the
// coefficients a_j(i) = (m0 + 2i + j) <rho^2>_{m0-j} of Eq. (def:a_l).  With the first and last m0
// modes fixed by quadrature (Eq. (offline:terms)), the others solve the banded system Eq. (Axb),
// A_ij = (2 m0 + i + j) <rho^2>_{i-j} for |i - j| <= m0.
//
// One warp per query:
//   1. rho^2 at 64 angles (cancellation-free differences), its modes n = 0..15 by a direct DFT,
//      m0 by Eq. (crt:M0) read as a bound on the whole tail (every |n| > m0 below eps0 of the
//      largest mode);
//   2. the real minimiser a of rho^2 (Newton on the trigonometric polynomial) and the distance b of
//      the nearest complex root, b = (2 rho^2(a) / rho^2''(a))^{1/2};
//   3. the 2 m0 boundary modes by 16-point Gauss-Legendre quadrature (the "adaptive Gauss-Legendre"
//      of the paper) on panels graded geometrically towards a, from b/4 up to pi on both sides, each
//      subdivided so that l times its half-width stays below kBandPhase for every boundary mode l;
//      a pass evaluates 32 nodes (one per lane, with two phasors), and the lanes, as (boundary mode,
//      node group) pairs, accumulate them;
//   4. Gaussian elimination with partial pivoting inside the band (Lemma after Eq. (root:x): A is
//      Hermitian and, under Eq. (cond:rho), positive definite; pivoting keeps the elimination stable
//      when the condition fails), rows k..k+m0 held in a circular shared-memory window; the rows of
//      U (2 m0 superdiagonals after pivoting) and the eliminated right-hand side go to the warp's
//      global scratch and are read back by the back substitution.
#include <cmath>
#include <mutex>

#include "bie_internal.cuh"
#include "surf_diff.cuh"

namespace bie {

constexpr int kBandMaxM0 = 15;                 // boundary modes one lane each; 2 m0 + 1 <= 31 lanes
constexpr int kBandWin = 2 * kBandMaxM0 + 1;   // row stride of the elimination window
constexpr int kBandSamples = 64;               // rho^2 samples: modes |n| <= 15 exact up to degree 48
constexpr int kBandMaxIv = 128;                // graded intervals (b >= 1e-12: at most 92)
constexpr int kBandWarps = 4;
constexpr double kBandPhase = 6.0;             // l * half-width of a panel, at most (GL16: 4e-16 at 8)
constexpr double kBandMinB = 1e-12;

struct BandSmem {
  double r2[kBandSamples];
  cplx c[kBandMaxM0 + 1];            // <rho^2>_n, n = 0..15; <rho^2>_{-n} = conj(<rho^2>_n)
  double qv[32];                     // one pass of quadrature nodes: weight / rho,
  cplx qe1[32], qeL[32];             // e^{-i (theta_s - a)} and e^{-i L (theta_s - a)}
  cplx bnd[2 * kBandMaxM0];          // modes 0..m0-1, then lmax-m0+1..lmax
  double ivlo[kBandMaxIv], ivhi[kBandMaxIv];
  int ivsub[kBandMaxIv + 1];         // prefix counts of subpanels
  int niv, pad;
  cplx win[(kBandMaxM0 + 1) * kBandWin];
  cplx wb[kBandMaxM0 + 1];
  cplx xs[kBandWin];                 // the last 2 m0 + 1 unknowns of the back substitution
  cplx red[32];                      // partial boundary sums of the node groups
};

__device__ __forceinline__ cplx warp_csum(cplx v) {
  for (int o = 16; o; o >>= 1) {
    v.re += __shfl_xor_sync(0xffffffffu, v.re, o);
    v.im += __shfl_xor_sync(0xffffffffu, v.im, o);
  }
  return v;
}

// hi + lo += a b, the rounding errors of the product (FMA) and of the sum (Knuth's TwoSum) kept in lo
// (intrinsics: the compiler may not contract them into FMAs, which would void the error terms)
__device__ __forceinline__ void dd_add_prod(double& hi, double& lo, double a, double b) {
  const double p = __dmul_rn(a, b), ep = fma(a, b, -p);
  const double s = __dadd_rn(hi, p), bb = __dsub_rn(s, hi);
  const double es = __dadd_rn(__dsub_rn(hi, __dsub_rn(s, bb)), __dsub_rn(p, bb));
  hi = s;
  lo += es + ep;
}

// e^{-i l x} with the product l x carried to twice the working precision before the reduction
__device__ __forceinline__ cplx phase_neg(int l, double x) {
  const double dl = (double)l;
  const double p = __dmul_rn(dl, x), e = fma(dl, x, -p);
  double s, c;
  sincos(p, &s, &c);
  return C(c + s * e, -(s - c * e));
}

// rho^2 as the trigonometric polynomial of its modes n = 0..m0, and its first two derivatives
__device__ __forceinline__ void r2_poly(const BandSmem& sm, int m0, double x, double* g, double* g1, double* g2) {
  double v = sm.c[0].re, d1 = 0.0, d2 = 0.0;
  for (int n = 1; n <= m0; ++n) {
    double s, c;
    sincos(n * x, &s, &c);
    const double re = sm.c[n].re * c - sm.c[n].im * s, im = sm.c[n].re * s + sm.c[n].im * c;
    v += 2.0 * re;
    d1 -= 2.0 * n * im;
    d2 -= 2.0 * n * n * re;
  }
  *g = v;
  *g1 = d1;
  *g2 = d2;
}

__device__ __forceinline__ cplx band_coef(const BandSmem& sm, int m0, int i, int c) {
  const int d = i - c;
  const cplx v = d >= 0 ? sm.c[d] : conj(sm.c[-d]);
  return (double)(2 * m0 + i + c) * v;
}

// the boundary value <rho^{-1}>_l of a column outside 0..M1 (column c is the unknown l = m0 + c)
__device__ __forceinline__ cplx band_boundary(const BandSmem& sm, int m0, int lmax, int c) {
  const int l = m0 + c;
  return l < m0 ? sm.bnd[l] : sm.bnd[l - (lmax - 2 * m0 + 1)];
}

// row i of A into its window slot (columns i - m0 .. i + m0, circular), its right-hand side
// -sum of the boundary columns into wb
__device__ __forceinline__ void band_load_row(BandSmem& sm, int m0, int lmax, int M1, int i) {
  const int lane = threadIdx.x & 31;
  const int wc = 2 * m0 + 1, slot = i % (m0 + 1);
  cplx rhs = C(0.0);
  if (lane < wc) {
    const int c = i - m0 + lane;
    const cplx v = band_coef(sm, m0, i, c);
    cplx stored = C(0.0);
    if (c >= 0 && c <= M1) {
      stored = v;
    } else {
      rhs = -1.0 * (v * band_boundary(sm, m0, lmax, c));
    }
    if (c >= 0) sm.win[slot * kBandWin + c % wc] = stored;
    else sm.win[slot * kBandWin + (c + wc) % wc] = C(0.0);   // initial rows: the slot of a column > i + m0
  }
  rhs = warp_csum(rhs);
  if (lane == 0) sm.wb[slot] = rhs;
}

// <rho^{-1}>_l, l = 0..lmax, of one query into out (global); U: this warp's scratch, ucols >= 2 m0cap + 2
// complex per row.  m0 is at most m0cap, twice the surface's theta-degree (the degree of rho^2), so
// that modes at rounding level cannot raise it when eps0 is very small.  Called by all 32 lanes.
// Returns m0, negated when the elimination met a zero or non-finite pivot.
__device__ int band_rho_inv(const SurfP& S, double t, double th, double ts, int lmax, double eps0, int m0cap,
                            BandSmem& sm, cplx* U, int ucols, cplx* out) {
  const int lane = threadIdx.x & 31;
  // 1. rho^2 samples and modes
  for (int i = lane; i < kBandSamples; i += 32) {
    const R3 Y = diff_ana<double>(S, ts, kTwoPi * i / kBandSamples, t, th);
    sm.r2[i] = dot(Y, Y);
  }
  __syncwarp();
  if (lane <= kBandMaxM0) {
    // compensated sums: the modes carry the samples' own rounding and little of the summation's,
    // which the banded system amplifies near the minimiser of rho^2
    double ch = 0.0, cl = 0.0, sh = 0.0, sl = 0.0;
    for (int i = 0; i < kBandSamples; ++i) {
      double s, c;
      sincospi((double)((lane * i) % kBandSamples) * (2.0 / kBandSamples), &s, &c);
      dd_add_prod(ch, cl, sm.r2[i], c);
      dd_add_prod(sh, sl, sm.r2[i], s);
    }
    sm.c[lane] = C((ch + cl) / kBandSamples, -(sh + sl) / kBandSamples);
  }
  __syncwarp();
  double big = 0.0;
  for (int n = 0; n <= kBandMaxM0; ++n) big = fmax(big, sqrt(abs2(sm.c[n])));
  int m0 = m0cap;
  while (m0 > 1 && sqrt(abs2(sm.c[m0])) <= eps0 * big) --m0;
  // 2. minimiser and root distance
  double best = 1e300;
  int bi = 0;
  for (int i = lane; i < kBandSamples; i += 32)
    if (sm.r2[i] < best) { best = sm.r2[i]; bi = i; }
  for (int o = 16; o; o >>= 1) {
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob < best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  double a = kTwoPi * bi / kBandSamples, g, g1, g2;
  for (int it = 0; it < 10; ++it) {
    r2_poly(sm, m0, a, &g, &g1, &g2);
    if (!(g2 > 0.0)) break;
    const double step = fmax(-kPi / 32, fmin(kPi / 32, g1 / g2));
    a -= step;
    if (fabs(step) <= 1e-15) break;
  }
  r2_poly(sm, m0, a, &g, &g1, &g2);
  const R3 Ya = diff_ana<double>(S, ts, a, t, th);
  double b = g2 > 0.0 ? sqrt(2.0 * dot(Ya, Ya) / g2) : 1e-3;
  b = fmin(1.0, fmax(kBandMinB, b));
  // 3. graded panels and the boundary modes
  if (lane == 0) {
    const double W = kBandPhase / (double)max(lmax, 1);   // largest half-width
    int n = 0, tot = 0;
    double lo = 0.0, hi = 0.25 * b;
    while (true) {
      if (n + 4 > kBandMaxIv) hi = kPi;
      hi = fmin(hi, kPi);
      for (int side = 0; side < 2; ++side) {
        const int sub = max(1, (int)ceil((hi - lo) / (2.0 * W)));
        sm.ivlo[n] = side ? -hi : lo;
        sm.ivhi[n] = side ? -lo : hi;
        sm.ivsub[n] = tot;
        tot += sub;
        ++n;
      }
      if (hi >= kPi) break;
      lo = hi;
      hi = 2.0 * hi;
    }
    sm.ivsub[n] = tot;
    sm.niv = n;
  }
  __syncwarp();
  const int niv = sm.niv, nodes = 16 * sm.ivsub[niv];
  // lane = (boundary mode jm, node group grp); a pass evaluates 32 nodes, one per lane, with the
  // phasors e^{-i x} and e^{-i L x} (L = lmax - m0 + 1, the first high mode); mode l then takes
  // e^{-i l x} as e^{-i x}^l (low modes, l < m0) or e^{-i L x} e^{-i x}^{l - L} (high modes)
  const int nbm = 2 * m0, groups = 32 / nbm, jm = lane % nbm, grp = lane / nbm;
  const bool own = grp < groups;
  const int l = jm < m0 ? jm : lmax - 2 * m0 + 1 + jm;
  const int Lh = lmax - m0 + 1, pw = jm < m0 ? jm : jm - m0;
  cplx acc = C(0.0);
  for (int base = 0; base < nodes; base += 32) {
    const int gidx = base + lane;
    double wv = 0.0;
    cplx e1 = C(1.0), eL = C(1.0);
    if (gidx < nodes) {
      const int spn = gidx >> 4, node = gidx & 15;
      int lo = 0, hi = niv - 1;   // interval holding subpanel spn
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (sm.ivsub[mid] <= spn) lo = mid; else hi = mid - 1;
      }
      const int ns = sm.ivsub[lo + 1] - sm.ivsub[lo], u = spn - sm.ivsub[lo];
      const double wd = (sm.ivhi[lo] - sm.ivlo[lo]) / ns;
      const double dv = sm.ivlo[lo] + wd * (u + S.gl.x[node]);
      const R3 Y = diff_ana<double>(S, ts, a + dv, t, th);
      wv = wd * S.gl.w[node] / sqrt(dot(Y, Y));
      e1 = phase_neg(1, dv);
      eL = phase_neg(Lh, dv);
    }
    sm.qv[lane] = wv;
    sm.qe1[lane] = e1;
    sm.qeL[lane] = eL;
    __syncwarp();
    if (own) {
      for (int i = grp; i < 32; i += groups) {
        cplx e = jm < m0 ? C(1.0) : sm.qeL[i];
        const cplx step = sm.qe1[i];
        for (int r = 0; r < pw; ++r) e = e * step;
        acc.re = fma(sm.qv[i], e.re, acc.re);
        acc.im = fma(sm.qv[i], e.im, acc.im);
      }
    }
    __syncwarp();
  }
  sm.red[lane] = acc;
  __syncwarp();
  if (lane < nbm) {
    cplx tot = C(0.0);
    for (int g = 0; g < groups; ++g) tot = tot + sm.red[lane + g * nbm];
    sm.bnd[lane] = (1.0 / kTwoPi) * (tot * phase_neg(l, a));
  }
  __syncwarp();
  // 4. the banded system, columns 0..M1 = modes m0..lmax-m0
  const int M1 = lmax - 2 * m0, wc = 2 * m0 + 1;
  int bad = 0;
  for (int i = 0; i <= min(m0, M1); ++i) band_load_row(sm, m0, lmax, M1, i);
  __syncwarp();
  for (int k = 0; k <= M1; ++k) {
    const int kend = min(k + m0, M1), ck = k % wc, sk = k % (m0 + 1);
    double mag = -1.0;
    int pj = 0;
    if (lane <= kend - k) {
      mag = abs2(sm.win[((k + lane) % (m0 + 1)) * kBandWin + ck]);
      pj = lane;
    }
    for (int o = 16; o; o >>= 1) {
      const double om = __shfl_xor_sync(0xffffffffu, mag, o);
      const int oj = __shfl_xor_sync(0xffffffffu, pj, o);
      if (om > mag || (om == mag && oj < pj)) { mag = om; pj = oj; }
    }
    if (!(mag > 0.0) || !isfinite(mag)) bad = 1;
    if (pj) {
      const int sp = (k + pj) % (m0 + 1);
      if (lane < wc) {
        const cplx u = sm.win[sk * kBandWin + lane];
        sm.win[sk * kBandWin + lane] = sm.win[sp * kBandWin + lane];
        sm.win[sp * kBandWin + lane] = u;
      }
      if (lane == 0) {
        const cplx u = sm.wb[sk];
        sm.wb[sk] = sm.wb[sp];
        sm.wb[sp] = u;
      }
    }
    __syncwarp();
    const cplx ipiv = cdiv(C(1.0), sm.win[sk * kBandWin + ck]);
    const int nr = kend - k, ncol = 2 * m0;
    for (int e = lane; e < nr * ncol; e += 32) {
      const int j = 1 + e / ncol, o = 1 + e % ncol;
      const int sj = (k + j) % (m0 + 1), cs = (k + o) % wc;
      const cplx mlt = sm.win[sj * kBandWin + ck] * ipiv;
      sm.win[sj * kBandWin + cs] = sm.win[sj * kBandWin + cs] - mlt * sm.win[sk * kBandWin + cs];
    }
    if (lane >= 1 && lane <= nr) {
      const int sj = (k + lane) % (m0 + 1);
      sm.wb[sj] = sm.wb[sj] - (sm.win[sj * kBandWin + ck] * ipiv) * sm.wb[sk];
    }
    __syncwarp();
    cplx* Uk = U + (int64_t)k * ucols;
    if (lane < wc) Uk[lane] = sm.win[sk * kBandWin + (k + lane) % wc];
    if (lane == 0) Uk[wc] = sm.wb[sk];
    if (lane >= 1 && lane <= nr) sm.win[((k + lane) % (m0 + 1)) * kBandWin + ck] = C(0.0);
    __syncwarp();
    if (k + m0 + 1 <= M1) band_load_row(sm, m0, lmax, M1, k + m0 + 1);
    __syncwarp();
  }
  // back substitution; the next row of U is loaded while this one is reduced
  cplx u = lane <= wc ? U[(int64_t)M1 * ucols + lane] : C(0.0);
  for (int k = M1; k >= 0; --k) {
    const cplx un = (k > 0 && lane <= wc) ? U[(int64_t)(k - 1) * ucols + lane] : C(0.0);
    cplx part = C(0.0);
    if (lane >= 1 && lane < wc && k + lane <= M1) part = u * sm.xs[(k + lane) % wc];
    part = warp_csum(part);
    const cplx u0 = shfl(u, 0), y = shfl(u, wc);
    if (lane == 0) {
      const cplx x = cdiv(y - part, u0);
      sm.xs[k % wc] = x;
      out[m0 + k] = x;
    }
    u = un;
    __syncwarp();
  }
  if (lane < nbm) out[lane < m0 ? lane : lmax - 2 * m0 + 1 + lane] = sm.bnd[lane];
  bad = __any_sync(0xffffffffu, bad);
  if (bad) {
    for (int i = lane; i <= lmax; i += 32) out[i] = C(__longlong_as_double(0x7ff8000000000000ll), __longlong_as_double(0x7ff8000000000000ll));
  }
  __syncwarp();
  return bad ? -m0 : m0;
}

struct BandArgs {
  SurfP S;
  const double* t;
  const double* th;
  const double* ts;
  int64_t n;
  int lmax;
  double eps0;
  int m0cap;            // twice the surface's theta-degree
  int ucols;            // complex per scratch row: the 2 m0 + 1 entries of a row of U and its y
  cplx* out;            // [n][lmax + 1]
  int* m0_out;          // [n] or null
  cplx* scratch;        // [warps][lmax + 1][ucols]
  int* status;          // status[2]: queries with a zero pivot or a non-finite value
};

__global__ void __launch_bounds__(32 * kBandWarps) band_rho_inv_kernel(BandArgs a) {
  extern __shared__ __align__(16) unsigned char band_smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  BandSmem& sm = reinterpret_cast<BandSmem*>(band_smem)[wib];
  const int64_t gw = (int64_t)blockIdx.x * kBandWarps + wib, nw = (int64_t)gridDim.x * kBandWarps;
  cplx* U = a.scratch + gw * (int64_t)(a.lmax + 1) * a.ucols;
  for (int64_t q = gw; q < a.n; q += nw) {
    const double t = a.t[q], th = a.th[q], ts = a.ts[q];
    cplx* out = a.out + q * (int64_t)(a.lmax + 1);
    if (!(t != ts) || !isfinite(t) || !isfinite(th) || !isfinite(ts)) {
      for (int i = lane; i <= a.lmax; i += 32) out[i] = C(__longlong_as_double(0x7ff8000000000000ll), __longlong_as_double(0x7ff8000000000000ll));
      if (lane == 0) {
        atomicAdd(a.status + 2, 1);
        if (a.m0_out) a.m0_out[q] = 0;
      }
      continue;
    }
    const int m0 = band_rho_inv(a.S, t, th, ts, a.lmax, a.eps0, a.m0cap, sm, U, a.ucols, out);
    if (lane == 0) {
      if (m0 <= 0) atomicAdd(a.status + 2, 1);
      if (a.m0_out) a.m0_out[q] = m0 > 0 ? m0 : -m0;
    }
  }
}

// Single-layer modes through the O(M) route, Eq. (Sphi:appr2) with M0 = M: the pair's
// <rho^{-1}>_l (l = 0..2M) from band_rho_inv, the grid modes C_j of cos(k rho) and G_j of
// sin(k rho)/rho (j = -M..M, the Nyquist mode split evenly between +M and -M) from one packed FFT
// of length Mth, and K_m = sum_j C_j <rho^{-1}>_{m-j} + i G_m, m = -M..M.
struct BandSArgs {
  SurfP S;
  int Mt, Np;
  int64_t N, n;
  double k, eps0;
  int m0cap;
  const double* t_nodes;
  const double* thg;
  const double* ring_t;
  const cplx* tw;
  int T;
  const int64_t* rows;
  const int32_t* srcs;
  int ucols;
  cplx* scratch;        // [warps][(Mt + 1) (ucols + 1)]: U rows, then <rho^{-1}>_l
  double* modes_out;    // [n][Mt + 1] complex
  int* status;          // status[0]: invalid pairs; status[2]: failed eliminations
  int warps;            // warps per block
  size_t smem_per_warp;
};

__global__ void __launch_bounds__(32 * kBandWarps) band_s_modes_kernel(BandSArgs a) {
  extern __shared__ __align__(16) unsigned char band_smem[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  unsigned char* base = band_smem + wib * a.smem_per_warp;
  BandSmem& sm = *reinterpret_cast<BandSmem*>(base);
  cplx* fx = reinterpret_cast<cplx*>(base + sizeof(BandSmem));
  cplx* fy = fx + (a.Mt + 1);
  const int Mt = a.Mt, M = Mt / 2, lmax = Mt;
  const int64_t gw = (int64_t)blockIdx.x * a.warps + wib, nw = (int64_t)gridDim.x * a.warps;
  cplx* U = a.scratch + gw * (int64_t)(lmax + 1) * (a.ucols + 1);
  cplx* R = U + (int64_t)(lmax + 1) * a.ucols;
  for (int64_t p = gw; p < a.n; p += nw) {
    double* out = a.modes_out + 2 * p * (int64_t)(Mt + 1);
    const int64_t row = a.rows[p];
    const int src = a.srcs[p];
    const int64_t tn = row / Mt;
    const int d = src / 16, g = src % 16;
    const int ip = (int)(tn / 16) + d - 1;
    const bool valid = row >= 0 && row < a.N && src >= 0 && src < 48 && (a.S.periodic || (ip >= 0 && ip < a.Np));
    if (!valid) {
      for (int i = lane; i < 2 * (Mt + 1); i += 32) out[i] = 0.0;
      if (lane == 0) atomicAdd(a.status, 1);
      continue;
    }
    const double t = a.t_nodes[tn], th = a.thg[3 * (int)(row % Mt)];
    const double ts = a.ring_t[(tn * 3 + d) * 16 + g];
    const int m0 = band_rho_inv(a.S, t, th, ts, lmax, a.eps0, a.m0cap, sm, U, a.ucols, R);
    if (m0 <= 0 && lane == 0) atomicAdd(a.status + 2, 1);
    // cos(k rho) + i sin(k rho)/rho on the grid, one transform
    for (int q = lane; q < Mt; q += 32) {
      const R3 Y = diff_ana<double>(a.S, ts, kTwoPi * q / Mt, t, th);
      const double rho = sqrt(dot(Y, Y));
      double s, c;
      sincos(a.k * rho, &s, &c);
      fx[q] = C(c, s / rho);
    }
    __syncwarp();
    const cplx* Z = warp_fft(fx, fy, Mt, a.tw, a.T, -1);
    cplx* CG = Z == fx ? fy : fx;   // C_j at CG[j + M], j = -M..M; G_j is read from Z below
    __syncwarp();
    const double inv = 1.0 / Mt;
    for (int j = lane; j <= M; j += 32) {
      const cplx zp = Z[j % Mt], zm = Z[(Mt - j) % Mt];
      cplx cj = 0.5 * inv * (zp + conj(zm));
      if (j == M) cj = 0.5 * cj;
      CG[M + j] = cj;
      CG[M - j] = conj(cj);
    }
    __syncwarp();
    // K_m = sum_j C_j R_{m-j} + i G_m
    for (int m = -M + lane; m <= M; m += 32) {
      cplx acc = C(0.0);
      for (int j = -M; j <= M; ++j) {
        const int l = m - j;
        const cplx r = l >= 0 ? R[l] : conj(R[-l]);
        acc = acc + CG[M + j] * r;
      }
      const int jm = m >= 0 ? m : -m;
      const cplx zp = Z[jm % Mt], zm = Z[(Mt - jm) % Mt];
      cplx gj = C(0.5 * inv * (zp.im + zm.im), -0.5 * inv * (zp.re - zm.re));
      if (jm == M) gj = 0.5 * gj;
      if (m < 0) gj = conj(gj);
      acc = acc + C(-gj.im, gj.re);   // + i G_m
      out[2 * (m + M)] = acc.re;
      out[2 * (m + M) + 1] = acc.im;
    }
    __syncwarp();
  }
}

}  // namespace bie

using namespace bie;

static int theta_degree(const SurfP& S) {
  if (S.kind == 1) {
    int d = 0;
    for (int i = 0; i < S.nt; ++i) d = max(d, abs((int)S.m[i]));
    return d + 1;
  }
  if (S.kind == 4) {
    int d = 0;
    for (int i = 0; i < S.nt; ++i) d = max(d, abs((int)S.m[i]));
    return max(d, 1);
  }
  return 1;
}

static bie_status band_grow(bie_ctx ctx, size_t need) {
  if (ctx->band_scratch_bytes >= need) return BIE_OK;
  cudaStreamSynchronize(ctx->stream);
  if (ctx->band_scratch) cudaFree(ctx->band_scratch);
  ctx->band_scratch = nullptr;
  ctx->band_scratch_bytes = 0;
  const cudaError_t e = cudaMalloc(&ctx->band_scratch, need);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(O(M) route scratch)");
  ctx->band_scratch_bytes = need;
  return BIE_OK;
}

static std::mutex g_band_attr_mu;
static int g_band_attr[2][64] = {};   // per device: dynamic shared memory set on the two kernels

static bie_status band_smem_attr(int which, int device, size_t smem) {
  std::lock_guard<std::mutex> lk(g_band_attr_mu);
  if (device < 0 || device >= 64) return BIE_EINVAL;
  int& cur = g_band_attr[which][device];
  if ((int)smem <= cur) return BIE_OK;
  const void* f = which == 0 ? (const void*)band_rho_inv_kernel : (const void*)band_s_modes_kernel;
  const cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(O(M) route)");
  cur = (int)smem;
  return BIE_OK;
}

// scratch budget of one launch: the warps in flight are capped so that their U rows fit in this
static constexpr size_t kBandScratchCap = size_t(512) << 20;

extern "C" {

bie_status bie_rho_inv_modes(bie_ctx ctx, bie_surface s, const double* t, const double* th, const double* ts,
                             int64_t n, int lmax, double eps0, double* modes_out, int32_t* m0_out) {
  if (!ctx || !s) { set_error("bie_rho_inv_modes: NULL handle"); return BIE_EINVAL; }
  bie_status st = check_device(ctx, "bie_rho_inv_modes");
  if (st != BIE_OK) return st;
  if (n < 0) { set_error("bie_rho_inv_modes: n < 0"); return BIE_EINVAL; }
  if (n == 0) return BIE_OK;
  if (!t || !th || !ts || !modes_out) { set_error("bie_rho_inv_modes: NULL buffer"); return BIE_EINVAL; }
  const int d = theta_degree(s->sp);
  if (2 * d > kBandMaxM0) {
    set_error("bie_rho_inv_modes: rho^2 has theta-degree %d (the route takes at most %d)", 2 * d, kBandMaxM0);
    return BIE_EINVAL;
  }
  if (lmax < 4 * d + 1 || lmax > (1 << 16)) {
    set_error("bie_rho_inv_modes: lmax %d outside [%d, 65536]", lmax, 4 * d + 1);
    return BIE_EINVAL;
  }
  if (!(eps0 > 0.0) || eps0 > 1e-6) { set_error("bie_rho_inv_modes: eps0 outside (0, 1e-6]"); return BIE_EINVAL; }
  const int ucols = 2 * (2 * d) + 2;
  const size_t per_warp = (size_t)(lmax + 1) * ucols * sizeof(cplx);
  int64_t warps = std::min<int64_t>((n + kBandWarps - 1) / kBandWarps * kBandWarps, (int64_t)ctx->sms * 8 * kBandWarps);
  warps = std::min<int64_t>(warps, std::max<int64_t>(kBandWarps, (int64_t)(kBandScratchCap / per_warp) / kBandWarps * kBandWarps));
  st = band_grow(ctx, per_warp * warps);
  if (st != BIE_OK) return st;
  const size_t smem = kBandWarps * sizeof(BandSmem);
  st = band_smem_attr(0, ctx->device, smem);
  if (st != BIE_OK) return st;
  BandArgs a = {};
  a.S = s->sp;
  a.t = t;
  a.th = th;
  a.ts = ts;
  a.n = n;
  a.lmax = lmax;
  a.eps0 = eps0;
  a.m0cap = 2 * d;
  a.ucols = ucols;
  a.out = reinterpret_cast<cplx*>(modes_out);
  a.m0_out = m0_out;
  a.scratch = reinterpret_cast<cplx*>(ctx->band_scratch);
  a.status = ctx->d_status;
  band_rho_inv_kernel<<<(unsigned)(warps / kBandWarps), 32 * kBandWarps, smem, ctx->stream>>>(a);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "band_rho_inv_kernel launch");
  return BIE_OK;
}

bie_status bie_kernel_modes_banded(bie_ctx ctx, bie_surface s, double k, const int64_t* pair_row,
                                   const int32_t* pair_src, int64_t n_pairs, double eps0, double* modes_out) {
  if (!ctx || !s) { set_error("bie_kernel_modes_banded: NULL handle"); return BIE_EINVAL; }
  bie_status st = check_device(ctx, "bie_kernel_modes_banded");
  if (st != BIE_OK) return st;
  if (n_pairs < 0) { set_error("bie_kernel_modes_banded: n_pairs < 0"); return BIE_EINVAL; }
  if (n_pairs == 0) return BIE_OK;
  if (!pair_row || !pair_src || !modes_out) { set_error("bie_kernel_modes_banded: NULL buffer"); return BIE_EINVAL; }
  if (!(k > 0.0) || !std::isfinite(k)) { set_error("bie_kernel_modes_banded: k must be positive"); return BIE_EINVAL; }
  if (!(eps0 > 0.0) || eps0 > 1e-6) { set_error("bie_kernel_modes_banded: eps0 outside (0, 1e-6]"); return BIE_EINVAL; }
  const int d = theta_degree(s->sp), Mt = s->Mt;
  if (2 * d > kBandMaxM0) {
    set_error("bie_kernel_modes_banded: rho^2 has theta-degree %d (the route takes at most %d)", 2 * d, kBandMaxM0);
    return BIE_EINVAL;
  }
  if (Mt < 4 * d + 1 || Mt > 1024) {
    set_error("bie_kernel_modes_banded: Mth %d outside [%d, 1024]", Mt, 4 * d + 1);
    return BIE_EINVAL;
  }
  const int ucols = 2 * (2 * d) + 2;
  const size_t per_warp = (size_t)(Mt + 1) * (ucols + 1) * sizeof(cplx);
  const size_t smem_per_warp = (sizeof(BandSmem) + 2 * (size_t)(Mt + 1) * sizeof(cplx) + 15) / 16 * 16;
  const int wpb = (int)std::min<size_t>(kBandWarps, (227 * 1024) / smem_per_warp);
  if (wpb < 1) { set_error("bie_kernel_modes_banded: Mth %d needs too much shared memory", Mt); return BIE_EINVAL; }
  int64_t warps = std::min<int64_t>((n_pairs + wpb - 1) / wpb * wpb, (int64_t)ctx->sms * 8 * wpb);
  warps = std::min<int64_t>(warps, std::max<int64_t>(wpb, (int64_t)(kBandScratchCap / per_warp) / wpb * wpb));
  st = band_grow(ctx, per_warp * warps);
  if (st != BIE_OK) return st;
  const size_t smem = wpb * smem_per_warp;
  st = band_smem_attr(1, ctx->device, smem);
  if (st != BIE_OK) return st;
  BandSArgs a = {};
  a.S = s->sp;
  a.Mt = Mt;
  a.Np = s->Np;
  a.N = s->N;
  a.n = n_pairs;
  a.k = k;
  a.eps0 = eps0;
  a.m0cap = 2 * d;
  a.t_nodes = s->t_nodes;
  a.thg = s->thgrid;
  a.ring_t = s->ring_t;
  a.tw = s->tw;
  a.T = s->tw_len;
  a.rows = pair_row;
  a.srcs = pair_src;
  a.ucols = ucols;
  a.scratch = reinterpret_cast<cplx*>(ctx->band_scratch);
  a.modes_out = modes_out;
  a.status = ctx->d_status;
  a.warps = wpb;
  a.smem_per_warp = smem_per_warp;
  band_s_modes_kernel<<<(unsigned)(warps / wpb), 32 * wpb, smem, ctx->stream>>>(a);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "band_s_modes_kernel launch");
  return BIE_OK;
}

}  // extern "C"
