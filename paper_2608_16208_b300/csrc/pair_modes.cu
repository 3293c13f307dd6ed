// Per-pair pipeline of the correction stage (Sections 3.2-3.4, 4): for a target
// node x = r(t_j^l, th_i) and a GGQ source ring t_s, the theta_s-Fourier modes
// of the single-layer kernel e^{ik rho}/rho by singularity swapping, and their
// Parseval weights on the theta grid.
//
// One warp per pair.  Steps (all FP64):
//   1. rho^2 on the ring (Eq. (rho)); samples with |t - t_s| + |th - th_q| <=
//      kStableDelta use the line integral of the Section 4 Remark, its 16
//      Gauss-Legendre nodes spread over 16 lanes.
//   2. a0 = grid argmin refined by real Newton, b0 = sqrt(2 rho^2(a0)/rho^2''(a0)),
//      complex Newton for theta_+ = a + ib on the analytic continuation
//      (Section 3.3); roots beyond kBCap are replaced by (a0, kBCap).
//   3. A_m(b), m = 0..3M (Eq. (Am)): closed-form A_0, A_1 by the AGM, then the
//      difference recurrence (Eq. (diff-recurrence)) if 3M b <= 7, else
//      Miller's backward recurrence on the ratios A_{m-1}/A_m.
//   4. Smooth factors F = (s_{a,b}/rho^2)^{1/2} (Eq. (F-smooth)) and cos(k rho)
//      packed as one complex FFT of length Mth.
//   5. Zero-padded FFT convolution (Eq. (convolution) followed by the
//      <cos k rho> (x) <rho^{-1}> product of Eq. (Sphi:appr2), merged by
//      associativity): the product of the two trigonometric interpolants is
//      sampled, shifted by a, on P = 3 Mth points (one inverse FFT), multiplied
//      by the transform of the circulant A_{|d|}, |d| <= 3M, and transformed
//      back; modes |m| <= M are exact linear-convolution values.
//   6. K_m = e^{-ima} y_m + i <sin(k rho)/rho>_m;  Parseval weights
//      W_l' = (1/Mth) sum'_m K_m e^{i m th_l'}  (Section 3.4).
#include <cmath>

#include "bie_internal.cuh"
#include "pair_args.cuh"

namespace bie {



__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// K(m), E(m) by the arithmetic-geometric mean (DLMF 19.8.1, 19.8.6); m1 = 1 - m.
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

// A_m(b), m = 0..L, sequential (one lane).  Same branches as the CPU restatement.
__device__ inline void a_modes_seq(double b, int L, double* A, double* D) {
  const double q = exp(-b);
  double K, E;
  ellipke(q * q, -expm1(-2 * b), &K, &E);
  const double A0 = 2 / kPi * K;
  const double sh2 = sinh(b / 2) * sinh(b / 2);
  if (L * b <= kForwardLimit) {
    double am = A0, dm = (2 / kPi) * ((K - E) / q - K);
    A[0] = am;
    if (D) D[0] = -dm;
    am += dm;
    A[1] = am;
    if (D) D[1] = dm;
    for (int m = 1; m < L; ++m) {
      dm = ((2 * m - 1) * dm + 8 * m * sh2 * am) / (2 * m + 1);
      am += dm;
      A[m + 1] = am;
      if (D) D[m + 1] = dm;
    }
    return;
  }
  // Miller: delta_m = A_{m-1}/A_m - 1 from m = N down to 1 (A_{N+1} = 0), stored for m <= L.
  const int N = L + (int)ceil(kMillerLog / (2 * b)) + 16;
  double dn = (2.0 * N + 1 + 8.0 * N * sh2) / (2.0 * N - 1);
  for (int m = N - 1; m > L; --m) dn = (8 * m * sh2 + (2 * m + 1) * dn / (1 + dn)) / (2 * m - 1);
  // dn = delta_{L+1}; now the stored range
  for (int m = L; m >= 1; --m) {
    dn = (8 * m * sh2 + (2 * m + 1) * dn / (1 + dn)) / (2 * m - 1);
    A[m] = dn;  // temporarily delta_m
  }
  double am = A0;
  A[0] = am;
  for (int m = 1; m <= L; ++m) {
    const double dl = A[m];
    const double an = am / (1 + dl);
    if (D) D[m] = -an * dl;
    am = an;
    A[m] = am;
  }
  if (D) D[0] = -D[1];
}

struct RootOut {
  double a, b, a0, b0;
  int capped;
};

// rho^2 and derivatives at real theta_s = z (warp-cooperative; identical on all lanes).
__device__ inline void eval_real(const PairArgs& a, double ts, double t, double th, const R3& x, double z, double* g0,
                                 double* g1, double* g2) {
  const int lane = threadIdx.x & 31;
  Geo G;
  surf_eval(a.S, ts, z, 2, &G);
  R3 Y = {G.r.x - x.x, G.r.y - x.y, G.r.z - x.z};
  const double dt = t - ts;
  const double dth = wrap_pi(th - z);
  const bool near = fabs(dt) + fabs(dth) <= kStableDelta;
  if (near) {
    double cx = 0, cy = 0, cz = 0;
    if (lane < 16) {
      Geo P;
      surf_eval(a.S, ts + a.gl.x[lane] * dt, z + a.gl.x[lane] * dth, 1, &P);
      const double w = a.gl.w[lane];
      cx = w * (dt * P.rt.x + dth * P.rth.x);
      cy = w * (dt * P.rt.y + dth * P.rth.y);
      cz = w * (dt * P.rt.z + dth * P.rth.z);
    }
    Y = {-warp_sum(cx), -warp_sum(cy), -warp_sum(cz)};
  }
  *g0 = dot(Y, Y);
  *g1 = 2 * dot(Y, G.rth);
  *g2 = 2 * (dot(G.rth, G.rth) + dot(Y, G.rthth));
}

// rho^2(zeta) and its derivative for complex zeta (warp-cooperative).
__device__ inline void eval_cplx(const PairArgs& a, double ts, double t, double th, const R3& x, cplx z, cplx* P,
                                 cplx* dP) {
  const int lane = threadIdx.x & 31;
  C3 r, rt, rth;
  surf_eval_c(a.S, ts, z, &r, &rt, &rth);
  C3 Y = {r.x - C(x.x), r.y - C(x.y), r.z - C(x.z)};
  const double dt = t - ts;
  const cplx dth = C(wrap_pi(th - z.re), -z.im);
  const bool near = fabs(dt) + fabs(dth.re) <= kStableDelta;
  if (near) {
    cplx cx = C(0), cy = C(0), cz = C(0);
    if (lane < 16) {
      C3 pr, prt, prth;
      surf_eval_c(a.S, ts + a.gl.x[lane] * dt, z + a.gl.x[lane] * dth, &pr, &prt, &prth);
      const double w = a.gl.w[lane];
      cx = w * (dt * prt.x + prth.x * dth);
      cy = w * (dt * prt.y + prth.y * dth);
      cz = w * (dt * prt.z + prth.z * dth);
    }
    Y = {C(-warp_sum(cx.re), -warp_sum(cx.im)), C(-warp_sum(cy.re), -warp_sum(cy.im)),
         C(-warp_sum(cz.re), -warp_sum(cz.im))};
  }
  *P = Y.x * Y.x + Y.y * Y.y + Y.z * Y.z;
  *dP = 2.0 * (Y.x * rth.x + Y.y * rth.y + Y.z * rth.z);
}

__device__ inline RootOut locate_root(const PairArgs& a, double ts, double t, double th, const R3& x, double a0) {
  const double hgrid = kTwoPi / a.Mt;
  const double start = a0;
  double g0, g1, g2;
  for (int it = 0; it < 40; ++it) {
    eval_real(a, ts, t, th, x, a0, &g0, &g1, &g2);
    double step = g2 > 0 ? g1 / g2 : 0.0;
    step = fmin(fmax(step, -hgrid), hgrid);
    a0 = fmin(fmax(a0 - step, start - hgrid), start + hgrid);
    if (fabs(step) <= 1e-15 * (1 + fabs(a0))) break;
  }
  eval_real(a, ts, t, th, x, a0, &g0, &g1, &g2);
  const double b0 = sqrt(2 * g0 / (g2 > 0 ? g2 : 0.0));
  RootOut o;
  o.a0 = a0;
  o.b0 = b0;
  o.capped = !(b0 <= kBCap);
  cplx z = C(a0, o.capped ? kBCap : b0);
  bool done = o.capped, extra = false;
  for (int it = 0; it < 60 && !done; ++it) {
    cplx P, dP;
    eval_cplx(a, ts, t, th, x, z, &P, &dP);
    const cplx dz = cdiv(P, dP);
    cplx zn = z - dz;
    if (zn.im < 0) zn = conj(zn);
    const bool over = !(zn.im <= kBCap);
    if (over) {
      o.capped = 1;
      zn = C(a0, kBCap);
    }
    z = zn;
    const bool small = sqrt(abs2(dz)) <= kRootTol * fabs(z.im) + 4e-16 * sqrt(abs2(z));
    if (over || extra) done = true;
    extra = extra || small;
  }
  o.a = z.re;
  o.b = z.im;
  return o;
}

__global__ void __launch_bounds__(128) pair_s_kernel(const PairArgs a) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int Mt = a.Mt, M = a.M, P = a.P, L = a.L;
  // per-warp shared memory (doubles): 6 Mt + 5 P + L + 5
  const int per_warp = 6 * Mt + 5 * P + L + 5;
  double* base = smem + (size_t)wib * per_warp;
  double* rho2 = base;                      // Mt
  double* sn = rho2 + Mt;                   // Mt
  double* Acal = sn + Mt;                   // P: transform of the circulant A_{|d|}
  cplx* bufA = (cplx*)(Acal + P);           // P
  cplx* bufB = bufA + P;                    // P
  double* Atab = (double*)(bufB + P);       // L + 1
  cplx* ph = (cplx*)(Atab + L + 1);         // 2M + 1: e^{i j a}, j = -M..M
  cplx* kc = ph + 2 * M + 1;                // 2M + 1: Kc_m, m = -M..M
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t p = warp; p < a.n_pairs; p += nwarps) {
    // ---- decode the pair
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
    const int64_t tn = row / Mt;
    const int i = (int)(row % Mt);
    const int j = (int)(tn / 16);
    const int ip = j + d - 1;
    if (row < 0 || row >= a.N || d < 0 || ip < 0 || ip >= a.Np) {
      if (a.modes_out)
        for (int m = lane; m < 2 * (Mt + 1); m += 32) a.modes_out[p * 2 * (Mt + 1) + m] = 0.0;
      if (a.weights_out)
        for (int m = lane; m < Mt; m += 32) a.weights_out[p * Mt + m] = C(0.0);
      if (!a.enumerate && lane == 0) atomicAdd(a.status, 1);
      continue;
    }
    const int64_t ring = (tn * 3 + d) * 16 + g;
    const double t = a.t_nodes[tn];
    const double th = kTwoPi * i / Mt;
    const double ts = a.ring_t[ring];
    const R3 x = {a.pts[3 * row], a.pts[3 * row + 1], a.pts[3 * row + 2]};
    const double* rr = a.ring_r + ring * 3 * Mt;
    const double dts = fabs(t - ts);
    // ---- 1. rho^2 on the ring (direct), then the near samples by the line integral
    for (int q = lane; q < Mt; q += 32) {
      const double yx = rr[3 * q] - x.x, yy = rr[3 * q + 1] - x.y, yz = rr[3 * q + 2] - x.z;
      rho2[q] = yx * yx + yy * yy + yz * yz;
    }
    __syncwarp();
    {
      const int K = (int)ceil(kStableDelta * Mt / kTwoPi) + 1;
      for (int c0 = -K; c0 <= K; c0 += 2) {
        const int c = c0 + (lane >> 4);
        const int q = ((i + c) % Mt + Mt) % Mt;
        const double thq = kTwoPi * q / Mt;
        const double dth = wrap_pi(th - thq);
        const bool nearq = (c <= K) && (dts + fabs(dth) <= kStableDelta);
        if (!__ballot_sync(0xffffffffu, nearq)) continue;
        double cx = 0, cy = 0, cz = 0;
        if (nearq) {
          const int jn = lane & 15;
          Geo G;
          const double dt = t - ts;
          surf_eval(a.S, ts + a.gl.x[jn] * dt, thq + a.gl.x[jn] * dth, 1, &G);
          const double w = a.gl.w[jn];
          cx = w * (dt * G.rt.x + dth * G.rth.x);
          cy = w * (dt * G.rt.y + dth * G.rth.y);
          cz = w * (dt * G.rt.z + dth * G.rth.z);
        }
        for (int o = 8; o; o >>= 1) {
          cx += __shfl_xor_sync(0xffffffffu, cx, o);
          cy += __shfl_xor_sync(0xffffffffu, cy, o);
          cz += __shfl_xor_sync(0xffffffffu, cz, o);
        }
        if (nearq && (lane & 15) == 0) rho2[q] = cx * cx + cy * cy + cz * cz;
      }
    }
    __syncwarp();
    // grid minimiser; near-ties (within 1e-12) go to the sample nearest the target angle
    // (integer grid distance), then to the lower index
    double bv = INFINITY;
    for (int q = lane; q < Mt; q += 32) bv = fmin(bv, rho2[q]);
    for (int o = 16; o; o >>= 1) bv = fmin(bv, __shfl_xor_sync(0xffffffffu, bv, o));
    int bkey = 0x7fffffff;
    for (int q = lane; q < Mt; q += 32) {
      if (rho2[q] <= bv * (1 + 1e-12)) {
        const int dq = q > i ? q - i : i - q;
        const int key = min(dq, Mt - dq) * Mt + q;
        bkey = min(bkey, key);
      }
    }
    for (int o = 16; o; o >>= 1) bkey = min(bkey, __shfl_xor_sync(0xffffffffu, bkey, o));
    const int bi = bkey % Mt;
    // ---- 2. complex root
    const RootOut ro = locate_root(a, ts, t, th, x, kTwoPi * bi / Mt);
    const double ra = ro.a, rb = ro.b;
    // ---- 3. A_m(b), m = 0..L, and the transform of the circulant A_{|d|}, |d| <= 3M
    if (lane == 0) a_modes_seq(rb, L, Atab, nullptr);
    __syncwarp();
    for (int pp = lane; pp < P; pp += 32) {
      const int dd = pp <= P / 2 ? pp : P - pp;
      bufA[pp] = C(dd <= 3 * M ? Atab[dd] : 0.0, 0.0);
    }
    __syncwarp();
    {
      const cplx* Af = warp_fft(bufA, bufB, P, a.tw, a.T, -1);
      for (int pp = lane; pp < P; pp += 32) Acal[pp] = Af[pp].re;
    }
    for (int jj = lane; jj <= 2 * M; jj += 32) ph[jj] = cexpi((jj - M) * ra);
    // ---- 4. smooth factors, packed: F + i cos(k rho)
    const double qb = exp(-rb), om = -expm1(-rb);
    for (int q = lane; q < Mt; q += 32) {
      const double phi = kTwoPi * q / Mt - ra;
      const double sp = sin(phi / 2);
      const double s = om * om + 4 * qb * sp * sp;
      const double r2 = rho2[q];
      const double rho = sqrt(r2);
      double skr, ckr;
      sincos(a.k * rho, &skr, &ckr);
      bufA[q] = C(sqrt(s / r2), ckr);
      sn[q] = skr / rho;
    }
    __syncwarp();
    cplx* Z = warp_fft(bufA, bufB, Mt, a.tw, a.T, -1);
    cplx* Xb = (Z == bufA) ? bufB : bufA;
    // ---- 5. e^{ija} Z_j / Mt on the P grid (Nyquist split evenly), inverse FFT
    for (int pp = lane; pp < P; pp += 32) Xb[pp] = C(0.0);
    __syncwarp();
    for (int jj = lane; jj <= 2 * M; jj += 32) {
      const int jv = jj - M;
      cplx z = Z[(jv + Mt) % Mt] * (1.0 / Mt);
      if (jv == M || jv == -M) z = 0.5 * z;
      Xb[(jv + P) % P] = ph[jj] * z;
    }
    __syncwarp();
    cplx* Zt = warp_fft(Xb, Z, P, a.tw, a.T, +1);
    // U_p = F~(phi_p + a) C~(phi_p + a) Acal_p
    for (int pp = lane; pp < P; pp += 32) Zt[pp] = C(Zt[pp].re * Zt[pp].im * Acal[pp], 0.0);
    __syncwarp();
    const cplx* Yf = warp_fft(Zt, (Zt == bufA) ? bufB : bufA, P, a.tw, a.T, -1);
    for (int mm = lane; mm <= 2 * M; mm += 32) {
      const int m = mm - M;
      kc[mm] = conj(ph[mm]) * Yf[(m + P) % P] * (1.0 / P);
    }
    __syncwarp();
    // ---- 6. outputs
    if (a.modes_out) {
      for (int q = lane; q < Mt; q += 32) bufA[q] = C(sn[q], 0.0);
      __syncwarp();
      const cplx* Sf = warp_fft(bufA, bufB, Mt, a.tw, a.T, -1);
      double* out = a.modes_out + p * 2 * (Mt + 1);
      for (int mm = lane; mm <= 2 * M; mm += 32) {
        const int m = mm - M;
        cplx sv = Sf[(m + Mt) % Mt] * (1.0 / Mt);
        if (m == M || m == -M) sv = 0.5 * sv;
        out[2 * mm] = kc[mm].re - sv.im;
        out[2 * mm + 1] = kc[mm].im + sv.re;
      }
      __syncwarp();
    }
    if (a.weights_out) {
      // Q[m mod Mt] = Kc_m (|m| < M), Q[M] = (Kc_M + Kc_{-M})/2;  W = IFFT(Q)/Mt + i sn/Mt
      for (int q = lane; q < Mt; q += 32) {
        const int m = q < M ? q : q - Mt;
        bufA[q] = (q == M) ? 0.5 * (kc[2 * M] + kc[0]) : kc[m + M];
      }
      __syncwarp();
      const cplx* Wt = warp_fft(bufA, bufB, Mt, a.tw, a.T, +1);
      for (int q = lane; q < Mt; q += 32) {
        const cplx w = Wt[q] * (1.0 / Mt);
        a.weights_out[p * Mt + q] = C(w.re, w.im + sn[q] / Mt);
      }
    }
    __syncwarp();
  }
}

size_t pair_s_smem_per_warp(int Mt) {
  const int P = 3 * Mt, L = 3 * (Mt / 2);
  return sizeof(double) * (size_t)(6 * Mt + 5 * P + L + 5);
}

PairArgs make_pair_args(bie_surface s, double k) {
  PairArgs a;
  a.S = s->sp;
  a.gl = s->gl01;
  a.Np = s->Np;
  a.Mt = s->Mt;
  a.M = s->Mt / 2;
  a.P = 3 * s->Mt;
  a.T = s->tw_len;
  a.L = 3 * a.M;
  a.h = s->h;
  a.k = k;
  a.N = s->N;
  a.t_nodes = s->t_nodes;
  a.pts = s->pts;
  a.ring_t = s->ring_t;
  a.ring_r = s->ring_r;
  a.ring_n = s->ring_n;
  a.tw = s->tw;
  a.rows = nullptr;
  a.srcs = nullptr;
  a.modes_out = nullptr;
  a.weights_out = nullptr;
  a.status = s->ctx->d_status;
  a.enumerate = 0;
  a.p0 = 0;
  a.n_pairs = 0;
  return a;
}

bie_status launch_pairs(bie_surface s, const PairArgs& a) {
  const int warps_per_block = 4;
  const size_t smem = pair_s_smem_per_warp(s->Mt) * warps_per_block;
  static int configured_smem = 0;
  cudaError_t e;
  if ((int)smem > configured_smem) {
    e = cudaFuncSetAttribute(pair_s_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(pair_s_kernel)");
    configured_smem = (int)smem;
  }
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pair_s_kernel, 32 * warps_per_block, smem);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy(pair_s_kernel)");
  if (per_sm < 1) { set_error("pair kernel does not fit (smem %zu)", smem); return BIE_EUNSUPPORTED; }
  int64_t blocks = (int64_t)s->ctx->sms * per_sm;
  const int64_t need = (a.n_pairs + warps_per_block - 1) / warps_per_block;
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  pair_s_kernel<<<(unsigned)blocks, 32 * warps_per_block, smem, s->ctx->stream>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "pair_s_kernel launch");
  return BIE_OK;
}

}  // namespace bie

using namespace bie;

extern "C" bie_status bie_kernel_modes(bie_ctx ctx, bie_surface s, unsigned kernels, double k,
                                       const int64_t* pair_row, const int32_t* pair_src, int64_t n_pairs,
                                       double* modes_out) {
  if (!ctx || !s || (n_pairs > 0 && (!pair_row || !pair_src || !modes_out)) || n_pairs < 0) {
    set_error("bie_kernel_modes: invalid arguments");
    return BIE_EINVAL;
  }
  if (!(k > 0) || !(k < 1e6)) { set_error("bie_kernel_modes: k must be in (0, 1e6)"); return BIE_EINVAL; }
  if (kernels != BIE_KERNEL_S) {
    set_error("bie_kernel_modes: this build computes BIE_KERNEL_S");
    return BIE_EUNSUPPORTED;
  }
  if (n_pairs == 0) return BIE_OK;
  PairArgs a = make_pair_args(s, k);
  a.rows = pair_row;
  a.srcs = pair_src;
  a.n_pairs = n_pairs;
  a.modes_out = modes_out;
  return launch_pairs(s, a);
}
