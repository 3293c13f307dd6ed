// Learned preconditioner: a 4-layer convolutional network on the (t, theta) grid of the unknowns,
// trained on systems the method generates, used inside FGMRES as a flexible preconditioner on top
// of the block-diagonal one:  z = B^{-1} r + s (o_0 + i o_1),  o = net(features(r)),  s = rms(r).
//
// Network: 3x3 convolutions 4 -> 32 -> 32 -> 32 -> 2 with dilations 1, 2, 4, 1 (both axes), ReLU
// after the first three, theta periodic and t zero-padded.  Input features of a residual r
// (unknown index t * M_theta + theta, t = panel * 16 + node): Re r / s, Im r / s, J / mean(J), k / 25.
// Weights: FP32 master copy (Adam); every forward and backward pass uses their BF16 rounding, with
// FP32 activations and FP32 accumulation.
//
// Training objective on a system A (FP32 copy), for a batch of residuals r_b:
//   L = (1/B) sum_b ||A z_b - r_b||^2 / ||r_b||^2,
//   dL/dz_b = (2 / (B ||r_b||^2)) A^H (A z_b - r_b)  (gradient w.r.t. (Re z, Im z) as a complex vector).
// Residual batches: half complex white noise, half A x with white x (the smooth part of the
// spectrum), drawn from splitmix64 (counter-based) and Box-Muller.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "bie_internal.cuh"

namespace bie {

constexpr int kNetW = 32, kNetIn = 4, kNetOut = 2;
constexpr int kOffW0 = 0;
constexpr int kOffB0 = kOffW0 + kNetW * kNetIn * 9;
constexpr int kOffW1 = kOffB0 + kNetW;
constexpr int kOffB1 = kOffW1 + kNetW * kNetW * 9;
constexpr int kOffW2 = kOffB1 + kNetW;
constexpr int kOffB2 = kOffW2 + kNetW * kNetW * 9;
constexpr int kOffW3 = kOffB2 + kNetW;
constexpr int kOffB3 = kOffW3 + kNetOut * kNetW * 9;
constexpr int kNetParams = kOffB3 + kNetOut;
static_assert(kNetParams == BIE_NET_PARAMS, "parameter count");

struct Layer {
  int cin, cout, dil, relu, w, b;
};
constexpr Layer kLayers[4] = {{kNetIn, kNetW, 1, 1, kOffW0, kOffB0},
                              {kNetW, kNetW, 2, 1, kOffW1, kOffB1},
                              {kNetW, kNetW, 4, 1, kOffW2, kOffB2},
                              {kNetW, kNetOut, 1, 0, kOffW3, kOffB3}};

// ------------------------------------------------------------------ convolution, forward form
// y[b][co][t][th] = bias[co] + sum_{ci, dt, dth} W[co][ci][dt][dth] x[b][ci][t + dil (dt - 1)][th + dil (dth - 1)]
// (theta index mod mt, zero outside 0 <= t < nt), ReLU if relu.  With TRANS the weights are those of
// the layer (COUT x CIN) transposed and flipped, which makes the kernel the adjoint (backward data);
// with mask, x is read as x * (mask > 0) (the ReLU derivative of the layer's output).
template <int CIN, int COUT, bool TRANS>
__global__ void __launch_bounds__(256) conv_fwd_kernel(int B, int nt, int mt, int dil, const float* __restrict__ x,
                                                       const float* __restrict__ mask, const float* __restrict__ w,
                                                       const float* __restrict__ bias, int relu,
                                                       float* __restrict__ y) {
  constexpr int CP = (COUT + 3) / 4 * 4;
  __shared__ __align__(16) float ws[CIN * 9 * CP];
  for (int e = threadIdx.x; e < CIN * 9 * CP; e += blockDim.x) {
    const int co = e % CP, tap = (e / CP) % 9, ci = e / (CP * 9);
    float v = 0.f;
    if (co < COUT) v = TRANS ? w[(ci * COUT + co) * 9 + (8 - tap)] : w[(co * CIN + ci) * 9 + tap];
    ws[e] = v;
  }
  __syncthreads();
  const int64_t plane = (int64_t)nt * mt;
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (int64_t)B * plane) return;
  const int b = (int)(p / plane);
  const int t = (int)((p / mt) % nt), th = (int)(p % mt);
  float acc[CP];
#pragma unroll
  for (int co = 0; co < CP; ++co) acc[co] = 0.f;
  const float* xb = x + (int64_t)b * CIN * plane;
  const float* mb = mask ? mask + (int64_t)b * CIN * plane : nullptr;
#pragma unroll
  for (int dt = 0; dt < 3; ++dt) {
    const int tt = t + dil * (dt - 1);
    if (tt < 0 || tt >= nt) continue;
#pragma unroll
    for (int dp = 0; dp < 3; ++dp) {
      int th2 = th + dil * (dp - 1);
      th2 = th2 < 0 ? th2 + mt : (th2 >= mt ? th2 - mt : th2);
      const int64_t off = (int64_t)tt * mt + th2;
      const int tap = dt * 3 + dp;
      for (int ci = 0; ci < CIN; ++ci) {
        float v = xb[(int64_t)ci * plane + off];
        if (mb && !(mb[(int64_t)ci * plane + off] > 0.f)) v = 0.f;
        const float4* wr = reinterpret_cast<const float4*>(ws + (ci * 9 + tap) * CP);
#pragma unroll
        for (int q = 0; q < CP / 4; ++q) {
          const float4 wq = wr[q];
          acc[4 * q + 0] = fmaf(wq.x, v, acc[4 * q + 0]);
          acc[4 * q + 1] = fmaf(wq.y, v, acc[4 * q + 1]);
          acc[4 * q + 2] = fmaf(wq.z, v, acc[4 * q + 2]);
          acc[4 * q + 3] = fmaf(wq.w, v, acc[4 * q + 3]);
        }
      }
    }
  }
  float* yb = y + (int64_t)b * COUT * plane + (int64_t)t * mt + th;
#pragma unroll
  for (int co = 0; co < COUT; ++co) {
    float v = acc[co] + (bias ? bias[co] : 0.f);
    if (relu) v = fmaxf(v, 0.f);
    yb[(int64_t)co * plane] = v;
  }
}

// ------------------------------------------------------------------ convolution, weight gradient
// Partial sums, per CTA, of gW[co][ci][tap] = sum g[b][co][t][th] x[b][ci][t + dil (dt - 1)][th + dil (dth - 1)]
// and gb[co] = sum g[b][co][t][th], over the CTA's image b and rows [r0, r0 + rows); g is read as
// g * (mask > 0) when mask is given.  One thread per (co, ci); input rows and the g row are staged
// in shared memory by theta chunks of 64.
constexpr int kWgChunk = 64;
template <int CIN, int COUT>
__global__ void __launch_bounds__(CIN * COUT) conv_wgrad_kernel(int B, int nt, int mt, int dil, int rows,
                                                                const float* __restrict__ x,
                                                                const float* __restrict__ g,
                                                                const float* __restrict__ mask,
                                                                float* __restrict__ partial) {
  constexpr int XW = kWgChunk + 8;  // chunk + halo (dil <= 4), padded stride
  __shared__ float xs[CIN][3][XW + 1];
  __shared__ float gs[COUT][kWgChunk];
  const int tiles = (nt + rows - 1) / rows;
  const int b = blockIdx.x / tiles, r0 = (blockIdx.x % tiles) * rows;
  const int co = threadIdx.x / CIN, ci = threadIdx.x % CIN;
  const int64_t plane = (int64_t)nt * mt;
  float acc[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) acc[i] = 0.f;
  float accb = 0.f;
  for (int t = r0; t < min(r0 + rows, nt); ++t) {
    for (int c0 = 0; c0 < mt; c0 += kWgChunk) {
      const int cw = min(kWgChunk, mt - c0);
      __syncthreads();
      for (int e = threadIdx.x; e < CIN * 3 * (cw + 2 * dil); e += blockDim.x) {
        const int j = e % (cw + 2 * dil), rr = (e / (cw + 2 * dil)) % 3, c = e / (3 * (cw + 2 * dil));
        const int tt = t + dil * (rr - 1);
        int th = c0 + j - dil;
        th = th < 0 ? th + mt : (th >= mt ? th - mt : th);
        xs[c][rr][j] = (tt >= 0 && tt < nt) ? x[((int64_t)b * CIN + c) * plane + (int64_t)tt * mt + th] : 0.f;
      }
      for (int e = threadIdx.x; e < COUT * cw; e += blockDim.x) {
        const int j = e % cw, c = e / cw;
        const int64_t idx = ((int64_t)b * COUT + c) * plane + (int64_t)t * mt + c0 + j;
        float v = g[idx];
        if (mask && !(mask[idx] > 0.f)) v = 0.f;
        gs[c][j] = v;
      }
      __syncthreads();
      for (int j = 0; j < cw; ++j) {
        const float gv = gs[co][j];
        accb += gv;
#pragma unroll
        for (int rr = 0; rr < 3; ++rr)
#pragma unroll
          for (int dp = 0; dp < 3; ++dp) acc[rr * 3 + dp] = fmaf(gv, xs[ci][rr][j + dil * dp], acc[rr * 3 + dp]);
      }
    }
  }
  float* out = partial + (int64_t)blockIdx.x * (COUT * CIN * 9 + COUT);
#pragma unroll
  for (int tap = 0; tap < 9; ++tap) out[(co * CIN + ci) * 9 + tap] = acc[tap];
  if (ci == 0) out[COUT * CIN * 9 + co] = accb;
}

// gparams[wOff + e] (e < COUT CIN 9) and gparams[bOff + co] = sums over the CTA partials (deterministic order).
__global__ void wgrad_reduce_kernel(int nblk, int nw, int nb, const float* __restrict__ partial, int wOff, int bOff,
                                    float* __restrict__ gparams) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nw + nb) return;
  float s = 0.f;
  for (int k = 0; k < nblk; ++k) s += partial[(int64_t)k * (nw + nb) + e];
  gparams[e < nw ? wOff + e : bOff + (e - nw)] = s;
}

// ------------------------------------------------------------------ skinny complex products (FP32)
// Y[v] = A X[v] for nv <= 16 vectors (A [N][N] row-major, vectors as rows [nv][N]); two rows per warp,
// X staged by chunks of 256 columns in shared memory.
constexpr int kMaxVec = 16;
__global__ void __launch_bounds__(256) cgemm_ax_kernel(int64_t N, int nv, const float2* __restrict__ A,
                                                       const float2* __restrict__ X, float2* __restrict__ Y) {
  __shared__ float2 xs[kMaxVec][256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i0 = (int64_t)blockIdx.x * 16 + warp * 2;
  float2 acc0[kMaxVec], acc1[kMaxVec];
#pragma unroll
  for (int v = 0; v < kMaxVec; ++v) acc0[v] = acc1[v] = make_float2(0.f, 0.f);
  for (int64_t c0 = 0; c0 < N; c0 += 256) {
    __syncthreads();
    for (int e = threadIdx.x; e < kMaxVec * 256; e += 256) {
      const int v = e >> 8, c = e & 255;
      xs[v][c] = (v < nv && c0 + c < N) ? X[(int64_t)v * N + c0 + c] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int cc = lane; cc < 256; cc += 32) {
      const int64_t c = c0 + cc;
      if (c >= N) break;
      const float2 a0 = i0 < N ? A[i0 * N + c] : make_float2(0.f, 0.f);
      const float2 a1 = i0 + 1 < N ? A[(i0 + 1) * N + c] : make_float2(0.f, 0.f);
#pragma unroll
      for (int v = 0; v < kMaxVec; ++v) {
        const float2 xv = xs[v][cc];
        acc0[v].x = fmaf(a0.x, xv.x, fmaf(-a0.y, xv.y, acc0[v].x));
        acc0[v].y = fmaf(a0.x, xv.y, fmaf(a0.y, xv.x, acc0[v].y));
        acc1[v].x = fmaf(a1.x, xv.x, fmaf(-a1.y, xv.y, acc1[v].x));
        acc1[v].y = fmaf(a1.x, xv.y, fmaf(a1.y, xv.x, acc1[v].y));
      }
    }
  }
#pragma unroll
  for (int v = 0; v < kMaxVec; ++v) {
    for (int o = 16; o > 0; o >>= 1) {
      acc0[v].x += __shfl_xor_sync(0xffffffffu, acc0[v].x, o);
      acc0[v].y += __shfl_xor_sync(0xffffffffu, acc0[v].y, o);
      acc1[v].x += __shfl_xor_sync(0xffffffffu, acc1[v].x, o);
      acc1[v].y += __shfl_xor_sync(0xffffffffu, acc1[v].y, o);
    }
  }
  if (lane == 0) {
#pragma unroll
    for (int v = 0; v < kMaxVec; ++v) {
      if (v >= nv) break;
      if (i0 < N) Y[(int64_t)v * N + i0] = acc0[v];
      if (i0 + 1 < N) Y[(int64_t)v * N + i0 + 1] = acc1[v];
    }
  }
}

// Y[v] = A^H E[v]: a CTA owns 32 columns (one per lane), its 8 warps split the rows; E staged by
// chunks of 64 rows in shared memory (broadcast reads).
__global__ void __launch_bounds__(256) cgemm_ahx_kernel(int64_t N, int nv, const float2* __restrict__ A,
                                                        const float2* __restrict__ E, float2* __restrict__ Y) {
  __shared__ float2 es[kMaxVec][64];
  __shared__ float2 red[8][kMaxVec][33];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t j = (int64_t)blockIdx.x * 32 + lane;
  float2 acc[kMaxVec];
#pragma unroll
  for (int v = 0; v < kMaxVec; ++v) acc[v] = make_float2(0.f, 0.f);
  for (int64_t i0 = 0; i0 < N; i0 += 64) {
    __syncthreads();
    for (int e = threadIdx.x; e < kMaxVec * 64; e += 256) {
      const int v = e >> 6, r = e & 63;
      es[v][r] = (v < nv && i0 + r < N) ? E[(int64_t)v * N + i0 + r] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int r = warp; r < 64; r += 8) {
      const int64_t i = i0 + r;
      if (i >= N) break;
      const float2 a = j < N ? A[i * N + j] : make_float2(0.f, 0.f);  // conj(a) e
#pragma unroll
      for (int v = 0; v < kMaxVec; ++v) {
        const float2 ev = es[v][r];
        acc[v].x = fmaf(a.x, ev.x, fmaf(a.y, ev.y, acc[v].x));
        acc[v].y = fmaf(a.x, ev.y, fmaf(-a.y, ev.x, acc[v].y));
      }
    }
  }
#pragma unroll
  for (int v = 0; v < kMaxVec; ++v) red[warp][v][lane] = acc[v];
  __syncthreads();
  for (int e = threadIdx.x; e < nv * 32; e += 256) {
    const int v = e >> 5, l = e & 31;
    float2 s = make_float2(0.f, 0.f);
    for (int w = 0; w < 8; ++w) { s.x += red[w][v][l].x; s.y += red[w][v][l].y; }
    const int64_t jj = (int64_t)blockIdx.x * 32 + l;
    if (jj < N) Y[(int64_t)v * N + jj] = s;
  }
}

// ------------------------------------------------------------------ elementwise and reductions
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  uint64_t z = x;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__device__ __forceinline__ double u01(uint64_t key, uint64_t ctr) {
  return (double)(splitmix64(key * 0x100000001B3ull + ctr) >> 11) * (1.0 / 9007199254740992.0);
}

// complex standard normal entries (E|z|^2 = 1) for [nv][N], counter = element index
__global__ void randn_kernel(int64_t total, uint64_t key, float2* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const double u1 = u01(key, 2 * e), u2 = u01(key, 2 * e + 1);
    const double rad = sqrt(-log1p(-u1));  // |z| with E|z|^2 = 1
    double s, c;
    sincospi(2.0 * u2, &s, &c);
    out[e] = make_float2((float)(rad * c), (float)(rad * s));
  }
}

// per-vector sums of |r|^2 (double accumulation); one CTA per vector
template <typename VT>
__global__ void sumsq_kernel(int64_t N, const VT* __restrict__ r, double* __restrict__ out) {
  const VT* rv = r + (int64_t)blockIdx.x * N;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
    const double a = rv[i].x, b = rv[i].y;
    s += a * a + b * b;
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) out[blockIdx.x] = s;
  }
}

// features [nv][4][nt][mt] of residuals r [nv][N] (N = nt mt): Re r / s, Im r / s, J / mean J, k / 25
template <typename VT>
__global__ void features_kernel(int nv, int64_t N, const VT* __restrict__ r, const double* __restrict__ sumsq,
                                const float* __restrict__ jn, float kfeat, float* __restrict__ f) {
  const int64_t total = (int64_t)nv * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = e / N, i = e - v * N;
    const double rms = sqrt(sumsq[v] / (double)N);
    const double inv = rms > 0.0 ? 1.0 / rms : 0.0;
    float* fv = f + v * 4 * N;
    fv[i] = (float)(r[e].x * inv);
    fv[N + i] = (float)(r[e].y * inv);
    fv[2 * N + i] = jn[i];
    fv[3 * N + i] = kfeat;
  }
}

// z = zb + s (o_0 + i o_1), per vector (VT = float2 in training, double2 in FGMRES)
template <typename VT>
__global__ void combine_kernel(int nv, int64_t N, const VT* __restrict__ zb, const float* __restrict__ o,
                               const double* __restrict__ sumsq, VT* __restrict__ z) {
  const int64_t total = (int64_t)nv * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = e / N, i = e - v * N;
    const double s = sqrt(sumsq[v] / (double)N);
    const float* ov = o + v * 2 * N;
    VT out;
    out.x = zb[e].x + s * ov[i];
    out.y = zb[e].y + s * ov[N + i];
    z[e] = out;
  }
}

// e = Az - r (in place into az) and per-vector |e|^2 into esq (atomic double adds)
__global__ void residual_kernel(int nv, int64_t N, const float2* __restrict__ r, float2* __restrict__ az,
                                double* __restrict__ esq) {
  const int v = blockIdx.y;
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = (int64_t)v * N + i;
    const float2 d = make_float2(az[e].x - r[e].x, az[e].y - r[e].y);
    az[e] = d;
    s += (double)d.x * d.x + (double)d.y * d.y;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(esq + v, s);
}

// go[v][0|1][i] = s_v c_v (Re|Im) gz[v][i], c_v = 2 / (nv |r_v|^2): gradient w.r.t. the network output
__global__ void outgrad_kernel(int nv, int64_t N, const float2* __restrict__ gz, const double* __restrict__ rsq,
                               float* __restrict__ go) {
  const int64_t total = (int64_t)nv * N;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t v = e / N, i = e - v * N;
    const double s = sqrt(rsq[v] / (double)N);
    const double c = rsq[v] > 0.0 ? 2.0 / ((double)nv * rsq[v]) : 0.0;
    go[v * 2 * N + i] = (float)(s * c * gz[e].x);
    go[v * 2 * N + N + i] = (float)(s * c * gz[e].y);
  }
}

__global__ void loss_kernel(int nv, const double* __restrict__ esq, const double* __restrict__ rsq,
                            float* __restrict__ loss) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int v = 0; v < nv; ++v) s += rsq[v] > 0.0 ? esq[v] / rsq[v] : 0.0;
  *loss = (float)(s / nv);
}

__global__ void round_bf16_kernel(int n, const float* __restrict__ w, float* __restrict__ wq) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < n) wq[e] = __bfloat162float(__float2bfloat16_rn(w[e]));
}

__global__ void adam_kernel(int n, float lr, float b1, float b2, float eps, float c1, float c2,
                            const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                            float* __restrict__ w, float* __restrict__ wq) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  const float ge = g[e];
  const float me = b1 * m[e] + (1.f - b1) * ge;
  const float ve = b2 * v[e] + (1.f - b2) * ge * ge;
  m[e] = me;
  v[e] = ve;
  const float we = w[e] - lr * (me / c1) / (sqrtf(ve / c2) + eps);
  w[e] = we;
  wq[e] = __bfloat162float(__float2bfloat16_rn(we));
}

__global__ void to_c64_kernel(int64_t total, const double2* __restrict__ a, float2* __restrict__ b) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    b[e] = make_float2((float)a[e].x, (float)a[e].y);
}

__global__ void jn_kernel(int64_t N, const double* __restrict__ J, float* __restrict__ jn) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) s += J[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) red[0] = s;
  }
  __syncthreads();
  const double mean = red[0] / (double)N;
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x) jn[i] = (float)(J[i] / mean);
}

}  // namespace bie

using namespace bie;

// ------------------------------------------------------------------ network object
struct bie_net_s {
  bie_ctx ctx;
  float* w = nullptr;     // FP32 master parameters
  float* wq = nullptr;    // their BF16 rounding (used by the kernels)
  float* m = nullptr;     // Adam moments
  float* v = nullptr;
  float* g = nullptr;     // gradient
  int64_t step = 0;
  // workspace, grown on demand
  float* act = nullptr;   // a0 | a1 | a2 | out, each [B][32][nt][mt] (out: [B][2])
  float* gbuf = nullptr;  // two [B][32][nt][mt] gradient buffers
  float* partial = nullptr;
  size_t act_elems = 0, partial_elems = 0;
};

struct bie_train_set_s {
  bie_ctx ctx;
  int64_t N;
  int nt, mt;
  double k;
  float2* A32 = nullptr;
  float* jn = nullptr;
  bie_blockdiag block = nullptr;
};

namespace bie {

static bie_status net_workspace(bie_net net, int B, int nt, int mt) {
  const size_t plane = (size_t)nt * mt;
  const size_t act = (size_t)B * plane * (3 * kNetW + kNetOut);
  const int tiles = (nt + 7) / 8;
  const size_t part = (size_t)B * tiles * (kNetW * kNetW * 9 + kNetW);
  if (act > net->act_elems) {
    cudaFree(net->act);
    cudaFree(net->gbuf);
    net->act = nullptr;
    net->gbuf = nullptr;
    net->act_elems = 0;
    cudaError_t e = cudaMalloc((void**)&net->act, sizeof(float) * act);
    if (e == cudaSuccess) e = cudaMalloc((void**)&net->gbuf, sizeof(float) * 2 * (size_t)B * plane * kNetW);
    if (e != cudaSuccess) return cuda_fail(e, "network workspace");
    net->act_elems = act;
  }
  if (part > net->partial_elems) {
    cudaFree(net->partial);
    net->partial = nullptr;
    net->partial_elems = 0;
    const cudaError_t e = cudaMalloc((void**)&net->partial, sizeof(float) * part);
    if (e != cudaSuccess) return cuda_fail(e, "network workspace");
    net->partial_elems = part;
  }
  return BIE_OK;
}

static float* act_ptr(bie_net net, int B, int nt, int mt, int l) {
  return net->act + (size_t)l * B * nt * mt * kNetW;  // l = 0, 1, 2: hidden; 3: output [B][2]
}

template <int CIN, int COUT, bool TRANS>
static void conv(cudaStream_t st, int B, int nt, int mt, int dil, const float* x, const float* mask, const float* w,
                 const float* bias, int relu, float* y) {
  const int64_t total = (int64_t)B * nt * mt;
  conv_fwd_kernel<CIN, COUT, TRANS><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(B, nt, mt, dil, x, mask, w,
                                                                                     bias, relu, y);
}

static bie_status net_forward_dev(bie_net net, int B, int nt, int mt, const float* x) {
  bie_status s = net_workspace(net, B, nt, mt);
  if (s) return s;
  const cudaStream_t st = net->ctx->stream;
  const float* wq = net->wq;
  float* a0 = act_ptr(net, B, nt, mt, 0);
  float* a1 = act_ptr(net, B, nt, mt, 1);
  float* a2 = act_ptr(net, B, nt, mt, 2);
  float* o = act_ptr(net, B, nt, mt, 3);
  conv<kNetIn, kNetW, false>(st, B, nt, mt, kLayers[0].dil, x, nullptr, wq + kOffW0, wq + kOffB0, 1, a0);
  conv<kNetW, kNetW, false>(st, B, nt, mt, kLayers[1].dil, a0, nullptr, wq + kOffW1, wq + kOffB1, 1, a1);
  conv<kNetW, kNetW, false>(st, B, nt, mt, kLayers[2].dil, a1, nullptr, wq + kOffW2, wq + kOffB2, 1, a2);
  conv<kNetW, kNetOut, false>(st, B, nt, mt, kLayers[3].dil, a2, nullptr, wq + kOffW3, wq + kOffB3, 0, o);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BIE_OK : cuda_fail(e, "network forward");
}

template <int CIN, int COUT>
static void wgrad(bie_net net, int B, int nt, int mt, int dil, const float* x, const float* g, const float* mask,
                  int wOff, int bOff) {
  const cudaStream_t st = net->ctx->stream;
  const int rows = 8, tiles = (nt + rows - 1) / rows;
  const int nblk = B * tiles;
  conv_wgrad_kernel<CIN, COUT><<<nblk, CIN * COUT, 0, st>>>(B, nt, mt, dil, rows, x, g, mask, net->partial);
  const int nw = COUT * CIN * 9;
  wgrad_reduce_kernel<<<(nw + COUT + 255) / 256, 256, 0, st>>>(nblk, nw, COUT, net->partial, wOff, bOff, net->g);
}

// gradient of sum(go * out) w.r.t. the parameters (into net->g) and the input x (into gx, if not null);
// the activations of the last forward pass on x are used.
static bie_status net_backward_dev(bie_net net, int B, int nt, int mt, const float* x, const float* go, float* gx) {
  const cudaStream_t st = net->ctx->stream;
  const float* wq = net->wq;
  const float* a0 = act_ptr(net, B, nt, mt, 0);
  const float* a1 = act_ptr(net, B, nt, mt, 1);
  const float* a2 = act_ptr(net, B, nt, mt, 2);
  float* g0 = net->gbuf;
  float* g1 = net->gbuf + (size_t)B * nt * mt * kNetW;
  // layer 3 (no ReLU): weights from (a2, go); data gradient w.r.t. a2 into g0
  wgrad<kNetW, kNetOut>(net, B, nt, mt, kLayers[3].dil, a2, go, nullptr, kOffW3, kOffB3);
  conv<kNetOut, kNetW, true>(st, B, nt, mt, kLayers[3].dil, go, nullptr, wq + kOffW3, nullptr, 0, g0);
  // layer 2: the gradient at its pre-activation is g0 * (a2 > 0)
  wgrad<kNetW, kNetW>(net, B, nt, mt, kLayers[2].dil, a1, g0, a2, kOffW2, kOffB2);
  conv<kNetW, kNetW, true>(st, B, nt, mt, kLayers[2].dil, g0, a2, wq + kOffW2, nullptr, 0, g1);
  // layer 1
  wgrad<kNetW, kNetW>(net, B, nt, mt, kLayers[1].dil, a0, g1, a1, kOffW1, kOffB1);
  conv<kNetW, kNetW, true>(st, B, nt, mt, kLayers[1].dil, g1, a1, wq + kOffW1, nullptr, 0, g0);
  // layer 0
  wgrad<kNetIn, kNetW>(net, B, nt, mt, kLayers[0].dil, x, g0, a0, kOffW0, kOffB0);
  if (gx) conv<kNetW, kNetIn, true>(st, B, nt, mt, kLayers[0].dil, g0, a0, wq + kOffW0, nullptr, 0, gx);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BIE_OK : cuda_fail(e, "network backward");
}

// One loss/gradient evaluation on residuals r [nv][N] (FP32 complex) of a training system: fills
// net->g and *loss_dev.  Work buffers: zb, z, az, f [nv][4][N], go [nv][2][N], d [3 nv] doubles.
struct TrainBufs {
  float2 *r, *zb, *z, *az;
  float *f, *go, *loss;
  double* d;
};

static bie_status loss_grad_dev(bie_net net, bie_train_set ts, int nv, TrainBufs& tb) {
  const cudaStream_t st = net->ctx->stream;
  const int64_t N = ts->N;
  const int G = net->ctx->sms * 4;
  double* rsq = tb.d;
  double* esq = tb.d + nv;
  // block-diagonal part zb = B^{-1} r (zero without a block preconditioner)
  if (ts->block) {
    const bie_status sb = blockdiag_apply_f32(ts->block, tb.r, nv, tb.zb);
    if (sb) return sb;
  } else {
    cudaMemsetAsync(tb.zb, 0, sizeof(float2) * nv * N, st);
  }
  sumsq_kernel<float2><<<nv, 256, 0, st>>>(N, tb.r, rsq);
  features_kernel<float2><<<G, 256, 0, st>>>(nv, N, tb.r, rsq, ts->jn, (float)(ts->k / 25.0), tb.f);
  bie_status s = net_forward_dev(net, nv, ts->nt, ts->mt, tb.f);
  if (s) return s;
  const float* o = act_ptr(net, nv, ts->nt, ts->mt, 3);
  combine_kernel<float2><<<G, 256, 0, st>>>(nv, N, tb.zb, o, rsq, tb.z);
  cgemm_ax_kernel<<<(unsigned)((N + 15) / 16), 256, 0, st>>>(N, nv, ts->A32, tb.z, tb.az);
  cudaMemsetAsync(esq, 0, sizeof(double) * nv, st);
  residual_kernel<<<dim3(64, nv), 256, 0, st>>>(nv, N, tb.r, tb.az, esq);
  loss_kernel<<<1, 32, 0, st>>>(nv, esq, rsq, tb.loss);
  cgemm_ahx_kernel<<<(unsigned)((N + 31) / 32), 256, 0, st>>>(N, nv, ts->A32, tb.az, tb.z);  // z <- A^H e
  outgrad_kernel<<<G, 256, 0, st>>>(nv, N, tb.z, rsq, tb.go);
  s = net_backward_dev(net, nv, ts->nt, ts->mt, tb.f, tb.go, nullptr);
  if (s) return s;
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BIE_OK : cuda_fail(e, "loss gradient");
}

}  // namespace bie

// ------------------------------------------------------------------ inference on FP64 vectors
namespace bie {

// Per-surface normalised Jacobians and feature buffers, cached on the network object.
struct NetInfer {
  const void* key = nullptr;
  int64_t N = 0;
  float* jn = nullptr;
  float* feat = nullptr;
  double* sq = nullptr;
  double2* zb = nullptr;
  int cap = 0;
};

}  // namespace bie

struct bie_net_infer_s : bie::NetInfer {};

namespace bie {

static bie_status infer_prepare(bie_net net, NetInfer& I, bie_surface s, int nv) {
  const cudaStream_t st = net->ctx->stream;
  if (I.key != (const void*)s || I.N != s->N || I.cap < nv) {
    cudaFree(I.jn);
    cudaFree(I.feat);
    cudaFree(I.sq);
    cudaFree(I.zb);
    I = NetInfer();
    cudaError_t e = cudaMalloc((void**)&I.jn, sizeof(float) * s->N);
    if (e == cudaSuccess) e = cudaMalloc((void**)&I.feat, sizeof(float) * 4 * s->N * nv);
    if (e == cudaSuccess) e = cudaMalloc((void**)&I.sq, sizeof(double) * nv);
    if (e == cudaSuccess) e = cudaMalloc((void**)&I.zb, sizeof(double2) * s->N * nv);
    if (e != cudaSuccess) return cuda_fail(e, "network inference buffers");
    jn_kernel<<<1, 1024, 0, st>>>(s->N, s->jac, I.jn);
    I.key = s;
    I.N = s->N;
    I.cap = nv;
  }
  return BIE_OK;
}

// z = B^{-1} v + s net(features(v)) for nv FP64 vectors of the surface's grid (B optional).
bie_status net_precond_apply_dev(bie_net net, bie_net_infer_s* I, bie_blockdiag block, bie_surface s, double k,
                                 const double2* v, int nv, double2* z) {
  const cudaStream_t st = net->ctx->stream;
  bie_status r = infer_prepare(net, *I, s, nv);
  if (r) return r;
  const int64_t N = s->N;
  const int nt = 16 * s->Np, mt = s->Mt;
  const int G = net->ctx->sms * 4;
  if (block) {
    r = blockdiag_apply_dev(block, v, nv, I->zb);
    if (r) return r;
  } else {
    cudaMemsetAsync(I->zb, 0, sizeof(double2) * N * nv, st);
  }
  sumsq_kernel<double2><<<nv, 256, 0, st>>>(N, v, I->sq);
  features_kernel<double2><<<G, 256, 0, st>>>(nv, N, v, I->sq, I->jn, (float)(k / 25.0), I->feat);
  r = net_forward_dev(net, nv, nt, mt, I->feat);
  if (r) return r;
  combine_kernel<double2><<<G, 256, 0, st>>>(nv, N, I->zb, act_ptr(net, nv, nt, mt, 3), I->sq, z);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BIE_OK : cuda_fail(e, "network preconditioner");
}

bie_net_infer_s* net_infer_new() { return new bie_net_infer_s(); }
void net_infer_free(bie_net_infer_s* I) {
  if (!I) return;
  cudaFree(I->jn);
  cudaFree(I->feat);
  cudaFree(I->sq);
  cudaFree(I->zb);
  delete I;
}

static void init_params(uint64_t seed, std::vector<float>& w) {
  // He-uniform for the hidden layers, zero output layer (the preconditioner starts as B^{-1}),
  // zero biases; uniforms from splitmix64 of (seed, index).
  w.assign(kNetParams, 0.f);
  auto u01h = [&](uint64_t ctr) {
    uint64_t x = (seed * 0x100000001B3ull + ctr) + 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    x ^= x >> 31;
    return (double)(x >> 11) * (1.0 / 9007199254740992.0);
  };
  for (int l = 0; l < 3; ++l) {
    const Layer& L = kLayers[l];
    const double a = std::sqrt(6.0 / (L.cin * 9));
    for (int e = 0; e < L.cout * L.cin * 9; ++e) w[L.w + e] = (float)(a * (2.0 * u01h(L.w + e) - 1.0));
  }
}

}  // namespace bie

extern "C" {

bie_status bie_net_create(bie_ctx ctx, const float* params, uint64_t seed, bie_net* out) {
  if (!ctx || !out) { set_error("bie_net_create: invalid arguments"); return BIE_EINVAL; }
  *out = nullptr;
  bie_net net = new bie_net_s();
  net->ctx = ctx;
  cudaError_t e = cudaMalloc((void**)&net->w, sizeof(float) * kNetParams * 5);
  if (e != cudaSuccess) { delete net; return cuda_fail(e, "bie_net_create"); }
  net->wq = net->w + kNetParams;
  net->m = net->w + 2 * kNetParams;
  net->v = net->w + 3 * kNetParams;
  net->g = net->w + 4 * kNetParams;
  std::vector<float> h;
  if (params) h.assign(params, params + kNetParams);
  else init_params(seed, h);
  const cudaStream_t st = ctx->stream;
  e = cudaMemcpyAsync(net->w, h.data(), sizeof(float) * kNetParams, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(net->m, 0, sizeof(float) * 3 * kNetParams, st);
  if (e == cudaSuccess) {
    round_bf16_kernel<<<(kNetParams + 255) / 256, 256, 0, st>>>(kNetParams, net->w, net->wq);
    e = cudaStreamSynchronize(st);
  }
  if (e != cudaSuccess) { bie_net_free(net); return cuda_fail(e, "bie_net_create"); }
  *out = net;
  return BIE_OK;
}

bie_status bie_net_get_params(bie_net net, float* params) {
  if (!net || !params) { set_error("bie_net_get_params: invalid arguments"); return BIE_EINVAL; }
  cudaError_t e = cudaMemcpyAsync(params, net->w, sizeof(float) * kNetParams, cudaMemcpyDeviceToHost, net->ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(net->ctx->stream);
  return e == cudaSuccess ? BIE_OK : cuda_fail(e, "bie_net_get_params");
}

void bie_net_free(bie_net net) {
  if (!net) return;
  cudaFree(net->w);
  cudaFree(net->act);
  cudaFree(net->gbuf);
  cudaFree(net->partial);
  delete net;
}

bie_status bie_net_forward(bie_net net, int B, int nt, int mt, const float* x, float* y) {
  if (!net || !x || !y || B < 1 || nt < 1 || mt < 8) { set_error("bie_net_forward: invalid arguments"); return BIE_EINVAL; }
  bie_status s = net_forward_dev(net, B, nt, mt, x);
  if (s) return s;
  const cudaError_t e = cudaMemcpyAsync(y, act_ptr(net, B, nt, mt, 3), sizeof(float) * (size_t)B * kNetOut * nt * mt,
                                        cudaMemcpyDeviceToDevice, net->ctx->stream);
  return e == cudaSuccess ? BIE_OK : cuda_fail(e, "bie_net_forward");
}

bie_status bie_net_backward(bie_net net, int B, int nt, int mt, const float* x, const float* gy, float* gparams,
                            float* gx) {
  if (!net || !x || !gy || !gparams || B < 1 || nt < 1 || mt < 8) {
    set_error("bie_net_backward: invalid arguments");
    return BIE_EINVAL;
  }
  bie_status s = net_forward_dev(net, B, nt, mt, x);
  if (s) return s;
  s = net_backward_dev(net, B, nt, mt, x, gy, gx);
  if (s) return s;
  const cudaError_t e = cudaMemcpyAsync(gparams, net->g, sizeof(float) * kNetParams, cudaMemcpyDeviceToDevice,
                                        net->ctx->stream);
  return e == cudaSuccess ? BIE_OK : cuda_fail(e, "bie_net_backward");
}

bie_status bie_train_set_create(bie_ctx ctx, bie_surface s, double k, const double* A, bie_blockdiag block,
                                bie_train_set* out) {
  if (!ctx || !s || !A || !out || !(k > 0)) { set_error("bie_train_set_create: invalid arguments"); return BIE_EINVAL; }
  if (block && bie_blockdiag_size(block) != s->N) { set_error("bie_train_set_create: block size mismatch"); return BIE_EINVAL; }
  *out = nullptr;
  bie_train_set ts = new bie_train_set_s();
  ts->ctx = ctx;
  ts->N = s->N;
  ts->nt = 16 * s->Np;
  ts->mt = s->Mt;
  ts->k = k;
  ts->block = block;
  const cudaStream_t st = ctx->stream;
  cudaError_t e = cudaMalloc((void**)&ts->A32, sizeof(float2) * (size_t)s->N * s->N);
  if (e == cudaSuccess) e = cudaMalloc((void**)&ts->jn, sizeof(float) * s->N);
  if (e != cudaSuccess) { bie_train_set_free(ts); return cuda_fail(e, "bie_train_set_create"); }
  to_c64_kernel<<<ctx->sms * 8, 256, 0, st>>>((int64_t)s->N * s->N, (const double2*)A, ts->A32);
  jn_kernel<<<1, 1024, 0, st>>>(s->N, s->jac, ts->jn);
  e = cudaGetLastError();
  if (e != cudaSuccess) { bie_train_set_free(ts); return cuda_fail(e, "bie_train_set_create"); }
  *out = ts;
  return BIE_OK;
}

void bie_train_set_free(bie_train_set ts) {
  if (!ts) return;
  cudaFree(ts->A32);
  cudaFree(ts->jn);
  delete ts;
}

static bie_status alloc_train_bufs(bie_ctx ctx, int nv, int64_t N, TrainBufs& tb, std::vector<void*>& owned) {
  cudaError_t e = cudaSuccess;
  auto get = [&](void** p, size_t bytes) {
    *p = nullptr;
    if (e != cudaSuccess) return;
    e = cudaMallocAsync(p, bytes, ctx->stream);
    if (e == cudaSuccess) owned.push_back(*p);
  };
  get((void**)&tb.r, sizeof(float2) * nv * N);
  get((void**)&tb.zb, sizeof(float2) * nv * N);
  get((void**)&tb.z, sizeof(float2) * nv * N);
  get((void**)&tb.az, sizeof(float2) * nv * N);
  get((void**)&tb.f, sizeof(float) * 4 * nv * N);
  get((void**)&tb.go, sizeof(float) * 2 * nv * N);
  get((void**)&tb.loss, sizeof(float) * 1);
  get((void**)&tb.d, sizeof(double) * 2 * nv);
  return e == cudaSuccess ? BIE_OK : cuda_fail(e, "training buffers");
}

static void free_owned(bie_ctx ctx, std::vector<void*>& owned) {
  for (void* p : owned) cudaFreeAsync(p, ctx->stream);
  owned.clear();
}

bie_status bie_net_loss_grad(bie_net net, bie_train_set ts, const float* r, int nv, float* gparams, float* loss) {
  if (!net || !ts || !r || nv < 1 || nv > kMaxVec) { set_error("bie_net_loss_grad: invalid arguments (nv <= 16)"); return BIE_EINVAL; }
  const cudaStream_t st = net->ctx->stream;
  TrainBufs tb;
  std::vector<void*> owned;
  bie_status s = alloc_train_bufs(net->ctx, nv, ts->N, tb, owned);
  if (s == BIE_OK) {
    cudaMemcpyAsync(tb.r, r, sizeof(float2) * nv * ts->N, cudaMemcpyDeviceToDevice, st);
    s = loss_grad_dev(net, ts, nv, tb);
  }
  float lh = 0.f;
  if (s == BIE_OK && gparams)
    cudaMemcpyAsync(gparams, net->g, sizeof(float) * kNetParams, cudaMemcpyDeviceToDevice, st);
  if (s == BIE_OK) cudaMemcpyAsync(&lh, tb.loss, sizeof(float), cudaMemcpyDeviceToHost, st);
  free_owned(net->ctx, owned);
  const cudaError_t e = cudaStreamSynchronize(st);
  if (s == BIE_OK && e != cudaSuccess) s = cuda_fail(e, "bie_net_loss_grad");
  if (loss) *loss = lh;
  return s;
}

bie_status bie_net_train(bie_net net, const bie_train_set* sets, int n_sets, const bie_train_opts* o,
                         float* loss_history) {
  if (!net || !sets || n_sets < 1 || !o || o->steps < 1 || o->batch < 2 || o->batch > kMaxVec || !(o->lr > 0)) {
    set_error("bie_net_train: invalid arguments (2 <= batch <= 16)");
    return BIE_EINVAL;
  }
  int64_t Nmax = 0;
  for (int i = 0; i < n_sets; ++i) {
    if (!sets[i]) { set_error("bie_net_train: NULL training set"); return BIE_EINVAL; }
    Nmax = std::max(Nmax, sets[i]->N);
  }
  const cudaStream_t st = net->ctx->stream;
  const int nv = o->batch, half = nv / 2;
  TrainBufs tb;
  std::vector<void*> owned;
  float* hist = nullptr;
  bie_status s = alloc_train_bufs(net->ctx, nv, Nmax, tb, owned);
  if (s == BIE_OK) {
    const cudaError_t e = cudaMallocAsync((void**)&hist, sizeof(float) * o->steps, st);
    if (e != cudaSuccess) s = cuda_fail(e, "bie_net_train");
    else owned.push_back(hist);
  }
  const int G = net->ctx->sms * 4;
  for (int it = 0; it < o->steps && s == BIE_OK; ++it) {
    bie_train_set ts = sets[it % n_sets];
    const int64_t N = ts->N;
    const uint64_t key = (o->seed << 32) ^ (uint64_t)(2 * it);
    // residual batch: complex white noise, and A x for white x in the second half
    randn_kernel<<<G, 256, 0, st>>>((int64_t)nv * N, key, tb.r);
    randn_kernel<<<G, 256, 0, st>>>((int64_t)(nv - half) * N, key + 1, tb.z);
    cgemm_ax_kernel<<<(unsigned)((N + 15) / 16), 256, 0, st>>>(N, nv - half, ts->A32, tb.z, tb.r + (int64_t)half * N);
    s = loss_grad_dev(net, ts, nv, tb);
    if (s) break;
    net->step += 1;
    const float c1 = 1.f - std::pow(o->beta1, (float)net->step), c2 = 1.f - std::pow(o->beta2, (float)net->step);
    adam_kernel<<<(kNetParams + 255) / 256, 256, 0, st>>>(kNetParams, o->lr, o->beta1, o->beta2, o->eps, c1, c2,
                                                          net->g, net->m, net->v, net->w, net->wq);
    cudaMemcpyAsync(hist + it, tb.loss, sizeof(float), cudaMemcpyDeviceToDevice, st);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) s = cuda_fail(e, "bie_net_train");
  }
  if (s == BIE_OK && loss_history)
    cudaMemcpyAsync(loss_history, hist, sizeof(float) * o->steps, cudaMemcpyDeviceToHost, st);
  free_owned(net->ctx, owned);
  const cudaError_t e = cudaStreamSynchronize(st);
  if (s == BIE_OK && e != cudaSuccess) s = cuda_fail(e, "bie_net_train");
  return s;
}

bie_status bie_net_precond_apply(bie_net net, bie_blockdiag block, bie_surface s, double k, const double* v, int nv,
                                 double* z) {
  if (!net || !s || !v || !z || nv < 1 || nv > kMaxVec || !(k > 0)) {
    set_error("bie_net_precond_apply: invalid arguments");
    return BIE_EINVAL;
  }
  if (block && bie_blockdiag_size(block) != s->N) { set_error("bie_net_precond_apply: block size mismatch"); return BIE_EINVAL; }
  bie_net_infer_s* I = net_infer_new();
  bie_status r = net_precond_apply_dev(net, I, block, s, k, (const double2*)v, nv, (double2*)z);
  const cudaError_t e = cudaStreamSynchronize(net->ctx->stream);
  net_infer_free(I);
  if (r == BIE_OK && e != cudaSuccess) r = cuda_fail(e, "bie_net_precond_apply");
  return r;
}

}  // extern "C"
