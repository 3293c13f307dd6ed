// Dense complex solve for the Nystrom system (the paper states the system, Section 3.4; the
// solver is this library's): restarted FGMRES, right preconditioned, classical Gram-Schmidt with
// one re-orthogonalisation, run for all right-hand sides in lockstep so that every iteration
// makes one pass over the matrix for all of them (a block product A [z_1 .. z_nr]).
//
// Matrix products (bie_matrix_matvec's prec):
//   0  FP64: the FP64 pipe (8 flops per complex entry and right-hand side).
//   1  FP32 storage (8 B per entry), FP32 products summed in FP32 over chunks, chunks in FP64.
//   2  split-BF16 storage (8 B per entry) on the tensor cores, FP32 accumulation (tc_matvec.cu).
//   3  FP64 storage, products in double-word arithmetic (about 2^-44): the refinement residual
//      of the mixed solves, on the FP32 pipe at the speed of the matrix read.
// Solve precisions (bie_solve_opts.prec): 0 = FP64 products throughout; 1 and 2 = FGMRES with
// the FP32 or split-BF16 products inside, and FP64-accurate iterative refinement outside
// (r = b - A x with product 3, solve A dx = r approximately, x += dx).
// Host-driven: one small device-to-host copy of the Hessenberg columns per Gram-Schmidt pass.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <vector>

#include "bie_internal.cuh"
#include "dw.cuh"
#include "tc_matvec.cuh"

struct bie_matrix_s {
  bie_ctx ctx;
  int64_t n;
  const double2* A64;      // caller-owned FP64 matrix
  float2* A32 = nullptr;   // FP32 copy (store & BIE_STORE_FP32)
  bie::TcImage tc;         // split-BF16 image (store & BIE_STORE_BF16X2)
  double2* work = nullptr; // [16][n] staging for products with strided inputs
};

namespace bie {

constexpr int kMaxBlock = 16;   // right-hand sides per block product

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------------ block products
// Y[j] = A X[j], j < NR, one warp per row, lanes over columns (16-byte loads of the row, the
// right-hand sides through L1/L2).  FP64.
template <int NR>
__global__ void __launch_bounds__(256) zgemm64_block_kernel(int64_t n, int nr, const double2* __restrict__ A,
                                                            const double2* __restrict__ X, int64_t ldx,
                                                            double2* __restrict__ Y, int64_t ldy) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = w; row < n; row += nw) {
    const double2* a = A + row * n;
    double re[NR], im[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) re[j] = im[j] = 0.0;
    for (int64_t c = lane; c < n; c += 32) {
      const double2 av = __ldcs(a + c);
#pragma unroll
      for (int j = 0; j < NR; ++j) {
        if (j < nr) {
          const double2 xv = __ldg(X + j * ldx + c);
          re[j] = fma(av.x, xv.x, fma(-av.y, xv.y, re[j]));
          im[j] = fma(av.x, xv.y, fma(av.y, xv.x, im[j]));
        }
      }
    }
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      if (j < nr) {
        const double r = warp_sum_d(re[j]), i = warp_sum_d(im[j]);
        if (lane == 0) Y[j * ldy + row] = make_double2(r, i);
      }
    }
  }
}

// FP32 storage.  A CTA of 8 warps takes 8 rows (one per warp) and walks the columns in chunks of
// kCh32 whose right-hand-side values it stages in shared memory once for all 8 rows (the block of
// right-hand sides is otherwise re-read from L2 for every row: NR times the row's own bytes).  Each
// lane sums its products in FP32 over 64 columns (8 chunks) and accumulates those sums in FP64.  The
// right-hand sides are converted to FP32 by the caller.
constexpr int kCh32 = 256;
template <int NR>
__global__ void __launch_bounds__(256) cgemm32_block_kernel(int64_t n, int nr, const float2* __restrict__ A,
                                                            const float2* __restrict__ X, int64_t ldx,
                                                            double2* __restrict__ Y, int64_t ldy) {
  __shared__ float2 xs[NR][kCh32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t g = blockIdx.x; g * 8 < n; g += gridDim.x) {
    const int64_t row = g * 8 + wid;
    const bool live = row < n;
    const float2* a = A + (live ? row : 0) * n;
    double dre[NR], dim[NR];
    float cr[NR], ci[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) {
      dre[j] = dim[j] = 0.0;
      cr[j] = ci[j] = 0.f;
    }
    int pending = 0;
    // the row's values of a chunk are loaded one chunk ahead (they do not wait for the staging)
    constexpr int U = kCh32 / 32;
    float2 av[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t c = lane + 32 * u;
      av[u] = (live && c < n) ? __ldcs(a + c) : make_float2(0.f, 0.f);
    }
    for (int64_t c0 = 0; c0 < n; c0 += kCh32) {
      __syncthreads();   // every warp is done with the previous chunk
      for (int e = threadIdx.x; e < nr * kCh32; e += 256) {
        const int j = e / kCh32, cc = e % kCh32;
        const int64_t c = c0 + cc;
        xs[j][cc] = c < n ? __ldg(X + j * ldx + c) : make_float2(0.f, 0.f);
      }
      float2 an[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t c = c0 + kCh32 + lane + 32 * u;
        an[u] = (live && c < n) ? __ldcs(a + c) : make_float2(0.f, 0.f);
      }
      __syncthreads();
      if (live) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
          for (int j = 0; j < NR; ++j) {
            if (j < nr) {
              const float2 xv = xs[j][lane + 32 * u];
              cr[j] = fmaf(av[u].x, xv.x, fmaf(-av[u].y, xv.y, cr[j]));
              ci[j] = fmaf(av[u].x, xv.y, fmaf(av[u].y, xv.x, ci[j]));
            }
          }
        }
        if (++pending == 8 || c0 + kCh32 >= n) {
#pragma unroll
          for (int j = 0; j < NR; ++j) {
            if (j < nr) {
              dre[j] += cr[j];
              dim[j] += ci[j];
              cr[j] = ci[j] = 0.f;
            }
          }
          pending = 0;
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) av[u] = an[u];
    }
    if (live) {
#pragma unroll
      for (int j = 0; j < NR; ++j) {
        if (j < nr) {
          const double r = warp_sum_d(dre[j]), i = warp_sum_d(dim[j]);
          if (lane == 0) Y[j * ldy + row] = make_double2(r, i);
        }
      }
    }
  }
}

// FP64 storage, double-word products: each real product a x = (a_h + a_l)(x_h + x_l) is taken as
// the exact a_h x_h (TwoProd) plus a_h x_l + a_l x_h; the high parts are summed with TwoSum and
// the low parts in FP32.  Relative error about 2^-44 of the sum of |terms| (FP64-accurate for the
// refinement residual), on the FP32 pipe.
struct DwAcc {
  float h, l;
};
__device__ __forceinline__ void dw_madd(DwAcc& s, float ah, float al, float xh, float xl) {
  const float p = __fmul_rn(ah, xh);
  float e = fmaf(ah, xh, -p);
  e = fmaf(ah, xl, e);
  e = fmaf(al, xh, e);
  const float t = __fadd_rn(s.h, p);
  const float bb = __fsub_rn(t, s.h);
  const float err = __fadd_rn(__fsub_rn(s.h, __fsub_rn(t, bb)), __fsub_rn(p, bb));
  s.h = t;
  s.l = __fadd_rn(s.l, __fadd_rn(err, e));
}
__device__ __forceinline__ double dw_acc_warp_sum(DwAcc s) {
  // exact conversion of each part, the warp sum in FP64 (32 terms)
  return warp_sum_d(f2d_bits(s.h) + f2d_bits(s.l));
}

// A CTA of 8 warps takes 8 rows (one per warp) and walks the columns in chunks of kChDw whose
// right-hand-side double words it stages in shared memory once for all 8 rows; each row's next chunk
// is loaded before the staging barrier.
constexpr int kChDw = 128;
template <int NR>
__global__ void __launch_bounds__(256) zgemm_dw_block_kernel(int64_t n, int nr, const double2* __restrict__ A,
                                                             const float4* __restrict__ X, int64_t ldx,
                                                             double2* __restrict__ Y, int64_t ldy) {
  __shared__ float4 xs[NR][kChDw];
  constexpr int U = kChDw / 32;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int64_t g = blockIdx.x; g * 8 < n; g += gridDim.x) {
    const int64_t row = g * 8 + wid;
    const bool live = row < n;
    const double2* a = A + (live ? row : 0) * n;
    DwAcc re[NR], im[NR];
#pragma unroll
    for (int j = 0; j < NR; ++j) re[j] = im[j] = DwAcc{0.f, 0.f};
    double2 av[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t c = lane + 32 * u;
      av[u] = (live && c < n) ? __ldcs(a + c) : make_double2(0.0, 0.0);
    }
    for (int64_t c0 = 0; c0 < n; c0 += kChDw) {
      __syncthreads();   // every warp is done with the previous chunk
      for (int e = threadIdx.x; e < nr * kChDw; e += 256) {
        const int j = e / kChDw, cc = e % kChDw;
        const int64_t c = c0 + cc;
        xs[j][cc] = c < n ? __ldg(X + j * ldx + c) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
      double2 an[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int64_t c = c0 + kChDw + lane + 32 * u;
        an[u] = (live && c < n) ? __ldcs(a + c) : make_double2(0.0, 0.0);
      }
      __syncthreads();
      if (live) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const float2 ar = dw_from(av[u].x), ai = dw_from(av[u].y);
#pragma unroll
          for (int j = 0; j < NR; ++j) {
            if (j < nr) {
              const float4 xv = xs[j][lane + 32 * u];   // (re.h, re.l, im.h, im.l)
              dw_madd(re[j], ar.x, ar.y, xv.x, xv.y);
              dw_madd(re[j], -ai.x, -ai.y, xv.z, xv.w);
              dw_madd(im[j], ar.x, ar.y, xv.z, xv.w);
              dw_madd(im[j], ai.x, ai.y, xv.x, xv.y);
            }
          }
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) av[u] = an[u];
    }
    if (live) {
#pragma unroll
      for (int j = 0; j < NR; ++j) {
        if (j < nr) {
          const double r = dw_acc_warp_sum(re[j]), i = dw_acc_warp_sum(im[j]);
          if (lane == 0) Y[j * ldy + row] = make_double2(r, i);
        }
      }
    }
  }
}

__global__ void to_f32_kernel(int64_t n, const double2* __restrict__ a, float2* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = make_float2((float)a[i].x, (float)a[i].y);
}
__global__ void to_dw_kernel(int64_t n, const double2* __restrict__ a, float4* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = mkc(dw_from(a[i].x), dw_from(a[i].y));
}

// ------------------------------------------------------------------ block vector kernels
// vectors of right-hand side c and basis index i live at V + (i nr + c) n
// partial[(c J + i) nb + block] = sum over the block's share of conj(V_i^c) W^c
__global__ void block_dots_kernel(int64_t n, int J, int nr, const double2* __restrict__ V,
                                  const double2* __restrict__ W, double2* __restrict__ partial) {
  __shared__ double sre[8], sim[8];
  const int i = blockIdx.y, c = blockIdx.z;
  const double2* v = V + ((int64_t)i * nr + c) * n;
  const double2* w = W + (int64_t)c * n;
  double re = 0, im = 0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const double2 a = v[k], b = w[k];
    re = fma(a.x, b.x, fma(a.y, b.y, re));
    im = fma(a.x, b.y, fma(-a.y, b.x, im));
  }
  re = warp_sum_d(re);
  im = warp_sum_d(im);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sre[wid] = re; sim[wid] = im; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0, m = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { r += sre[q]; m += sim[q]; }
    partial[((int64_t)c * J + i) * gridDim.x + blockIdx.x] = make_double2(r, m);
  }
}
__global__ void reduce_partials_kernel(int nb, const double2* __restrict__ partial, double2* __restrict__ h) {
  const int j = blockIdx.x;   // c J + i
  double re = 0, im = 0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    re += partial[(int64_t)j * nb + b].x;
    im += partial[(int64_t)j * nb + b].y;
  }
  re = warp_sum_d(re);
  im = warp_sum_d(im);
  __shared__ double sre[8], sim[8];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sre[wid] = re; sim[wid] = im; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0, m = 0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) { r += sre[q]; m += sim[q]; }
    h[j] = make_double2(r, m);
  }
}
// W^c -= sum_{i<J} h[c J + i] V_i^c
__global__ void block_axpy_kernel(int64_t n, int J, int nr, const double2* __restrict__ V,
                                  const double2* __restrict__ h, double2* __restrict__ W) {
  const int c = blockIdx.y;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    double2 acc = W[(int64_t)c * n + k];
    for (int i = 0; i < J; ++i) {
      const double2 a = V[((int64_t)i * nr + c) * n + k], s = h[c * J + i];
      acc.x -= s.x * a.x - s.y * a.y;
      acc.y -= s.x * a.y + s.y * a.x;
    }
    W[(int64_t)c * n + k] = acc;
  }
}
// Y^c = s[c] X^c
__global__ void block_scale_kernel(int64_t n, const double* __restrict__ s, const double2* __restrict__ X,
                                   double2* __restrict__ Y) {
  const int c = blockIdx.y;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const double2 x = X[(int64_t)c * n + k];
    Y[(int64_t)c * n + k] = make_double2(s[c] * x.x, s[c] * x.y);
  }
}
// R^c = B^c - Y^c
__global__ void block_sub_kernel(int64_t n, const double2* __restrict__ B, const double2* __restrict__ Y,
                                 double2* __restrict__ R) {
  const int c = blockIdx.y;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const double2 b = B[(int64_t)c * n + k], y = Y[(int64_t)c * n + k];
    R[(int64_t)c * n + k] = make_double2(b.x - y.x, b.y - y.y);
  }
}
// X^c += sum_{i<J} y[c J + i] Z_i^c
__global__ void block_update_kernel(int64_t n, int J, int nr, const double2* __restrict__ Z,
                                    const double2* __restrict__ y, double2* __restrict__ X) {
  const int c = blockIdx.y;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    double2 acc = X[(int64_t)c * n + k];
    for (int i = 0; i < J; ++i) {
      const double2 z = Z[((int64_t)i * nr + c) * n + k], s = y[c * J + i];
      acc.x += s.x * z.x - s.y * z.y;
      acc.y += s.x * z.y + s.y * z.x;
    }
    X[(int64_t)c * n + k] = acc;
  }
}

// ------------------------------------------------------------------ matrix products (host)
static int pick_nr(int nr) { return nr <= 1 ? 1 : nr <= 2 ? 2 : nr <= 4 ? 4 : nr <= 8 ? 8 : 16; }

#define BIE_DISPATCH_NR(NRV, KERNEL, ...)                                   \
  switch (pick_nr(NRV)) {                                                   \
    case 1: KERNEL<1><<<grid, 256, 0, st>>>(__VA_ARGS__); break;            \
    case 2: KERNEL<2><<<grid, 256, 0, st>>>(__VA_ARGS__); break;            \
    case 4: KERNEL<4><<<grid, 256, 0, st>>>(__VA_ARGS__); break;            \
    case 8: KERNEL<8><<<grid, 256, 0, st>>>(__VA_ARGS__); break;            \
    default: KERNEL<16><<<grid, 256, 0, st>>>(__VA_ARGS__); break;          \
  }

// Y [nr][n] = A X [nr][n]; nr <= 16; scratch: FP32 or double-word copies of X (16 n float4)
bie_status matrix_product(bie_matrix M, int prec, const double2* X, int nr, double2* Y, float4* scratch) {
  const bie_ctx ctx = M->ctx;
  const cudaStream_t st = ctx->stream;
  const int64_t n = M->n;
  const int grid = ctx->sms * 8;
  if (nr < 1 || nr > kMaxBlock) { set_error("matrix product: 1 <= nr <= %d", kMaxBlock); return BIE_EINVAL; }
  switch (prec) {
    case 0:
      BIE_DISPATCH_NR(nr, zgemm64_block_kernel, n, nr, M->A64, X, n, Y, n);
      break;
    case 1: {
      if (!M->A32) { set_error("matrix product: no FP32 copy (BIE_STORE_FP32)"); return BIE_EINVAL; }
      float2* x32 = reinterpret_cast<float2*>(scratch);
      to_f32_kernel<<<ctx->sms * 4, 256, 0, st>>>(n * nr, X, x32);
      BIE_DISPATCH_NR(nr, cgemm32_block_kernel, n, nr, M->A32, x32, n, Y, n);
      break;
    }
    case 2:
      if (!M->tc.a_img) { set_error("matrix product: no split-BF16 copy (BIE_STORE_BF16X2)"); return BIE_EINVAL; }
      return tc_matvec(ctx, M->tc, X, n, nr, Y, n);
    case 3:
      to_dw_kernel<<<ctx->sms * 4, 256, 0, st>>>(n * nr, X, scratch);
      BIE_DISPATCH_NR(nr, zgemm_dw_block_kernel, n, nr, M->A64, scratch, n, Y, n);
      break;
    default:
      set_error("matrix product: prec %d not in 0..3", prec);
      return BIE_EINVAL;
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BIE_OK : cuda_fail(e, "matrix product");
}

// ------------------------------------------------------------------ lockstep FGMRES
struct BlockSolver {
  bie_ctx ctx;
  bie_matrix M;
  int64_t n;
  int m;                 // restart length
  int nr;                // right-hand sides in the block
  double2 *V = nullptr, *Z = nullptr, *W = nullptr, *R = nullptr, *T = nullptr;
  double2 *hdev = nullptr, *partial = nullptr;
  double* sdev = nullptr;
  float4* xs = nullptr;  // FP32 / double-word copies of a block of vectors
  int dot_blocks = 0;
  int matvecs = 0;
  // right preconditioner
  int pkind = 0;
  bie_blockdiag block = nullptr;
  bie_net net = nullptr;
  bie_surface surface = nullptr;
  double k = 0.0;
  bie_net_infer_s* infer = nullptr;

  bie_status product(int prec, const double2* X, double2* Y) {
    ++matvecs;
    return matrix_product(M, prec, X, nr, Y, xs);
  }
  bie_status precond(const double2* Vb, double2* Zb, const std::vector<char>& live) {
    bie_status s = BIE_OK;
    if (pkind == 1) s = blockdiag_apply_dev(block, Vb, nr, Zb);
    else if (pkind == 2) s = net_precond_apply_dev(net, infer, block, surface, k, Vb, nr, Zb);
    else {
      const cudaError_t e = cudaMemcpyAsync(Zb, Vb, sizeof(double2) * n * nr, cudaMemcpyDeviceToDevice, ctx->stream);
      if (e != cudaSuccess) return cuda_fail(e, "precond copy");
    }
    if (s) return s;
    for (int c = 0; c < nr; ++c)   // columns that are done carry zeros (a network maps 0 to NaN)
      if (!live[c]) cudaMemsetAsync(Zb + (int64_t)c * n, 0, sizeof(double2) * n, ctx->stream);
    return BIE_OK;
  }
  // hh[c J + i] = V_i^c^H W^c, i < J (copied to the host)
  bie_status dots(int J, const double2* Vb, const double2* Wb, std::complex<double>* hh) {
    const cudaStream_t st = ctx->stream;
    dim3 g(dot_blocks, J, nr);
    block_dots_kernel<<<g, 256, 0, st>>>(n, J, nr, Vb, Wb, partial);
    reduce_partials_kernel<<<J * nr, 256, 0, st>>>(dot_blocks, partial, hdev);
    cudaError_t e = cudaMemcpyAsync(hh, hdev, sizeof(double2) * J * nr, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? BIE_OK : cuda_fail(e, "dots");
  }
  bie_status norms(const double2* Xb, double* out) {
    std::vector<std::complex<double>> h(nr);
    // the diagonal dots <X^c, X^c>: V = X with J = 1
    const bie_status s = dots(1, Xb, Xb, h.data());
    for (int c = 0; c < nr; ++c) out[c] = std::sqrt(std::max(h[c].real(), 0.0));
    return s;
  }
  bie_status scale(const double* s, const double2* X, double2* Y) {
    cudaError_t e = cudaMemcpyAsync(sdev, s, sizeof(double) * nr, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(e, "scale");
    block_scale_kernel<<<dim3(ctx->sms * 2, nr), 256, 0, ctx->stream>>>(n, sdev, X, Y);
    return BIE_OK;
  }

  // FGMRES for all columns of B (x in/out), relative tolerances tol[c]; *iters = block iterations,
  // relres[c] = final true residual (computed with product prec) / ||b^c||.
  bie_status fgmres(const double2* B, double2* X, const double* tol, int maxit, int prec, int* iters,
                    double* relres) {
    const cudaStream_t st = ctx->stream;
    std::vector<double> bnorm(nr), beta(nr), res(nr), hn(nr), sc(nr);
    bie_status s = norms(B, bnorm.data());
    if (s) return s;
    std::vector<char> live(nr), cyc(nr);
    for (int c = 0; c < nr; ++c)
      if (bnorm[c] == 0.0) cudaMemsetAsync(X + (int64_t)c * n, 0, sizeof(double2) * n, st);
    for (int c = 0; c < nr; ++c)
      if (!(bnorm[c] == bnorm[c])) return BIE_ENAN;
    const size_t HM = (size_t)(m + 1) * m;
    std::vector<std::complex<double>> H(HM * nr), cs((size_t)m * nr), sn((size_t)m * nr), g((size_t)(m + 1) * nr),
        hh((size_t)(m + 1) * nr), hsum((size_t)(m + 1) * nr), y((size_t)m * nr);
    std::vector<int> jdone(nr);
    int total = 0;
    *iters = 0;
    while (true) {
      s = product(prec, X, T);
      if (s) return s;
      block_sub_kernel<<<dim3(ctx->sms * 2, nr), 256, 0, st>>>(n, B, T, R);
      s = norms(R, beta.data());
      if (s) return s;
      bool any = false;
      for (int c = 0; c < nr; ++c) {
        res[c] = bnorm[c] > 0 ? beta[c] / bnorm[c] : 0.0;
        if (!(res[c] == res[c])) return BIE_ENAN;
        live[c] = res[c] > tol[c];
        any = any || live[c];
      }
      if (!any || total >= maxit) break;
      for (int c = 0; c < nr; ++c) sc[c] = live[c] ? 1.0 / beta[c] : 0.0;
      s = scale(sc.data(), R, V);
      if (s) return s;
      std::fill(g.begin(), g.end(), 0.0);
      for (int c = 0; c < nr; ++c) {
        g[(size_t)c * (m + 1)] = live[c] ? beta[c] : 0.0;
        cyc[c] = live[c];
        jdone[c] = 0;
      }
      for (int j = 0; j < m && total < maxit; ++j) {
        double2* Vj = V + (int64_t)j * nr * n;
        double2* Zj = Z + (int64_t)j * nr * n;
        s = precond(Vj, Zj, cyc);
        if (s) return s;
        s = product(prec, Zj, W);
        if (s) return s;
        // classical Gram-Schmidt, twice, for every column at once
        std::fill(hsum.begin(), hsum.end(), 0.0);
        for (int pass = 0; pass < 2; ++pass) {
          s = dots(j + 1, V, W, hh.data());
          if (s) return s;
          for (int c = 0; c < nr; ++c)
            if (!cyc[c])
              for (int i = 0; i <= j; ++i) hh[(size_t)c * (j + 1) + i] = 0.0;
          cudaMemcpyAsync(hdev, hh.data(), sizeof(double2) * (j + 1) * nr, cudaMemcpyHostToDevice, st);
          block_axpy_kernel<<<dim3(ctx->sms * 2, nr), 256, 0, st>>>(n, j + 1, nr, V, hdev, W);
          for (size_t q = 0; q < (size_t)(j + 1) * nr; ++q) hsum[q] += hh[q];
        }
        s = norms(W, hn.data());
        if (s) return s;
        for (int c = 0; c < nr; ++c) sc[c] = (cyc[c] && hn[c] > 0) ? 1.0 / hn[c] : 0.0;
        s = scale(sc.data(), W, V + (int64_t)(j + 1) * nr * n);
        if (s) return s;
        bool still = false;
        for (int c = 0; c < nr; ++c) {
          if (!cyc[c]) continue;
          std::complex<double>* Hc = H.data() + (size_t)c * HM;
          std::complex<double>* csc = cs.data() + (size_t)c * m;
          std::complex<double>* snc = sn.data() + (size_t)c * m;
          std::complex<double>* gc = g.data() + (size_t)c * (m + 1);
          for (int i = 0; i <= j; ++i) Hc[(size_t)i * m + j] = hsum[(size_t)c * (j + 1) + i];
          Hc[(size_t)(j + 1) * m + j] = hn[c];
          for (int i = 0; i < j; ++i) {   // Givens rotations
            const std::complex<double> a = Hc[(size_t)i * m + j], bb = Hc[(size_t)(i + 1) * m + j];
            Hc[(size_t)i * m + j] = std::conj(csc[i]) * a + std::conj(snc[i]) * bb;
            Hc[(size_t)(i + 1) * m + j] = -snc[i] * a + csc[i] * bb;
          }
          const std::complex<double> a = Hc[(size_t)j * m + j], bb = Hc[(size_t)(j + 1) * m + j];
          const double den = std::sqrt(std::norm(a) + std::norm(bb));
          csc[j] = den > 0 ? a / den : 1.0;
          snc[j] = den > 0 ? bb / den : 0.0;
          Hc[(size_t)j * m + j] = den;
          Hc[(size_t)(j + 1) * m + j] = 0.0;
          gc[j + 1] = -snc[j] * gc[j];
          gc[j] = std::conj(csc[j]) * gc[j];
          jdone[c] = j + 1;
          const double est = std::abs(gc[j + 1]) / bnorm[c];
          if (!(est == est)) return BIE_ENAN;
          if (est <= tol[c] * 0.5 || hn[c] == 0) cyc[c] = 0;
          still = still || cyc[c];
        }
        ++total;
        if (!still) break;
      }
      // back substitution and x^c += Z y^c
      int Jmax = 0;
      std::fill(y.begin(), y.end(), 0.0);
      for (int c = 0; c < nr; ++c) {
        const int J = jdone[c];
        Jmax = std::max(Jmax, J);
        const std::complex<double>* Hc = H.data() + (size_t)c * HM;
        const std::complex<double>* gc = g.data() + (size_t)c * (m + 1);
        for (int i = J - 1; i >= 0; --i) {
          std::complex<double> acc = gc[i];
          for (int k2 = i + 1; k2 < J; ++k2) acc -= Hc[(size_t)i * m + k2] * y[(size_t)c * m + k2];
          y[(size_t)c * m + i] = acc / Hc[(size_t)i * m + i];
        }
      }
      if (Jmax > 0) {
        std::vector<std::complex<double>> yy((size_t)Jmax * nr, 0.0);
        for (int c = 0; c < nr; ++c)
          for (int i = 0; i < jdone[c]; ++i) yy[(size_t)c * Jmax + i] = y[(size_t)c * m + i];
        cudaMemcpyAsync(hdev, yy.data(), sizeof(double2) * Jmax * nr, cudaMemcpyHostToDevice, st);
        block_update_kernel<<<dim3(ctx->sms * 2, nr), 256, 0, st>>>(n, Jmax, nr, Z, hdev, X);
        // the host vector yy must outlive the copy
        const cudaError_t e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "fgmres update");
      }
    }
    *iters = total;
    for (int c = 0; c < nr; ++c) relres[c] = res[c];
    return BIE_OK;
  }
};

bie_status matrix_create(bie_ctx ctx, int64_t n, const double* A, unsigned store, bie_matrix* out) {
  bie_matrix M = new bie_matrix_s();
  M->ctx = ctx;
  M->n = n;
  M->A64 = (const double2*)A;
  const cudaStream_t st = ctx->stream;
  cudaError_t e = cudaSuccess;
  bie_status s = BIE_OK;
  if (store & BIE_STORE_FP32) {
    e = cudaMallocAsync((void**)&M->A32, sizeof(float2) * n * n, st);
    if (e == cudaSuccess) {
      to_f32_kernel<<<ctx->sms * 8, 256, 0, st>>>(n * n, (const double2*)A, M->A32);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) s = cuda_fail(e, "bie_matrix_create (FP32 copy)");
  }
  if (s == BIE_OK && (store & BIE_STORE_BF16X2)) s = tc_image_create(ctx, n, A, &M->tc);
  if (s != BIE_OK) {
    if (M->A32) cudaFreeAsync(M->A32, st);
    delete M;
    return s;
  }
  *out = M;
  return BIE_OK;
}

}  // namespace bie

using namespace bie;

extern "C" {

bie_status bie_matrix_create(bie_ctx ctx, int64_t n, const double* A, unsigned store, bie_matrix* out) {
  if (!ctx || !A || !out || n <= 0 || (store & ~(BIE_STORE_FP32 | BIE_STORE_BF16X2))) {
    set_error("bie_matrix_create: invalid arguments");
    return BIE_EINVAL;
  }
  const bie_status ds = check_device(ctx, "bie_matrix_create");
  if (ds != BIE_OK) return ds;
  return matrix_create(ctx, n, A, store, out);
}

void bie_matrix_free(bie_matrix M) {
  if (!M) return;
  const cudaStream_t st = M->ctx->stream;
  if (M->A32) cudaFreeAsync(M->A32, st);
  tc_image_free(M->ctx, &M->tc);
  if (M->work) cudaFreeAsync(M->work, st);
  cudaStreamSynchronize(st);
  delete M;
}

int64_t bie_matrix_size(bie_matrix M) { return M ? M->n : 0; }

bie_status bie_matrix_matvec(bie_matrix M, int prec, const double* x, int nr, double* y) {
  if (!M || !x || !y || nr < 1 || nr > kMaxBlock || prec < 0 || prec > 3) {
    set_error("bie_matrix_matvec: invalid arguments");
    return BIE_EINVAL;
  }
  const bie_status ds = check_device(M->ctx, "bie_matrix_matvec");
  if (ds != BIE_OK) return ds;
  float4* xs = nullptr;
  const cudaStream_t st = M->ctx->stream;
  cudaError_t e = cudaMallocAsync((void**)&xs, sizeof(float4) * M->n * nr, st);
  if (e != cudaSuccess) return cuda_fail(e, "bie_matrix_matvec scratch");
  const bie_status s = matrix_product(M, prec, (const double2*)x, nr, (double2*)y, xs);
  cudaFreeAsync(xs, st);
  return s;
}

bie_status bie_solve_matrix(bie_ctx ctx, bie_matrix Mx, const double* rhs, int nrhs, double* x,
                            const bie_solve_opts* opts, bie_solve_report* report) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!ctx || !Mx || !rhs || !x || nrhs <= 0 || !opts) { set_error("bie_solve_matrix: invalid arguments"); return BIE_EINVAL; }
  const int64_t n = Mx->n;
  if (!(opts->tol > 0) || opts->restart < 1 || opts->restart > 1000 || opts->maxit < 1 || opts->prec < 0 ||
      opts->prec > 2 || opts->precond < 0 || opts->precond > 2) {
    set_error("bie_solve_matrix: invalid options");
    return BIE_EINVAL;
  }
  if (opts->prec == 1 && !Mx->A32) { set_error("bie_solve_matrix: prec = 1 needs the FP32 copy (BIE_STORE_FP32)"); return BIE_EINVAL; }
  if (opts->prec == 2 && !Mx->tc.a_img) {
    set_error("bie_solve_matrix: prec = 2 needs the split-BF16 copy (BIE_STORE_BF16X2)");
    return BIE_EINVAL;
  }
  if (opts->precond == 1 && (!opts->block || bie_blockdiag_size(opts->block) != n)) {
    set_error("bie_solve_matrix: precond = 1 needs a block preconditioner of size n");
    return BIE_EINVAL;
  }
  if (opts->precond == 2 && (!opts->net || !opts->surface || opts->surface->N != n || !(opts->k > 0) ||
                             (opts->block && bie_blockdiag_size(opts->block) != n))) {
    set_error("bie_solve_matrix: precond = 2 needs a network, the surface of the unknowns and k > 0");
    return BIE_EINVAL;
  }
  {
    const bie_status ds = check_device(ctx, "bie_solve_matrix");
    if (ds != BIE_OK) return ds;
  }
  const cudaStream_t st = ctx->stream;
  std::vector<void*> owned;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** p, size_t bytes) {
    *p = nullptr;
    if (e != cudaSuccess) return;
    e = cudaMallocAsync(p, bytes, st);
    if (e == cudaSuccess) owned.push_back(*p);
  };
  const int nb_max = std::min(nrhs, kMaxBlock);
  BlockSolver S;
  S.ctx = ctx;
  S.M = Mx;
  S.n = n;
  S.m = opts->restart;
  S.pkind = opts->precond;
  S.block = opts->block;
  S.net = opts->net;
  S.surface = opts->surface;
  S.k = opts->k;
  S.dot_blocks = ctx->sms;
  if (S.pkind == 2) S.infer = net_infer_new();
  double2 *dX = nullptr, *Rr = nullptr, *X0 = nullptr;
  alloc((void**)&S.V, sizeof(double2) * n * nb_max * (S.m + 1));
  alloc((void**)&S.Z, sizeof(double2) * n * nb_max * S.m);
  alloc((void**)&S.W, sizeof(double2) * n * nb_max);
  alloc((void**)&S.R, sizeof(double2) * n * nb_max);
  alloc((void**)&S.T, sizeof(double2) * n * nb_max);
  alloc((void**)&S.xs, sizeof(float4) * n * nb_max);
  alloc((void**)&S.hdev, sizeof(double2) * (S.m + 2) * nb_max);
  alloc((void**)&S.sdev, sizeof(double) * nb_max);
  alloc((void**)&S.partial, sizeof(double2) * (S.m + 1) * nb_max * S.dot_blocks);
  if (opts->prec > 0) {
    alloc((void**)&dX, sizeof(double2) * n * nb_max);
    alloc((void**)&Rr, sizeof(double2) * n * nb_max);
  }
  if (S.pkind == 2 && opts->block) alloc((void**)&X0, sizeof(double2) * n * nb_max);
  bie_status status = e == cudaSuccess ? BIE_OK : cuda_fail(e, "bie_solve allocation");
  int total_iters = 0, refinements = 0, fallback = 0;
  double worst = 0.0;
  const int low = opts->prec;   // product precision inside FGMRES for prec 1, 2
  for (int c0 = 0; c0 < nrhs && status == BIE_OK; c0 += nb_max) {
    const int nr = std::min(nb_max, nrhs - c0);
    S.nr = nr;
    const double2* B = (const double2*)rhs + (int64_t)c0 * n;
    double2* Xc = (double2*)x + (int64_t)c0 * n;
    if (X0) cudaMemcpyAsync(X0, Xc, sizeof(double2) * n * nr, cudaMemcpyDeviceToDevice, st);
    int budget0 = total_iters;
    std::vector<double> rr(nr, 0.0), tolv(nr, opts->tol);
  retry:
    if (opts->prec == 0) {
      int it = 0;
      status = S.fgmres(B, Xc, tolv.data(), opts->maxit - (total_iters - budget0), 0, &it, rr.data());
      total_iters += it;
    } else {
      std::vector<double> bnorm(nr), rn(nr), itol(nr);
      status = S.norms(B, bnorm.data());
      for (int outer = 0; outer < 40 && status == BIE_OK; ++outer) {
        // FP64-accurate residual with the double-word product
        status = S.product(3, Xc, S.T);
        if (status) break;
        block_sub_kernel<<<dim3(ctx->sms * 2, nr), 256, 0, st>>>(n, B, S.T, Rr);
        status = S.norms(Rr, rn.data());
        if (status) break;
        bool done = true;
        for (int c = 0; c < nr; ++c) {
          rr[c] = bnorm[c] > 0 ? rn[c] / bnorm[c] : (bnorm[c] == 0.0 ? 0.0 : NAN);
          if (!(rr[c] == rr[c])) status = BIE_ENAN;
          done = done && rr[c] <= opts->tol;
        }
        if (status || done || total_iters - budget0 >= opts->maxit) break;
        for (int c = 0; c < nr; ++c) {
          // converged columns get a zero right-hand side (inactive inside); the others need what the
          // outer step asks, but not below the floor of the low-precision products (the FP32 sums
          // and the split-BF16 operator carry about 1e-7 and 1e-5 relative error)
          if (rr[c] <= opts->tol) {
            cudaMemsetAsync(Rr + (int64_t)c * n, 0, sizeof(double2) * n, st);
            itol[c] = 1.0;
          } else {
            itol[c] = std::max(low == 2 ? 1e-4 : 1e-5, 0.5 * opts->tol / rr[c]);
          }
        }
        cudaMemsetAsync(dX, 0, sizeof(double2) * n * nr, st);
        int it = 0;
        std::vector<double> inner(nr);
        status = S.fgmres(Rr, dX, itol.data(), opts->maxit - (total_iters - budget0), low, &it, inner.data());
        total_iters += it;
        ++refinements;
        if (status) break;
        {
          // x^c += dx^c as an update with one basis vector of coefficient 1
          std::vector<std::complex<double>> ones(nr, 1.0);
          cudaMemcpyAsync(S.hdev, ones.data(), sizeof(double2) * nr, cudaMemcpyHostToDevice, st);
          block_update_kernel<<<dim3(ctx->sms * 2, nr), 256, 0, st>>>(n, 1, nr, dX, S.hdev, Xc);
          const cudaError_t e2 = cudaStreamSynchronize(st);
          if (e2 != cudaSuccess) { status = cuda_fail(e2, "refinement update"); break; }
        }
      }
    }
    double wr = 0.0;
    for (int c = 0; c < nr; ++c) wr = std::max(wr, rr[c]);
    if (status == BIE_OK && !(wr <= opts->tol)) status = BIE_ENOCONV;
    // the learned preconditioner gave no convergence (or a NaN): the block-diagonal one takes over
    if ((status == BIE_ENOCONV || status == BIE_ENAN) && S.pkind == 2 && X0) {
      S.pkind = 1;
      fallback = 1;
      budget0 = total_iters;   // the fallback solve gets a fresh iteration budget
      status = BIE_OK;
      cudaMemcpyAsync(Xc, X0, sizeof(double2) * n * nr, cudaMemcpyDeviceToDevice, st);
      goto retry;
    }
    worst = std::max(worst, wr);
  }
  for (void* p : owned) cudaFreeAsync(p, st);
  cudaError_t e2 = cudaStreamSynchronize(st);
  if (status == BIE_OK && e2 != cudaSuccess) status = cuda_fail(e2, "bie_solve");
  if (status == BIE_OK) {
    int flags[4] = {0, 0, 0, 0};
    if (cudaMemcpy(flags, ctx->d_status, sizeof(flags), cudaMemcpyDeviceToHost) == cudaSuccess && flags[1]) {
      cudaMemsetAsync(ctx->d_status + 1, 0, sizeof(int), st);
      set_error("bie_solve_matrix: a bounded wait in the tensor-core product expired");
      status = BIE_ETIMEOUT;
    }
  }
  if (report) {
    report->iterations = total_iters;
    report->refinements = refinements;
    report->rel_residual = worst;
    report->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    report->fallback_used = fallback;
    report->matvecs = S.matvecs;
  }
  net_infer_free(S.infer);
  if (status == BIE_ENOCONV) set_error("bie_solve_matrix: tolerance not reached within maxit");
  if (status == BIE_ENAN) set_error("bie_solve_matrix: NaN in the residual");
  return status;
}

bie_status bie_solve(bie_ctx ctx, int64_t n, const double* A, const double* rhs, int nrhs, double* x,
                     const bie_solve_opts* opts, bie_solve_report* report) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!ctx || !A || !rhs || !x || n <= 0 || nrhs <= 0 || !opts) { set_error("bie_solve: invalid arguments"); return BIE_EINVAL; }
  if (opts->prec < 0 || opts->prec > 2) { set_error("bie_solve: invalid options"); return BIE_EINVAL; }
  const bie_status ds = check_device(ctx, "bie_solve");
  if (ds != BIE_OK) return ds;
  bie_matrix M = nullptr;
  const unsigned store = opts->prec == 1 ? BIE_STORE_FP32 : opts->prec == 2 ? BIE_STORE_BF16X2 : 0u;
  bie_status s = matrix_create(ctx, n, A, store, &M);
  if (s != BIE_OK) return s;
  s = bie_solve_matrix(ctx, M, rhs, nrhs, x, opts, report);
  bie_matrix_free(M);
  if (report) report->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return s;
}

}  // extern "C"
