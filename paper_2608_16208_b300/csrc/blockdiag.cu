// Block-diagonal preconditioner for FGMRES: LU factors, with partial pivoting, of the diagonal
// blocks of the Nystrom matrix (one block per panel: 16 Gauss-Legendre rings x M_theta samples,
// which holds every self-panel GGQ correction of Section 3.4).  The factors are FP32 complex: a
// preconditioner only has to be an approximate inverse, and FGMRES keeps the outer residual in FP64.
//
// Factorisation: right-looking blocked LU, panel width 32, all blocks of the matrix at once.
//   panel_kernel   one CTA per block; one warp per row, lane c <-> panel column c (coalesced rows);
//                  pivot search, row interchange, scaling and the rank-1 update of the panel, with
//                  the next column's pivot search fused into the update pass
//   swap_kernel    the panel's row interchanges on every column outside the panel
//   trsm_kernel    U12 = L11^{-1} A12 (unit lower, one thread per column)
//   gemm_kernel    A22 -= L21 U12, 64 x 64 complex tiles staged in shared memory
// Apply: z = U^{-1} L^{-1} P r per block and vector, one CTA each; the vector lives in shared memory
// and the triangular solves go by 32-row tiles (a warp-per-row product with the solved part, then a
// one-warp solve of the 32 x 32 diagonal tile).
#include <algorithm>
#include <vector>

#include "bie_internal.cuh"

namespace bie {

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 csubmulf(float2 acc, float2 a, float2 b) {  // acc - a b
  return make_float2(acc.x - fmaf(a.x, b.x, -a.y * b.y), acc.y - fmaf(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ float2 crecipf(float2 a) {
  const float d = a.x * a.x + a.y * a.y;
  return d > 0.f ? make_float2(a.x / d, -a.y / d) : make_float2(0.f, 0.f);
}
__device__ __forceinline__ float2 shflf(float2 v, int src) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

constexpr int kPanel = 32;

__global__ void bd_extract_kernel(int64_t n, int bs, int nb, const double2* __restrict__ A, float2* __restrict__ lu) {
  const int64_t total = (int64_t)nb * bs * bs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e / ((int64_t)bs * bs);
    const int64_t rem = e - b * bs * bs;
    const int64_t i = rem / bs, j = rem - (rem / bs) * bs;
    const double2 v = A[(b * bs + i) * n + b * bs + j];
    lu[e] = make_float2((float)v.x, (float)v.y);
  }
}

// Reduce (magnitude, row) over the CTA: larger magnitude wins, ties go to the smaller row.
__device__ __forceinline__ void argmax_merge(float& m, int& r, float m2, int r2) {
  if (m2 > m || (m2 == m && r2 < r)) { m = m2; r = r2; }
}

__global__ void __launch_bounds__(1024) bd_panel_kernel(int bs, int k, float2* __restrict__ lu, int* __restrict__ piv,
                                                        int* __restrict__ singular) {
  const int b = blockIdx.x;
  float2* a = lu + (int64_t)b * bs * bs;
  const int pw = min(kPanel, bs - k);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  __shared__ float s_mag[32];
  __shared__ int s_row[32];
  __shared__ float2 s_prow[kPanel];
  // pivot search for the first panel column
  float bm = -1.f;
  int br = bs;
  for (int i = k + threadIdx.x; i < bs; i += blockDim.x) {
    const float2 v = a[(int64_t)i * bs + k];
    argmax_merge(bm, br, v.x * v.x + v.y * v.y, i);
  }
  for (int j = k; j < k + pw; ++j) {
    const int cj = j - k;
    // CTA-wide argmax of the candidates (bm, br) of column j
    for (int o = 16; o > 0; o >>= 1) {
      const float m2 = __shfl_xor_sync(0xffffffffu, bm, o);
      const int r2 = __shfl_xor_sync(0xffffffffu, br, o);
      argmax_merge(bm, br, m2, r2);
    }
    if (lane == 0) { s_mag[warp] = bm; s_row[warp] = br; }
    __syncthreads();
    if (warp == 0) {
      float m = lane < nwarps ? s_mag[lane] : -1.f;
      int r = lane < nwarps ? s_row[lane] : bs;
      for (int o = 16; o > 0; o >>= 1) {
        const float m2 = __shfl_xor_sync(0xffffffffu, m, o);
        const int r2 = __shfl_xor_sync(0xffffffffu, r, o);
        argmax_merge(m, r, m2, r2);
      }
      if (r >= bs) r = j;
      if (lane == 0) {
        piv[(int64_t)b * bs + j] = r;
        if (!(m > 0.f) && singular[b] == 0) singular[b] = j + 1;
      }
      // interchange rows j and p inside the panel and publish the pivot row
      const int p = r;
      if (lane < pw) {
        const float2 vj = a[(int64_t)j * bs + k + lane];
        const float2 vp = a[(int64_t)p * bs + k + lane];
        if (p != j) {
          a[(int64_t)j * bs + k + lane] = vp;
          a[(int64_t)p * bs + k + lane] = vj;
        }
        s_prow[lane] = (p != j) ? vp : vj;
      }
    }
    __syncthreads();
    const float2 inv = crecipf(s_prow[cj]);
    const float2 pr = lane < pw ? s_prow[lane] : make_float2(0.f, 0.f);
    // scale column j and update the panel columns right of it; candidates for column j + 1
    bm = -1.f;
    br = bs;
    for (int i = j + 1 + warp; i < bs; i += nwarps) {
      float2 v = lane < pw ? a[(int64_t)i * bs + k + lane] : make_float2(0.f, 0.f);
      const float2 l = cmulf(shflf(v, cj), inv);
      if (lane == cj) v = l;
      else if (lane > cj) v = csubmulf(v, l, pr);
      if (lane >= cj && lane < pw) a[(int64_t)i * bs + k + lane] = v;
      if (lane == cj + 1) argmax_merge(bm, br, v.x * v.x + v.y * v.y, i);
    }
    // the candidate sits on lane cj + 1: broadcast it to the warp for the reduction
    if (cj + 1 < 32) {
      bm = __shfl_sync(0xffffffffu, bm, cj + 1);
      br = __shfl_sync(0xffffffffu, br, cj + 1);
    }
    __syncthreads();
  }
}

__global__ void bd_swap_kernel(int bs, int k, float2* __restrict__ lu, const int* __restrict__ piv) {
  const int b = blockIdx.y;
  float2* a = lu + (int64_t)b * bs * bs;
  const int pw = min(kPanel, bs - k);
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= bs || (c >= k && c < k + pw)) return;
  for (int j = k; j < k + pw; ++j) {
    const int p = piv[(int64_t)b * bs + j];
    if (p != j) {
      const float2 t = a[(int64_t)j * bs + c];
      a[(int64_t)j * bs + c] = a[(int64_t)p * bs + c];
      a[(int64_t)p * bs + c] = t;
    }
  }
}

__global__ void __launch_bounds__(128) bd_trsm_kernel(int bs, int k, float2* __restrict__ lu) {
  const int b = blockIdx.y;
  float2* a = lu + (int64_t)b * bs * bs;
  const int pw = min(kPanel, bs - k);
  __shared__ float2 L[kPanel][kPanel + 1];
  for (int e = threadIdx.x; e < pw * pw; e += blockDim.x) L[e / pw][e % pw] = a[(int64_t)(k + e / pw) * bs + k + e % pw];
  __syncthreads();
  const int c = k + pw + blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= bs) return;
  float2 x[kPanel];
#pragma unroll
  for (int i = 0; i < kPanel; ++i) x[i] = i < pw ? a[(int64_t)(k + i) * bs + c] : make_float2(0.f, 0.f);
#pragma unroll
  for (int i = 1; i < kPanel; ++i) {
#pragma unroll
    for (int j = 0; j < i; ++j) x[i] = csubmulf(x[i], L[i][j], x[j]);
  }
#pragma unroll
  for (int i = 1; i < kPanel; ++i)
    if (i < pw) a[(int64_t)(k + i) * bs + c] = x[i];
}

// A22 -= L21 U12 on 64 x 64 tiles; 256 threads, each 4 x 4 outputs (rows ty + 16 r, columns tx + 16 q).
__global__ void __launch_bounds__(256) bd_gemm_kernel(int bs, int k, float2* __restrict__ lu) {
  const int b = blockIdx.z;
  float2* a = lu + (int64_t)b * bs * bs;
  const int pw = min(kPanel, bs - k);
  const int r0 = k + pw + blockIdx.y * 64, c0 = k + pw + blockIdx.x * 64;
  __shared__ float2 Ls[64][kPanel + 1];
  __shared__ float2 Us[kPanel][64];
  const int tid = threadIdx.x;
  for (int e = tid; e < 64 * kPanel; e += 256) {
    const int i = e / kPanel, j = e % kPanel;
    Ls[i][j] = (r0 + i < bs && j < pw) ? a[(int64_t)(r0 + i) * bs + k + j] : make_float2(0.f, 0.f);
  }
  for (int e = tid; e < kPanel * 64; e += 256) {
    const int j = e / 64, c = e % 64;
    Us[j][c] = (c0 + c < bs && j < pw) ? a[(int64_t)(k + j) * bs + c0 + c] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int tx = tid & 15, ty = tid >> 4;
  float2 acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int q = 0; q < 4; ++q) acc[r][q] = make_float2(0.f, 0.f);
#pragma unroll 8
  for (int j = 0; j < kPanel; ++j) {
    float2 l[4], u[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) l[r] = Ls[ty + 16 * r][j];
#pragma unroll
    for (int q = 0; q < 4; ++q) u[q] = Us[j][tx + 16 * q];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc[r][q].x = fmaf(l[r].x, u[q].x, fmaf(-l[r].y, u[q].y, acc[r][q].x));
        acc[r][q].y = fmaf(l[r].x, u[q].y, fmaf(l[r].y, u[q].x, acc[r][q].y));
      }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = r0 + ty + 16 * r;
    if (i >= bs) continue;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = c0 + tx + 16 * q;
      if (c < bs) {
        float2 v = a[(int64_t)i * bs + c];
        v.x -= acc[r][q].x;
        v.y -= acc[r][q].y;
        a[(int64_t)i * bs + c] = v;
      }
    }
  }
}

// perm[i]: the row of the original block that the interchanges bring to position i.
__global__ void bd_perm_kernel(int bs, int nb, const int* __restrict__ piv, int* __restrict__ perm) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  int* p = perm + (int64_t)b * bs;
  for (int i = 0; i < bs; ++i) p[i] = i;
  for (int j = 0; j < bs; ++j) {
    const int q = piv[(int64_t)b * bs + j];
    const int t = p[j];
    p[j] = p[q];
    p[q] = t;
  }
}

// z = U^{-1} L^{-1} P r for block blockIdx.y and vector blockIdx.x (VT: double2 or float2 vectors).
template <typename VT>
__global__ void __launch_bounds__(1024) bd_apply_kernel(int64_t n, int bs, const float2* __restrict__ lu,
                                                        const int* __restrict__ perm, const VT* __restrict__ r,
                                                        VT* __restrict__ z) {
  extern __shared__ float2 x[];
  const int v = blockIdx.x, b = blockIdx.y;
  const float2* a = lu + (int64_t)b * bs * bs;
  const int* p = perm + (int64_t)b * bs;
  const VT* rv = r + (int64_t)v * n + (int64_t)b * bs;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int i = threadIdx.x; i < bs; i += blockDim.x) {
    const VT t = rv[p[i]];
    x[i] = make_float2((float)t.x, (float)t.y);
  }
  __syncthreads();
  // forward: unit lower L
  for (int t0 = 0; t0 < bs; t0 += 32) {
    for (int w = warp; w < 32; w += nwarps) {
      const int i = t0 + w;
      if (i >= bs) break;
      float2 acc = make_float2(0.f, 0.f);
      for (int j = lane; j < t0; j += 32) {
        const float2 l = a[(int64_t)i * bs + j];
        acc.x = fmaf(l.x, x[j].x, fmaf(-l.y, x[j].y, acc.x));
        acc.y = fmaf(l.x, x[j].y, fmaf(l.y, x[j].x, acc.y));
      }
      for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      }
      if (lane == 0) { x[i].x -= acc.x; x[i].y -= acc.y; }
    }
    __syncthreads();
    if (warp == 0) {
      const int i = t0 + lane;
      float2 xi = i < bs ? x[i] : make_float2(0.f, 0.f);
      for (int j = 0; j < 32 && t0 + j < bs; ++j) {
        const float2 xj = shflf(xi, j);
        if (lane > j && i < bs) xi = csubmulf(xi, a[(int64_t)i * bs + t0 + j], xj);
      }
      if (i < bs) x[i] = xi;
    }
    __syncthreads();
  }
  // backward: upper U with its diagonal
  const int last = ((bs - 1) / 32) * 32;
  for (int t0 = last; t0 >= 0; t0 -= 32) {
    const int t1 = min(t0 + 32, bs);
    for (int w = warp; w < 32; w += nwarps) {
      const int i = t0 + w;
      if (i >= bs) break;
      float2 acc = make_float2(0.f, 0.f);
      for (int j = t1 + lane; j < bs; j += 32) {
        const float2 u = a[(int64_t)i * bs + j];
        acc.x = fmaf(u.x, x[j].x, fmaf(-u.y, x[j].y, acc.x));
        acc.y = fmaf(u.x, x[j].y, fmaf(u.y, x[j].x, acc.y));
      }
      for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
      }
      if (lane == 0) { x[i].x -= acc.x; x[i].y -= acc.y; }
    }
    __syncthreads();
    if (warp == 0) {
      const int i = t0 + lane;
      float2 xi = i < bs ? x[i] : make_float2(0.f, 0.f);
      for (int j = t1 - t0 - 1; j >= 0; --j) {
        if (lane == j) xi = cmulf(xi, crecipf(a[(int64_t)i * bs + i]));
        const float2 xj = shflf(xi, j);
        if (lane < j && i < bs) xi = csubmulf(xi, a[(int64_t)i * bs + t0 + j], xj);
      }
      if (i < bs) x[i] = xi;
    }
    __syncthreads();
  }
  VT* zv = z + (int64_t)v * n + (int64_t)b * bs;
  for (int i = threadIdx.x; i < bs; i += blockDim.x) {
    VT o;
    o.x = x[i].x;
    o.y = x[i].y;
    zv[i] = o;
  }
}

}  // namespace bie

struct bie_blockdiag_s {
  bie_ctx ctx;
  int64_t n;
  int bs, nb;
  float2* lu;
  int* piv;
  int* perm;
};

using namespace bie;

namespace bie {
template <typename VT>
static bie_status blockdiag_apply_t(bie_blockdiag P, const VT* r, int nv, VT* z) {
  const cudaStream_t st = P->ctx->stream;
  dim3 grid(nv, P->nb);
  bd_apply_kernel<VT><<<grid, 1024, sizeof(float2) * P->bs, st>>>(P->n, P->bs, P->lu, P->perm, r, z);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BIE_OK : cuda_fail(e, "bd_apply_kernel");
}
bie_status blockdiag_apply_dev(bie_blockdiag P, const double2* r, int nv, double2* z) {
  return blockdiag_apply_t<double2>(P, r, nv, z);
}
bie_status blockdiag_apply_f32(bie_blockdiag P, const float2* r, int nv, float2* z) {
  return blockdiag_apply_t<float2>(P, r, nv, z);
}
}  // namespace bie

extern "C" {

bie_status bie_blockdiag_create(bie_ctx ctx, int64_t n, const double* A, int block, bie_blockdiag* out) {
  if (!ctx || !A || !out || n <= 0) { set_error("bie_blockdiag_create: invalid arguments"); return BIE_EINVAL; }
  if (block < 32 || block > 4096 || n % block != 0) {
    set_error("bie_blockdiag_create: block = %d must be in [32, 4096] and divide n = %lld", block, (long long)n);
    return BIE_EINVAL;
  }
  *out = nullptr;
  const cudaStream_t st = ctx->stream;
  bie_blockdiag P = new bie_blockdiag_s();
  P->ctx = ctx;
  P->n = n;
  P->bs = block;
  P->nb = (int)(n / block);
  int* singular = nullptr;
  cudaError_t e = cudaMalloc((void**)&P->lu, sizeof(float2) * (size_t)P->nb * block * block);
  if (e == cudaSuccess) e = cudaMalloc((void**)&P->piv, sizeof(int) * (size_t)P->nb * block);
  if (e == cudaSuccess) e = cudaMalloc((void**)&P->perm, sizeof(int) * (size_t)P->nb * block);
  if (e == cudaSuccess) e = cudaMalloc((void**)&singular, sizeof(int) * P->nb);
  if (e != cudaSuccess) {
    bie_blockdiag_free(P);
    cudaFree(singular);
    return cuda_fail(e, "bie_blockdiag_create allocation");
  }
  cudaMemsetAsync(singular, 0, sizeof(int) * P->nb, st);
  const int bs = block, nb = P->nb;
  bd_extract_kernel<<<ctx->sms * 8, 256, 0, st>>>(n, bs, nb, (const double2*)A, P->lu);
  for (int k = 0; k < bs; k += kPanel) {
    const int pw = std::min(kPanel, bs - k);
    bd_panel_kernel<<<nb, 1024, 0, st>>>(bs, k, P->lu, P->piv, singular);
    bd_swap_kernel<<<dim3((bs + 255) / 256, nb), 256, 0, st>>>(bs, k, P->lu, P->piv);
    const int rest = bs - k - pw;
    if (rest > 0) {
      bd_trsm_kernel<<<dim3((rest + 127) / 128, nb), 128, 0, st>>>(bs, k, P->lu);
      bd_gemm_kernel<<<dim3((rest + 63) / 64, (rest + 63) / 64, nb), 256, 0, st>>>(bs, k, P->lu);
    }
  }
  bd_perm_kernel<<<(nb + 127) / 128, 128, 0, st>>>(bs, nb, P->piv, P->perm);
  e = cudaGetLastError();
  std::vector<int> sing(nb, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(sing.data(), singular, sizeof(int) * nb, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(singular);
  if (e != cudaSuccess) {
    bie_blockdiag_free(P);
    return cuda_fail(e, "bie_blockdiag_create");
  }
  for (int b = 0; b < nb; ++b)
    if (sing[b]) {
      set_error("bie_blockdiag_create: block %d is singular (zero pivot at column %d)", b, sing[b] - 1);
      bie_blockdiag_free(P);
      return BIE_ENAN;
    }
  *out = P;
  return BIE_OK;
}

bie_status bie_blockdiag_apply(bie_blockdiag P, const double* r, int nv, double* z) {
  if (!P || !r || !z || nv < 1 || nv > 65535) { set_error("bie_blockdiag_apply: invalid arguments"); return BIE_EINVAL; }
  if (r == z) { set_error("bie_blockdiag_apply: z must not alias r"); return BIE_EINVAL; }
  return blockdiag_apply_dev(P, (const double2*)r, nv, (double2*)z);
}

int64_t bie_blockdiag_size(bie_blockdiag P) { return P ? P->n : 0; }

void bie_blockdiag_free(bie_blockdiag P) {
  if (!P) return;
  cudaFree(P->lu);
  cudaFree(P->piv);
  cudaFree(P->perm);
  delete P;
}

}  // extern "C"
