// Dense complex solve for the Nystrom system (the paper states the system,
// Section 3.4; the solver is this library's): restarted FGMRES, right
// preconditioned, classical Gram-Schmidt with one re-orthogonalisation.
//   prec = 0: FP64 matrix-vector products throughout.
//   prec = 1: FP32 copy of the matrix for the inner FGMRES (FP32 products,
//             FP32 accumulation), FP64 iterative refinement outside: r = b - A x
//             with the FP64 matrix, solve A dx = r approximately, x += dx.
// Host-driven: one small device->host copy of the Hessenberg column per step.
#include <chrono>
#include <cmath>
#include <complex>
#include <vector>

#include "bie_internal.cuh"

namespace bie {

__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum_f(float v) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// y = A x, FP64, one warp per row, 16-byte coalesced loads of the row.
__global__ void __launch_bounds__(256) zgemv64_kernel(int64_t n, const double2* __restrict__ A,
                                                      const double2* __restrict__ x, double2* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = w; row < n; row += nw) {
    const double2* a = A + row * n;
    double re = 0, im = 0;
    for (int64_t c = lane; c < n; c += 32) {
      const double2 av = __ldcs(a + c);
      const double2 xv = __ldg(x + c);
      re = fma(av.x, xv.x, fma(-av.y, xv.y, re));
      im = fma(av.x, xv.y, fma(av.y, xv.x, im));
    }
    re = warp_sum_d(re);
    im = warp_sum_d(im);
    if (lane == 0) y[row] = make_double2(re, im);
  }
}

// y = A32 x32 with FP32 products summed in FP32 over chunks of 32 terms per lane, the chunk sums
// accumulated in FP64 (1/64 of the work in FP64, so the kernel stays bound by the FP32 matrix read);
// y written in FP64.
__global__ void __launch_bounds__(256) cgemv32_kernel(int64_t n, const float2* __restrict__ A,
                                                      const float2* __restrict__ x, double2* __restrict__ y) {
  const int lane = threadIdx.x & 31;
  const int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = w; row < n; row += nw) {
    double dre = 0.0, dim = 0.0;
    float re = 0.f, im = 0.f;
    if (n & 1) {  // rows not 16-byte aligned: plain 8-byte loads
      int cnt = 0;
      for (int64_t c = lane; c < n; c += 32) {
        const float2 av = __ldcs(A + row * n + c), xv = __ldg(x + c);
        re = fmaf(av.x, xv.x, fmaf(-av.y, xv.y, re));
        im = fmaf(av.x, xv.y, fmaf(av.y, xv.x, im));
        if (++cnt == 32) { dre += re; dim += im; re = im = 0.f; cnt = 0; }
      }
    } else {
      const float4* a = reinterpret_cast<const float4*>(A + row * n);   // two complex entries per load
      const float4* xv4 = reinterpret_cast<const float4*>(x);
      const int64_t n2 = n / 2;
      for (int64_t c0 = lane; c0 < n2; c0 += 32 * 16) {   // chunks of 16 loads (32 complex terms) per lane
        float cr = 0.f, ci = 0.f;
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          const int64_t c = c0 + 32 * u;
          if (c < n2) {
            const float4 av = __ldcs(a + c);
            const float4 xv = __ldg(xv4 + c);
            cr = fmaf(av.x, xv.x, fmaf(-av.y, xv.y, cr));
            ci = fmaf(av.x, xv.y, fmaf(av.y, xv.x, ci));
            cr = fmaf(av.z, xv.z, fmaf(-av.w, xv.w, cr));
            ci = fmaf(av.z, xv.w, fmaf(av.w, xv.z, ci));
          }
        }
        dre += cr;
        dim += ci;
      }
    }
    dre = warp_sum_d(dre + re);
    dim = warp_sum_d(dim + im);
    if (lane == 0) y[row] = make_double2(dre, dim);
  }
}

__global__ void to_f32_kernel(int64_t n, const double2* __restrict__ a, float2* __restrict__ b) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = make_float2((float)a[i].x, (float)a[i].y);
}

// h[j] = sum_i conj(V[j][i]) w[i], j < J; partial sums per block, reduced on the host side kernel.
__global__ void multi_dot_kernel(int64_t n, int J, const double2* __restrict__ V, const double2* __restrict__ w,
                                 double2* __restrict__ partial) {
  __shared__ double sre[8], sim[8];
  const int j = blockIdx.y;
  double re = 0, im = 0;
  const double2* v = V + (int64_t)j * n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double2 a = v[i], b = w[i];
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
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { r += sre[k]; m += sim[k]; }
    partial[(int64_t)j * gridDim.x + blockIdx.x] = make_double2(r, m);
  }
}

__global__ void reduce_partials_kernel(int J, int nb, const double2* __restrict__ partial, double2* __restrict__ h) {
  const int j = blockIdx.x;
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
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { r += sre[k]; m += sim[k]; }
    h[j] = make_double2(r, m);
  }
}

// w -= sum_j h[j] V[j]
__global__ void multi_axpy_kernel(int64_t n, int J, const double2* __restrict__ V, const double2* __restrict__ h,
                                  double2* __restrict__ w) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double2 acc = w[i];
    for (int j = 0; j < J; ++j) {
      const double2 a = V[(int64_t)j * n + i], c = h[j];
      acc.x -= c.x * a.x - c.y * a.y;
      acc.y -= c.x * a.y + c.y * a.x;
    }
    w[i] = acc;
  }
}

// y = alpha x (+ beta y) helpers
__global__ void scale_copy_kernel(int64_t n, double s, const double2* __restrict__ x, double2* __restrict__ y) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = make_double2(s * x[i].x, s * x[i].y);
}
__global__ void sub_kernel(int64_t n, const double2* __restrict__ b, const double2* __restrict__ ax,
                           double2* __restrict__ r) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    r[i] = make_double2(b[i].x - ax[i].x, b[i].y - ax[i].y);
}
// x += sum_j c[j] Z[j]
__global__ void update_kernel(int64_t n, int J, const double2* __restrict__ Z, const double2* __restrict__ c,
                              double2* __restrict__ x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double2 acc = x[i];
    for (int j = 0; j < J; ++j) {
      const double2 z = Z[(int64_t)j * n + i], cj = c[j];
      acc.x += cj.x * z.x - cj.y * z.y;
      acc.y += cj.x * z.y + cj.y * z.x;
    }
    x[i] = acc;
  }
}

// x += dx
__global__ void add_kernel(int64_t n, const double2* __restrict__ dx, double2* __restrict__ x) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] = make_double2(x[i].x + dx[i].x, x[i].y + dx[i].y);
}

struct Solver {
  bie_ctx ctx;
  int64_t n;
  int m;
  const double2* A64;
  float2* A32 = nullptr;
  float2* x32 = nullptr;
  double2 *V = nullptr, *Z = nullptr, *w = nullptr, *r = nullptr, *tmp = nullptr, *hdev = nullptr, *partial = nullptr;
  int dot_blocks = 0;
  int gemv_blocks = 0;

  bie_status matvec(const double2* x, double2* y, bool low) {
    const cudaStream_t st = ctx->stream;
    if (low) {
      to_f32_kernel<<<ctx->sms * 4, 256, 0, st>>>(n, x, x32);
      cgemv32_kernel<<<gemv_blocks, 256, 0, st>>>(n, A32, x32, y);
    } else {
      zgemv64_kernel<<<gemv_blocks, 256, 0, st>>>(n, A64, x, y);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? BIE_OK : cuda_fail(e, "matvec");
  }

  // right preconditioner, flexible slot Z_j = M(V_j): none, block-diagonal, or learned (+ block)
  int pkind = 0;
  bie_blockdiag block = nullptr;
  bie_net net = nullptr;
  bie_surface surface = nullptr;
  double k = 0.0;
  bie_net_infer_s* infer = nullptr;
  bie_status precond(const double2* v, double2* z) {
    if (pkind == 1) return blockdiag_apply_dev(block, v, 1, z);
    if (pkind == 2) return net_precond_apply_dev(net, infer, block, surface, k, v, 1, z);
    const cudaError_t e = cudaMemcpyAsync(z, v, sizeof(double2) * n, cudaMemcpyDeviceToDevice, ctx->stream);
    return e == cudaSuccess ? BIE_OK : cuda_fail(e, "precond");
  }

  // h[0..J) = V[0..J)^H w  (copied to the host)
  bie_status dots(int J, const double2* Vb, const double2* wv, std::complex<double>* hh) {
    const cudaStream_t st = ctx->stream;
    dim3 g(dot_blocks, J);
    multi_dot_kernel<<<g, 256, 0, st>>>(n, J, Vb, wv, partial);
    reduce_partials_kernel<<<J, 256, 0, st>>>(J, dot_blocks, partial, hdev);
    cudaError_t e = cudaMemcpyAsync(hh, hdev, sizeof(double2) * J, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? BIE_OK : cuda_fail(e, "dots");
  }

  double norm(const double2* v) {
    std::complex<double> h;
    dots(1, v, v, &h);
    return std::sqrt(std::max(h.real(), 0.0));
  }

  // FGMRES on A x = b (x in/out), relative tolerance tol w.r.t. ||b||; returns iterations.
  bie_status fgmres(const double2* b, double2* x, double tol, int maxit, bool low, int* iters, double* relres) {
    const cudaStream_t st = ctx->stream;
    const int G = ctx->sms * 4;
    const double bnorm = norm(b);
    *iters = 0;
    if (bnorm == 0.0) {
      cudaMemsetAsync(x, 0, sizeof(double2) * n, st);
      *relres = 0.0;
      return BIE_OK;
    }
    std::vector<std::complex<double>> H((size_t)(m + 1) * m), cs(m), sn(m), g(m + 1), hh(m + 1), y(m);
    int total = 0;
    double res = 0.0;
    while (true) {
      bie_status s = matvec(x, tmp, low);
      if (s) return s;
      sub_kernel<<<G, 256, 0, st>>>(n, b, tmp, r);
      const double beta = norm(r);
      res = beta / bnorm;
      if (!(res == res)) return BIE_ENAN;
      if (res <= tol || total >= maxit) break;
      scale_copy_kernel<<<G, 256, 0, st>>>(n, 1.0 / beta, r, V);
      std::fill(g.begin(), g.end(), 0.0);
      g[0] = beta;
      int jdone = 0;
      for (int j = 0; j < m && total < maxit; ++j) {
        s = precond(V + (int64_t)j * n, Z + (int64_t)j * n);
        if (s) return s;
        s = matvec(Z + (int64_t)j * n, w, low);
        if (s) return s;
        // classical Gram-Schmidt, twice
        std::vector<std::complex<double>> hsum(j + 1, 0.0);
        for (int pass = 0; pass < 2; ++pass) {
          s = dots(j + 1, V, w, hh.data());
          if (s) return s;
          cudaMemcpyAsync(hdev, hh.data(), sizeof(double2) * (j + 1), cudaMemcpyHostToDevice, st);
          multi_axpy_kernel<<<G, 256, 0, st>>>(n, j + 1, V, hdev, w);
          for (int i = 0; i <= j; ++i) hsum[i] += hh[i];
        }
        const double hn = norm(w);
        for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hsum[i];
        H[(size_t)(j + 1) * m + j] = hn;
        if (hn > 0) scale_copy_kernel<<<G, 256, 0, st>>>(n, 1.0 / hn, w, V + (int64_t)(j + 1) * n);
        // Givens rotations
        for (int i = 0; i < j; ++i) {
          const std::complex<double> a = H[(size_t)i * m + j], bb = H[(size_t)(i + 1) * m + j];
          H[(size_t)i * m + j] = std::conj(cs[i]) * a + std::conj(sn[i]) * bb;
          H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * bb;
        }
        const std::complex<double> a = H[(size_t)j * m + j], bb = H[(size_t)(j + 1) * m + j];
        const double den = std::sqrt(std::norm(a) + std::norm(bb));
        cs[j] = den > 0 ? a / den : 1.0;
        sn[j] = den > 0 ? bb / den : 0.0;
        H[(size_t)j * m + j] = den;
        H[(size_t)(j + 1) * m + j] = 0.0;
        g[j + 1] = -sn[j] * g[j];
        g[j] = std::conj(cs[j]) * g[j];
        ++total;
        jdone = j + 1;
        const double est = std::abs(g[j + 1]) / bnorm;
        if (!(est == est)) return BIE_ENAN;
        if (est <= tol * 0.5 || hn == 0) break;
      }
      // back substitution and update x += Z y
      for (int i = jdone - 1; i >= 0; --i) {
        std::complex<double> acc = g[i];
        for (int k2 = i + 1; k2 < jdone; ++k2) acc -= H[(size_t)i * m + k2] * y[k2];
        y[i] = acc / H[(size_t)i * m + i];
      }
      cudaMemcpyAsync(hdev, y.data(), sizeof(double2) * jdone, cudaMemcpyHostToDevice, st);
      update_kernel<<<G, 256, 0, st>>>(n, jdone, Z, hdev, x);
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_fail(e, "fgmres update");
    }
    *iters = total;
    *relres = res;
    return BIE_OK;
  }
};

}  // namespace bie

using namespace bie;

extern "C" bie_status bie_solve(bie_ctx ctx, int64_t n, const double* A, const double* rhs, int nrhs, double* x,
                                const bie_solve_opts* opts, bie_solve_report* report) {
  const auto t0 = std::chrono::steady_clock::now();
  if (!ctx || !A || !rhs || !x || n <= 0 || nrhs <= 0 || !opts) { set_error("bie_solve: invalid arguments"); return BIE_EINVAL; }
  if (!(opts->tol > 0) || opts->restart < 1 || opts->restart > 1000 || opts->maxit < 1 || opts->prec < 0 ||
      opts->prec > 1 || opts->precond < 0 || opts->precond > 2) {
    set_error("bie_solve: invalid options");
    return BIE_EINVAL;
  }
  if (opts->precond == 1 && (!opts->block || bie_blockdiag_size(opts->block) != n)) {
    set_error("bie_solve: precond = 1 needs a block preconditioner of size n");
    return BIE_EINVAL;
  }
  if (opts->precond == 2 && (!opts->net || !opts->surface || opts->surface->N != n || !(opts->k > 0) ||
                             (opts->block && bie_blockdiag_size(opts->block) != n))) {
    set_error("bie_solve: precond = 2 needs a network, the surface of the unknowns and k > 0");
    return BIE_EINVAL;
  }
  Solver S;
  S.ctx = ctx;
  S.n = n;
  S.pkind = opts->precond;
  S.block = opts->block;
  S.net = opts->net;
  S.surface = opts->surface;
  S.k = opts->k;
  if (S.pkind == 2) S.infer = net_infer_new();
  S.m = opts->restart;
  S.A64 = (const double2*)A;
  S.dot_blocks = ctx->sms * 2;
  S.gemv_blocks = ctx->sms * 8;
  const cudaStream_t st = ctx->stream;
  std::vector<void*> owned;
  cudaError_t e = cudaSuccess;
  auto alloc = [&](void** p, size_t bytes) {
    *p = nullptr;
    if (e != cudaSuccess) return;
    e = cudaMallocAsync(p, bytes, st);
    if (e == cudaSuccess) owned.push_back(*p);
  };
  double2 *dx = nullptr, *res = nullptr;
  alloc((void**)&S.V, sizeof(double2) * n * (S.m + 1));
  alloc((void**)&S.Z, sizeof(double2) * n * S.m);
  alloc((void**)&S.w, sizeof(double2) * n);
  alloc((void**)&S.r, sizeof(double2) * n);
  alloc((void**)&S.tmp, sizeof(double2) * n);
  alloc((void**)&S.hdev, sizeof(double2) * (S.m + 2));
  alloc((void**)&S.partial, sizeof(double2) * (S.m + 1) * S.dot_blocks);
  if (opts->prec == 1) {
    alloc((void**)&S.A32, sizeof(float2) * n * n);
    alloc((void**)&S.x32, sizeof(float2) * (n + 1));
    alloc((void**)&dx, sizeof(double2) * n);
    alloc((void**)&res, sizeof(double2) * n);
  }
  bie_status status = BIE_OK;
  int total_iters = 0, refinements = 0;
  double worst = 0.0;
  if (e != cudaSuccess) status = cuda_fail(e, "bie_solve allocation");
  if (status == BIE_OK && opts->prec == 1) {
    to_f32_kernel<<<ctx->sms * 8, 256, 0, st>>>(n * n, (const double2*)A, S.A32);
    e = cudaGetLastError();
    if (e != cudaSuccess) status = cuda_fail(e, "to_f32");
  }
  int fallback = 0, budget0 = 0;
  double2* x0 = nullptr;
  if (S.pkind == 2 && opts->block) alloc((void**)&x0, sizeof(double2) * n);
  if (e != cudaSuccess && status == BIE_OK) status = cuda_fail(e, "bie_solve allocation");
  for (int c = 0; c < nrhs && status == BIE_OK; ++c) {
    const double2* b = (const double2*)rhs + (int64_t)c * n;
    double2* xc = (double2*)x + (int64_t)c * n;
    if (x0) cudaMemcpyAsync(x0, xc, sizeof(double2) * n, cudaMemcpyDeviceToDevice, st);
  retry:
    int it = 0;
    double rr = 0.0;
    if (opts->prec == 0) {
      status = S.fgmres(b, xc, opts->tol, opts->maxit - (total_iters - budget0), false, &it, &rr);
      total_iters += it;
    } else {
      const double bnorm = S.norm(b);
      for (int outer = 0; outer < 40 && status == BIE_OK; ++outer) {
        status = S.matvec(xc, S.tmp, false);
        if (status) break;
        sub_kernel<<<ctx->sms * 4, 256, 0, st>>>(n, b, S.tmp, res);
        rr = bnorm > 0 ? S.norm(res) / bnorm : 0.0;
        if (!(rr == rr)) { status = BIE_ENAN; break; }
        if (rr <= opts->tol || total_iters - budget0 >= opts->maxit) break;
        cudaMemsetAsync(dx, 0, sizeof(double2) * n, st);
        double inner_res = 0.0;
        // inner relative tolerance: what the outer step needs, but not below 1e-5: FP32 products of a
        // first-kind operator applied to rough Krylov vectors lose digits to cancellation
        const double inner_tol = std::max(1e-5, 0.5 * opts->tol / rr);
        status = S.fgmres(res, dx, inner_tol, opts->maxit - (total_iters - budget0), true, &it, &inner_res);
        total_iters += it;
        ++refinements;
        if (status) break;
        add_kernel<<<ctx->sms * 4, 256, 0, st>>>(n, dx, xc);
      }
    }
    if (status == BIE_OK && !(rr <= opts->tol)) status = BIE_ENOCONV;
    // learned preconditioner gave no convergence (or a NaN): the block-diagonal one takes over
    if ((status == BIE_ENOCONV || status == BIE_ENAN) && S.pkind == 2 && x0) {
      S.pkind = 1;
      fallback = 1;
      budget0 = total_iters;  // the fallback solve gets a fresh iteration budget
      status = BIE_OK;
      cudaMemcpyAsync(xc, x0, sizeof(double2) * n, cudaMemcpyDeviceToDevice, st);
      goto retry;
    }
    worst = std::max(worst, rr);
  }
  for (void* p : owned) cudaFreeAsync(p, st);
  cudaError_t e2 = cudaStreamSynchronize(st);
  if (status == BIE_OK && e2 != cudaSuccess) status = cuda_fail(e2, "bie_solve");
  if (report) {
    report->iterations = total_iters;
    report->refinements = refinements;
    report->rel_residual = worst;
    report->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    report->fallback_used = fallback;
  }
  net_infer_free(S.infer);
  if (status == BIE_ENOCONV) set_error("bie_solve: tolerance not reached within maxit");
  if (status == BIE_ENAN) set_error("bie_solve: NaN in the residual");
  return status;
}
