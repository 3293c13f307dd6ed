// Dense Nystrom assembly (Section 3.4; Section 3.1 Eqs. (S123), (S1); Section 4).
//
// Preparation stage: every entry of the N x N matrix from the 16-point
// Gauss-Legendre rule in t and the trapezoid rule in theta (Eq. (S1) with
// Eq. (Sphi:sm)); entries of near blocks (|i - j| <= 1) are set to zero and the
// identity of K +- I / CFIE is added on the diagonal (identity acting on the
// weighted density = diag(1/J)).
//
// Correction stage: for every target node and near panel, the Parseval weights
// of the 16 GGQ source rings (pair pipeline) are combined with the GGQ weights
// and the Lagrange basis of the source panel's Legendre nodes:
//   A[x, (i',n,l')] += (h/2) sum_g w_g L_n(s_g) W_{l'}(x, s_g).
// One target panel at a time, so the weight buffer holds 16*48*Mth pairs.
#include <cmath>

#include "bie_internal.cuh"
#include "dw.cuh"
#include "pair_args.cuh"

namespace bie {

struct FarArgs {
  SurfP S;
  int Np, Mt, periodic;
  int kprime;           // the double-layer part is K' (tau_0 with the target's normal)
  int64_t N;
  double h, k, wid;
  int unweighted;
  cplx ws, wk;
  const double* pts;
  const double* nrm;
  const double* jac;
  double wq[16];        // (h/2) w_n / Mt: Gauss-Legendre weight on [-1, 1] times the panel and trapezoid factors
  cplx* A;
};

// k rho below which the entry's phase goes through the double-word sin/cos (FP64 reduction by pi/2)
constexpr double kFarDwMaxPhase = 4096.0;
// rows per thread of the far fill: a thread keeps its column's node, normal and weight in registers
constexpr int kFarRows = 16;

// Thread per column, kFarRows consecutive rows per block (row tiles grid-strided over blockIdx.y);
// a row's 256 entries of a block are stored contiguously.  FP64 for the differences, rho^2, rsqrt
// and k rho (the phase keeps FP64 accuracy); the sin/cos series and the products of the entry in
// double words, so that the FP64 pipe carries about a third of the instructions of an all-FP64 entry.
__global__ void far_fill_kernel(const FarArgs a) {
  const int N = (int)a.N;
  const int per_panel = 16 * a.Mt;
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= N) return;
  const bool wantS = a.ws.re != 0.0 || a.ws.im != 0.0;
  const bool wantK = a.wk.re != 0.0 || a.wk.im != 0.0;
  const float4 wsd = dwc_from(a.ws), wkd = dwc_from(a.wk);
  const int jcol = col / per_panel;
  const int n = (col / a.Mt) & 15;
  const double w = a.unweighted ? a.wq[n] * a.jac[col] : a.wq[n];
  const float2 wd = dw_from(w);
  const double sx = a.pts[3 * col], sy = a.pts[3 * col + 1], sz = a.pts[3 * col + 2];
  const double nx = a.nrm[3 * col], ny = a.nrm[3 * col + 1], nz = a.nrm[3 * col + 2];
  for (int r0 = blockIdx.y * kFarRows; r0 < N; r0 += gridDim.y * kFarRows) {
    const int rend = min(r0 + kFarRows, N);
    for (int row = r0; row < rend; ++row) {
      const int jrow = row / per_panel;
      cplx v = C(0.0);
      int dj = abs(jcol - jrow);
      if (a.periodic && a.Np - dj < dj) dj = a.Np - dj;   // torus: the first and last panels are neighbours
      if (dj >= 2) {
        const double yx = sx - a.pts[3 * row], yy = sy - a.pts[3 * row + 1], yz = sz - a.pts[3 * row + 2];
        const double r2 = yx * yx + yy * yy + yz * yz;
        const double rinv = rsqrt(r2);
        const double x = a.k * (r2 * rinv);
        const double tau0 = !wantK ? 0.0
                            : a.kprime ? -(a.nrm[3 * row] * yx + a.nrm[3 * row + 1] * yy + a.nrm[3 * row + 2] * yz)
                                       : nx * yx + ny * yy + nz * yz;
        if (x < kFarDwMaxPhase) {
          float2 sn, cs;
          dw_sincos(x, &sn, &cs);
          const float2 ri = dw_from(rinv);
          float4 val = dwc_zero();
          if (wantS) val = dwc_mul(wsd, mkc(dw_mul(cs, ri), dw_mul(sn, ri)));   // ws e^{ik rho} / rho
          if (wantK) {
            // wk tau0 / rho^3 e^{ik rho} (ik rho - 1) = wk tau0 / rho^3 ((-cos - x sin) + i (x cos - sin))
            const float2 xd = dw_from(x);
            const float2 f = dw_mul(dw_from(tau0), dw_mul(ri, dw_mul(ri, ri)));
            const float4 g = mkc(dw_sub(dw_neg(cs), dw_mul(xd, sn)), dw_sub(dw_mul(xd, cs), sn));
            val = dwc_add(val, dwc_mul(wkd, dwc_mulr(g, f)));
          }
          v = dwc_to(dwc_mulr(val, wd));
        } else {
          double s, c;
          sincos(x, &s, &c);
          const cplx e = C(c, s);
          cplx val = C(0.0);
          if (wantS) val = rinv * (a.ws * e);
          if (wantK) val = val + (tau0 * rinv * rinv * rinv) * (a.wk * (e * C(-1.0, x)));
          v = w * val;
        }
      }
      if (col == row && a.wid != 0.0) v = v + C(a.unweighted ? a.wid : a.wid / a.jac[row], 0.0);
      a.A[(int64_t)row * N + col] = v;
    }
  }
}

// Where the near fill writes: the dense matrix (row-major, leading dimension N, entries added
// to what is there), or the near band (row - row0, leading dimension 3*16*Mt, slot delta of
// 16*Mt entries per row; entries overwritten, slots of source panels outside the surface zeroed).
struct NearOut {
  cplx* A;
  int64_t ld, row0;
  int band;
};

// Near fill of one target panel: block per (local target node tl in [0, 16 Mt), delta).
// A[row, block] += sS * sum_g coef W_S + sK * sum_g coef W_K   (W_K may be null).
// kDW: single layer alone with double-word weights (re.h, re.l, im.h, im.l); the GGQ fold, the
// scaling and the Jacobian run in double words, and only the update of A in FP64.
template <bool kDW>
__global__ void near_fill_kernel(int Np, int Mt, int periodic, int jpanel, cplx sS, cplx sK,
                                 const double* __restrict__ coef, const float2* __restrict__ coefw,
                                 const cplx* __restrict__ WS, const cplx* __restrict__ WK,
                                 const double* __restrict__ jcol, const NearOut out) {
  const int tl = blockIdx.x;            // l * Mt + i
  const int d = blockIdx.y;
  const int l = tl / Mt, i = tl % Mt;
  int ip = jpanel + d - 1;
  if (periodic) ip = (ip + Np) % Np;   // torus: cyclic neighbours
  const bool inside = ip >= 0 && ip < Np;
  if (!inside && !out.band) return;
  const int64_t tn = (int64_t)jpanel * 16 + l;
  const int64_t row = tn * Mt + i;
  cplx* Arow = out.band ? out.A + (row - out.row0) * out.ld + (int64_t)d * 16 * Mt
                        : out.A + row * out.ld + (int64_t)ip * 16 * Mt;
  if (!inside) {
    for (int e = threadIdx.x; e < 16 * Mt; e += blockDim.x) Arow[e] = C(0.0);
    return;
  }
  // weight index within the panel chunk: (((l*3 + d)*16 + g)*Mt + i)
  const int64_t base = ((((int64_t)l * 3 + d) * 16) * Mt + i) * Mt;
  const double* cf = coef + ((d * 16 + l) * 16) * 16;   // [g][n]
  if constexpr (kDW) {
    // thread per (source angle lp, group of npt source nodes n): the 16 weights of lp (one per GGQ
    // node g) are loaded once and folded into the group's npt outputs (they were loaded once per output)
    const float2* cw = coefw + ((d * 16 + l) * 16) * 16;
    const float4* W = reinterpret_cast<const float4*>(WS);
    const float4 sw = dwc_from(sS);
    const int npt = Mt >= 128 ? 8 : 4;
    for (int it = threadIdx.x; it < (16 / npt) * Mt; it += blockDim.x) {
      const int lp = it % Mt, n0 = (it / Mt) * npt;
      float4 w[16];
#pragma unroll
      for (int g = 0; g < 16; ++g) w[g] = W[base + (int64_t)g * Mt * Mt + lp];
      for (int n = n0; n < n0 + npt; ++n) {
        float2 ar = make_float2(0.f, 0.f), ai = make_float2(0.f, 0.f);
#pragma unroll
        for (int g = 0; g < 16; ++g) {
          const float2 c = cw[g * 16 + n];
          ar = dw_add(ar, dw_mul(c, cre(w[g])));
          ai = dw_add(ai, dw_mul(c, cim(w[g])));
        }
        const int e = n * Mt + lp;
        float4 add = dwc_mul(sw, mkc(ar, ai));
        if (jcol) add = dwc_mulr(add, dw_from(jcol[(int64_t)ip * 16 * Mt + e]));   // times J of the source node
        const cplx ad = dwc_to(add);
        Arow[e] = out.band ? ad : Arow[e] + ad;
      }
    }
  } else {
  for (int e = threadIdx.x; e < 16 * Mt; e += blockDim.x) {
    const int n = e / Mt, lp = e % Mt;
    cplx accS = C(0.0), accK = C(0.0);
#pragma unroll 4
    for (int g = 0; g < 16; ++g) {
      const int64_t w = base + (int64_t)g * Mt * Mt + lp;
      if (WS) accS = accS + cf[g * 16 + n] * WS[w];
      if (WK) accK = accK + cf[g * 16 + n] * WK[w];
    }
    cplx add = sS * accS + sK * accK;
    if (jcol) add = jcol[(int64_t)ip * 16 * Mt + e] * add;   // unweighted unknown: times J of the source node
    Arow[e] = out.band ? add : Arow[e] + add;
  }
  }
}

// Near fill of one target panel into its near band from Parseval weights kept in a ring of pair
// rows (the batch scheduler's throughput mode): the weights of pair pp of the panel (pp in the
// panel's enumeration order) at ring row (pbase + pp) % ring, row length w_ld.  Single layer,
// weighted density; band [16 Mt rows][3][16 Mt], entries overwritten, slots of source panels outside
// the surface zeroed.  Block per (local target node, delta), as near_fill_kernel.
__global__ void near_fill_ring_kernel(int Np, int Mt, int periodic, int jpanel, cplx sS,
                                      const double* __restrict__ coef, const cplx* __restrict__ W, int64_t pbase,
                                      int64_t ring, int w_ld, cplx* __restrict__ band) {
  const int tl = blockIdx.x;            // l * Mt + i
  const int d = blockIdx.y;
  const int l = tl / Mt, i = tl % Mt;
  int ip = jpanel + d - 1;
  if (periodic) ip = (ip + Np) % Np;
  cplx* Arow = band + (int64_t)tl * 3 * 16 * Mt + (int64_t)d * 16 * Mt;
  if (ip < 0 || ip >= Np) {
    for (int e = threadIdx.x; e < 16 * Mt; e += blockDim.x) Arow[e] = C(0.0);
    return;
  }
  const int64_t pp0 = (((int64_t)l * 3 + d) * 16) * Mt + i;   // pair (l, d, g = 0, i) of the panel
  const double* cf = coef + ((d * 16 + l) * 16) * 16;          // [g][n]
  // thread per (source angle lp, group of npt source nodes n), as near_fill_kernel
  const int npt = Mt >= 128 ? 8 : 4;
  for (int it = threadIdx.x; it < (16 / npt) * Mt; it += blockDim.x) {
    const int lp = it % Mt, n0 = (it / Mt) * npt;
    cplx w[16];
#pragma unroll
    for (int g = 0; g < 16; ++g) w[g] = W[((pbase + pp0 + (int64_t)g * Mt) % ring) * w_ld + lp];
    for (int n = n0; n < n0 + npt; ++n) {
      cplx acc = C(0.0);
#pragma unroll
      for (int g = 0; g < 16; ++g) acc = acc + cf[g * 16 + n] * w[g];
      Arow[n * Mt + lp] = sS * acc;
    }
  }
}

bie_status near_fill_ring(bie_surface s, int jpanel, const cplx* W, int64_t pbase, int64_t ring, int w_ld,
                          cplx* band, cudaStream_t st) {
  const int Mt = s->Mt;
  const cplx sS = C(0.5 * s->h);
  near_fill_ring_kernel<<<dim3(16 * Mt, 3), 256, 0, st>>>(s->Np, Mt, s->sp.periodic, jpanel, sS, s->near_coef, W, pbase,
                                                          ring, w_ld, band);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BIE_OK : cuda_fail(e, "near_fill_ring_kernel");
}

}  // namespace bie

using namespace bie;

extern "C" {

// Correction stage over all target panels, in groups of panels whose pair weights fit a ~4 GB
// buffer.  dst: where the near fill writes (NearOut; row0 is set per group when staging).
// host_band: page-locked host memory for the near band [N][3][16 Mt]; the fill then writes two
// device staging slots of one group's band rows each, and the copy of a finished group to the
// host runs on a second stream while the next group's pair kernels run.  The ctx stream waits for
// the last copy, so the band is complete when the ctx stream reaches the end of this call.
static bie_status near_stage(bie_ctx ctx, bie_surface s, unsigned kernels, double k, cplx ws, cplx wk,
                             const double* jac, NearOut dst, cplx* host_band) {
  const int Mt = s->Mt;
  const unsigned dl = kernels & (BIE_KERNEL_K | BIE_KERNEL_KP);   // the double layer (at most one kind)
  const int nk = ((kernels & BIE_KERNEL_S) ? 1 : 0) + (dl ? 1 : 0);
  const int64_t panel_pairs = (int64_t)16 * 48 * Mt;
  const int64_t panel_rows = (int64_t)16 * Mt;
  // panels per launch: enough pairs for many waves, weight buffer at most ~4 GB
  const size_t per_panel_bytes = sizeof(cplx) * (size_t)panel_pairs * Mt * nk;
  int group = (int)(((size_t)4 << 30) / per_panel_bytes);
  if (group < 1) group = 1;
  if (group > s->Np) group = s->Np;
  // >= 8 groups: every copy but the last overlaps the next group's pair kernels, and the last one
  // (the exposed part of the copy) is an eighth of the band (16 groups of one panel were slower:
  // launches of 98,304 pairs leave the root kernel's last wave mostly empty)
  if (host_band && group > (s->Np + 7) / 8) group = (s->Np + 7) / 8;
  const int64_t chunk_pairs = panel_pairs * group;
  const cudaStream_t st0 = ctx->stream;
  cplx* W = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&W, sizeof(cplx) * chunk_pairs * Mt * nk, st0);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync(weights)");
  cplx* stage = nullptr;
  cudaStream_t cs = nullptr;
  cudaEvent_t ev_fill[2] = {nullptr, nullptr}, ev_copy[2] = {nullptr, nullptr};
  const int64_t slot_elems = (int64_t)group * panel_rows * dst.ld;
  bie_status st = BIE_OK;
  if (host_band) {
    e = cudaMallocAsync((void**)&stage, sizeof(cplx) * 2 * slot_elems, st0);
    if (e != cudaSuccess) st = cuda_fail(e, "cudaMallocAsync(band staging)");
    if (st == BIE_OK && (e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess)
      st = cuda_fail(e, "cudaStreamCreate(band copies)");
    for (int q = 0; q < 2 && st == BIE_OK; ++q) {
      if ((e = cudaEventCreateWithFlags(&ev_fill[q], cudaEventDisableTiming)) != cudaSuccess ||
          (e = cudaEventCreateWithFlags(&ev_copy[q], cudaEventDisableTiming)) != cudaSuccess)
        st = cuda_fail(e, "cudaEventCreate(band copies)");
    }
  }
  const cplx sS = ws * (0.5 * s->h), sK = wk * (0.5 * s->h);
  // single layer alone: double-word weights and fold (unless the context runs the transforms in FP64)
  const bool dw = kernels == BIE_KERNEL_S && !ctx->fp64_transforms;
  for (int j0 = 0, gi = 0; j0 < s->Np && st == BIE_OK; j0 += group, ++gi) {
    const int nj = (j0 + group <= s->Np) ? group : s->Np - j0;
    const int slot = gi & 1;
    NearOut o = dst;
    if (host_band) {
      if (gi >= 2 && (e = cudaStreamWaitEvent(st0, ev_copy[slot], 0)) != cudaSuccess) {
        st = cuda_fail(e, "cudaStreamWaitEvent(band slot)");
        break;
      }
      o.A = stage + slot * slot_elems;
      o.row0 = (int64_t)j0 * panel_rows;
    }
    PairArgs a = make_pair_args(s, k, kernels);
    a.enumerate = 1;
    a.p0 = (int64_t)j0 * panel_pairs;
    a.n_pairs = panel_pairs * nj;
    a.weights_out = W;
    a.weights_stride = panel_pairs * nj * Mt;
    a.weights_dw = dw;
    st = launch_pairs(s, a);
    if (st != BIE_OK) break;
    const cplx* WS = (kernels & BIE_KERNEL_S) ? W : nullptr;
    const cplx* WK = dl ? W + (nk - 1) * a.weights_stride : nullptr;
    const int tm = trace_begin(ctx, kTraceNearFill);
    for (int jj = 0; jj < nj; ++jj) {
      const int64_t off = (int64_t)jj * panel_pairs * Mt;
      dim3 grid(16 * Mt, 3);
      if (dw)
        near_fill_kernel<true><<<grid, 256, 0, st0>>>(s->Np, Mt, s->sp.periodic, j0 + jj, sS, sK, s->near_coef, s->near_coef_dw,
                                                      WS + off, nullptr, jac, o);
      else
        near_fill_kernel<false><<<grid, 256, 0, st0>>>(s->Np, Mt, s->sp.periodic, j0 + jj, sS, sK, s->near_coef, s->near_coef_dw,
                                                       WS ? WS + off : nullptr, WK ? WK + off : nullptr, jac, o);
    }
    trace_end(ctx, tm);
    e = cudaGetLastError();
    if (e != cudaSuccess) { st = cuda_fail(e, "near_fill_kernel"); break; }
    if (host_band) {
      if ((e = cudaEventRecord(ev_fill[slot], st0)) != cudaSuccess ||
          (e = cudaStreamWaitEvent(cs, ev_fill[slot], 0)) != cudaSuccess ||
          (e = cudaMemcpyAsync(host_band + o.row0 * dst.ld, o.A, sizeof(cplx) * nj * panel_rows * dst.ld,
                               cudaMemcpyDeviceToHost, cs)) != cudaSuccess ||
          (e = cudaEventRecord(ev_copy[slot], cs)) != cudaSuccess)
        st = cuda_fail(e, "near band copy to the host");
    }
  }
  if (cs) {
    // join: the ctx stream (and so the staging free and the caller) follow the last copy
    cudaEvent_t done = nullptr;
    if (cudaEventCreateWithFlags(&done, cudaEventDisableTiming) == cudaSuccess) {
      cudaEventRecord(done, cs);
      cudaStreamWaitEvent(st0, done, 0);
      cudaEventDestroy(done);
    } else {
      cudaStreamSynchronize(cs);
    }
    cudaStreamDestroy(cs);
  }
  for (int q = 0; q < 2; ++q) {
    if (ev_fill[q]) cudaEventDestroy(ev_fill[q]);
    if (ev_copy[q]) cudaEventDestroy(ev_copy[q]);
  }
  if (stage) cudaFreeAsync(stage, st0);
  cudaFreeAsync(W, st0);
  return st;
}

static bie_status check_near_args(const char* who, bie_ctx ctx, bie_surface s, unsigned kernels, double k,
                                  const void* out) {
  if (!ctx || !s || !out) { set_error("%s: NULL argument", who); return BIE_EINVAL; }
  if (!(k > 0) || !(k < 1e6)) { set_error("%s: k must be in (0, 1e6)", who); return BIE_EINVAL; }
  if (kernels == 0 || (kernels & ~(BIE_KERNEL_S | BIE_KERNEL_K | BIE_KERNEL_KP)) ||
      ((kernels & BIE_KERNEL_K) && (kernels & BIE_KERNEL_KP))) {
    set_error("%s: bad kernel mask %u (S and at most one of K, KP)", who, kernels);
    return BIE_EINVAL;
  }
  return BIE_OK;
}

bie_status bie_assemble_near(bie_ctx ctx, bie_surface s, unsigned kernels, double k, double ws_re, double ws_im,
                             double wk_re, double wk_im, double* A_out) {
  const bie_status st = check_near_args("bie_assemble_near", ctx, s, kernels, k, A_out);
  if (st != BIE_OK) return st;
  const NearOut o = {(cplx*)A_out, s->N, 0, 0};
  return near_stage(ctx, s, kernels, k, C(ws_re, ws_im), C(wk_re, wk_im), nullptr, o, nullptr);
}

bie_status bie_assemble_near_band(bie_ctx ctx, bie_surface s, unsigned kernels, double k, double ws_re,
                                  double ws_im, double wk_re, double wk_im, double* band_out) {
  const bie_status st = check_near_args("bie_assemble_near_band", ctx, s, kernels, k, band_out);
  if (st != BIE_OK) return st;
  cudaPointerAttributes at;
  const cudaError_t e = cudaPointerGetAttributes(&at, band_out);
  if (e != cudaSuccess) return cuda_fail(e, "bie_assemble_near_band: cudaPointerGetAttributes(band_out)");
  const NearOut o = {(cplx*)band_out, (int64_t)3 * 16 * s->Mt, 0, 1};
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)
    return near_stage(ctx, s, kernels, k, C(ws_re, ws_im), C(wk_re, wk_im), nullptr, o, nullptr);
  if (at.type == cudaMemoryTypeHost)
    return near_stage(ctx, s, kernels, k, C(ws_re, ws_im), C(wk_re, wk_im), nullptr, o, (cplx*)band_out);
  set_error("bie_assemble_near_band: band_out is pageable host memory; give device memory or page-locked "
            "host memory (cudaHostAlloc / cudaHostRegister)");
  return BIE_EINVAL;
}

bie_status bie_assemble(bie_ctx ctx, bie_surface s, int op_flags, double k, double eta, double* A_out) {
  const bool unweighted = op_flags & BIE_UNWEIGHTED;
  const int op = op_flags & ~BIE_UNWEIGHTED;
  if (!ctx || !s || !A_out) { set_error("bie_assemble: NULL argument"); return BIE_EINVAL; }
  if (op < BIE_OP_S || op > BIE_OP_KP_MINUS_I) { set_error("bie_assemble: unknown operator %d", op); return BIE_EINVAL; }
  if (!(k > 0) || !(k < 1e6)) { set_error("bie_assemble: k must be in (0, 1e6)"); return BIE_EINVAL; }
  cplx ws = C(0.0), wk = C(0.0);
  double wid = 0.0;
  switch (op) {
    case BIE_OP_S: ws = C(1.0); break;
    case BIE_OP_K: wk = C(1.0); break;
    case BIE_OP_K_PLUS_I: wk = C(1.0); wid = 1.0; break;
    case BIE_OP_K_MINUS_I: wk = C(1.0); wid = -1.0; break;
    case BIE_OP_CFIE: wk = C(1.0); wid = 1.0; ws = C(0.0, -eta); break;
    case BIE_OP_KP: wk = C(1.0); break;
    case BIE_OP_KP_PLUS_I: wk = C(1.0); wid = 1.0; break;
    case BIE_OP_KP_MINUS_I: wk = C(1.0); wid = -1.0; break;
  }
  const bool kp = op >= BIE_OP_KP;
  FarArgs fa;
  fa.S = s->sp;
  fa.Np = s->Np;
  fa.Mt = s->Mt;
  fa.periodic = s->sp.periodic;
  fa.kprime = kp ? 1 : 0;
  fa.N = s->N;
  fa.h = s->h;
  fa.k = k;
  fa.ws = ws;
  fa.wk = wk;
  fa.wid = wid;
  fa.unweighted = unweighted ? 1 : 0;
  fa.pts = s->pts;
  fa.nrm = s->nrm;
  fa.jac = s->jac;
  for (int n = 0; n < 16; ++n) fa.wq[n] = s->h * 0.5 * s->gl_w[n] / s->Mt;
  fa.A = (cplx*)A_out;
  const int64_t row_tiles = (s->N + kFarRows - 1) / kFarRows;
  dim3 grid((unsigned)((s->N + 255) / 256), (unsigned)(row_tiles < 65535 ? row_tiles : 65535));
  const int tm = trace_begin(ctx, kTraceFarFill);
  far_fill_kernel<<<grid, 256, 0, ctx->stream>>>(fa);
  trace_end(ctx, tm);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "far_fill_kernel");
  unsigned kernels = 0;
  if (ws.re != 0.0 || ws.im != 0.0) kernels |= BIE_KERNEL_S;
  if (wk.re != 0.0 || wk.im != 0.0) kernels |= kp ? BIE_KERNEL_KP : BIE_KERNEL_K;
  const NearOut o = {(cplx*)A_out, s->N, 0, 0};
  return near_stage(ctx, s, kernels, k, ws, wk, unweighted ? s->jac : nullptr, o, nullptr);
}

}  // extern "C"
