// Boundary data on the collocation nodes and layer-potential evaluation away
// from the surface (Section 3.4: 16-point Gauss-Legendre in t times the
// trapezoid rule in theta; Section 5 data).
#include <cmath>

#include "bie_internal.cuh"
#include "dw.cuh"

namespace bie {

__global__ void rhs_kernel(int64_t N, const double* __restrict__ pts, const double* __restrict__ nrm, int kind,
                           double px, double py, double pz, double k, double2* __restrict__ g) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = pts[3 * i], y = pts[3 * i + 1], z = pts[3 * i + 2];
    double s, c;
    if (kind == 0) {  // sound-soft plane wave: -e^{ik d.x}
      sincos(k * (px * x + py * y + pz * z), &s, &c);
      g[i] = make_double2(-c, -s);
    } else {
      const double dx = x - px, dy = y - py, dz = z - pz;
      const double r = sqrt(dx * dx + dy * dy + dz * dz);
      sincos(k * r, &s, &c);
      const double f = 1.0 / (4 * kPi * r);
      if (kind == 1) {   // point source e^{ik r}/(4 pi r)
        g[i] = make_double2(c * f, s * f);
      } else {           // its normal derivative nu.(x - src) e^{ik r} (ik r - 1) / (4 pi r^3)
        const double nd = (nrm[3 * i] * dx + nrm[3 * i + 1] * dy + nrm[3 * i + 2] * dz) * f / (r * r);
        // e^{ikr} (ikr - 1) = (-cos - kr sin) + i (kr cos - sin)
        g[i] = make_double2(nd * (-c - k * r * s), nd * (k * r * c - s));
      }
    }
  }
}

struct FieldArgs {
  int64_t N;
  int Mt;
  double h, k, eta;
  int rep, far, unweighted;
  double wq[16];        // (h/2) w_n / Mt: Gauss-Legendre weight on [-1, 1] times the panel and trapezoid factors
  const double* pts;
  const double* nrm;
  const double* jac;
  const double2* dens;
  const double* tgt;
  double2* out;
};

// |phase| below which the kernel's e^{i phase} goes through the double-word sin/cos
constexpr double kFieldDwMaxPhase = 4096.0;

// One CTA per evaluation point; threads over the surface nodes.  FP64 for the differences, rho^2,
// rsqrt and the phase; the sin/cos series, the kernel, its product with the density and the
// per-thread sums in double words (a thread adds about N / 256 terms, so the sloppy sums stay near
// 1e-13 of the sum of magnitudes); the block reduction in FP64.
__global__ void field_kernel(const FieldArgs a) {
  const int64_t p = blockIdx.x;
  const double x = a.tgt[3 * p], y = a.tgt[3 * p + 1], z = a.tgt[3 * p + 2];
  const float4 ceta = mkc(dw_from(0.0), dw_from(-a.eta));   // -i eta
  float4 acc = dwc_zero();
  double re = 0, im = 0;   // terms whose phase is beyond the double-word sin/cos range
  for (int64_t i = threadIdx.x; i < a.N; i += blockDim.x) {
    const int n = (int)((i / a.Mt) % 16);
    const double w = a.unweighted ? a.wq[n] * a.jac[i] : a.wq[n];
    const double yx = a.pts[3 * i], yy = a.pts[3 * i + 1], yz = a.pts[3 * i + 2];
    const double nx = a.nrm[3 * i], ny = a.nrm[3 * i + 1], nz = a.nrm[3 * i + 2];
    const double2 d = a.dens[i];
    if (!a.far) {
      const double dx = yx - x, dy = yy - y, dz = yz - z;
      const double r2 = dx * dx + dy * dy + dz * dz;
      const double rinv = rsqrt(r2);
      const double ph = a.k * (r2 * rinv);
      const double tau0 = a.rep == BIE_OP_S ? 0.0 : nx * dx + ny * dy + nz * dz;
      if (ph < kFieldDwMaxPhase) {
        float2 sn, cs;
        dw_sincos(ph, &sn, &cs);
        const float2 ri = dw_from(rinv);
        const float4 sl = mkc(dw_mul(cs, ri), dw_mul(sn, ri));   // e^{ik rho} / rho
        float4 kern = sl;
        if (a.rep != BIE_OP_S) {
          // tau0 / rho^3 e^{ik rho} (ik rho - 1)
          const float2 xd = dw_from(ph);
          const float2 f = dw_mul(dw_from(tau0), dw_mul(ri, dw_mul(ri, ri)));
          kern = dwc_mulr(mkc(dw_sub(dw_neg(cs), dw_mul(xd, sn)), dw_sub(dw_mul(xd, cs), sn)), f);
          if (a.rep == BIE_OP_CFIE) kern = dwc_add(kern, dwc_mul(ceta, sl));
        }
        acc = dwc_add(acc, dwc_mulr(dwc_mul(kern, dwc_from(C(d.x, d.y))), dw_from(w)));
        continue;
      }
      const double rho = r2 * rinv;
      const cplx e = cexpi(ph);
      const cplx sl = e * rinv;
      cplx kern = sl;
      if (a.rep != BIE_OP_S) {
        kern = (tau0 * rinv * rinv * rinv) * (e * C(-1.0, a.k * rho));
        if (a.rep == BIE_OP_CFIE) kern = kern + C(0.0, -a.eta) * sl;
      }
      const cplx v = w * (kern * C(d.x, d.y));
      re += v.re;
      im += v.im;
    } else {  // far-field pattern in direction (x, y, z) (unit vector)
      const double ph = -a.k * (x * yx + y * yy + z * yz);
      const double kn = -a.k * (x * nx + y * ny + z * nz);
      if (fabs(ph) < kFieldDwMaxPhase) {
        float2 sn, cs;
        dw_sincos(ph, &sn, &cs);
        const float4 e = mkc(cs, sn);
        float4 kern = e;
        if (a.rep != BIE_OP_S) {
          kern = dwc_mul(mkc(dw_from(0.0), dw_from(kn)), e);   // -i k (d . nu) e
          if (a.rep == BIE_OP_CFIE) kern = dwc_add(kern, dwc_mul(ceta, e));
        }
        acc = dwc_add(acc, dwc_mulr(dwc_mul(kern, dwc_from(C(d.x, d.y))), dw_from(w)));
        continue;
      }
      const cplx e = cexpi(ph);
      cplx kern = e;
      if (a.rep != BIE_OP_S) {
        kern = C(0.0, kn) * e;
        if (a.rep == BIE_OP_CFIE) kern = kern + C(0.0, -a.eta) * e;
      }
      const cplx v = w * (kern * C(d.x, d.y));
      re += v.re;
      im += v.im;
    }
  }
  re += dw_to(cre(acc));
  im += dw_to(cim(acc));
  for (int o = 16; o; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  __shared__ double sre[32], sim[32];
  if ((threadIdx.x & 31) == 0) { sre[threadIdx.x >> 5] = re; sim[threadIdx.x >> 5] = im; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0, m = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { r += sre[k]; m += sim[k]; }
    a.out[p] = make_double2(r, m);
  }
}

}  // namespace bie

using namespace bie;

extern "C" {

bie_status bie_rhs(bie_ctx ctx, bie_surface s, int kind, const double* param, double k, double* g) {
  if (!ctx || !s || !param || !g || kind < 0 || kind > 2) { set_error("bie_rhs: invalid arguments"); return BIE_EINVAL; }
  rhs_kernel<<<ctx->sms * 4, 256, 0, ctx->stream>>>(s->N, s->pts, s->nrm, kind, param[0], param[1], param[2], k,
                                                    (double2*)g);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BIE_OK : cuda_fail(e, "rhs_kernel");
}

bie_status bie_field_eval(bie_ctx ctx, bie_surface s, int rep_flags, double k, double eta, const double* density,
                          const double* pts, int64_t n, int far_field, double* out) {
  const int rep = rep_flags & ~BIE_UNWEIGHTED;
  if (!ctx || !s || !density || !pts || !out || n < 0 || n > (1 << 30) ||
      (rep != BIE_OP_S && rep != BIE_OP_K && rep != BIE_OP_CFIE)) {
    set_error("bie_field_eval: invalid arguments");
    return BIE_EINVAL;
  }
  if (n == 0) return BIE_OK;
  FieldArgs a;
  a.N = s->N;
  a.Mt = s->Mt;
  a.h = s->h;
  a.k = k;
  a.eta = eta;
  a.rep = rep;
  a.unweighted = (rep_flags & BIE_UNWEIGHTED) ? 1 : 0;
  a.jac = s->jac;
  a.far = far_field ? 1 : 0;
  for (int i = 0; i < 16; ++i) a.wq[i] = s->h * 0.5 * s->gl_w[i] / s->Mt;
  a.pts = s->pts;
  a.nrm = s->nrm;
  a.dens = (const double2*)density;
  a.tgt = pts;
  a.out = (double2*)out;
  field_kernel<<<(unsigned)n, 256, 0, ctx->stream>>>(a);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? BIE_OK : cuda_fail(e, "field_kernel");
}

}  // extern "C"
