// Surface sampling (Section 2, Eq. (para); Section 3.1 panels and GGQ rings).
#include <cmath>
#include <cstring>
#include <vector>

#include "bie_internal.cuh"

namespace bie {

// Collocation grid: N = 16 Np Mt nodes; position, unit normal, Jacobian.
__global__ void sample_grid_kernel(SurfP S, const double* __restrict__ t_nodes, int Mt, int64_t N,
                                   double* __restrict__ pts, double* __restrict__ nrm, double* __restrict__ jac) {
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < N; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t tn = idx / Mt;
    const int i = (int)(idx % Mt);
    Geo g;
    surf_eval(S, t_nodes[tn], kTwoPi * i / Mt, 1, &g);
    R3 n = cross(g.rt, g.rth);
    const double J = sqrt(dot(n, n));
    pts[3 * idx + 0] = g.r.x; pts[3 * idx + 1] = g.r.y; pts[3 * idx + 2] = g.r.z;
    nrm[3 * idx + 0] = n.x / J; nrm[3 * idx + 1] = n.y / J; nrm[3 * idx + 2] = n.z / J;
    jac[idx] = J;
  }
}

// GGQ source rings: ring (target node tn, d, g) at t_s = ring_t[ring], Mt angles.
__global__ void sample_rings_kernel(SurfP S, const double* __restrict__ ring_t, int Mt, int64_t n_rings,
                                    double* __restrict__ rr, double* __restrict__ rn) {
  const int64_t total = n_rings * Mt;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total; idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ring = idx / Mt;
    const int q = (int)(idx % Mt);
    const double ts = ring_t[ring];
    if (!(ts == ts)) {  // ring of a panel that does not exist
      for (int c = 0; c < 3; ++c) { rr[3 * idx + c] = 0.0; rn[3 * idx + c] = 0.0; }
      continue;
    }
    Geo g;
    surf_eval(S, ts, kTwoPi * q / Mt, 1, &g);
    R3 n = cross(g.rt, g.rth);
    const double J = sqrt(dot(n, n));
    rr[3 * idx + 0] = g.r.x; rr[3 * idx + 1] = g.r.y; rr[3 * idx + 2] = g.r.z;
    rn[3 * idx + 0] = n.x / J; rn[3 * idx + 1] = n.y / J; rn[3 * idx + 2] = n.z / J;
  }
}

static bool valid_length(int Mt) {
  if (Mt < 8 || Mt > 1024 || (Mt & 1)) return false;
  int m = Mt;
  while (m % 2 == 0) m /= 2;
  while (m % 3 == 0) m /= 3;
  while (m % 5 == 0) m /= 5;
  return m == 1;
}

}  // namespace bie

using namespace bie;

extern "C" {

bie_status bie_surface_sample(bie_ctx ctx, const bie_surface_desc* desc, int Np, int Mt,
                              const bie_quad_tables* ggq, bie_surface* out) {
  if (!ctx || !desc || !ggq || !out) { set_error("bie_surface_sample: NULL argument"); return BIE_EINVAL; }
  if (Np < 2 || Np > 4096) { set_error("bie_surface_sample: n_panels %d out of [2, 4096]", Np); return BIE_EINVAL; }
  if (!valid_length(Mt)) { set_error("bie_surface_sample: m_theta %d must be even, 2^a 3^b 5^c, in [8, 1024]", Mt); return BIE_EINVAL; }
  if (desc->kind < 0 || desc->kind > 4) { set_error("bie_surface_sample: unknown kind %d", desc->kind); return BIE_EINVAL; }
  const bool with_terms = desc->kind == 1 || desc->kind == 3 || desc->kind == 4;
  if (with_terms && (desc->n_terms < 0 || desc->n_terms > BIE_MAX_TERMS || (desc->n_terms && !desc->terms))) {
    set_error("bie_surface_sample: n_terms %d out of [0, %d]", desc->n_terms, BIE_MAX_TERMS);
    return BIE_EINVAL;
  }
  if (desc->kind == 3 && desc->n_terms != 1) { set_error("bie_surface_sample: the torus takes one term (R, eps, m)"); return BIE_EINVAL; }
  const bool periodic = desc->kind == 3 || desc->kind == 4;
  if (periodic && Np < 3) { set_error("bie_surface_sample: a torus needs n_panels >= 3"); return BIE_EINVAL; }
  {
    // non-finite descriptor values or tables would sample NaN geometry: refuse them here
    bool finite = true;
    for (int c = 0; c < 3; ++c) finite = finite && std::isfinite(desc->axes[c]);
    if (with_terms)
      for (int i = 0; i < 5 * desc->n_terms; ++i) finite = finite && std::isfinite(desc->terms[i]);
    for (int i = 0; i < 3 * 16 * 16; ++i)
      finite = finite && std::isfinite((&ggq->x[0][0][0])[i]) && std::isfinite((&ggq->w[0][0][0])[i]);
    if (!finite) { set_error("bie_surface_sample: NaN or Inf in the surface descriptor or the quadrature tables"); return BIE_ENAN; }
  }
  {
    const bie_status ds = check_device(ctx, "bie_surface_sample");
    if (ds != BIE_OK) return ds;
  }
  bie_surface s = new bie_surface_s();
  memset(&s->sp, 0, sizeof(s->sp));
  s->ctx = ctx;
  s->sp.kind = desc->kind;
  s->sp.ax = desc->axes[0]; s->sp.ay = desc->axes[1]; s->sp.az = desc->axes[2];
  s->sp.periodic = periodic ? 1 : 0;
  s->sp.L = periodic ? 2 * kPi : kPi;
  if (desc->kind == 3) {
    s->sp.R = desc->terms[0];
    s->sp.eps = desc->terms[1];
    s->sp.mm = (int)lrint(desc->terms[2]);
    if (fabs(desc->terms[2]) > 100) { delete s; set_error("bie_surface_sample: torus m out of range"); return BIE_EINVAL; }
  }
  if (desc->kind == 4) {
    s->sp.R = desc->axes[0];
    s->sp.nt = desc->n_terms;
    for (int i = 0; i < desc->n_terms; ++i) {
      const double* tr = desc->terms + 5 * i;
      if (fabs(tr[1]) > 100 || fabs(tr[2]) > 100) { delete s; set_error("bie_surface_sample: term %d out of range", i); return BIE_EINVAL; }
      s->sp.c[i] = tr[0];
      s->sp.m[i] = (int8_t)lrint(tr[1]);   // theta frequency
      s->sp.q[i] = (int8_t)lrint(tr[2]);   // t frequency
    }
  }
  if (desc->kind == 1) {
    s->sp.nt = desc->n_terms;
    for (int i = 0; i < desc->n_terms; ++i) {
      const double* tr = desc->terms + 5 * i;
      s->sp.c[i] = tr[0];
      s->sp.p[i] = (int8_t)lrint(tr[1]);
      s->sp.q[i] = (int8_t)lrint(tr[2]);
      s->sp.m[i] = (int8_t)lrint(tr[3]);
      s->sp.s[i] = (int8_t)lrint(tr[4]);
      if (tr[1] < 0 || tr[2] < 0 || tr[3] < 0 || tr[1] > 40 || tr[2] > 40 || tr[3] > 100) {
        delete s;
        set_error("bie_surface_sample: term %d has exponents out of range", i);
        return BIE_EINVAL;
      }
    }
  }
  s->Np = Np;
  s->Mt = Mt;
  s->L = s->sp.L;
  s->h = s->L / Np;
  s->N = (int64_t)16 * Np * Mt;
  s->n_rings = (int64_t)16 * Np * 48;
  // Gauss-Legendre rule from the tables: validate, keep, map to [0, 1]
  {
    double wsum = 0.0;
    for (int l = 0; l < 16; ++l) {
      wsum += ggq->gl_w[l];
      if (!(ggq->gl_x[l] > -1.0 && ggq->gl_x[l] < 1.0) || !(ggq->gl_w[l] > 0) ||
          (l && !(ggq->gl_x[l] > ggq->gl_x[l - 1]))) {
        delete s;
        set_error("bie_surface_sample: Gauss-Legendre table is not an ascending rule on (-1, 1)");
        return BIE_EINVAL;
      }
      s->gl_x[l] = ggq->gl_x[l];
      s->gl_w[l] = ggq->gl_w[l];
      s->gl01.x[l] = (ggq->gl_x[l] + 1) / 2;
      s->gl01.w[l] = ggq->gl_w[l] / 2;
    }
    s->sp.gl = s->gl01;
    if (fabs(wsum - 2.0) > 1e-13) {
      delete s;
      set_error("bie_surface_sample: Gauss-Legendre weights do not sum to 2");
      return BIE_EINVAL;
    }
  }
  std::vector<double> tn(16 * Np), rt(s->n_rings);
  for (int j = 0; j < Np; ++j)
    for (int l = 0; l < 16; ++l) tn[j * 16 + l] = (j + 0.5) * s->h + (s->h / 2) * s->gl_x[l];
  for (int j = 0; j < Np; ++j)
    for (int l = 0; l < 16; ++l)
      for (int d = 0; d < 3; ++d)
        for (int g = 0; g < 16; ++g) {
          const int ip = j + d - 1;   // past an end of a torus: the last / first panel, shifted by -L / +L
          const int64_t ring = (((int64_t)(j * 16 + l) * 3 + d) * 16 + g);
          rt[ring] = (!periodic && (ip < 0 || ip >= Np)) ? NAN : (ip + 0.5) * s->h + (s->h / 2) * ggq->x[d][l][g];
        }
  // near-fill coefficients w_g L_n(x_g) (Lagrange basis on the 16 Legendre nodes)
  std::vector<double> coef(3 * 16 * 16 * 16);
  for (int d = 0; d < 3; ++d)
    for (int l = 0; l < 16; ++l)
      for (int g = 0; g < 16; ++g) {
        const double x = ggq->x[d][l][g];
        for (int n = 0; n < 16; ++n) {
          double Ln = 1.0;
          const double xn = s->gl_x[n];
          for (int m = 0; m < 16; ++m)
            if (m != n) Ln *= (x - s->gl_x[m]) / (xn - s->gl_x[m]);
          coef[((d * 16 + l) * 16 + g) * 16 + n] = ggq->w[d][l][g] * Ln;
        }
      }
  std::vector<float2> coefw(coef.size());   // the same as double words
  for (size_t e = 0; e < coef.size(); ++e) {
    const float h = (float)coef[e];
    coefw[e] = make_float2(h, (float)(coef[e] - (double)h));
  }
  // twiddles for length 12 Mt
  const int T = 12 * Mt;
  std::vector<cplx> tw(T);
  std::vector<float4> twf(T);   // the same table as double words (h + l, rounded from long double)
  for (int k = 0; k < T; ++k) {
    long double a = -2.0L * 3.14159265358979323846264338327950288L * k / T;
    const long double c = cosl(a), sn = sinl(a);
    tw[k] = C((double)c, (double)sn);
    const float ch = (float)c, sh = (float)sn;
    twf[k] = make_float4(ch, (float)(c - (long double)ch), sh, (float)(sn - (long double)sh));
  }
  s->tw_len = T;
  std::vector<double> thg(3 * Mt);
  for (int q = 0; q < Mt; ++q) {
    const double th = kTwoPi * q / Mt;
    thg[3 * q] = th;
    thg[3 * q + 1] = sin(0.5 * th);
    thg[3 * q + 2] = cos(0.5 * th);
  }
  s->host_t_nodes = new double[16 * Np];
  memcpy(s->host_t_nodes, tn.data(), sizeof(double) * 16 * Np);
  cudaError_t e;
  const size_t N = s->N;
#define ALLOC(ptr, bytes)                                   \
  e = cudaMalloc((void**)&(ptr), (bytes));                  \
  if (e != cudaSuccess) { bie_surface_free(s); return cuda_fail(e, "cudaMalloc(surface)"); }
  ALLOC(s->t_nodes, sizeof(double) * 16 * Np);
  ALLOC(s->pts, sizeof(double) * 3 * N);
  ALLOC(s->nrm, sizeof(double) * 3 * N);
  ALLOC(s->jac, sizeof(double) * N);
  ALLOC(s->ring_t, sizeof(double) * s->n_rings);
  ALLOC(s->ring_r, sizeof(double) * 3 * s->n_rings * Mt);
  ALLOC(s->ring_n, sizeof(double) * 3 * s->n_rings * Mt);
  ALLOC(s->near_coef, sizeof(double) * coef.size());
  ALLOC(s->near_coef_dw, sizeof(float2) * coef.size());
  ALLOC(s->ggq_x, sizeof(double) * 3 * 16 * 16);
  ALLOC(s->tw, sizeof(cplx) * T);
  ALLOC(s->twf, sizeof(float4) * T);
  ALLOC(s->thgrid, sizeof(double) * 3 * Mt);
#undef ALLOC
  cudaStream_t st = ctx->stream;
#define H2D(dst, src, bytes)                                                          \
  e = cudaMemcpyAsync((dst), (src), (bytes), cudaMemcpyHostToDevice, st);             \
  if (e != cudaSuccess) { bie_surface_free(s); return cuda_fail(e, "cudaMemcpyAsync(surface)"); }
  H2D(s->t_nodes, tn.data(), sizeof(double) * 16 * Np);
  H2D(s->ring_t, rt.data(), sizeof(double) * s->n_rings);
  H2D(s->near_coef, coef.data(), sizeof(double) * coef.size());
  H2D(s->near_coef_dw, coefw.data(), sizeof(float2) * coefw.size());
  H2D(s->ggq_x, &ggq->x[0][0][0], sizeof(double) * 3 * 16 * 16);
  H2D(s->tw, tw.data(), sizeof(cplx) * T);
  H2D(s->twf, twf.data(), sizeof(float4) * T);
  H2D(s->thgrid, thg.data(), sizeof(double) * 3 * Mt);
#undef H2D
  const int threads = 256;
  const int blocks = ctx->sms * 8;
  sample_grid_kernel<<<blocks, threads, 0, st>>>(s->sp, s->t_nodes, Mt, s->N, s->pts, s->nrm, s->jac);
  sample_rings_kernel<<<blocks, threads, 0, st>>>(s->sp, s->ring_t, Mt, s->n_rings, s->ring_r, s->ring_n);
  e = cudaGetLastError();
  if (e != cudaSuccess) { bie_surface_free(s); return cuda_fail(e, "sample kernels"); }
  // the host vectors die at return: make the copies complete first
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { bie_surface_free(s); return cuda_fail(e, "bie_surface_sample sync"); }
  *out = s;
  return BIE_OK;
}

void bie_surface_free(bie_surface s) {
  if (!s) return;
  cudaFree(s->t_nodes); cudaFree(s->pts); cudaFree(s->nrm); cudaFree(s->jac);
  cudaFree(s->ring_t); cudaFree(s->ring_r); cudaFree(s->ring_n);
  cudaFree(s->near_coef); cudaFree(s->near_coef_dw); cudaFree(s->ggq_x); cudaFree(s->tw); cudaFree(s->twf); cudaFree(s->thgrid);
  delete[] s->host_t_nodes;
  delete s;
}

int64_t bie_surface_unknowns(bie_surface s) { return s ? s->N : 0; }
int64_t bie_surface_near_pairs(bie_surface s) {
  return s ? (int64_t)256 * s->Mt * (3 * s->Np - (s->sp.periodic ? 0 : 2)) : 0;
}
const double* bie_surface_points(bie_surface s) { return s ? s->pts : nullptr; }
const double* bie_surface_normals(bie_surface s) { return s ? s->nrm : nullptr; }
const double* bie_surface_jacobians(bie_surface s) { return s ? s->jac : nullptr; }

}  // extern "C"
