// Double-word (float-float) arithmetic and a warp-cooperative FFT on it.
//
// A value is an unevaluated sum h + l of two floats with |l| <= ulp(h) / 2: 48 significant bits,
// relative rounding about 2^-48.  The FP32 pipe of this GPU runs about 70 times the FP64 rate, so
// the linear parts of the pair pipeline (FFTs, upsampling, products, unpacking) run in this
// format, and FP64 is kept for what needs its range or its elementary functions.
//
// Building blocks (Knuth's TwoSum; Dekker's FastTwoSum; the FMA form of TwoProd; the double-word
// sum and product as analysed by Joldes, Muller and Popescu, ACM TOMS 44(2), 2017):
//   two_sum       s + e = a + b exactly                                   (6 flops)
//   fast_two_sum  the same when |a| >= |b| or a = 0                        (3 flops)
//   dw_add        "sloppy" double-word sum: error <= ~2^-47 (|x| + |y|)    (11 flops)
//   dw_mul        double-word product, relative error <= ~5 2^-48          (7 flops)
//   dwc_mul       complex product with one renormalisation per component   (~36 flops)
// The sloppy sum has no bound relative to |x + y| under cancellation, but its error relative to
// |x| + |y| is what the normwise error analysis of an FFT uses.
// Complex values are float4 (re.h, re.l, im.h, im.l), 16 bytes, the size of a complex double.
#pragma once
#include <cuda_runtime.h>

#include "bie_internal.cuh"

namespace bie {

__device__ __forceinline__ float2 two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return make_float2(s, e);
}
__device__ __forceinline__ float2 fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return make_float2(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ float2 dw_add(float2 x, float2 y) {
  const float2 s = two_sum(x.x, y.x);
  return fast_two_sum(s.x, __fadd_rn(s.y, __fadd_rn(x.y, y.y)));
}
__device__ __forceinline__ float2 dw_neg(float2 x) { return make_float2(-x.x, -x.y); }
__device__ __forceinline__ float2 dw_sub(float2 x, float2 y) { return dw_add(x, dw_neg(y)); }
__device__ __forceinline__ float2 dw_mul(float2 x, float2 y) {
  const float p = __fmul_rn(x.x, y.x);
  float e = fmaf(x.x, y.x, -p);
  e = fmaf(x.x, y.y, e);
  e = fmaf(x.y, y.x, e);
  return fast_two_sum(p, e);
}
__device__ __forceinline__ float2 dw_scale2(float2 x, float s) {   // s a power of two: exact
  return make_float2(x.x * s, x.y * s);
}
__device__ __forceinline__ float2 dw_from(double v) {
  const float h = __double2float_rn(v);
  return make_float2(h, __double2float_rn(v - (double)h));
}
__device__ __forceinline__ double dw_to(float2 a) { return (double)a.x + (double)a.y; }

// complex helpers on float4 = (re.h, re.l, im.h, im.l)
__device__ __forceinline__ float2 cre(float4 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ float2 cim(float4 a) { return make_float2(a.z, a.w); }
__device__ __forceinline__ float4 mkc(float2 re, float2 im) { return make_float4(re.x, re.y, im.x, im.y); }
__device__ __forceinline__ float4 dwc_add(float4 a, float4 b) { return mkc(dw_add(cre(a), cre(b)), dw_add(cim(a), cim(b))); }
__device__ __forceinline__ float4 dwc_sub(float4 a, float4 b) { return mkc(dw_sub(cre(a), cre(b)), dw_sub(cim(a), cim(b))); }
__device__ __forceinline__ float4 dwc_conj(float4 a) { return make_float4(a.x, a.y, -a.z, -a.w); }
__device__ __forceinline__ float4 dwc_scale2(float4 a, float s) { return make_float4(a.x * s, a.y * s, a.z * s, a.w * s); }
__device__ __forceinline__ float4 dwc_from(cplx v) { return mkc(dw_from(v.re), dw_from(v.im)); }
__device__ __forceinline__ cplx dwc_to(float4 a) { return C(dw_to(cre(a)), dw_to(cim(a))); }
__device__ __forceinline__ float4 dwc_zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }

// x * y (complex): each component is sum of two exact products (TwoProd) and their low-order
// cross terms, renormalised once
__device__ __forceinline__ float4 dwc_mul(float4 x, float4 y) {
  float2 re, im;
  {
    const float p1 = __fmul_rn(x.x, y.x), e1 = fmaf(x.x, y.x, -p1);
    const float p2 = __fmul_rn(x.z, y.z), e2 = fmaf(x.z, y.z, -p2);
    const float2 s = two_sum(p1, -p2);
    float c = __fadd_rn(s.y, __fsub_rn(e1, e2));
    c = fmaf(x.x, y.y, c);
    c = fmaf(x.y, y.x, c);
    c = fmaf(-x.z, y.w, c);
    c = fmaf(-x.w, y.z, c);
    re = two_sum(s.x, c);
  }
  {
    const float p1 = __fmul_rn(x.x, y.z), e1 = fmaf(x.x, y.z, -p1);
    const float p2 = __fmul_rn(x.z, y.x), e2 = fmaf(x.z, y.x, -p2);
    const float2 s = two_sum(p1, p2);
    float c = __fadd_rn(s.y, __fadd_rn(e1, e2));
    c = fmaf(x.x, y.w, c);
    c = fmaf(x.y, y.z, c);
    c = fmaf(x.z, y.y, c);
    c = fmaf(x.w, y.x, c);
    im = two_sum(s.x, c);
  }
  return mkc(re, im);
}
// complex times real double-word
__device__ __forceinline__ float4 dwc_mulr(float4 x, float2 r) { return mkc(dw_mul(cre(x), r), dw_mul(cim(x), r)); }

// ------------------------------------------------------------------ warp FFT
// Same transform and buffer contract as warp_fft (Stockham, radices 4, 2, 3; the result lands in
// x or y, returned), on double-word complex values; tw: the twiddle table e^{-2 pi i k / T} in
// double-word form.
__device__ __forceinline__ float4 tw_load(const float4* __restrict__ tw, int idx, int sign) {
  const float4 w = __ldg(tw + idx);
  return sign > 0 ? dwc_conj(w) : w;
}
__device__ __forceinline__ float4 mul_i(float4 a, int sign) {   // sign * i * a
  return sign < 0 ? make_float4(a.z, a.w, -a.x, -a.y) : make_float4(-a.z, -a.w, a.x, a.y);
}

static __device__ __noinline__ float4* warp_fft_dw(float4* x, float4* y, int n, const float4* __restrict__ tw, int T,
                                                   int sign) {
  const int lane = threadIdx.x & 31;
  const FFTPlan p = make_plan(n);
  float4* src = x;
  float4* dst = y;
  int Ns = 1;
  // sign * sqrt(3)/2 as a double word
  const float2 s3 = make_float2(sign * 0.8660253882408142f, sign * 1.5543625053737742e-08f);
  for (int st = 0; st < p.nst; ++st) {
    const int R = p.rad[st];
    const int stride = n / R;
    const int tstep = (T / n) * (n / (Ns * R));   // r * jm * tstep < T
    if (R == 4) {
      for (int j = lane; j < stride; j += 32) {
        const int jm = j % Ns;
        float4 v0 = src[j], v1 = src[j + stride], v2 = src[j + 2 * stride], v3 = src[j + 3 * stride];
        if (jm) {
          v1 = dwc_mul(v1, tw_load(tw, jm * tstep, sign));
          v2 = dwc_mul(v2, tw_load(tw, 2 * jm * tstep, sign));
          v3 = dwc_mul(v3, tw_load(tw, 3 * jm * tstep, sign));
        }
        const float4 s02 = dwc_add(v0, v2), d02 = dwc_sub(v0, v2), s13 = dwc_add(v1, v3);
        const float4 jd = mul_i(dwc_sub(v1, v3), sign);
        const int idx = (j / Ns) * Ns * 4 + jm;
        dst[idx] = dwc_add(s02, s13);
        dst[idx + Ns] = dwc_add(d02, jd);
        dst[idx + 2 * Ns] = dwc_sub(s02, s13);
        dst[idx + 3 * Ns] = dwc_sub(d02, jd);
      }
    } else if (R == 2) {
      for (int j = lane; j < stride; j += 32) {
        const int jm = j % Ns;
        const float4 v0 = src[j];
        float4 v1 = src[j + stride];
        if (jm) v1 = dwc_mul(v1, tw_load(tw, jm * tstep, sign));
        const int idx = (j / Ns) * Ns * 2 + jm;
        dst[idx] = dwc_add(v0, v1);
        dst[idx + Ns] = dwc_sub(v0, v1);
      }
    } else {
      for (int j = lane; j < stride; j += 32) {
        const int jm = j % Ns;
        const float4 v0 = src[j];
        float4 v1 = src[j + stride], v2 = src[j + 2 * stride];
        if (jm) {
          v1 = dwc_mul(v1, tw_load(tw, jm * tstep, sign));
          v2 = dwc_mul(v2, tw_load(tw, 2 * jm * tstep, sign));
        }
        const float4 t1 = dwc_add(v1, v2), d = dwc_sub(v1, v2);
        // t2 = s3 * i * d (s3 carries the sign)
        const float4 t2 = mkc(dw_neg(dw_mul(s3, cim(d))), dw_mul(s3, cre(d)));
        const float4 base = dwc_sub(v0, dwc_scale2(t1, 0.5f));
        const int idx = (j / Ns) * Ns * 3 + jm;
        dst[idx] = dwc_add(v0, t1);
        dst[idx + Ns] = dwc_add(base, t2);
        dst[idx + 2 * Ns] = dwc_sub(base, t2);
      }
    }
    __syncwarp();
    float4* tmp = src;
    src = dst;
    dst = tmp;
    Ns *= R;
  }
  return src;
}

}  // namespace bie
