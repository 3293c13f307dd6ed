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
// double -> double word by splitting the significand with integer operations (the FP32 <-> FP64
// conversion instructions run on the narrow FP64 pipe): h = the top 24 significand bits (truncated),
// l = the remaining 29 bits rounded to a float, same sign.  Outside 2^-126 .. 2^115 plain conversions.
__device__ __forceinline__ float2 dw_from(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7ff);
  if (e < 897 || e > 1138) {
    const float h = __double2float_rn(v);
    return make_float2(h, __double2float_rn(v - (double)h));
  }
  const unsigned sgn = (unsigned)(b >> 32) & 0x80000000u;
  const float h = __uint_as_float(sgn | ((unsigned)(e - 896) << 23) | (unsigned)((b >> 29) & 0x7fffffu));
  // the 29-bit remainder r as a float, rounded to nearest, with FP32 instructions only (an integer
  // conversion instruction would run on the FP64 pipe): r = 64 rh + rl with rh < 2^23 and rl < 64 are
  // exact floats by the 2^23 bias trick, and one FMA rounds 64 rh + rl once
  const unsigned r = (unsigned)(b & 0x1fffffffu);
  const float fh = __uint_as_float(0x4B000000u | (r >> 6)) - 8388608.0f;
  const float fl = __uint_as_float(0x4B000000u | (r & 63u)) - 8388608.0f;
  const float rest = fmaf(fh, 64.0f, fl);
  const float l = (__uint_as_float(sgn | __float_as_uint(rest)) * 5.421010862427522e-20f)   // * 2^-64
                  * __uint_as_float((unsigned)(e - 884) << 23);                            // * 2^(e - 1011)
  return make_float2(h, l);
}
// float -> double exactly from the bit pattern (zero and subnormal floats give a signed zero)
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned ef = (u >> 23) & 0xffu;
  if (ef == 0xffu) return (double)f;
  const unsigned long long sg = (unsigned long long)(u & 0x80000000u) << 32;
  if (ef == 0) return __longlong_as_double((long long)sg);
  return __longlong_as_double((long long)(sg | ((unsigned long long)(ef + 896) << 52) |
                                          ((unsigned long long)(u & 0x7fffffu) << 29)));
}
__device__ __forceinline__ double dw_to(float2 a) { return f2d_bits(a.x) + f2d_bits(a.y); }

// sqrt of a double word a >= 0 (Dekker's double-length square root, Numer. Math. 18, 1971): s =
// sqrt(h) in FP32, then one Newton step on the residual a - s^2 with s^2 = p + e exact by FMA (h - p
// is exact: p is within a few ulps of h); about 2^-47 relative.
__device__ __forceinline__ float2 dw_sqrt(float2 a) {
  if (!(a.x > 0.f)) return make_float2(0.f, 0.f);
  const float s = __fsqrt_rn(a.x);
  const float p = __fmul_rn(s, s);
  const float e = fmaf(s, s, -p);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.x, p), e), a.y);
  return fast_two_sum(s, __fdividef(r, 2.f * s));
}

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

// ------------------------------------------------------------------ sin and cos
// sin x, cos x for |x| < 1e4 (FP64 argument): Cody-Waite reduction by pi/2 in FP64 (two-part constant
// with FMA: r = x - n pi/2 to about 1e-16 absolute), then the Taylor series of sin r / r and cos r in
// r^2 for |r| <= pi/4: the terms r^10 .. r^16 (below 2.3e-9) in FP32, the leading five in double
// words.  Absolute error about 1e-14.
__device__ __forceinline__ void dw_sincos(double x, float2* sn, float2* cs) {
  const double n = rint(x * 0.63661977236758138);
  double r = fma(-n, 1.5707963267948966, x);
  r = fma(-n, 6.123233995736766e-17, r);
  const float2 rw = dw_from(r);
  const float2 r2 = dw_mul(rw, rw);
  const float xf = r2.x;
  // (-1)^k / (2k+1)! and (-1)^k / (2k)!, k = 5..8 (FP32) and k = 0..4 (double words)
  float ts = fmaf(fmaf(fmaf(2.8114573589663704e-15f, xf, -7.647163609812713e-13f), xf, 1.6059044372074283e-10f), xf,
                  -2.5052107943679403e-08f);
  float tc = fmaf(fmaf(fmaf(4.7794772561329454e-14f, xf, -1.147074536050896e-11f), xf, 2.0876755879584152e-09f), xf,
                  -2.755731998149713e-07f);
  float2 ps = make_float2(ts, 0.f), pc = make_float2(tc, 0.f);
  ps = dw_add(dw_mul(ps, r2), make_float2(2.7557318844628753e-06f, 3.793571224297229e-14f));
  pc = dw_add(dw_mul(pc, r2), make_float2(2.4801587642286904e-05f, -3.40699609366682e-13f));
  ps = dw_add(dw_mul(ps, r2), make_float2(-0.00019841270113829523f, 2.725596874933456e-12f));
  pc = dw_add(dw_mul(pc, r2), make_float2(-0.0013888889225199819f, 3.3631094437103215e-11f));
  ps = dw_add(dw_mul(ps, r2), make_float2(0.008333333767950535f, -4.34617203337595e-10f));
  pc = dw_add(dw_mul(pc, r2), make_float2(0.0416666679084301f, -1.2417634698280722e-09f));
  ps = dw_add(dw_mul(ps, r2), make_float2(-0.1666666716337204f, 4.967053879312289e-09f));
  pc = dw_add(dw_mul(pc, r2), make_float2(-0.5f, 0.f));
  ps = dw_add(dw_mul(ps, r2), make_float2(1.f, 0.f));
  pc = dw_add(dw_mul(pc, r2), make_float2(1.f, 0.f));
  const float2 sr = dw_mul(ps, rw);
  switch ((int)n & 3) {
    case 0: *sn = sr; *cs = pc; break;
    case 1: *sn = pc; *cs = dw_neg(sr); break;
    case 2: *sn = dw_neg(sr); *cs = dw_neg(pc); break;
    default: *sn = dw_neg(pc); *cs = sr; break;
  }
}

// ------------------------------------------------------------------ warp FFT
// Same transform and buffer contract as warp_fft (Stockham, radices 4, 2, 3, 5; the result lands in
// x or y, returned), on double-word complex values; tw: the twiddle table e^{-2 pi i k / T} in
// double-word form.
__device__ __forceinline__ float4 tw_load(const float4* __restrict__ tw, int idx, int sign) {
  const float4 w = __ldg(tw + idx);
  return sign > 0 ? dwc_conj(w) : w;
}
__device__ __forceinline__ float4 mul_i(float4 a, int sign) {   // sign * i * a
  return sign < 0 ? make_float4(a.z, a.w, -a.x, -a.y) : make_float4(-a.z, -a.w, a.x, a.y);
}

// j = q Ns + jm: by shift and mask when Ns is a power of two (every stage of the power-of-two
// plans), by division otherwise
struct StageIdx {
  int Ns, sh;   // sh >= 0: Ns = 2^sh
  __device__ __forceinline__ int rem(int j) const { return sh >= 0 ? (j & (Ns - 1)) : j % Ns; }
  __device__ __forceinline__ int quo(int j) const { return sh >= 0 ? (j >> sh) : j / Ns; }
};

// st0 > 0: the first st0 stages are done (x holds their output).
static __device__ __noinline__ float4* warp_fft_dw(float4* x, float4* y, int n, const float4* __restrict__ tw, int T,
                                                   int sign, int st0 = 0) {
  const int lane = threadIdx.x & 31;
  const FFTPlan p = make_plan(n);
  float4* src = x;
  float4* dst = y;
  int Ns = 1;
  for (int st = 0; st < st0; ++st) Ns *= p.rad[st];
  // sign * sqrt(3)/2 as a double word
  const float2 s3 = make_float2(sign * 0.8660253882408142f, sign * 1.5543625053737742e-08f);
  for (int st = st0; st < p.nst; ++st) {
    const int R = p.rad[st];
    const int stride = n / R;
    const int tstep = (T / n) * (n / (Ns * R));   // r * jm * tstep < T
    const StageIdx ix = {Ns, (Ns & (Ns - 1)) == 0 ? __ffs(Ns) - 1 : -1};
    if (R == 4) {
      for (int j = lane; j < stride; j += 32) {
        const int jm = ix.rem(j);
        float4 v0 = src[j], v1 = src[j + stride], v2 = src[j + 2 * stride], v3 = src[j + 3 * stride];
        if (jm) {
          v1 = dwc_mul(v1, tw_load(tw, jm * tstep, sign));
          v2 = dwc_mul(v2, tw_load(tw, 2 * jm * tstep, sign));
          v3 = dwc_mul(v3, tw_load(tw, 3 * jm * tstep, sign));
        }
        const float4 s02 = dwc_add(v0, v2), d02 = dwc_sub(v0, v2), s13 = dwc_add(v1, v3);
        const float4 jd = mul_i(dwc_sub(v1, v3), sign);
        const int idx = ix.quo(j) * Ns * 4 + jm;
        dst[idx] = dwc_add(s02, s13);
        dst[idx + Ns] = dwc_add(d02, jd);
        dst[idx + 2 * Ns] = dwc_sub(s02, s13);
        dst[idx + 3 * Ns] = dwc_sub(d02, jd);
      }
    } else if (R == 2) {
      for (int j = lane; j < stride; j += 32) {
        const int jm = ix.rem(j);
        const float4 v0 = src[j];
        float4 v1 = src[j + stride];
        if (jm) v1 = dwc_mul(v1, tw_load(tw, jm * tstep, sign));
        const int idx = ix.quo(j) * Ns * 2 + jm;
        dst[idx] = dwc_add(v0, v1);
        dst[idx + Ns] = dwc_sub(v0, v1);
      }
    } else if (R == 5) {
      // cos and sin of 2 pi / 5 and 4 pi / 5 as double words (the sines carry the sign)
      const float2 c1 = make_float2(0.30901700258255005f, -8.207602597565256e-09f);
      const float2 c2 = make_float2(-0.80901700258255f, 8.207602597565256e-09f);
      const float2 s1 = make_float2(sign * 0.9510565400123596f, sign * -2.3717205976936384e-08f);
      const float2 s2 = make_float2(sign * 0.5877852439880371f, sign * 8.304436249773062e-09f);
      for (int j = lane; j < stride; j += 32) {
        const int jm = ix.rem(j);
        const float4 v0 = src[j];
        float4 v1 = src[j + stride], v2 = src[j + 2 * stride], v3 = src[j + 3 * stride], v4 = src[j + 4 * stride];
        if (jm) {
          v1 = dwc_mul(v1, tw_load(tw, jm * tstep, sign));
          v2 = dwc_mul(v2, tw_load(tw, 2 * jm * tstep, sign));
          v3 = dwc_mul(v3, tw_load(tw, 3 * jm * tstep, sign));
          v4 = dwc_mul(v4, tw_load(tw, 4 * jm * tstep, sign));
        }
        const float4 t1 = dwc_add(v1, v4), t2 = dwc_add(v2, v3), t3 = dwc_sub(v1, v4), t4 = dwc_sub(v2, v3);
        const float4 a1 = dwc_add(v0, dwc_add(dwc_mulr(t1, c1), dwc_mulr(t2, c2)));
        const float4 a2 = dwc_add(v0, dwc_add(dwc_mulr(t1, c2), dwc_mulr(t2, c1)));
        const float4 b1 = dwc_add(dwc_mulr(t3, s1), dwc_mulr(t4, s2));
        const float4 b2 = dwc_sub(dwc_mulr(t3, s2), dwc_mulr(t4, s1));
        const float4 ib1 = make_float4(-b1.z, -b1.w, b1.x, b1.y), ib2 = make_float4(-b2.z, -b2.w, b2.x, b2.y);
        const int idx = ix.quo(j) * Ns * 5 + jm;
        dst[idx] = dwc_add(v0, dwc_add(t1, t2));
        dst[idx + Ns] = dwc_add(a1, ib1);
        dst[idx + 2 * Ns] = dwc_add(a2, ib2);
        dst[idx + 3 * Ns] = dwc_sub(a2, ib2);
        dst[idx + 4 * Ns] = dwc_sub(a1, ib1);
      }
    } else {
      for (int j = lane; j < stride; j += 32) {
        const int jm = ix.rem(j);
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
        const int idx = ix.quo(j) * Ns * 3 + jm;
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
