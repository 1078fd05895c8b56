// Arithmetic of the Bluestein FFT passes: FP64 complex, or "double-float"
// complex (every real part held as an unevaluated sum hi + lo of two FP32
// numbers, about 48 significant bits) computed with error-free transformations
// on the FP32 pipes:
//   two-sum (Knuth, TAOCP vol. 2, 4.2.2) and fast-two-sum (Dekker 1971) for
//   sums, the fused multiply-add form of Dekker's exact product for products,
//   following the double-word algorithms of Joldes, Muller and Popescu
//   ("Tight and rigorous error bounds for basic building blocks of
//   double-word arithmetic", ACM TOMS 2017).
// Inside a butterfly the sums are left unnormalised (the error of the high
// parts is kept exactly, the low parts added in FP32) and renormalised once
// when a value is stored, which keeps the normwise error at about 2^-48 and
// saves a fast-two-sum per addition.
// Every FP32 operation below uses a round-to-nearest intrinsic, which the
// compiler never contracts or reassociates, so the transformations stay exact.
#pragma once

#include "common.cuh"

namespace mr1l {

// FP64 complex in registers and memory (double2).
struct OpsF64 {
  typedef cplx V;
  static __device__ __forceinline__ V zero() { return cmake(0.0, 0.0); }
  static __device__ __forceinline__ V add(V a, V b) { return cadd(a, b); }
  static __device__ __forceinline__ V sub(V a, V b) { return csub(a, b); }
  static __device__ __forceinline__ V mul(V a, V b) { return cmul(a, b); }
  static __device__ __forceinline__ V mulc(V a, V b) { return cmulc(a, b); }
  // acc + a * b as four FMAs
  static __device__ __forceinline__ V mac(V acc, V a, V b) {
    return cmake(fma(a.x, b.x, fma(-a.y, b.y, acc.x)), fma(a.x, b.y, fma(a.y, b.x, acc.y)));
  }
  static __device__ __forceinline__ V conj(V a) { return cconj(a); }
  template <bool INV>
  static __device__ __forceinline__ V mi(V a) { return mul_mi<INV>(a); }
  // a * s for a real s given as double (FP64) or as the FP32 pair hi + lo
  static __device__ __forceinline__ V scale(V a, double s) { return cmake(a.x * s, a.y * s); }
  static __device__ __forceinline__ V scalec(V a, double s, float, float) { return cmake(a.x * s, a.y * s); }
  static __device__ __forceinline__ V half(V a) { return cmake(0.5 * a.x, 0.5 * a.y); }
  static __device__ __forceinline__ V from(cplx a) { return a; }
  static __device__ __forceinline__ cplx to(V a) { return a; }
  static __device__ __forceinline__ bool nonzero(V a) { return a.x != 0.0 || a.y != 0.0; }
  static __device__ __forceinline__ V norm(V a) { return a; }
};

// ---------------------------------------------------------------------------
// Double-float
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
// (ah + al) + (bh + bl)
__device__ __forceinline__ void dw_add(float ah, float al, float bh, float bl, float& rh, float& rl) {
  float s, e;
  two_sum(ah, bh, s, e);
  e = __fadd_rn(e, __fadd_rn(al, bl));
  fast_two_sum(s, e, rh, rl);
}
// (ah + al) + (bh + bl) left unnormalised: the high parts are added
// error-free and the low parts and the rounding error summed in FP32; the
// pair (rh, rl) represents the sum to the same accuracy, with |rl| possibly a
// few units of the last place of rh.  Callers renormalise (fast-two-sum)
// before a value leaves the registers.
__device__ __forceinline__ void dw_add_lazy(float ah, float al, float bh, float bl, float& rh, float& rl) {
  float e;
  two_sum(ah, bh, rh, e);
  rl = __fadd_rn(e, __fadd_rn(al, bl));
}
// (ah + al) * (bh + bl)
__device__ __forceinline__ void dw_mul(float ah, float al, float bh, float bl, float& rh, float& rl) {
  float p = __fmul_rn(ah, bh);
  float e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
  fast_two_sum(p, e, rh, rl);
}
// x*y + s*u*v in double-word (s = +1 or -1): the two exact products are summed
// with one two-sum, their low parts and the cross terms folded into the error.
__device__ __forceinline__ void dw_dot2(float xh, float xl, float yh, float yl, float uh, float ul, float vh,
                                       float vl, float sgn, float& rh, float& rl) {
  float p1 = __fmul_rn(xh, yh);
  float e1 = __fmaf_rn(xh, yh, -p1);
  float p2 = __fmul_rn(sgn * uh, vh);
  float e2 = __fmaf_rn(sgn * uh, vh, -p2);
  float s, e;
  two_sum(p1, p2, s, e);
  e = __fadd_rn(e, __fadd_rn(e1, e2));
  e = __fmaf_rn(xh, yl, e);
  e = __fmaf_rn(xl, yh, e);
  e = __fmaf_rn(sgn * uh, vl, e);
  e = __fmaf_rn(sgn * ul, vh, e);
  fast_two_sum(s, e, rh, rl);
}

// complex double-float: x = re.hi, y = re.lo, z = im.hi, w = im.lo (16 bytes)
struct OpsDF {
  typedef float4 V;
  static __device__ __forceinline__ V zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  // sums inside a butterfly are left unnormalised (dw_add_lazy); norm()
  // renormalises before a value is stored or converted
  static __device__ __forceinline__ V add(V a, V b) {
    V r;
    dw_add_lazy(a.x, a.y, b.x, b.y, r.x, r.y);
    dw_add_lazy(a.z, a.w, b.z, b.w, r.z, r.w);
    return r;
  }
  static __device__ __forceinline__ V sub(V a, V b) {
    V r;
    dw_add_lazy(a.x, a.y, -b.x, -b.y, r.x, r.y);
    dw_add_lazy(a.z, a.w, -b.z, -b.w, r.z, r.w);
    return r;
  }
  static __device__ __forceinline__ V norm(V a) {
    V r;
    fast_two_sum(a.x, a.y, r.x, r.y);
    fast_two_sum(a.z, a.w, r.z, r.w);
    return r;
  }
  // a * b
  static __device__ __forceinline__ V mul(V a, V b) {
    V r;
    dw_dot2(a.x, a.y, b.x, b.y, a.z, a.w, b.z, b.w, -1.f, r.x, r.y);  // ar br - ai bi
    dw_dot2(a.x, a.y, b.z, b.w, a.z, a.w, b.x, b.y, 1.f, r.z, r.w);   // ar bi + ai br
    return r;
  }
  static __device__ __forceinline__ V mac(V acc, V a, V b) { return add(acc, mul(a, b)); }
  // a * conj(b)
  static __device__ __forceinline__ V mulc(V a, V b) {
    V r;
    dw_dot2(a.x, a.y, b.x, b.y, a.z, a.w, b.z, b.w, 1.f, r.x, r.y);   // ar br + ai bi
    dw_dot2(a.z, a.w, b.x, b.y, a.x, a.y, b.z, b.w, -1.f, r.z, r.w);  // ai br - ar bi
    return r;
  }
  static __device__ __forceinline__ V conj(V a) { return make_float4(a.x, a.y, -a.z, -a.w); }
  template <bool INV>
  static __device__ __forceinline__ V mi(V a) {
    return INV ? make_float4(-a.z, -a.w, a.x, a.y) : make_float4(a.z, a.w, -a.x, -a.y);
  }
  // a * s, s split on the fly (FP64 work: keep out of inner loops)
  static __device__ __forceinline__ V scale(V a, double s) {
    float sh = __double2float_rn(s);
    float sl = __double2float_rn(s - (double)sh);
    return scalec(a, s, sh, sl);
  }
  // a * (sh + sl) for a constant given as its FP32 pair
  static __device__ __forceinline__ V scalec(V a, double, float sh, float sl) {
    V r;
    dw_mul(a.x, a.y, sh, sl, r.x, r.y);
    dw_mul(a.z, a.w, sh, sl, r.z, r.w);
    return r;
  }
  static __device__ __forceinline__ V half(V a) {  // exact
    return make_float4(0.5f * a.x, 0.5f * a.y, 0.5f * a.z, 0.5f * a.w);
  }
  static __device__ __forceinline__ V from(cplx a) {
    float rh = __double2float_rn(a.x), ih = __double2float_rn(a.y);
    return make_float4(rh, __double2float_rn(a.x - (double)rh), ih, __double2float_rn(a.y - (double)ih));
  }
  static __device__ __forceinline__ cplx to(V a) {
    a = norm(a);
    return cmake((double)a.x + (double)a.y, (double)a.z + (double)a.w);
  }
  static __device__ __forceinline__ bool nonzero(V a) { return a.x != 0.f || a.z != 0.f; }
};

}  // namespace mr1l
