// Compensated FP32 arithmetic: float-float values (hi, lo) and error-free transformations.
//
// A float-float value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi) / 2, a
// 48-bit significand with the FP32 exponent range.  The transformations are the published ones:
//   TwoSum  (Knuth, TAOCP vol. 2, Sec. 4.2.2): a + b = s + e exactly, s = fl(a + b);
//   TwoProd (Dekker 1971, with a fused multiply-add): a * b = p + e exactly, p = fl(a * b);
//   Dot2    (Ogita, Rump, Oishi, "Accurate sum and dot product", SISC 2005): a dot product or sum
//           computed as if in twice the working precision and then rounded.
// On GB300 the FP64 units run at 1/64 of the FP32 rate, so sums that must be accurate to about
// 2^-48 are formed here on the FP32 units instead.  Conversions to and from double (dval, dsplit)
// use the FP64 units and are meant for per-row results and small vectors, not for inner loops.
#pragma once

#include <cuda_runtime.h>

namespace sgks {

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// Dot2 accumulator: the running value is p + s (p carries the rounded sum, s the collected errors).
struct Dot2 {
    float p = 0.f, s = 0.f;
    __device__ __forceinline__ void add_prod(float a, float b) {
        float h, r, q;
        two_prod(a, b, h, r);
        two_sum(p, h, p, q);
        s = __fadd_rn(s, __fadd_rn(q, r));
    }
    // a * (bh + bl) with bh + bl a float-float value
    __device__ __forceinline__ void add_prod2(float a, float bh, float bl) {
        add_prod(a, bh);
        s = __fmaf_rn(a, bl, s);
    }
    // (ah + al) * (bh + bl)
    __device__ __forceinline__ void add_prod22(float ah, float al, float bh, float bl) {
        add_prod(ah, bh);
        s = __fmaf_rn(ah, bl, s);
        s = __fmaf_rn(al, bh, s);
    }
    __device__ __forceinline__ void add(float a) {
        float q;
        two_sum(p, a, p, q);
        s = __fadd_rn(s, q);
    }
    // add the float-float value (ah, al)
    __device__ __forceinline__ void add2(float ah, float al) {
        add(ah);
        s = __fadd_rn(s, al);
    }
    __device__ __forceinline__ void merge(const Dot2& o) {
        float q;
        two_sum(p, o.p, p, q);
        s = __fadd_rn(s, __fadd_rn(q, o.s));
    }
    // (p, s) <- (fl(p + s), its error): the same value, with the collected errors folded in, so that
    // the FP32 sum of later errors starts small again
    __device__ __forceinline__ void renorm() { two_sum(p, s, p, s); }
    __device__ __forceinline__ void negate() {
        p = -p;
        s = -s;
    }
    __device__ __forceinline__ float2 value() const {   // renormalised float-float pair
        float hi, lo;
        two_sum(p, s, hi, lo);
        return make_float2(hi, lo);
    }
    __device__ __forceinline__ float rounded() const { return __fadd_rn(p, s); }   // nearest float of p + s
    __device__ __forceinline__ double to_double() const { return (double)p + (double)s; }
};

// Dot2's error grows with the number of terms in one accumulator: the collected errors are
// summed in plain FP32 (the bound is u|sum| + gamma_n^2 sum|p_i|, gamma_n ~ n u).  A CPU emulation
// of these kernels' Dot2 on 229-term dot products with terms of both signs measured the error at
// ~17x one rounding of u^2 per term (28x at 460 terms).  Long sums therefore take their terms in
// blocks of kDot2Block into a fresh accumulator that is merged into the running one after each
// block (measured ~2.6x), at one merge (eight operations) per block.  Where registers do not
// allow a second accumulator, renorm() every few terms folds the errors back (every 4 terms:
// ~4.6x at 229 terms).
constexpr int kDot2Block = 16;

__device__ __forceinline__ double dval(float2 v) { return (double)v.x + (double)v.y; }
__device__ __forceinline__ float2 dsplit(double v) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}

// Shuffle-xor exchange of a Dot2 accumulator with lane ^ off, merged in place.
__device__ __forceinline__ void dot2_xor_merge(Dot2& a, int off) {
    Dot2 b;
    b.p = __shfl_xor_sync(0xffffffffu, a.p, off);
    b.s = __shfl_xor_sync(0xffffffffu, a.s, off);
    a.merge(b);
}

// Warp-cooperative Dot2 reduction (lanes combine their accumulators in a fixed tree).
__device__ __forceinline__ Dot2 warp_dot2(Dot2 a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dot2_xor_merge(a, o);
    return a;
}

}  // namespace sgks
