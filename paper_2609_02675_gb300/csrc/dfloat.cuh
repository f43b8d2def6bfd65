// Double-float ("double-word") arithmetic on the FP32 pipes: a value is the unevaluated sum
// hi + lo of two floats with |lo| <= ulp(hi)/2, about 48 significand bits.  It stands in for
// FP64 in the ill-conditioned per-body solves, because this GPU's FP64 rate is a small
// fraction of its FP32 rate.
//
// Error-free transformations: TwoSum (Knuth / Moller), FastTwoSum (Dekker 1971, |a| >= |b|),
// TwoProd through one fused multiply-add.  Double-word operations after Joldes, Muller and
// Popescu, "Tight and rigorous error bounds for basic building blocks of double-word
// arithmetic" (ACM TOMS 2017): the accurate sum of two double-words, the product with
// FMA, the quotient by one correction step; the square root by one Newton correction of the
// single-precision root.  Every sum and product in the transformations goes through the
// round-to-nearest intrinsics so that no contraction into an FMA changes them.
#pragma once

namespace pabd {

// keep the float and double overloads visible beside the double-float one declared below
using ::sqrt;

struct df {
    float hi, lo;
    df() = default;
    __host__ __device__ constexpr df(float a) : hi(a), lo(0.f) {}
    __host__ __device__ constexpr df(int a) : hi((float)a), lo(0.f) {}
    // constants written as double literals: split once (folded at compile time)
    __host__ __device__ constexpr df(double a) : hi((float)a), lo((float)(a - (double)(float)a)) {}
    __host__ __device__ constexpr df(float h, float l, int) : hi(h), lo(l) {}
    __device__ explicit operator float() const { return __fadd_rn(hi, lo); }
};

__device__ __forceinline__ df two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df(s, e, 0);
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return df(s, __fsub_rn(b, __fsub_rn(s, a)), 0);
}

__device__ __forceinline__ df two_prod(float a, float b) {
    const float p = __fmul_rn(a, b);
    return df(p, __fmaf_rn(a, b, -p), 0);
}

__device__ __forceinline__ df operator+(df x, df y) {
    const df s = two_sum(x.hi, y.hi);
    const df t = two_sum(x.lo, y.lo);
    const df v = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}

// a double-word plus a float (JMP's DWPlusFP)
__device__ __forceinline__ df operator+(df x, float y) {
    const df s = two_sum(x.hi, y);
    return fast_two_sum(s.hi, __fadd_rn(x.lo, s.lo));
}

__device__ __forceinline__ df operator-(df x) { return df(-x.hi, -x.lo, 0); }
__device__ __forceinline__ df operator-(df x, df y) { return x + (-y); }

__device__ __forceinline__ df operator*(df x, df y) {
    const df c = two_prod(x.hi, y.hi);
    const float t = __fmaf_rn(x.hi, y.lo, __fmul_rn(x.lo, y.lo));
    return fast_two_sum(c.hi, __fadd_rn(c.lo, __fmaf_rn(x.lo, y.hi, t)));
}

// a double-word times a float (JMP's DWTimesFP with FMA)
__device__ __forceinline__ df operator*(df x, float y) {
    const df c = two_prod(x.hi, y);
    return fast_two_sum(c.hi, __fmaf_rn(x.lo, y, c.lo));
}
__device__ __forceinline__ df operator*(float y, df x) { return x * y; }

__device__ __forceinline__ df operator/(df x, df y) {
    const float th = __fdiv_rn(x.hi, y.hi);
    const df r = two_prod(y.hi, th);                    // y * th, hi part exact
    const float rl = __fmaf_rn(y.lo, th, r.lo);
    const float d = __fadd_rn(__fsub_rn(x.hi, r.hi), __fsub_rn(x.lo, rl));
    return fast_two_sum(th, __fdiv_rn(d, y.hi));
}

__device__ __forceinline__ df& operator+=(df& x, df y) { return x = x + y; }
__device__ __forceinline__ df& operator+=(df& x, float y) { return x = x + y; }
__device__ __forceinline__ df& operator-=(df& x, df y) { return x = x - y; }
__device__ __forceinline__ df& operator*=(df& x, df y) { return x = x * y; }

__device__ __forceinline__ bool operator<(df x, df y) { return x.hi < y.hi || (x.hi == y.hi && x.lo < y.lo); }
__device__ __forceinline__ bool operator>(df x, df y) { return y < x; }
__device__ __forceinline__ bool operator<=(df x, df y) { return !(y < x); }
__device__ __forceinline__ bool operator>=(df x, df y) { return !(x < y); }

// square root: s = sqrt(hi) in single precision, then s + (x - s^2) / (2 s)
__device__ __forceinline__ df sqrt(df x) {
    if (!(x.hi > 0.f)) return df(0.f);
    const float s = __fsqrt_rn(x.hi);
    const df p = two_prod(s, s);
    const float r = __fadd_rn(__fsub_rn(__fsub_rn(x.hi, p.hi), p.lo), x.lo);
    return fast_two_sum(s, __fdiv_rn(r, __fmul_rn(2.f, s)));
}

__device__ __forceinline__ df inv_sqrt(df x) { return df(1.f) / sqrt(x); }

// Fused multiply-add a * b + c of double-words in the "sloppy" form (the products' and the
// sum's rounding errors added in single precision, one renormalisation): its error is a few
// units of 2^-48 of |a b| + |c| -- the bound of an FP64 multiply-add's inputs rather than of
// its result -- at about half the cost of a product followed by the accurate sum.
__device__ __forceinline__ df fma_dd(df a, df b, df c) {
    const df p = two_prod(a.hi, b.hi);
    const df t = two_sum(p.hi, c.hi);
    const float e = __fadd_rn(__fadd_rn(__fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, p.lo)), c.lo), t.lo);
    return fast_two_sum(t.hi, e);
}

// reciprocal 1 / x of a double-word: the single-precision reciprocal th, corrected once by
// the double-word residual 1 - x th (Newton's step)
__device__ __forceinline__ df recip_dd(df x) {
    const float th = __fdiv_rn(1.f, x.hi);
    const df r = two_prod(x.hi, th);
    const float e = __fsub_rn(__fsub_rn(1.f, r.hi), __fmaf_rn(x.lo, th, r.lo));
    return fast_two_sum(th, __fmul_rn(th, e));
}

__device__ __forceinline__ df shfl_xor(unsigned mask, df v, int o) {
    return df(__shfl_xor_sync(mask, v.hi, o), __shfl_xor_sync(mask, v.lo, o), 0);
}

}  // namespace pabd
