// lbm_df64.cuh -- double-word ("double-float") arithmetic: a value is the unevaluated
// sum hi + lo of two FP32 numbers with |lo| <= ulp(hi) / 2, which carries about 48
// significant bits.  On GB300 the FP32 pipes issue 64 times as many instructions per
// clock as the FP64 pipe, so a step written in this type runs its arithmetic on the
// FP32 pipes while staying within ~1e-14 of FP64 per operation.
//
// The building blocks are the error-free transformations of Knuth (2Sum), Dekker
// (Fast2Sum, exact when |a| >= |b|) and the FMA product 2Prod (a b = p + e exactly).
// Sums and products follow the double-word algorithms of Joldes, Muller and Popescu,
// "Tight and rigorous error bounds for basic building blocks of double-word
// arithmetic", ACM TOMS 44 (2017):
//   sum       -- SloppyDWPlusDW (error <= ~3u^2 (|x| + |y|), u = 2^-24);
//   product   -- DWTimesDW2 without the final renormalisation (relative error ~4u^2);
//   x * float -- DWTimesFP1 likewise (relative error ~2u^2);
//   quotient  -- DWDivDW2, with one correctly rounded reciprocal of the divisor's high word.
// The reciprocal square root is one FP32 Newton step on rsqrtf, then one Newton step
// with the residual 1 - x y^2 evaluated in double-word arithmetic (tiny arguments are
// scaled by a power of two first).
// The exponent range is FP32's: magnitudes below ~1e-38 lose precision and below
// ~1e-45 become zero (an absolute error below 1e-38, far under every tolerance here).
//
// Every float operation of the transformations uses the _rn intrinsics, so the compiler
// neither contracts nor reorders them.
#pragma once

namespace lbm {

struct __align__(8) df64 {
    float hi, lo;
    df64() = default;
    __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
    // Nearest double word of a double: hi = fl32(d); d - hi is exact in FP64.
    __host__ __device__ explicit constexpr df64(double d)
        : hi(static_cast<float>(d)), lo(static_cast<float>(d - static_cast<double>(static_cast<float>(d)))) {}
    __host__ __device__ explicit constexpr df64(float f) : hi(f), lo(0.0f) {}
    __host__ __device__ explicit constexpr df64(int i) : df64(static_cast<double>(i)) {}
    __host__ __device__ explicit constexpr operator double() const
    {
        return static_cast<double>(hi) + static_cast<double>(lo);
    }
    __host__ __device__ explicit constexpr operator float() const { return hi; }
};

// ---- error-free transformations --------------------------------------------------
// a + b = s + e exactly, if |a| >= |b| (or a = 0).
__device__ __forceinline__ df64 dw_fast2sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return df64(s, __fsub_rn(b, __fsub_rn(s, a)));
}
// a + b = s + e exactly, any a, b.
__device__ __forceinline__ df64 dw_2sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bp = __fsub_rn(s, a);
    const float ap = __fsub_rn(s, bp);
    return df64(s, __fadd_rn(__fsub_rn(a, ap), __fsub_rn(b, bp)));
}
// a b = p + e exactly (no underflow).
__device__ __forceinline__ df64 dw_2prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return df64(p, __fmaf_rn(a, b, -p));
}

// ---- arithmetic --------------------------------------------------------------------
__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }

// SloppyDWPlusDW: the exact sum of the high words, then the low words added with one
// rounding.  Its error is at most ~3u^2 (|x| + |y|): relative to the operands, not to
// the result, which is what an absolute tolerance on the fields needs.  (The accurate
// variant, relative to the result, costs 9 more instructions per sum; on the parity
// cases it lowered the largest error of any field by 3 % at most.)
// The high-word sum and the low-word sum are independent: on the GPU they are one packed
// FP32-pair add (add.rn.f32x2, two IEEE round-to-nearest sums in one instruction), which
// frees an issue slot per sum and gives the same values.
__device__ __forceinline__ df64 operator+(df64 x, df64 y)
{
    float s, t;
#ifdef __CUDA_ARCH__
    unsigned long long a, b, st;
    asm("mov.b64 %0, {%1, %2};" : "=l"(a) : "f"(x.hi), "f"(x.lo));
    asm("mov.b64 %0, {%1, %2};" : "=l"(b) : "f"(y.hi), "f"(y.lo));
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(st) : "l"(a), "l"(b));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(s), "=f"(t) : "l"(st));
#else
    s = __fadd_rn(x.hi, y.hi);
    t = __fadd_rn(x.lo, y.lo);
#endif
    // the rounding error of s = x.hi + y.hi (2Sum), then one rounding of the low words
    const float bp = __fsub_rn(s, x.hi);
    const float ap = __fsub_rn(s, bp);
    const float e = __fadd_rn(__fsub_rn(x.hi, ap), __fsub_rn(y.hi, bp));
    return dw_fast2sum(s, __fadd_rn(e, t));
}
__device__ __forceinline__ df64 operator-(df64 x, df64 y) { return x + (-y); }

// Products are left unnormalised: hi is the rounded product of the high words and lo
// collects its exact rounding error plus the cross terms, so |lo| <= ~3u |hi| instead of
// u/2 |hi|.  Every operation here takes such pairs as they are (a sum starts with the
// exact 2Sum of the high words and then renormalises), and the dropped lo.lo term and
// the two roundings of lo keep the relative error near 4u^2 (DWTimesDW2 of Joldes et al.
// without its final Fast2Sum).  4 FP32 instructions instead of 9.
__device__ __forceinline__ df64 operator*(df64 x, df64 y)
{
    const float p = __fmul_rn(x.hi, y.hi);
    const float e = __fmaf_rn(x.hi, y.hi, -p);
    return df64(p, __fmaf_rn(x.lo, y.hi, __fmaf_rn(x.hi, y.lo, e)));
}
// x times a float, unnormalised likewise (3 instructions)
__device__ __forceinline__ df64 operator*(df64 x, float y)
{
    const float p = __fmul_rn(x.hi, y);
    return df64(p, __fmaf_rn(x.lo, y, __fmaf_rn(x.hi, y, -p)));
}
__device__ __forceinline__ df64 operator*(float y, df64 x) { return x * y; }

__device__ __forceinline__ df64 operator/(df64 x, df64 y)
{
    const float r = __frcp_rn(y.hi);
    const float th = __fmul_rn(x.hi, r);
    // y th as a double word
    const df64 c = dw_2prod(y.hi, th);
    const df64 rr = dw_fast2sum(c.hi, __fmaf_rn(y.lo, th, c.lo));
    const float ph = __fsub_rn(x.hi, rr.hi);  // exact (Sterbenz)
    const float dl = __fsub_rn(x.lo, rr.lo);
    const float d = __fadd_rn(ph, dl);
    return dw_fast2sum(th, __fmul_rn(d, r));
}

__device__ __forceinline__ df64& operator+=(df64& a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64& operator-=(df64& a, df64 b) { return a = a - b; }
__device__ __forceinline__ df64& operator*=(df64& a, df64 b) { return a = a * b; }

__device__ __forceinline__ bool operator<(df64 a, df64 b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool operator>(df64 a, df64 b) { return b < a; }
__device__ __forceinline__ bool operator<=(df64 a, df64 b) { return !(b < a); }
__device__ __forceinline__ bool operator>=(df64 a, df64 b) { return !(a < b); }

// a b + c
__device__ __forceinline__ df64 rfma(df64 a, df64 b, df64 c) { return a * b + c; }
__device__ __forceinline__ df64 rfma(float a, df64 b, df64 c) { return b * a + c; }
__device__ __forceinline__ df64 rfma(df64 a, df64 b, float c) { return a * b + df64(c); }
__device__ __forceinline__ df64 rfma(df64 a, float b, df64 c) { return a * b + c; }

// 1 / sqrt(x) for x > 0.  An argument below 2^-60 is first scaled by 2^100 (exact), so
// that y^2 below stays in range; the result is scaled back by 2^50.
__device__ __forceinline__ df64 rrsqrt(df64 x)
{
    const bool tiny = x.hi < 0x1p-60f;
    const float pre = tiny ? 0x1p100f : 1.0f, post = tiny ? 0x1p50f : 1.0f;
    x = df64(__fmul_rn(x.hi, pre), __fmul_rn(x.lo, pre));
    float y = rsqrtf(x.hi);
    // FP32 Newton step: y (3 - x y^2) / 2
    y = __fmul_rn(y, __fmaf_rn(__fmul_rn(-0.5f * x.hi, y), y, 1.5f));
    // residual e = 1 - x y^2, with x y^2 as a double word (it is 1 to ~2^-23)
    const df64 t = x * dw_2prod(y, y);
    const float e = __fsub_rn(__fsub_rn(1.0f, t.hi), t.lo);
    const df64 r = dw_fast2sum(y, __fmul_rn(__fmul_rn(0.5f, y), e));
    return df64(__fmul_rn(r.hi, post), __fmul_rn(r.lo, post));
}

}  // namespace lbm
