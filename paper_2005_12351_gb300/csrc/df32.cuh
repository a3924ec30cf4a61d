// df32.cuh -- double-float arithmetic for the few pair terms of the FP32
// forms that decide their accuracy (the closest particle pairs of the near
// field, §2 Eq. (1) P2P).
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits.  The operations are built from error-free
// transformations: TwoSum (Knuth, TAOCP vol. 2, 4.2.2), FastTwoSum (Dekker,
// "A floating-point technique for extending the available precision", 1971)
// and the FMA form of TwoProduct; add and multiply are the short ("sloppy")
// double-word forms analysed by Joldes, Muller & Popescu (ACM TOMS 44, 2017):
// their error is a few units of 2^-44 relative to the operands' magnitudes,
// which for summing pair terms behaves like FP64 rounding.  Every operation is
// spelled with the _rn intrinsics so that the compiler neither contracts nor
// reassociates them.
#pragma once

namespace fmm {

struct df32 {
    float hi, lo;
};

__device__ __forceinline__ df32 df_make(float hi, float lo) { return {hi, lo}; }

// |a| >= |b| (or a == 0): a + b = s + e exactly
__device__ __forceinline__ df32 df_fast2(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// a + b = s + e exactly, any magnitudes
__device__ __forceinline__ df32 df_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

// a * b = p + e exactly
__device__ __forceinline__ df32 df_two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ df32 df_neg(df32 a) { return {-a.hi, -a.lo}; }

__device__ __forceinline__ df32 df_add(df32 a, df32 b)
{
    const df32 s = df_two_sum(a.hi, b.hi);
    return df_fast2(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df32 df_sub(df32 a, df32 b) { return df_add(a, df_neg(b)); }

// a + b for a float b
__device__ __forceinline__ df32 df_addf(df32 a, float b)
{
    const df32 s = df_two_sum(a.hi, b);
    return df_fast2(s.hi, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ df32 df_mul(df32 a, df32 b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return df_fast2(p, e);
}

// times a float (exact small constants such as 3 or 15 included)
__device__ __forceinline__ df32 df_mulf(df32 a, float b)
{
    const float p = __fmul_rn(a.hi, b);
    return df_fast2(p, __fmaf_rn(a.lo, b, __fmaf_rn(a.hi, b, -p)));
}

__device__ __forceinline__ df32 df_sqr(df32 a)
{
    const float p = __fmul_rn(a.hi, a.hi);
    return df_fast2(p, __fmaf_rn(__fadd_rn(a.hi, a.hi), a.lo, __fmaf_rn(a.hi, a.hi, -p)));
}

// 1/sqrt(x) for x > 0 (normal floats): an FP32 seed y = rsqrtf(x.hi), relative
// error ~2^-22, then one Newton step for f(y) = y^-2 - x carried in double-
// float, y' = y + y (1 - x y^2) / 2, which leaves ~(3/2)(2^-22)^2 ~ 2^-43.
// 1 - x y^2 is formed without cancellation loss: x y^2 lies in [1/2, 2], so
// 1 - its high part is exact (Sterbenz) and its low part follows.
__device__ __forceinline__ df32 df_rsqrt(df32 x)
{
    const float y = rsqrtf(x.hi);
    const df32 t = df_mul(x, df_two_prod(y, y));
    const float e = __fsub_rn(__fsub_rn(1.0f, t.hi), t.lo);
    return df_fast2(y, __fmul_rn(__fmul_rn(y, e), 0.5f));
}

__device__ __forceinline__ double df_to_double(df32 a) { return (double)a.hi + (double)a.lo; }

// One source seen from one target in double-float (§2 Eq. (1), the same sums
// as the FP64 pair terms): R = x_i - x_j given as double-floats, the moments S
// as float pairs (Sh, Sl) in the layout of the FP32 forms (quadrupoles: six
// components and their trace).  r = 0 is the caller's to exclude.
template <int S, bool PHI, bool FIELD>
__device__ __forceinline__ void pair_df(df32 dx, df32 dy, df32 dz, const float *Sh, const float *Sl,
                                        df32 &f, df32 &e0, df32 &e1, df32 &e2)
{
    const df32 r2 = df_add(df_sqr(dx), df_add(df_sqr(dy), df_sqr(dz)));
    const df32 y = df_rsqrt(r2);
    const df32 y2 = df_mul(y, y);
    if (S == 0) {
        const df32 q = {Sh[0], Sl[0]};
        if (PHI) f = df_add(f, df_mul(q, y));
        if (FIELD) {
            const df32 w = df_mul(q, df_mul(y, y2));
            e0 = df_add(e0, df_mul(w, dx));
            e1 = df_add(e1, df_mul(w, dy));
            e2 = df_add(e2, df_mul(w, dz));
        }
    } else if (S == 1) {
        const df32 s0 = {Sh[0], Sl[0]}, s1 = {Sh[1], Sl[1]}, s2 = {Sh[2], Sl[2]};
        const df32 y3 = df_mul(y, y2);
        const df32 sr = df_add(df_mul(s0, dx), df_add(df_mul(s1, dy), df_mul(s2, dz)));
        if (PHI) f = df_sub(f, df_mul(sr, y3));
        if (FIELD) {
            const df32 w = df_mulf(df_mul(sr, df_mul(y3, y2)), 3.0f);
            e0 = df_add(e0, df_sub(df_mul(s0, y3), df_mul(w, dx)));
            e1 = df_add(e1, df_sub(df_mul(s1, y3), df_mul(w, dy)));
            e2 = df_add(e2, df_sub(df_mul(s2, y3), df_mul(w, dz)));
        }
    } else {
        const df32 y3 = df_mul(y, y2), y5 = df_mul(y3, y2);
        const df32 a0 = {Sh[0], Sl[0]}, a1 = {Sh[1], Sl[1]}, a2 = {Sh[2], Sl[2]};
        const df32 a3 = {Sh[3], Sl[3]}, a4 = {Sh[4], Sl[4]}, a5 = {Sh[5], Sl[5]};
        const df32 tr = {Sh[6], Sl[6]};
        // grad q for q(R) = sum_{|a|=2} S_a R^a
        const df32 g0 = df_add(df_mulf(df_mul(a0, dx), 2.0f), df_add(df_mul(a1, dy), df_mul(a2, dz)));
        const df32 g1 = df_add(df_mul(a1, dx), df_add(df_mulf(df_mul(a3, dy), 2.0f), df_mul(a4, dz)));
        const df32 g2 = df_add(df_mul(a2, dx), df_add(df_mul(a4, dy), df_mulf(df_mul(a5, dz), 2.0f)));
        const df32 q = df_mulf(df_add(df_mul(g0, dx), df_add(df_mul(g1, dy), df_mul(g2, dz))), 0.5f);
        if (PHI) f = df_add(f, df_sub(df_mulf(df_mul(q, y5), 3.0f), df_mul(tr, y3)));
        if (FIELD) {
            const df32 a = df_mulf(y5, 3.0f);
            const df32 w = df_sub(df_mulf(df_mul(q, df_mul(y5, y2)), 15.0f), df_mul(tr, a));
            e0 = df_add(e0, df_sub(df_mul(w, dx), df_mul(a, g0)));
            e1 = df_add(e1, df_sub(df_mul(w, dy), df_mul(a, g1)));
            e2 = df_add(e2, df_sub(df_mul(w, dz), df_mul(a, g2)));
        }
    }
}

}  // namespace fmm
