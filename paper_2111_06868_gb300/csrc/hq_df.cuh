// hq_df.cuh -- double-float arithmetic on the FP32 pipes: a double carried as
// an unevaluated sum hi + lo of two floats (48 significant bits).
//   * products by Dekker's method with an FMA: p = x_h y_h exactly as
//     p + fma(x_h, y_h, -p), plus the cross terms x_h y_l + x_l y_h;
//   * sums by Knuth's two-sum: s = a + b and its exact rounding error
//     (a - (s - bb)) + (b - bb), bb = s - a, collected in a float beside s;
//   * a result renormalised by a fast two-sum (|lo| <= ulp(hi) / 2);
//   * doubles split into (hi, lo) and rebuilt from them with integer
//     operations on their bit fields: no instruction here runs on the FP64
//     pipe.
// Every rounding is to nearest in FP32 (the intrinsics are never contracted
// into FMAs).  Magnitudes below 2^-126 are flushed to zero (2^-74 for the
// lo part of a split).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hq {
namespace df {

struct C {
    float rh, rl, ih, il;  // re = rh + rl, im = ih + il
};

// d = hi + lo to 48 bits: hi = d truncated to 24 significant bits, lo = the
// remaining 29 mantissa bits (rounded to 24); |d| < 2^-126 gives 0.
__device__ __forceinline__ void split(double d, float &hi, float &lo)
{
    const unsigned long long b = __double_as_longlong(d);
    const uint32_t hw = uint32_t(b >> 32), lw = uint32_t(b);
    const uint32_t sgn = hw & 0x80000000u;
    const uint32_t ex = (hw >> 20) & 0x7FFu;  // biased exponent (1023)
    // exponent rebiased to 127, top 23 of the 52 mantissa bits
    const uint32_t hb = sgn | (((hw & 0x7FFFFFFFu) - 0x38000000u) << 3) | (lw >> 29);
    // remaining 29 mantissa bits, scaled by 2^(e - 52): exponent field e - 52 + 127
    const float lo_mag = __fmul_rn(__uint2float_rn(lw & 0x1FFFFFFFu), __uint_as_float((ex - 948u) << 23));
    hi = ex > 896u ? __uint_as_float(hb) : 0.f;
    lo = ex > 948u ? __uint_as_float(__float_as_uint(lo_mag) | sgn) : 0.f;
}

// The double nearest below |h + l| in magnitude (truncated to 53 bits), for a
// normalised pair (|l| <= ulp(h) / 2); |h| < 2^-126 gives 0.
__device__ __forceinline__ double join(float h, float l)
{
    const uint32_t hb = __float_as_uint(h), lb = __float_as_uint(l);
    const int eh = int((hb >> 23) & 0xFFu), el = int((lb >> 23) & 0xFFu);
    if (eh == 0) return 0.0;
    // h = M 2^(eh - 127 - 52) with M of 53 bits
    unsigned long long M = (unsigned long long)((hb & 0x7FFFFFu) | 0x800000u) << 29;
    if (el != 0) {
        const unsigned long long ml = (lb & 0x7FFFFFu) | 0x800000u;
        const int sh = el - eh + 29;  // l = (ml << sh) 2^(eh - 127 - 52)
        const unsigned long long Ml = sh >= 0 ? (ml << sh) : (sh > -24 ? (ml >> -sh) : 0ull);
        M = ((hb ^ lb) >> 31) ? M - Ml : M + Ml;
    }
    int e = eh + 896;  // biased double exponent of h
    if (M >> 53) {
        M >>= 1;
        ++e;
    } else if (!(M >> 52)) {
        M <<= 1;
        --e;
    }
    return __longlong_as_double((long long)((((unsigned long long)(hb >> 31)) << 63) |
                                            ((unsigned long long)e << 52) | (M & ((1ull << 52) - 1))));
}

__device__ __forceinline__ C load(const double2 v)
{
    C c;
    split(v.x, c.rh, c.rl);
    split(v.y, c.ih, c.il);
    return c;
}

// (re_h, re_l, im_h, im_l) of a complex double, for matrix entries
__device__ __forceinline__ float4 entry(double re, double im)
{
    float4 e;
    split(re, e.x, e.y);
    split(im, e.z, e.w);
    return e;
}

// value s + c, c collecting the exact rounding errors
struct Acc {
    float s, c;
};

// a = (x_h + x_l)(y_h + y_l), the first term of a sum
__device__ __forceinline__ Acc first(float xh, float xl, float yh, float yl)
{
    const float p = __fmul_rn(xh, yh);
    float e = __fmaf_rn(xh, yh, -p);
    e = __fmaf_rn(xh, yl, e);
    e = __fmaf_rn(xl, yh, e);
    return {p, e};
}

// a += (x_h + x_l)(y_h + y_l)
__device__ __forceinline__ void add_prod(Acc &a, float xh, float xl, float yh, float yl)
{
    const float p = __fmul_rn(xh, yh);
    float e = __fmaf_rn(xh, yh, -p);
    e = __fmaf_rn(xh, yl, e);
    e = __fmaf_rn(xl, yh, e);
    const float s = __fadd_rn(a.s, p);
    const float bb = __fsub_rn(s, a.s);
    const float t = __fadd_rn(__fsub_rn(a.s, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    a.s = s;
    a.c = __fadd_rn(a.c, __fadd_rn(t, e));
}

// the normalised pair (h, l) of an accumulator
__device__ __forceinline__ void norm(const Acc &a, float &h, float &l)
{
    h = __fadd_rn(a.s, a.c);
    l = __fsub_rn(a.c, __fsub_rn(h, a.s));
}

__device__ __forceinline__ double finish(const Acc &a)
{
    float h, l;
    norm(a, h, l);
    return join(h, l);
}

// out = sum_c m[c] v[c] (complex) over NC entries, as normalised pairs
template <int NC>
__device__ __forceinline__ C row(const float4 *m, const C *v)
{
    Acc re = first(m[0].x, m[0].y, v[0].rh, v[0].rl);
    add_prod(re, -m[0].z, -m[0].w, v[0].ih, v[0].il);
    Acc im = first(m[0].x, m[0].y, v[0].ih, v[0].il);
    add_prod(im, m[0].z, m[0].w, v[0].rh, v[0].rl);
#pragma unroll
    for (int c = 1; c < NC; ++c) {
        add_prod(re, m[c].x, m[c].y, v[c].rh, v[c].rl);
        add_prod(re, -m[c].z, -m[c].w, v[c].ih, v[c].il);
        add_prod(im, m[c].x, m[c].y, v[c].ih, v[c].il);
        add_prod(im, m[c].z, m[c].w, v[c].rh, v[c].rl);
    }
    C out;
    norm(re, out.rh, out.rl);
    norm(im, out.ih, out.il);
    return out;
}

// the same, rebuilt as a complex double
template <int NC>
__device__ __forceinline__ double2 row_d(const float4 *m, const C *v)
{
    const C o = row<NC>(m, v);
    return make_double2(join(o.rh, o.rl), join(o.ih, o.il));
}

}  // namespace df
}  // namespace hq
