// Helpers of the mixed-precision path that keep FP64 work off the FP64 pipe.
//
// On GB300 the FP64 pipe issues ~1.6 operations per SM clock against ~116
// FP32 FMAs, and double<->float conversions run on the FP64 pipe too.  The
// mixed sweep therefore (1) splits each loaded double into a float pair
// hi + lo with integer bit operations, (2) recovers the thermal pressure
// p = (gamma-1)(E - |m|^2/(2 rho) - |B'|^2/2) in double-float arithmetic on the
// FP32 pipe (error-free transformations: Knuth's two-sum and the FMA-based
// two-product, about 44-48 significant bits -- enough to keep the cancellation
// of E against the kinetic and magnetic energies harmless), and (3) widens the
// FP32 increment back to double with one conversion, so that the FP64 pipe
// sees two instructions per conserved variable (conversion, accumulate) --
// about a third of its capacity at the sweeps' rate.
#pragma once
#include <math.h>

namespace ppmlr {

struct df { float h, l; };

// Truncating split of a double into floats: x = h + l + (below 2^-48 |x|).
// |x| outside the normal float range flushes to zero (tiny) or infinity;
// NaN stays NaN.
__device__ __forceinline__ df split_double(double x)
{
    const long long b = __double_as_longlong(x);
    const unsigned hi = (unsigned)((unsigned long long)b >> 32), lo = (unsigned)b;
    const unsigned sgn = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7FFu);
    df r;
    if (e >= 897 && e <= 1150) {
        const unsigned mh = ((hi & 0xFFFFFu) << 3) | (lo >> 29);
        r.h = __uint_as_float(sgn | ((unsigned)(e - 896) << 23) | mh);
        const unsigned rem = lo & 0x1FFFFFFFu;            // value rem * 2^(e-1075)
        float lf = 0.0f;
        if (e >= 949 && rem) lf = __uint2float_rn(rem) * __uint_as_float((unsigned)(e - 948) << 23);
        r.l = sgn ? -lf : lf;
    } else if (e == 0x7FF) {
        const bool nan = ((hi & 0xFFFFFu) | lo) != 0u;
        r.h = __uint_as_float(sgn | 0x7F800000u | (nan ? 0x400000u : 0u));
        r.l = 0.0f;
    } else if (e > 1150) {
        r.h = __uint_as_float(sgn | 0x7F800000u);
        r.l = 0.0f;
    } else {
        r.h = __uint_as_float(sgn);
        r.l = 0.0f;
    }
    return r;
}

// Fast split for doubles in the normal float range (the common case: one
// funnel shift and two logic operations for h, h's bits being those of the
// truncated double): the double's exponent e in [897, 1150] maps to the
// float exponent e - 896 = (e mod 256) with its top bit flipped; the rest
// (zero, tiny, huge, non-finite) takes split_double.
__device__ __forceinline__ df split_double_fast(double x)
{
    const long long b = __double_as_longlong(x);
    const unsigned hi = (unsigned)((unsigned long long)b >> 32), lo = (unsigned)b;
    const unsigned e = (hi >> 20) & 0x7FFu;
    if (e - 897u >= 254u) return split_double(x);
    const unsigned t = __funnelshift_l(lo, hi, 3);       // hi << 3 | lo >> 29: exponent bits 8..0, mantissa 23
    const unsigned sgn = hi & 0x80000000u;
    df r;
    r.h = __uint_as_float(sgn | ((t ^ 0x40000000u) & 0x7FFFFFFFu));
    const unsigned rem = lo & 0x1FFFFFFFu;               // value rem * 2^(e-1075)
    const float scale = e >= 949u ? __uint_as_float((e - 948u) << 23) : 0.0f;
    r.l = __uint_as_float(__float_as_uint(__uint2float_rn(rem) * scale) ^ sgn);
    return r;
}

// Exact float -> double (one conversion; denormal floats are zero under
// flush-to-zero).
__device__ __forceinline__ double widen(float f) { return (double)f; }

// Error-free transformations (no multiply appears, so contraction cannot fuse them).
__device__ __forceinline__ df two_sum(float a, float b)
{
    const float s = a + b;
    const float bp = s - a;
    return {s, (a - (s - bp)) + (b - bp)};
}
__device__ __forceinline__ df quick_two_sum(float a, float b)   // |a| >= |b|
{
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ df df_add(df x, df y)
{
    df s = two_sum(x.h, y.h);
    s.l += x.l + y.l;
    return quick_two_sum(s.h, s.l);
}
__device__ __forceinline__ df df_neg(df x) { return {-x.h, -x.l}; }
__device__ __forceinline__ df df_sqr(df x)
{
    const float p = x.h * x.h;
    float e = fmaf(x.h, x.h, -p);
    e += 2.0f * x.h * x.l;
    return quick_two_sum(p, e);
}
__device__ __forceinline__ df df_div(df x, df y)
{
    const float q1 = x.h / y.h;
    const float p = q1 * y.h;
    const float pe = fmaf(q1, y.h, -p);
    const float r = ((x.h - p) - pe + x.l) - q1 * y.l;
    return quick_two_sum(q1, r / y.h);
}

// Thermal pressure from conserved values split into float pairs (mu0 = 1).
__device__ __forceinline__ float pressure_df(df rho, df m0, df m1, df m2, df b0, df b1, df b2, df E, float gm1)
{
    const df mm = df_add(df_add(df_sqr(m0), df_sqr(m1)), df_sqr(m2));
    const df bb = df_add(df_add(df_sqr(b0), df_sqr(b1)), df_sqr(b2));
    df t = df_add(df_div(mm, rho), bb);
    t.h *= 0.5f;
    t.l *= 0.5f;
    const df q = df_add(E, df_neg(t));
    return gm1 * (q.h + q.l);
}

// The same pressure as a float pair h + l (about 44-48 significant bits):
// gm1 times the double-float difference, the product split by the FMA
// two-product.  The mixed sweeps form p - p_ref from it without first
// rounding p to a float.
__device__ __forceinline__ df pressure_df_pair(df rho, df m0, df m1, df m2, df b0, df b1, df b2, df E, float gm1)
{
    const df mm = df_add(df_add(df_sqr(m0), df_sqr(m1)), df_sqr(m2));
    const df bb = df_add(df_add(df_sqr(b0), df_sqr(b1)), df_sqr(b2));
    df t = df_add(df_div(mm, rho), bb);
    t.h *= 0.5f;
    t.l *= 0.5f;
    const df q = df_add(E, df_neg(t));
    const float ph = gm1 * q.h;
    return {ph, fmaf(gm1, q.h, -ph) + gm1 * q.l};
}

// Earth dipole in float (moment along -z).
__device__ __forceinline__ void dipole_f(float M, float x, float y, float z, float *B)
{
    const float r2 = x * x + y * y + z * z;
    if (M == 0.0f || r2 == 0.0f) { B[0] = B[1] = B[2] = 0.0f; return; }
    const float r = sqrtf(r2);
    const float f = M / (r2 * r2 * r);
    const float mr = -z;
    B[0] = f * (3.0f * mr * x);
    B[1] = f * (3.0f * mr * y);
    B[2] = f * (3.0f * mr * z + r2);
}

}  // namespace ppmlr
