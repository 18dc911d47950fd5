// One directional PPMLR sweep on sm_103a: PPM reconstruction with its limiter,
// characteristic domain-of-dependence states, a linearised Lagrangian MHD
// Riemann solve per interface, the Lagrangian update, the conservative remap to
// the Eulerian grid, the directional dipole/Powell sources, the inner-sphere
// reset and the boundary ghosts -- all fused in one kernel (Sec. II scheme,
// Sec. III-A split, Secs. II / IV-A boundaries).
//
// Thread layout: a tile is L pencils ("lanes") x NP = C + 2*GH positions along
// the sweep axis; one thread owns one (position, lane) for the whole kernel
// and keeps its own cell's values in registers between phases.  Only what a
// neighbour needs crosses threads, through NSM shared-memory values per slot
// (slot-major with an odd pitch NSMP, so a warp's accesses to one value hit 32
// distinct banks and every value of a slot sits at a constant offset from the
// slot's address) that are reused from phase to phase (barrier-separated).  The thread
// index is the shared-memory slot: x sweeps run positions fastest (contiguous
// global rows), y and z sweeps run lanes fastest (consecutive x cells, so every
// global access of a warp is a set of contiguous row segments: coalesced, no
// transpose).  A neighbour at position offset k is slot + k*PS.
//
// R is the arithmetic type of reconstruction, Riemann, remap and sources:
// double for the FP64 path (expression trees identical to the CPU reference,
// compiled without contraction), float for the mixed path (pressure recovery
// and the state accumulation stay in double).
#pragma once
#include <cuda.h>

#include <type_traits>

#include "mixed_util.cuh"
#include "ppmlr_internal.h"

namespace ppmlr {

// Checked build (-DPPMLR_CHECK): every shared-memory, staged-box, geometry and
// state index of the tile body is tested against the extent of its array; an
// out-of-range index raises FLAG_BOUNDS (status PPMLR_E_BOUNDS) and the access
// goes to element 0 of the same array instead.  The plain build compiles the
// bare index.
#ifdef PPMLR_CHECK
#define CHK(i, n) ((i) >= 0 && (i) < (n) ? (i) : (atomicOr(a.flags, FLAG_BOUNDS), 0))
#else
#define CHK(i, n) (i)
#endif

template <typename R> struct K;
template <> struct K<double> {
    static __device__ __forceinline__ double sq(double x) { return sqrt(x); }
    static __device__ __forceinline__ double ab(double x) { return fabs(x); }
    static __device__ __forceinline__ double rs(double x) { return rsqrt(x); }
};
template <> struct K<float> {
    static __device__ __forceinline__ float sq(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float ab(float x) { return fabsf(x); }
    static __device__ __forceinline__ float rs(float x) { return rsqrtf(x); }
};

// Sign and magnitude tests of doubles on the integer pipe (the GB300's FP64
// pipe is its scarcest unit).  For finite values they decide exactly as the
// floating-point comparisons they replace.
__device__ __forceinline__ bool pos_d(double x) { return __double_as_longlong(x) > 0; }          // x > 0
__device__ __forceinline__ bool neg_d(double x)                                                   // x < 0
{
    const long long b = __double_as_longlong(x);
    return b < 0 && (b << 1) != 0;
}
__device__ __forceinline__ long long mag_d(double x) { return __double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFLL; }
// Sign flip and absolute value of a double on the integer pipe: on the GB300
// a double negation or fabs that is not an operand of a fused multiply-add
// is an FP64 add (measured with ncu), doublings likewise.
__device__ __forceinline__ double neg_i(double x)
{
    return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ULL);
}
template <typename R, bool EX>
__device__ __forceinline__ R negx(R x)
{
    if constexpr (!EX && std::is_same<R, double>::value) return neg_i(x);
    else return -x;
}
template <typename R, bool EX>
__device__ __forceinline__ R absx(R x)
{
    if constexpr (!EX && std::is_same<R, double>::value) return __longlong_as_double(mag_d(x));
    else return K<R>::ab(x);
}
// x * y > 0 (both non-zero, same sign; ignores underflow of the product)
__device__ __forceinline__ bool same_sign_d(double x, double y)
{
    const long long a = __double_as_longlong(x), b = __double_as_longlong(y);
    return (a ^ b) >= 0 && (a << 1) != 0 && (b << 1) != 0;
}

// x * 2^k for a finite double whose result stays a normal number, on the
// integer pipe (the exponent field moved; zero stays zero): the same value as
// the multiplication, without an instruction on the GB300's FP64 pipe.
__device__ __forceinline__ double pow2_scale(double x, int k)
{
    const long long b = __double_as_longlong(x);
    return (b << 1) == 0 ? x : __longlong_as_double(b + ((long long)k << 52));
}

// 1/x of a double on the integer and FP32 pipes, correctly rounded (no FP64
// instruction; the hardware-seeded FP64 refinement costs the GB300's FP64
// pipe three fused multiply-adds).  With x = m 2^(e-1075), m the 53-bit
// significand, 1/x = Q 2^(970-e), Q = 2^105 / m in (2^52, 2^53], and the
// result's significand is R = round(Q):
//  1. float seed: h ~ 1/mh from the hardware's approximate reciprocal of
//     the top 24 bits mh = m >> 29; with eh = 1 - mh h (exact by one fused
//     multiply-add) and delta = (m - mh 2^29) / (mh 2^29) < 2^-23,
//     1/m ~ h 2^-29 (1 + d + d^2), d = eh - delta, so R1 = h 2^76 +
//     round(h (d + d^2) 2^76) lies within ~2^8.3 of Q (the omitted
//     eh delta term and the float roundings);
//  2. one Newton step on the exact integer remainder r = 2^105 - m R1
//     (|r| < 2^63, so its low 64 bits are the value): R2 = R1 + round(r / m),
//     r / m from r >> 41 and h in float, within one of Q;
//  3. R = R2 + k, k in {-1, 0, 1}, such that |2^105 - m R| < m / 2 (round
//     to nearest; a tie would need m to be a power of two, where Q is
//     exact).
// Floats are built from and read back to integers by exponent-field
// arithmetic (the 1.5 2^23 offset), not by conversion instructions.
// Zero or subnormal x gives a signed inf, inf a signed zero, NaN itself; a
// result below the normal range flushes to a signed zero.
__device__ __forceinline__ double recip_int(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned ex = (unsigned)(b >> 52) & 0x7FFu;
    const unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
    const unsigned mh = (unsigned)(m >> 29);                                     // [2^23, 2^24)
    const float xh = __uint_as_float((150u << 23) | (mh & 0x7FFFFFu));           // = mh
    const float xl = __uint_as_float(0x4B000000u | ((unsigned)(m >> 6) & 0x7FFFFFu)) - 8388608.0f;  // (m mod 2^29) >> 6
    float h;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(h) : "f"(xh));
    const float eh = fmaf(-xh, h, 1.0f);
    const float d = fmaf(-xl * 0x1p-23f, h, eh);
    const float l = h * fmaf(d, d, d);
    const unsigned hb = __float_as_uint(h);                                      // h in (2^-24, 2^-23]
    long long R = (long long)((hb & 0x7FFFFFu) | 0x800000u) << ((int)(hb >> 23) - 74);
    const float l66 = fmaf(l, 0x1p66f, 12582912.0f);                            // round(l 2^66), |.| < 2^22
    const float lr = fmaf(-(l66 - 12582912.0f), 0x1p-66f, l);                   // its remainder (exact)
    R += ((long long)(__float_as_int(l66) - 0x4B400000) << 10) +
         (long long)(__float_as_int(fmaf(lr, 0x1p76f, 12582912.0f)) - 0x4B400000);
    long long r = -(long long)(m * (unsigned long long)R);                     // 2^105 - m R
    const float vr = __int_as_float(0x4B400000 + (int)(r >> 41)) - 12582912.0f;  // r 2^-41, |.| < 2^22
    const long long k = (long long)(__float_as_int(fmaf(vr, h * 0x1p12f, 12582912.0f)) - 0x4B400000);
    R += k;
    r -= k * (long long)m;
    const long long mm = (long long)m;
    R += (long long)(2 * r > mm) - (long long)(2 * r < -mm);
    const unsigned long long sgn = b & 0x8000000000000000ull;
    unsigned long long res = (sgn | ((unsigned long long)(2044u - ex) << 52)) + (unsigned long long)R;
    res = ex >= 2045u ? sgn : res;                                               // result below the normal range
    res = ex == 0u ? (sgn | 0x7FF0000000000000ull) : res;                       // zero, subnormal
    res = ex == 0x7FFu ? ((b << 12) != 0 ? b : sgn) : res;                       // NaN, inf
    return __longlong_as_double((long long)res);
}

// 1/x: recip_int in the contracted double form; other forms divide.
template <typename R, bool EX>
__device__ __forceinline__ R recip(R x)
{
    if constexpr (!EX && std::is_same<R, double>::value) return recip_int(x);
    else return R(1) / x;
}

// The remap's donor fraction y (> 0 where it is used) reaches the zone width:
// y >= 1, on the bit patterns for the fast double form.
template <typename R, bool EX>
__device__ __forceinline__ bool sliver_too_wide(R y)
{
    if constexpr (!EX && std::is_same<R, double>::value)
        return __double_as_longlong(y) >= 0x3FF0000000000000LL;       // the bits of 1.0
    else return !(R(1) - y > R(0));
}

// x > 0 and x < 0 on the integer pipe for the fast double form, plain
// comparisons otherwise.
template <typename R, bool EX>
__device__ __forceinline__ bool gt0(R x)
{
    if constexpr (!EX && std::is_same<R, double>::value) return pos_d(x);
    else return x > R(0);
}
template <typename R, bool EX>
__device__ __forceinline__ bool lt0(R x)
{
    if constexpr (!EX && std::is_same<R, double>::value) return neg_d(x);
    else return x < R(0);
}

// Correctly rounded square root of a positive normal double with no FP64
// instruction (integer and FP32 pipes; the GB300's FP64 pipe would spend
// ~8.6 slots on it).  With x = m 2^(e-52), m the 53-bit significand, made
// m in [2^52, 2^54) with e even: sqrt(x) = sqrt(N) 2^(e/2 - 52), N = m 2^52,
// and the significand of the result is R = round(sqrt(N)) in [2^52, 2^53).
//  1. sqrt(m / 2^30) = sqrt(xh + xl) as a float pair h + l: xh = m >> 30
//     exact, h the correctly rounded float root, l = (xh - h^2 + xl) / (2h)
//     with the residual xh - h^2 exact by one fused multiply-add; R1 =
//     (h + l) 2^41 is within ~2^8.3 of sqrt(N) (the series' next term
//     (xh - h^2 + xl)^2 / (8 h^3) < 2^-34 and the float roundings of l).
//  2. One Newton step on the exact integer remainder: R2 = R1 +
//     round((N - R1^2) / (2 R1)) (N - R1^2 from a 128-bit square), within
//     one of sqrt(N).
//  3. R = R2 + k, k in {-1, 0, 1}, such that -R < N - R^2 <= R (round to
//     nearest; sqrt(N) of an integer N is never a half-integer, so there
//     are no ties).
__device__ __forceinline__ double sqrt_int(double x)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    int e = (int)(b >> 52) - 1023;
    unsigned long long m = (b & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
    if (e & 1) { m <<= 1; e -= 1; }
    // 1. float-pair seed
    const float xh = (float)(unsigned)(m >> 30);                  // < 2^24: exact
    const float xl = (float)(unsigned)(m & 0x3FFFFFFFull) * 0x1p-30f;
    const float h = __fsqrt_rn(xh);
    const float l = (fmaf(-h, h, xh) + xl) * (0.5f * __frcp_rn(h));
    const unsigned hb = __float_as_uint(h);                         // h in [2^11, 2^12]
    const long long Rh = (long long)((hb & 0x7FFFFFu) | 0x800000u) << ((int)(hb >> 23) - 127 + 18);
    long long R = Rh + (long long)__float2int_rn(l * 0x1p41f);       // |l 2^41| < 2^30
    // 2. Newton step on the exact remainder N - R^2: |N - R^2| < 2^63 (R is
    //    within ~2^8.3 of sqrt(N)), so its low 64 bits are the value
    const unsigned long long ur = (unsigned long long)R;
    long long d = (long long)((m << 52) - ur * ur);
    const long long k = (long long)__float2int_rn((float)(int)(d >> 32) * __fdividef(0x1p-10f, h));
    d -= k * (2 * R + k);                                           // N - (R + k)^2
    R += k;
    // 3. round to nearest
    if (d > R) { d -= 2 * R + 1; R += 1; }
    else if (d <= -R) { d += 2 * R - 1; R -= 1; }
    return __longlong_as_double((long long)(((unsigned long long)((e >> 1) + 1022) << 52) + (unsigned long long)R));
}

// Product of two doubles on the integer pipes.  The GB300's FP64 pipe
// retires ~1.7 lanes per SM and clock and the FP64 sweeps keep it the
// busiest unit, while integer instructions issue beside it: a product moved
// here frees an FP64 slot.  With a = ma 2^(ea-1075), b = mb 2^(eb-1075)
// (53-bit significands): the 106-bit P = ma mb from four 32 x 32 -> 64-bit
// partial products; the result's significand is P >> (52 + t), t = 1 when
// P >= 2^105, rounded up when the next bit is set and the rest (sticky bits)
// or the significand's last bit is; the exponent field is ea + eb - 1023 + t
// (the carry of a significand rounded to 2^53 moves into it).  Normal
// operands with a normal result: the correctly rounded (to nearest, ties to
// even) IEEE product, bit for bit.  Otherwise, with selects and no branch
// (an inline fallback to the hardware product was compiled into a DMUL
// issued every time, which took away the gain): a zero or subnormal operand
// or an underflowing result gives a signed zero, an overflowing one
// infinity, and an inf or NaN operand a result with an all-ones exponent
// (inf or NaN), so a non-finite state stays non-finite.
__device__ __forceinline__ double dmul_int(double a, double b)
{
    const unsigned long long A = (unsigned long long)__double_as_longlong(a);
    const unsigned long long B = (unsigned long long)__double_as_longlong(b);
    const unsigned ah = (unsigned)(A >> 32), al = (unsigned)A;
    const unsigned bh = (unsigned)(B >> 32), bl = (unsigned)B;
    const unsigned ea = (ah >> 20) & 0x7FFu, eb = (bh >> 20) & 0x7FFu;
    const unsigned mah = (ah & 0xFFFFFu) | 0x100000u, mbh = (bh & 0xFFFFFu) | 0x100000u;
    const unsigned long long p0 = (unsigned long long)al * bl;
    const unsigned long long p1 = (unsigned long long)al * mbh + (p0 >> 32);
    const unsigned long long p2 = (unsigned long long)mah * bl + p1;              // < 2^54
    const unsigned long long p3 = (unsigned long long)mah * mbh + (p2 >> 32);     // P >> 64, < 2^42
    const unsigned t = (unsigned)(p3 >> 41);
    const unsigned long long G = (p3 << 22) | ((unsigned)p2 >> 10);              // P >> 42
    const unsigned sh = 10u + t;
    unsigned long long M = G >> sh;
    const unsigned g = (unsigned)G;
    const unsigned rb = (g >> (sh - 1u)) & 1u;
    const unsigned st = (g & ((1u << (sh - 1u)) - 1u)) | ((unsigned)p2 & 0x3FFu) | (unsigned)p0;
    M += rb & ((st != 0u) | (unsigned)M);
    const int E = (int)(ea + eb) - 1023 + (int)t;
    const unsigned long long sgn = (unsigned long long)((ah ^ bh) & 0x80000000u) << 32;
    unsigned long long r = (sgn | ((unsigned long long)(E - 1) << 52)) + M;
    r = E > 2046 ? (sgn | 0x7FF0000000000000ull) : r;                          // overflow: inf
    r = (E < 1 || ea == 0u || eb == 0u) ? sgn : r;                             // zero, subnormal, underflow
    r = (ea == 0x7FFu || eb == 0x7FFu) ? (sgn | 0x7FF0000000000000ull | ((A | B) & 0xFFFFFFFFFFFFFull)) : r;
    return __longlong_as_double((long long)r);
}

// A product that the contracted FP64 form takes on the integer pipes
// (dmul_int; not fused with a following add); elsewhere a * b.
template <typename R, bool EX>
__device__ __forceinline__ R imul(R a, R b)
{
    if constexpr (!EX && std::is_same<R, double>::value) return dmul_int(a, b);
    else return a * b;
}

// Square root of a non-negative value.  Contracted FP64 form: sqrt_int
// (correctly rounded, no FP64 instruction); zero for x = 0, for a negative x
// (a rounded discriminant) and, as x is a sum of squares or a density here,
// for subnormal x; +inf and NaN pass through, so a non-finite state stays
// non-finite.  Otherwise the library square root.
template <typename R, bool EX>
__device__ __forceinline__ R fsqrt(R x)
{
    if constexpr (!EX && std::is_same<R, double>::value) {
        const long long b = __double_as_longlong(x);
        if (b >= 0x7FF0000000000000LL) return x;                      // +inf, NaN
        return b >= 0x0010000000000000LL ? sqrt_int(x) : 0.0;         // the smallest normal double
    } else {
        return K<R>::sq(x);
    }
}

// Fast magnetosonic speed squared along the normal (mu0 = 1).  EX: the
// reference's expression; otherwise one reciprocal of rho shared by the three
// quotients.
template <typename R, bool EX = true>
__device__ __forceinline__ R fast2(R rho, R p, R Bn, R B1, R B2, R gam)
{
    if constexpr (!EX) {
        const R ir = recip<R, EX>(rho);
        const R a2 = gam * p * ir;
        const R b2 = (Bn * Bn + B1 * B1 + B2 * B2) * ir;
        const R bn2 = Bn * Bn * ir;
        const R s = a2 + b2;
        R disc = s * s - R(4) * a2 * bn2;
        if constexpr (!std::is_same<R, double>::value)      // (the double square root below returns 0 for disc <= 0)
            if (disc < R(0)) disc = R(0);
        return R(0.5) * (s + fsqrt<R, EX>(disc));
    }
    R a2 = gam * p / rho;
    R b2 = (Bn * Bn + B1 * B1 + B2 * B2) / rho;
    R bn2 = Bn * Bn / rho;
    R s = a2 + b2;
    R disc = s * s - R(4) * a2 * bn2;
    if (disc < R(0)) disc = R(0);
    return R(0.5) * (s + K<R>::sq(disc));
}

// Nonlinear (two-shock) normal subsystem of the Lagrangian Riemann problem:
// each side's fast wave is a shock whose Lagrangian speed depends on the
// middle total pressure, W(P) = C sqrt(1 + (gamma+1)/(2 gamma) (P/P_s - 1)),
// C = rho c_f (Colella & Woodward 1984 two-shock solver, fast speed and total
// pressure for the gas's).  Starting from the two-wave P*, `iters` Newton steps
// on u*_R(P) - u*_L(P) = 0 (slope of each shock curve dP/du =
// 2 W^3 / (W^2 + C^2)); on return WL, WR hold W at the final P (clipped at 0),
// and the caller's two-wave formulas give u*, P*.  EX: the reference's
// expression trees; otherwise one reciprocal square root per side and one
// division per step (W = C / rsqrt(q), 1/Z = (1 + 1/q) / (2 W)).
template <typename R, bool EX>
__device__ __forceinline__ void two_shock(const int iters, const R uL, const R uR, const R PL, const R PR,
                                          const R gam, R &WL, R &WR)
{
    const R CL = WL, CR = WR;
    if constexpr (EX) {
        const R a = (gam + R(1)) / (R(2) * gam);
        R P = (WR * PL + WL * PR + WL * WR * (uL - uR)) / (WL + WR);
        for (int k = 0; k < iters; k++) {
            const R Pc = P > R(0) ? P : R(0);
            const R WLk = CL * K<R>::sq(R(1) + a * (Pc / PL - R(1)));
            const R WRk = CR * K<R>::sq(R(1) + a * (Pc / PR - R(1)));
            const R uLk = uL - (Pc - PL) / WLk;
            const R uRk = uR + (Pc - PR) / WRk;
            const R ZL = R(2) * WLk * WLk * WLk / (WLk * WLk + CL * CL);
            const R ZR = R(2) * WRk * WRk * WRk / (WRk * WRk + CR * CR);
            P = Pc - ZL * ZR * (uRk - uLk) / (ZL + ZR);
        }
        const R Pc = P > R(0) ? P : R(0);
        WL = CL * K<R>::sq(R(1) + a * (Pc / PL - R(1)));
        WR = CR * K<R>::sq(R(1) + a * (Pc / PR - R(1)));
    } else {
        const R a = (gam + R(1)) / (R(2) * gam);
        const R aL = a / PL, aR = a / PR, b = R(1) - a;       // q = 1 + a (P/P_s - 1) = b + (a/P_s) P
        const R iCL = R(1) / CL, iCR = R(1) / CR;
        R P = (WR * PL + WL * PR + WL * WR * (uL - uR)) / (WL + WR);
        for (int k = 0; k < iters; k++) {
            const R Pc = gt0<R, false>(P) ? P : R(0);
            const R rqL = K<R>::rs(b + aL * Pc), rqR = K<R>::rs(b + aR * Pc);
            const R rWL = rqL * iCL, rWR = rqR * iCR;         // 1 / W
            const R f = (uR - uL) + (Pc - PR) * rWR + (Pc - PL) * rWL;
            const R izL = R(0.5) * (R(1) + rqL * rqL) * rWL, izR = R(0.5) * (R(1) + rqR * rqR) * rWR;   // 1 / Z
            P = Pc - f / (izL + izR);
        }
        const R Pc = gt0<R, false>(P) ? P : R(0);
        WL = CL * fsqrt<R, false>(b + aL * Pc);
        WR = CR * fsqrt<R, false>(b + aR * Pc);
    }
}

// Lagrangian fast impedance W = rho c_f without a reciprocal of rho:
// W^2 = rho (rho c_f^2) = rho (S + sqrt(S^2 - 4 gamma p Bn^2)) / 2 with
// S = gamma p + |B|^2 (the fast-speed formula multiplied through by rho).
// Contracted FP64 form, from parts its callers share: b2 = |B|^2 and
// bn4 = 4 Bn^2 (the factors 4 and 1/2 as exponent moves on the integer pipe).
__device__ __forceinline__ double fast_impedance(double rho, double p, double b2, double bn4, double gam)
{
    const double gp = dmul_int(gam, p);
    const double S = gp + b2;
    const double D = fma(-gp, bn4, dmul_int(S, S));     // fsqrt gives 0 for D <= 0
    return fsqrt<double, false>(dmul_int(rho, pow2_scale(S + fsqrt<double, false>(D), -1)));
}

// Earth dipole along -z: B_d = M [3 (m.r) r - m r^2] / r^5, m = -z.
template <bool EX = true>
__device__ __forceinline__ void dipole(double M, double x, double y, double z, double *B)
{
    if constexpr (!EX) {
        const double r2 = x * x + y * y + z * z;
        if (M == 0.0 || r2 == 0.0) { B[0] = B[1] = B[2] = 0.0; return; }
        const double f = M / (r2 * r2 * sqrt(r2));
        const double mr = -z;
        B[0] = f * (3.0 * mr * x);
        B[1] = f * (3.0 * mr * y);
        B[2] = f * (3.0 * mr * z + r2);
        return;
    }
    double r2 = x * x + y * y + z * z;
    if (M == 0.0 || r2 == 0.0) { B[0] = B[1] = B[2] = 0.0; return; }
    double r = sqrt(r2);
    double r5 = r2 * r2 * r;
    double mr = -z;
    B[0] = M * (3.0 * mr * x) / r5;
    B[1] = M * (3.0 * mr * y) / r5;
    B[2] = M * (3.0 * mr * z + r2) / r5;
}

// Limited PPM slope of zone i from its neighbours (Colella & Woodward 1984):
// da = c1 (c2 dp + c3 dm), limited to 2 min(|dm|, |dp|) and zero at an
// extremum.  Contracted forms: c2 and c3 arrive with c1 folded in (c1 is not
// used), and the two limits as one doubling of the smaller difference.
template <typename R, bool EX = true>
__device__ __forceinline__ R limit_slope(R am, R a0, R ap, R c1, R c2, R c3, R *dp_out = nullptr)
{
    if constexpr (!EX && std::is_same<R, double>::value) {
        const double dp = ap - a0, dm = a0 - am;
        if (dp_out) *dp_out = dp;
        if (!same_sign_d(dp, dm)) return 0.0;
        const double da = fma(c2, dp, dmul_int(c3, dm));
        // twice the smaller difference (both non-zero here): the exponent field
        // + 1; |da| limited to it and da's sign put back, on the bit patterns
        // (+0 for da = 0)
        const long long lim = min(mag_d(dm), mag_d(dp)) + (1LL << 52);
        const long long m = min(lim, mag_d(da));
        return __longlong_as_double(m == 0 ? 0LL : (m | (__double_as_longlong(da) & (long long)0x8000000000000000ULL)));
    }
    if constexpr (!EX && std::is_same<R, float>::value) {   // branch-free: min/max and selects
        const float dp = ap - a0, dm = a0 - am;
        if (dp_out) *dp_out = dp;
        const float da = c2 * dp + c3 * dm;
        const float m = fminf(fabsf(da), 2.0f * fminf(fabsf(dm), fabsf(dp)));
        return dp * dm > 0.0f ? copysignf(m, da) : 0.0f;
    }
    R dp = ap - a0;
    R dm = a0 - am;
    R da = c1 * (c2 * dp + c3 * dm);
    if (dp * dm > R(0)) {
        R m = K<R>::ab(da);
        R lim_m = R(2) * K<R>::ab(dm), lim_p = R(2) * K<R>::ab(dp);
        if (lim_m < m) m = lim_m;
        if (lim_p < m) m = lim_p;
        return da > R(0) ? m : (da < R(0) ? -m : R(0));
    }
    return R(0);
}

// Monotonicity constraint of the parabola; returns a6 and updates l, r.
// Fast double form, on the one-sided differences dl = ai - l, dr = r - ai
// (da = dl + dr, a6 = 3 (dl - dr)): the extremum test is a sign test; with dl,
// dr of one sign the overshoot tests da*a6 > da^2 and -da^2 > da*a6 reduce to
// |dl| > 2 |dr| and |dr| > 2 |dl|, compared on the bit patterns with the
// doubling as an exponent increment (exact for normal numbers; for a
// subnormal difference the threshold moves by less than 2^-1021, and the
// constraint is continuous at both switch points); the moved end and a6 then
// have closed forms: l = ai - 2 dr, a6 = 3 dr, or r = ai + 2 dl, a6 = -3 dl.
template <typename R, bool EX = true>
__device__ __forceinline__ R monotone(R ai, R &l, R &r)
{
    if constexpr (!EX && std::is_same<R, double>::value) {
        const double dl = ai - l, dr = r - ai;
        if (!same_sign_d(dr, dl)) {
            l = ai; r = ai;
            return 0.0;
        }
        constexpr long long twice = 1LL << 52;
        const long long ml = mag_d(dl), mr = mag_d(dr);
        if (ml > mr + twice) {
            l = ai - 2.0 * dr;
            return 3.0 * dr;
        }
        if (mr > ml + twice) {
            r = ai + 2.0 * dl;
            return -3.0 * dl;
        }
        return 3.0 * (dl - dr);
    }
    if constexpr (!EX && std::is_same<R, float>::value) {
        // branch-free, on the one-sided differences as in the fast double
        // form: extremum when dl, dr differ in sign; otherwise the overshoot
        // tests |dl| > 2 |dr| (l = ai - 2 dr) and |dr| > 2 |dl| (r = ai + 2 dl),
        // and a6 = 3 (dl - dr) of the adjusted ends
        const float dl = ai - l, dr = r - ai;
        const bool ext = dl * dr <= 0.0f;
        const float adl = fabsf(dl), adr = fabsf(dr);
        float dl2 = adl > adr + adr ? dr + dr : dl;
        float dr2 = adr > adl + adl ? dl + dl : dr;
        dl2 = ext ? 0.0f : dl2;
        dr2 = ext ? 0.0f : dr2;
        l = ai - dl2;
        r = ai + dr2;
        return 3.0f * (dl2 - dr2);
    }
    if ((r - ai) * (ai - l) <= R(0)) {
        l = ai; r = ai;
    } else {
        R da = r - l;
        R m6 = R(6) * (ai - R(0.5) * (l + r));
        if (da * m6 > da * da) l = R(3) * ai - R(2) * r;
        else if (-(da * da) > da * m6) r = R(3) * ai - R(2) * l;
    }
    return R(6) * (ai - R(0.5) * (l + r));
}

// The monotonicity constraint as the one-sided differences of the constrained
// parabola (contracted and mixed forms): with dl = ai - l, dr = r - ai its
// ends are ai - dl2 and ai + dr2 and a6 = 3 (dl2 - dr2): dl2 = dr2 = 0 at an
// extremum (dl, dr of different sign or zero), dl2 = 2 dr where |dl| > 2 |dr|,
// dr2 = 2 dl where |dr| > 2 |dl|, else dl2 = dl, dr2 = dr (the same cases as
// `monotone`).  Double: the tests on the bit patterns and the doublings as
// exponent increments on the integer pipe (exact for normal numbers; a
// subnormal difference is doubled to within 2^-1022), two FP64 instructions.
__device__ __forceinline__ void monotone_d(double ai, double l, double r, double &dl2, double &dr2)
{
    const double dl = ai - l, dr = r - ai;
    constexpr long long twice = 1LL << 52;
    const long long bl = __double_as_longlong(dl), br = __double_as_longlong(dr);
    const long long ml = mag_d(dl), mr = mag_d(dr);
    long long l2 = ml > mr + twice ? br + twice : bl;
    long long r2 = mr > ml + twice ? bl + twice : br;
    if (!same_sign_d(dr, dl)) { l2 = 0; r2 = 0; }
    dl2 = __longlong_as_double(l2);
    dr2 = __longlong_as_double(r2);
}
__device__ __forceinline__ void monotone_d(float ai, float l, float r, float &dl2, float &dr2)
{
    const float dl = ai - l, dr = r - ai;
    const bool ext = dl * dr <= 0.0f;
    const float adl = fabsf(dl), adr = fabsf(dr);
    const float l2 = adl > adr + adr ? dr + dr : dl;
    const float r2 = adr > adl + adl ? dl + dl : dr;
    dl2 = ext ? 0.0f : l2;
    dr2 = ext ? 0.0f : r2;
}

// Averages of the parabola over the fraction y of the zone at its right and
// left ends (below), written with the one-sided differences of monotone_d:
// right: ai + (1 - y)^2 dr2 + y (1 - y) dl2; left: ai - (1 - y)^2 dl2 -
// y (1 - y) dr2 (the same polynomials in y as avg_right / avg_left with
// l = ai - dl2, r = ai + dr2, a6 = 3 (dl2 - dr2)); two fused multiply-adds
// each once P = (1 - y)^2 and Q = y (1 - y) are formed for the fraction.
template <typename R> struct AvgCoef { R P, Q; };
template <typename R>
__device__ __forceinline__ AvgCoef<R> avg_coef(R y)
{
    const R u = R(1) - y;
    return AvgCoef<R>{imul<R, false>(u, u), imul<R, false>(y, u)};
}
template <typename R>
__device__ __forceinline__ R avg_right_d(R ai, R dl2, R dr2, const AvgCoef<R> &k)
{
    return fma(k.Q, dl2, fma(k.P, dr2, ai));
}
template <typename R>
__device__ __forceinline__ R avg_left_d(R ai, R dl2, R dr2, const AvgCoef<R> &k)
{
    return fma(-k.Q, dr2, fma(-k.P, dl2, ai));
}

template <typename R>
__device__ __forceinline__ R avg_right(R l, R r, R a6, R y)
{
    return r - R(0.5) * y * ((r - l) - (R(1) - R(2.0 / 3.0) * y) * a6);
}
template <typename R>
__device__ __forceinline__ R avg_left(R l, R r, R a6, R y)
{
    return l + R(0.5) * y * ((r - l) + (R(1) - R(2.0 / 3.0) * y) * a6);
}

// Coefficients of the PPM slope and interface formulas on a non-uniform
// coordinate (they depend only on the zone widths, so they are shared by all
// reconstructed variables).
template <typename R> struct SlopeCoef { R c1, c2, c3; };
// EX: three quotients as in the reference; otherwise one reciprocal of the
// product of the three denominators, and c1 folded into c2 and c3
// (c1 c2 = x0 (2 xm + x0) / (d1 d2), c1 c3 = x0 (x0 + 2 xp) / (d1 d3);
// c1 is returned as 1).
template <typename R, bool EX = true>
__device__ __forceinline__ SlopeCoef<R> slope_coef(R xm, R x0, R xp)
{
    if constexpr (!EX) {
        const R d1 = xm + x0 + xp, d2 = xp + x0, d3 = xm + x0;
        const R q = imul<R, EX>(x0, recip<R, EX>(imul<R, EX>(d1, imul<R, EX>(d2, d3))));
        SlopeCoef<R> k;
        k.c1 = R(1);
        k.c2 = imul<R, EX>(imul<R, EX>(R(2) * xm + x0, d3), q);
        k.c3 = imul<R, EX>(imul<R, EX>(x0 + R(2) * xp, d2), q);
        return k;
    }
    R s3 = xm + x0 + xp;
    SlopeCoef<R> k;
    k.c1 = x0 / s3;
    k.c2 = (R(2) * xm + x0) / (xp + x0);
    k.c3 = (x0 + R(2) * xp) / (xm + x0);
    return k;
}
template <typename R> struct EdgeCoef { R k1, k2, k3, k4, k5; };
// EX: the reference's five quotients; otherwise one reciprocal of the
// product of the four denominators, and k2 folded into the others (see
// edge_value): k1 + k2 k3, k2 k4, k2 k5 are returned in k1, k4, k5.
template <typename R, bool EX = true>
__device__ __forceinline__ EdgeCoef<R> edge_coef(R x0, R x1, R x2, R x3)
{
    if constexpr (!EX) {
        const R d1 = R(2) * x1 + x2, d2 = R(2) * x2 + x1, d3 = x1 + x2, d4 = x0 + x1 + x2 + x3;
        const R d12 = imul<R, EX>(d1, d2), d34 = imul<R, EX>(d3, d4);
        const R inv = recip<R, EX>(imul<R, EX>(d12, d34));
        const R i12 = imul<R, EX>(d34, inv), i34 = imul<R, EX>(d12, inv);          // 1 / d12, 1 / d34
        const R r1 = imul<R, EX>(d2, i12), r2 = imul<R, EX>(d1, i12);
        const R r3 = imul<R, EX>(d4, i34), r4 = imul<R, EX>(d3, i34);
        const R z1 = imul<R, EX>(x0 + x1, r1), z2 = imul<R, EX>(x3 + x2, r2);
        // k1 = (x1/d3) (1 + 2 (x2/d4)(z1 - z2)), k4 = (x1/d4) z1, k5 = (x2/d4) z2
        const R x1r3 = imul<R, EX>(x1, r3), x2r4 = imul<R, EX>(x2, r4);
        EdgeCoef<R> k;
        R x2r4_2;                                          // 2 x2r4 (an exponent move for doubles)
        if constexpr (std::is_same<R, double>::value) x2r4_2 = pow2_scale(x2r4, 1);
        else x2r4_2 = R(2) * x2r4;
        k.k1 = x1r3 + x1r3 * imul<R, EX>(x2r4_2, z1 - z2);
        k.k2 = R(0);
        k.k3 = R(0);
        k.k4 = imul<R, EX>(imul<R, EX>(x1, r4), z1);
        k.k5 = imul<R, EX>(x2r4, z2);
        return k;
    }
    R z1 = (x0 + x1) / (R(2) * x1 + x2);
    R z2 = (x3 + x2) / (R(2) * x2 + x1);
    R s4 = x0 + x1 + x2 + x3;
    EdgeCoef<R> k;
    k.k1 = x1 / (x1 + x2);
    k.k2 = R(1) / s4;
    k.k3 = R(2) * x2 * x1 / (x1 + x2) * (z1 - z2);
    k.k4 = x1 * z1;
    k.k5 = x2 * z2;
    return k;
}
// Interface value a_{i+1/2} = a0 + k1 d + k2 (k3 d - k4 dm_{i+1} + k5 dm_i),
// d = a1 - a0; contracted forms with the folded coefficients of edge_coef.
template <typename R, bool EX = true>
__device__ __forceinline__ R edge_value(const EdgeCoef<R> &k, R a0, R a1, R dmi, R dmi1)
{
    const R d = a1 - a0;
    if constexpr (!EX) return a0 + k.k1 * d - k.k4 * dmi1 + k.k5 * dmi;
    return a0 + k.k1 * d + k.k2 * (k.k3 * d - k.k4 * dmi1 + k.k5 * dmi);
}
// Contracted forms, with d = a1 - a0 as the slope step computed it.
template <typename R>
__device__ __forceinline__ R edge_value_d(const EdgeCoef<R> &k, R a0, R d, R dmi, R dmi1)
{
    return a0 + k.k1 * d - k.k4 * dmi1 + k.k5 * dmi;
}

// Shared-memory array indices.  Phase by phase (barrier between phases):
//  P1 writes A (primitives of every position, mass width, total pressure,
//     normal field, v x B_d);
//  P2 reads A, writes B (7 limited slopes, flattening indicator);
//  P3 reads A, B, writes C (7 interface values);
//  P4 reads C, writes A[0..8] (traced state right of each zone's left edge);
//  P5 reads A[0..8], A_BN, writes C (Riemann output per interface);
//  P6 reads C, writes B (7 Lagrangian densities, Lagrangian width);
//  P7 reads B, writes A[0..6] (7 remap slopes);
//  P8 reads A, B, writes C (7 remap interface values);
//  P9 reads C (and, steepening, A[0..6] and B of the neighbours), writes the
//     remap flux through each Eulerian edge (flux_slot);
//  P10 reads the fluxes and writes the new state.
enum : int {
    A_RHO = 0, A_U, A_V1, A_V2, A_B1, A_B2, A_P, A_DM, A_PT, A_BN, A_AX, A_AY, A_AZ,
    SB0 = 13, SC0 = 21
};
// P7 -> P8: second differences of the Lagrangian density (contact steepening)
// in the pad value NSM; P9 -> P10: the remap fluxes in values that are free
// by then (A_DM .. A_AZ and the pad), so that P9 can still read its
// neighbours' remap densities and slopes.
__device__ __forceinline__ constexpr int flux_slot(int v) { return v < 6 ? A_DM + v : NSM; }

// Contact-steepening constants (Colella & Woodward 1984, Sec. 1).
constexpr double ST_ETA1 = 20.0, ST_ETA2 = 0.05, ST_EPS = 0.01, ST_K0 = 0.1;

// Layout of a tile's input box staged in shared memory (8 arrays).  y/z
// sweeps: NP positions x L lanes in slot order (position-major, lanes
// consecutive x cells).  x sweep: the box starts one cell before the tile's
// first position so that the copy starts on an even x (16-byte aligned) and
// holds NP + 2 cells per lane row, lane-major.
template <int DIR>
__device__ __forceinline__ int stage_index(int l, int ps, int NP, int L)
{
    return DIR == 0 ? l * (NP + 2) + ps + 1 : ps * L + l;
}
template <int DIR>
__device__ __forceinline__ int stage_array_stride(int NP, int L) { return DIR == 0 ? (NP + 2) * L : NP * L; }

// ---- TMA staging (y and z sweeps) -------------------------------------------
__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// Bounded wait on the mbarrier phase (at most `polls` try_wait polls); false
// if it gave up.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, int polls = 1 << 22)
{
    for (int it = 0; it < polls; it++) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}
// After a bounded wait gave up: one more bounded wait on each buffer that still
// has a box copy in flight, so that the block, when it returns, does not
// leave the copy engine writing into shared memory it no longer owns.  If a
// copy still has not landed after this second wait the block returns anyway
// (FLAG_TIMEOUT is already raised and the status reports it).
__device__ __forceinline__ void mbar_drain(unsigned long long *bar, unsigned parity)
{
    (void)mbar_wait(bar, parity);
}

// One 4D box (x, y, z, variable) of the state into shared memory.
__device__ __forceinline__ void tma_load_4d(void *dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
        : "memory");
}

// One tile of one sweep, processed by the calling block.  `a` describes the
// domain (the single-domain kernel passes its launch argument, the ensemble
// kernel a per-instance copy in shared memory); `tile` is the tile index
// within that domain; `smem_raw` holds NSMP * NP * L values of type R.
// EX (double only): every stage evaluates the reference's expression trees;
// otherwise quotients sharing a denominator use one reciprocal.
// `stage` (optional): this tile's input box staged in shared memory by TMA,
// 8 arrays of NP * L doubles in the tile's slot order (position p of lane l
// at the slot of (p, l)); cells outside the box come from global memory.
// `stage_bar` (optional): the mbarrier (phase 0) that completes when the box
// has landed; the tile loads its geometry and evaluates the dipole while the
// copy is in flight, then waits (bounded: on giving up it raises
// FLAG_TIMEOUT, waits once more for the copy and returns).
template <int DIR, typename R, bool EX, typename ARGS>
__device__ __forceinline__ void sweep_tile(ARGS &a, const int tile, unsigned char *smem_raw, const int flip,
                                           const double *__restrict__ stage = nullptr,
                                           unsigned long long *stage_bar = nullptr)
{
    // input and output state (flip = 1 exchanges them); array v at base + v * vs
    const double *Uin = flip ? a.Un : a.U;
    double *Uout = flip ? const_cast<double *>(a.U) : a.Un;
    const long long vs = a.vs;
    constexpr int T1 = (DIR + 1) % 3, T2 = (DIR + 2) % 3;
    constexpr bool F64 = std::is_same<R, double>::value;
    R *sm = reinterpret_cast<R *>(smem_raw);
    // opaque copies: inside a persistent loop the addresses derived from the
    // tile shape are then recomputed per tile instead of held in registers
    int L_, NP_;
    asm volatile("mov.b32 %0, %1;" : "=r"(L_) : "r"(a.L));
    asm volatile("mov.b32 %0, %1;" : "=r"(NP_) : "r"(a.NP));
    const int L = L_, NP = NP_, NT = NP * L;
    const int PS = DIR == 0 ? 1 : L;
    const int s = threadIdx.x;
    // extents for the checked build: cells of the domain, ghost-extended
    // positions along the sweep axis and across it
    const long long NCELL = (long long)a.n[0] * a.n[1] * a.n[2];
    const int NG = a.N + 2 * GH, NG0 = a.n[0] + 2 * GH, NG1 = a.n[1] + 2 * GH, NG2 = a.n[2] + 2 * GH;
    (void)NCELL; (void)NG; (void)NG0; (void)NG1; (void)NG2;
#define SM(k, slot) sm[CHK((slot) * NSMP + (k), NT * NSMP)]

    // ---- tile decode ----
    const int chunk = tile % a.nchunk;
    const int grp = tile / a.nchunk;
    int p, l;
    if (DIR == 0) { l = s / NP; p = s - l * NP; }
    else { p = s / L; l = s - p * L; }
    const int g0 = chunk * a.C;
    const int Ce = min(a.C, a.N - g0);           // output cells of this chunk
    const int NPe = Ce + 2 * GH;                 // positions in use
    int ix = 0, iy = 0, iz = 0;
    bool lane_ok;
    if (DIR == 0) {
        int q = grp * L + l;
        lane_ok = q < a.n[1] * a.n[2];
        if (lane_ok) { iy = q % a.n[1]; iz = q / a.n[1]; }
    } else {
        int xg = grp % a.ngx, t = grp / a.ngx;
        ix = xg * L + l;
        lane_ok = ix < a.n[0];
        if (DIR == 1) iz = t; else iy = t;
    }
    const bool act = (s < NT) && lane_ok && (p < NPe);
    const int g = g0 - GH + p;                   // cell index along the axis (ghosts < 0 or >= N)
    const double dt = a.dt_dev ? *a.dt_dev : a.dt;
    const R dtr = R(dt);
    R gam;
    if constexpr (F64) gam = R(a.gamma);
    else gam = a.gammaf;

    // base offset and stride of this lane's pencil
    long long base, stride;
    if (DIR == 0) { base = ((long long)iz * a.n[1] + iy) * a.n[0]; stride = 1; }
    else if (DIR == 1) { base = (long long)iz * a.n[1] * a.n[0] + ix; stride = a.n[0]; }
    else { base = (long long)iy * a.n[0] + ix; stride = (long long)a.n[0] * a.n[1]; }

    // ---------------- P1: load, ghosts, primitives ----------------
    double dx = 0.0, pos[3] = {0.0, 0.0, 0.0}, Bdg[3] = {0.0, 0.0, 0.0};
    R rho = 0, u = 0, v1 = 0, v2 = 0, Bn = 0, B1 = 0, B2 = 0, pr = 0, W = 0, dm = 0, e = 0;
    R pdel = 0;                // reconstructed pressure: p - p_reff (mixed path), p (FP64 forms)
    R Bd0 = 0, Bd1 = 0, Bd2 = 0;
    R dtm_k = 0;               // contracted forms: dt / dm (P1 or P4 -> P6)
    bool floored = false;
    const bool out_cell = act && p >= GH && p < GH + Ce;
    float dxf = 0.0f;          // mixed path: the cell width
    // geometry and dipole first: they do not depend on the staged box
    if (act && F64) {
        dx = a.w[CHK(g + GH, NG)];
        pos[0] = a.cx[CHK((DIR == 0 ? g : ix) + GH, NG0)];
        pos[1] = a.cy[CHK((DIR == 1 ? g : iy) + GH, NG1)];
        pos[2] = a.cz[CHK((DIR == 2 ? g : iz) + GH, NG2)];
        if (a.bd && g >= 0 && g < a.N) {      // interior cell: the dipole table
            const long long gi = base + (long long)g * stride;
            Bdg[0] = __ldg(a.bd + CHK(gi, NCELL));
            Bdg[1] = __ldg(a.bd + a.vs + CHK(gi, NCELL));
            Bdg[2] = __ldg(a.bd + 2 * a.vs + CHK(gi, NCELL));
        } else {
            dipole<EX>(a.M, pos[0], pos[1], pos[2], Bdg);
        }
    } else if (act) {
        dxf = a.wf[CHK(g + GH, NG)];
        const float px = a.cxf[CHK((DIR == 0 ? g : ix) + GH, NG0)];
        const float py = a.cyf[CHK((DIR == 1 ? g : iy) + GH, NG1)];
        const float pz = a.czf[CHK((DIR == 2 ? g : iz) + GH, NG2)];
        float Bdf[3];
        dipole_f(a.Mf, px, py, pz, Bdf);
        Bd0 = Bdf[DIR]; Bd1 = Bdf[T1]; Bd2 = Bdf[T2];
    }
    if (stage_bar && !mbar_wait(stage_bar, 0u)) {     // every thread of the block waits
        if (threadIdx.x == 0) atomicOr(a.flags, FLAG_TIMEOUT);
        mbar_drain(stage_bar, 0u);
        return;
    }
    if (act && F64) {
        double Uc[8];
        int src = g;
        bool fixed = false;
        if (g < 0 || g >= a.N) {
            int kind = g < 0 ? a.bc_lo : a.bc_hi;
            if (kind == PPMLR_BC_PERIODIC) src = ((g % a.N) + a.N) % a.N;
            else if (kind == PPMLR_BC_OUTFLOW) src = g < 0 ? 0 : a.N - 1;
            else {
                fixed = true;
                const auto *f = a.inflow;
                double Bp0 = f[4] - Bdg[0], Bp1 = f[5] - Bdg[1], Bp2 = f[6] - Bdg[2];
                double rh = f[0];
                Uc[0] = rh;
                Uc[1] = rh * f[1]; Uc[2] = rh * f[2]; Uc[3] = rh * f[3];
                Uc[4] = Bp0; Uc[5] = Bp1; Uc[6] = Bp2;
                Uc[7] = f[7] / (a.gamma - 1.0) + 0.5 * rh * (f[1] * f[1] + f[2] * f[2] + f[3] * f[3])
                        + 0.5 * (Bp0 * Bp0 + Bp1 * Bp1 + Bp2 * Bp2);
            }
        }
        if (!fixed) {
            const int ps = src - (g0 - GH);                 // position of the source cell in the box
            if (stage && ps >= 0 && ps < NP) {
                const int slot = stage_index<DIR>(l, ps, NP, L), sv = stage_array_stride<DIR>(NP, L);
#pragma unroll
                for (int v = 0; v < 8; v++) Uc[v] = stage[CHK(v * sv + slot, 8 * sv)];
            } else {
                const long long gi = base + (long long)src * stride;
#pragma unroll
                for (int v = 0; v < 8; v++) Uc[v] = __ldg(Uin + v * vs + CHK(gi, NCELL));
            }
        }
        double rd = Uc[0];
        double mn = Uc[1 + DIR], m1 = Uc[1 + T1], m2 = Uc[1 + T2];
        double bn = Uc[4 + DIR], b1 = Uc[4 + T1], b2 = Uc[4 + T2];
        double E = Uc[7];
        double prd;
        Bd0 = R(Bdg[DIR]); Bd1 = R(Bdg[T1]); Bd2 = R(Bdg[T2]);
        if constexpr (EX) {
            prd = (a.gamma - 1.0) * (E - 0.5 * (mn * mn + m1 * m1 + m2 * m2) / rd
                                     - 0.5 * (bn * bn + b1 * b1 + b2 * b2));
            rho = R(rd); u = R(mn / rd); v1 = R(m1 / rd); v2 = R(m2 / rd);
            e = R(E / rd);
        } else {
            const double ir = recip<double, EX>(rd);
            prd = dmul_int(a.gamma - 1.0, E - pow2_scale(dmul_int(mn, mn) + m1 * m1 + m2 * m2, -1) * ir
                                          - 0.5 * (dmul_int(bn, bn) + b1 * b1 + b2 * b2));
            rho = R(rd); u = R(dmul_int(mn, ir)); v1 = R(dmul_int(m1, ir)); v2 = R(dmul_int(m2, ir));
            e = R(dmul_int(E, ir));
            if (a.iw) dtm_k = R(dmul_int(dmul_int(dt, ir), a.iw[CHK(g + GH, NG)]));    // dt / (rho dx) without a division
        }
        // p_min >= 0: the floor test is a signed comparison of the bit patterns in
        // the contracted form (integer pipe); the exact form compares doubles
        const bool below = EX ? prd < a.p_min : __double_as_longlong(prd) < __double_as_longlong(a.p_min);
        if (below) { prd = a.p_min; floored = out_cell; }
        Bn = R(bn); B1 = R(b1); B2 = R(b2); pr = R(prd);
        dm = R(imul<double, EX>(rd, dx));
    } else if (act) {
        // mixed path: float geometry, float dipole, integer double->float
        // splits and a double-float pressure recovery (no FP64 instructions)
        int src = g;
        bool fixed = false;
        if (g < 0 || g >= a.N) {
            int kind = g < 0 ? a.bc_lo : a.bc_hi;
            if (kind == PPMLR_BC_PERIODIC) src = ((g % a.N) + a.N) % a.N;
            else if (kind == PPMLR_BC_OUTFLOW) src = g < 0 ? 0 : a.N - 1;
            else fixed = true;
        }
        const float gm1 = a.gammaf - 1.0f;
        if (fixed) {
            const auto *f = a.inflowf;
            rho = f[0];
            u = f[1 + DIR]; v1 = f[1 + T1]; v2 = f[1 + T2];
            Bn = f[4 + DIR] - Bd0; B1 = f[4 + T1] - Bd1; B2 = f[4 + T2] - Bd2;
            pr = f[7];
            pdel = f[7] - a.p_reff;
            e = pr / (gm1 * rho) + 0.5f * (u * u + v1 * v1 + v2 * v2) + 0.5f * (Bn * Bn + B1 * B1 + B2 * B2) / rho;
        } else {
            df q[8];
            const int ps = src - (g0 - GH);                 // position of the source cell in the box
            if (stage && ps >= 0 && ps < NP) {
                const int slot = stage_index<DIR>(l, ps, NP, L), sv = stage_array_stride<DIR>(NP, L);
#pragma unroll
                for (int v = 0; v < 8; v++) q[v] = split_double_fast(stage[CHK(v * sv + slot, 8 * sv)]);
            } else {
                const long long gi = base + (long long)src * stride;
#pragma unroll
                for (int v = 0; v < 8; v++) q[v] = split_double_fast(__ldg(Uin + v * vs + CHK(gi, NCELL)));
            }
            const df pp = pressure_df_pair(q[0], q[1 + DIR], q[1 + T1], q[1 + T2], q[4 + DIR], q[4 + T1],
                                           q[4 + T2], q[7], gm1);
            rho = q[0].h;
            const float ir = 1.0f / rho;
            u = q[1 + DIR].h * ir; v1 = q[1 + T1].h * ir; v2 = q[1 + T2].h * ir;
            Bn = q[4 + DIR].h; B1 = q[4 + T1].h; B2 = q[4 + T2].h;
            e = q[7].h * ir;
            pr = pp.h + pp.l;
            pdel = (pp.h - a.p_reff) + pp.l;
        }
        if (pr < a.p_minf) { pr = a.p_minf; pdel = a.p_minf - a.p_reff; floored = out_cell; }
        dm = rho * dxf;
    }
    if constexpr (F64) pdel = pr;
    if (act) {
        R Pt;
        if constexpr (F64 && !EX) {     // |B|^2 shared by the total pressure and the impedance
            const double bn2 = dmul_int(Bn, Bn), b2 = fma(B2, B2, fma(B1, B1, bn2));
            Pt = fma(0.5, b2, pr);
            W = fast_impedance(rho, pr, b2, pow2_scale(bn2, 2), gam);
        } else {
            Pt = pr + R(0.5) * (Bn * Bn + B1 * B1 + B2 * B2);
            W = rho * fsqrt<R, EX>(fast2<R, EX>(rho, pr, Bn, B1, B2, gam));
        }
        SM(A_RHO, s) = rho; SM(A_U, s) = u; SM(A_V1, s) = v1; SM(A_V2, s) = v2;
        SM(A_B1, s) = B1; SM(A_B2, s) = B2; SM(A_P, s) = pdel; SM(A_DM, s) = dm;
        SM(A_PT, s) = Pt; SM(A_BN, s) = Bn;
        if (a.do_src) {   // v x B_d in the local frame
            SM(A_AX, s) = v1 * Bd2 - imul<R, EX>(v2, Bd1);
            SM(A_AY, s) = v2 * Bd0 - imul<R, EX>(u, Bd2);
            SM(A_AZ, s) = u * Bd1 - imul<R, EX>(v1, Bd0);
        }
    }
    {
        int nf = __syncthreads_count(floored);
        if (s == 0 && nf) atomicAdd(a.floors, (unsigned long long)nf);
    }

    // ---------------- P2: slopes, flattening indicator, sources ----------------
    R dmv[7];
    R dpv[7];                  // contracted forms: a_{i+1} - a_i, reused by the interface values (P3)
    R src_m[3] = {0, 0, 0}, src_b[3] = {0, 0, 0}, src_e = 0;
    if (act && p >= 1 && p <= NPe - 2) {
        SlopeCoef<R> k = slope_coef<R, EX>(SM(A_DM, s - PS), dm, SM(A_DM, s + PS));
        const R own[7] = {rho, u, v1, v2, B1, B2, pdel};
#pragma unroll
        for (int v = 0; v < 7; v++) {
            dmv[v] = limit_slope<R, EX>(SM(A_RHO + v, s - PS), own[v], SM(A_RHO + v, s + PS), k.c1, k.c2, k.c3,
                                        EX ? nullptr : &dpv[v]);
            SM(SB0 + v, s) = dmv[v];
        }
        R ft = 0;
        if (p >= 2 && p <= NPe - 3) {
            R Pp = SM(A_PT, s + PS), Pm = SM(A_PT, s - PS);
            R dP = Pp - Pm;
            R pmin;
            if constexpr (!EX && F64)      // total pressures >= 0: ordered as their bit patterns
                pmin = __longlong_as_double(min(__double_as_longlong(Pp), __double_as_longlong(Pm)));
            else
                pmin = Pp < Pm ? Pp : Pm;
            bool shock;
            if constexpr (!EX && F64)      // the same tests on the bit patterns (integer pipe)
                shock = mag_d(dP) > mag_d(dmul_int(0.33, pmin)) && pos_d(SM(A_U, s - PS) - SM(A_U, s + PS));
            else
                shock = K<R>::ab(dP) > R(0.33) * pmin && SM(A_U, s - PS) - SM(A_U, s + PS) > R(0);
            if (shock) {
                R den = SM(A_PT, s + 2 * PS) - SM(A_PT, s - 2 * PS);
                R steep = den != R(0) ? dP / den : R(1);
                R f = (steep - R(0.75)) * R(10);
                if (f < R(0)) f = R(0);
                if (f > R(1)) f = R(1);
                ft = f;
            }
        }
        SM(SB0 + 7, s) = ft;
        if (a.do_src && out_cell) {
            // centred-difference span h; the contracted FP64 form reads 1 / h from
            // the geometry table when the context has one
            const bool h_table = F64 && !EX && a.ih;
            R h = R(1);
            if constexpr (F64) {
                if (!h_table) h = R(0.5) * R(a.w[CHK(g + GH - 1, NG)]) + R(dx) + R(0.5) * R(a.w[CHK(g + GH + 1, NG)]);
            } else {
                h = R(0.5) * a.wf[CHK(g + GH - 1, NG)] + a.wf[CHK(g + GH, NG)] + R(0.5) * a.wf[CHK(g + GH + 1, NG)];
            }
            R DB0, DB1, DB2, DA1, DA2;
            if constexpr (EX) {
                DB0 = (SM(A_BN, s + PS) - SM(A_BN, s - PS)) / h;
                DB1 = (SM(A_B1, s + PS) - SM(A_B1, s - PS)) / h;
                DB2 = (SM(A_B2, s + PS) - SM(A_B2, s - PS)) / h;
                DA1 = (SM(A_AY, s + PS) - SM(A_AY, s - PS)) / h;
                DA2 = (SM(A_AZ, s + PS) - SM(A_AZ, s - PS)) / h;
            } else {
                const R ih = h_table ? R(a.ih[CHK(g + GH, NG)]) : R(1) / h;
                DB0 = imul<R, EX>(SM(A_BN, s + PS) - SM(A_BN, s - PS), ih);
                DB1 = imul<R, EX>(SM(A_B1, s + PS) - SM(A_B1, s - PS), ih);
                DB2 = imul<R, EX>(SM(A_B2, s + PS) - SM(A_B2, s - PS), ih);
                DA1 = imul<R, EX>(SM(A_AY, s + PS) - SM(A_AY, s - PS), ih);
                DA2 = imul<R, EX>(SM(A_AZ, s + PS) - SM(A_AZ, s - PS), ih);
            }
            R J0 = 0, J1 = negx<R, EX>(DB2), J2 = DB1;
            R cA0 = 0, cA1 = negx<R, EX>(DA2), cA2 = DA1;
            R divB = DB0;
            if constexpr (EX) {
                src_m[0] = J1 * Bd2 - J2 * Bd1;
                src_m[1] = J2 * Bd0 - J0 * Bd2;
                src_m[2] = J0 * Bd1 - J1 * Bd0;
                R pw = a.powell ? R(1) : R(0);
                src_b[0] = cA0 - pw * u * divB;
                src_b[1] = cA1 - pw * v1 * divB;
                src_b[2] = cA2 - pw * v2 * divB;
                src_e = u * src_m[0] + v1 * src_m[1] + v2 * src_m[2] + Bn * cA0 + B1 * cA1 + B2 * cA2;
            } else {            // the same terms without the products with J0 = cA0 = 0
                src_m[0] = J1 * Bd2 - imul<R, EX>(J2, Bd1);
                src_m[1] = imul<R, EX>(J2, Bd0);
                src_m[2] = negx<R, EX>(imul<R, EX>(J1, Bd0));
                src_b[0] = R(0); src_b[1] = cA1; src_b[2] = cA2;
                if (a.powell) {
                    src_b[0] = negx<R, EX>(imul<R, EX>(u, divB));
                    src_b[1] = cA1 - v1 * divB;
                    src_b[2] = cA2 - v2 * divB;
                }
                src_e = imul<R, EX>(u, src_m[0]) + v1 * src_m[1] + v2 * src_m[2] + B1 * cA1 + B2 * cA2;
            }
        }
    }
    __syncthreads();

    // ---------------- P3: interface values, flattening coefficient ----------------
    R edg[7];
    R flat = 0;
    bool shock_k = false;      // contact steepening: this zone sits in a shock
    if (act && p >= 1 && p <= NPe - 3) {
        EdgeCoef<R> k = edge_coef<R, EX>(SM(A_DM, s - PS), dm, SM(A_DM, s + PS), SM(A_DM, s + 2 * PS));
        const R own[7] = {rho, u, v1, v2, B1, B2, pdel};
#pragma unroll
        for (int v = 0; v < 7; v++) {
            if constexpr (EX) edg[v] = edge_value<R, EX>(k, own[v], SM(A_RHO + v, s + PS), dmv[v], SM(SB0 + v, s + PS));
            else edg[v] = edge_value_d<R>(k, own[v], dpv[v], dmv[v], SM(SB0 + v, s + PS));
            SM(SC0 + v, s) = edg[v];
        }
        if (p >= 3 && p <= NPe - 4) {
            R up = lt0<R, EX>(SM(A_PT, s + PS) - SM(A_PT, s - PS)) ? SM(SB0 + 7, s + PS) : SM(SB0 + 7, s - PS);
            R ft = SM(SB0 + 7, s);
            if constexpr (!EX && F64)      // ft, up in [0, 1]: ordered as their bit patterns
                flat = __double_as_longlong(ft) > __double_as_longlong(up) ? ft : up;
            else
                flat = ft > up ? ft : up;
        }
        if (a.steepen) {   // shock exclusion of contact steepening: relative total-pressure jump vs density jump
            const R Pp = SM(A_PT, s + PS), Pm = SM(A_PT, s - PS), rp = SM(A_RHO, s + PS), rm = SM(A_RHO, s - PS);
            shock_k = gam * R(ST_K0) * K<R>::ab(Pp - Pm) / (Pp < Pm ? Pp : Pm) >= K<R>::ab(rp - rm) / (rp < rm ? rp : rm);
        }
    }
    __syncthreads();

    // reciprocal kept from one phase to a later one (contracted forms only):
    // 1 / dxL (P6 -> P9)
    R idxL_k = 0;

    // ---------------- P4: parabolas and characteristic tracing ----------------
    // left state of interface p+1/2 (this zone, right end): kept in registers;
    // right state of interface p-1/2 (this zone, left end): to A[0..8] for p-1.
    R sl[9];
    if (act && p >= 3 && p <= NPe - 4) {
        R yf, ya;
        if constexpr (EX) {
            yf = W * dtr / dm;
            ya = K<R>::sq(rho) * K<R>::ab(Bn) * dtr / dm;
        } else {
            if (!(F64 && a.iw)) dtm_k = dtr / dm;       // else from P1
            const R dtm = dtm_k;
            yf = imul<R, EX>(W, dtm);
            ya = imul<R, EX>(imul<R, EX>(fsqrt<R, EX>(rho), absx<R, EX>(Bn)), dtm);
        }
        const R own[7] = {rho, u, v1, v2, B1, B2, pdel};
        R srv[9];
        // contracted forms: no blend where the zone is not flattened (flat is +0;
        // the double test on its bit pattern)
        bool blend = true;
        if constexpr (!EX && F64) blend = __double_as_longlong(flat) != 0;
        else if constexpr (!EX) blend = flat != R(0);
        AvgCoef<R> kf{}, ka{};
        if constexpr (!EX) { kf = avg_coef<R>(yf); ka = avg_coef<R>(ya); }
#pragma unroll
        for (int v = 0; v < 7; v++) {
            R lft = SM(SC0 + v, s - PS), rgt = edg[v];
            if (blend) {
                lft = flat * own[v] + (R(1) - flat) * lft;
                rgt = flat * own[v] + (R(1) - flat) * rgt;
            }
            if constexpr (EX) {
                R a6 = monotone<R, EX>(own[v], lft, rgt);
                R y = (v == 2 || v == 3) ? ya : yf;
                sl[v] = avg_right<R>(lft, rgt, a6, y);
                srv[v] = avg_left<R>(lft, rgt, a6, y);
                if (v == 4 || v == 5) {
                    sl[v + 3] = avg_right<R>(lft, rgt, a6, ya);
                    srv[v + 3] = avg_left<R>(lft, rgt, a6, ya);
                }
            } else {
                R dl2, dr2;
                monotone_d(own[v], lft, rgt, dl2, dr2);
                const AvgCoef<R> &k = (v == 2 || v == 3) ? ka : kf;
                sl[v] = avg_right_d<R>(own[v], dl2, dr2, k);
                srv[v] = avg_left_d<R>(own[v], dl2, dr2, k);
                if (v == 4 || v == 5) {
                    sl[v + 3] = avg_right_d<R>(own[v], dl2, dr2, ka);
                    srv[v + 3] = avg_left_d<R>(own[v], dl2, dr2, ka);
                }
            }
        }
#pragma unroll
        for (int v = 0; v < 9; v++) SM(v, s) = srv[v];
    }
    __syncthreads();

    // ---------------- P5: Riemann problem at p+1/2 ----------------
    R rs_u = 0, rs_S = 0, rs_s1 = 0, rs_s2 = 0, rs_b1 = 0, rs_b2 = 0, rs_fe = 0;
    if (act && p >= 3 && p <= NPe - 5) {
        R Rs[9];
#pragma unroll
        for (int v = 0; v < 9; v++) Rs[v] = SM(v, s + PS);
        R Bnf;
        if constexpr (F64 && !EX) Bnf = pow2_scale(Bn + SM(A_BN, s + PS), -1);
        else Bnf = R(0.5) * (Bn + SM(A_BN, s + PS));
        // total pressures relative to p_reff (mixed path; 0 for the FP64
        // forms): u*, P* - p_reff and the Lagrangian momentum update need only
        // their differences and weighted means
        R PL, PR;
        R pref = R(0);
        if constexpr (!F64) pref = a.p_reff;
        R WL, WR;
        if constexpr (F64 && !EX) {     // the transverse |B|^2 of each side shared by P and W
            const double bn2 = dmul_int(Bnf, Bnf), bn4 = pow2_scale(bn2, 2);
            const double btL = fma(sl[5], sl[5], dmul_int(sl[4], sl[4])), btR = fma(Rs[5], Rs[5], dmul_int(Rs[4], Rs[4]));
            PL = fma(0.5, btL, sl[6]);
            PR = fma(0.5, btR, Rs[6]);
            WL = fast_impedance(sl[0], sl[6], btL + bn2, bn4, gam);
            WR = fast_impedance(Rs[0], Rs[6], btR + bn2, bn4, gam);
        } else {
            PL = sl[6] + R(0.5) * (sl[4] * sl[4] + sl[5] * sl[5]);
            PR = Rs[6] + R(0.5) * (Rs[4] * Rs[4] + Rs[5] * Rs[5]);
        }
        if constexpr (!F64) {
            WL = sl[0] * K<R>::sq(fast2<R, EX>(sl[0], sl[6] + pref, Bnf, sl[4], sl[5], gam));
            WR = Rs[0] * K<R>::sq(fast2<R, EX>(Rs[0], Rs[6] + pref, Bnf, Rs[4], Rs[5], gam));
        } else if constexpr (EX) {
            WL = sl[0] * K<R>::sq(fast2<R, EX>(sl[0], sl[6], Bnf, sl[4], sl[5], gam));
            WR = Rs[0] * K<R>::sq(fast2<R, EX>(Rs[0], Rs[6], Bnf, Rs[4], Rs[5], gam));
        }
        if constexpr (!F64) {
            const R PLa = PL + pref, PRa = PR + pref;          // the nonlinear solver takes absolute pressures
            if (a.riemann_iters > 0 && PLa > R(0) && PRa > R(0))
                two_shock<R, EX>(a.riemann_iters, sl[1], Rs[1], PLa, PRa, gam, WL, WR);
        } else {
            if (a.riemann_iters > 0 && gt0<R, EX>(PL) && gt0<R, EX>(PR))
                two_shock<R, EX>(a.riemann_iters, sl[1], Rs[1], PL, PR, gam, WL, WR);
        }
        R us, Ps;
        if constexpr (EX) {
            us = (WL * sl[1] + WR * Rs[1] + PL - PR) / (WL + WR);
            Ps = (WR * PL + WL * PR + WL * WR * (sl[1] - Rs[1])) / (WL + WR);
        } else if constexpr (F64) {
            // P* = PL - WL (u* - uL): the same value in exact arithmetic
            // (the left wave's jump condition), two instructions
            us = dmul_int(fma(WR, Rs[1], dmul_int(WL, sl[1])) + PL - PR, recip<R, EX>(WL + WR));
            Ps = fma(-WL, us - sl[1], PL);
        } else {
            const R iW = recip<R, EX>(WL + WR);
            us = (WL * sl[1] + WR * Rs[1] + PL - PR) * iW;
            Ps = (WR * PL + WL * PR + WL * WR * (sl[1] - Rs[1])) * iW;
        }
        R Ss;
        if constexpr (F64 && !EX) Ss = Ps - pow2_scale(Bnf, -1) * Bnf;
        else Ss = Ps - R(0.5) * Bnf * Bnf;
        R vs[2], ss[2];
        if constexpr (F64 && !EX) {
            // Alfven impedances Z = sqrt(rho) |Bn|: with s = Bn B_t the common
            // factor |Bn| cancels from v* = (ZL vL + ZR vR + sR - sL)/(ZL + ZR),
            // v* = (qL vL + qR vR + sgn(Bn)(B_tR - B_tL))/(qL + qR) with
            // q = sqrt(rho), and s* = sL + ZL (v* - vL) (as P* above) =
            // Bn (B_tL + sgn(Bn) qL (v* - vL)); Bn = 0: v* the mean, s* = 0
            const bool zero_z = (__double_as_longlong(Bnf) << 1) == 0;
            const double qL = fsqrt<R, EX>(sl[0]), qR = fsqrt<R, EX>(Rs[0]);
            const double iQ = recip<R, EX>(qL + qR);
            const long long sgn = __double_as_longlong(Bnf) & 0x8000000000000000LL;
            const double sqL = __longlong_as_double(__double_as_longlong(qL) ^ sgn);     // sgn(Bn) qL
#pragma unroll
            for (int t = 0; t < 2; t++) {
                const double vL = sl[2 + t], vR = Rs[2 + t];
                const double dB = __longlong_as_double(__double_as_longlong(Rs[7 + t] - sl[7 + t]) ^ sgn);
                if (zero_z) {
                    vs[t] = 0.5 * (vL + vR);
                    ss[t] = 0.0;
                } else {
                    vs[t] = dmul_int(fma(qL, vL, dmul_int(qR, vR)) + dB, iQ);
                    ss[t] = dmul_int(Bnf, fma(sqL, vs[t] - vL, sl[7 + t]));
                }
            }
        } else {
            R ZL = fsqrt<R, EX>(sl[0]) * K<R>::ab(Bnf);
            R ZR = fsqrt<R, EX>(Rs[0]) * K<R>::ab(Bnf);
            const R zsum = ZL + ZR;
            const bool zero_z = zsum == R(0);
            const R iZ = (EX || zero_z) ? R(0) : recip<R, EX>(zsum);
#pragma unroll
            for (int t = 0; t < 2; t++) {
                R vL = sl[2 + t], vR = Rs[2 + t];
                R sL = Bnf * sl[7 + t], sR = Bnf * Rs[7 + t];
                if (zero_z) {
                    vs[t] = R(0.5) * (vL + vR);
                    ss[t] = R(0);
                } else if constexpr (EX) {
                    vs[t] = (ZL * vL + ZR * vR + sR - sL) / (ZL + ZR);
                    ss[t] = (ZR * sL + ZL * sR + ZL * ZR * (vR - vL)) / (ZL + ZR);
                } else {
                    vs[t] = (ZL * vL + ZR * vR + sR - sL) * iZ;
                    ss[t] = (ZR * sL + ZL * sR + ZL * ZR * (vR - vL)) * iZ;
                }
            }
        }
        rs_u = us; rs_S = Ss; rs_s1 = ss[0]; rs_s2 = ss[1];
        rs_b1 = imul<R, EX>(Bnf, vs[0]); rs_b2 = imul<R, EX>(Bnf, vs[1]);
        if constexpr (F64) rs_fe = imul<R, EX>(Ss, us) - ss[0] * vs[0] - ss[1] * vs[1];
        else rs_fe = (Ss + pref) * us - ss[0] * vs[0] - ss[1] * vs[1];     // absolute S* in the energy flux
        SM(SC0 + 0, s) = rs_u; SM(SC0 + 1, s) = rs_S; SM(SC0 + 2, s) = rs_s1; SM(SC0 + 3, s) = rs_s2;
        SM(SC0 + 4, s) = rs_b1; SM(SC0 + 5, s) = rs_b2; SM(SC0 + 6, s) = rs_fe;
    }
    __syncthreads();

    // ---------------- P6: Lagrangian update ----------------
    R dC[6], qL[7], dxL = 0, del_p = 0, del_m = 0;
    if (act && p >= 4 && p <= NPe - 5) {
        R lu = SM(SC0 + 0, s - PS), lS = SM(SC0 + 1, s - PS), ls1 = SM(SC0 + 2, s - PS), ls2 = SM(SC0 + 3, s - PS);
        R lb1 = SM(SC0 + 4, s - PS), lb2 = SM(SC0 + 5, s - PS), lfe = SM(SC0 + 6, s - PS);
        R dxr;
        if constexpr (F64) dxr = R(dx);
        else dxr = a.wf[CHK(g + GH, NG)];
        dxL = dxr + dtr * (rs_u - lu);
        if (!gt0<R, EX>(dxL)) atomicOr(a.flags, FLAG_CFL);
        R bv1 = imul<R, EX>(dtr, rs_b1 - lb1);
        R bv2 = imul<R, EX>(dtr, rs_b2 - lb2);
        R B1dx = B1 * dxr + bv1;
        R B2dx = B2 * dxr + bv2;
        if constexpr (EX) {
            R uL = u - dtr * (rs_S - lS) / dm;
            R v1L = v1 + dtr * (rs_s1 - ls1) / dm;
            R v2L = v2 + dtr * (rs_s2 - ls2) / dm;
            R eL = e - dtr * (rs_fe - lfe) / dm;
            R rhoL = dm / dxL;
            qL[0] = rhoL; qL[1] = rhoL * uL; qL[2] = rhoL * v1L; qL[3] = rhoL * v2L;
            qL[4] = B1dx / dxL; qL[5] = B2dx / dxL; qL[6] = rhoL * eL;
        } else {
            const R dtm = dtm_k, idxL = recip<R, EX>(dxL);     // dt / dm from P1 or P4
            idxL_k = idxL;
            R uL = u - (rs_S - lS) * dtm;
            R v1L = v1 + (rs_s1 - ls1) * dtm;
            R v2L = v2 + (rs_s2 - ls2) * dtm;
            R eL = e - (rs_fe - lfe) * dtm;
            R rhoL = imul<R, EX>(dm, idxL);
            qL[0] = rhoL; qL[1] = imul<R, EX>(rhoL, uL); qL[2] = imul<R, EX>(rhoL, v1L); qL[3] = imul<R, EX>(rhoL, v2L);
            qL[4] = imul<R, EX>(B1dx, idxL); qL[5] = imul<R, EX>(B2dx, idxL); qL[6] = imul<R, EX>(rhoL, eL);
        }
        dC[0] = negx<R, EX>(imul<R, EX>(dtr, rs_S - lS));
        dC[1] = imul<R, EX>(dtr, rs_s1 - ls1);
        dC[2] = imul<R, EX>(dtr, rs_s2 - ls2);
        dC[3] = bv1;
        dC[4] = bv2;
        dC[5] = negx<R, EX>(imul<R, EX>(dtr, rs_fe - lfe));
        del_p = imul<R, EX>(dtr, rs_u);
        del_m = imul<R, EX>(dtr, lu);
#pragma unroll
        for (int v = 0; v < 7; v++) SM(SB0 + v, s) = qL[v];
        SM(SB0 + 7, s) = dxL;
    }
    __syncthreads();

    // ---------------- P7: remap slopes ----------------
    R rmv[7];
    R rpv[7];                  // contracted forms: q_{i+1} - q_i, reused by the remap interface values (P8)
    if (act && p >= 5 && p <= NPe - 6) {
        SlopeCoef<R> k = slope_coef<R, EX>(SM(SB0 + 7, s - PS), dxL, SM(SB0 + 7, s + PS));
#pragma unroll
        for (int v = 0; v < 7; v++) {
            rmv[v] = limit_slope<R, EX>(SM(SB0 + v, s - PS), qL[v], SM(SB0 + v, s + PS), k.c1, k.c2, k.c3,
                                        EX ? nullptr : &rpv[v]);
            SM(v, s) = rmv[v];
        }
        if (a.steepen) {   // second difference of the Lagrangian density on the Lagrangian widths
            const R rl = SM(SB0, s - PS), rr = SM(SB0, s + PS), wl = SM(SB0 + 7, s - PS), wr = SM(SB0 + 7, s + PS);
            SM(NSM, s) = ((rr - qL[0]) / (wr + dxL) - (qL[0] - rl) / (dxL + wl)) / (wl + dxL + wr);
        }
    }
    __syncthreads();

    // ---------------- P8: remap interface values ----------------
    R red[7];
    R eta_k = 0;               // contact-steepening weight of this zone
    if (act && p >= 5 && p <= NPe - 7) {
        EdgeCoef<R> k = edge_coef<R, EX>(SM(SB0 + 7, s - PS), dxL, SM(SB0 + 7, s + PS), SM(SB0 + 7, s + 2 * PS));
#pragma unroll
        for (int v = 0; v < 7; v++) {
            if constexpr (EX) red[v] = edge_value<R, EX>(k, qL[v], SM(SB0 + v, s + PS), rmv[v], SM(v, s + PS));
            else red[v] = edge_value_d<R>(k, qL[v], rpv[v], rmv[v], SM(v, s + PS));
            SM(SC0 + v, s) = red[v];
        }
        if (a.steepen && p >= 6 && !shock_k) {   // contact weight of this zone
            const R dp2 = SM(NSM, s + PS), dm2 = SM(NSM, s - PS);
            const R rr = SM(SB0, s + PS), rl = SM(SB0, s - PS);
            const R dr = rr - rl;
            const R rmin = K<R>::ab(rr) < K<R>::ab(rl) ? K<R>::ab(rr) : K<R>::ab(rl);
            if (dp2 * dm2 < R(0) && K<R>::ab(dr) - R(ST_EPS) * rmin > R(0)) {
                const R wl = SM(SB0 + 7, s - PS), wr = SM(SB0 + 7, s + PS);
                const R xl = R(0.5) * (wl + dxL), xr = R(0.5) * (dxL + wr);
                const R et = -(dp2 - dm2) / dr * (xl * xl * xl + xr * xr * xr) / (xl + xr);
                R e = R(ST_ETA1) * (et - R(ST_ETA2));
                if (e < R(0)) e = R(0);
                if (e > R(1)) e = R(1);
                eta_k = e;
            }
        }
    }
    __syncthreads();

    // ---------------- P9: remap parabolas and donor fluxes ----------------
    if (act && p >= 6 && p <= NPe - 7) {
        // exact form: the constrained ends and a6; otherwise the one-sided
        // differences of the constrained parabola (pl, pr_ reused for them)
        R pl[7], pr_[7], p6[7];
#pragma unroll
        for (int v = 0; v < 7; v++) {
            pl[v] = SM(SC0 + v, s - PS);
            pr_[v] = red[v];
            if (gt0<R, EX>(eta_k)) {   // steepened ends: towards the neighbours' one-sided values
                const R ld = SM(SB0 + v, s - PS) + R(0.5) * SM(v, s - PS);
                const R rd = SM(SB0 + v, s + PS) - R(0.5) * SM(v, s + PS);
                pl[v] = pl[v] * (R(1) - eta_k) + eta_k * ld;
                pr_[v] = pr_[v] * (R(1) - eta_k) + eta_k * rd;
            }
            if constexpr (EX) p6[v] = monotone<R, EX>(qL[v], pl[v], pr_[v]);
            else monotone_d(qL[v], pl[v], pr_[v], pl[v], pr_[v]);
        }
        if (p <= NPe - 8) {                       // edge p+1/2: donor is this zone when del >= 0
            if (gt0<R, EX>(del_p)) {
                R y = EX ? del_p / dxL : imul<R, EX>(del_p, idxL_k);
                if (sliver_too_wide<R, EX>(y)) atomicOr(a.flags, FLAG_CFL);
                if constexpr (EX) {
#pragma unroll
                    for (int v = 0; v < 7; v++) SM(flux_slot(v), s) = del_p * avg_right<R>(pl[v], pr_[v], p6[v], y);
                } else {
                    const AvgCoef<R> k = avg_coef<R>(y);
#pragma unroll
                    for (int v = 0; v < 7; v++) SM(flux_slot(v), s) = imul<R, EX>(del_p, avg_right_d<R>(qL[v], pl[v], pr_[v], k));
                }
            } else if (!lt0<R, EX>(del_p)) {
#pragma unroll
                for (int v = 0; v < 7; v++) SM(flux_slot(v), s) = R(0);
            }
        }
        if (p >= 7 && lt0<R, EX>(del_m)) {       // edge p-1/2: donor is this zone when del < 0
            R y = EX ? -del_m / dxL : imul<R, EX>(negx<R, EX>(del_m), idxL_k);
            if (sliver_too_wide<R, EX>(y)) atomicOr(a.flags, FLAG_CFL);
            if constexpr (EX) {
#pragma unroll
                for (int v = 0; v < 7; v++) SM(flux_slot(v), s - PS) = del_m * avg_left<R>(pl[v], pr_[v], p6[v], y);
            } else {
                const AvgCoef<R> k = avg_coef<R>(y);
#pragma unroll
                for (int v = 0; v < 7; v++) SM(flux_slot(v), s - PS) = imul<R, EX>(del_m, avg_left_d<R>(qL[v], pl[v], pr_[v], k));
            }
        }
    }
    __syncthreads();

    // ---------------- P10: new state, sources, inner sphere, store ----------------
    if (out_cell) {
        const long long gi = base + (long long)g * stride;
        double Un[8];
        if (stage) {
            const int slot = stage_index<DIR>(l, p, NP, L), sv = stage_array_stride<DIR>(NP, L);
#pragma unroll
            for (int v = 0; v < 8; v++) Un[v] = stage[CHK(v * sv + slot, 8 * sv)];
        } else {
#pragma unroll
            for (int v = 0; v < 8; v++) Un[v] = __ldg(Uin + v * vs + CHK(gi, NCELL));
        }
        const int cmap[7] = {0, 1 + DIR, 1 + T1, 1 + T2, 4 + T1, 4 + T2, 7};
        const R dCv[7] = {R(0), dC[0], dC[1], dC[2], dC[3], dC[4], dC[5]};
        if constexpr (F64) {
            const double idx = EX ? 0.0 : (a.iw ? a.iw[CHK(g + GH, NG)] : 1.0 / dx);
#pragma unroll
            for (int v = 0; v < 7; v++) {
                double dU;
                if constexpr (EX) dU = (dCv[v] + SM(flux_slot(v), s - PS) - SM(flux_slot(v), s)) / dx;
                else if (v == 0) dU = (SM(flux_slot(v), s - PS) - SM(flux_slot(v), s)) * idx;   // no Lagrangian term
                else dU = (dCv[v] + SM(flux_slot(v), s - PS) - SM(flux_slot(v), s)) * idx;
                Un[cmap[v]] = Un[cmap[v]] + dU;
            }
            if (a.do_src) {
                const int mi[3] = {1 + DIR, 1 + T1, 1 + T2}, bi[3] = {4 + DIR, 4 + T1, 4 + T2};
#pragma unroll
                for (int m = 0; m < 3; m++) {
                    Un[mi[m]] = Un[mi[m]] + dt * src_m[m];
                    Un[bi[m]] = Un[bi[m]] + dt * src_b[m];
                }
                Un[7] = Un[7] + dt * src_e;
            }
        } else {
            const R idx = R(1) / a.wf[CHK(g + GH, NG)];
            R dU[8];
#pragma unroll
            for (int v = 0; v < 7; v++) dU[cmap[v]] = (dCv[v] + SM(flux_slot(v), s - PS) - SM(flux_slot(v), s)) * idx;
            dU[4 + DIR] = R(0);
            if (a.do_src) {
                dU[1 + DIR] += dtr * src_m[0]; dU[1 + T1] += dtr * src_m[1]; dU[1 + T2] += dtr * src_m[2];
                dU[4 + DIR] += dtr * src_b[0]; dU[4 + T1] += dtr * src_b[1]; dU[4 + T2] += dtr * src_b[2];
                dU[7] += dtr * src_e;
            }
#pragma unroll
            for (int v = 0; v < 8; v++) Un[v] = Un[v] + widen(dU[v]);
        }
        bool inner = false;
        if (a.inner_mask) {
            inner = a.inner_mask[CHK(gi, NCELL)] != 0;
        } else if constexpr (F64) {
            inner = a.r_inner > 0.0 &&
                    pos[0] * pos[0] + pos[1] * pos[1] + pos[2] * pos[2] < a.r_inner * a.r_inner;
        } else if (a.r_innerf > 0.0f) {
            // float test with an exact double test for centres within 1e-5 of the sphere
            const float px = a.cxf[CHK((DIR == 0 ? g : ix) + GH, NG0)], py = a.cyf[CHK((DIR == 1 ? g : iy) + GH, NG1)],
                        pz = a.czf[CHK((DIR == 2 ? g : iz) + GH, NG2)];
            const float r2 = px * px + py * py + pz * pz, ri2 = a.r_innerf * a.r_innerf;
            if (r2 < ri2 * (1.0f - 1e-5f)) inner = true;
            else if (r2 < ri2 * (1.0f + 1e-5f)) {
                const double x = a.cx[CHK((DIR == 0 ? g : ix) + GH, NG0)], y = a.cy[CHK((DIR == 1 ? g : iy) + GH, NG1)],
                             z = a.cz[CHK((DIR == 2 ? g : iz) + GH, NG2)];
                inner = x * x + y * y + z * z < a.r_inner * a.r_inner;
            }
        }
        if (inner && a.inner_cells) {     // the ionosphere's state of this cell
            int lo = 0, hi = a.n_inner - 1;
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (a.inner_cells[mid] < gi) lo = mid + 1; else hi = mid;
            }
            if (a.inner_cells[lo] == gi) {
#pragma unroll
                for (int v = 0; v < 8; v++) Un[v] = a.inner_state[(long long)v * a.n_inner + lo];
                inner = false;
            }
        }
        if (inner) {
            const auto *q = a.inner;
            double rh = q[0];
            Un[0] = rh;
            Un[1] = rh * q[1]; Un[2] = rh * q[2]; Un[3] = rh * q[3];
            Un[4] = 0.0; Un[5] = 0.0; Un[6] = 0.0;
            Un[7] = q[7] / (a.gamma - 1.0) + 0.5 * rh * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3])
                    + 0.5 * (0.0 * 0.0 + 0.0 * 0.0 + 0.0 * 0.0);
        }
        bool bad = false;
#pragma unroll
        for (int v = 0; v < 8; v++) {   // non-finite test on the exponent bits (integer pipe)
            bad |= ((__double2hiint(Un[v]) >> 20) & 0x7FF) == 0x7FF;
            Uout[v * vs + CHK(gi, NCELL)] = Un[v];
        }
        if (bad) atomicOr(a.flags, FLAG_NONFINITE);
    }
#undef SM
}

template <typename R> struct MaxThreads { static constexpr int value = MAXT; };
template <> struct MaxThreads<double> { static constexpr int value = MAXT_F64; };

// Box origin (x, y, z) of a tile.  y/z sweeps: lanes along x from xg * L,
// positions along the sweep axis from g0 - GH.  x sweep: positions from
// g0 - GH - 1 (even: C is even for this form), lanes = L consecutive pencils
// of one z plane (ny is a multiple of L for this form).
template <int DIR>
__device__ __forceinline__ void tile_box_origin(const SweepArgs &a, int tile, int &cx, int &cy, int &cz)
{
    const int chunk = tile % a.nchunk, grp = tile / a.nchunk;
    if (DIR == 0) {
        const int q = grp * a.L;
        cx = chunk * a.C - GH - 1;
        cy = q % a.n[1];
        cz = q / a.n[1];
        return;
    }
    const int xg = grp % a.ngx, t = grp / a.ngx;
    cx = xg * a.L;
    if (DIR == 1) { cy = chunk * a.C - GH; cz = t; }
    else { cy = t; cz = chunk * a.C - GH; }
}

// Resident blocks the TMA kernels are compiled for: the persistent loop
// otherwise roughly doubles the register allocation of the tile body.
template <typename R, bool PERSIST> struct TmaMinBlocks { static constexpr int value = 1; };
template <bool PERSIST> struct TmaMinBlocks<float, PERSIST> { static constexpr int value = 2; };
// The mixed ensemble's one-block-per-tile kernels are held to the same 64
// registers (two 512-thread blocks per SM): left free, the tile body takes
// 78-87 and the resident warps halve.
template <typename R> struct EnsMinBlocks { static constexpr int value = 1; };
template <> struct EnsMinBlocks<float> { static constexpr int value = 2; };

// Single domain, input staged by TMA (any direction).  PERSIST: each block
// takes tiles blockIdx.x, blockIdx.x + gridDim.x, ...; while it computes one
// tile, the tensor memory accelerator copies the next tile's input box (all 8
// state arrays, NP positions x L lanes) into the other of two shared buffers.
// Otherwise one tile per block: the box is copied at the start and the other
// resident blocks overlap it.  Waits are bounded: a block that gives up raises
// FLAG_TIMEOUT and returns.
template <int DIR, typename R, bool EX, bool PERSIST>
__global__ void __launch_bounds__(MaxThreads<R>::value, TmaMinBlocks<R, PERSIST>::value)
    sweep_tma_kernel(SweepArgs a, const __grid_constant__ CUtensorMap map)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long bar[2];
    const size_t stage_bytes = (size_t)8 * stage_array_stride<DIR>(a.NP, a.L) * sizeof(double);
    const size_t stage_pad = (stage_bytes + 1023) / 1024 * 1024;
    double *stage0 = reinterpret_cast<double *>(smem_raw);
    double *stage1 = reinterpret_cast<double *>(smem_raw + (PERSIST ? stage_pad : 0));
    unsigned char *work = smem_raw + (PERSIST ? 2 : 1) * stage_pad;
    const int ntiles = DIR == 0 ? a.nchunk * a.ngx : a.nchunk * a.ngx * (DIR == 1 ? a.n[2] : a.n[1]);
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    int t = blockIdx.x;
    if (t >= ntiles) return;
    if (threadIdx.x == 0) {
        int cx, cy, cz;
        tile_box_origin<DIR>(a, t, cx, cy, cz);
        mbar_expect_tx(&bar[0], (unsigned)stage_bytes);
        tma_load_4d(stage0, &map, cx, cy, cz, 0, &bar[0]);
    }
    if constexpr (!PERSIST) {                            // one tile per block, no loop
        // the tile waits for the box itself, after its geometry loads
        sweep_tile<DIR, R, EX, const SweepArgs>(a, t, work, 0, stage0, &bar[0]);
    } else {
    unsigned phase[2] = {0u, 0u};
    for (int k = 0; t < ntiles; k++, t += gridDim.x) {
        const int b = k & 1;
        const int tn = t + gridDim.x;
        if (PERSIST && threadIdx.x == 0 && tn < ntiles) {   // prefetch the next tile into the other buffer
            // the buffer's previous contents were read by every thread before
            // the barrier that ended the last iteration; order those reads
            // before the copy engine's writes
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            int cx, cy, cz;
            tile_box_origin<DIR>(a, tn, cx, cy, cz);
            mbar_expect_tx(&bar[b ^ 1], (unsigned)stage_bytes);
            tma_load_4d(b ? stage0 : stage1, &map, cx, cy, cz, 0, &bar[b ^ 1]);
        }
        if (!mbar_wait(&bar[b], phase[b])) {
            if (threadIdx.x == 0) atomicOr(a.flags, FLAG_TIMEOUT);
            // no further prefetch; drain this tile's copy and the next tile's,
            // issued above into the other buffer
            mbar_drain(&bar[b], phase[b]);
            if (tn < ntiles) mbar_drain(&bar[b ^ 1], phase[b ^ 1]);
            return;
        }
        phase[b] ^= 1u;
        sweep_tile<DIR, R, EX, const SweepArgs>(a, t, work, 0, b ? stage1 : stage0);
        __syncthreads();
    }
    }
}

// Register cap of the single-domain kernel: the tile-size limit's share of
// the register file, except for the contracted FP64 form, where a tighter
// cap (a few spilled values) lets two blocks of the usual tile shapes reside
// on an SM: 72 for y and z (2 x 416 threads; measured on GB300 at
// 256x192x192: 16.8 -> 15.9 ms per sweep), 96 for x (two blocks of 288
// threads, or one of two whole 256-cell pencils, 544 threads: each of the
// SM's four schedulers holds a quarter of its registers, so a block of 17 to
// 20 warps needs 5 x 32 x 96 <= 16384 registers per scheduler).
template <int DIR, typename R, bool EX> struct SweepRegCap {
    static constexpr int value = 65536 / MaxThreads<R>::value;
};
template <int DIR> struct SweepRegCap<DIR, double, false> {
    static constexpr int value = DIR == 0 ? 96 : 72;
};
static_assert(SweepRegCap<0, double, false>::value * 32 * ((MAXT_F64_X / 32 + 3) / 4) <= 16384,
              "FP64 x tile budget vs register cap (registers per scheduler)");
static_assert(SweepRegCap<1, double, false>::value * MAXT_F64 <= 65536, "FP64 tile budget vs register cap");

// Single domain: one block per tile.
template <int DIR, typename R, bool EX>
__global__ void __maxnreg__((SweepRegCap<DIR, R, EX>::value)) sweep_kernel(SweepArgs a)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    sweep_tile<DIR, R, EX, const SweepArgs>(a, blockIdx.x, smem_raw, 0);
}

// Ensemble: a persistent kernel.  Each block repeatedly takes the next tile
// from a global work counter (one atomic per tile, no waiting), finds the
// instance that owns it from the per-instance first-tile table and processes
// the tile with that instance's arguments (read-only device table).
// Instances of different sizes and boundary data share the launch.
template <int DIR, typename R, bool EX>
__global__ void __launch_bounds__(MaxThreads<R>::value) sweep_ensemble_kernel(EnsSweepArgs e)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ SweepArgs args;
    __shared__ int next, inst_cur;
    if (threadIdx.x == 0) inst_cur = -1;
    for (;;) {
        if (threadIdx.x == 0) next = (int)atomicAdd(e.queue, 1u);
        __syncthreads();
        const int t = next;
        const int cur = inst_cur;
        __syncthreads();
        if (t >= e.total_tiles) break;
        // instance owning tile t: last i with first_tile[i] <= t
        int lo = 0, hi = e.count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (__ldg(e.first_tile + mid) <= t) lo = mid; else hi = mid - 1;
        }
        if (lo != cur) {   // uniform across the block
            const int *src = reinterpret_cast<const int *>(e.args + lo);
            int *dst = reinterpret_cast<int *>(&args);
            for (int k = threadIdx.x; k < (int)(sizeof(SweepArgs) / sizeof(int)); k += blockDim.x) dst[k] = src[k];
            if (threadIdx.x == 0) inst_cur = lo;
            __syncthreads();
        }
        // read through a volatile view: each use is a shared-memory load
        // rather than a register held across the tile's phases
        const volatile SweepArgs &va = args;
        sweep_tile<DIR, R, EX, const volatile SweepArgs>(va, t - __ldg(e.first_tile + lo), smem_raw, e.flip);
        __syncthreads();
    }
}

// Ensemble, one block per tile: the block scheduler hands out (instance,
// tile) items in order; the block finds its instance from the first-tile
// table and copies that instance's arguments to shared memory.
template <int DIR, typename R, bool EX>
__global__ void __launch_bounds__(MaxThreads<R>::value, EnsMinBlocks<R>::value) sweep_ensemble_grid_kernel(EnsSweepArgs e)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ SweepArgs args;
    const int t = blockIdx.x;
    int lo = 0, hi = e.count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(e.first_tile + mid) <= t) lo = mid; else hi = mid - 1;
    }
    const int *src = reinterpret_cast<const int *>(e.args + lo);
    int *dst = reinterpret_cast<int *>(&args);
    for (int k = threadIdx.x; k < (int)(sizeof(SweepArgs) / sizeof(int)); k += blockDim.x) dst[k] = src[k];
    __syncthreads();
    sweep_tile<DIR, R, EX, const SweepArgs>(args, t - __ldg(e.first_tile + lo), smem_raw, e.flip);
}

// Ensemble, one block per tile with the tile's input box staged by TMA: the block finds its instance, copies its arguments to shared
// memory and loads the box through that instance's tensor map (maps[2 * i +
// b], b = the buffer holding the input: 0 = the instance's first state set,
// 1 = its second; the array lives in global memory, written before the
// launch).  The wait is bounded; a block that gives up raises FLAG_TIMEOUT.
template <int DIR, typename R, bool EX>
__global__ void __launch_bounds__(MaxThreads<R>::value, EnsMinBlocks<R>::value) sweep_ensemble_tma_kernel(EnsSweepArgs e,
                                                                                  const CUtensorMap *maps)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ SweepArgs args;
    __shared__ __align__(8) unsigned long long bar;
    const int t = blockIdx.x;
    int lo = 0, hi = e.count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(e.first_tile + mid) <= t) lo = mid; else hi = mid - 1;
    }
    const int *src = reinterpret_cast<const int *>(e.args + lo);
    int *dst = reinterpret_cast<int *>(&args);
    for (int k = threadIdx.x; k < (int)(sizeof(SweepArgs) / sizeof(int)); k += blockDim.x) dst[k] = src[k];
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const int tile = t - __ldg(e.first_tile + lo);
    const size_t stage_bytes = (size_t)8 * stage_array_stride<DIR>(args.NP, args.L) * sizeof(double);
    const size_t stage_pad = (stage_bytes + 1023) / 1024 * 1024;
    double *stage = reinterpret_cast<double *>(smem_raw);
    if (threadIdx.x == 0) {
        int cx, cy, cz;
        tile_box_origin<DIR>(args, tile, cx, cy, cz);
        mbar_expect_tx(&bar, (unsigned)stage_bytes);
        tma_load_4d(stage, maps + 2 * lo + e.flip, cx, cy, cz, 0, &bar);
    }
    sweep_tile<DIR, R, EX, const SweepArgs>(args, tile, smem_raw + stage_pad, e.flip, stage, &bar);
}

// Ensemble, one block per tile with the tile's input box staged by TMA and
// every instance's arguments in the kernel parameter (constant bank): the
// block finds its instance by a search in the parameter space, thread 0
// issues the box copy at once, and the tile loads its geometry while the copy
// is in flight (no per-block copy of the arguments, no device-table search).
template <int DIR, typename R, bool EX>
__global__ void __launch_bounds__(MaxThreads<R>::value, EnsMinBlocks<R>::value)
    sweep_ensemble_tma_param_kernel(const __grid_constant__ EnsSweepParams p, const CUtensorMap *maps)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long bar;
    const int t = blockIdx.x;
    int lo = 0, hi = p.count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.first_tile[mid] <= t) lo = mid; else hi = mid - 1;
    }
    const SweepArgs &a = p.args[lo];
    const int tile = t - p.first_tile[lo];
    const size_t stage_bytes = (size_t)8 * stage_array_stride<DIR>(a.NP, a.L) * sizeof(double);
    const size_t stage_pad = (stage_bytes + 1023) / 1024 * 1024;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        int cx, cy, cz;
        tile_box_origin<DIR>(a, tile, cx, cy, cz);
        mbar_expect_tx(&bar, (unsigned)stage_bytes);
        tma_load_4d(smem_raw, maps + 2 * lo + p.flip, cx, cy, cz, 0, &bar);
    }
    __syncthreads();                           // the mbarrier is initialised before anyone waits on it
    sweep_tile<DIR, R, EX, const SweepArgs>(a, tile, smem_raw + stage_pad, p.flip,
                                            reinterpret_cast<const double *>(smem_raw), &bar);
}

// Ensemble, one block per tile, arguments of all instances in the kernel
// parameter (constant bank): the block finds its instance from the first-tile
// table and reads that instance's fields straight from the parameter space.
template <int DIR, typename R, bool EX>
__global__ void __launch_bounds__(MaxThreads<R>::value, EnsMinBlocks<R>::value) sweep_ensemble_param_kernel(const __grid_constant__ EnsSweepParams p)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int t = blockIdx.x;
    int lo = 0, hi = p.count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p.first_tile[mid] <= t) lo = mid; else hi = mid - 1;
    }
    sweep_tile<DIR, R, EX, const SweepArgs>(p.args[lo], t - p.first_tile[lo], smem_raw, p.flip);
}

// Ensemble, persistent blocks with all instances' arguments in the kernel
// parameter: each block repeatedly takes the next tile from the work counter
// (one atomic per tile, no waiting), finds its instance from the first-tile
// table and runs the tile with that instance's fields read straight from the
// parameter space (no per-block copy of the arguments, so the tile body keeps
// the one-block-per-tile form's register budget).
template <int DIR, typename R, bool EX>
__global__ void __launch_bounds__(MaxThreads<R>::value, EnsMinBlocks<R>::value)
    sweep_ensemble_param_persist_kernel(const __grid_constant__ EnsSweepParams p, unsigned int *queue)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    __shared__ int next;
    for (;;) {
        if (threadIdx.x == 0) next = (int)atomicAdd(queue, 1u);
        __syncthreads();
        const int t = next;
        __syncthreads();                       // every thread has read `next` before it is rewritten
        if (t >= p.total_tiles) break;
        int lo = 0, hi = p.count - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (p.first_tile[mid] <= t) lo = mid; else hi = mid - 1;
        }
        sweep_tile<DIR, R, EX, const SweepArgs>(p.args[lo], t - p.first_tile[lo], smem_raw, p.flip);
        __syncthreads();                       // the tile's shared memory is free again
    }
}

// Dipole table of a single domain (FP64 forms): B_d at every cell centre,
// component k at bd + k * vs + cell, evaluated by the same dipole<EX> as the
// sweeps evaluate on the fly (ghost cells still do).
template <bool EX>
__global__ void dipole_table_kernel(double M, int nx, int ny, int nz, const double *cx, const double *cy,
                                    const double *cz, double *bd, long long vs)
{
    const long long ncell = (long long)nx * ny * nz;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < ncell;
         i += (long long)gridDim.x * blockDim.x) {
        const int ix = (int)(i % nx), iy = (int)((i / nx) % ny), iz = (int)(i / ((long long)nx * ny));
        double B[3];
        dipole<EX>(M, cx[ix + GH], cy[iy + GH], cz[iz + GH], B);
        bd[i] = B[0];
        bd[vs + i] = B[1];
        bd[2 * vs + i] = B[2];
    }
}

}  // namespace ppmlr
