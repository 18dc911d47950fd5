// FP64 sweep kernels, default form: IEEE double throughout, compiled with
// contraction (fused multiply-add) and one reciprocal per shared denominator;
// products, reciprocals and square roots partly on the integer and FP32 pipes
// (each correctly rounded), sign flips and compares on the bit patterns.
// Agrees with the CPU reference to roundoff (parity bar: relative L1 1e-11).
#include "launch.cuh"

namespace ppmlr {
const SweepLaunchers k_sweep_fp64 = SweepVariant<double, false>::table();

namespace {

// Error, in ulps of the correctly rounded result, of this form's square root
// and reciprocal over n arguments x = (1 + f) 2^e, e cycling over
// -1000..1000 and f from a Weyl sequence, every fourth argument an exact
// square s^2 2^(2j) instead (s a 26-bit integer, 2j = e - 52 with e first
// made even toward zero) moved by -3..3 units in its last place, so that
// the root is exact or lies within a fraction of an ulp of s 2^j: out[0]
// square root, out[1] reciprocal (non-negative doubles compared as their
// bit patterns), out[2] the arguments whose square root differs from the
// correctly rounded one, out[3] the pairs (x, y) whose integer-pipe product
// differs from the IEEE product; y = (1 + f') 2^e', e' cycling over
// -500..500, or for every fourth pair x = 1 + k 2^-52 (k < 2^10) and
// y = (2c + 1) 2^-8 (c < 2^8), products whose discarded bits are often
// exactly one half (ties).
__global__ void __launch_bounds__(256) arith_selftest_kernel(long long n, unsigned long long *out)
{
    double m_sqrt = 0.0, m_rcp = 0.0;
    unsigned long long wrong = 0, wrong_mul = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int ex = (int)(i % 2001) - 1000;
        const double f = (double)(((unsigned long long)i * 0x9E3779B97F4A7C15ULL) >> 11) * 0x1.0p-53;
        double x = ldexp(1.0 + f, ex);
        if ((i & 3) == 3) {
            const unsigned long long q = (1ull << 25) + ((((unsigned long long)i * 0x2545F4914F6CDD1DULL) >> 20) &
                                                         ((1ull << 25) - 1));
            const double sq = ldexp((double)(q * q), 2 * (ex / 2) - 52);     // q^2 < 2^52: exact; sq < 2^1000
            x = __longlong_as_double(__double_as_longlong(sq) + (i % 7) - 3);
        }
        const double s = fsqrt<double, false>(x), s_ref = sqrt(x);
        const double r = recip<double, false>(x), r_ref = 1.0 / x;
        m_sqrt = fmax(m_sqrt, fabs(s - s_ref) / ldexp(1.0, ilogb(s_ref) - 52));
        m_rcp = fmax(m_rcp, fabs(r - r_ref) / ldexp(1.0, ilogb(r_ref) - 52));
        wrong += __double_as_longlong(s) != __double_as_longlong(s_ref);
        const unsigned long long h = (unsigned long long)i * 0xD1B54A32D192ED03ULL;
        double xa = ldexp(1.0 + f, ex / 2), ya = ldexp(1.0 + (double)(h >> 11) * 0x1.0p-53, (int)(h % 1001) - 500);
        if ((i & 3) == 1) {
            xa = 1.0 + (double)((h >> 20) & 1023) * 0x1.0p-52;
            ya = (double)(2 * ((h >> 40) & 255) + 1) * 0x1.0p-8;
        }
        if ((i & 8) != 0) xa = -xa;
        wrong_mul += __double_as_longlong(dmul_int(xa, ya)) != __double_as_longlong(__dmul_rn(xa, ya));
    }
    atomicMax(out, (unsigned long long)__double_as_longlong(m_sqrt));
    atomicMax(out + 1, (unsigned long long)__double_as_longlong(m_rcp));
    atomicAdd(out + 2, wrong);
    atomicAdd(out + 3, wrong_mul);
}

}  // namespace
}  // namespace ppmlr

extern "C" ppmlr_status ppmlr_selftest_fp64_arith(void *cuda_stream, long long n, double max_ulp[4])
{
    if (!max_ulp || n < 1) return PPMLR_E_INVALID;
    unsigned long long *d = nullptr, h[4] = {0, 0, 0, 0};   // max ulp bits (2), mismatch counts (2)
    if (cudaMalloc(&d, sizeof(h)) != cudaSuccess) return PPMLR_E_OOM;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(h), s);
    if (e == cudaSuccess) {
        const long long want = (n + 255) / 256;
        ppmlr::arith_selftest_kernel<<<(unsigned)(want < 4096 ? want : 4096), 256, 0, s>>>(n, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    if (e != cudaSuccess) return PPMLR_E_CUDA;
    for (int k = 0; k < 2; k++) memcpy(&max_ulp[k], &h[k], sizeof(double));
    max_ulp[2] = (double)h[2];
    max_ulp[3] = (double)h[3];
    return PPMLR_OK;
}
