// FP64 sweep kernels, default form: IEEE double throughout, compiled with
// contraction (fused multiply-add) and one reciprocal per shared denominator.
// Agrees with the CPU reference to roundoff (parity bar: relative L1 1e-11).
#include "launch.cuh"

namespace ppmlr {
const SweepLaunchers k_sweep_fp64 = SweepVariant<double, false>::table();

namespace {

// Error, in ulps of the correctly rounded result, of this form's square root
// and reciprocal over n arguments x = (1 + f) 2^e, e cycling over
// -1000..1000 and f from a Weyl sequence: out[0] square root, out[1]
// reciprocal (non-negative doubles compared as their bit patterns).
__global__ void __launch_bounds__(256) arith_selftest_kernel(long long n, unsigned long long *out)
{
    double m_sqrt = 0.0, m_rcp = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const int ex = (int)(i % 2001) - 1000;
        const double f = (double)(((unsigned long long)i * 0x9E3779B97F4A7C15ULL) >> 11) * 0x1.0p-53;
        const double x = ldexp(1.0 + f, ex);
        const double s = fsqrt<double, false>(x), s_ref = sqrt(x);
        const double r = recip<double, false>(x), r_ref = 1.0 / x;
        m_sqrt = fmax(m_sqrt, fabs(s - s_ref) / ldexp(1.0, ilogb(s_ref) - 52));
        m_rcp = fmax(m_rcp, fabs(r - r_ref) / ldexp(1.0, ilogb(r_ref) - 52));
    }
    atomicMax(out, (unsigned long long)__double_as_longlong(m_sqrt));
    atomicMax(out + 1, (unsigned long long)__double_as_longlong(m_rcp));
}

}  // namespace
}  // namespace ppmlr

extern "C" ppmlr_status ppmlr_selftest_fp64_arith(void *cuda_stream, long long n, double max_ulp[2])
{
    if (!max_ulp || n < 1) return PPMLR_E_INVALID;
    unsigned long long *d = nullptr, h[2] = {0, 0};
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
    return PPMLR_OK;
}
