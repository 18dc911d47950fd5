// Arithmetic-pipe rates of this GPU, the denominators of the "alu" roofline
// that bench.py reports for the FP64 sweeps: FP64 fused multiply-add, add and
// multiply (one instruction each), FP64 division, square root and reciprocal
// square root (several instruction slots each), FP32 fused multiply-add, and a double->float->double
// round trip (the conversions also run on the FP64 pipe).
//
// Every thread runs eight independent dependency chains so that the pipe, not
// the latency of one chain, sets the rate; the grid is 8 blocks of 256
// threads per SM.  Build and run on the GPU:
//   nvcc -gencode arch=compute_103a,code=sm_103a -O3 -o fp64_rate bench_fp64_rate.cu && ./fp64_rate
#include <cstdio>

#include <cuda_runtime.h>

#define CK(x)                                                                          \
    do {                                                                               \
        cudaError_t e_ = (x);                                                          \
        if (e_ != cudaSuccess) {                                                       \
            std::printf("CUDA error %s at line %d\n", cudaGetErrorString(e_), __LINE__); \
            return 1;                                                                  \
        }                                                                              \
    } while (0)

enum Op { DFMA, DADD, DMUL, DDIV, DSQRT, DRSQRT, FFMA, F2F };

template <int OP>
__global__ void chains(double *out, int iters, double seed)
{
    double a[8];
    float f[8];
    for (int k = 0; k < 8; k++) { a[k] = seed + threadIdx.x * 1e-3 + k; f[k] = (float)a[k]; }
    const double m = 0.999999, c = 1e-7;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < 8; k++) {
            if (OP == DFMA) a[k] = fma(a[k], m, c);
            if (OP == DADD) a[k] = a[k] + c;
            if (OP == DMUL) a[k] = a[k] * m;
            if (OP == DDIV) a[k] = c + 1.0 / a[k];
            if (OP == DSQRT) a[k] = sqrt(a[k]) + c;
            if (OP == DRSQRT) a[k] = rsqrt(a[k]) + 1.0;
            if (OP == FFMA) {
#pragma unroll
                for (int r = 0; r < 8; r++) f[k] = fmaf(f[k], 0.999f, 1e-3f);
            }
            if (OP == F2F) { f[k] = (float)a[k]; a[k] = (double)f[k] * m; }
        }
    }
    double s = 0.0;
    for (int k = 0; k < 8; k++) s += a[k] + f[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int OP>
int measure(const char *name, double ops_per_iter, int iters, int blocks, int threads, double *out, double sms)
{
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    chains<OP><<<blocks, threads>>>(out, 10, 1.0);      // warm-up
    CK(cudaDeviceSynchronize());
    CK(cudaEventRecord(e0));
    chains<OP><<<blocks, threads>>>(out, iters, 1.0);
    CK(cudaEventRecord(e1));
    CK(cudaEventSynchronize(e1));
    float ms = 0.0f;
    CK(cudaEventElapsedTime(&ms, e0, e1));
    int khz = 0;
    CK(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, 0));
    const double ops = ops_per_iter * iters * (double)blocks * threads;
    const double rate = ops / (ms * 1e-3);
    std::printf("%-6s %9.3f ms  %9.1f G op/s  %6.2f op per SM per clock (at %d MHz)\n", name, ms, rate * 1e-9,
                rate / (sms * khz * 1e3), khz / 1000);
    CK(cudaEventDestroy(e0));
    CK(cudaEventDestroy(e1));
    return 0;
}

int main()
{
    cudaDeviceProp p;
    CK(cudaGetDeviceProperties(&p, 0));
    std::printf("%s, %d SMs\n", p.name, p.multiProcessorCount);
    const int blocks = p.multiProcessorCount * 8, threads = 256;
    double *out = nullptr;
    CK(cudaMalloc(&out, sizeof(double) * blocks * threads));
    const double sms = p.multiProcessorCount;
    int rc = 0;
    rc |= measure<DFMA>("DFMA", 8, 2000, blocks, threads, out, sms);
    rc |= measure<DADD>("DADD", 8, 2000, blocks, threads, out, sms);
    rc |= measure<DMUL>("DMUL", 8, 2000, blocks, threads, out, sms);
    rc |= measure<DDIV>("DDIV", 8, 200, blocks, threads, out, sms);
    rc |= measure<DSQRT>("DSQRT", 8, 200, blocks, threads, out, sms);
    rc |= measure<DRSQRT>("DRSQRT", 8, 200, blocks, threads, out, sms);
    rc |= measure<FFMA>("FFMA", 64, 2000, blocks, threads, out, sms);
    rc |= measure<F2F>("F2F", 8, 2000, blocks, threads, out, sms);   // round trips: two conversions and a DMUL each
    CK(cudaFree(out));
    return rc;
}
