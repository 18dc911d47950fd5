// Arithmetic-pipe rates of the GPU the library runs on: the denominators of
// the FP64 "alu" roofline of the sweeps.  Each thread runs eight independent
// dependency chains of one operation so that the pipe, not the latency of a
// chain, sets the rate; 8 blocks of 256 threads per SM; CUDA events on the
// caller's stream around one launch after a warm-up launch.
#include "sweep.cuh"

namespace ppmlr {
namespace {

// OP_IMUL: the integer-pipe double product of the contracted FP64 sweeps
// (dmul_int); OP_MIX: four chains of FP64 FMAs beside four of dmul_int
enum PipeOp { OP_DFMA = 0, OP_DADD = 1, OP_FFMA = 2, OP_IMUL = 3, OP_MIX = 4 };

template <int OP>
__global__ void __launch_bounds__(256) pipe_chains_kernel(double *out, int iters, double seed)
{
    double a[8];
    float f[8];
#pragma unroll
    for (int k = 0; k < 8; k++) {
        a[k] = seed + threadIdx.x * 1e-3 + k;
        f[k] = (float)(seed + k);
    }
    const double m = 0.999999, c = 1e-7;
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < 8; k++) {
            if (OP == OP_DFMA) a[k] = fma(a[k], m, c);
            if (OP == OP_DADD) a[k] = a[k] + c;
            if (OP == OP_IMUL) a[k] = dmul_int(a[k], m);
            if (OP == OP_MIX) a[k] = (k & 1) ? dmul_int(a[k], m) : fma(a[k], m, c);
            if (OP == OP_FFMA) {
#pragma unroll
                for (int r = 0; r < 8; r++) f[k] = fmaf(f[k], 0.999f, 1e-3f);
            }
        }
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < 8; k++) s += a[k] + f[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int OP>
cudaError_t time_chains(double *out, int blocks, int iters, cudaStream_t s, float *ms)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        pipe_chains_kernel<OP><<<blocks, 256, 0, s>>>(out, 16, 1.0);      // warm-up
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
        pipe_chains_kernel<OP><<<blocks, 256, 0, s>>>(out, iters, 1.0);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return e;
}

}  // namespace
}  // namespace ppmlr

using namespace ppmlr;

extern "C" ppmlr_status ppmlr_measure_pipe_rates(void *cuda_stream, double rates[3])
{
    if (!rates) return PPMLR_E_INVALID;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return PPMLR_E_CUDA;
    const int blocks = 8 * sms, threads = 256;
    double *out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * blocks * threads) != cudaSuccess) return PPMLR_E_OOM;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int iters[3] = {4000, 4000, 1000};
    const double ops_per_iter[3] = {8, 8, 64};
    ppmlr_status st = PPMLR_OK;
    for (int op = 0; op < 3 && st == PPMLR_OK; op++) {
        float ms = 0.0f;
        cudaError_t e = op == OP_DFMA   ? time_chains<OP_DFMA>(out, blocks, iters[op], s, &ms)
                        : op == OP_DADD ? time_chains<OP_DADD>(out, blocks, iters[op], s, &ms)
                                        : time_chains<OP_FFMA>(out, blocks, iters[op], s, &ms);
        if (e != cudaSuccess || !(ms > 0.0f)) st = PPMLR_E_CUDA;
        else rates[op] = ops_per_iter[op] * iters[op] * (double)blocks * threads / (ms * 1e-3);
    }
    cudaFree(out);
    return st;
}

extern "C" ppmlr_status ppmlr_measure_coissue(void *cuda_stream, double rates[2])
{
    if (!rates) return PPMLR_E_INVALID;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
        return PPMLR_E_CUDA;
    const int blocks = 8 * sms, threads = 256, iters = 2000;
    double *out = nullptr;
    if (cudaMalloc(&out, sizeof(double) * blocks * threads) != cudaSuccess) return PPMLR_E_OOM;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    ppmlr_status st = PPMLR_OK;
    for (int k = 0; k < 2 && st == PPMLR_OK; k++) {
        float ms = 0.0f;
        cudaError_t e = k == 0 ? time_chains<OP_IMUL>(out, blocks, iters, s, &ms)
                               : time_chains<OP_MIX>(out, blocks, iters, s, &ms);
        if (e != cudaSuccess || !(ms > 0.0f)) st = PPMLR_E_CUDA;
        else rates[k] = 8.0 * iters * (double)blocks * threads / (ms * 1e-3);
    }
    cudaFree(out);
    return st;
}
