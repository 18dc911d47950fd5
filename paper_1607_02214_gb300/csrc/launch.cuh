// Launchers of the sweep kernels for one arithmetic variant (R, EX); each
// kernel translation unit instantiates one variant with its own compiler
// flags and exports a SweepLaunchers table.
#pragma once
#include "march.cuh"
#include "sweep.cuh"

namespace ppmlr {

template <typename R, bool EX>
struct SweepVariant {
    template <int DIR>
    static cudaError_t single_dir(const SweepArgs &a, const Tile &t, cudaStream_t s)
    {
        static bool attr = false;
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(sweep_kernel<DIR, R, EX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 227 * 1024);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        sweep_kernel<DIR, R, EX><<<t.ntiles, t.threads, t.smem, s>>>(a);
        return cudaGetLastError();
    }
    template <int DIR>
    static cudaError_t ens_dir(const EnsSweepArgs &e, int blocks, int threads, size_t smem, cudaStream_t s)
    {
        // (the shared-memory attribute is set by per_sm_dir, which planning always calls first)
        if (blocks == e.total_tiles) {   // one block per tile
            sweep_ensemble_grid_kernel<DIR, R, EX><<<blocks, threads, smem, s>>>(e);
            return cudaGetLastError();
        }
        sweep_ensemble_kernel<DIR, R, EX><<<blocks, threads, smem, s>>>(e);
        return cudaGetLastError();
    }
    template <int DIR>
    static cudaError_t param_dir(const EnsSweepParams &p, int blocks, int threads, size_t smem, cudaStream_t s)
    {
        static bool attr = false;
        if (!attr) {
            cudaError_t r = cudaFuncSetAttribute(sweep_ensemble_param_kernel<DIR, R, EX>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            if (r != cudaSuccess) return r;
            attr = true;
        }
        sweep_ensemble_param_kernel<DIR, R, EX><<<blocks, threads, smem, s>>>(p);
        return cudaGetLastError();
    }
    template <int DIR>
    static cudaError_t param_persist_dir(const EnsSweepParams &p, unsigned int *queue, int blocks, int threads,
                                         size_t smem, cudaStream_t s)
    {
        static bool attr = false;
        if (!attr) {
            cudaError_t r = cudaFuncSetAttribute(sweep_ensemble_param_persist_kernel<DIR, R, EX>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
            if (r != cudaSuccess) return r;
            attr = true;
        }
        sweep_ensemble_param_persist_kernel<DIR, R, EX><<<blocks, threads, smem, s>>>(p, queue);
        return cudaGetLastError();
    }
    template <int DIR>
    static int param_persist_per_sm_dir(int threads, size_t smem)
    {
        cudaFuncSetAttribute(sweep_ensemble_param_persist_kernel<DIR, R, EX>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_ensemble_param_persist_kernel<DIR, R, EX>,
                                                          threads, smem) != cudaSuccess)
            return 1;
        return n > 0 ? n : 1;
    }
    static cudaError_t param_persist(int dir, const EnsSweepParams &p, unsigned int *queue, int blocks, int threads,
                                     size_t smem, cudaStream_t s)
    {
        return dir == 0 ? param_persist_dir<0>(p, queue, blocks, threads, smem, s)
               : dir == 1 ? param_persist_dir<1>(p, queue, blocks, threads, smem, s)
                          : param_persist_dir<2>(p, queue, blocks, threads, smem, s);
    }
    static int param_persist_per_sm(int dir, int threads, size_t smem)
    {
        return dir == 0 ? param_persist_per_sm_dir<0>(threads, smem)
               : dir == 1 ? param_persist_per_sm_dir<1>(threads, smem) : param_persist_per_sm_dir<2>(threads, smem);
    }
    template <int DIR>
    static int per_sm_dir(int threads, size_t smem)
    {
        cudaFuncSetAttribute(sweep_ensemble_kernel<DIR, R, EX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024);
        cudaFuncSetAttribute(sweep_ensemble_grid_kernel<DIR, R, EX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             200 * 1024);
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_ensemble_kernel<DIR, R, EX>, threads, smem) !=
            cudaSuccess)
            return 1;
        return n > 0 ? n : 1;
    }
    // dynamic shared memory up to the 227 KB per block less the kernel's
    // static part (its mbarriers)
    template <int DIR, bool P>
    static cudaError_t allow_tma_smem()
    {
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, sweep_tma_kernel<DIR, R, EX, P>);
        if (e != cudaSuccess) return e;
        return cudaFuncSetAttribute(sweep_tma_kernel<DIR, R, EX, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    227 * 1024 - (int)fa.sharedSizeBytes);
    }
    template <int DIR, bool P>
    static cudaError_t tma_dir(const SweepArgs &a, const CUtensorMap &map, int blocks, int threads, size_t smem,
                               cudaStream_t s)
    {
        static bool attr = false;
        if (!attr) {
            cudaError_t e = allow_tma_smem<DIR, P>();
            if (e != cudaSuccess) return e;
            attr = true;
        }
        sweep_tma_kernel<DIR, R, EX, P><<<blocks, threads, smem, s>>>(a, map);
        return cudaGetLastError();
    }
    template <int DIR, bool P>
    static int tma_per_sm_dir(int threads, size_t smem)
    {
        if (allow_tma_smem<DIR, P>() != cudaSuccess) return 0;
        int n = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_tma_kernel<DIR, R, EX, P>, threads, smem) !=
            cudaSuccess)
            return 0;
        return n;
    }
    // persist: 1 = persistent double-buffered, 0 = one tile per block
    static cudaError_t tma(int dir, int persist, const SweepArgs &a, const CUtensorMap &map, int blocks,
                           int threads, size_t smem, cudaStream_t s)
    {
        if (persist)
            return dir == 1 ? tma_dir<1, true>(a, map, blocks, threads, smem, s)
                   : dir == 2 ? tma_dir<2, true>(a, map, blocks, threads, smem, s)
                              : cudaErrorInvalidValue;      // x: one tile per block only
        return dir == 0 ? tma_dir<0, false>(a, map, blocks, threads, smem, s)
               : dir == 1 ? tma_dir<1, false>(a, map, blocks, threads, smem, s)
                          : tma_dir<2, false>(a, map, blocks, threads, smem, s);
    }
    // ensemble y/z sweep with TMA-staged input boxes (one block per tile)
    template <int DIR>
    static cudaError_t allow_ens_tma_smem()
    {
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, sweep_ensemble_tma_kernel<DIR, R, EX>);
        if (e != cudaSuccess) return e;
        return cudaFuncSetAttribute(sweep_ensemble_tma_kernel<DIR, R, EX>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024 - (int)fa.sharedSizeBytes);
    }
    static cudaError_t ens_tma(int dir, const EnsSweepArgs &e, const CUtensorMap *maps, int blocks, int threads,
                               size_t smem, cudaStream_t s)
    {
        static bool attr[3] = {false, false, false};
        if (dir < 0 || dir > 2) return cudaErrorInvalidValue;
        if (!attr[dir]) {
            cudaError_t r = dir == 0 ? allow_ens_tma_smem<0>() : dir == 1 ? allow_ens_tma_smem<1>()
                                                                          : allow_ens_tma_smem<2>();
            if (r != cudaSuccess) return r;
            attr[dir] = true;
        }
        if (dir == 0) sweep_ensemble_tma_kernel<0, R, EX><<<blocks, threads, smem, s>>>(e, maps);
        else if (dir == 1) sweep_ensemble_tma_kernel<1, R, EX><<<blocks, threads, smem, s>>>(e, maps);
        else sweep_ensemble_tma_kernel<2, R, EX><<<blocks, threads, smem, s>>>(e, maps);
        return cudaGetLastError();
    }
    template <int DIR>
    static int ens_tma_per_sm_dir(int threads, size_t smem)
    {
        if (allow_ens_tma_smem<DIR>() != cudaSuccess) return 0;
        int n = 0;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_ensemble_tma_kernel<DIR, R, EX>, threads,
                                                             smem) == cudaSuccess ? n : 0;
    }
    static int ens_tma_per_sm(int dir, int threads, size_t smem)
    {
        return dir == 0 ? ens_tma_per_sm_dir<0>(threads, smem)
               : dir == 1 ? ens_tma_per_sm_dir<1>(threads, smem) : ens_tma_per_sm_dir<2>(threads, smem);
    }
    // ensemble, one block per tile, TMA-staged box, arguments in the kernel parameter
    template <int DIR>
    static cudaError_t allow_ens_tma_param_smem()
    {
        cudaFuncAttributes fa;
        cudaError_t e = cudaFuncGetAttributes(&fa, sweep_ensemble_tma_param_kernel<DIR, R, EX>);
        if (e != cudaSuccess) return e;
        return cudaFuncSetAttribute(sweep_ensemble_tma_param_kernel<DIR, R, EX>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024 - (int)fa.sharedSizeBytes);
    }
    template <int DIR>
    static cudaError_t ens_tma_param_dir(const EnsSweepParams &p, const CUtensorMap *maps, int blocks, int threads,
                                         size_t smem, cudaStream_t s)
    {
        static bool attr = false;
        if (!attr) {
            cudaError_t r = allow_ens_tma_param_smem<DIR>();
            if (r != cudaSuccess) return r;
            attr = true;
        }
        sweep_ensemble_tma_param_kernel<DIR, R, EX><<<blocks, threads, smem, s>>>(p, maps);
        return cudaGetLastError();
    }
    static cudaError_t ens_tma_param(int dir, const EnsSweepParams &p, const CUtensorMap *maps, int blocks,
                                     int threads, size_t smem, cudaStream_t s)
    {
        return dir == 0 ? ens_tma_param_dir<0>(p, maps, blocks, threads, smem, s)
               : dir == 1 ? ens_tma_param_dir<1>(p, maps, blocks, threads, smem, s)
                          : ens_tma_param_dir<2>(p, maps, blocks, threads, smem, s);
    }
    template <int DIR>
    static int ens_tma_param_per_sm_dir(int threads, size_t smem)
    {
        if (allow_ens_tma_param_smem<DIR>() != cudaSuccess) return 0;
        int n = 0;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_ensemble_tma_param_kernel<DIR, R, EX>,
                                                             threads, smem) == cudaSuccess ? n : 0;
    }
    static int ens_tma_param_per_sm(int dir, int threads, size_t smem)
    {
        if (threads > MaxThreads<R>::value) return 0;
        return dir == 0 ? ens_tma_param_per_sm_dir<0>(threads, smem)
               : dir == 1 ? ens_tma_param_per_sm_dir<1>(threads, smem) : ens_tma_param_per_sm_dir<2>(threads, smem);
    }
    static cudaError_t dipole_table(double M, const int n[3], const double *cx, const double *cy, const double *cz,
                                    double *bd, long long vs, cudaStream_t s)
    {
        if constexpr (std::is_same<R, double>::value) {
            const long long ncell = (long long)n[0] * n[1] * n[2];
            long long blocks = (ncell + 255) / 256;
            if (blocks > 152 * 16) blocks = 152 * 16;
            dipole_table_kernel<EX><<<(int)blocks, 256, 0, s>>>(M, n[0], n[1], n[2], cx, cy, cz, bd, vs);
            return cudaGetLastError();
        } else {
            return cudaErrorNotSupported;
        }
    }
    template <int DIR>
    static cudaError_t march_dir(const SweepArgs &a, cudaStream_t s)
    {
        const int warps = march_warps(a, DIR);
        const int blocks = (warps + MARCH_WARPS - 1) / MARCH_WARPS;
        sweep_march_kernel<DIR><<<blocks, 32 * MARCH_WARPS, march_smem_bytes(), s>>>(a);
        return cudaGetLastError();
    }
    static cudaError_t march(int dir, const SweepArgs &a, cudaStream_t s)
    {
        if constexpr (std::is_same<R, float>::value && !EX)
            return dir == 0 ? march_dir<0>(a, s) : dir == 1 ? march_dir<1>(a, s) : march_dir<2>(a, s);
        else
            return cudaErrorNotSupported;
    }
    static int tma_per_sm(int dir, int persist, int threads, size_t smem)
    {
        if (persist)
            return dir == 1 ? tma_per_sm_dir<1, true>(threads, smem)
                   : dir == 2 ? tma_per_sm_dir<2, true>(threads, smem) : 0;
        return dir == 0 ? tma_per_sm_dir<0, false>(threads, smem)
               : dir == 1 ? tma_per_sm_dir<1, false>(threads, smem) : tma_per_sm_dir<2, false>(threads, smem);
    }
    static cudaError_t single(int dir, const SweepArgs &a, const Tile &t, cudaStream_t s)
    {
        return dir == 0 ? single_dir<0>(a, t, s) : dir == 1 ? single_dir<1>(a, t, s) : single_dir<2>(a, t, s);
    }
    static cudaError_t ens(int dir, const EnsSweepArgs &e, int blocks, int threads, size_t smem, cudaStream_t s)
    {
        return dir == 0 ? ens_dir<0>(e, blocks, threads, smem, s)
                        : dir == 1 ? ens_dir<1>(e, blocks, threads, smem, s) : ens_dir<2>(e, blocks, threads, smem, s);
    }
    static cudaError_t param(int dir, const EnsSweepParams &p, int blocks, int threads, size_t smem, cudaStream_t s)
    {
        return dir == 0 ? param_dir<0>(p, blocks, threads, smem, s)
                        : dir == 1 ? param_dir<1>(p, blocks, threads, smem, s)
                                   : param_dir<2>(p, blocks, threads, smem, s);
    }
    static int per_sm(int dir, int threads, size_t smem)
    {
        return dir == 0 ? per_sm_dir<0>(threads, smem)
                        : dir == 1 ? per_sm_dir<1>(threads, smem) : per_sm_dir<2>(threads, smem);
    }
    static constexpr SweepLaunchers table()
    {
        return {single, ens, param, per_sm, tma, tma_per_sm,
                std::is_same<R, double>::value ? &dipole_table : nullptr, ens_tma, ens_tma_per_sm,
                param_persist, param_persist_per_sm, ens_tma_param, ens_tma_param_per_sm, march};
    }
};

}  // namespace ppmlr
