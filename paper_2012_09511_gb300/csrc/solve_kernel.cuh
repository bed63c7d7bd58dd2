// solve_kernel.cuh -- the explorer-pool kernel template and its launch
// helpers, instantiated by solve_kernel.cu (plain solver), solve_learned.cu
// (solver with the ordering network) and solve_coop.cu (solver exchanging
// with the host heuristic threads), translation units that compile in
// parallel.
#pragma once

#include <cuda_runtime.h>

#include "explorer_device.cuh"

namespace pfsp {

template <int NW, int MT, int KIND>
__global__ void __launch_bounds__((KIND == kKindLearned ? kSolveWarpsLearned : kSolveWarps) * 32, 1)
    solve_kernel(SolveArgs a) {
    constexpr bool LEARNED = KIND == kKindLearned;
    extern __shared__ __align__(128) int smem[];
    __shared__ uint64_t bar;
    stage_tables(smem, a.tab, a.tab_words, &bar);
    SmemTables T;
    T.pm = smem + a.off_pm;
    T.pq = nullptr;  // the max-scan fronts are the bounding kernel's
    T.tot = smem + a.off_tot;
    T.kl = smem + a.off_kl;
    T.rank = reinterpret_cast<const uint8_t *>(smem + a.off_rank);
    T.ptab = reinterpret_cast<const int2 *>(smem + a.off_ptab);
    T.S = (a.off_ptab - a.off_rank) / (8 * a.n);
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int warps = blockDim.x >> 5;
    const int rows_words = a.rows_smem ? solve_row_words(a.n) : 0;
    int *wbase = smem + a.warp_base + wib * (a.warp_words + kExplorerWords + rows_words);
    WarpScratch W = carve_warp(wbase, a.n, a.m);
    ExplorerSmem &X = *reinterpret_cast<ExplorerSmem *>(wbase + a.warp_words);
    const int me = blockIdx.x * warps + wib;
    // the ordering network's inference image (read from global memory)
    __shared__ MlpImage net;
    if (LEARNED && a.net_image) {
        if (threadIdx.x == 0) net = mlp_image_view(a.net_image, a.net_D0, a.net_O3);
        __syncthreads();
    }
    if (me >= a.K) return;

    for (int i = lane; i < a.n; i += 32) {
        X.D[i] = a.in_start[(size_t)me * 64 + i];
        X.E[i] = a.in_end[(size_t)me * 65 + 1 + i];
    }
    if (lane == 0) {
        X.etop = a.in_end[(size_t)me * 65];
        X.seq = 0;
        const int lv = a.in_level ? a.in_level[me] : 0xff;
        X.lvl = lv == 0xff ? -1 : lv;
    }
    __syncwarp();
    run_explorer<NW, MT, KIND>(a, T, W, X, me, LEARNED && a.net_image ? &net : nullptr);
}

template <int NW, int MT, int KIND>
inline cudaError_t launch_solve_t(const SolveArgs &a, int blocks, int warps, size_t smem, cudaStream_t st) {
    auto kern = solve_kernel<NW, MT, KIND>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&a};
    return cudaLaunchCooperativeKernel((const void *)kern, dim3(blocks), dim3(warps * 32), args, smem, st);
}

template <int NW, int MT, int KIND>
inline int occupancy_t(int warps, size_t smem) {
    auto kern = solve_kernel<NW, MT, KIND>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem) != cudaSuccess) return 0;
    return per_sm;
}

#define PFSP_DISPATCH(NWV, LV, FN, ...)                                   \
    switch (a.m) {                                                         \
        case 5: return FN<NWV, 5, LV>(__VA_ARGS__);                        \
        case 10: return FN<NWV, 10, LV>(__VA_ARGS__);                      \
        case 20: return FN<NWV, 20, LV>(__VA_ARGS__);                      \
        default: return FN<NWV, 0, LV>(__VA_ARGS__);                       \
    }

}  // namespace pfsp
