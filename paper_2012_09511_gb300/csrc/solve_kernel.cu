// solve_kernel.cu -- device-resident pool of depth-first explorers
// (Sections 2.5, 2.6, 3.1-3.4 of the paper), one explorer per warp for the
// whole life of a persistent, cooperatively launched kernel.
//
// Explorer state (IVM-like, Section 2.5): the current level I, the digit V[i]
// selected at every level i (the factoradic position of Section 2.6), the
// branching direction of every level, and per level a row of the jobs still
// to place with the bound of the child each one makes (INT32_MAX once the
// child is pruned).  Rows live in global memory (L2 resident); digits and
// directions in shared memory.
//
// Work units are factoradic intervals [start, end) of leaf indices.  An
// explorer decomposes a node only while the node's leftmost leaf lo(node) is
// below its end, and counts a decomposition only when lo(node) >= start; the
// ancestors it re-decomposes to rebuild its rows at start (lo < start) are not
// counted.  As the intervals partition [0, n!), every node of the search tree
// is counted by exactly one explorer, so with a fixed incumbent the counts
// equal those of a sequential depth-first search.
//
// Work stealing (Section 3.4, redesigned for an asynchronous pool): an idle
// explorer (thief) posts its id in the mailbox of a victim chosen by the
// published log2 length of its interval; the victim itself, at the top of its
// next iteration, splits its remaining interval [pos, end) at the floor
// midpoint, keeps [pos, mid) and hands [mid, end) to the thief.  Only the owner
// ever changes its own interval, so no position can be explored twice.  Every
// wait is bounded; on expiry the kernel records an error and stops.
#include <cuda_runtime.h>

#include <cfloat>

#include "explorer_device.cuh"

namespace pfsp {

template <int NW, int MT, bool LEARNED>
__global__ void __launch_bounds__((LEARNED ? kSolveWarpsLearned : kSolveWarps) * 32, 1) solve_kernel(SolveArgs a) {
    extern __shared__ __align__(128) int smem[];
    __shared__ uint64_t bar;
    stage_tables(smem, a.tab, a.tab_words, &bar);
    SmemTables T;
    T.pm = smem + a.off_pm;
    T.tot = smem + a.off_tot;
    T.kl = smem + a.off_kl;
    T.rank = reinterpret_cast<const uint8_t *>(smem + a.off_rank);
    T.ptab = reinterpret_cast<const int2 *>(smem + a.off_ptab);
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int warps = blockDim.x >> 5;
    int *wbase = smem + a.warp_base + wib * (a.warp_words + kExplorerWords);
    WarpScratch W = carve_warp(wbase, a.n, a.m);
    ExplorerSmem &X = *reinterpret_cast<ExplorerSmem *>(wbase + a.warp_words);
    const int me = blockIdx.x * warps + wib;
    // the ordering network's inference image, copied once per CTA
    __shared__ MlpImage net;
    if (LEARNED && a.net_words) {
        stage_tables(smem + a.net_base, reinterpret_cast<const int32_t *>(a.net_image), a.net_words, &bar);
        if (threadIdx.x == 0) net = mlp_image_view(smem + a.net_base, a.net_D0, a.net_O3);
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
    }
    __syncwarp();
    run_explorer<NW, MT, LEARNED>(a, T, W, X, me, LEARNED && a.net_words ? &net : nullptr);
}

int solve_warp_words(int n, int m, int bound) {
    return warp_words(n, m, n > 32, bound == PFSP_LB2 && m >= 2) + kExplorerWords;
}


int mlp_scratch_place(int n, int m, int bound, int D0, int *off) {
    const int need = (mlp_scratch_bytes(D0) + 3) / 4;
    const int bw = warp_words(n, m, n > 32, bound == PFSP_LB2 && m >= 2);
    if (bound == PFSP_LB2 && m >= 2) {
        // alias the prefix-record / C region, free outside the LB2 sweep
        const int nr = round4(n);
        const int e_off = kWarpHead + 3 * round4(nr * (m | 1));
        const int start = (e_off + 7) & ~7;
        if (start + need <= bw) {
            *off = start;
            return 0;
        }
    }
    *off = (bw + 7) & ~7;
    return *off + need - bw;
}

template <int NW, int MT, bool LEARNED>
static cudaError_t launch_solve_t(const SolveArgs &a, int blocks, int warps, size_t smem, cudaStream_t st) {
    auto kern = solve_kernel<NW, MT, LEARNED>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&a};
    return cudaLaunchCooperativeKernel((const void *)kern, dim3(blocks), dim3(warps * 32), args, smem, st);
}

template <int NW, int MT, bool LEARNED>
static int occupancy_t(int warps, size_t smem) {
    auto kern = solve_kernel<NW, MT, LEARNED>;
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

int solve_occupancy(const SolveArgs &a, int warps, size_t smem) {
    const bool learned = a.net_words > 0;
    if (a.n <= 32 && learned) { PFSP_DISPATCH(1, true, occupancy_t, warps, smem) }
    if (a.n <= 32) { PFSP_DISPATCH(1, false, occupancy_t, warps, smem) }
    if (learned) { PFSP_DISPATCH(2, true, occupancy_t, warps, smem) }
    PFSP_DISPATCH(2, false, occupancy_t, warps, smem)
}

cudaError_t launch_solve(const SolveArgs &a, int blocks, int warps, size_t smem, cudaStream_t st) {
    const bool learned = a.net_words > 0;
    if (a.n <= 32 && learned) { PFSP_DISPATCH(1, true, launch_solve_t, a, blocks, warps, smem, st) }
    if (a.n <= 32) { PFSP_DISPATCH(1, false, launch_solve_t, a, blocks, warps, smem, st) }
    if (learned) { PFSP_DISPATCH(2, true, launch_solve_t, a, blocks, warps, smem, st) }
    PFSP_DISPATCH(2, false, launch_solve_t, a, blocks, warps, smem, st)
}

}  // namespace pfsp
