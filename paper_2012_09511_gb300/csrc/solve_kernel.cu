// solve_kernel.cu -- device-resident pool of depth-first explorers
// (Sections 2.5, 2.6, 3.1-3.4 of the paper), one explorer per warp for the
// whole life of a persistent, cooperatively launched kernel.
//
// Explorer state (IVM-like, Section 2.5): the current level I, the digit V[i]
// selected at every level i (the factoradic position of Section 2.6), the
// branching direction of every level, and per level a row of the jobs still
// to place with the bound of the child each one makes (INT32_MAX once the
// child is pruned).  Digits and directions live in shared memory, and so do
// the rows when they fit without costing explorer warps (else in L2-resident
// global memory).
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

#include "solve_kernel.cuh"

namespace pfsp {

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

int solve_occupancy(const SolveArgs &a, int warps, size_t smem) {
    if (a.net_image) return solve_occupancy_learned(a, warps, smem);
    if (a.coop) return solve_occupancy_coop(a, warps, smem);
    if (a.minht) return solve_occupancy_minht(a, warps, smem);
    if (a.diag) return solve_occupancy_diag(a, warps, smem);
    if (a.bound == PFSP_LB2 && (a.learned & PFSP_EARLY_EXIT)) return solve_occupancy_ee(a, warps, smem);
    if (a.bound == PFSP_LB1) {
        if (a.n <= 32) { PFSP_DISPATCH(1, kKindLb1, occupancy_t, warps, smem) }
        PFSP_DISPATCH(2, kKindLb1, occupancy_t, warps, smem)
    }
    if (a.n <= 32) { PFSP_DISPATCH(1, kKindPlain, occupancy_t, warps, smem) }
    PFSP_DISPATCH(2, kKindPlain, occupancy_t, warps, smem)
}

cudaError_t launch_solve(const SolveArgs &a, int blocks, int warps, size_t smem, cudaStream_t st) {
    if (a.net_image) return launch_solve_learned(a, blocks, warps, smem, st);
    if (a.coop) return launch_solve_coop(a, blocks, warps, smem, st);
    if (a.minht) return launch_solve_minht(a, blocks, warps, smem, st);
    if (a.diag) return launch_solve_diag(a, blocks, warps, smem, st);
    if (a.bound == PFSP_LB2 && (a.learned & PFSP_EARLY_EXIT)) return launch_solve_ee(a, blocks, warps, smem, st);
    if (a.bound == PFSP_LB1) {
        if (a.n <= 32) { PFSP_DISPATCH(1, kKindLb1, launch_solve_t, a, blocks, warps, smem, st) }
        PFSP_DISPATCH(2, kKindLb1, launch_solve_t, a, blocks, warps, smem, st)
    }
    if (a.n <= 32) { PFSP_DISPATCH(1, kKindPlain, launch_solve_t, a, blocks, warps, smem, st) }
    PFSP_DISPATCH(2, kKindPlain, launch_solve_t, a, blocks, warps, smem, st)
}

}  // namespace pfsp
