// solve_coop.cu -- the explorer-pool kernel that exchanges with the host
// heuristic threads (Section 4.2): it folds their incumbent into its own and
// answers their snapshot requests.  Its own translation unit, so that it
// compiles in parallel with the plain solver, which carries none of its code.
#include <cuda_runtime.h>

#include "solve_kernel.cuh"

namespace pfsp {

int solve_occupancy_coop(const SolveArgs &a, int warps, size_t smem) {
    if (a.n <= 32) { PFSP_DISPATCH(1, kKindCoop, occupancy_t, warps, smem) }
    PFSP_DISPATCH(2, kKindCoop, occupancy_t, warps, smem)
}

cudaError_t launch_solve_coop(const SolveArgs &a, int blocks, int warps, size_t smem, cudaStream_t st) {
    if (a.n <= 32) { PFSP_DISPATCH(1, kKindCoop, launch_solve_t, a, blocks, warps, smem, st) }
    PFSP_DISPATCH(2, kKindCoop, launch_solve_t, a, blocks, warps, smem, st)
}

}  // namespace pfsp
