// solve_ee.cu -- the explorer-pool kernel with the early exit of the LB2
// sweep (PFSP_EARLY_EXIT, PFSP_EARLY_EXIT_SLOTS).  Its own translation unit,
// compiled in parallel; the plain kernel carries none of the exit checks.
#include <cuda_runtime.h>

#include "solve_kernel.cuh"

namespace pfsp {

int solve_occupancy_ee(const SolveArgs &a, int warps, size_t smem) {
    if (a.n <= 32) { PFSP_DISPATCH(1, kKindEE, occupancy_t, warps, smem) }
    PFSP_DISPATCH(2, kKindEE, occupancy_t, warps, smem)
}

cudaError_t launch_solve_ee(const SolveArgs &a, int blocks, int warps, size_t smem, cudaStream_t st) {
    if (a.n <= 32) { PFSP_DISPATCH(1, kKindEE, launch_solve_t, a, blocks, warps, smem, st) }
    PFSP_DISPATCH(2, kKindEE, launch_solve_t, a, blocks, warps, smem, st)
}

}  // namespace pfsp
