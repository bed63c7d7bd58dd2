// solve_minht.cu -- the explorer-pool kernel with the heads and tails
// refinement of LB1 (pfsp_options.lb1_minht; not in the paper).  Its own
// translation unit, compiled in parallel; the plain kernel carries none of it.
#include <cuda_runtime.h>

#include "solve_kernel.cuh"

namespace pfsp {

int solve_occupancy_minht(const SolveArgs &a, int warps, size_t smem) {
    if (a.n <= 32) { PFSP_DISPATCH(1, kKindMinht, occupancy_t, warps, smem) }
    PFSP_DISPATCH(2, kKindMinht, occupancy_t, warps, smem)
}

cudaError_t launch_solve_minht(const SolveArgs &a, int blocks, int warps, size_t smem, cudaStream_t st) {
    if (a.n <= 32) { PFSP_DISPATCH(1, kKindMinht, launch_solve_t, a, blocks, warps, smem, st) }
    PFSP_DISPATCH(2, kKindMinht, launch_solve_t, a, blocks, warps, smem, st)
}

}  // namespace pfsp
