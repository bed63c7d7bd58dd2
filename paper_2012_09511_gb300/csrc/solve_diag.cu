// solve_diag.cu -- the explorer-pool kernel with phase timers and
// decomposition traces (pfsp_options.phase_timers, pfsp_solve_trace), for
// either bound.  Its own translation unit, compiled in parallel; the fast
// kernels carry none of this code.
#include <cuda_runtime.h>

#include "solve_kernel.cuh"

namespace pfsp {

int solve_occupancy_diag(const SolveArgs &a, int warps, size_t smem) {
    if (a.n <= 32) { PFSP_DISPATCH(1, kKindDiag, occupancy_t, warps, smem) }
    PFSP_DISPATCH(2, kKindDiag, occupancy_t, warps, smem)
}

cudaError_t launch_solve_diag(const SolveArgs &a, int blocks, int warps, size_t smem, cudaStream_t st) {
    if (a.n <= 32) { PFSP_DISPATCH(1, kKindDiag, launch_solve_t, a, blocks, warps, smem, st) }
    PFSP_DISPATCH(2, kKindDiag, launch_solve_t, a, blocks, warps, smem, st)
}

}  // namespace pfsp
