// solve_learned.cu -- the explorer-pool kernel with the ordering network
// (learned child and slot order, not in the paper), in its own translation
// unit so that it compiles in parallel with the plain solver.
#include <cuda_runtime.h>

#include "solve_kernel.cuh"

namespace pfsp {

int solve_occupancy_learned(const SolveArgs &a, int warps, size_t smem) {
    if (a.n <= 32) { PFSP_DISPATCH(1, kKindLearned, occupancy_t, warps, smem) }
    PFSP_DISPATCH(2, kKindLearned, occupancy_t, warps, smem)
}

cudaError_t launch_solve_learned(const SolveArgs &a, int blocks, int warps, size_t smem, cudaStream_t st) {
    if (a.n <= 32) { PFSP_DISPATCH(1, kKindLearned, launch_solve_t, a, blocks, warps, smem, st) }
    PFSP_DISPATCH(2, kKindLearned, launch_solve_t, a, blocks, warps, smem, st)
}

}  // namespace pfsp
