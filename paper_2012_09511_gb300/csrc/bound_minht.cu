// bound_minht.cu -- batched bounding with the heads and tails refinement of
// LB1 (pfsp_bound_batch with PFSP_MINHT; an option, not in the paper).  The
// same decomposition as bound_kernel.cu, then refine_minht on the parents
// whose sigma1 or sigma2 is empty; one warp per parent, generic in m.  It is
// a separate kernel so that the plain one carries none of its code.
#include <cuda_runtime.h>

#include <algorithm>

#include "minht_device.cuh"
#include "pfsp_internal.h"

namespace pfsp {

struct MinhtArgs {
    const uint8_t *perm, *d1, *d2;
    int32_t *lb1, *lb2;
    long long num_nodes;
    const int32_t *tab;
    int tab_words;
    int n, m, S;
    int off_pm, off_tot, off_kl, off_rank, off_ptab;
    int warp_words;
    int kind;  // PFSP_LB1 / PFSP_LB2 bits
};

template <int NW>
__global__ void __launch_bounds__(8 * 32, 1) bound_minht_kernel(MinhtArgs a) {
    extern __shared__ __align__(16) int smem[];
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
    const int n = a.n, m = a.m;
    WarpScratch W = carve_warp(smem + a.tab_words + wib * a.warp_words, n, m, false);
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long node = (long long)blockIdx.x * (blockDim.x >> 5) + wib; node < a.num_nodes; node += warps) {
        const int d1 = a.d1[node], d2 = a.d2[node];
        int32_t *o1 = a.lb1 ? a.lb1 + node * 2 * n : nullptr;
        int32_t *o2 = a.lb2 ? a.lb2 + node * 2 * n : nullptr;
        if (d1 + d2 > n) {
            for (int i = lane; i < 2 * n; i += 32) {
                if (o1) o1[i] = -1;
                if (o2) o2[i] = -1;
            }
            continue;
        }
        const uint8_t *pr = a.perm + node * n;
        const int nj0 = lane < n ? pr[lane] : 0;
        const int nj1 = (NW == 2 && lane + 32 < n) ? pr[lane + 32] : 0;
        const int job0 = nj0 < n ? nj0 : 0, job1 = nj1 < n ? nj1 : 0;
        ChildBounds<NW> cb;
        decompose_lb1<NW, 0>(T, W, n, m, a.kind, job0, job1, d1, d2, cb);
        if (d1 == 0 || d2 == 0) refine_minht<NW, 0>(T, W, n, m, d1, d2, cb);
        if ((a.kind & PFSP_LB2) && m >= 2) decompose_lb2<NW, 0, 0>(T, W, n, m, a.S, cb, INT_MAX, false, nullptr);
#pragma unroll
        for (int h = 0; h < NW; ++h) {
            const int j = lane + 32 * h;
            const bool in = j < n && has_job<NW>(cb.U, j);
            const int c = in ? popcnt<NW>(cb.U & low_bits<NW>(j)) : 0;
            const int v1f = gather_child<NW>(cb.lb1f, c), v1b = gather_child<NW>(cb.lb1b, c);
            const int v2f = gather_child<NW>(cb.lb2f, c), v2b = gather_child<NW>(cb.lb2b, c);
            if (j < n) {
                if (o1 && (a.kind & PFSP_LB1)) {
                    o1[j] = in ? v1f : -1;
                    o1[n + j] = in ? v1b : -1;
                }
                if (o2 && (a.kind & PFSP_LB2)) {
                    o2[j] = in ? v2f : -1;
                    o2[n + j] = in ? v2b : -1;
                }
            }
        }
        __syncwarp();
    }
}

template <int NW>
static cudaError_t launch_minht_t(const MinhtArgs &a, cudaStream_t stream) {
    int dev = 0, nsm = 1, optin = 48 * 1024;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const long long fit = ((long long)optin - 64 - (long long)a.tab_words * 4) / ((long long)a.warp_words * 4);
    const int warps = (int)std::min<long long>(8, fit);
    if (warps < 1) return cudaErrorInvalidConfiguration;
    const size_t smem = (size_t)(a.tab_words + warps * a.warp_words) * 4;
    auto kern = bound_minht_kernel<NW>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long need = (a.num_nodes + warps - 1) / warps;
    const long long grid = std::max<long long>(1, std::min<long long>((long long)nsm * per_sm, need));
    kern<<<(unsigned)grid, warps * 32, smem, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_bound_batch_minht(const pfsp_instance *inst, int kind, long long num_nodes, const uint8_t *perm,
                                     const uint8_t *d1, const uint8_t *d2, int32_t *lb1, int32_t *lb2,
                                     cudaStream_t stream) {
    if (num_nodes <= 0) return cudaSuccess;
    const TableLayout &L = inst->lay;
    MinhtArgs a;
    a.perm = perm;
    a.d1 = d1;
    a.d2 = d2;
    a.lb1 = lb1;
    a.lb2 = lb2;
    a.num_nodes = num_nodes;
    a.tab = inst->d_tab;
    a.tab_words = (kind & PFSP_LB2) ? L.words : L.off_rank;
    a.n = L.n;
    a.m = L.m;
    a.S = (kind & PFSP_LB2) ? L.Ssweep : 0;
    a.off_pm = L.off_pm;
    a.off_tot = L.off_tot;
    a.off_kl = L.off_kl;
    a.off_rank = L.off_rank;
    a.off_ptab = L.off_ptab;
    a.kind = kind & (PFSP_LB1 | PFSP_LB2);
    const int nw = L.n <= 32 ? 1 : 2;
    a.warp_words = warp_words(L.n, L.m, nw == 2, (kind & PFSP_LB2) && L.m >= 2, false);
    return nw == 1 ? launch_minht_t<1>(a, stream) : launch_minht_t<2>(a, stream);
}

}  // namespace pfsp
