// bound_kernel.cu -- batched bounding of the children of many partial
// schedules (the bounding operator of Sections 2.3-2.4 applied to a batch).
//
// One warp decomposes one parent at a time; the grid is persistent (a whole
// number of CTAs per SM) and walks the batch with a warp-stride loop.  Each
// CTA stages the instance tables (processing times by machine, machine
// totals, per-pair Johnson tables) into shared memory once with a bulk copy.
// The epilogue either writes every child's bounds (materialize) or reduces
// them per parent and direction to what branching and pruning consume
// (reduce: least bound, its count, the sum, the survivors).
#include <cuda_runtime.h>

#include <algorithm>

#include "bound_device.cuh"
#include "pfsp_internal.h"

namespace pfsp {

struct BoundArgs {
    const uint8_t *perm, *d1, *d2;
    int32_t *lb1, *lb2;
    long long num_nodes;
    const int32_t *tab;
    int tab_words;
    int n, m, S;
    int off_pm, off_tot, off_pq, off_kl, off_rank, off_ptab;
    int warp_words;
    int kind;
    pfsp_node_summary *summary;  // reduce mode: one per node
    int ub;                      // reduce mode: exclusive incumbent of the survivor masks
};

// Reduce-mode epilogue: lane c holds the bounds of the children of compact
// index c (and c + 32); warp reductions give each direction's least bound,
// its count, the sum and the job mask of the children below ub.
template <int NW>
__device__ __forceinline__ void write_summary(const ChildBounds<NW> &cb, const WarpScratch &W, bool use2, int ub,
                                              pfsp_node_summary *out) {
    const int lane = threadIdx.x & 31;
    int mn[2] = {INT_MAX, INT_MAX}, sm[2] = {0, 0};
    unsigned klo[2] = {0u, 0u}, khi[2] = {0u, 0u};
    int v[2][NW];
#pragma unroll
    for (int h = 0; h < NW; ++h) {
        const int c = lane + 32 * h;
        const bool on = c < cb.u;
        const int j = on ? W.ul[c] : 0;
        v[0][h] = use2 ? cb.lb2f[h] : cb.lb1f[h];
        v[1][h] = use2 ? cb.lb2b[h] : cb.lb1b[h];
#pragma unroll
        for (int d = 0; d < 2; ++d) {
            if (on) {
                mn[d] = min(mn[d], v[d][h]);
                sm[d] += v[d][h];  // at most 64 bounds below 2^21 each: no overflow
            }
            if (on && v[d][h] < ub) {
                if (j < 32) klo[d] |= 1u << j;
                else khi[d] |= 1u << (j - 32);
            }
        }
    }
    int cnt[2];
#pragma unroll
    for (int d = 0; d < 2; ++d) {
        mn[d] = __reduce_min_sync(PFSP_FULL, mn[d]);
        sm[d] = __reduce_add_sync(PFSP_FULL, sm[d]);
        klo[d] = __reduce_or_sync(PFSP_FULL, klo[d]);
        khi[d] = __reduce_or_sync(PFSP_FULL, khi[d]);
        cnt[d] = 0;
#pragma unroll
        for (int h = 0; h < NW; ++h)
            cnt[d] += __popc(__ballot_sync(PFSP_FULL, lane + 32 * h < cb.u && v[d][h] == mn[d]));
    }
    if (lane == 0) {
#pragma unroll
        for (int d = 0; d < 2; ++d) {
            out->min[d] = mn[d];
            out->count[d] = cnt[d];
            out->sum[d] = sm[d];
            out->keep[d] = ((unsigned long long)khi[d] << 32) | klo[d];
        }
    }
}

// Each CTA owns a contiguous range of nodes; its warps claim them one at a
// time from a shared counter, so that warps on less busy schedulers of the
// SM take more nodes.
template <int NW, int MT, int WALK, bool REDUCE>
__global__ void __launch_bounds__(kWarpsPerCta * 32, 1) bound_batch_kernel(BoundArgs a) {
    extern __shared__ __align__(16) int smem[];
    __shared__ uint64_t bar;
    __shared__ unsigned long long next_node;
    const long long per_cta = (a.num_nodes + gridDim.x - 1) / gridDim.x;
    const long long first = (long long)blockIdx.x * per_cta;
    const long long end = min(a.num_nodes, first + per_cta);
    if (threadIdx.x == 0) next_node = (unsigned long long)first;
    stage_tables(smem, a.tab, a.tab_words, &bar);  // its first barrier publishes next_node

    SmemTables T;
    T.pm = smem + a.off_pm;
    T.pq = smem + a.off_pq;
    T.tot = smem + a.off_tot;
    T.kl = smem + a.off_kl;
    T.rank = reinterpret_cast<const uint8_t *>(smem + a.off_rank);
    T.ptab = reinterpret_cast<const int2 *>(smem + a.off_ptab);
    T.S = (a.off_ptab - a.off_rank) / (8 * a.n);

    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int n = a.n, m = a.m;
    WarpScratch W = carve_warp(smem + a.tab_words + wib * a.warp_words, n, m, WALK == 1);

    // the next node's depths and permutation entries are loaded while the
    // current node is decomposed
    auto claim = [&]() -> long long {
        unsigned long long c = 0;
        if (lane == 0) c = atomicAdd(&next_node, 1ull);
        return (long long)__shfl_sync(PFSP_FULL, c, 0);
    };
    int nd1 = 0, nd2 = 0, nj0 = 0, nj1 = 0;
    auto fetch = [&](long long v) {
        if (v < end) {
            nd1 = a.d1[v];
            nd2 = a.d2[v];
            const uint8_t *pr = a.perm + v * n;
            nj0 = lane < n ? pr[lane] : 0;
            nj1 = (NW == 2 && lane + 32 < n) ? pr[lane + 32] : 0;
        }
    };
    long long next = claim();
    fetch(next);
    for (;;) {
        const long long node = next;
        if (node >= end) break;
        const int d1 = nd1, d2 = nd2;
        int job0 = nj0 < n ? nj0 : 0;  // keep indexes in range on malformed rows
        int job1 = nj1 < n ? nj1 : 0;
        next = claim();
        fetch(next);
        int32_t *o1 = a.lb1 ? a.lb1 + node * 2 * n : nullptr;
        int32_t *o2 = a.lb2 ? a.lb2 + node * 2 * n : nullptr;
        if (d1 + d2 > n) {
            if constexpr (REDUCE) {
                if (lane == 0) {
                    pfsp_node_summary *s = a.summary + node;
                    for (int d = 0; d < 2; ++d) {
                        s->min[d] = -1;
                        s->count[d] = -1;
                        s->sum[d] = 0;
                        s->keep[d] = 0;
                    }
                }
                continue;
            }
            for (int i = lane; i < 2 * n; i += 32) {
                if (o1) o1[i] = -1;
                if (o2) o2[i] = -1;
            }
            continue;
        }
        ChildBounds<NW> cb;
        decompose_node<NW, MT, WALK, true>(T, W, n, m, a.S, a.kind, job0, job1, d1, d2, cb);
        if constexpr (REDUCE) {
            write_summary<NW>(cb, W, (a.kind & PFSP_LB2) != 0, a.ub, a.summary + node);
            __syncwarp();
            continue;
        }
#pragma unroll
        for (int h = 0; h < NW; ++h) {
            int j = lane + 32 * h;
            bool in = j < n && has_job<NW>(cb.U, j);
            int c = in ? popcnt<NW>(cb.U & low_bits<NW>(j)) : 0;
            int v1f = gather_child<NW>(cb.lb1f, c), v1b = gather_child<NW>(cb.lb1b, c);
            int v2f = gather_child<NW>(cb.lb2f, c), v2b = gather_child<NW>(cb.lb2b, c);
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

static int g_num_sms = 0;

static int num_sms() {
    if (g_num_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 1;
    }
    return g_num_sms;
}

static int g_smem_optin = 0;

static int smem_optin() {
    if (g_smem_optin == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        if (g_smem_optin <= 0) g_smem_optin = 48 * 1024;
    }
    return g_smem_optin;
}

// Warps per CTA: up to `want`, as many as the shared-memory cap allows.
static int fit_warps(const BoundArgs &a, int want) {
    long long avail = (long long)smem_optin() - 64 - (long long)a.tab_words * 4;
    long long w = avail / ((long long)a.warp_words * 4);
    return (int)std::max<long long>(0, std::min<long long>(want, w));
}

template <int NW, int MT, int WALK>
static cudaError_t launch_t(const BoundArgs &a, int want_warps, cudaStream_t stream) {
    const int warps = fit_warps(a, want_warps);
    if (warps < 1) return cudaErrorInvalidConfiguration;
    size_t smem = (size_t)(a.tab_words + warps * a.warp_words) * 4;
    auto kern = a.summary ? bound_batch_kernel<NW, MT, WALK, true> : bound_batch_kernel<NW, MT, WALK, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    long long blocks_needed = (a.num_nodes + warps - 1) / warps;
    long long grid = std::min<long long>((long long)num_sms() * per_sm, blocks_needed);
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, warps * 32, smem, stream>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_bound_batch(const pfsp_instance *inst, int kind, long long num_nodes, const uint8_t *perm,
                               const uint8_t *d1, const uint8_t *d2, int32_t *lb1, int32_t *lb2,
                               cudaStream_t stream, pfsp_node_summary *summary, int ub) {
    if (num_nodes <= 0) return cudaSuccess;
    const TableLayout &L = inst->lay;
    BoundArgs a;
    a.summary = summary;
    a.ub = ub;
    a.perm = perm;
    a.d1 = d1;
    a.d2 = d2;
    a.lb1 = lb1;
    a.lb2 = lb2;
    a.num_nodes = num_nodes;
    a.tab = inst->d_tab;
    // LB1 alone needs only the processing times, totals and pair indexes
    a.tab_words = (kind & PFSP_LB2) ? L.words : L.off_rank;
    a.n = L.n;
    a.m = L.m;
    a.S = (kind & PFSP_LB2) ? L.Ssweep : 0;
    a.off_pm = L.off_pm;
    a.off_tot = L.off_tot;
    a.off_pq = L.off_pq;
    a.off_kl = L.off_kl;
    a.off_rank = L.off_rank;
    a.off_ptab = L.off_ptab;
    a.kind = kind;
    const int warps = kWarpsPerCta;
    const bool want2 = (kind & PFSP_LB2) && L.m >= 2;
    const int nw = L.n <= 32 ? 1 : 2;
    const bool reg_walk = nw == 1 && L.n <= kRegWalk;
    a.warp_words = warp_words(L.n, L.m, nw == 2, want2, reg_walk);
    if (reg_walk) {
        switch (L.m) {
            case 5: return launch_t<1, 5, 1>(a, warps, stream);
            case 10: return launch_t<1, 10, 1>(a, warps, stream);
            case 20: return launch_t<1, 20, 1>(a, warps, stream);
            default: return launch_t<1, 0, 1>(a, warps, stream);
        }
    }
    if (nw == 1) {
        switch (L.m) {
            case 5: return launch_t<1, 5, 0>(a, warps, stream);
            case 10: return launch_t<1, 10, 0>(a, warps, stream);
            case 20: return launch_t<1, 20, 0>(a, warps, stream);
            default: return launch_t<1, 0, 0>(a, warps, stream);
        }
    }
    switch (L.m) {
        case 5: return launch_t<2, 5, 0>(a, warps, stream);
        case 10: return launch_t<2, 10, 0>(a, warps, stream);
        case 20: return launch_t<2, 20, 0>(a, warps, stream);
        default: return launch_t<2, 0, 0>(a, warps, stream);
    }
}

}  // namespace pfsp
