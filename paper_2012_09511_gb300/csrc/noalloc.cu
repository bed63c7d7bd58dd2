// noalloc.cu -- pfsp_solve_noalloc: the explorer-pool solve for callers that
// must not allocate device memory.
//
// Some programs cannot call cudaMalloc at the point where they want a solve:
// a service that reserves all its device memory up front and treats any later
// allocation as a fault, a host application whose device memory is owned by
// another allocator (a framework's caching pool) that it may not bypass, or a
// latency-bound caller for which the implicit device synchronisation of
// cudaMalloc/cudaFree is unacceptable.  For them this file keeps the solve's
// device scratch -- the instance tables and the whole explorer pool state --
// in one file-scope __device__ array of fixed size, created when the library
// is loaded on a device and kept until the process exits.
//
// The array is shared by every call on a device and keeps the contents of the
// last call: each call rewrites or clears everything the kernel reads before
// launching.  Two calls that overlap on the GPU (from different host threads
// or streams) would use the same memory and race; callers must serialise them.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cstring>
#include <vector>

#include "explorer_device.cuh"

namespace pfsp {

// Fixed capacity of the scratch array: 8 MiB per device.
constexpr size_t kNoAllocBytes = 8u << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the array on the current device.  In host code the
// symbol g_noalloc_scratch is only a host-side stand-in, not a device address.
// The address is looked up on every call (a cheap query that allocates
// nothing): a cached address could go stale when the primary context is
// reset and the module is loaded again.  The first call on a device loads the
// library's module there, and the array with it.
static int scratch_for_current_device(void **out) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
        return set_error(PFSP_ERR_CUDA, "cudaGetSymbolAddress of the static scratch: %s", cudaGetErrorString(e));
    *out = p;
    return PFSP_OK;
}

}  // namespace pfsp

using namespace pfsp;

extern "C" int pfsp_solve_noalloc(int n, int m, const int32_t *p, const pfsp_options *opt, int32_t *best_cmax,
                                  int32_t *best_perm, int *outcome, pfsp_stats_t *stats) {
    if (!p || !opt || !best_cmax || !outcome) return set_error(PFSP_ERR_INVALID, "NULL argument");
    if (n < 1 || m < 1) return set_error(PFSP_ERR_INVALID, "n and m must be >= 1 (n=%d, m=%d)", n, m);
    if (n > kMaxJobs || m > kMaxMachines)
        return set_error(PFSP_ERR_UNSUPPORTED, "n <= %d and m <= %d required", kMaxJobs, kMaxMachines);
    long long total = 0;
    for (long long i = 0; i < (long long)n * m; ++i) {
        if (p[i] < 0) return set_error(PFSP_ERR_INVALID, "negative processing time at index %lld", i);
        if (p[i] > kMaxTime) return set_error(PFSP_ERR_UNSUPPORTED, "processing time above 2^22-1 at %lld", i);
        total += p[i];
    }
    if (total >= kMaxTotal) return set_error(PFSP_ERR_UNSUPPORTED, "sum of processing times >= 2^28");
    if (opt->bound != PFSP_LB1 && opt->bound != PFSP_LB2)
        return set_error(PFSP_ERR_INVALID, "bound must be PFSP_LB1 or PFSP_LB2");
    if (opt->branching < PFSP_MINMIN || opt->branching > PFSP_MINSUM)
        return set_error(PFSP_ERR_INVALID, "branching must be PFSP_MINMIN, PFSP_MINMIN_CAPPED, PFSP_MINBRANCH or PFSP_MINSUM");
    if (opt->node_limit < 0 || opt->time_limit_s < 0) return set_error(PFSP_ERR_INVALID, "negative limit");

    void *scratch = nullptr;
    int rc = scratch_for_current_device(&scratch);
    if (rc != PFSP_OK) return rc;

    const TableLayout L = table_layout(n, m);
    if (opt->bound == PFSP_LB2 && (size_t)(L.words - (L.off_kl - L.off_pq)) * 4 > (size_t)kMaxTableBytes)
        return set_error(PFSP_ERR_UNSUPPORTED, "LB2 tables exceed shared memory for this instance");
    std::vector<int32_t> blob;
    build_tables(L, p, blob, nullptr, L.P);

    std::vector<int> neh_perm;
    int ub0 = opt->init_ub;
    bool from_neh = false;
    if (ub0 == INT32_MAX) {
        ub0 = neh(n, m, p, neh_perm);
        from_neh = true;
    }

    SolveArgs a;
    memset(&a, 0, sizeof(a));
    a.tab_words = opt->bound == PFSP_LB2 ? L.words : L.off_rank;
    a.n = n;
    a.m = m;
    a.S = opt->bound == PFSP_LB2 ? L.Ssweep : 0;
    a.off_pm = L.off_pm;
    a.off_tot = L.off_tot;
    a.off_kl = L.off_kl;
    a.off_rank = L.off_rank;
    a.off_ptab = L.off_ptab;
    a.bound = opt->bound;
    a.branching = opt->branching;
    a.cap = ub0;
    if (opt->learned) return set_error(PFSP_ERR_UNSUPPORTED, "pfsp_solve_noalloc runs the plain solver only");
    if (opt->heuristic_threads) return set_error(PFSP_ERR_UNSUPPORTED, "pfsp_solve_noalloc runs no heuristic threads");
    if (opt->lb1_minht) return set_error(PFSP_ERR_UNSUPPORTED, "pfsp_solve_noalloc runs the plain bounds only");
    a.warp_words = (warp_words(n, m, n > 32, opt->bound == PFSP_LB2 && m >= 2) + 7) & ~7;
    a.warp_base = (a.tab_words + 7) & ~7;
    const int per_warp = a.warp_words + kExplorerWords;
    int dev = 0, nsm = 1, optin = 48 * 1024;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    int want = opt->warps_per_sm > 0 ? std::min(opt->warps_per_sm, kSolveWarps) : kSolveWarps;
    long long fit = ((long long)optin - 256 - (long long)a.warp_base * 4) / ((long long)per_warp * 4);
    want = (int)std::min<long long>(want, fit);

    // layout inside the static array: tables, then the explorer pool; the
    // pool shrinks (fewer explorers per SM) until it fits
    auto layout_bytes = [&](int K, size_t *offs) {
        size_t off = 0;
        auto take = [&](size_t bytes) {
            size_t o = off;
            off = (off + bytes + 255) & ~(size_t)255;
            return o;
        };
        offs[0] = take((size_t)L.words * 4);
        offs[1] = take((size_t)K * n * n);
        offs[2] = take((size_t)K * n * n * 4);
        offs[3] = take((size_t)K * 64);
        offs[4] = take((size_t)K * 65);
        offs[5] = take((size_t)K * 8);
        offs[6] = take((size_t)K * 8);
        offs[7] = take((size_t)K * 4);
        offs[8] = take((size_t)K * 64);
        offs[9] = take(8 * 8);
        offs[10] = take(64);
        return off;
    };
    // explorers per SM are chosen directly: a cooperative launch may use
    // fewer CTAs per SM than can be resident, so the pool can shrink to one
    // explorer per SM (one single-warp CTA on each SM); the largest pool that
    // fits is used (ties: more warps per CTA)
    size_t offs[11];
    int warps = 0, blocks = 0, K = 0;
    size_t smem = 0;
    for (int w = want; w >= 1; --w) {
        const size_t sm_w = (size_t)(a.warp_base + w * per_warp) * 4;
        const int per_sm = solve_occupancy(a, w, sm_w);
        for (int c = per_sm; c >= 1; --c) {
            const int Kc = nsm * c * w;
            if (Kc <= K) break;
            if (layout_bytes(Kc, offs) <= kNoAllocBytes) {
                warps = w;
                blocks = nsm * c;
                K = Kc;
                smem = sm_w;
                break;
            }
        }
    }
    if (K < 1) {
        const size_t need = layout_bytes(nsm, offs);
        return set_error(PFSP_ERR_UNSUPPORTED,
                         "instance %dx%d needs more than the %zu-byte static scratch of pfsp_solve_noalloc "
                         "(%zu bytes with one explorer per SM)",
                         n, m, kNoAllocBytes, need);
    }
    layout_bytes(K, offs);
    a.K = K;
    a.row_stride = n * n;
    a.inst_of = nullptr;
    a.my_inst = 0;
    a.inst_perm = nullptr;
    a.perm_lock = nullptr;
    a.perm_cmax = nullptr;
    char *b = (char *)scratch;
    a.tab = (const int32_t *)(b + offs[0]);
    a.rows_job = (uint8_t *)(b + offs[1]);
    a.rows_lb = (int32_t *)(b + offs[2]);
    a.in_start = (uint8_t *)(b + offs[3]);
    a.in_end = (uint8_t *)(b + offs[4]);
    a.mailbox = (unsigned long long *)(b + offs[5]);
    a.response = (unsigned long long *)(b + offs[6]);
    a.len_est = (float *)(b + offs[7]);
    a.best_perm = (uint8_t *)(b + offs[8]);
    a.counters = (unsigned long long *)(b + offs[9]);
    int *sc = (int *)(b + offs[10]);
    a.active = sc + 0;
    a.ub = sc + 1;
    a.stop = sc + 2;
    a.err = sc + 3;
    a.best_key = (unsigned long long *)(sc + 4);
    a.node_limit = opt->node_limit;
    a.time_limit_ns = opt->time_limit_s > 0 ? (unsigned long long)(opt->time_limit_s * 1e9) : 0ull;
    a.min_steal = opt->min_steal > 0 ? (float)opt->min_steal : default_min_steal(n);
    int ce = opt->check_every > 0 ? opt->check_every : kDefaultCheckEvery, pw = 1;
    while (pw < ce) pw <<= 1;
    a.check_every = pw;

    // initial partition of [0, n!) into equal chunks of the first levels
    int Lv = 0;
    long long PL = 1;
    while (Lv < n && PL < K) {
        PL *= (n - Lv);
        ++Lv;
    }
    const long long Kp = std::min<long long>(K, PL);
    std::vector<uint8_t> hs((size_t)K * 64, 0), he((size_t)K * 65, 0);
    auto digits = [&](long long x, uint8_t *d) {
        for (int lvl = Lv - 1; lvl >= 0; --lvl) {
            int r = n - lvl;
            d[lvl] = (uint8_t)(x % r);
            x /= r;
        }
    };
    for (long long i = 0; i < Kp; ++i) {
        long long s = (long long)((__int128)i * PL / Kp), e = (long long)((__int128)(i + 1) * PL / Kp);
        digits(s, &hs[(size_t)i * 64]);
        if (e == PL) he[(size_t)i * 65] = 1;
        else digits(e, &he[(size_t)i * 65 + 1]);
    }

    // every region the kernel reads is rewritten here: the array still holds
    // whatever the previous call left in it
    auto t0 = std::chrono::steady_clock::now();
    int hsc[6] = {(int)Kp, ub0, 0, 0, -1, -1};
    cudaStream_t st = 0;
    cudaError_t e = cudaMemcpyAsync((void *)a.tab, blob.data(), (size_t)L.words * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.mailbox, 0xff, (size_t)K * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.response, 0, (size_t)K * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.len_est, 0, (size_t)K * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.counters, 0, 64, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(a.in_start, hs.data(), hs.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(a.in_end, he.data(), he.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sc, hsc, sizeof(hsc), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_solve(a, blocks, warps, smem, st);
    int rsc[6];
    unsigned long long cnt[8];
    if (e == cudaSuccess) e = cudaMemcpyAsync(rsc, sc, sizeof(rsc), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cnt, a.counters, sizeof(cnt), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return set_error(PFSP_ERR_CUDA, "pfsp_solve_noalloc: %s", cudaGetErrorString(e));
    if (rsc[3] != 0)
        return set_error(PFSP_ERR_TIMEOUT, "a bounded device wait expired (detail %d)", rsc[3]);
    unsigned long long key;
    memcpy(&key, &rsc[4], sizeof(key));
    const bool found = key != ~0ull;
    uint8_t bp[64];
    if (found) {
        e = cudaMemcpy(bp, a.best_perm + (size_t)(key & 0xffffffffu) * 64, 64, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return set_error(PFSP_ERR_CUDA, "pfsp_solve_noalloc: %s", cudaGetErrorString(e));
    }
    if (rsc[2] == 1) *outcome = PFSP_LIMIT_NODES;
    else if (rsc[2] == 2) *outcome = PFSP_LIMIT_TIME;
    else if (found || from_neh) *outcome = PFSP_OPTIMAL;
    else *outcome = PFSP_PROVEN_NO_BETTER;
    *best_cmax = rsc[1];
    if (best_perm) {
        if (found)
            for (int j = 0; j < n; ++j) best_perm[j] = bp[j];
        else if (from_neh)
            for (int j = 0; j < n; ++j) best_perm[j] = neh_perm[j];
    }
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->decomposed = cnt[0];
        stats->bounded_children = cnt[1];
        stats->leaves = cnt[2];
        stats->pruned = cnt[3];
        stats->steals = cnt[4];
        stats->iterations = cnt[5];
        stats->final_ub = rsc[1];
        stats->explorers = K;
        stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return PFSP_OK;
}
