// solve_batch.cu -- many independent instances of uneven n and m solved by
// one persistent launch of the explorer pool, captured in a CUDA graph, with
// an autotuner for the pool's launch parameters.  (Batching instances is not
// in the paper; each instance is solved exactly as by pfsp_solve.)
//
// Scheduling: every CTA claims the next unclaimed instance from a global
// counter, stages that instance's tables into its shared memory and runs its
// warps as explorers on it, the instance's leaf interval split evenly among
// them.  Once every instance has been claimed, a CTA that finishes joins the
// running instance with the most explorers holding work; its warps start idle
// and obtain work by stealing from that instance's explorers only (a steal
// request from an explorer now on another instance is denied).  An instance
// is done when none of its explorers holds work.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cstring>
#include <vector>

#include "explorer_device.cuh"

namespace pfsp {

struct InstDesc {
    const int32_t *tab;
    int tab_words, n, m, S;
    int off_pm, off_tot, off_kl, off_rank, off_ptab;
    int warp_words;
    int cap;
};

struct BatchArgs {
    const InstDesc *desc;
    int count;
    int bound, branching;
    int K, row_stride, warp_stride, max_tab_words;
    uint8_t *rows_job;
    int32_t *rows_lb;
    uint8_t *hand_job;   // [K][row_stride] rows handed over with stolen intervals
    int32_t *hand_lb;    // [K][row_stride]
    uint8_t *hand_dir;   // [K][64]
    int *hand_lc;        // [K]
    uint8_t *in_start, *in_end;
    unsigned long long *mailbox, *response;
    float *len_est;
    uint8_t *best_perm;  // [K][64]
    uint8_t *inst_perm;  // [count][64] best permutation per instance
    int *perm_lock;      // [count]
    int *perm_cmax;      // [count]
    int *inst_of;        // [K]
    int *next;           // next instance to claim
    int *started;        // [count]
    int *active;         // [count]
    int *ub;             // [count]
    unsigned long long *best_key;  // [count]
    unsigned long long *counters;  // [count][8]
    int *stop;                     // [count]
    int *err;
    unsigned long long *t0;        // kernel start on the device clock
    long long node_limit;          // per instance
    unsigned long long time_limit_ns;
    float min_steal;
    int check_every;
};

// Interval of warp w among the W explorers that open an instance: the first
// L levels (n!/(n-L)! >= W prefixes) are cut into W equal runs of prefixes.
__device__ inline void opening_interval(int n, int W, int w, ExplorerSmem &X) {
    for (int i = 0; i < 64; ++i) {
        X.D[i] = 0;
        X.E[i] = 0;
    }
    X.etop = 0;
    X.lvl = -1;
    int L = 0;
    long long PL = 1;
    while (L < n && PL < W) {
        PL *= (n - L);
        ++L;
    }
    const long long Kp = PL < W ? PL : W;
    if (w >= Kp) return;  // empty: start == end
    long long s = (long long)w * PL / Kp, e = (long long)(w + 1) * PL / Kp;
    for (int lvl = L - 1; lvl >= 0; --lvl) {
        int r = n - lvl;
        X.D[lvl] = (int)(s % r);
        s /= r;
    }
    if (e == PL) {
        X.etop = 1;
    } else {
        for (int lvl = L - 1; lvl >= 0; --lvl) {
            int r = n - lvl;
            X.E[lvl] = (int)(e % r);
            e /= r;
        }
    }
}

__device__ inline int opening_count(int n, int W) {
    int L = 0;
    long long PL = 1;
    while (L < n && PL < W) {
        PL *= (n - L);
        ++L;
    }
    return (int)(PL < W ? PL : W);
}

template <int NW>
__global__ void __launch_bounds__(kSolveWarps * 32, 1) solve_batch_kernel(BatchArgs b) {
    extern __shared__ __align__(128) int smem[];
    __shared__ uint64_t bar;
    __shared__ SolveArgs sa;
    __shared__ int s_inst, s_mode;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    const int me = blockIdx.x * W + wib;
    int *wbase = smem + b.max_tab_words + wib * b.warp_stride;
    ExplorerSmem &X = *reinterpret_cast<ExplorerSmem *>(wbase + b.warp_stride - kExplorerWords);
    if (threadIdx.x == 0) atomicCAS(b.t0, 0ull, global_ns());
    if (lane == 0) X.seq = 0;

    while (true) {
        if (threadIdx.x == 0) {
            int i = atomicAdd(b.next, 1), mode = 1;
            if (i >= b.count) {
                // every instance claimed: help the one with the most busy explorers
                i = -1;
                mode = 0;
                int best = 0;
                for (int q = 0; q < b.count; ++q) {
                    if (ld_volatile(b.started + q) != 1) continue;
                    int act = ld_volatile(b.active + q);
                    if (act > best) {
                        best = act;
                        i = q;
                    }
                }
                if (i >= 0) mode = 2;
            }
            s_inst = i;
            s_mode = mode;
            if (mode) {
                const InstDesc d = b.desc[i];
                memset(&sa, 0, sizeof(sa));
                sa.tab = d.tab;
                sa.tab_words = d.tab_words;
                sa.n = d.n;
                sa.m = d.m;
                sa.S = d.S;
                sa.off_pm = d.off_pm;
                sa.off_tot = d.off_tot;
                sa.off_kl = d.off_kl;
                sa.off_rank = d.off_rank;
                sa.off_ptab = d.off_ptab;
                sa.warp_words = d.warp_words;
                sa.bound = b.bound;
                sa.branching = b.branching;
                sa.cap = d.cap;
                sa.K = b.K;
                sa.row_stride = b.row_stride;
                sa.rows_job = b.rows_job;
                sa.rows_lb = b.rows_lb;
                sa.hand_job = b.hand_job;
                sa.hand_lb = b.hand_lb;
                sa.hand_dir = b.hand_dir;
                sa.hand_lc = b.hand_lc;
                sa.inst_of = b.inst_of;
                sa.my_inst = i;
                sa.in_start = b.in_start;
                sa.in_end = b.in_end;
                sa.mailbox = b.mailbox;
                sa.response = b.response;
                sa.len_est = b.len_est;
                sa.active = b.active + i;
                sa.ub = b.ub + i;
                sa.best_key = b.best_key + i;
                sa.best_perm = b.best_perm;
                sa.inst_perm = b.inst_perm + (size_t)64 * i;
                sa.perm_lock = b.perm_lock + i;
                sa.perm_cmax = b.perm_cmax + i;
                sa.counters = b.counters + 8 * i;
                sa.node_limit = b.node_limit;
                unsigned long long now = global_ns(), t0 = *(volatile unsigned long long *)b.t0;
                if (b.time_limit_ns) {
                    unsigned long long end = t0 + b.time_limit_ns;
                    sa.time_limit_ns = now < end ? end - now : 1ull;
                }
                sa.stop = b.stop + i;
                sa.err = b.err;
                sa.min_steal = b.min_steal;
                sa.check_every = b.check_every;
            }
        }
        __syncthreads();
        const int mode = s_mode, i = s_inst;
        if (mode == 0) break;
        stage_tables(smem, sa.tab, sa.tab_words, &bar);
        if (mode == 1 && threadIdx.x == 0) {
            atomicExch(b.active + i, opening_count(sa.n, W));
            __threadfence();
            atomicExch(b.started + i, 1);
        }
        __syncthreads();
        SmemTables T;
        T.pm = smem + sa.off_pm;
        T.pq = nullptr;  // the max-scan fronts are the bounding kernel's
        T.tot = smem + sa.off_tot;
        T.kl = smem + sa.off_kl;
        T.rank = reinterpret_cast<const uint8_t *>(smem + sa.off_rank);
        T.ptab = reinterpret_cast<const int2 *>(smem + sa.off_ptab);
    T.S = (sa.off_ptab - sa.off_rank) / (8 * sa.n);
        WarpScratch Ws = carve_warp(wbase, sa.n, sa.m);
        if (lane == 0) {
            if (mode == 1) opening_interval(sa.n, W, wib, X);
            else {
                for (int q = 0; q < 64; ++q) {
                    X.D[q] = 0;
                    X.E[q] = 0;
                }
                X.etop = 0;
                X.lvl = -1;
            }
            b.len_est[me] = -1.0f;
            __threadfence();
            atomicExch(b.inst_of + me, i);
        }
        __syncwarp();
        switch (sa.m) {
            case 5: run_explorer<NW, 5, kKindBatch>(sa, T, Ws, X, me, nullptr); break;
            case 10: run_explorer<NW, 10, kKindBatch>(sa, T, Ws, X, me, nullptr); break;
            case 20: run_explorer<NW, 20, kKindBatch>(sa, T, Ws, X, me, nullptr); break;
            default: run_explorer<NW, 0, kKindBatch>(sa, T, Ws, X, me, nullptr); break;
        }
        if (lane == 0) atomicExch(b.inst_of + me, -1);
        __syncthreads();
    }
}

template <int NW>
static int batch_occupancy(int warps, size_t smem) {
    auto kern = solve_batch_kernel<NW>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, warps * 32, smem) != cudaSuccess) return 0;
    return per_sm;
}

template <int NW>
static cudaError_t batch_launch(const BatchArgs &b, int blocks, int warps, size_t smem, cudaStream_t st) {
    auto kern = solve_batch_kernel<NW>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg;
    memset(&cfg, 0, sizeof(cfg));
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(warps * 32);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, b);
}

struct BatchPlan {
    int warps = 0, blocks = 0, K = 0;
    size_t smem = 0;
    int nw = 1;
    int max_n = 1, max_tab = 0, warp_stride = 0;
};

static int plan_batch(const pfsp_instance *const *insts, int count, const pfsp_options *opt, BatchPlan &P) {
    for (int i = 0; i < count; ++i) {
        const pfsp_instance *I = insts[i];
        P.max_n = std::max(P.max_n, I->n);
        int tw = opt->bound == PFSP_LB2 ? I->lay.words : I->lay.off_rank;
        P.max_tab = std::max(P.max_tab, tw);
        P.warp_stride = std::max(P.warp_stride, solve_warp_words(I->n, I->m, opt->bound));
    }
    P.nw = P.max_n <= 32 ? 1 : 2;
    int dev = 0, nsm = 1, optin = 48 * 1024;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // a slot (CTA) of `warps` explorers per instance in flight; explorers
    // per SM as asked (a cooperative launch may use fewer CTAs per SM than
    // can be resident), else every resident slot
    const int per_sm_want = opt->warps_per_sm > 0 ? opt->warps_per_sm : 0;
    int warps = opt->slot_warps > 0 ? opt->slot_warps : (per_sm_want > 0 ? per_sm_want : kSolveWarps);
    warps = std::min(warps, kSolveWarps);
    long long fit = ((long long)optin - 256 - (long long)P.max_tab * 4) / ((long long)P.warp_stride * 4);
    warps = (int)std::min<long long>(warps, fit);
    if (warps < 1) return set_error(PFSP_ERR_UNSUPPORTED, "batch explorer state does not fit in shared memory");
    P.smem = (size_t)(P.max_tab + warps * P.warp_stride) * 4;
    int per_sm = P.nw == 1 ? batch_occupancy<1>(warps, P.smem) : batch_occupancy<2>(warps, P.smem);
    if (per_sm < 1) return set_error(PFSP_ERR_CUDA, "batch solve kernel cannot be resident");
    if (per_sm_want > 0) per_sm = std::max(1, std::min(per_sm, per_sm_want / warps));
    P.warps = warps;
    P.blocks = nsm * per_sm;
    P.K = P.blocks * warps;
    return PFSP_OK;
}

}  // namespace pfsp

using namespace pfsp;

extern "C" int pfsp_solve_batch(const pfsp_instance *const *insts, int count, const pfsp_options *opt,
                                const int32_t *init_ubs, int32_t *best_cmax, int32_t *best_perms, int *outcomes,
                                pfsp_stats_t *stats) {
    if (!insts || !opt || !best_cmax || !outcomes || count < 0) return set_error(PFSP_ERR_INVALID, "bad argument");
    if (count == 0) return PFSP_OK;
    if (opt->bound != PFSP_LB1 && opt->bound != PFSP_LB2)
        return set_error(PFSP_ERR_INVALID, "bound must be PFSP_LB1 or PFSP_LB2");
    if (opt->branching < PFSP_MINMIN || opt->branching > PFSP_MINSUM)
        return set_error(PFSP_ERR_INVALID, "branching must be PFSP_MINMIN, PFSP_MINMIN_CAPPED, PFSP_MINBRANCH or PFSP_MINSUM");
    if (opt->node_limit < 0 || opt->time_limit_s < 0) return set_error(PFSP_ERR_INVALID, "negative limit");
    if (opt->learned) return set_error(PFSP_ERR_UNSUPPORTED, "pfsp_solve_batch runs the plain solver only");
    if (opt->heuristic_threads) return set_error(PFSP_ERR_UNSUPPORTED, "pfsp_solve_batch runs no heuristic threads");
    if (opt->lb1_minht) return set_error(PFSP_ERR_UNSUPPORTED, "pfsp_solve_batch runs the plain bounds only");
    int dev = 0;
    cudaGetDevice(&dev);
    for (int i = 0; i < count; ++i) {
        if (!insts[i]) return set_error(PFSP_ERR_INVALID, "instance %d is NULL", i);
        if (insts[i]->device != dev) return set_error(PFSP_ERR_INVALID, "instance %d lives on another device", i);
        if (opt->bound == PFSP_LB2 && !insts[i]->lb2_ok)
            return set_error(PFSP_ERR_UNSUPPORTED, "instance %d: LB2 tables exceed shared memory", i);
    }
    auto t0 = std::chrono::steady_clock::now();
    BatchPlan P;
    int rc = plan_batch(insts, count, opt, P);
    if (rc != PFSP_OK) return rc;

    // incumbents: given, or from NEH per instance
    std::vector<int> ub0(count);
    std::vector<std::vector<int>> neh_perm(count);
    std::vector<char> from_neh(count, 0);
    for (int i = 0; i < count; ++i) {
        if (init_ubs && init_ubs[i] != INT32_MAX) ub0[i] = init_ubs[i];
        else {
            ub0[i] = neh(insts[i]->n, insts[i]->m, insts[i]->p_host, neh_perm[i]);
            from_neh[i] = 1;
        }
    }
    std::vector<InstDesc> desc(count);
    for (int i = 0; i < count; ++i) {
        const pfsp_instance *I = insts[i];
        InstDesc &d = desc[i];
        d.tab = I->d_tab;
        d.tab_words = opt->bound == PFSP_LB2 ? I->lay.words : I->lay.off_rank;
        d.n = I->n;
        d.m = I->m;
        d.S = opt->bound == PFSP_LB2 ? I->lay.Ssweep : 0;
        d.off_pm = I->lay.off_pm;
        d.off_tot = I->lay.off_tot;
        d.off_kl = I->lay.off_kl;
        d.off_rank = I->lay.off_rank;
        d.off_ptab = I->lay.off_ptab;
        d.warp_words = warp_words(I->n, I->m, I->n > 32, opt->bound == PFSP_LB2 && I->m >= 2);
        d.cap = ub0[i];
    }
    const int K = P.K, rs = P.max_n * P.max_n;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = (off + bytes + 255) & ~(size_t)255;
        return o;
    };
    const size_t o_desc = take(sizeof(InstDesc) * count), o_rj = take((size_t)K * rs), o_rl = take((size_t)K * rs * 4);
    const size_t o_is = take((size_t)K * 64), o_ie = take((size_t)K * 65), o_mb = take((size_t)K * 8);
    const size_t o_rs = take((size_t)K * 8), o_le = take((size_t)K * 4), o_bp = take((size_t)K * 64);
    const size_t o_io = take((size_t)K * 4), o_st = take((size_t)count * 4), o_ac = take((size_t)count * 4);
    const size_t o_ub = take((size_t)count * 4), o_bk = take((size_t)count * 8), o_ct = take((size_t)count * 64);
    const size_t o_sp = take((size_t)count * 4), o_misc = take(64);
    const size_t o_ip = take((size_t)count * 64), o_pl = take((size_t)count * 4), o_pc = take((size_t)count * 4);
    const size_t o_hj = take((size_t)K * rs), o_hl = take((size_t)K * rs * 4), o_hd = take((size_t)K * 64),
                 o_hc = take((size_t)K * 4);
    void *blob = nullptr;
    cudaError_t e = cudaMalloc(&blob, off);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(PFSP_ERR_OOM, "cudaMalloc of %zu bytes for the batch explorer pool failed", off);
    }
    char *B = (char *)blob;
    BatchArgs b;
    memset(&b, 0, sizeof(b));
    b.desc = (const InstDesc *)(B + o_desc);
    b.count = count;
    b.bound = opt->bound;
    b.branching = opt->branching;
    b.K = K;
    b.row_stride = rs;
    b.warp_stride = P.warp_stride;
    b.max_tab_words = P.max_tab;
    b.rows_job = (uint8_t *)(B + o_rj);
    b.rows_lb = (int32_t *)(B + o_rl);
    b.hand_job = (uint8_t *)(B + o_hj);
    b.hand_lb = (int32_t *)(B + o_hl);
    b.hand_dir = (uint8_t *)(B + o_hd);
    b.hand_lc = (int *)(B + o_hc);
    b.in_start = (uint8_t *)(B + o_is);
    b.in_end = (uint8_t *)(B + o_ie);
    b.mailbox = (unsigned long long *)(B + o_mb);
    b.response = (unsigned long long *)(B + o_rs);
    b.len_est = (float *)(B + o_le);
    b.best_perm = (uint8_t *)(B + o_bp);
    b.inst_of = (int *)(B + o_io);
    b.started = (int *)(B + o_st);
    b.active = (int *)(B + o_ac);
    b.ub = (int *)(B + o_ub);
    b.best_key = (unsigned long long *)(B + o_bk);
    b.counters = (unsigned long long *)(B + o_ct);
    b.stop = (int *)(B + o_sp);
    b.inst_perm = (uint8_t *)(B + o_ip);
    b.perm_lock = (int *)(B + o_pl);
    b.perm_cmax = (int *)(B + o_pc);
    int *misc = (int *)(B + o_misc);
    b.next = misc;
    b.err = misc + 1;
    b.t0 = (unsigned long long *)(misc + 2);
    b.node_limit = opt->node_limit;
    b.time_limit_ns = opt->time_limit_s > 0 ? (unsigned long long)(opt->time_limit_s * 1e9) : 0ull;
    b.min_steal = opt->min_steal > 0 ? (float)opt->min_steal : 2.0f;
    int ce = opt->check_every > 0 ? opt->check_every : kDefaultCheckEvery, pw = 1;
    while (pw < ce) pw <<= 1;
    b.check_every = pw;

    cudaStream_t st = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    float ms = 0.f;
    std::vector<int> hub(count), hstop(count);
    std::vector<unsigned long long> hkey(count), hcnt((size_t)count * 8);
    int herr = 0;
    e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&ev1);
    // inputs that come from the host are copied before the graph; the graph
    // holds the state resets and the one persistent launch
    if (e == cudaSuccess) e = cudaMemcpyAsync((void *)b.desc, desc.data(), sizeof(InstDesc) * count,
                                              cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.ub, ub0.data(), sizeof(int) * count, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b.perm_cmax, ub0.data(), sizeof(int) * count, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t c = cudaMemsetAsync(b.mailbox, 0xff, (size_t)K * 8, st);
        if (c == cudaSuccess) c = cudaMemsetAsync(b.response, 0, (size_t)K * 8, st);
        if (c == cudaSuccess) c = cudaMemsetAsync(b.len_est, 0, (size_t)K * 4, st);
        if (c == cudaSuccess) c = cudaMemsetAsync(b.inst_of, 0xff, (size_t)K * 4, st);
        if (c == cudaSuccess) c = cudaMemsetAsync(b.started, 0, (size_t)count * 4, st);
        if (c == cudaSuccess) c = cudaMemsetAsync(b.active, 0, (size_t)count * 4, st);
        if (c == cudaSuccess) c = cudaMemsetAsync(b.best_key, 0xff, (size_t)count * 8, st);
        if (c == cudaSuccess) c = cudaMemsetAsync(b.counters, 0, (size_t)count * 64, st);
        if (c == cudaSuccess) c = cudaMemsetAsync(b.stop, 0, (size_t)count * 4, st);
        if (c == cudaSuccess) c = cudaMemsetAsync(b.perm_lock, 0, (size_t)count * 4, st);
        if (c == cudaSuccess) c = cudaMemsetAsync(b.hand_lc, 0xff, (size_t)K * 4, st);
        if (c == cudaSuccess) c = cudaMemsetAsync(misc, 0, 64, st);
        if (c == cudaSuccess) c = P.nw == 1 ? batch_launch<1>(b, P.blocks, P.warps, P.smem, st)
                                            : batch_launch<2>(b, P.blocks, P.warps, P.smem, st);
        e = cudaStreamEndCapture(st, &graph);
        if (c != cudaSuccess) e = c;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
    if (e == cudaSuccess) e = cudaEventRecord(ev0, st);
    if (e == cudaSuccess) e = cudaGraphLaunch(exec, st);
    if (e == cudaSuccess) e = cudaEventRecord(ev1, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hub.data(), b.ub, sizeof(int) * count, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hstop.data(), b.stop, sizeof(int) * count, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hkey.data(), b.best_key, 8 * count, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hcnt.data(), b.counters, 64 * count, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&herr, b.err, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, ev0, ev1);
    std::vector<uint8_t> bp;
    if (e == cudaSuccess && best_perms) {
        bp.resize((size_t)count * 64);
        e = cudaMemcpy(bp.data(), b.inst_perm, bp.size(), cudaMemcpyDeviceToHost);
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    if (st) cudaStreamDestroy(st);
    cudaFree(blob);
    if (e != cudaSuccess) return set_error(PFSP_ERR_CUDA, "pfsp_solve_batch: %s", cudaGetErrorString(e));
    if (herr) return set_error(PFSP_ERR_TIMEOUT, "a bounded device wait expired (detail %d)", herr);

    pfsp_stats_t agg;
    memset(&agg, 0, sizeof(agg));
    for (int i = 0; i < count; ++i) {
        const bool found = hkey[i] != ~0ull;
        if (hstop[i] == 1) outcomes[i] = PFSP_LIMIT_NODES;
        else if (hstop[i] == 2) outcomes[i] = PFSP_LIMIT_TIME;
        else if (found || from_neh[i]) outcomes[i] = PFSP_OPTIMAL;
        else outcomes[i] = PFSP_PROVEN_NO_BETTER;
        best_cmax[i] = hub[i];
        if (best_perms) {
            int32_t *row = best_perms + (size_t)i * 64;
            for (int j = 0; j < 64; ++j) row[j] = -1;
            if (found) {
                const uint8_t *src = bp.data() + (size_t)i * 64;
                for (int j = 0; j < insts[i]->n; ++j) row[j] = src[j];
            } else if (from_neh[i]) {
                for (int j = 0; j < insts[i]->n; ++j) row[j] = neh_perm[i][j];
            }
        }
        agg.decomposed += hcnt[i * 8 + 0];
        agg.bounded_children += hcnt[i * 8 + 1];
        agg.leaves += hcnt[i * 8 + 2];
        agg.pruned += hcnt[i * 8 + 3];
        agg.steals += hcnt[i * 8 + 4];
        agg.iterations += hcnt[i * 8 + 5];
    }
    agg.kernel_seconds = ms * 1e-3;
    agg.explorers = K;
    agg.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = agg;
    return PFSP_OK;
}

// Autotuner: time the batch solve on a sample of the instances for a small
// grid of pool parameters (explorers per SM, explorers per instance slot --
// hence instances in flight per SM --, iterations between publications,
// smallest interval a victim splits) and keep the fastest.  The sample takes
// every (count / k)-th instance, so that it spreads over the batch's mix of
// sizes, and each setting keeps the better of two timings.
extern "C" int pfsp_autotune_batch(const pfsp_instance *const *insts, int count, const pfsp_options *base,
                                   int sample, pfsp_options *best) {
    if (!insts || !base || !best || count < 1) return set_error(PFSP_ERR_INVALID, "bad argument");
    const int k = sample > 0 ? std::min(sample, count) : std::min(count, 32);
    std::vector<const pfsp_instance *> pick(k);
    for (int i = 0; i < k; ++i) pick[i] = insts[(int)((long long)i * count / k)];
    std::vector<int32_t> cm(k), perms;
    std::vector<int> out(k);
    const int per_sm_grid[] = {8, 12};
    const int slot_grid[] = {4, 6, 12};
    const int check_grid[] = {8, 32};
    const double steal_grid[] = {2.0, 40320.0};
    double best_t = 1e300;
    pfsp_options bo = *base;
    for (int e : per_sm_grid)
        for (int w : slot_grid)
            for (int c : check_grid)
                for (double st : steal_grid) {
                    if (w > e) continue;
                    pfsp_options o = *base;
                    o.warps_per_sm = e;
                    o.slot_warps = w;
                    o.check_every = c;
                    o.min_steal = st;
                    double t = 1e300;
                    for (int rep = 0; rep < 2; ++rep) {
                        pfsp_stats_t stt;
                        int rc = pfsp_solve_batch(pick.data(), k, &o, nullptr, cm.data(), nullptr, out.data(), &stt);
                        if (rc != PFSP_OK) return rc;
                        t = std::min(t, stt.kernel_seconds);
                    }
                    if (t < best_t) {
                        best_t = t;
                        bo = o;
                    }
                }
    *best = bo;
    return PFSP_OK;
}
