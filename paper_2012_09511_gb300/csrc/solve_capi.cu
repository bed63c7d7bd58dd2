// solve_capi.cu -- host side of pfsp_solve: initial incumbent (NEH), initial
// partition of the leaf interval [0, n!) among the explorers, device state,
// cooperative launch of the explorer pool and collection of the result.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <cstring>
#include <memory>
#include <thread>
#include <vector>

#include "bound_device.cuh"
#include "heuristic.h"
#include "pfsp_internal.h"
#include "solve_internal.h"

namespace pfsp {

// Completion time of the last job on the last machine of a sequence (Eq. 1).
static int makespan_of(int m, const int32_t *p, const int *seq, int len, std::vector<int> &C) {
    std::fill(C.begin(), C.end(), 0);
    for (int i = 0; i < len; ++i) {
        const int32_t *pj = p + (size_t)seq[i] * m;
        int prev = 0;
        for (int k = 0; k < m; ++k) {
            C[k] = std::max(C[k], prev) + pj[k];
            prev = C[k];
        }
    }
    return C[m - 1];
}

// NEH insertion heuristic (Nawaz, Enscore, Ham 1983) for the initial
// incumbent: jobs by decreasing total time (ties: lower id first), each
// inserted where the partial makespan is least (ties: earliest position).
int neh(int n, int m, const int32_t *p, std::vector<int> &perm) {
    std::vector<int> order(n), tot(n, 0);
    for (int j = 0; j < n; ++j) {
        order[j] = j;
        for (int k = 0; k < m; ++k) tot[j] += p[j * m + k];
    }
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return tot[x] > tot[y]; });
    std::vector<int> seq, cand;
    std::vector<int> C(m);
    for (int j : order) {
        int best_pos = 0, best = INT_MAX;
        for (int pos = 0; pos <= (int)seq.size(); ++pos) {
            cand = seq;
            cand.insert(cand.begin() + pos, j);
            int c = makespan_of(m, p, cand.data(), (int)cand.size(), C);
            if (c < best) {
                best = c;
                best_pos = pos;
            }
        }
        seq.insert(seq.begin() + best_pos, j);
    }
    perm = seq;
    return makespan_of(m, p, seq.data(), n, C);
}

struct DeviceSolveState {
    void *blob = nullptr;
    size_t bytes = 0;
    ~DeviceSolveState() {
        if (blob) cudaFree(blob);
    }
};

}  // namespace pfsp

using namespace pfsp;

// Polls of a thief's answer wait in pfsp_solve (0: the default kWaitLimit);
// set only through the test hook pfsp_set_steal_wait_limit.
static std::atomic<int> g_steal_wait_limit{0};

extern "C" {

int pfsp_set_steal_wait_limit(int polls) {
    if (polls < 0) return set_error(PFSP_ERR_INVALID, "polls must be >= 0");
    g_steal_wait_limit.store(polls);
    return PFSP_OK;
}

void pfsp_default_options(pfsp_options *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->init_ub = INT32_MAX;
    o->bound = PFSP_LB1;
    o->branching = PFSP_MINMIN;
}

struct TraceRequest {
    int64_t capacity;
    int stride;
    uint8_t *perm, *d1, *d2;
    int64_t *count;
};

// Checkpoint buffer (pfsp_solve_resumable): this header, then `count`
// explorer records of kCkptRecord bytes (layout in solve_internal.h).
struct CkptHeader {
    char magic[8];       // "PFSPCKP1"
    int32_t n, m, bound, branching;
    int32_t cap;         // the first segment's initial incumbent (capped MinMin and early exit)
    int32_t ub;          // incumbent (exclusive) when the segment stopped
    int32_t count;       // records that follow
    int32_t have_perm;   // 1: best_perm is a schedule of makespan ub
    uint8_t best_perm[64];
};
static const char kCkptMagic[8] = {'P', 'F', 'S', 'P', 'C', 'K', 'P', '1'};

struct ResumeIO {
    const uint8_t *resume;  // NULL: start from the whole tree
    int64_t resume_bytes;
    uint8_t **ckpt;         // NULL: record nothing
    int64_t *ckpt_bytes;
};

static int solve_impl(const pfsp_instance *inst_c, const pfsp_options *opt, const TraceRequest *tr,
                      const ResumeIO *rio, int32_t *best_cmax, int32_t *best_perm, int *outcome) {
    pfsp_instance *inst = const_cast<pfsp_instance *>(inst_c);
    if (!inst || !opt || !best_cmax || !outcome) return set_error(PFSP_ERR_INVALID, "NULL argument");
    if (opt->bound != PFSP_LB1 && opt->bound != PFSP_LB2)
        return set_error(PFSP_ERR_INVALID, "bound must be PFSP_LB1 or PFSP_LB2");
    if (opt->branching < PFSP_MINMIN || opt->branching > PFSP_MINSUM)
        return set_error(PFSP_ERR_INVALID, "branching must be PFSP_MINMIN, PFSP_MINMIN_CAPPED, PFSP_MINBRANCH or PFSP_MINSUM");
    if (opt->node_limit < 0 || opt->time_limit_s < 0) return set_error(PFSP_ERR_INVALID, "negative limit");
    if (opt->bound == PFSP_LB2 && !inst->lb2_ok)
        return set_error(PFSP_ERR_UNSUPPORTED, "LB2 tables exceed shared memory for this instance");
    if (opt->learned & ~(PFSP_LEARN_CHILD_ORDER | PFSP_LEARN_PAIR_ORDER | PFSP_EARLY_EXIT | PFSP_EARLY_EXIT_SLOTS |
                         PFSP_EARLY_EXIT_CHILDREN))
        return set_error(PFSP_ERR_INVALID, "unknown bits in learned");
    if ((opt->learned & PFSP_EARLY_EXIT_SLOTS) && !(opt->learned & PFSP_EARLY_EXIT))
        return set_error(PFSP_ERR_INVALID, "PFSP_EARLY_EXIT_SLOTS needs PFSP_EARLY_EXIT");
    if ((opt->learned & PFSP_EARLY_EXIT_CHILDREN) && !(opt->learned & PFSP_EARLY_EXIT))
        return set_error(PFSP_ERR_INVALID, "PFSP_EARLY_EXIT_CHILDREN needs PFSP_EARLY_EXIT");
    if ((opt->learned & PFSP_EARLY_EXIT) && opt->branching == PFSP_MINSUM)
        return set_error(PFSP_ERR_INVALID, "PFSP_EARLY_EXIT keeps the tree of MinMin and MinBranch only");
    if (opt->heuristic_threads < 0 || opt->heuristic_threads > 256)
        return set_error(PFSP_ERR_INVALID, "heuristic_threads must be in 0..256");
    if (opt->heuristic_kind < 0 || opt->heuristic_kind > 2)
        return set_error(PFSP_ERR_INVALID, "heuristic_kind must be 0, 1 or 2");
    if (opt->heuristic_threads && (opt->learned & (PFSP_LEARN_CHILD_ORDER | PFSP_LEARN_PAIR_ORDER)))
        return set_error(PFSP_ERR_UNSUPPORTED, "heuristic threads run beside the plain solver only");
    if (opt->lb1_minht != 0 && opt->lb1_minht != 1) return set_error(PFSP_ERR_INVALID, "lb1_minht must be 0 or 1");
    if (opt->heuristic_threads && (opt->phase_timers || tr))
        return set_error(PFSP_ERR_UNSUPPORTED, "phase timers and traces are not taken beside heuristic threads");
    if (opt->lb1_minht && (opt->heuristic_threads || (opt->learned & (PFSP_LEARN_CHILD_ORDER | PFSP_LEARN_PAIR_ORDER))))
        return set_error(PFSP_ERR_UNSUPPORTED, "lb1_minht runs in the plain solver only");
    const bool use_net = (opt->learned & (PFSP_LEARN_CHILD_ORDER | PFSP_LEARN_PAIR_ORDER)) != 0;
    int net_m = 0, net_D0 = 0, net_O = 0;
    if (use_net) {
        if (!opt->mlp) return set_error(PFSP_ERR_INVALID, "learned ordering requested without a network");
        mlp_dims(opt->mlp, &net_m, &net_D0, &net_O);
        if (net_m != inst->m)
            return set_error(PFSP_ERR_INVALID, "network built for m=%d, instance has m=%d", net_m, inst->m);
    }
    auto t0 = std::chrono::steady_clock::now();
    const int n = inst->n, m = inst->m;
    const TableLayout &L = inst->lay;

    // a resumed checkpoint: its header fixes the incumbent and the cap
    CkptHeader rh;
    memset(&rh, 0, sizeof(rh));
    const bool resuming = rio && rio->resume;
    if (resuming) {
        if (rio->resume_bytes < (int64_t)sizeof(CkptHeader))
            return set_error(PFSP_ERR_INVALID, "checkpoint shorter than its header");
        memcpy(&rh, rio->resume, sizeof(rh));
        if (memcmp(rh.magic, kCkptMagic, 8) != 0) return set_error(PFSP_ERR_INVALID, "not a pfsp checkpoint");
        if (rh.n != n || rh.m != m) return set_error(PFSP_ERR_INVALID, "checkpoint of a %d x %d instance", rh.n, rh.m);
        // the bound field carries PFSP_MINHT when the refinement was on
        if (rh.bound != (opt->bound | (opt->lb1_minht ? PFSP_MINHT : 0)) || rh.branching != opt->branching)
            return set_error(PFSP_ERR_INVALID, "checkpoint taken with another bound or branching rule");
        if (rh.count < 0 || rio->resume_bytes != (int64_t)sizeof(CkptHeader) + (int64_t)rh.count * kCkptRecord)
            return set_error(PFSP_ERR_INVALID, "checkpoint size does not match its record count");
    }

    // incumbent: exclusive; INT32_MAX means "start from the NEH schedule"
    std::vector<int> neh_perm;
    int ub0 = opt->init_ub;
    bool from_neh = false;
    if (resuming) {
        ub0 = rh.ub;
        if (rh.have_perm) {
            from_neh = true;  // a schedule of makespan ub0 is known (returned if nothing better is found)
            neh_perm.assign(rh.best_perm, rh.best_perm + n);
        }
    } else if (ub0 == INT32_MAX) {
        ub0 = neh(n, m, inst->p_host, neh_perm);
        from_neh = true;
    }

    // launch shape: explorers per CTA limited by shared memory, one CTA per SM
    SolveArgs a;
    memset(&a, 0, sizeof(a));
    a.tab = inst->d_tab;
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
    a.minht = opt->lb1_minht;
    a.diag = (opt->phase_timers || tr) ? 1 : 0;
    a.cap = resuming ? rh.cap : ub0;
    a.wait_limit = g_steal_wait_limit.load();
    a.warp_words = warp_words(n, m, n > 32, opt->bound == PFSP_LB2 && m >= 2);
    // the network's inference image: every output column when it orders the
    // LB2 slots, else only the descend-first column (one 16-column tile)
    const int net_O3 = use_net ? ((opt->learned & PFSP_LEARN_PAIR_ORDER) ? net_O : 16) : 0;
    const int img_bytes = use_net ? mlp_image_bytes(net_D0, net_O3) : 0;
    if (use_net) {
        a.warp_words += mlp_scratch_place(n, m, opt->bound, net_D0, &a.mlp_off);
        a.net_D0 = net_D0;
        a.net_O3 = net_O3;
        long long tot = 0;
        for (int j = 0; j < n * m; ++j) tot += inst->p_host[j];
        a.inv_scale = tot > 0 ? (float)m / (float)tot : 1.0f;
    }
    a.learned = opt->learned;
    a.learn_depth = opt->learn_depth > 0 ? opt->learn_depth : n;
    a.warp_words = (a.warp_words + 7) & ~7;  // keeps every warp's scratch 32-byte aligned
    a.warp_base = (a.tab_words + 7) & ~7;
    const int per_warp = a.warp_words + (solve_warp_words(n, m, opt->bound) -
                                         warp_words(n, m, n > 32, opt->bound == PFSP_LB2 && m >= 2));
    int dev = 0, nsm = 1, optin = 48 * 1024;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int max_warps = use_net ? kSolveWarpsLearned : kSolveWarps;
    int warps = opt->warps_per_sm > 0 ? std::min(opt->warps_per_sm, max_warps) : max_warps;
    // the network's image stays in global memory (its weights are read there
    // by the tensor-core fragments), so it costs no explorer warps
    long long fit = ((long long)optin - 256 - (long long)a.warp_base * 4) / ((long long)per_warp * 4);
    // each explorer's rows (jobs and bounds of every level) go to shared
    // memory, after its explorer state, when that costs no explorer warps:
    // selection and decoding then read them on chip instead of from L2
    const int rows_words = solve_row_words(n);
    long long fit_rows =
        ((long long)optin - 256 - (long long)a.warp_base * 4) / ((long long)(per_warp + rows_words) * 4);
    int per_warp_eff = per_warp;
    if (std::min<long long>(warps, fit_rows) >= std::min<long long>(warps, fit)) {
        a.rows_smem = 1;
        per_warp_eff = per_warp + rows_words;
        fit = fit_rows;
    }
    warps = (int)std::min<long long>(warps, fit);
    if (warps < 1) return set_error(PFSP_ERR_UNSUPPORTED, "explorer state does not fit in shared memory");
    size_t smem = (size_t)(a.warp_base + warps * per_warp_eff) * 4;
    // host heuristic threads (Section 4.2), exchanging with the explorers
    // through host-mapped memory; a.coop also selects their kernel
    std::unique_ptr<HeuristicPool> hp;
    std::vector<int> h_start;
    if (opt->heuristic_threads > 0) {
        hp.reset(new HeuristicPool(n, m, inst->p_host, opt->heuristic_threads, (uint64_t)(uint32_t)opt->heuristic_seed,
                                   opt->heuristic_kind));
        if (!hp->ok()) return set_error(PFSP_ERR_OOM, "host-mapped memory for the heuristic threads");
        a.coop = hp->device_shared();
        if ((int)neh_perm.size() == n) h_start = neh_perm;
        else neh(n, m, inst->p_host, h_start);
    }
    int per_sm = solve_occupancy(a, warps, smem);
    if (per_sm < 1) return set_error(PFSP_ERR_CUDA, "solve kernel cannot be resident (occupancy 0)");
    // explorers per SM as asked: a cooperative launch may use fewer CTAs per
    // SM than can be resident (default: every resident CTA)
    if (opt->warps_per_sm > 0) per_sm = std::max(1, std::min(per_sm, opt->warps_per_sm / warps));
    const int blocks = nsm * per_sm;
    const int K = blocks * warps;
    a.K = K;
    a.row_stride = n * n;
    a.inst_of = nullptr;
    a.my_inst = 0;
    a.inst_perm = nullptr;
    a.perm_lock = nullptr;
    a.perm_cmax = nullptr;

    if (hp) {
        if (!hp->attach(K)) return set_error(PFSP_ERR_OOM, "host-mapped memory for the heuristic threads");
        a.coop_slots = hp->device_slots();
    }

    // initial partition of [0, n!): equal chunks of the first L levels
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
    std::vector<uint8_t> hl((size_t)K, 0xff);
    int active0 = (int)Kp;
    if (resuming) {
        if (rh.count > K)
            return set_error(PFSP_ERR_UNSUPPORTED, "checkpoint holds %d intervals, this launch has %d explorers",
                             rh.count, K);
        std::fill(hs.begin(), hs.end(), 0);
        std::fill(he.begin(), he.end(), 0);
        const uint8_t *rec = rio->resume + sizeof(CkptHeader);
        for (int i = 0; i < rh.count; ++i, rec += kCkptRecord) {
            for (int q = 0; q < n; ++q) {
                if (rec[4 + q] >= n - q || rec[68 + q] >= n - q)
                    return set_error(PFSP_ERR_INVALID, "checkpoint record %d holds an invalid digit", i);
                hs[(size_t)i * 64 + q] = rec[4 + q];
                he[(size_t)i * 65 + 1 + q] = rec[68 + q];
            }
            if (rec[1] != 0xff && rec[1] > n - 2)
                return set_error(PFSP_ERR_INVALID, "checkpoint record %d holds an invalid level", i);
            he[(size_t)i * 65] = rec[2] ? 1 : 0;
            hl[(size_t)i] = rec[1];
        }
        active0 = rh.count;
    }

    // device state, one allocation
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = (off + bytes + 255) & ~(size_t)255;
        return o;
    };
    const size_t o_rj = take((size_t)K * n * n), o_rl = take((size_t)K * n * n * 4);
    const size_t o_is = take((size_t)K * 64), o_ie = take((size_t)K * 65);
    const size_t o_mb = take((size_t)K * 8), o_rs = take((size_t)K * 8), o_le = take((size_t)K * 4);
    const size_t o_bp = take((size_t)K * 64), o_ct = take(8 * 8), o_sc = take(64), o_ph = take(8 * kPhases);
    const size_t o_lv = take((size_t)K), o_sp = take((size_t)K * 4), o_sq = take((size_t)K * 4);
    const size_t o_hd = take((size_t)K * 64), o_hc = take((size_t)K * 4);
    // hand-off rows: the explorers' own global rows when their rows live in
    // shared memory (unused then), else a buffer of their own
    const size_t o_hj = take(a.rows_smem ? 0 : (size_t)K * n * n), o_hl = take(a.rows_smem ? 0 : (size_t)K * n * n * 4);
    const bool want_ckpt = rio && rio->ckpt;
    const size_t o_ck = take(want_ckpt ? (size_t)K * kCkptRecord : 0);
    const int64_t tcap = tr ? tr->capacity : 0;
    const size_t o_tp = take((size_t)tcap * n), o_t1 = take((size_t)tcap), o_t2 = take((size_t)tcap),
                 o_tc = take(8);
    const size_t o_img = take((size_t)img_bytes);
    DeviceSolveState D;
    cudaError_t e = cudaMalloc(&D.blob, off);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return set_error(PFSP_ERR_OOM, "cudaMalloc of %zu bytes for the explorer pool failed", off);
    }
    char *b = (char *)D.blob;
    a.rows_job = (uint8_t *)(b + o_rj);
    a.rows_lb = (int32_t *)(b + o_rl);
    a.in_start = (uint8_t *)(b + o_is);
    a.in_end = (uint8_t *)(b + o_ie);
    a.mailbox = (unsigned long long *)(b + o_mb);
    a.response = (unsigned long long *)(b + o_rs);
    a.len_est = (float *)(b + o_le);
    a.best_perm = (uint8_t *)(b + o_bp);
    a.in_level = (uint8_t *)(b + o_lv);
    a.seq_posted = (unsigned *)(b + o_sp);
    a.seq_taken = (unsigned *)(b + o_sq);
    a.hand_dir = (uint8_t *)(b + o_hd);
    a.hand_lc = (int *)(b + o_hc);
    a.hand_job = a.rows_smem ? a.rows_job : (uint8_t *)(b + o_hj);
    a.hand_lb = a.rows_smem ? a.rows_lb : (int32_t *)(b + o_hl);
    a.ckpt = want_ckpt ? (uint8_t *)(b + o_ck) : nullptr;
    a.counters = (unsigned long long *)(b + o_ct);
    a.phase = opt->phase_timers ? (unsigned long long *)(b + o_ph) : nullptr;
    int *sc = (int *)(b + o_sc);  // active, ub, stop, err, best_key (8 bytes at +16)
    a.active = sc + 0;
    a.ub = sc + 1;
    a.stop = sc + 2;
    a.err = sc + 3;
    a.best_key = (unsigned long long *)(sc + 4);
    if (use_net) a.net_image = (const unsigned char *)(b + o_img);
    a.node_limit = opt->node_limit;
    a.time_limit_ns = opt->time_limit_s > 0 ? (unsigned long long)(opt->time_limit_s * 1e9) : 0ull;
    a.min_steal = opt->min_steal > 0 ? (float)opt->min_steal : default_min_steal(n);
    if (tcap > 0) {
        a.trace_perm = (uint8_t *)(b + o_tp);
        a.trace_d1 = (uint8_t *)(b + o_t1);
        a.trace_d2 = (uint8_t *)(b + o_t2);
        a.trace_count = (unsigned long long *)(b + o_tc);
        a.trace_cap = tcap;
        a.trace_stride = tr->stride > 0 ? tr->stride : 1;
    }
    int ce = opt->check_every > 0 ? opt->check_every : kDefaultCheckEvery;
    int pw = 1;
    while (pw < ce) pw <<= 1;
    a.check_every = pw;

    int hsc[6] = {active0, ub0, 0, 0, -1, -1};  // best_key = ~0
    cudaStream_t st = 0;
    cudaEvent_t ev0, ev1;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    e = cudaMemsetAsync(a.mailbox, 0xff, (size_t)K * 8, st);
    if (e == cudaSuccess && use_net) e = mlp_build_image(opt->mlp, net_O3, (void *)a.net_image, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.response, 0, (size_t)K * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.len_est, 0, (size_t)K * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.counters, 0, 64, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(b + o_ph, 0, 8 * kPhases, st);
    if (e == cudaSuccess && tcap > 0) e = cudaMemsetAsync(a.trace_count, 0, 8, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(a.in_start, hs.data(), hs.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(a.in_end, he.data(), he.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(a.in_level, hl.data(), hl.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.seq_posted, 0, (size_t)K * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.seq_taken, 0, (size_t)K * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.hand_lc, 0xff, (size_t)K * 4, st);
    if (e == cudaSuccess && want_ckpt) e = cudaMemsetAsync(a.ckpt, 0, (size_t)K * kCkptRecord, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sc, hsc, sizeof(hsc), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaEventRecord(ev0, st);
    if (e == cudaSuccess) e = launch_solve(a, blocks, warps, smem, st);
    if (e == cudaSuccess) e = cudaEventRecord(ev1, st);
    if (e == cudaSuccess && hp) {
        // the heuristic threads search while the explorers run; this thread
        // drives the snapshots until the kernel is done (before the result
        // copies below, which wait for it)
        hp->start(ub0, h_start);
        cudaError_t q;
        while ((q = cudaEventQuery(ev1)) == cudaErrorNotReady) {
            hp->tick();
            std::this_thread::sleep_for(std::chrono::microseconds(50));
        }
        hp->stop();
        if (q != cudaSuccess) e = q;
    }
    int rsc[6];
    unsigned long long cnt[8], ph[kPhases];
    if (e == cudaSuccess) e = cudaMemcpyAsync(rsc, sc, sizeof(rsc), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(cnt, a.counters, sizeof(cnt), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ph, b + o_ph, sizeof(ph), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, ev0, ev1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (e != cudaSuccess) return set_error(PFSP_ERR_CUDA, "pfsp_solve: %s", cudaGetErrorString(e));
    if (rsc[3] != 0) return set_error(PFSP_ERR_TIMEOUT, "a bounded device wait expired (detail %d)", rsc[3]);

    unsigned long long key;
    memcpy(&key, &rsc[4], sizeof(key));
    const int final_ub = rsc[1];
    bool found = key != ~0ull;
    std::vector<uint8_t> bp(64);
    if (found) {
        int eid = (int)(key & 0xffffffffu);
        e = cudaMemcpy(bp.data(), a.best_perm + (size_t)eid * 64, 64, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return set_error(PFSP_ERR_CUDA, "pfsp_solve readback: %s", cudaGetErrorString(e));
    }
    // the best schedule: the explorers' record when it reaches the final
    // incumbent, else the heuristic threads' (whose makespan the explorers
    // took as their incumbent, or found after the explorers stopped at a
    // limit), else the initial one
    std::vector<int> hperm;
    const int hc = hp ? hp->best(&hperm) : INT_MAX;
    const int best = std::min(final_ub, hc);
    const bool dev_best = found && (int)(key >> 32) == best;
    const bool heur_best = !dev_best && hc == best && hc != INT_MAX;
    const bool have_perm = dev_best || heur_best || from_neh;
    std::vector<int> fperm(n, -1);
    for (int j = 0; j < n && have_perm; ++j) fperm[j] = dev_best ? bp[j] : heur_best ? hperm[j] : neh_perm[j];
    if (rsc[2] == 1) *outcome = PFSP_LIMIT_NODES;
    else if (rsc[2] == 2) *outcome = PFSP_LIMIT_TIME;
    else if (have_perm) *outcome = PFSP_OPTIMAL;
    else *outcome = PFSP_PROVEN_NO_BETTER;
    *best_cmax = best;
    if (best_perm && have_perm)
        for (int j = 0; j < n; ++j) best_perm[j] = fperm[j];
    if (want_ckpt) {
        *rio->ckpt = nullptr;
        *rio->ckpt_bytes = 0;
    }
    if (want_ckpt && (rsc[2] == 1 || rsc[2] == 2)) {
        // the explorers' own records, plus intervals granted to thieves that
        // stopped before taking them in (their answer sits in the response slot)
        std::vector<uint8_t> rec((size_t)K * kCkptRecord), ins((size_t)K * 64), ine((size_t)K * 65), inl((size_t)K);
        std::vector<unsigned long long> resp((size_t)K);
        std::vector<unsigned> sp((size_t)K), sq((size_t)K);
        e = cudaMemcpy(rec.data(), a.ckpt, rec.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(ins.data(), a.in_start, ins.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(ine.data(), a.in_end, ine.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(inl.data(), a.in_level, inl.size(), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(resp.data(), a.response, resp.size() * 8, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(sp.data(), a.seq_posted, sp.size() * 4, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(sq.data(), a.seq_taken, sq.size() * 4, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return set_error(PFSP_ERR_CUDA, "checkpoint readback: %s", cudaGetErrorString(e));
        std::vector<uint8_t> out;
        for (int t = 0; t < K; ++t) {
            const uint8_t *r = &rec[(size_t)t * kCkptRecord];
            if (r[0]) out.insert(out.end(), r, r + kCkptRecord);
            const unsigned long long v = resp[t];
            if ((v & 3ull) == 1ull && (unsigned)(v >> 2) == sp[t] && sq[t] != sp[t]) {
                uint8_t g[kCkptRecord];
                memset(g, 0, sizeof(g));
                g[0] = 1;
                g[1] = inl[t];
                g[2] = ine[(size_t)t * 65];
                memcpy(g + 4, &ins[(size_t)t * 64], 64);
                memcpy(g + 68, &ine[(size_t)t * 65 + 1], 64);
                out.insert(out.end(), g, g + kCkptRecord);
            }
        }
        CkptHeader h;
        memset(&h, 0, sizeof(h));
        memcpy(h.magic, kCkptMagic, 8);
        h.n = n;
        h.m = m;
        h.bound = opt->bound | (opt->lb1_minht ? PFSP_MINHT : 0);
        h.branching = opt->branching;
        h.cap = a.cap;
        h.ub = best;
        h.count = (int32_t)(out.size() / kCkptRecord);
        h.have_perm = have_perm ? 1 : 0;
        for (int j = 0; j < n; ++j) h.best_perm[j] = (uint8_t)(have_perm ? fperm[j] : 0xff);
        const size_t bytes = sizeof(h) + out.size();
        uint8_t *buf = (uint8_t *)malloc(bytes);
        if (!buf) return set_error(PFSP_ERR_OOM, "host allocation of the checkpoint failed");
        memcpy(buf, &h, sizeof(h));
        if (!out.empty()) memcpy(buf + sizeof(h), out.data(), out.size());
        *rio->ckpt = buf;
        *rio->ckpt_bytes = (int64_t)bytes;
    }
    if (tcap > 0) {
        unsigned long long tc = 0;
        e = cudaMemcpy(&tc, a.trace_count, 8, cudaMemcpyDeviceToHost);
        const int64_t got = (int64_t)std::min<unsigned long long>(tc, (unsigned long long)tcap);
        if (e == cudaSuccess && got > 0) e = cudaMemcpy(tr->perm, a.trace_perm, (size_t)got * n, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && got > 0) e = cudaMemcpy(tr->d1, a.trace_d1, (size_t)got, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && got > 0) e = cudaMemcpy(tr->d2, a.trace_d2, (size_t)got, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return set_error(PFSP_ERR_CUDA, "trace readback: %s", cudaGetErrorString(e));
        *tr->count = got;
    }
    memset(&inst->stats, 0, sizeof(inst->stats));
    inst->stats.decomposed = cnt[0];
    inst->stats.bounded_children = cnt[1];
    inst->stats.leaves = cnt[2];
    inst->stats.pruned = cnt[3];
    inst->stats.steals = cnt[4];
    inst->stats.iterations = cnt[5];
    inst->stats.lb2_slots = cnt[7];
    inst->stats.kernel_seconds = ms * 1e-3;
    inst->stats.final_ub = best;
    inst->stats.explorers = K;
    inst->stats.heuristic_improvements = hp ? hp->improvements() : 0;
    inst->stats.promoted = hp ? hp->promoted() : 0;
    inst->stats.heuristic_cmax = hp ? hp->own_best() : INT_MAX;
    inst->stats.snapshots = hp ? hp->snapshots() : 0;
    for (int p = 0; p < kPhases; ++p) inst->stats.phase_cycles[p] = ph[p];
    inst->stats.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return PFSP_OK;
}

int pfsp_solve(const pfsp_instance *inst, const pfsp_options *opt, int32_t *best_cmax, int32_t *best_perm,
               int *outcome) {
    return solve_impl(inst, opt, nullptr, nullptr, best_cmax, best_perm, outcome);
}

int pfsp_solve_resumable(const pfsp_instance *inst, const pfsp_options *opt, const uint8_t *resume,
                         int64_t resume_bytes, uint8_t **checkpoint, int64_t *checkpoint_bytes, int32_t *best_cmax,
                         int32_t *best_perm, int *outcome) {
    if (resume && resume_bytes <= 0) return set_error(PFSP_ERR_INVALID, "resume buffer without a size");
    if (checkpoint && !checkpoint_bytes) return set_error(PFSP_ERR_INVALID, "checkpoint_bytes is NULL");
    ResumeIO rio{resume, resume_bytes, checkpoint, checkpoint_bytes};
    return solve_impl(inst, opt, nullptr, &rio, best_cmax, best_perm, outcome);
}

void pfsp_free_checkpoint(uint8_t *checkpoint) { free(checkpoint); }

int pfsp_solve_trace(const pfsp_instance *inst, const pfsp_options *opt, int64_t capacity, int stride,
                     uint8_t *perm, uint8_t *d1, uint8_t *d2, int64_t *count, int32_t *best_cmax, int *outcome) {
    if (capacity < 0 || !count || (capacity > 0 && (!perm || !d1 || !d2)))
        return set_error(PFSP_ERR_INVALID, "bad trace buffers");
    TraceRequest tr{capacity, stride, perm, d1, d2, count};
    *count = 0;
    return solve_impl(inst, opt, &tr, nullptr, best_cmax, nullptr, outcome);
}

}  // extern "C"
