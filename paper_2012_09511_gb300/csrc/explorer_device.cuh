// explorer_device.cuh -- one depth-first explorer per warp: IVM-like state,
// selection, decomposition with MinMin, interval work stealing (Sections 2.5,
// 2.6, 3.1-3.4 of the paper).  Shared by the single-instance and the batched
// explorer-pool kernels.
#pragma once

#include <cfloat>
#include <climits>

#include "bound_device.cuh"
#include "minht_device.cuh"
#include "pfsp_internal.h"
#include "solve_internal.h"

namespace pfsp {

__device__ inline unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ inline int ld_volatile(const int *p) { return *(const volatile int *)p; }

// Per-warp explorer scratch in shared memory (int words).
// LB2 slots of the largest machine count the ordering network supports
// (m = 20: 190 pairs).
constexpr int kMaxSlots = 6;

struct ExplorerSmem {
    int V[64];      // digit selected at each level
    int dir[64];    // branching direction of each level (0 fwd, 1 bwd)
    int E[64];      // end of the interval (digits); etop = coefficient of n!
    int D[64];      // start of an incoming interval
    int perm[64];   // staging of the decoded node
    float lw[64];   // log2 (n-1-i)!, for length estimates
    int etop;
    unsigned seq;   // sequence number of this explorer's last steal request
    int lvl;        // start level of the interval (-1: the first level below which D is all zero)
    int last_d1, last_d2;  // depths of the node staged in perm (the last one decomposed)
    int pad[3];
    float score[64];   // descend-first logits of the children being ordered
    float sscore[16];  // summed pair probabilities per LB2 slot
    int sorder[16];    // LB2 slot order of the current node
    unsigned long long ph[kPhases];  // SM clock cycles spent in each phase (lane 0 updates)
};
constexpr int kExplorerWords = (64 * 5 + 64 + 8 + 64 + 16 + 16 + 2 * kPhases);  // a multiple of 8 words
static_assert(sizeof(ExplorerSmem) == 4 * kExplorerWords, "explorer scratch size");
static_assert(kExplorerWords % 8 == 0, "explorer scratch keeps 32-byte alignment");

struct Stats {
    unsigned long long decomposed, bounded, leaves, pruned, steals, iters, slots;
};

// KIND selects the instantiation: kKindPlain, kKindLearned (runs the ordering
// network), kKindCoop (exchanges with the host heuristic threads), kKindMinht
// (refined LB1), kKindLb1 (LB1 solves, without the LB2 sweep), kKindDiag
// (phase timers and traces) or kKindEE (early exit of the LB2 sweep).  Each
// kernel carries only its own code: the explorer loop is bound by
// instruction fetch, so even code that never runs slows it down.
template <int NW, int MT, int KIND>
struct Explorer {
    static constexpr bool LEARNED = KIND == kKindLearned;
    static constexpr bool COOP = KIND == kKindCoop;
    static constexpr bool MINHT = KIND == kKindMinht;
    static constexpr bool LB1_ONLY = KIND == kKindLb1;
    // phase timers and decomposition traces: compiled out of the fast kernels
    // (plain LB2, LB1-only, and the one beside the heuristic threads), which
    // run solves that ask for neither
    static constexpr bool DIAG = KIND != kKindPlain && KIND != kKindBatch && KIND != kKindLb1 && KIND != kKindCoop &&
                                 KIND != kKindEE;
    // early exit of the LB2 sweep: compiled out of the plain kernels
    static constexpr bool EARLY = KIND != kKindPlain && KIND != kKindBatch && KIND != kKindLb1;
    // the batched pool inlines one explorer per machine count into a single
    // kernel: its sweep leaves out the code that only saves instructions
    // (lb2_sweep's LEAN), which there costs spills
    static constexpr bool LEAN = KIND == kKindBatch;
    const SolveArgs &a;
    const SmemTables &T;
    const WarpScratch &W;
    ExplorerSmem &X;
    const MlpImage *net;  // view of the network's image in global memory (NULL: plain solver)
    int n, m, S, lane, me;
    uint8_t *rj;
    int32_t *rl;
    int I;  // current level (-1: at the root)
    Stats st;
    unsigned rng;
    unsigned long long pending_nodes;
    unsigned long long deadline;
    long long t_mark;  // SM clock at the end of the last timed phase (lane 0)
    bool timed;        // phase timers on (a.phase != NULL)
    int ub_seen;       // incumbent read at the top of the current iteration
    int hand_level;    // >= 0: rows 0..hand_level of a new interval's path were handed over
    int snap_seen;     // last snapshot request of the host heuristic threads answered

    __device__ Explorer(const SolveArgs &a_, const SmemTables &T_, const WarpScratch &W_, ExplorerSmem &X_, int me_,
                        const MlpImage *net_)
        : a(a_), T(T_), W(W_), X(X_), net(net_), me(me_) {
        n = a.n;
        m = a.m;
        S = a.S;
        lane = threadIdx.x & 31;
        rj = a.rows_job + (size_t)me * a.row_stride;
        rl = a.rows_lb + (size_t)me * a.row_stride;
        if (a.rows_smem) {  // rows in shared memory, right after the explorer state
            int32_t *rb = reinterpret_cast<int32_t *>(&X_) + kExplorerWords;
            rl = rb;
            rj = reinterpret_cast<uint8_t *>(rb + a.n * a.n);
        }
        I = -1;
        st = Stats{0, 0, 0, 0, 0, 0, 0};
        rng = 0x9e3779b9u * (me + 1) ^ 0x85ebca6bu;
        pending_nodes = 0;
        deadline = a.time_limit_ns ? global_ns() + a.time_limit_ns : 0ull;
        for (int i = lane; i < 64; i += 32) {
            float lw = 0.0f;
            for (int t = 2; t <= n - 1 - i; ++t) lw += log2f((float)t);
            X.lw[i] = lw;
        }
        timed = a.phase != nullptr;
        ub_seen = INT_MAX;
        snap_seen = 0;
        hand_level = -1;
        if (lane < kPhases) X.ph[lane] = 0ull;
        t_mark = timed ? clock64() : 0;
        __syncwarp();
    }

    // Charge the cycles since the last mark to phase p (lane 0; the sums are
    // reported per solve).  A uniform test when the timers are off.
    __device__ __forceinline__ void tick(int p) {
        if (DIAG && timed && lane == 0) {
            const long long t = clock64();
            X.ph[p] += (unsigned long long)(t - t_mark);
            t_mark = t;
        }
    }

    // warp-uniform reads of shared counters (lane 0 loads, all lanes agree)
    __device__ int ub() const {
        int v = 0;
        if (lane == 0) v = ld_volatile(a.ub);
        return __shfl_sync(PFSP_FULL, v, 0);
    }
    // rows handed over with stolen intervals (SolveArgs.hand_*)
    __device__ bool handoff_on() const { return a.hand_dir != nullptr; }

    __device__ int active_count() const {
        int v = 0;
        if (lane == 0) v = ld_volatile(a.active);
        return __shfl_sync(PFSP_FULL, v, 0);
    }

    // lo(current position) < end ?  Position digits are V[0..I], zeros below.
    __device__ bool pos_before_end() const {
        if (X.etop) return true;
        for (int h = 0; h < NW; ++h) {
            int i = lane + 32 * h;
            int v = (i < n && i <= I) ? X.V[i] : 0;
            int e = i < n ? X.E[i] : 0;
            unsigned diff = __ballot_sync(PFSP_FULL, v != e);
            if (diff) {
                int f = __ffs(diff) - 1;
                int vf = __shfl_sync(PFSP_FULL, v, f), ef = __shfl_sync(PFSP_FULL, e, f);
                return vf < ef;
            }
        }
        return false;  // equal
    }

    // The length of the remaining interval [pos, end) (pos = V[0..I] with
    // zeros below, end = E plus etop * n!) as acc * (n-1-lv)!, in integer
    // arithmetic (the FP64 units of this GPU are few and slow).  The digit
    // differences are folded level by level with Horner's rule in the
    // factorial base (the weight of level i-1 is n-i times that of level i),
    // from level i0 (every level above it equal in pos and end; 0 with etop)
    // until acc reaches 2^24 or the last level is folded.  The levels left out
    // add less than one unit of (n-1-lv)!, so acc * (n-1-lv)! is the length to
    // within a relative 2^-24, and exactly when lv = n - 1.  A prefix of end is
    // never below the same prefix of pos, so acc >= 0.  One lane.
    __device__ int fold_length(int i0, int &lv) const {
        int acc = X.etop, i = X.etop ? 0 : i0;
        for (; i < n; ++i) {
            acc = acc * (n - i) + (X.E[i] - (i <= I ? X.V[i] : 0));  // < 2^30
            if (acc >= (1 << 24)) break;
        }
        lv = min(i, n - 1);
        return acc;
    }

    // log2 of (end - pos), or -1 if empty (estimate for victim choice only);
    // the value of lane 0
    __device__ float log2_length() const {
        int i0 = n;
        for (int h = NW - 1; h >= 0; --h) {
            const int i = lane + 32 * h;
            const unsigned d = __ballot_sync(PFSP_FULL, i < n && X.E[i] != (i <= I ? X.V[i] : 0));
            if (d) i0 = 32 * h + __ffs(d) - 1;
        }
        float l = -1.0f;
        if (lane == 0) {
            int lv;
            const int acc = fold_length(i0, lv);
            if (acc >= 1) l = __log2f((float)acc) + X.lw[lv];
        }
        return l;
    }

    // Find the next node: the first live cell at or after V[I] on level I,
    // backtracking when a row is exhausted (Section 2.5, selection).
    __device__ bool select() {
        while (I >= 0) {
            const int len = n - I;
            const int v = X.V[I];
            const int ubv = ub_seen;
            unsigned b0 = 0, b1 = 0;
            {
                int c = lane;
                bool ok = c < len && c >= v && rl[I * n + c] < ubv;
                b0 = __ballot_sync(PFSP_FULL, ok);
            }
            if (NW == 2 && !b0) {
                int c = lane + 32;
                bool ok = c < len && c >= v && rl[I * n + c] < ubv;
                b1 = __ballot_sync(PFSP_FULL, ok);
            }
            if (b0 | b1) {
                int c = b0 ? __ffs(b0) - 1 : 32 + __ffs(b1) - 1;
                if (lane == 0) X.V[I] = c;
                __syncwarp();
                return true;
            }
            --I;
            if (I >= 0 && lane == 0) X.V[I] += 1;
            __syncwarp();
        }
        return false;
    }

    // Network scratch of this warp (32-byte aligned).
    __device__ unsigned char *mlp_scratch() const { return (unsigned char *)((int *)W.FRB + a.mlp_off); }

    // Layers 1 and 2 of the network on the tile Xs (fused, in registers),
    // layer 2's activations handed to sink k-tile by k-tile.
    template <class Sink>
    __device__ void net_hidden(const __nv_bfloat16 *Xs, __nv_bfloat16 *H1, Sink &&sink) const {
        constexpr int KT = MT ? (3 * MT + 15) / 16 : 0;
        if constexpr (KT > 0) {
            mlp_fused_hidden<KT>(*net, Xs, H1, sink);
        } else {
            switch (net->D0 >> 4) {
                case 1: mlp_fused_hidden<1>(*net, Xs, H1, sink); break;
                case 2: mlp_fused_hidden<2>(*net, Xs, H1, sink); break;
                case 3: mlp_fused_hidden<3>(*net, Xs, H1, sink); break;
                default: mlp_fused_hidden<4>(*net, Xs, H1, sink); break;
            }
        }
    }

    // Order of the LB2 slots for the node whose front, back and remaining
    // work sit in W.FRB: by decreasing sum over the slot's pairs of
    // the network's probability that the pair attains a child's LB2.
    __device__ void slot_order() {
        const MlpImage &P = *net;
        const int ldx = P.D0 + 8;
        __nv_bfloat16 *Xs = (__nv_bfloat16 *)mlp_scratch();
        for (int e = lane; e < 16 * ldx; e += 32) Xs[e] = __float2bfloat16_rn(0.0f);
        __syncwarp();
        if (lane < m) {
            const int4 F = W.FRB[lane];
            Xs[lane] = __float2bfloat16_rn(F.x * a.inv_scale);
            Xs[m + lane] = __float2bfloat16_rn(F.z * a.inv_scale);
            Xs[2 * m + lane] = __float2bfloat16_rn(F.y * a.inv_scale);
        }
        if (lane < 16) X.sscore[lane] = 0.0f;
        __syncwarp();
        __nv_bfloat16 *H1 = Xs + 16 * ldx, *H2 = H1 + 16 * (kMlpHidden + 8);
        net_hidden(Xs, H1, MlpPark{H2});
        // row 0 (the parent) sits in lanes 0..3: columns 16p + 2t (+1) and
        // 16p + 8 + 2t (+1).  The pair probabilities go to the input tile,
        // free once layer 1 has run, one float per pair in column order.
        const int npairs = m * (m - 1) / 2;
        const int t = lane & 3;
        float *prob = reinterpret_cast<float *>(Xs);
        for (int p = 0; p < P.O3 / 16; ++p) {
            float c0[4], c1[4];
            mlp_tile_cols<kMlpHidden / 16>(H2, kMlpHidden + 8, P.W3t, kMlpHidden + 8, p, c0, c1);
            if (lane < 4) {
                const int cols[4] = {16 * p + 2 * t, 16 * p + 2 * t + 1, 16 * p + 8 + 2 * t, 16 * p + 9 + 2 * t};
                const float z[4] = {c0[0], c0[1], c1[0], c1[1]};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int col = cols[i];
                    if (col >= 1 && col <= npairs) prob[col - 1] = 1.0f / (1.0f + expf(-(z[i] + P.b3[col])));
                }
            }
        }
        __syncwarp();
        // summed over the pairs that each slot holds (the instance's pair order)
        for (int s2 = 0; s2 < S; ++s2) {
            const int klw = T.kl[s2 * 32 + lane];
            const int k = klw & 0xff, l = klw >> 8;
            float v = l > k ? prob[pair_index(k, l, m)] : 0.0f;
            for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(PFSP_FULL, v, o);
            if (lane == 0) X.sscore[s2] = v;
        }
        __syncwarp();
        if (lane == 0) {
            for (int s2 = 0; s2 < S; ++s2) X.sorder[s2] = s2;
            for (int a1 = 1; a1 < S; ++a1) {
                int v = X.sorder[a1], b1 = a1 - 1;
                while (b1 >= 0 && X.sscore[X.sorder[b1]] < X.sscore[v]) {
                    X.sorder[b1 + 1] = X.sorder[b1];
                    --b1;
                }
                X.sorder[b1 + 1] = v;
            }
        }
        __syncwarp();
    }

    // Row positions of the u children of direction `dir` (compact index c held
    // by lane c and c + 32): decreasing descend-first logit, ties by job id.
    // Depends on the node alone (never on the incumbent), so every explorer
    // that rebuilds this row orders it the same way.
    __device__ void child_order(int dir, int u, int (&pos)[NW]) {
        const MlpImage &P = *net;
        const int ldx = P.D0 + 8;
        __nv_bfloat16 *Xs = (__nv_bfloat16 *)mlp_scratch();
        const int nj = (n + 3) & ~3;
        for (int t0 = 0; t0 < u; t0 += 16) {
            for (int e = lane; e < 16 * ldx; e += 32) Xs[e] = __float2bfloat16_rn(0.0f);
            __syncwarp();
            const int c = t0 + lane;
            if (lane < 16 && c < u) {
                const int j = W.ul[c];
                __nv_bfloat16 *xr = Xs + lane * ldx;
                if (dir == 0) {
                    int f = 0;
                    for (int k = 0; k < m; ++k) {
                        const int pk = T.pm[k * nj + j];
                        const int4 F = W.FRB[k];
                        f = max(f, F.x) + pk;
                        xr[k] = __float2bfloat16_rn(f * a.inv_scale);
                        xr[m + k] = __float2bfloat16_rn(F.z * a.inv_scale);
                        xr[2 * m + k] = __float2bfloat16_rn((F.y - pk) * a.inv_scale);
                    }
                } else {
                    int b = 0;
                    for (int k = m - 1; k >= 0; --k) {
                        const int pk = T.pm[k * nj + j];
                        const int4 F = W.FRB[k];
                        b = max(b, F.z) + pk;
                        xr[k] = __float2bfloat16_rn(F.x * a.inv_scale);
                        xr[m + k] = __float2bfloat16_rn(b * a.inv_scale);
                        xr[2 * m + k] = __float2bfloat16_rn((F.y - pk) * a.inv_scale);
                    }
                }
            }
            __syncwarp();
            float c0[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            net_hidden(Xs, Xs + 16 * ldx, MlpFirstCols{P.W3t, c0});
            // column 0 of rows g and g + 8 sits in lane 4g
            if ((lane & 3) == 0) {
                const int g = lane >> 2;
                const float z0 = c0[0] + P.b3[0], z1 = c0[2] + P.b3[0];
                if (t0 + g < u) X.score[t0 + g] = (z0 == z0) ? z0 : -1e30f;  // a NaN never breaks the ranking
                if (t0 + g + 8 < u) X.score[t0 + g + 8] = (z1 == z1) ? z1 : -1e30f;
            }
            __syncwarp();
        }
        for (int h = 0; h < NW; ++h) {
            const int c = lane + 32 * h;
            if (c < u) {
                const float key = X.score[c];
                int r = 0;
                for (int c2 = 0; c2 < u; ++c2) {
                    const float k2 = X.score[c2];
                    r += (k2 > key) || (k2 == key && c2 < c);
                }
                pos[h] = r;
            }
        }
        __syncwarp();
    }

    // Decompose the node at level I (I = -1: the root): bound both children
    // sets, choose the direction by MinMin, write row I+1, handle leaves.
    __device__ void expand(bool counted) {
        // ---- decode the node into [sigma1 | unscheduled | sigma2] -------------
        unsigned long long sched = 0;
        int d1 = 0, d2 = 0;
        {
            unsigned fw[2] = {0, 0}, bw[2] = {0, 0};
            int jobv[2] = {0, 0}, dv[2] = {0, 0};
            for (int h = 0; h < NW; ++h) {
                int i = lane + 32 * h;
                bool on = i <= I && i < n;
                if (on) {
                    jobv[h] = rj[i * n + X.V[i]];
                    dv[h] = X.dir[i];
                }
                fw[h] = __ballot_sync(PFSP_FULL, on && dv[h] == PFSP_FWD_DIR);
                bw[h] = __ballot_sync(PFSP_FULL, on && dv[h] != PFSP_FWD_DIR);
                unsigned long long bit = on ? (1ull << jobv[h]) : 0ull;
                unsigned lo = __reduce_or_sync(PFSP_FULL, (unsigned)(bit & 0xffffffffull));
                unsigned hi = __reduce_or_sync(PFSP_FULL, (unsigned)(bit >> 32));
                sched |= ((unsigned long long)hi << 32) | lo;
            }
            d1 = __popc(fw[0]) + __popc(fw[1]);
            d2 = __popc(bw[0]) + __popc(bw[1]);
            if (COOP && lane == 0) {
                X.last_d1 = d1;
                X.last_d2 = d2;
            }
            for (int h = 0; h < NW; ++h) {
                int i = lane + 32 * h;
                if (i <= I && i < n) {
                    unsigned below = (1u << lane) - 1;
                    int pos;
                    if (dv[h] == PFSP_FWD_DIR) pos = (h ? __popc(fw[0]) : 0) + __popc(fw[h] & below);
                    else pos = n - 1 - ((h ? __popc(bw[0]) : 0) + __popc(bw[h] & below));
                    X.perm[pos] = jobv[h];
                }
            }
            for (int h = 0; h < NW; ++h) {
                int j = lane + 32 * h;
                if (j < n && !((sched >> j) & 1ull)) {
                    unsigned long long free_below = ~sched & ((1ull << j) - 1);
                    X.perm[d1 + __popcll(free_below)] = j;
                }
            }
            __syncwarp();
        }
        const int job0 = lane < n ? X.perm[lane] : 0;
        const int job1 = (NW == 2 && lane + 32 < n) ? X.perm[lane + 32] : 0;
        tick(counted ? kPhDecode : kPhInit);
        if (DIAG && counted && a.trace_cap > 0 && (st.decomposed % (unsigned long long)a.trace_stride) == 0) {
            unsigned long long slot = 0;
            if (lane == 0) slot = atomicAdd(a.trace_count, 1ull);
            slot = __shfl_sync(PFSP_FULL, slot, 0);
            if (slot < (unsigned long long)a.trace_cap) {
                for (int i = lane; i < n; i += 32) a.trace_perm[slot * n + i] = (uint8_t)X.perm[i];
                if (lane == 0) {
                    a.trace_d1[slot] = (uint8_t)d1;
                    a.trace_d2[slot] = (uint8_t)d2;
                }
            }
        }
        ChildBounds<NW> cb;
        const int kind = (!LB1_ONLY && a.bound == PFSP_LB2) ? (PFSP_LB1 | PFSP_LB2) : PFSP_LB1;
        decompose_lb1<NW, MT>(T, W, n, m, kind, job0, job1, d1, d2, cb);
        if constexpr (MINHT) {
            if (d1 == 0 || d2 == 0) refine_minht<NW, MT>(T, W, n, m, d1, d2, cb);
        }
        tick(counted ? kPhLB1 : kPhInit);
        if (!LB1_ONLY && (kind & PFSP_LB2) && m >= 2) {
            const int *order = nullptr;
            if constexpr (LEARNED) {
                if ((a.learned & PFSP_LEARN_PAIR_ORDER) && net && S >= 2 && cb.u > 0 && I + 1 < a.learn_depth) {
                    slot_order();
                    order = X.sorder;
                }
            }
            // early-exit threshold: the incumbent of this iteration (never
            // above the initial one, equal to it in proof mode); MinBranch
            // counts children against the initial incumbent, so it keeps that
            const int ee_cap = !(a.learned & PFSP_EARLY_EXIT) ? INT_MAX
                               : a.branching == PFSP_MINBRANCH ? a.cap
                                                               : min(a.cap, ub_seen);
            const int swept =
                EARLY ? decompose_lb2<NW, MT, 0, true>(T, W, n, m, S, cb, ee_cap,
                                                       (a.learned & PFSP_EARLY_EXIT_SLOTS) != 0, order,
                                                       (a.learned & PFSP_EARLY_EXIT_CHILDREN) != 0)
                      : decompose_lb2<NW, MT, 0, false, LEAN>(T, W, n, m, S, cb, INT_MAX, false, nullptr);
            if (counted) st.slots += swept;
        }
        tick(counted ? kPhLB2 : kPhInit);
        const int u = cb.u;

        // ---- branching rule: MinMin (Section 2.3); MinBranch, MinSum (Table 4)
        // Each rule counts the children of each set at or below a threshold:
        // MinMin the overall minimum (nothing lies below it), MinBranch the
        // initial incumbent minus one, MinSum nothing; fewer wins, then the
        // larger sum of bounds, then forward.
        const int rule = a.branching;
        const bool capped = rule == PFSP_MINMIN_CAPPED;
        int vf[NW], vb[NW];
        int mn = INT_MAX;
        for (int h = 0; h < NW; ++h) {
            int c = lane + 32 * h;
            vf[h] = (!LB1_ONLY && a.bound == PFSP_LB2) ? cb.lb2f[h] : cb.lb1f[h];
            vb[h] = (!LB1_ONLY && a.bound == PFSP_LB2) ? cb.lb2b[h] : cb.lb1b[h];
            if (c < u) {
                int xf = capped ? min(vf[h], a.cap) : vf[h];
                int xb = capped ? min(vb[h], a.cap) : vb[h];
                mn = min(mn, min(xf, xb));
            }
        }
        mn = __reduce_min_sync(PFSP_FULL, mn);
        // MinBranch: a child counts when its bound is below the solve's initial
        // incumbent (a constant: every node's decision is fixed for the run, as
        // the intervals need); MinSum: no bound (all >= 0) is at or below -1
        const int thr = rule == PFSP_MINBRANCH ? max(a.cap, 0) - 1 : rule == PFSP_MINSUM ? -1 : mn;
        int cf = 0, cbk = 0;
        long long sf = 0, sb = 0;
        for (int h = 0; h < NW; ++h) {
            int c = lane + 32 * h;
            bool on = c < u;
            int xf = capped ? min(vf[h], a.cap) : vf[h];
            int xb = capped ? min(vb[h], a.cap) : vb[h];
            cf += __popc(__ballot_sync(PFSP_FULL, on && xf <= thr));
            cbk += __popc(__ballot_sync(PFSP_FULL, on && xb <= thr));
            sf += on ? xf : 0;
            sb += on ? xb : 0;
        }
        for (int o = 16; o; o >>= 1) {
            sf += __shfl_xor_sync(PFSP_FULL, sf, o);
            sb += __shfl_xor_sync(PFSP_FULL, sb, o);
        }
        int dir;
        if (cf != cbk) dir = cf < cbk ? 0 : 1;
        else if (sf != sb) dir = sf > sb ? 0 : 1;
        else dir = 0;

        // ---- new row: children of the chosen direction, pruned against UB ------
        const int row = I + 1;
        int ubv = ub_seen;  // read at the top of this iteration (never below the current incumbent)
        int npruned = 0;
        int pos[NW];
        for (int h = 0; h < NW; ++h) pos[h] = lane + 32 * h;
        if constexpr (LEARNED) {
            if ((a.learned & PFSP_LEARN_CHILD_ORDER) && net && u >= 2 && row < a.learn_depth) child_order(dir, u, pos);
        }
        for (int h = 0; h < NW; ++h) {
            int c = lane + 32 * h;
            int lb = dir ? vb[h] : vf[h];
            bool on = c < u;
            bool leaf = on && u == 1;
            if (leaf && lb < ubv) {
                // a complete schedule better than the incumbent (its bound is
                // its makespan): record it, then lower the incumbent
                int j = W.ul[c];
                int prev = atomicMin(a.ub, lb);
                if (lb < prev && !a.inst_perm) {
                    uint8_t *bp = a.best_perm + (size_t)me * 64;
                    for (int q = 0; q < n; ++q) bp[q] = (uint8_t)(q == d1 ? j : X.perm[q]);
                    if constexpr (COOP) {
                        // the host heuristic threads promote with the incumbent's order
                        for (int q = 0; q < n; ++q) a.coop->dev_perm[q] = bp[q];
                        __threadfence_system();
                        a.coop->dev_cmax = lb;
                    }
                    __threadfence();
                    atomicMin(a.best_key, ((unsigned long long)(unsigned)lb << 32) | (unsigned)me);
                } else if (lb < prev) {
                    // batched solves: explorers move between instances, so the
                    // record is per instance, written under a short bounded lock
                    bool got = false;
                    for (int it = 0; it < kLockLimit && !got; ++it) {
                        got = atomicCAS(a.perm_lock, 0, 1) == 0;
                        if (!got) __nanosleep(64);
                    }
                    if (got) {
                        __threadfence();
                        if (lb < *(volatile int *)a.perm_cmax) {
                            for (int q = 0; q < n; ++q) a.inst_perm[q] = (uint8_t)(q == d1 ? j : X.perm[q]);
                            *(volatile int *)a.perm_cmax = lb;
                        }
                        __threadfence();
                        atomicExch(a.perm_lock, 0);
                        atomicMin(a.best_key, ((unsigned long long)(unsigned)lb << 32) | (unsigned)me);
                    } else {
                        atomicExch(a.err, kErrRecordLock);
                        atomicCAS(a.stop, 0, 3);
                    }
                }
            }
            bool keep = on && !leaf && lb < ubv;
            npruned += __popc(__ballot_sync(PFSP_FULL, on && !keep && !(leaf && lb < ubv)));
            if (on) {
                rj[row * n + pos[h]] = (uint8_t)W.ul[c];
                rl[row * n + pos[h]] = keep ? lb : kPrunedLB;
            }
        }
        if (lane == 0) {
            X.dir[row] = dir;
            X.V[row] = 0;
        }
        I = row;
        __syncwarp();
        if (counted) {
            st.decomposed += 1;
            st.bounded += 2 * u;
            if (u == 1) st.leaves += 2;
            st.pruned += npruned;
            pending_nodes += 1;
        }
        tick(counted ? kPhBranch : kPhInit);
    }

    // Rebuild the rows along the path to the start digits D and position the
    // explorer on the first live node at or after start.  Returns false when
    // no such node exists.  The node that starts the interval is the first
    // one on the path whose remaining digits are all zero (X.lvl < 0: a
    // stolen or initial interval), or the node at level X.lvl (a resumed
    // checkpoint, whose ancestors on the path were decomposed before it even
    // when they share its leftmost leaf).  Ancestors are not counted.
    // One step of rebuilding the path to the start digits D after a new
    // interval arrived (init_phase 0: the root is next; 1: the row of level I
    // was just built).  Returns 1 when the next node on the path must be
    // decomposed (*counted says whether it counts), 0 when the explorer stands
    // on the first node of its interval (have_node), -1 when no node of the
    // interval is left on this path and selection took over (have_node as
    // select() returned).  The decompositions happen at the loop's single
    // expand call site, so that the kernel carries one copy of it.
    __device__ int init_step(int &init_phase, bool &counted, bool &have_node) {
        if (init_phase == 0 && hand_level >= 0) {
            // rows 0..hand_level were handed over with the interval: carry on
            // as if row hand_level had just been built
            I = hand_level;
            hand_level = -1;
            init_phase = 1;
        }
        if (init_phase == 0) {
            I = -1;
            bool zero = true;
            for (int h = 0; h < NW; ++h) {
                int i = lane + 32 * h;
                zero &= __all_sync(PFSP_FULL, i >= n || X.D[i] == 0);
            }
            init_phase = 1;
            counted = zero && X.lvl < 0;  // the root; counted only by the explorer starting at 0
            return 1;
        }
        // I is the level whose row has just been built; follow the digit D[I]
        const int d = X.D[I];
        if (lane == 0) X.V[I] = d;
        __syncwarp();
        if (!(rl[I * n + d] < ub_seen)) {
            if (lane == 0) X.V[I] = d + 1;
            __syncwarp();
            have_node = select();
            return -1;
        }
        bool rest_zero = true;
        for (int h = 0; h < NW; ++h) {
            int i = lane + 32 * h;
            rest_zero &= __all_sync(PFSP_FULL, i >= n || i <= I || X.D[i] == 0);
        }
        const int lvl = X.lvl;
        if ((lvl < 0 ? rest_zero : I >= lvl) || I >= n - 2) {  // this node starts the interval
            have_node = true;
            return 0;
        }
        counted = false;
        return 1;
    }

    // Answer a steal request if one is waiting (victim side).  A request
    // names the thief, the thief's sequence number and the instance it is for;
    // only a request for this explorer's current instance can be granted, and
    // the answer carries the sequence number so that a thief never takes an
    // answer meant for an earlier request of its own.
    __device__ void service(bool active) {
        unsigned long long req = 0;
        if (lane == 0) req = *(volatile unsigned long long *)(a.mailbox + me);
        service_req(__shfl_sync(PFSP_FULL, req, 0), active);
    }

    // The stop flag, this explorer's mailbox and the incumbent, read together
    // (one L2 round trip) one iteration ahead: prefetch_poll issues the loads
    // (lane 0) and take_poll consumes them at the top of the next iteration,
    // so that the round trip overlaps the decomposition in between.
    // take_poll returns the stop flag, *req receives the request and ub_seen
    // the incumbent that this iteration's selection and pruning use.  The
    // values are at most one iteration old: a request or a stop is seen one
    // iteration later, and the incumbent is never below the current one (it
    // only decreases), so it prunes no more than the current one would.
    int pf_stop = 0, pf_ub = INT_MAX;
    unsigned long long pf_req = kNoRequest;
    __device__ __forceinline__ void prefetch_poll() {
        if (lane == 0) {
            pf_stop = ld_volatile(a.stop);
            pf_req = *(volatile unsigned long long *)(a.mailbox + me);
            pf_ub = ld_volatile(a.ub);
        }
    }
    __device__ __forceinline__ int take_poll(unsigned long long *req) {
        *req = __shfl_sync(PFSP_FULL, pf_req, 0);
        ub_seen = __shfl_sync(PFSP_FULL, pf_ub, 0);
        return __shfl_sync(PFSP_FULL, pf_stop, 0);
    }

    __device__ void service_req(unsigned long long req, bool active) {
        if (req == kNoRequest) return;
        const int t = (int)(req & 0xfffffull);
        const unsigned long long rseq = (req >> 20) & 0xfffffull;
        const bool same = (int)(req >> 40) == (a.my_inst & 0xffffff);
        int granted = 0;
        int lc = -1;  // last level of the path the thief shares with this explorer
        if (lane == 0 && active && same && t < a.K) {
            // remaining territory [pos, end): pos = V[0..I], zeros below
            int s[64], q[64];
            int carry = 0;
            for (int i = n - 1; i >= 0; --i) {
                int p = i <= I ? X.V[i] : 0;
                int v = p + X.E[i] + carry;
                int r = n - i;
                carry = v >= r;
                s[i] = v - (carry ? r : 0);
            }
            int top = X.etop + carry;
            int rem = top & 1;
            for (int i = 0; i < n; ++i) {
                int cur = rem * (n - i) + s[i];
                q[i] = cur >> 1;
                rem = cur & 1;
            }
            // mid > pos ?
            int cmp = 0;
            for (int i = 0; i < n && cmp == 0; ++i) {
                int p = i <= I ? X.V[i] : 0;
                cmp = q[i] > p ? 1 : (q[i] < p ? -1 : 0);
            }
            // the minimum steal size: compared exactly when the fold reached
            // the last level, else (a length of 2^24 leaves or more) on the
            // log2 scale
            int lv;
            const int acc = fold_length(0, lv);
            const bool big = lv == n - 1 ? (float)acc >= a.min_steal
                                         : __log2f((float)acc) + X.lw[lv] >= log2f(fmaxf(a.min_steal, 1.0f));
            if (cmp > 0 && big) {
                uint8_t *ds = a.in_start + (size_t)t * 64;
                uint8_t *de = a.in_end + (size_t)t * 65;
                for (int i = 0; i < n; ++i) {
                    ds[i] = (uint8_t)q[i];
                    de[1 + i] = (uint8_t)X.E[i];
                }
                de[0] = (uint8_t)X.etop;
                if (a.in_level) a.in_level[t] = 0xff;
                for (int i = 0; i < n; ++i) X.E[i] = q[i];
                X.etop = 0;
                atomicAdd(a.active, 1);
                granted = 1;
                // the thief's path follows q: its nodes above the first
                // level L where q leaves this explorer's position are this
                // explorer's, and so are rows 0..min(L, I)
                int L = 0;
                while (L < n && q[L] == (L <= I ? X.V[L] : 0)) ++L;
                lc = min(L, I);
            }
        }
        if (handoff_on()) {
            granted = __shfl_sync(PFSP_FULL, granted, 0);
            lc = __shfl_sync(PFSP_FULL, lc, 0);
            if (granted && lc >= 0) {
                int32_t *tl = a.hand_lb + (size_t)t * a.row_stride;
                uint8_t *tj = a.hand_job + (size_t)t * a.row_stride;
                for (int i = lane; i < (lc + 1) * n; i += 32) {
                    tl[i] = rl[i];
                    tj[i] = rj[i];
                }
                for (int i = lane; i <= lc; i += 32) a.hand_dir[(size_t)t * 64 + i] = (uint8_t)X.dir[i];
                if (lane == 0) a.hand_lc[t] = lc;
                __threadfence();  // before lane 0's answer below
            } else if (granted && lane == 0) {
                a.hand_lc[t] = -1;
            }
            __syncwarp();
        }
        if (lane == 0) {
            __threadfence();
            if (t < a.K) atomicExch(a.response + t, (rseq << 2) | (granted ? 1ull : 2ull));
            atomicExch(a.mailbox + me, kNoRequest);
        }
        __syncwarp();
    }

    __device__ void publish_length(bool active) {
        float l = active ? log2_length() : -1.0f;
        if (lane == 0) a.len_est[me] = l;
    }

    __device__ bool stopped() const {
        int s = 0;
        if (lane == 0) s = ld_volatile(a.stop);
        return __shfl_sync(PFSP_FULL, s, 0) != 0;
    }

    __device__ void flush_limits() {
        if (lane == 0 && pending_nodes) {
            unsigned long long tot = atomicAdd(a.counters + 6, pending_nodes) + pending_nodes;
            pending_nodes = 0;
            if (a.node_limit > 0 && tot >= (unsigned long long)a.node_limit) atomicCAS(a.stop, 0, 1);
        }
        if (lane == 0 && deadline && global_ns() > deadline) atomicCAS(a.stop, 0, 2);
        if constexpr (COOP) coop_exchange();
        __syncwarp();
    }

    // Host heuristic threads (Section 4.2): take their incumbent if it is
    // better, and answer a snapshot request with the node last decomposed.
    __device__ void coop_exchange() {
        int req = 0;
        if (lane == 0) {
            const int hub = a.coop->host_ub;
            req = a.coop->snap_req;
            if (hub < ub_seen) atomicMin(a.ub, hub);
        }
        req = __shfl_sync(PFSP_FULL, req, 0);
        if (req == snap_seen) return;
        snap_seen = req;
        CoopSlot &s = a.coop_slots[me];
        for (int i = lane; i < n; i += 32) s.perm[i] = (uint8_t)X.perm[i];
        if (lane == 0) {
            s.d1 = (uint8_t)X.last_d1;
            s.d2 = (uint8_t)X.last_d2;
        }
        __threadfence_system();
        __syncwarp();
        if (lane == 0) s.seq = req;
    }

    // Thief side: pick a victim, post a request, wait (bounded) for the answer.
    // Returns 1 = got an interval (in D / E), 0 = nothing now, -1 = give up.
    __device__ int try_steal() {
        const float min_log = log2f(fmaxf(a.min_steal, 1.0f));
        // scan a random window first, then everything
        int best = -1;
        float bestv = min_log;
        const int K = a.K;
        for (int pass = 0; pass < 2 && best < 0; ++pass) {
            int start = 0, count = K;
            if (pass == 0) {
                rng = rng * 1664525u + 1013904223u;
                start = (int)(rng % (unsigned)K);
                count = min(K, 64);
            }
            for (int o = lane; o < count; o += 32) {
                int e = (start + o) % K;
                float l = e == me ? -1.0f : *(volatile float *)(a.len_est + e);
                if (a.inst_of && ld_volatile(a.inst_of + e) != a.my_inst) l = -1.0f;
                if (l > bestv) {
                    bestv = l;
                    best = e;
                }
            }
            for (int o = 16; o; o >>= 1) {
                float ov = __shfl_xor_sync(PFSP_FULL, bestv, o);
                int oe = __shfl_xor_sync(PFSP_FULL, best, o);
                if (ov > bestv || (ov == bestv && oe > best)) {
                    bestv = ov;
                    best = oe;
                }
            }
        }
        if (best < 0) return 0;
        int posted = 0;
        unsigned long long myseq = 0;
        if (lane == 0) {
            X.seq = (X.seq + 1) & 0xfffffu;
            myseq = X.seq;
            const unsigned long long req = ((unsigned long long)(a.my_inst & 0xffffff) << 40) | (myseq << 20) |
                                           (unsigned long long)me;
            posted = atomicCAS(a.mailbox + best, kNoRequest, req) == kNoRequest;
            if (posted && a.seq_posted) a.seq_posted[me] = (unsigned)myseq;
        }
        posted = __shfl_sync(PFSP_FULL, posted, 0);
        myseq = __shfl_sync(PFSP_FULL, myseq, 0);
        if (!posted) return 0;
        int r = 0;
        const int wait_limit = a.wait_limit > 0 ? a.wait_limit : kWaitLimit;
        for (int it = 0; it < wait_limit; ++it) {
            if (lane == 0) {
                unsigned long long v = *(volatile unsigned long long *)(a.response + me);
                r = (v >> 2) == myseq ? (int)(v & 3ull) : 0;
            }
            r = __shfl_sync(PFSP_FULL, r, 0);
            if (r) break;
            service(false);  // deny requests addressed to this idle explorer
            if (stopped() || active_count() == 0) return -1;
            __nanosleep(200);
        }
        if (r == 0) {
            if (lane == 0) {
                atomicExch(a.err, kErrStealWait);
                atomicCAS(a.stop, 0, 3);
            }
            return -1;
        }
        if (r == 2) return 0;
        __threadfence();
        const uint8_t *ds = a.in_start + (size_t)me * 64;
        const uint8_t *de = a.in_end + (size_t)me * 65;
        for (int i = lane; i < n; i += 32) {
            X.D[i] = ((volatile const uint8_t *)ds)[i];
            X.E[i] = ((volatile const uint8_t *)de)[1 + i];
        }
        if (lane == 0) {
            X.etop = ((volatile const uint8_t *)de)[0];
            X.lvl = -1;
            if (a.seq_taken) a.seq_taken[me] = (unsigned)myseq;
        }
        __syncwarp();
        // never index with digits that are not a valid factoradic number
        bool bad = false;
        for (int h = 0; h < NW; ++h) {
            int i = lane + 32 * h;
            bad |= __any_sync(PFSP_FULL, i < n && (X.D[i] >= n - i || X.E[i] >= n - i || X.D[i] < 0 || X.E[i] < 0));
        }
        if (bad) {
            if (lane == 0) {
                atomicExch(a.err, kErrBadInterval);
                atomicCAS(a.stop, 0, 3);
            }
            return -1;
        }
        hand_level = -1;
        if (handoff_on()) {
            // rows 0..lc of the path to D, as the victim wrote them (read
            // from L2, past this SM's L1, and stored into this explorer's
            // rows by itself): the path is rebuilt below them only
            const int lc = __ldcg(a.hand_lc + me);
            if (lc >= 0 && lc <= n - 2) {
                const int32_t *hl = a.hand_lb + (size_t)me * a.row_stride;
                const volatile uint8_t *hj = a.hand_job + (size_t)me * a.row_stride;
                for (int i = lane; i < (lc + 1) * n; i += 32) {
                    rl[i] = __ldcg(hl + i);
                    rj[i] = hj[i];
                }
                const volatile uint8_t *hd = a.hand_dir + (size_t)me * 64;
                for (int i = lane; i <= lc; i += 32) {
                    X.dir[i] = hd[i];
                    X.V[i] = X.D[i];
                }
                hand_level = lc;
            }
            __syncwarp();
        }
        st.steals += 1;
        return 1;
    }
};

// One explorer's life on one instance: initialise from the interval held in
// X.D / X.E / X.etop (empty if start >= end), then select, decompose, answer
// steal requests and steal until no explorer of the instance holds work or
// the solve is stopped.  Counters are added to a.counters on return.
template <int NW, int MT, int KIND = kKindPlain>
__device__ void run_explorer(const SolveArgs &a, const SmemTables &T, const WarpScratch &W, ExplorerSmem &X,
                             int me, const MlpImage *net) {
    const int lane = threadIdx.x & 31;
    Explorer<NW, MT, KIND> ex(a, T, W, X, me, net);
    bool nonempty = false;
    {
        // start < end ?
        if (X.etop) nonempty = true;
        else {
            int f = -1;
            for (int h = 0; h < NW && f < 0; ++h) {
                int i = lane + 32 * h;
                unsigned diff = __ballot_sync(PFSP_FULL, i < a.n && X.D[i] != X.E[i]);
                if (diff) {
                    int b = __ffs(diff) - 1;
                    int di = __shfl_sync(PFSP_FULL, i < a.n ? X.D[i] : 0, b);
                    int ei = __shfl_sync(PFSP_FULL, i < a.n ? X.E[i] : 0, b);
                    nonempty = di < ei;
                    f = b;
                }
            }
        }
    }
    int state = nonempty ? 1 : 0;  // 0 empty, 1 rebuilding the path to a new interval, 2 active
    int init_phase = 0;
    bool have_node = false;
    unsigned iter = 0;
    // watchdog of idle explorers: the global decomposition count must keep
    // moving while some explorer holds work
    unsigned long long seen = ~0ull, seen_at = global_ns();
    ex.prefetch_poll();
    while (true) {
        ++iter;
        if ((iter & (a.check_every - 1)) == 0) {
            ex.flush_limits();
            ex.publish_length(state == 2);
        }
        unsigned long long req;
        // a stop is taken between nodes of the interval, never in the middle
        // of a path rebuild (at most n decompositions): a checkpoint then
        // records the interval's start, and the root, counted when it starts
        // an interval, is never decomposed twice
        if (ex.take_poll(&req) && state != 1) break;
        ex.service_req(req, state == 2);
        ex.tick(kPhService);
        bool counted = false, go = false;
        if (state == 1) {
            const int r = ex.init_step(init_phase, counted, have_node);
            if (r == 1) go = true;
            else {
                state = 2;
                ex.publish_length(true);
            }
            ex.tick(kPhInit);
        }
        if (state == 2 && !go) {
            ex.st.iters += 1;
            if (!have_node) have_node = ex.select();
            go = have_node && ex.pos_before_end();
            counted = true;
            ex.tick(kPhSelect);
            if (!go) {
                // interval exhausted
                state = 0;
                have_node = false;
                ex.publish_length(false);
                if (lane == 0) atomicSub(a.active, 1);
                __syncwarp();
            }
        }
        if (go) {
            // the next iteration's poll is issued now: its L2 round trip
            // overlaps the decomposition
            ex.prefetch_poll();
            ex.expand(counted);
            have_node = false;
            continue;
        }
        ex.prefetch_poll();
        // idle
        if (ex.active_count() == 0) break;
        {
            int trip = 0;
            if (lane == 0) {
                unsigned long long now_cnt = *(volatile unsigned long long *)(a.counters + 6);
                unsigned long long now = global_ns();
                if (now_cnt != seen) {
                    seen = now_cnt;
                    seen_at = now;
                } else if (now - seen_at > kWatchdogNs) {
                    atomicExch(a.err, kErrNoProgress);
                    atomicCAS(a.stop, 0, 3);
                    trip = 1;
                }
            }
            if (__shfl_sync(PFSP_FULL, trip, 0)) break;
        }
        int r = ex.try_steal();
        ex.tick(kPhIdle);
        if (r < 0) break;
        if (r == 1) {
            state = 1;
            init_phase = 0;
            ex.prefetch_poll();
            continue;
        }
        __nanosleep(500);
        ex.prefetch_poll();
        ex.tick(kPhIdle);
    }
    ex.flush_limits();
    // stopped at a limit with work left: record the rest of the interval so
    // that a later launch resumes exactly where this one stopped
    if (a.ckpt && state != 0 && (ld_volatile(a.stop) == 1 || ld_volatile(a.stop) == 2)) {
        int lvl = -1;
        bool rec = false;
        if (state == 1) {
            rec = true;
            lvl = X.lvl;
        } else {
            if (!have_node) have_node = ex.select();
            if (have_node && ex.pos_before_end()) {
                rec = true;
                lvl = ex.I;
                for (int i = lane; i < a.n; i += 32) X.D[i] = i <= ex.I ? X.V[i] : 0;
                __syncwarp();
            }
        }
        uint8_t *rp = a.ckpt + (size_t)me * kCkptRecord;
        if (rec) {
            for (int i = lane; i < 64; i += 32) {
                rp[4 + i] = (uint8_t)(i < a.n ? X.D[i] : 0);
                rp[68 + i] = (uint8_t)(i < a.n ? X.E[i] : 0);
            }
            if (lane == 0) {
                rp[1] = (uint8_t)(lvl < 0 ? 0xff : lvl);
                rp[2] = (uint8_t)X.etop;
                rp[0] = 1;
            }
        }
        __syncwarp();
    }
    ex.publish_length(false);
    ex.tick(kPhService);
    if (lane == 0 && a.phase) {
        for (int p = 0; p < kPhases; ++p) atomicAdd(a.phase + p, X.ph[p]);
    }
    if (lane == 0) {
        atomicAdd(a.counters + 0, ex.st.decomposed);
        atomicAdd(a.counters + 1, ex.st.bounded);
        atomicAdd(a.counters + 2, ex.st.leaves);
        atomicAdd(a.counters + 3, ex.st.pruned);
        atomicAdd(a.counters + 4, ex.st.steals);
        atomicAdd(a.counters + 5, ex.st.iters);
        atomicAdd(a.counters + 7, ex.st.slots);
    }
}

}  // namespace pfsp
