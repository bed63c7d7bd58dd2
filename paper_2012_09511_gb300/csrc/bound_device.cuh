// bound_device.cuh -- warp-level decomposition of one parent node: front,
// back and remaining work (Section 2.4, steps 1-3), LB1 of all 2u children by
// the incremental rule of Section 2.4, and LB2 of all children over all
// machine pairs.
//
// LB2 per pair (k, l) runs the unscheduled jobs of the child, in the pair's
// Johnson order, through  t0 += p_jk;  t1 = max(t1, t0 + g_j) + p_jl  from
// (t0, t1) = (F_k, F_l) and takes max(t0 + B_k, t1 + B_l).  Written in the gap
// u = t1 - t0, one job is the max-plus map  u -> max(u + a_j, b_j)  with
// a_j = p_jl - p_jk and b_j = g_j + p_jl.  Maps of this form compose into a
// map of the same form, (A1, B1) then (A2, B2) = (A1 + A2, max(B1 + A2, B2)),
// so for the child that leaves out job j the composed map is the prefix of
// the order before j followed by the suffix after it: its constant part is
//     C_j = max(PB_j + SA_j, SB_j).
// Expanding the pair value with it gives
//     v_kl = max(F_k + R_k + B_k,  F_l + R_l + B_l,  F_k + R_k + C_j + B_l)
// with F, R, B the child's front, remaining work and back.  The first two
// terms, maximised over pairs, are exactly LB1 of the child (m >= 2), so
//     LB2(child) = max(LB1(child), max_{k<l} (F_k + R_k + C_j(k,l) + B_l)).
// All arithmetic is exact int32: the result is bit-identical to running the
// recurrence job by job, at O(P u) work per parent instead of O(P u^2).
#pragma once

#include <climits>
#include <cstdint>
#include <type_traits>

#include "pfsp_internal.h"

namespace pfsp {

#define PFSP_FULL 0xffffffffu

template <int NW>
using umask_t = typename std::conditional<NW == 1, uint32_t, unsigned long long>::type;

template <int NW>
__device__ __forceinline__ bool has_job(umask_t<NW> U, int j) {
    return (U >> j) & 1;
}

template <int NW>
__device__ __forceinline__ umask_t<NW> low_bits(int j) {
    return (umask_t<NW>(1) << j) - 1;
}

template <int NW>
__device__ __forceinline__ int popcnt(umask_t<NW> x) {
    if constexpr (NW == 1) return __popc(x);
    else return __popcll(x);
}

// Shared-memory views of one CTA's instance tables.
struct SmemTables {
    const int *pm;        // [m][nj]
    const int *tot;       // [32]
    const int *kl;        // [S*32]
    const int *pq;        // int2 [n][m] per job and machine: {P_k, Q_k}, its times summed over 0..k and k..m-1
    const uint8_t *rank;  // [n][S][32] bit of job j in the lane's position masks (see pos_of_bit)
    const int2 *ptab;     // [S][n][32]
    int S;                // slots of the table layout (stride of rank); the sweep may use fewer
};

__host__ __device__ inline int round4(int w) { return (w + 3) & ~3; }

// Per-warp scratch.  Every region starts on a multiple of 4 words (16 bytes);
// child-indexed tables have round4(n) rows so that the evaluation loop, which
// walks children in groups of four, stays inside them.
struct WarpScratch {
    int4 *FRB;        // [32] per machine k: {front F_k, remaining work R_k, back B_k, F_k + R_k} of the parent
    int *ul;          // [64] compact list: ul[c] = c-th unscheduled job
    int *cidx;        // [64] cidx[j] = compact index of job j
    int2 *G;          // [nr][mp] {forward child: F'_k + R_k - p_jk, backward child: F_k + R_k - p_jk}
    int *Bb;          // [nr][mp] backward child back B'_k minus the parent's B_k
    int *Epb;         // [nr][32] prefix pass records: the prefix constant PB of each step (per lane)
    uint8_t *Et;      // [nr][32] the bit of the step's position (per lane); both NULL for register walks
    int *Cb;          // [nr][32] C of child c plus the parent's B_l (per lane)
    int2 *X;          // [u][33] transpose buffer (shared accumulators only), aliasing the records and Cb
    int2 *Acc;        // [nr][32] accumulators (only when not kept in registers)
};

// Words before the child tables: FRB, ul, cidx.
constexpr int kWarpHead = 256;

// Walks of up to kRegWalk jobs keep their records in registers (scan_slot_reg).
constexpr int kRegWalk = 20;

// reg_walk: the layout of kernels whose LB2 walks keep their records in
// registers (n <= kRegWalk, register accumulators): no record region and no
// transpose buffer.
__host__ __device__ inline int warp_words(int n, int m, bool smem_acc, bool lb2, bool reg_walk = false) {
    if (!lb2) return kWarpHead;
    int nr = round4(n);
    int g = round4(nr * (m | 1));
    // G takes 2g words, Bb g; then the records (Epb 32 nr + Et 8 nr) and Cb
    // (32 nr): 72 nr, which the transpose buffer of shared accumulators (66 nr)
    // aliases; Cb alone (32 nr) with register walks
    const int walk = reg_walk ? 32 * nr : 72 * nr;
    return kWarpHead + 3 * g + walk + (smem_acc ? 64 * nr : 0);
}

__device__ inline WarpScratch carve_warp(int *base, int n, int m, bool reg_walk = false) {
    int nr = round4(n);
    int g = round4(nr * (m | 1));
    WarpScratch w;
    w.FRB = reinterpret_cast<int4 *>(base);
    w.ul = base + 128;
    w.cidx = base + 192;
    w.G = reinterpret_cast<int2 *>(base + kWarpHead);
    w.Bb = base + kWarpHead + 2 * g;
    if (reg_walk) {
        // register walks come with register accumulators: neither the
        // records, the transpose buffer nor shared accumulators are used
        w.Epb = nullptr;
        w.Et = nullptr;
        w.Cb = w.Bb + g;
        w.X = nullptr;
        w.Acc = nullptr;
    } else {
        w.Epb = w.Bb + g;
        w.Et = reinterpret_cast<uint8_t *>(w.Epb + 32 * nr);
        w.Cb = w.Epb + 40 * nr;
        // shared accumulators (n > 32) only: the transpose buffer from the
        // records on, the accumulators after the 72 nr words of the walk
        w.X = reinterpret_cast<int2 *>(w.Epb);
        w.Acc = n > 32 ? reinterpret_cast<int2 *>(w.Epb + 72 * nr) : nullptr;
    }
    return w;
}

// Result of one decomposition, distributed over lanes: lane c (and c + 32)
// holds the bounds of the children of compact index c (the c-th unscheduled
// job in ascending id order).
template <int NW>
struct ChildBounds {
    umask_t<NW> U;  // unscheduled jobs
    int u;          // number of unscheduled jobs
    int lb1f[NW], lb1b[NW];
    int lb2f[NW], lb2b[NW];
};

template <int NW>
__device__ __forceinline__ int lowest_bit(umask_t<NW> x) {
    if constexpr (NW == 1) return __ffs(x) - 1;
    else return __ffsll((long long)x) - 1;
}

// Bit walks.  32-bit masks are walked from the highest set bit (bfind, one
// instruction, -1 for an empty mask) and 64-bit masks from the lowest (a
// 64-bit bfind and variable shift cost more than the 64-bit ffs and
// x & (x - 1)).  The position masks of a pair's Johnson order follow the walk:
// position t sits in bit 31 - t (n <= 32) or t (n > 32), so that every walk
// meets the positions in ascending order.
template <int NW>
__device__ __forceinline__ int next_bit(umask_t<NW> x) {
    if constexpr (NW == 1) {
        int r;
        asm("bfind.u32 %0, %1;" : "=r"(r) : "r"(x));
        return r;
    } else {
        return lowest_bit<NW>(x);
    }
}

// x without bit t = next_bit(x).  shl clamps shift amounts past the width,
// so t = -1 (an empty mask) leaves x = 0 unchanged.
template <int NW>
__device__ __forceinline__ umask_t<NW> drop_bit(umask_t<NW> x, int t) {
    if constexpr (NW == 1) {
        uint32_t b;
        asm("shl.b32 %0, 1, %1;" : "=r"(b) : "r"(t));
        return x & ~b;
    } else {
        return x & (x - 1);
    }
}

// Position of bit b of a position mask (its own inverse).
template <int NW>
__device__ __forceinline__ int pos_of_bit(int b) {
    return NW == 1 ? 31 - b : b;
}

// The mask of positions 0..n-1.
template <int NW>
__device__ __forceinline__ umask_t<NW> all_positions(int n) {
    if constexpr (NW == 1) return ~0u << (32 - n);  // 1 <= n <= 32
    else return n >= 64 ? ~0ull : ((1ull << n) - 1);
}

// __shfl_down_sync with the source lane clamped to max_lane: lanes whose
// source lies above it keep their own value.
__device__ __forceinline__ int shfl_down_clamped(int v, int delta, int max_lane) {
    int r;
    asm volatile("shfl.sync.down.b32 %0, %1, %2, %3, 0xffffffff;" : "=r"(r) : "r"(v), "r"(delta), "r"(max_lane));
    return r;
}

// max(a + b, c): the step of every max-plus recurrence below, one DPX
// add-max instruction on sm_90 and later.
__device__ __forceinline__ int addmax(int a, int b, int c) { return __viaddmax_s32(a, b, c); }

// Decompose the node whose permutation entries are held one per lane
// (job0 = position lane, job1 = position lane + 32) with depths d1, d2.
// kind: bit 0 = LB1 wanted, bit 1 = LB2 wanted.  MT is the machine count
// when known at compile time (0: take m_rt).  SCAN: fronts and backs by
// max-scans over the machines, one per scheduled job (needs T.pq), when there
// are at least 16 machines; otherwise, and below 16 machines, by the
// wavefront (its m - 1 fill steps cost less than log2 m shuffles per job
// there).  All 32 lanes must call.
template <int NW, int MT, bool SCAN = false>
__device__ __forceinline__ void decompose_lb1(const SmemTables &T, const WarpScratch &W, int n, int m_rt, int kind,
                                              int job0, int job1, int d1, int d2, ChildBounds<NW> &out) {
    using mask_t = umask_t<NW>;
    const int m = MT ? MT : m_rt;
    const int lane = threadIdx.x & 31;
    const int mp = m | 1;
    const int nj = (n + 3) & ~3;

    // ---- unscheduled set, its compact list and the compact index of each job --
    bool un0 = lane < n && lane >= d1 && lane < n - d2;
    bool un1 = (NW == 2) && (lane + 32 < n) && (lane + 32 >= d1) && (lane + 32 < n - d2);
    mask_t mine = (un0 ? (mask_t(1) << job0) : mask_t(0));
    if constexpr (NW == 2) mine |= (un1 ? (mask_t(1) << job1) : mask_t(0));
    mask_t U;
    if constexpr (NW == 1) {
        U = __reduce_or_sync(PFSP_FULL, mine);
    } else {
        unsigned lo = __reduce_or_sync(PFSP_FULL, (unsigned)(mine & 0xffffffffull));
        unsigned hi = __reduce_or_sync(PFSP_FULL, (unsigned)(mine >> 32));
        U = ((mask_t)hi << 32) | lo;
    }
    const int u = popcnt<NW>(U);
#pragma unroll
    for (int h = 0; h < NW; ++h) {
        int j = lane + 32 * h;
        if (j < n) {
            int c = popcnt<NW>(U & low_bits<NW>(j));
            W.cidx[j] = c;
            if (has_job<NW>(U, j)) W.ul[c] = j;
        }
    }

    // ---- steps 1 and 3: front (Eq. 1 over sigma1) and back (Eq. 1 over the
    // reversed sigma2 on reversed machines), lane = machine -------------------
    int Fk = 0, Bk = 0, Sk = 0;
    if (SCAN && (MT ? MT >= 16 : m >= 16)) {
        // Appending job j to the front, F'_k = max(F_k, F'_{k-1}) + p_jk,
        // unrolls to F'_k = P_k + max_{k' <= k} (F_k' - P_k' + p_jk') with P the
        // job's prefix sums over machines: one inclusive max-scan over lanes.
        // Prepending it to the back is the mirror image with the suffix sums
        // Q: B'_k = Q_k + max_{k' >= k} (B_k' - Q_k' + p_jk').  As
        // P_k + Q_k = T_j + p_jk (T_j the job's total, P at the last machine),
        // p_jk - P_k = Q_k - T_j and p_jk - Q_k = P_k - T_j: one 8-byte load of
        // {P_k, Q_k} per lane and job (job-major rows, so the lanes read
        // consecutive words) and T_j from the last machine's lane.  The front's
        // scan reads lower lanes only; the back's is clamped to the last
        // machine, so lanes past it (entries of machine 0) feed no machine.
        constexpr int LG = MT == 0 ? 5 : MT <= 2 ? 1 : MT <= 4 ? 2 : MT <= 8 ? 3 : MT <= 16 ? 4 : 5;
        const int2 *pqrow = reinterpret_cast<const int2 *>(T.pq) + (lane < m ? lane : 0);
        const int steps = max(d1, d2);
        for (int s = 0; s < steps; ++s) {
            const int pos = n - 1 - s;
            int jf = __shfl_sync(PFSP_FULL, job0, s);
            int jb = __shfl_sync(PFSP_FULL, job0, pos);
            if constexpr (NW == 2) {
                const int jf1 = __shfl_sync(PFSP_FULL, job1, s);
                const int jb1 = __shfl_sync(PFSP_FULL, job1, pos);
                jf = s >= 32 ? jf1 : jf;
                jb = pos >= 32 ? jb1 : jb;
            }
            if (s < d1) {
                const int2 v = pqrow[jf * m];
                const int Tj = __shfl_sync(PFSP_FULL, v.x, m - 1);
                int x = Fk + v.y - Tj;
#pragma unroll
                for (int o = 0; o < LG; ++o) x = max(x, __shfl_up_sync(PFSP_FULL, x, 1 << o));
                Fk = v.x + x;
                Sk += v.x + v.y - Tj;
            }
            if (s < d2) {
                const int2 v = pqrow[jb * m];
                const int Tj = __shfl_sync(PFSP_FULL, v.x, m - 1);
                int x = Bk + v.x - Tj;
#pragma unroll
                for (int o = 0; o < LG; ++o) x = max(x, shfl_down_clamped(x, 1 << o, m - 1));
                Bk = v.y + x;
                Sk += v.x + v.y - Tj;
            }
        }
    } else {
        const int stepsF = d1 > 0 ? d1 + m - 1 : 0;
        const int stepsB = d2 > 0 ? d2 + m - 1 : 0;
        const int steps = max(stepsF, stepsB);
        const int r = m - 1 - lane;
        // lanes past the last machine take no part (their depths are zero);
        // lane 0 receives its own F from shfl_up and the lane after the last
        // machine holds B = 0, both of which leave the recurrence unchanged
        const unsigned ud1 = lane < m ? d1 : 0, ud2 = lane < m ? d2 : 0;
        const int *pmrow = T.pm + lane * nj;
        for (int s = 0; s < steps; ++s) {
            const int i = s - lane;  // sigma1 position this machine handles now
            const int ib = s - r;    // position from the end of sigma2
            const int left = __shfl_up_sync(PFSP_FULL, Fk, 1);
            const int right = __shfl_down_sync(PFSP_FULL, Bk, 1);
            const int pos = n - 1 - ib;
            // source lanes are taken modulo 32
            int jf = __shfl_sync(PFSP_FULL, job0, i);
            int jb = __shfl_sync(PFSP_FULL, job0, pos);
            if constexpr (NW == 2) {
                int jf1 = __shfl_sync(PFSP_FULL, job1, i);
                int jb1 = __shfl_sync(PFSP_FULL, job1, pos);
                jf = i >= 32 ? jf1 : jf;
                jb = pos >= 32 ? jb1 : jb;
            }
            if ((unsigned)i < ud1) {
                const int pk = pmrow[jf];
                Fk = max(Fk, left) + pk;
                Sk += pk;
            }
            if ((unsigned)ib < ud2) {
                const int pk = pmrow[jb];
                Bk = max(Bk, right) + pk;
                Sk += pk;
            }
        }
    }
    // ---- step 2: remaining work = totals minus scheduled work -----------------
    if (lane < m) {
        const int Rk = T.tot[lane] - Sk;
        W.FRB[lane] = make_int4(Fk, Rk, Bk, Fk + Rk);
    }
    __syncwarp();

    // ---- LB1 of all children, incrementally from the parent (Section 2.4) -----
    const bool want2 = (kind & PFSP_LB2) && m >= 2;
#pragma unroll
    for (int h = 0; h < NW; ++h) {
        out.lb1f[h] = kNegInf;
        out.lb1b[h] = kNegInf;
        int c = lane + 32 * h;
        if (c < u) {
            // forward child: machines upwards from the parent's front;
            // backward child: machines downwards from its back (two
            // independent chains in one loop)
            const int j = W.ul[c];
            int f = 0, lf = kNegInf, b = 0, lb = kNegInf;
#pragma unroll
            for (int i = 0; i < m; ++i) {
                const int kf = i, kb = m - 1 - i;
                const int pf = T.pm[kf * nj + j], pb = T.pm[kb * nj + j];
                const int4 Pf = W.FRB[kf], Pb = W.FRB[kb];  // broadcast loads
                f = max(f, Pf.x) + pf;
                b = max(b, Pb.z) + pb;
                const int gf = f + Pf.y - pf;
                const int gb = Pb.w - pb;
                lf = addmax(gf, Pf.z, lf);
                lb = addmax(gb, b, lb);
                if (want2) {
                    W.G[c * mp + kf].x = gf;
                    W.G[c * mp + kb].y = gb;
                    W.Bb[c * mp + kb] = b - Pb.z;
                }
            }
            out.lb1f[h] = lf;
            out.lb1b[h] = lb;
        }
        out.lb2f[h] = out.lb1f[h];
        out.lb2b[h] = out.lb1b[h];
    }
    out.U = U;
    out.u = u;
}

// One slot of the LB2 sweep for this lane's pair: walk the unscheduled jobs
// (bit mask Upos of their positions in the pair's Johnson order, walked in
// ascending position order by next_bit) recording the prefix constant PB
// before each job, then backwards composing the suffix maps, leaving C of
// every child (compact index c) plus Bl in W.Cb[c][lane].  The suffix walk
// starts from the map (Bl, -inf) instead of the identity (0, -inf): every
// constant it builds, and so C, comes out shifted by Bl (the parent's B_l),
// which saves the evaluation an addition.  Both walks take four jobs per
// round: the next positions come off the mask by dropping the walked bit (a
// short chain), so the table loads of the four jobs issue together
// instead of each waiting for the previous job's.
template <int NW>
__device__ __forceinline__ void scan_slot(const WarpScratch &W, const int2 *pt, umask_t<NW> Upos, int u, int lane,
                                          int Bl) {
    int *Epb = W.Epb + lane;
    uint8_t *Et = W.Et + lane;
    int PB = kNegInf;
    for (int i = 0; i < u; i += 4) {
        int t[4];
        int2 e[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            t[q] = next_bit<NW>(Upos);  // -1 once the mask is empty
            Upos = drop_bit<NW>(Upos, t[q]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) e[q] = (i + q < u) ? pt[pos_of_bit<NW>(t[q]) * 32] : make_int2(0, kNegInf);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            // rows u..round4(u)-1 get a record that the backward walk never reads
            Epb[(i + q) * 32] = PB;
            Et[(i + q) * 32] = (uint8_t)t[q];
            PB = addmax(PB, e[q].x >> 8, e[q].y);  // identity for a padding step
        }
    }
    int SA = Bl, SB = kNegInf;
    for (int i = u - 1; i >= 0; i -= 4) {
        int pb[4], c[4];
        int2 e[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            pb[r] = (i - r >= 0) ? Epb[(i - r) * 32] : 0;
            e[r] = (i - r >= 0) ? pt[pos_of_bit<NW>(Et[(i - r) * 32]) * 32] : make_int2(0, kNegInf);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) c[r] = W.cidx[e[r].x & 0xff];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            if (i - r >= 0) {
                W.Cb[c[r] * 32 + lane] = addmax(pb[r], SA, SB);
                SB = addmax(e[r].y, SA, SB);
                SA += e[r].x >> 8;
            }
        }
    }
}

// Register walks keep the forward records in registers: the prefix
// constant of step i in PBr[i] and the position of its job in byte i % 4 of
// tb[i / 4].  All indices below are compile-time constants.

// Backward steps 4G+3 .. 4G (those below u) of scan_slot_reg (n <= 32:
// masks of 32 bits).
template <int G>
__device__ __forceinline__ void scan_back_group(const WarpScratch &W, const int2 *pt, const int (&PBr)[kRegWalk],
                                                const unsigned (&tb)[kRegWalk / 4], int u, int lane, int &SA,
                                                int &SB) {
    int2 e[4];
    int c[4];
#pragma unroll
    for (int r = 3; r >= 0; --r) {
        const int t = (tb[G] >> (8 * r)) & 0xff;
        e[r] = (4 * G + r < u) ? pt[pos_of_bit<1>(t) * 32] : make_int2(0, kNegInf);
    }
#pragma unroll
    for (int r = 3; r >= 0; --r) c[r] = W.cidx[e[r].x & 0xff];
#pragma unroll
    for (int r = 3; r >= 0; --r) {
        if (4 * G + r < u) {
            W.Cb[c[r] * 32 + lane] = addmax(PBr[4 * G + r], SA, SB);
            SB = addmax(e[r].y, SA, SB);
            SA += e[r].x >> 8;
        }
    }
}

// scan_slot for u <= kRegWalk without the per-step records in shared memory:
// the forward walk keeps them in registers, the backward walk re-reads the
// job's table entry (for a, b and the job) and the compact index.  It is
// entered at the group holding step u - 1.
template <int NW>
__device__ __forceinline__ void scan_slot_reg(const WarpScratch &W, const int2 *pt, umask_t<NW> Upos, int u,
                                              int lane, int Bl) {
    static_assert(NW == 1, "register walks need n <= 32");
    int PBr[kRegWalk];
    unsigned tb[kRegWalk / 4];
    int PB = kNegInf;
#pragma unroll
    for (int g = 0; g < kRegWalk / 4; ++g) {
        if (4 * g >= u) break;
        int t[4];
        int2 e[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            t[q] = next_bit<NW>(Upos);  // -1 once the mask is empty
            Upos = drop_bit<NW>(Upos, t[q]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) e[q] = (4 * g + q < u) ? pt[pos_of_bit<NW>(t[q]) * 32] : make_int2(0, kNegInf);
        tb[g] = (unsigned)(t[0] & 0xff) | ((unsigned)(t[1] & 0xff) << 8) | ((unsigned)(t[2] & 0xff) << 16) |
                ((unsigned)(t[3] & 0xff) << 24);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            PBr[4 * g + q] = PB;
            PB = addmax(PB, e[q].x >> 8, e[q].y);  // identity for a padding step
        }
    }
    int SA = Bl, SB = kNegInf;  // shifted by Bl, as in scan_slot
    static_assert(kRegWalk == 20, "the entry switch below lists kRegWalk / 4 groups");
    switch ((u + 3) >> 2) {
        case 5: scan_back_group<4>(W, pt, PBr, tb, u, lane, SA, SB); [[fallthrough]];
        case 4: scan_back_group<3>(W, pt, PBr, tb, u, lane, SA, SB); [[fallthrough]];
        case 3: scan_back_group<2>(W, pt, PBr, tb, u, lane, SA, SB); [[fallthrough]];
        case 2: scan_back_group<1>(W, pt, PBr, tb, u, lane, SA, SB); [[fallthrough]];
        case 1: scan_back_group<0>(W, pt, PBr, tb, u, lane, SA, SB); [[fallthrough]];
        default: break;
    }
}

template <int NW>
__device__ __forceinline__ umask_t<NW> warp_or(umask_t<NW> x) {
    if constexpr (NW == 1) {
        return __reduce_or_sync(PFSP_FULL, (unsigned)x);
    } else {
        const unsigned lo = __reduce_or_sync(PFSP_FULL, (unsigned)(x & 0xffffffffull));
        const unsigned hi = __reduce_or_sync(PFSP_FULL, (unsigned)(x >> 32));
        return ((umask_t<NW>)hi << 32) | lo;
    }
}

// LB2 sweep over the slots.  NC > 0: the children's accumulators are NC
// registers per direction (u <= NC); NC = 0: they live in W.Acc.  RW: the
// walks keep their records in registers (u <= kRegWalk).  LEAN: without the
// first-slot peel and the masks built from the scheduled jobs, code that only
// saves instructions (for kernels that inline several sweeps and would spill
// with it).
//
// SURV with live_only (the early exit per child, cap < INT_MAX): a job both
// of whose children have an LB1 at or above cap is not evaluated (a
// warp-uniform test per job); the other jobs are, in both directions.  Such
// children keep their LB1, a lower bound of their LB2 at or above cap, so
// they are pruned as with the full sweep and min(bound, cap) is unchanged:
// capped MinMin decides every node as with full LB2.  The walks over the
// unscheduled jobs are those of the full sweep (every job is in every
// child's sequence).  With slot checks, a job whose children are both
// decided after a slot (a pair term or its LB1 at or above cap) is not
// evaluated in the later slots either.  Without live_only every child is
// evaluated, as in the full sweep.
template <int NW, int MT, int NC, bool RW, bool SURV = false, bool LEAN = false>
__device__ __forceinline__ int lb2_sweep(const SmemTables &T, const WarpScratch &W, int n, int m_rt, int S_rt,
                                         ChildBounds<NW> &out, int cap, bool slot_checks, const int *order,
                                         bool live_only = false) {
    using mask_t = umask_t<NW>;
    constexpr bool REGACC = NC > 0;
    const int m = MT ? MT : m_rt;
    const int S = S_rt;  // slots swept: those holding the instance's pairs
    const int lane = threadIdx.x & 31;
    const int mp = m | 1;
    const mask_t U = out.U;
    const int u = out.u;
    __syncwarp();
    const mask_t all = (u >= 8 * (int)sizeof(mask_t)) ? ~mask_t(0) : ((mask_t(1) << u) - 1);
    // children already decided (only with a cap); when every child of one
    // direction is, the node is a dead end and no pair is needed
    mask_t done_f = 0, done_b = 0;
    if (cap != INT_MAX) {
#pragma unroll
        for (int h = 0; h < NW; ++h) {
            unsigned bf = __ballot_sync(PFSP_FULL, lane + 32 * h < u && out.lb1f[h] >= cap);
            unsigned bb = __ballot_sync(PFSP_FULL, lane + 32 * h < u && out.lb1b[h] >= cap);
            done_f |= (mask_t)bf << (32 * h);
            done_b |= (mask_t)bb << (32 * h);
        }
        if ((done_f & all) == all || (done_b & all) == all) return 0;
    }
    // jobs evaluated (warp-uniform): every job, or (SURV, live_only) those
    // with a child still below cap
    mask_t ev = all;
    if constexpr (SURV) {
        if (live_only) ev = all & ~(done_f & done_b);
    }
    // jobs evaluated in at least one slot: their accumulators are reduced
    // at the end (a job dropped at a slot check holds terms >= cap)
    const mask_t ev0 = ev;
    // register accumulators: with PEEL the first slot swept assigns every
    // accumulator that is read later (children below u), so none is set here.
    // Not in the register-walk kernel of 20 or more machines, which sits at
    // its 128-register cap (there the second copy of the evaluation costs a
    // spill and was measured slower), not in the early-exit sweep (SURV) at 20
    // machines, not with a run-time machine count, and not LEAN: those kernels
    // spill with it.
    constexpr bool PEEL = REGACC && !LEAN && MT > 0 && !((RW || SURV) && MT >= 20);
    int accf[REGACC ? NC : 1], accb[REGACC ? NC : 1];
    if constexpr (REGACC && !PEEL) {
#pragma unroll
        for (int c = 0; c < NC; ++c) { accf[c] = kNegInf; accb[c] = kNegInf; }
    } else if constexpr (!REGACC) {
        for (int c = 0; c < u; ++c) W.Acc[c * 32 + lane] = make_int2(kNegInf, kNegInf);
    }
    const int u4 = (u + 3) & ~3;
    // positions of the unscheduled jobs in each pair's Johnson order, one
    // bit mask per slot; with a compile-time slot count all masks are built
    // in a single walk over the unscheduled jobs, or, when fewer jobs are
    // scheduled than not, over the scheduled ones (their positions, taken
    // out of the mask of all n positions)
    constexpr int SC = MT ? (MT * (MT - 1) / 2 + 31) / 32 : 1;
    mask_t UposAll[SC];
    if constexpr (MT > 0) {
#pragma unroll
        for (int q = 0; q < SC; ++q) UposAll[q] = 0;
        const bool flip = !LEAN && 2 * u > n;
        const mask_t jobs_n = (n >= 8 * (int)sizeof(mask_t)) ? ~mask_t(0) : ((mask_t(1) << n) - 1);
        for (mask_t um = flip ? (jobs_n & ~U) : U; um;) {
            const int j = next_bit<NW>(um);
            um = drop_bit<NW>(um, j);
            const uint8_t *rj = T.rank + (size_t)j * SC * 32 + lane;
#pragma unroll
            for (int q = 0; q < SC; ++q) UposAll[q] |= mask_t(1) << rj[q * 32];
        }
        if (flip) {
            const mask_t all_pos = all_positions<NW>(n);
#pragma unroll
            for (int q = 0; q < SC; ++q) UposAll[q] ^= all_pos;
        }
    }
    int swept = 0;
#pragma unroll 1
    for (int si = 0; si < S; ++si) {
        swept = si + 1;
        const int sl = order ? order[si] : si;
        const int klw = T.kl[sl * 32 + lane];
        const int k = klw & 0xff, l = klw >> 8;
        const int Bl = W.FRB[l].z;
        const int2 *pt = T.ptab + (size_t)sl * n * 32 + lane;
        mask_t Upos;
        if constexpr (MT > 0) {
            if (order) {
                Upos = 0;
#pragma unroll
                for (int q = 0; q < SC; ++q) Upos = q == sl ? UposAll[q] : Upos;
            } else {
                Upos = UposAll[0];
#pragma unroll
                for (int q = 0; q + 1 < SC; ++q) UposAll[q] = UposAll[q + 1];
            }
        } else {
            Upos = 0;
            for (mask_t um = U; um;) {
                const int j = next_bit<NW>(um);
                um = drop_bit<NW>(um, j);
                Upos |= mask_t(1) << T.rank[((size_t)j * T.S + sl) * 32 + lane];
            }
        }
        if constexpr (RW) scan_slot_reg<NW>(W, pt, Upos, u, lane, Bl);
        else scan_slot<NW>(W, pt, Upos, u, lane, Bl);
        // evaluation: the third pair term of every evaluated child,
        // F_k + R_k + C + B_l of the child; Cb holds C + B_l(parent) and Bb
        // holds B'_l - B_l(parent), so the forward child's term is G.x + Cb
        // and the backward child's G.y + Cb + Bb
        const int2 *gk = W.G + k;
        const int *bb = W.Bb + l;
        const int *cb = W.Cb + lane;
        if constexpr (PEEL) {
            if (si == 0) {
                // every accumulator below u4 is written here (a child left
                // out gets -inf), since the slot checks read them all
#pragma unroll
                for (int c0 = 0; c0 < NC; c0 += 4) {
                    if (c0 >= u4) break;
#pragma unroll
                    for (int c = c0; c < c0 + 4; ++c) {
                        if (SURV && !((ev >> c) & 1)) {  // warp-uniform
                            accf[c] = kNegInf;
                            accb[c] = kNegInf;
                            continue;
                        }
                        const int C = cb[c * 32];
                        const int2 g = gk[c * mp];
                        accf[c] = g.x + C;
                        accb[c] = g.y + C + bb[c * mp];
                    }
                }
            } else {
                const int cend = SURV ? ((ev ? 32 - __clz((unsigned)ev) : 0) + 3) & ~3 : u4;
#pragma unroll
                for (int c0 = 0; c0 < NC; c0 += 4) {
                    if (c0 >= cend) break;
#pragma unroll
                    for (int c = c0; c < c0 + 4; ++c) {
                        if (SURV && !((ev >> c) & 1)) continue;  // warp-uniform
                        const int C = cb[c * 32];
                        const int2 g = gk[c * mp];
                        accf[c] = addmax(g.x, C, accf[c]);
                        accb[c] = max(accb[c], g.y + C + bb[c * mp]);
                    }
                }
            }
        } else if constexpr (REGACC) {
            // children past the last evaluated one cost nothing (ev is a
            // 32-bit mask here: register accumulators hold u <= 32)
            const int cend = SURV ? ((ev ? 32 - __clz((unsigned)ev) : 0) + 3) & ~3 : u4;
#pragma unroll
            for (int c0 = 0; c0 < NC; c0 += 4) {
                if (c0 >= cend) break;
#pragma unroll
                for (int c = c0; c < c0 + 4; ++c) {
                    if (SURV && !((ev >> c) & 1)) continue;  // warp-uniform
                    const int C = cb[c * 32];
                    const int2 g = gk[c * mp];
                    accf[c] = addmax(g.x, C, accf[c]);
                    accb[c] = max(accb[c], g.y + C + bb[c * mp]);
                }
            }
        } else {
            for (int c = 0; c < u; ++c) {
                if (SURV && !((ev >> c) & 1)) continue;  // warp-uniform
                const int C = cb[c * 32];
                const int2 g = gk[c * mp];
                int2 v = W.Acc[c * 32 + lane];
                v.x = addmax(g.x, C, v.x);
                v.y = max(v.y, g.y + C + bb[c * mp]);
                W.Acc[c * 32 + lane] = v;
            }
        }
        if (slot_checks && cap != INT_MAX && si + 1 < S) {
            // every child of one direction decided? (its LB1 or some pair
            // term already >= cap)
            mask_t mf = 0, mb = 0;
            if constexpr (REGACC) {
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    if (c >= u) break;
                    mf |= (mask_t)(accf[c] >= cap) << c;
                    mb |= (mask_t)(accb[c] >= cap) << c;
                }
            } else {
                for (int c = 0; c < u; ++c) {
                    int2 v = W.Acc[c * 32 + lane];
                    mf |= (mask_t)(v.x >= cap) << c;
                    mb |= (mask_t)(v.y >= cap) << c;
                }
            }
            done_f |= warp_or<NW>(mf);
            done_b |= warp_or<NW>(mb);
            if ((done_f & all) == all || (done_b & all) == all) break;
            if constexpr (SURV) {
                if (live_only) ev &= ~(done_f & done_b);
            }
        }
    }
    // ---- max over lanes (pairs) per child -------------------------------------
    if constexpr (REGACC) {
        // register accumulators (u <= 32): one warp max-reduction per
        // evaluated child and direction, kept by the child's lane
        static_assert(NW == 1, "register accumulators hold at most 32 children");
        int mf = kNegInf, mb = kNegInf;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            if (c >= u) break;
            if (SURV && !((ev0 >> c) & 1)) continue;  // warp-uniform
            const int xf = __reduce_max_sync(PFSP_FULL, accf[c]);
            const int xb = __reduce_max_sync(PFSP_FULL, accb[c]);
            mf = lane == c ? xf : mf;
            mb = lane == c ? xb : mb;
        }
        if (lane < u) {
            out.lb2f[0] = max(out.lb1f[0], mf);
            out.lb2b[0] = max(out.lb1b[0], mb);
        }
        return swept;
    }
    // shared accumulators: transpose through padded rows (rows of children
    // never evaluated stay at kNegInf)
    __syncwarp();
    int2 *X = W.X;  // [u][33], aliases the walk records and Cb
    for (int c = 0; c < u; ++c) X[c * 33 + lane] = W.Acc[c * 32 + lane];
    __syncwarp();
#pragma unroll
    for (int h = 0; h < NW; ++h) {
        int c = lane + 32 * h;
        if (c < u) {
            const int2 *row = X + c * 33;
            int mf = kNegInf, mb = kNegInf;
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                int2 v = row[i];
                mf = max(mf, v.x);
                mb = max(mb, v.y);
            }
            out.lb2f[h] = max(out.lb1f[h], mf);
            out.lb2b[h] = max(out.lb1b[h], mb);
        }
    }
    return swept;
}

// LB2 phase: lanes = machine pairs, S slots of 32 pairs.  Needs the tables
// written by decompose_lb1.  `order` (may be NULL) gives the order in which
// the slots are swept.  With cap < INT_MAX the sweep is skipped when every
// child of one direction has an LB1 >= cap, and, with slot_checks, stopped
// after the first slot at which every child of one direction has a bound
// known to be >= cap (its LB1 or a pair term already seen reaches cap).  The values returned are
// then lower bounds of the children's LB2 (each is the LB1 or the largest pair
// term seen).  Such a node has no child below cap in either MinMin rule: the
// decided direction holds no minimum below cap, so it is chosen whenever the
// other holds one, and every child of both is >= cap otherwise.
// WALK = 1: register walks (n <= kRegWalk, scratch carved with reg_walk);
// WALK = 0: walks through shared memory (any n).  Fixed per kernel, so that
// a kernel carries the register demand of one path only.
// Returns the number of 32-pair slots swept (fewer than S after an early exit).
template <int NW, int MT, int WALK = 0, bool SURV = false, bool LEAN = false>
__device__ __forceinline__ int decompose_lb2(const SmemTables &T, const WarpScratch &W, int n, int m_rt, int S_rt,
                                             ChildBounds<NW> &out, int cap, bool slot_checks, const int *order,
                                             bool live_only = false) {
    if (out.u == 0 || (MT ? MT : m_rt) < 2) return 0;
    static_assert(WALK == 0 || NW == 1, "register walks need n <= 32");
    if constexpr (WALK == 1)
        return lb2_sweep<NW, MT, kRegWalk, true, SURV, LEAN>(T, W, n, m_rt, S_rt, out, cap, slot_checks, order,
                                                               live_only);
    else
        return lb2_sweep<NW, MT, NW == 1 ? 32 : 0, false, SURV, LEAN>(T, W, n, m_rt, S_rt, out, cap, slot_checks,
                                                                        order, live_only);
}

// Both phases: the bounds of all 2u children of the node.
template <int NW, int MT, int WALK = 0, bool SCAN = false>
__device__ __forceinline__ void decompose_node(const SmemTables &T, const WarpScratch &W, int n, int m_rt,
                                               int S_rt, int kind, int job0, int job1, int d1, int d2,
                                               ChildBounds<NW> &out) {
    decompose_lb1<NW, MT, SCAN>(T, W, n, m_rt, kind, job0, job1, d1, d2, out);
    if ((kind & PFSP_LB2) && (MT ? MT : m_rt) >= 2)
        decompose_lb2<NW, MT, WALK>(T, W, n, m_rt, S_rt, out, INT_MAX, false, nullptr);
}

// Stage `words` int32 (a multiple of 4, 16-byte aligned on both sides) from
// global into shared memory with the bulk-copy engine, completion tracked by
// an mbarrier.  The wait is bounded; on expiry the block falls back to plain
// loads so that no thread can wait forever.
__device__ inline void stage_tables(int *dst, const int32_t *src, int words, uint64_t *bar) {
    const unsigned bytes = (unsigned)words * 4u;
    const unsigned sbar = (unsigned)__cvta_generic_to_shared(bar);
    bool ok = true;
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(sbar));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(sbar), "r"(bytes)
                     : "memory");
        const unsigned sdst = (unsigned)__cvta_generic_to_shared(dst);
        // copies of at most 64 KiB - 16 bytes each
        unsigned done = 0;
        while (done < bytes) {
            unsigned chunk = min(bytes - done, 65536u - 16u);
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                    sdst + done),
                "l"(reinterpret_cast<const char *>(src) + done), "r"(chunk), "r"(sbar)
                : "memory");
            done += chunk;
        }
    }
    // phase 0 completes when all bytes have landed
    unsigned ready = 0;
    for (int it = 0; it < (1 << 22) && !ready; ++it) {
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ready)
            : "r"(sbar)
            : "memory");
    }
    ok = ready != 0;
    if (!__syncthreads_and(ok)) {
        // bounded wait expired (never expected): copy with plain loads instead
        for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
        __syncthreads();
    }
    // every thread is past the wait: retire the barrier so that a later call
    // (a CTA that moves to another instance) can initialise it again
    if (threadIdx.x == 0) asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(sbar) : "memory");
    __syncthreads();
}

constexpr int kWarpsPerCta = 16;

// Value of child compact index c held by lanes (c & 31) of register h = c >> 5.
template <int NW>
__device__ __forceinline__ int gather_child(const int (&v)[NW], int c) {
    int a = __shfl_sync(PFSP_FULL, v[0], c & 31);
    if constexpr (NW == 2) {
        int b = __shfl_sync(PFSP_FULL, v[1], c & 31);
        return c >= 32 ? b : a;
    }
    return a;
}

}  // namespace pfsp
