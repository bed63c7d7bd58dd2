// minht_device.cuh -- the heads and tails refinement of LB1 (an option, not
// in the paper, which leaves the front of an empty sigma1 and the back of an
// empty sigma2 at zero).  With sigma1 empty no unscheduled job can start on
// machine k before its own work on machines 0..k-1, and with sigma2 empty none
// can end before its own work on machines k+1..m-1 is added: the front (back)
// is raised to the least such work over the child's unscheduled jobs.
#pragma once

#include <climits>

#include "bound_device.cuh"

namespace pfsp {

// Per machine k (lane k), the two least values and the job of the least of
// a job's work before k (head) and after k (tail), over the jobs of U.
struct HeadTailMins {
    int h1, h2, hj, t1, t2, tj;
};

template <int NW, int MT>
__device__ __forceinline__ HeadTailMins head_tail_mins(const SmemTables &T, const WarpScratch &W, int n, int m_rt,
                                                       int u) {
    const int m = MT ? MT : m_rt;
    const int lane = threadIdx.x & 31;
    const int nj = (n + 3) & ~3;
    HeadTailMins r{INT_MAX, INT_MAX, -1, INT_MAX, INT_MAX, -1};
    for (int c = 0; c < u; ++c) {
        const int j = W.ul[c];
        const int v = lane < m ? T.pm[lane * nj + j] : 0;
        int incl = v;  // inclusive prefix sum over machines (lanes)
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(PFSP_FULL, incl, o);
            if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(PFSP_FULL, incl, m - 1);
        const int head = incl - v, tail = total - incl;
        if (head < r.h1) {
            r.h2 = r.h1;
            r.h1 = head;
            r.hj = j;
        } else if (head < r.h2) {
            r.h2 = head;
        }
        if (tail < r.t1) {
            r.t2 = r.t1;
            r.t1 = tail;
            r.tj = j;
        } else if (tail < r.t2) {
            r.t2 = tail;
        }
    }
    return r;
}

// The least value over U without job j (0 over an empty set).
__device__ __forceinline__ int min_without(int v1, int v2, int vj, int j) {
    const int v = vj == j ? v2 : v1;
    return v == INT_MAX ? 0 : v;
}

// Raise the LB1 of the children whose sigma1 (backward children of a node with
// d1 = 0) or sigma2 (forward children of a node with d2 = 0) is empty, after
// decompose_lb1 (W.FRB and W.ul of the parent, out.lb1*); LB2 entries become
// at least the refined LB1.  Call with d1 == 0 || d2 == 0; warp-uniform.
template <int NW, int MT>
__device__ __forceinline__ void refine_minht(const SmemTables &T, const WarpScratch &W, int n, int m_rt, int d1,
                                             int d2, ChildBounds<NW> &out) {
    const int m = MT ? MT : m_rt;
    const int lane = threadIdx.x & 31;
    const int nj = (n + 3) & ~3;
    const int u = out.u;
    const HeadTailMins s = head_tail_mins<NW, MT>(T, W, n, m, u);
#pragma unroll
    for (int h = 0; h < NW; ++h) {
        const int c = lane + 32 * h;
        const bool on = c < u;
        const int j = on ? W.ul[c] : 0;
        int f = 0, lf = kNegInf, b = 0, lb = kNegInf;
        // one loop over the machines, uniform across the warp (the shuffles
        // broadcast machine k's minima): forward children upwards, backward
        // children downwards
#pragma unroll
        for (int i = 0; i < (MT ? MT : 32); ++i) {
            if (!MT && i >= m) break;
            const int kf = i, kb = m - 1 - i;
            const int t1 = __shfl_sync(PFSP_FULL, s.t1, kf), t2 = __shfl_sync(PFSP_FULL, s.t2, kf);
            const int tj = __shfl_sync(PFSP_FULL, s.tj, kf);
            const int h1 = __shfl_sync(PFSP_FULL, s.h1, kb), h2 = __shfl_sync(PFSP_FULL, s.h2, kb);
            const int hj = __shfl_sync(PFSP_FULL, s.hj, kb);
            const int4 Pf = W.FRB[kf], Pb = W.FRB[kb];
            const int pf = T.pm[kf * nj + j], pb = T.pm[kb * nj + j];
            // forward child (sigma1 j, ()): front from the parent's, remaining
            // work without j, back the least tail of the others
            f = max(f, Pf.x) + pf;
            lf = max(lf, f + Pf.y - pf + min_without(t1, t2, tj, j));
            // backward child ((), j sigma2): back from the parent's, front the
            // least head of the others
            b = max(b, Pb.z) + pb;
            lb = max(lb, min_without(h1, h2, hj, j) + Pb.y - pb + b);
        }
        if (on && d2 == 0) {
            out.lb1f[h] = max(out.lb1f[h], lf);
            out.lb2f[h] = max(out.lb2f[h], out.lb1f[h]);
        }
        if (on && d1 == 0) {
            out.lb1b[h] = max(out.lb1b[h], lb);
            out.lb2b[h] = max(out.lb2b[h], out.lb1b[h]);
        }
    }
}

}  // namespace pfsp
