// mlp_rows.cu -- training rows for the ordering network, built on the GPU
// from nodes the solver decomposed (not in the paper).
//
// Each node [perm, d1, d2] yields 1 + 2n rows:
//   row 0          the parent: features = front F_k, back B_k, remaining work
//                  R_k of every machine divided by the instance's mean machine
//                  load; targets on columns 1..P: pair (k, l) is 1 when its
//                  two-machine term is the LB2 of at least one child and that
//                  LB2 is above the child's LB1.
//   row 1 + j      the forward child of job j, features of the child (front
//                  after j, same back, remaining work minus j); column-0
//                  target 1 for the child of least LB2 among the forward
//                  children (ties: lowest job id).
//   row 1 + n + j  the backward child of job j, likewise.
// Rows of scheduled jobs have zero features and a zero mask.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <vector>

#include "bound_device.cuh"
#include "pfsp_internal.h"

struct pfsp_mlp;

namespace pfsp {

int mlp_dims(const pfsp_mlp *M, int *m, int *D0, int *O);

struct RowsArgs {
    const uint8_t *perm, *d1, *d2;
    long long num_nodes;
    const int32_t *tab;
    int tab_words, n, m, S;
    int off_pm, off_tot, off_kl, off_rank, off_ptab;
    int warp_words;  // bound scratch + 256 words of per-child bounds
    int D0, O;
    float inv_scale;
    float *X, *T, *M;
    int parents_only;  // 1: only the parent row of each node (features, no targets)
};

template <int NW, int MT>
__global__ void __launch_bounds__(256) mlp_rows_kernel(RowsArgs a) {
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
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int n = a.n, m = MT ? MT : a.m, S = a.S, mp = m | 1, nj = (n + 3) & ~3;
    int *base = smem + a.tab_words + wib * a.warp_words;
    WarpScratch W = carve_warp(base, n, m);
    int *lb = base + a.warp_words - 256;  // [0..63] lb1f, [64..] lb1b, [128..] lb2f, [192..] lb2b by compact index
    const int rows = a.parents_only ? 1 : 1 + 2 * n;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long node = (long long)blockIdx.x * (blockDim.x >> 5) + wib; node < a.num_nodes; node += nw) {
        float *X = a.X + (size_t)node * rows * a.D0;
        for (int e = lane; e < rows * a.D0; e += 32) X[e] = 0.0f;
        float *Tt = nullptr, *Mk = nullptr;
        if (!a.parents_only) {
            Tt = a.T + (size_t)node * rows * a.O;
            Mk = a.M + (size_t)node * rows * a.O;
            for (int e = lane; e < rows * a.O; e += 32) {
                Tt[e] = 0.0f;
                Mk[e] = 0.0f;
            }
        }
        int d1 = a.d1[node], d2 = a.d2[node];
        if (d1 + d2 > n) continue;
        const uint8_t *pr = a.perm + node * n;
        int job0 = lane < n ? pr[lane] : 0;
        int job1 = (NW == 2 && lane + 32 < n) ? pr[lane + 32] : 0;
        job0 = job0 < n ? job0 : 0;
        job1 = job1 < n ? job1 : 0;
        ChildBounds<NW> cb;
        decompose_lb1<NW, MT>(T, W, n, m, a.parents_only ? PFSP_LB1 : PFSP_LB1 | PFSP_LB2, job0, job1, d1, d2, cb);
        __syncwarp();
        // parent features
        if (lane < m) {
            const int4 P = W.FRB[lane];
            X[lane] = P.x * a.inv_scale;
            X[m + lane] = P.z * a.inv_scale;
            X[2 * m + lane] = P.y * a.inv_scale;
        }
        if (a.parents_only) continue;
        decompose_lb2<NW, MT>(T, W, n, m, S, cb, INT_MAX, false, nullptr);
        const int u = cb.u;
        __syncwarp();
        // children: features, bounds for the pair pass, descend-first targets
        for (int h = 0; h < NW; ++h) {
            int c = lane + 32 * h;
            if (c < u) {
                lb[c] = cb.lb1f[h];
                lb[64 + c] = cb.lb1b[h];
                lb[128 + c] = cb.lb2f[h];
                lb[192 + c] = cb.lb2b[h];
                const int j = W.ul[c];
                float *xf = X + (size_t)(1 + j) * a.D0, *xb = X + (size_t)(1 + n + j) * a.D0;
                for (int k = 0; k < m; ++k) {
                    const int pk = T.pm[k * nj + j];
                    const int rc = W.FRB[k].y - pk;
                    xf[k] = (W.G[c * mp + k].x - rc) * a.inv_scale;  // front after j
                    xf[m + k] = W.FRB[k].z * a.inv_scale;
                    xf[2 * m + k] = rc * a.inv_scale;
                    xb[k] = W.FRB[k].x * a.inv_scale;
                    xb[m + k] = (W.Bb[c * mp + k] + W.FRB[k].z) * a.inv_scale;  // back after j
                    xb[2 * m + k] = rc * a.inv_scale;
                }
                Mk[(size_t)(1 + j) * a.O] = 1.0f;
                Mk[(size_t)(1 + n + j) * a.O] = 1.0f;
            }
        }
        __syncwarp();
        if (lane == 0 && u > 0) {
            int bf = 0, bb = 0;
            for (int c = 1; c < u; ++c) {
                if (lb[128 + c] < lb[128 + bf]) bf = c;
                if (lb[192 + c] < lb[192 + bb]) bb = c;
            }
            Tt[(size_t)(1 + W.ul[bf]) * a.O] = 1.0f;
            Tt[(size_t)(1 + n + W.ul[bb]) * a.O] = 1.0f;
        }
        // pair targets: sweep the slots again and compare each pair's term
        // with the children's final LB2
        for (int s = 0; s < S && m >= 2 && u > 0; ++s) {
            const int klw = T.kl[s * 32 + lane];
            const int k = klw & 0xff, l = klw >> 8;
            const int Bl = W.FRB[l].z;
            umask_t<NW> Upos = 0;
            for (umask_t<NW> um = cb.U; um;) {
                const int j = next_bit<NW>(um);
                um = drop_bit<NW>(um, j);
                Upos |= umask_t<NW>(1) << T.rank[((size_t)j * T.S + s) * 32 + lane];
            }
            scan_slot<NW>(W, T.ptab + (size_t)s * n * 32 + lane, Upos, u, lane, Bl);
            bool hit = false;
            for (int c = 0; c < u; ++c) {
                // Cb holds C + B_l and Bb holds B'_l - B_l (parent's B_l)
                const int C = W.Cb[c * 32 + lane];
                const int ef = W.G[c * mp + k].x + C;
                const int eb = W.G[c * mp + k].y + C + W.Bb[c * mp + l];
                hit |= (ef == lb[128 + c] && lb[128 + c] > lb[c]) || (eb == lb[192 + c] && lb[192 + c] > lb[64 + c]);
            }
            // the lane's pair (k < l; dummy lanes hold k = l = 0), in the
            // network's column order whatever the instance's pair order
            if (l > k) {
                const int q = pair_index(k, l, m);
                Tt[1 + q] = hit ? 1.0f : 0.0f;
                Mk[1 + q] = 1.0f;
            }
        }
        __syncwarp();
    }
}

template <int NW, int MT>
static cudaError_t launch_rows(const RowsArgs &a, int warps) {
    size_t smem = (size_t)(a.tab_words + warps * a.warp_words) * 4;
    auto kern = mlp_rows_kernel<NW, MT>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    kern<<<nsm, warps * 32, smem>>>(a);
    return cudaGetLastError();
}

}  // namespace pfsp

using namespace pfsp;

namespace pfsp {

cudaError_t mlp_forward_dev(const pfsp_mlp *M, const float *dX, long long rows, float *dY);

// Arguments of the rows kernel for `inst` and `mlp` (checked by the caller).
static RowsArgs rows_args(const pfsp_instance *inst, int D0, int O, long long num_nodes) {
    const TableLayout &L = inst->lay;
    long long total = 0;
    for (int j = 0; j < inst->n * inst->m; ++j) total += inst->p_host[j];
    RowsArgs a;
    memset(&a, 0, sizeof(a));
    a.num_nodes = num_nodes;
    a.tab = inst->d_tab;
    a.tab_words = L.words;
    a.n = inst->n;
    a.m = inst->m;
    a.S = L.Ssweep;
    a.off_pm = L.off_pm;
    a.off_tot = L.off_tot;
    a.off_kl = L.off_kl;
    a.off_rank = L.off_rank;
    a.off_ptab = L.off_ptab;
    a.warp_words = warp_words(inst->n, inst->m, inst->n > 32, true) + 256;
    a.D0 = D0;
    a.O = O;
    a.inv_scale = total > 0 ? (float)inst->m / (float)total : 1.0f;
    return a;
}

static cudaError_t run_rows(const pfsp_instance *inst, const RowsArgs &a) {
    int optin = 48 * 1024, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    int warps = (int)std::min<long long>(8, ((long long)optin - 64 - (long long)a.tab_words * 4) / (a.warp_words * 4));
    if (warps < 1) return cudaErrorInvalidConfiguration;
    if (inst->n <= 32) {
        switch (inst->m) {
            case 5: return launch_rows<1, 5>(a, warps);
            case 10: return launch_rows<1, 10>(a, warps);
            case 20: return launch_rows<1, 20>(a, warps);
            default: return launch_rows<1, 0>(a, warps);
        }
    }
    return inst->m == 5 ? launch_rows<2, 5>(a, warps) : launch_rows<2, 0>(a, warps);
}

static int check_rows_args(const pfsp_instance *inst, const pfsp_mlp *mlp, int64_t num_nodes, const uint8_t *perm,
                           const uint8_t *d1, const uint8_t *d2, int *D0, int *O) {
    if (!inst || !mlp || num_nodes < 0) return set_error(PFSP_ERR_INVALID, "bad argument");
    if (num_nodes > 0 && (!perm || !d1 || !d2)) return set_error(PFSP_ERR_INVALID, "NULL node buffer");
    int mm = 0;
    mlp_dims(mlp, &mm, D0, O);
    if (mm != inst->m) return set_error(PFSP_ERR_INVALID, "network built for m=%d, instance has m=%d", mm, inst->m);
    if (!inst->lb2_ok) return set_error(PFSP_ERR_UNSUPPORTED, "LB2 tables exceed shared memory");
    for (int64_t i = 0; i < num_nodes; ++i)
        if (d1[i] + d2[i] > inst->n) return set_error(PFSP_ERR_INVALID, "node %lld: d1 + d2 > n", (long long)i);
    return PFSP_OK;
}

// Nodes to the device: perm [N][n], then d1 [N], then d2 [N].
static cudaError_t upload_nodes(int n, int64_t N, const uint8_t *perm, const uint8_t *d1, const uint8_t *d2,
                                uint8_t **dp) {
    cudaError_t e = cudaMalloc(dp, (size_t)N * (n + 2));
    if (e == cudaSuccess) e = cudaMemcpy(*dp, perm, (size_t)N * n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(*dp + (size_t)N * n, d1, N, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(*dp + (size_t)N * (n + 1), d2, N, cudaMemcpyHostToDevice);
    return e;
}

}  // namespace pfsp

extern "C" int pfsp_mlp_rows(const pfsp_instance *inst, const pfsp_mlp *mlp, int64_t num_nodes, const uint8_t *perm,
                             const uint8_t *d1, const uint8_t *d2, float *X, float *T, float *M) {
    int D0 = 0, O = 0;
    int rc = check_rows_args(inst, mlp, num_nodes, perm, d1, d2, &D0, &O);
    if (rc != PFSP_OK) return rc;
    if (num_nodes == 0) return PFSP_OK;
    if (!X || !T || !M) return set_error(PFSP_ERR_INVALID, "NULL buffer");
    const int n = inst->n;
    RowsArgs a = rows_args(inst, D0, O, num_nodes);
    const size_t rows = (size_t)num_nodes * (1 + 2 * n);
    uint8_t *dp = nullptr;
    float *dX = nullptr, *dT = nullptr, *dM = nullptr;
    cudaError_t e = upload_nodes(n, num_nodes, perm, d1, d2, &dp);
    if (e == cudaSuccess) e = cudaMalloc(&dX, rows * D0 * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dT, rows * O * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dM, rows * O * 4);
    a.perm = dp;
    a.d1 = dp + (size_t)num_nodes * n;
    a.d2 = dp + (size_t)num_nodes * (n + 1);
    a.X = dX;
    a.T = dT;
    a.M = dM;
    if (e == cudaSuccess) e = run_rows(inst, a);
    if (e == cudaSuccess) e = cudaMemcpy(X, dX, rows * D0 * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(T, dT, rows * O * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(M, dM, rows * O * 4, cudaMemcpyDeviceToHost);
    cudaFree(dp);
    cudaFree(dX);
    cudaFree(dT);
    cudaFree(dM);
    return e == cudaSuccess ? PFSP_OK : set_error(PFSP_ERR_CUDA, "pfsp_mlp_rows: %s", cudaGetErrorString(e));
}

extern "C" int pfsp_mlp_pair_scores(const pfsp_instance *inst, const pfsp_mlp *mlp, int64_t num_nodes,
                                    const uint8_t *perm, const uint8_t *d1, const uint8_t *d2, float *score) {
    int D0 = 0, O = 0;
    int rc = check_rows_args(inst, mlp, num_nodes, perm, d1, d2, &D0, &O);
    if (rc != PFSP_OK) return rc;
    if (!score) return set_error(PFSP_ERR_INVALID, "NULL score buffer");
    if (num_nodes == 0) return set_error(PFSP_ERR_INVALID, "no nodes to score");
    const int n = inst->n, P = inst->lay.P;
    RowsArgs a = rows_args(inst, D0, O, num_nodes);
    a.parents_only = 1;
    uint8_t *dp = nullptr;
    float *dX = nullptr, *dY = nullptr;
    cudaError_t e = upload_nodes(n, num_nodes, perm, d1, d2, &dp);
    if (e == cudaSuccess) e = cudaMalloc(&dX, (size_t)num_nodes * D0 * 4);
    if (e == cudaSuccess) e = cudaMalloc(&dY, (size_t)num_nodes * O * 4);
    a.perm = dp;
    a.d1 = dp + (size_t)num_nodes * n;
    a.d2 = dp + (size_t)num_nodes * (n + 1);
    a.X = dX;
    if (e == cudaSuccess) e = run_rows(inst, a);
    if (e == cudaSuccess) e = mlp_forward_dev(mlp, dX, num_nodes, dY);
    std::vector<float> Y;
    if (e == cudaSuccess) {
        Y.resize((size_t)num_nodes * O);
        e = cudaMemcpy(Y.data(), dY, Y.size() * 4, cudaMemcpyDeviceToHost);
    }
    cudaFree(dp);
    cudaFree(dX);
    cudaFree(dY);
    if (e != cudaSuccess) return set_error(PFSP_ERR_CUDA, "pfsp_mlp_pair_scores: %s", cudaGetErrorString(e));
    // mean over the nodes of the probability of each pair column
    for (int q = 0; q < P; ++q) {
        double acc = 0.0;
        for (int64_t i = 0; i < num_nodes; ++i) acc += 1.0 / (1.0 + std::exp(-(double)Y[(size_t)i * O + 1 + q]));
        score[q] = (float)(acc / (double)num_nodes);
    }
    return PFSP_OK;
}

extern "C" int pfsp_learn_pair_order(pfsp_instance *inst, const pfsp_mlp *mlp, int64_t num_nodes,
                                     const uint8_t *perm, const uint8_t *d1, const uint8_t *d2, int32_t *order) {
    if (!inst) return set_error(PFSP_ERR_INVALID, "instance is NULL");
    const int P = inst->lay.P;
    std::vector<float> score(P > 0 ? P : 1);
    int rc = pfsp_mlp_pair_scores(inst, mlp, num_nodes, perm, d1, d2, score.data());
    if (rc != PFSP_OK) return rc;
    std::vector<int32_t> ord(P);
    for (int q = 0; q < P; ++q) ord[q] = q;
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t x, int32_t y) { return score[x] > score[y]; });
    rc = pfsp_set_pair_order(inst, ord.data());
    if (rc == PFSP_OK && order) memcpy(order, ord.data(), sizeof(int32_t) * P);
    return rc;
}

extern "C" int pfsp_learn_lb2_pairs(pfsp_instance *inst, const pfsp_mlp *mlp, int64_t num_nodes, const uint8_t *perm,
                                    const uint8_t *d1, const uint8_t *d2, int keep, int32_t *pairs) {
    if (!inst) return set_error(PFSP_ERR_INVALID, "instance is NULL");
    const int n = inst->n, P = inst->lay.P;
    if (keep < 1) return set_error(PFSP_ERR_INVALID, "keep must be >= 1");
    if (P == 0) return set_error(PFSP_ERR_INVALID, "an instance with one machine has no machine pair");
    // default sample: the 2n children of the root (job j first, or job j last)
    std::vector<uint8_t> rp, r1, r2;
    if (!perm) {
        num_nodes = 2 * (int64_t)n;
        rp.resize((size_t)num_nodes * n);
        r1.resize(num_nodes);
        r2.resize(num_nodes);
        for (int j = 0; j < n; ++j)
            for (int side = 0; side < 2; ++side) {
                uint8_t *row = &rp[((size_t)2 * j + side) * n];
                int c = 0;
                if (side == 0) row[c++] = (uint8_t)j;
                for (int x = 0; x < n; ++x)
                    if (x != j) row[c++] = (uint8_t)x;
                if (side == 1) row[c++] = (uint8_t)j;
                r1[2 * j + side] = side == 0 ? 1 : 0;
                r2[2 * j + side] = side == 1 ? 1 : 0;
            }
        perm = rp.data();
        d1 = r1.data();
        d2 = r2.data();
    }
    std::vector<float> score(P);
    int rc = pfsp_mlp_pair_scores(inst, mlp, num_nodes, perm, d1, d2, score.data());
    if (rc != PFSP_OK) return rc;
    std::vector<int32_t> ord(P);
    for (int q = 0; q < P; ++q) ord[q] = q;
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t x, int32_t y) { return score[x] > score[y]; });
    const int k = std::min(keep, P);
    rc = pfsp_set_lb2_pairs(inst, ord.data(), k);
    if (rc == PFSP_OK && pairs) memcpy(pairs, ord.data(), sizeof(int32_t) * k);
    return rc;
}
