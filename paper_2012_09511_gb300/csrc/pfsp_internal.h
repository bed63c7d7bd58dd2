// pfsp_internal.h -- host/device layout shared by the library's translation
// units (not part of the public ABI).
#pragma once

#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/pfsp.h"

namespace pfsp {

constexpr int kMaxJobs = 64;
constexpr int kMaxMachines = 32;
constexpr int kNegInf = -(1 << 29);         // "minus infinity" of the max-plus maps
constexpr int kMaxTime = (1 << 22) - 1;     // largest accepted processing time
constexpr long long kMaxTotal = 1LL << 28;  // largest accepted sum of all times
constexpr int kMaxTableBytes = 160 * 1024;  // LB2 tables must fit in shared memory
constexpr long long kBoundChunk = 1 << 18;  // nodes per chunk of the host-pointer bounding pipeline
constexpr int kDefaultCheckEvery = 8;      // explorer iterations between limit checks and length publications

// Default smallest interval (in leaves) a victim splits for a thief: the
// leaves of a subtree with min(floor(2n/5), 9) jobs left (8! at n = 20, 9!
// from n = 23 on).  Smaller intervals cost the thief more to rebuild (a path
// of decompositions down to the interval's start) than the work they hold;
// much larger ones leave thieves idle (12! was slower than 8!-10! on 30-job
// proofs).
inline float default_min_steal(int n) {
    double f = 1.0;
    const int jobs = (2 * n) / 5 < 9 ? (2 * n) / 5 : 9;
    for (int k = 2; k <= jobs; ++k) f *= k;
    return (float)f;
}

// Instance tables, one contiguous int32 blob in device memory that every CTA
// copies into its shared memory.  Word offsets are multiples of 4 (16 bytes):
//   pm   [m][nj]       processing times by machine (nj = n rounded up to 4)
//   tot  [32]          per-machine totals T_k = sum_j p[j][k]
//   pq   [n][m] int2  per job j and machine k: {P_k, Q_k} with
//                      P_k = sum_{k' <= k} p[j][k'], Q_k = sum_{k' >= k} p[j][k']
//                      (2 n m words, rounded up to a multiple of 4)
//   kl   [S*32]        machine pair at slot position i: k | l << 8 (dummy: 0);
//                      pairs sit in the instance's pair order (default: k = 0..m-2,
//                      l = k+1..m-1), position i in slot i / 32, lane i % 32
//   rank [n][S][32]    uint8: bit of job j in the lane's position masks:
//                      31 - t (n <= 32) or t (n > 32), t its position in the
//                      Johnson order of the lane's pair (dummy lanes: t = j)
//   ptab [S][n][32]    int2 per (slot, position, lane): the lane's pair,
//                      x = (a << 8) | job, y = b, for the job at position t of
//                      the pair's Johnson order, with a = p[j][l] - p[j][k]
//                      and b = g_j + p[j][l] (g_j = lag).  Dummy lanes (pairs
//                      past the last one) hold job i at position i with a = 0,
//                      b = kNegInf: the identity map.
struct TableLayout {
    int n, m, P, S, nj;
    int Ssweep;  // slots holding the pairs LB2 uses (S unless LB2 uses a subset of the pairs)
    int off_pm, off_tot, off_pq, off_kl, off_rank, off_ptab, words;
};

TableLayout table_layout(int n, int m);

}  // namespace pfsp

struct pfsp_instance {
    int n, m;
    int device;
    int32_t *p_host;             // n*m job-major copy
    pfsp::TableLayout lay;
    int32_t *d_tab;              // device table blob (lay.words int32)
    bool lb2_ok;                 // LB2 tables fit in shared memory
    // grow-only device scratch of the host-pointer entry points
    void *d_scratch;
    size_t scratch_bytes;
    pfsp_stats_t stats;
    int32_t *pair_order;         // pair at each slot position (NULL: k < l lexicographic)
    int pair_count;              // pairs LB2 uses (the first ones of pair_order; P by default)
};

namespace pfsp {

// Kernel launchers (bound_kernel.cu).  Return cudaError_t of the launch.
// With summary != NULL the reduce mode: one pfsp_node_summary per node
// (survivors below ub) instead of the bound arrays.
cudaError_t launch_bound_batch(const pfsp_instance *inst, int kind, long long num_nodes,
                               const uint8_t *perm, const uint8_t *d1, const uint8_t *d2,
                               int32_t *lb1, int32_t *lb2, cudaStream_t stream,
                               pfsp_node_summary *summary = nullptr, int ub = 0);
// With the heads and tails refinement of LB1 (bound_minht.cu).
cudaError_t launch_bound_batch_minht(const pfsp_instance *inst, int kind, long long num_nodes,
                                     const uint8_t *perm, const uint8_t *d1, const uint8_t *d2,
                                     int32_t *lb1, int32_t *lb2, cudaStream_t stream);

// Error reporting shared by the C-ABI translation units.
int set_error(int code, const char *fmt, ...);

struct MlpDev;
// The network's device view and dimensions (mlp.cu).
MlpDev mlp_view(const pfsp_mlp *M);
// Writes the network's inference image of O3 output columns (layout in
// mlp_device.cuh) to the device buffer dst, on stream st.
cudaError_t mlp_build_image(const pfsp_mlp *M, int O3, void *dst, cudaStream_t st);
int mlp_dims(const pfsp_mlp *M, int *m, int *D0, int *O);

// Host-side builders shared by the entry points (capi.cu, solve_capi.cu).
// pair_order: the pair (index in k < l lexicographic order) placed at each
// slot position, NULL for the lexicographic order itself; only the first
// `count` positions hold pairs (count < P: LB2 over that subset), the others
// are dummy lanes (identity maps).
void build_tables(const TableLayout &L, const int32_t *p, std::vector<int32_t> &blob, const int32_t *pair_order,
                  int count);

// Index of machine pair k < l in the lexicographic order of all m(m-1)/2 pairs.
__host__ __device__ inline int pair_index(int k, int l, int m) { return k * (2 * m - k - 1) / 2 + (l - k - 1); }
int neh(int n, int m, const int32_t *p, std::vector<int> &perm);

}  // namespace pfsp
