// solve_internal.h -- arguments and constants of the explorer-pool kernel.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "mlp_device.cuh"

namespace pfsp {

constexpr int kSolveWarps = 12;          // explorers (warps) per CTA at most
constexpr int kSolveWarpsLearned = 12;   // with the ordering network (same as the plain solver)
constexpr int kPrunedLB = 0x7fffffff;     // bound stored for a pruned cell
constexpr int kWaitLimit = 1 << 21;       // polls of a thief waiting for an answer
constexpr int kErrStealWait = 1;          // error detail: a steal answer never came
constexpr int kErrNoProgress = 2;         // error detail: no decomposition for kWatchdogNs
constexpr int kErrBadInterval = 3;        // error detail: a received interval was not valid
constexpr int kErrRecordLock = 4;         // error detail: the best-permutation record stayed locked
constexpr int kLockLimit = 1 << 20;       // attempts to take that lock
constexpr unsigned long long kNoRequest = ~0ull;  // empty mailbox
constexpr unsigned long long kWatchdogNs = 10ull * 1000 * 1000 * 1000;
#define PFSP_FWD_DIR 0

// Explorer-pool kernel instantiations
constexpr int kKindPlain = 0;    // the paper's solver
constexpr int kKindLearned = 1;  // with the ordering network
constexpr int kKindCoop = 2;     // with the host heuristic threads' exchange
constexpr int kKindMinht = 3;    // with the heads and tails refinement of LB1
constexpr int kKindLb1 = 4;      // LB1 solves: the loop carries no LB2 code
constexpr int kKindDiag = 5;     // with phase timers and decomposition traces (both bounds)
constexpr int kKindEE = 6;       // with the early exit of the LB2 sweep (PFSP_EARLY_EXIT)
constexpr int kKindBatch = 7;    // the paper's solver inside the batched pool (lean LB2 sweep)

// Phases of an explorer's loop whose SM clock cycles are summed per solve
// (pfsp_stats_t.phase_cycles) when the timers are on.  Each reading of the SM
// clock costs enough that a timed solve runs several times slower, so they
// are off unless asked for.
constexpr int kPhService = 0;  // limit checks, steal requests answered, length publication
constexpr int kPhSelect = 1;   // next live cell, backtracking, interval-end check
constexpr int kPhDecode = 2;   // node decoding into [sigma1 | unscheduled | sigma2]
constexpr int kPhLB1 = 3;      // front/back wavefronts and LB1 of all children
constexpr int kPhLB2 = 4;      // LB2 sweep over the machine pairs
constexpr int kPhBranch = 5;   // MinMin, pruning, the new row, leaves (and the network's row order)
constexpr int kPhInit = 6;     // rebuilding the path to a new interval's start
constexpr int kPhIdle = 7;     // stealing and waiting without work
constexpr int kPhases = 8;

// Exchange with the host heuristic threads, in host-mapped memory.  The
// explorers read host_ub and snap_req at their limit checks: host_ub is folded
// into the device incumbent, and a new snap_req asks each explorer to copy the
// node it last decomposed into its slot, then to set the slot's seq to it.  An
// explorer that lowers the incumbent with a leaf also copies that schedule to
// dev_perm and then its makespan to dev_cmax (concurrent writers may tear the
// copy: the host recomputes the makespan of what it reads).
struct CoopShared {
    volatile int host_ub;
    volatile int snap_req;
    volatile int dev_cmax;
    int pad[13];
    uint8_t dev_perm[64];
};
struct CoopSlot {
    volatile int seq;  // snap_req answered
    uint8_t d1, d2, pad[2];
    uint8_t perm[64];  // [sigma1 | unscheduled | sigma2]
};
static_assert(sizeof(CoopShared) == 128 && sizeof(CoopSlot) == 72, "exchange layout");

// Checkpoint record of one explorer (device and host): [0] valid, [1] start
// level (0xff: the first level below which the start digits are all zero),
// [2] coefficient of n! of the end, [3] unused, [4..67] start digits,
// [68..131] end digits.
constexpr int kCkptRecord = 132;

struct SolveArgs {
    // instance tables (same layout as the bounding kernel)
    const int32_t *tab;
    int tab_words;
    int n, m, S;
    int off_pm, off_tot, off_kl, off_rank, off_ptab;
    int warp_words;  // bound scratch words per warp (excluding explorer words)
    int bound;       // PFSP_LB1 or PFSP_LB2
    int branching;   // PFSP_MINMIN, PFSP_MINMIN_CAPPED, PFSP_MINBRANCH or PFSP_MINSUM
    int cap;
    int K;           // explorers = warps in the grid
    int row_stride;       // row elements per explorer (n * n, or the batch's largest n squared)
    uint8_t *rows_job;    // [K][row_stride]
    int32_t *rows_lb;     // [K][row_stride]
    const int *inst_of;   // batched solves: [K] instance each explorer works on (NULL otherwise)
    int my_inst;          // batched solves: this CTA's instance
    int *perm_lock;       // batched solves: lock of this instance's best-permutation record
    int *perm_cmax;       // batched solves: makespan of the recorded permutation
    uint8_t *inst_perm;   // batched solves: [64] recorded permutation (NULL: per-explorer slots)
    uint8_t *in_start;    // [K][64] start digits of an incoming interval
    uint8_t *in_end;      // [K][65] end: [0] = coefficient of n!, [1..n] digits
    uint8_t *in_level;    // [K] start level of an incoming interval (0xff: first zero-rest level), or NULL
    unsigned *seq_posted; // [K] sequence number of each explorer's last posted steal request (or NULL)
    unsigned *seq_taken;  // [K] sequence number of the last answer it took in (or NULL)
    // rows handed over with a stolen interval (hand_dir NULL: none): the
    // victim writes rows 0..L of the shared path into the thief's slot of
    // hand_job / hand_lb (the unused rows_job / rows_lb when the rows live in
    // shared memory), their directions into hand_dir and L into hand_lc; the
    // thief copies them into its own rows
    uint8_t *hand_job;    // [K][row_stride]
    int32_t *hand_lb;     // [K][row_stride]
    uint8_t *hand_dir;    // [K][64]
    int *hand_lc;         // [K]
    uint8_t *ckpt;        // [K][kCkptRecord] remaining interval of each explorer at a limit stop (NULL: off)
    unsigned long long *mailbox;   // [K] request: instance << 40 | sequence << 20 | thief, or kNoRequest
    unsigned long long *response;  // [K] answer to a thief: sequence << 2 | 1 granted / 2 denied
    float *len_est;       // [K] log2 of the remaining interval length, -1 if empty
    int *active;          // explorers holding work
    int *ub;              // incumbent (exclusive)
    unsigned long long *best_key;  // (cmax << 32) | explorer
    uint8_t *best_perm;   // [K][64]
    unsigned long long *counters;  // decomposed, bounded, leaves, pruned, steals, iters, limit count, LB2 slots
    unsigned long long *phase;     // [kPhases] cycles per phase summed over explorers (NULL: timers off)
    long long node_limit;
    unsigned long long time_limit_ns;  // stop after this long on the device clock; 0 = none
    int *stop;            // 0 run, 1 node limit, 2 time limit, 3 error
    int *err;
    float min_steal;      // smallest interval length (leaves) a victim gives away
    int check_every;      // power of two: iterations between limit checks
    int warp_base;        // word offset of the first warp's scratch (32-byte aligned)
    // recorded decompositions (pfsp_solve_trace); trace_cap = 0: off
    uint8_t *trace_perm, *trace_d1, *trace_d2;
    unsigned long long *trace_count;
    long long trace_cap;
    int trace_stride;
    // learned ordering (PFSP_LEARN_* / PFSP_EARLY_EXIT bits; 0: off)
    int learned;
    const unsigned char *net_image;  // the network's inference image in global memory (mlp_device.cuh)
    int net_D0, net_O3;   // its input width and staged output columns
    float inv_scale;      // 1 / (mean machine load) for the network's features
    int mlp_off;          // word offset of the network's scratch from the warp's base
    int learn_depth;      // rows of level < learn_depth are ordered by the network
    CoopShared *coop;     // host heuristic threads' exchange (NULL: none)
    CoopSlot *coop_slots; // [K] the explorers' snapshot slots
    int minht;            // 1: LB1 with the heads and tails refinement (its own kernel)
    int diag;             // 1: phase timers or a trace requested (the kernel that carries them)
    int rows_smem;        // 1: each explorer's rows live in shared memory after its explorer state
    int wait_limit;       // polls of a thief's answer wait (0: kWaitLimit; lowered only by a test hook)
};

// Words of one explorer's rows in shared memory: bounds [n][n] int32, then
// jobs [n][n] uint8; a multiple of 8 words.
__host__ __device__ inline int solve_row_words(int n) { return ((n * n + (n * n + 3) / 4) + 7) & ~7; }

int solve_warp_words(int n, int m, int bound);
// Network scratch placement for a learned solve: sets *off (words from the
// warp base) and returns the extra words to add to the per-warp stride.
int mlp_scratch_place(int n, int m, int bound, int D0, int *off);
int solve_occupancy(const SolveArgs &a, int warps, size_t smem);
cudaError_t launch_solve(const SolveArgs &a, int blocks, int warps, size_t smem, cudaStream_t st);
// The same for the kernels with the ordering network (solve_learned.cu).
int solve_occupancy_learned(const SolveArgs &a, int warps, size_t smem);
cudaError_t launch_solve_learned(const SolveArgs &a, int blocks, int warps, size_t smem, cudaStream_t st);
int solve_occupancy_coop(const SolveArgs &a, int warps, size_t smem);
cudaError_t launch_solve_coop(const SolveArgs &a, int blocks, int warps, size_t smem, cudaStream_t st);
int solve_occupancy_ee(const SolveArgs &a, int warps, size_t smem);
cudaError_t launch_solve_ee(const SolveArgs &a, int blocks, int warps, size_t smem, cudaStream_t st);
int solve_occupancy_diag(const SolveArgs &a, int warps, size_t smem);
cudaError_t launch_solve_diag(const SolveArgs &a, int blocks, int warps, size_t smem, cudaStream_t st);
int solve_occupancy_minht(const SolveArgs &a, int warps, size_t smem);
cudaError_t launch_solve_minht(const SolveArgs &a, int blocks, int warps, size_t smem, cudaStream_t st);

}  // namespace pfsp
