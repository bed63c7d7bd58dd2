/*
 * pfsp.h -- C ABI of the GB300 (sm_103a) permutation flow-shop branch-and-bound
 * library: batched lower bounds for the children of many partial schedules,
 * and a device-resident depth-first explorer pool that solves instances.
 *
 * Problem (Gmys, arXiv 2012.09511, Section 2.1): n jobs, m machines, integer
 * processing times p[j][k]; find a permutation minimising the completion time
 * of the last job on the last machine (Eq. 1 gives the completion times).
 *
 * General rules of every call:
 *   - Every function returns PFSP_OK (0) or a negative PFSP_ERR_* code; on an
 *     error nothing is written to the outputs and pfsp_last_error() holds a
 *     one-line message for the calling thread.
 *   - Host-pointer functions are synchronous: they return after the results
 *     are in the caller's buffers.  Buffers are owned by the caller and only
 *     read or written during the call.
 *   - Functions with the _dev suffix take device pointers and a CUDA stream
 *     (cudaStream_t passed as void*, NULL = legacy default stream); they only
 *     enqueue work and return.  The caller keeps the buffers alive until the
 *     stream has passed the work.
 *   - Jobs and machines are numbered from 0.  p is job-major: p[j*m + k].
 *   - Limits: 1 <= n <= 64, 1 <= m <= 32, 0 <= p[j][k] < 2^22 and the sum of
 *     all p[j][k] below 2^28 (all bound arithmetic is int32 and exact);
 *     otherwise PFSP_ERR_UNSUPPORTED.  LB2 also needs its per-pair tables to
 *     fit in shared memory (m(m-1)/2 pairs x n jobs x 8 bytes <= 160 KiB).
 *   - All calls act on the CUDA device that is current in the calling thread
 *     when pfsp_load_instance runs; the instance lives on that device.
 */
#ifndef PFSP_H
#define PFSP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Return codes. */
#define PFSP_OK 0
#define PFSP_ERR_INVALID (-1)      /* bad argument: NULL pointer, size, depth, negative time */
#define PFSP_ERR_OOM (-2)          /* device or host allocation failed */
#define PFSP_ERR_CUDA (-3)         /* a CUDA runtime call failed (message has the CUDA error) */
#define PFSP_ERR_UNSUPPORTED (-4)  /* outside the limits above */
#define PFSP_ERR_TIMEOUT (-5)      /* a bounded device-side wait gave up; the context stays usable */

/* Outcome of a solve (not an error). */
#define PFSP_OPTIMAL 0             /* search finished; best_cmax is optimal */
#define PFSP_PROVEN_NO_BETTER 1    /* search finished; no schedule below init_ub exists */
#define PFSP_LIMIT_NODES 2         /* stopped at node_limit; best_cmax is the best found */
#define PFSP_LIMIT_TIME 3          /* stopped at time_limit_s; best_cmax is the best found */

/* Bound kinds (bit mask for pfsp_bound_batch; a single value for solves). */
#define PFSP_LB1 1   /* one-machine bound, Section 2.4 steps 1-4 */
#define PFSP_LB2 2   /* two-machine Johnson bound over all m(m-1)/2 machine pairs, Section 2.4 */
#define PFSP_MINHT 4 /* with LB1 or LB2: raise the front of an empty sigma1 (back of an empty sigma2)
                        to the least work of an unscheduled job on the machines before (after) each
                        machine -- the heads and tails refinement of LB1, not in the paper, off by
                        default; LB2 is then the larger of that LB1 and the pair values */

/* Dynamic branching rules: MinMin (Section 2.3) and its capped variant, and
 * readings of MinBranch and MinSum, which Table 4 names for earlier solvers
 * without defining them.  Every rule compares the two children sets of a
 * node; a tie goes to the set with the larger sum of bounds, then forward. */
#define PFSP_MINMIN 0          /* the paper's rule on the exact bounds of all children: the set
                                  where the smallest bound of both sets occurs less often */
#define PFSP_MINMIN_CAPPED 1   /* the same rule on min(bound, incumbent) */
#define PFSP_MINBRANCH 2       /* the set with fewer children below the solve's initial incumbent
                                  (fewer subproblems to explore) */
#define PFSP_MINSUM 3          /* the set whose children leave the smaller total gap sum(c - LB) to
                                  the incumbent c: with as many children in both sets, the set with
                                  the larger sum of bounds */

typedef struct pfsp_instance pfsp_instance; /* opaque, owned by the library */

/*
 * Load an instance (Section 2.1): copies p (n*m int32, job-major) and builds
 * the device tables used by the bounds: processing times by machine, the
 * per-machine totals, and for every machine pair k < l the Johnson order of
 * the jobs on (p[j][k] + g_j, p[j][l] + g_j) with lag g_j the sum of job j's
 * times on the machines strictly between k and l (Section 2.4, LB2 with
 * pre-sorted Johnson schedules).  *out receives the new instance.
 * Errors: PFSP_ERR_INVALID (NULL, n < 1, m < 1, negative time),
 * PFSP_ERR_UNSUPPORTED (limits), PFSP_ERR_OOM, PFSP_ERR_CUDA.
 */
int pfsp_load_instance(int n, int m, const int32_t *p, pfsp_instance **out);

/* Release an instance and every device buffer it holds.  NULL is ignored. */
void pfsp_free_instance(pfsp_instance *inst);

/*
 * Bounds of both children sets of num_nodes partial schedules (Sections 2.3
 * and 2.4).  Node i is perm[i*n .. i*n+n-1] (a permutation of 0..n-1) with
 * depths d1[i], d2[i], d1 + d2 <= n: positions [0, d1) hold sigma1 in order,
 * positions [n-d2, n) hold sigma2 in order, the rest are unscheduled.
 * For every unscheduled job j the forward child is (sigma1 j, sigma2) and the
 * backward child is (sigma1, j sigma2).  Outputs are int32 arrays of
 * num_nodes*2*n entries laid out [node][dir][job] (dir 0 = forward,
 * 1 = backward); entries of scheduled jobs are -1.  kind is a bit mask of
 * PFSP_LB1 | PFSP_LB2, optionally with PFSP_MINHT (a separate, generic
 * kernel); the output of a kind not requested may be NULL and is not
 * touched.  With m = 1 there is no machine pair and LB2 equals LB1.
 * Bounds are exact int32 values, identical to their definitions.
 * num_nodes = 0 is allowed and does nothing.
 * Errors: PFSP_ERR_INVALID (NULL pointer for a requested output or input,
 * d1 + d2 > n, kind without LB1 or LB2 or with other bits),
 * PFSP_ERR_UNSUPPORTED (LB2 tables too large),
 * PFSP_ERR_OOM, PFSP_ERR_CUDA.  On an error the outputs are not written
 * (the depths are validated while the first chunks of the batch are bounded
 * on the device, and results are copied back only after that).
 */
int pfsp_bound_batch(const pfsp_instance *inst, int kind, int64_t num_nodes, const uint8_t *perm,
                     const uint8_t *d1, const uint8_t *d2, int32_t *lb1_out, int32_t *lb2_out);

/* (pfsp_bound_batch moves the batch in chunks of 262,144 nodes over two CUDA
 * streams, so that the copies of one chunk overlap the kernel of another; the
 * overlap is complete with page-locked host buffers.  When both requested
 * outputs are page-locked memory that the GPU maps, the chunks after the
 * first two are written in place by the kernel over the host link, so that
 * no copy is left after the last kernel; the first two, like every chunk of
 * pageable outputs, go through device buffers, and nothing reaches the
 * outputs before the depths are validated.  The same holds for the summaries
 * of pfsp_bound_reduce.) */

/* Same as pfsp_bound_batch on device buffers, enqueued on `stream`.  Depths
 * are not validated on the device beyond clamping (a node with d1 + d2 > n
 * gets all -1 outputs); the host variant validates them. */
int pfsp_bound_batch_dev(const pfsp_instance *inst, int kind, int64_t num_nodes, const uint8_t *perm,
                         const uint8_t *d1, const uint8_t *d2, int32_t *lb1_out, int32_t *lb2_out,
                         void *stream);

/*
 * Per-parent summary of the bounds of its children (Sections 2.3-2.4): what
 * the branching rule and the pruning consume, without the 2n bounds each.
 * Index 0 is the forward children set, 1 the backward one.
 */
typedef struct {
    int32_t min[2];    /* least bound of the set (INT32_MAX when the node has no child; -1 for
                          invalid depths on the device entry point) */
    int32_t count[2];  /* children of the set at that least bound (-1 for invalid depths) */
    int64_t sum[2];    /* sum of the set's bounds */
    uint64_t keep[2];  /* bit j: the child of job j has a bound below ub (it survives pruning) */
} pfsp_node_summary;

/*
 * Bounding with the children reduced per parent (the "reduce" mode; the
 * arrays of pfsp_bound_batch are the "materialize" mode): the same nodes,
 * layout and validation as pfsp_bound_batch; kind is PFSP_LB1 or PFSP_LB2
 * (one bound: the one summarised).  ub is the exclusive incumbent that keep
 * tests against.  out (num_nodes entries) receives one summary per node.
 * MinMin's count of the overall least bound mu is count[d] where min[d] == mu
 * and 0 elsewhere.  Returns the codes of pfsp_bound_batch.
 */
int pfsp_bound_reduce(const pfsp_instance *inst, int kind, int64_t num_nodes, const uint8_t *perm,
                      const uint8_t *d1, const uint8_t *d2, int32_t ub, pfsp_node_summary *out);

/* Same on device buffers, enqueued on `stream` (depths clamped as in
 * pfsp_bound_batch_dev; invalid ones get min = count = -1). */
int pfsp_bound_reduce_dev(const pfsp_instance *inst, int kind, int64_t num_nodes, const uint8_t *perm,
                          const uint8_t *d1, const uint8_t *d2, int32_t ub, pfsp_node_summary *out,
                          void *stream);

/* Counters reported by pfsp_stats, pfsp_solve_batch and pfsp_solve_noalloc. */
typedef struct {
    uint64_t decomposed;       /* parents whose children were bounded (root counts 1) */
    uint64_t bounded_children; /* children bounded: sum of 2(n - d1 - d2) over parents */
    uint64_t leaves;           /* complete schedules evaluated */
    uint64_t pruned;           /* children of the chosen direction discarded (bound >= incumbent) */
    uint64_t steals;           /* successful device work-stealing operations */
    uint64_t iterations;       /* explorer loop iterations summed over explorers */
    double seconds;            /* wall time of the call (host clock) */
    double kernel_seconds;     /* device time of the main kernel (CUDA events) */
    int32_t final_ub;          /* incumbent at the end of a solve */
    int32_t explorers;         /* explorers used by a solve */
    /* pfsp_solve with pfsp_options.phase_timers only (zero elsewhere): SM clock
     * cycles spent by the explorers in each phase of their loop, summed over
     * explorers: [0] limit checks and
     * answering steal requests, [1] selecting the next node, [2] decoding it,
     * [3] LB1 (wavefronts and children), [4] the LB2 sweep, [5] MinMin,
     * pruning and the new row, [6] rebuilding the path to a stolen interval's
     * start, [7] stealing and waiting without work. */
    uint64_t phase_cycles[8];
    /* pfsp_solve only: 32-pair slots swept by LB2, summed over decompositions
     * (fewer than decomposed x ceil(m(m-1)/2 / 32) with PFSP_EARLY_EXIT). */
    uint64_t lb2_slots;
    /* pfsp_solve with heuristic_threads only: times the host threads lowered
     * the incumbent, explorer nodes promoted to complete schedules, the best
     * makespan the threads found below the initial incumbent (INT32_MAX:
     * none), and the snapshot rounds the explorers answered. */
    uint64_t heuristic_improvements;
    uint64_t promoted;
    int32_t heuristic_cmax;
    int32_t snapshots;
} pfsp_stats_t;

/*
 * Options of a solve.  Call pfsp_default_options first, then change fields.
 *   init_ub      exclusive incumbent: only schedules with makespan < init_ub
 *                are sought (the paper initialises it at the optimum plus one
 *                or at a known value, Section 5); INT32_MAX (default) starts
 *                from the NEH schedule's makespan.  With init_ub equal to the
 *                optimum, the search proves that nothing better exists and
 *                the decomposed-node count is that of the fixed critical tree.
 *   node_limit   stop after about this many counted decompositions (checked
 *                every check_every iterations per explorer); 0 = no limit.
 *   time_limit_s stop after this many seconds of device time; 0 = no limit.
 *   bound        PFSP_LB1 or PFSP_LB2 (Section 2.4).
 *   branching    PFSP_MINMIN (default), PFSP_MINMIN_CAPPED (the MinMin rule
 *                on min(bound, c) with c the solve's initial incumbent, a
 *                constant, so that every node's decision is fixed for the
 *                run), PFSP_MINBRANCH or PFSP_MINSUM.  MinBranch counts the
 *                children below that same constant c: the explorers'
 *                intervals number the leaves of one fixed tree (Section
 *                2.6), so no decision may depend on the incumbent as it
 *                improves.  PFSP_EARLY_EXIT is refused with PFSP_MINSUM (the
 *                skipped sweep could change its decision).
 *   warps_per_sm explorers per SM; 0 = as many as fit in shared memory (at
 *                most 12).
 *   check_every  iterations between limit checks and length publications
 *                (rounded up to a power of two); 0 = default (8).
 *   min_steal    smallest remaining interval (in leaves) a victim splits;
 *                0 = default: pfsp_solve and pfsp_solve_noalloc take the
 *                leaves of a subtree with min(floor(2n/5), 9) jobs left (8!
 *                at n = 20), pfsp_solve_batch takes 2 (any splittable
 *                interval; pfsp_autotune_batch chooses between 2 and 8!).
 */
typedef struct pfsp_mlp pfsp_mlp; /* ordering network, see pfsp_mlp_create */

/* Learned-ordering flags (pfsp_options.learned; not in the paper). */
#define PFSP_LEARN_CHILD_ORDER 1  /* order each new row by the network's descend-first logits */
#define PFSP_LEARN_PAIR_ORDER 2   /* sweep LB2's 32-pair slots in the order of the network's pair logits */
#define PFSP_EARLY_EXIT 4         /* skip the LB2 sweep of a node when every child of one direction
                                     has an LB1 at least the incumbent c (the incumbent the explorer
                                     read for this node, never above the initial one and equal to it
                                     in proof mode; under PFSP_MINBRANCH the initial one): such a node
                                     has no child below the incumbent under either MinMin rule (the
                                     decided direction holds no minimum below it, so MinMin picks
                                     it) nor under MinBranch (it has no child below the incumbent, so
                                     MinBranch picks it unless the other direction has none either),
                                     hence the search tree and every counter are those of the full
                                     sweep; refused with PFSP_MINSUM */
#define PFSP_EARLY_EXIT_SLOTS 8   /* with PFSP_EARLY_EXIT: also stop the sweep after the first
                                     32-pair slot at which every child of one direction has a pair
                                     term at least the incumbent (same exactness argument); pairs in
                                     the instance's order (pfsp_learn_pair_order puts the pairs most
                                     likely to decide first). */
#define PFSP_EARLY_EXIT_CHILDREN 16 /* with PFSP_EARLY_EXIT: the sweep evaluates only the jobs one of
                                     whose children has an LB1 below the incumbent c of
                                     PFSP_EARLY_EXIT; a child left out keeps its LB1, a lower bound of
                                     its LB2 that is at least c.  It is pruned as with the full
                                     sweep, and in proof mode (c fixed at the initial incumbent)
                                     min(bound, c) is unchanged, so under PFSP_MINMIN_CAPPED the
                                     search tree and every counter are those of the full sweep.
                                     Under PFSP_MINMIN and PFSP_MINBRANCH the sums of bounds that
                                     break ties may differ, so trees may differ too; pruning and the
                                     optimum stay exact (not in the paper) */

typedef struct {
    int32_t init_ub;
    int64_t node_limit;
    double time_limit_s;
    int bound;
    int branching;
    int warps_per_sm;
    int check_every;
    double min_steal;
    const pfsp_mlp *mlp;  /* network used by the PFSP_LEARN_* flags (built for the instance's m) */
    int learned;          /* PFSP_LEARN_* / PFSP_EARLY_EXIT bits; 0 = plain solver */
    int learn_depth;      /* the network orders rows of level < learn_depth only (0 = every level) */
    int phase_timers;     /* 1: fill pfsp_stats_t.phase_cycles (reads the SM clock at every phase
                             boundary, which slows the solve down several times: for relative
                             profiling only; runs in a kernel instantiation of its own, not
                             beside heuristic threads); 0 (default): off */
    int heuristic_threads; /* pfsp_solve / pfsp_solve_resumable: host threads running the iterated
                              greedy beside the explorer pool (Section 4.2's heuristic threads);
                              0 (default): none.  Their improved schedules lower the explorers'
                              incumbent, so node counts then vary from run to run: a
                              finding-mode option.  The optimum found stays exact. */
    int heuristic_seed;   /* seed of the heuristic threads' random choices */
    int lb1_minht;        /* 1: LB1 (and the LB1 inside LB2) with the heads and tails refinement of
                             PFSP_MINHT; pfsp_solve / pfsp_solve_resumable with the plain solver
                             only (no heuristic threads, no ordering network); 0 (default): off */
    int heuristic_kind;   /* search of the heuristic threads: 0 (default) the iterated greedy
                             (pfsp_iterated_greedy) from the promoted schedules, 1 beam search
                             (pfsp_beam_search) below the promoted explorer nodes with their
                             prefix and suffix fixed, widths 1, 2, 4, ... 256, 2 both (odd
                             threads beam search) */
    int slot_warps;       /* pfsp_solve_batch only: explorers per instance slot.  A slot is one CTA
                             that claims an instance and explores it with its warps (then joins
                             the busiest running instance); with warps_per_sm explorers per SM,
                             warps_per_sm / slot_warps slots run on each SM, so this sets how many
                             instances are in flight at once.  0 (default): one slot per SM of
                             warps_per_sm explorers (12 when that is 0 too) */
    int reserved[2];
} pfsp_options;

void pfsp_default_options(pfsp_options *opt);

/*
 * Solve an instance with the device-resident pool of depth-first explorers
 * (Sections 2.2-3.4): dynamic branching with MinMin, pruning of children whose
 * bound is not below the incumbent, interval work stealing on the device.
 * Writes the best makespan found (or init_ub when nothing better exists) to
 * *best_cmax, a permutation reaching it to best_perm (n int32 job ids; may be
 * NULL; untouched when *outcome is PFSP_PROVEN_NO_BETTER), and the outcome
 * code (PFSP_OPTIMAL, PFSP_PROVEN_NO_BETTER, PFSP_LIMIT_NODES,
 * PFSP_LIMIT_TIME) to *outcome.  pfsp_stats then reports the counters.
 * Errors: PFSP_ERR_INVALID, PFSP_ERR_UNSUPPORTED, PFSP_ERR_OOM, PFSP_ERR_CUDA,
 * PFSP_ERR_TIMEOUT (a bounded device-side wait expired; no result).
 */
int pfsp_solve(const pfsp_instance *inst, const pfsp_options *opt, int32_t *best_cmax, int32_t *best_perm,
               int *outcome);

/*
 * pfsp_solve in resumable segments: the checkpoint of the paper's coordinator
 * (Section 4.1, a file of the unexplored intervals plus the best solution,
 * read back on restart), here for the explorer pool of one GPU.
 *   resume       NULL: search the whole tree; else a checkpoint written by an
 *                earlier call on this instance with the same bound and
 *                branching options (resume_bytes its size): the search covers
 *                exactly the intervals it holds, from its incumbent (opt->init_ub
 *                is ignored) and with its cap (the first segment's initial
 *                incumbent, used by PFSP_MINMIN_CAPPED and PFSP_EARLY_EXIT).
 *   checkpoint   NULL: nothing is recorded.  Else, when the call stops at
 *                node_limit or time_limit_s, *checkpoint receives a buffer
 *                allocated by the library (free it with pfsp_free_checkpoint)
 *                and *checkpoint_bytes its size: the incumbent, a schedule
 *                reaching it (when one is known) and, for every explorer with
 *                work left, the rest of its interval and the level of the next
 *                node it would have decomposed.  When the search finishes,
 *                *checkpoint is NULL and *checkpoint_bytes 0.
 * Every node is decomposed in exactly one segment: in proof mode the counters
 * of the segments add up to those of one uninterrupted pfsp_solve.  The buffer
 * is plain bytes and can be written to a file; it is only valid for a launch
 * with at least as many explorers as records (the same device and options).
 * Errors: those of pfsp_solve; PFSP_ERR_INVALID for a malformed or foreign
 * checkpoint; PFSP_ERR_UNSUPPORTED when it holds more intervals than the
 * launch has explorers.
 */
int pfsp_solve_resumable(const pfsp_instance *inst, const pfsp_options *opt, const uint8_t *resume,
                         int64_t resume_bytes, uint8_t **checkpoint, int64_t *checkpoint_bytes, int32_t *best_cmax,
                         int32_t *best_perm, int *outcome);
/* Release a checkpoint returned by pfsp_solve_resumable.  NULL is ignored. */
void pfsp_free_checkpoint(uint8_t *checkpoint);

/*
 * Solve `count` independent instances (any mix of n and m, all loaded on the
 * current device) in one persistent launch of the explorer pool, recorded in
 * a CUDA graph and launched from it.  Batching is not in the paper; each
 * instance is solved exactly as pfsp_solve would (same bounds, MinMin,
 * pruning, work stealing among the explorers working on that instance).
 * Every CTA first takes the next unclaimed instance; when none is left, CTAs
 * that finish join the running instance with the most busy explorers.
 *   init_ubs    count exclusive incumbents, or NULL (NEH for every instance;
 *               an entry INT32_MAX also means NEH).
 *   best_cmax   count outputs; outcomes: count outcome codes.
 *   best_perms  NULL or count rows of 64 int32: row i holds instance i's best
 *               permutation in its first n_i entries (-1 elsewhere, and -1
 *               throughout when the outcome is PFSP_PROVEN_NO_BETTER).
 *   stats       NULL or the counters summed over the batch.
 * node_limit applies to each instance; time_limit_s to the whole launch.
 * Errors: as pfsp_solve; PFSP_ERR_INVALID also for an instance on another
 * device.
 */
int pfsp_solve_batch(const pfsp_instance *const *insts, int count, const pfsp_options *opt,
                     const int32_t *init_ubs, int32_t *best_cmax, int32_t *best_perms, int *outcomes,
                     pfsp_stats_t *stats);

/*
 * Autotuner of the batched pool (not in the paper): runs pfsp_solve_batch on
 * `sample` instances spread evenly over the batch (every (count / sample)-th;
 * 0 = up to 32) for each point of a small grid of launch parameters --
 * explorers per SM {8, 12}, explorers per instance slot {4, 6, 12} (at most
 * the explorers per SM), iterations between limit checks and length
 * publications {8, 32}, smallest interval a victim splits {2, 8!} -- and
 * writes to *best the options (base plus the fastest point by device time,
 * the better of two timings each).  The children handled per warp are not a
 * parameter: a warp always bounds every child of the node it decomposes.
 */
int pfsp_autotune_batch(const pfsp_instance *const *insts, int count, const pfsp_options *base, int sample,
                        pfsp_options *best);

/*
 * Order of the machine pairs in the LB2 sweep (not in the paper; LB2 of
 * Section 2.4 is the maximum over all pairs, so no bound value depends on it).
 * order[i] (i = 0 .. m(m-1)/2 - 1) is the index of the pair placed at sweep
 * position i, pairs being indexed k = 0..m-2, l = k+1..m-1 (the network's
 * column order); positions 0..31 form the first 32-pair slot, and so on.  The
 * order matters only to PFSP_EARLY_EXIT_SLOTS, which can stop after a slot.
 * Every pair is used (this also undoes pfsp_set_lb2_pairs).  order NULL
 * restores the index order.  The instance's device tables are rebuilt (the
 * call synchronises the device first; no call using the instance may run
 * meanwhile).
 * Errors: PFSP_ERR_INVALID (NULL instance, order not a permutation),
 * PFSP_ERR_CUDA.
 */
int pfsp_set_pair_order(pfsp_instance *inst, const int32_t *order);
/*
 * LB2 over a subset of the machine pairs: Section 2.4 notes that the bound
 * can use anything between m and all m(m-1)/2 pairs (for instance the m - 1
 * adjacent pairs (k, k+1), whose indices are k (2m - k - 1) / 2).  After this
 * call LB2 of the instance (bounding and solves alike) is the largest of LB1
 * and the values of the `count` pairs listed (distinct indices in the order
 * of pfsp_set_pair_order), swept in that order.  It is a weaker but valid
 * lower bound, so solves stay exact; their trees differ from the full LB2's.
 * pairs NULL restores all pairs in index order.  Same synchronisation as
 * pfsp_set_pair_order.
 * Errors: PFSP_ERR_INVALID (NULL instance, m = 1, count outside 1..m(m-1)/2,
 * repeated or out-of-range index), PFSP_ERR_CUDA.
 */
int pfsp_set_lb2_pairs(pfsp_instance *inst, const int32_t *pairs, int count);
/* The pairs LB2 uses, in sweep order, in the first entries of `order`
 * (m(m-1)/2 int32); entries past the pairs in use are -1. */
int pfsp_get_pair_order(const pfsp_instance *inst, int32_t *order);

/*
 * Test hook (no counterpart in the paper): the number of polls a thief makes
 * while it waits for a victim's answer in pfsp_solve and pfsp_solve_resumable
 * (the steal handshake of Section 3.4; each poll also answers requests sent to
 * the waiting thief and sleeps about 200 ns).  0 restores the default
 * (2^21 polls, about half a second).  When a wait runs out, the kernel records
 * the error, stops every explorer and the call returns PFSP_ERR_TIMEOUT with
 * nothing written; the context stays usable.  A small limit makes that
 * happen on purpose, so that callers can test their handling of the error.
 * Process-wide; read when a solve starts.  Errors: PFSP_ERR_INVALID
 * (polls < 0).
 */
int pfsp_set_steal_wait_limit(int polls);

/* Counters of the last pfsp_bound_batch or pfsp_solve call on `inst`. */
int pfsp_stats(const pfsp_instance *inst, pfsp_stats_t *out);

/*
 * pfsp_solve for callers that cannot allocate device memory (the paper has no
 * counterpart; this is a deployment variant).  It solves the instance given
 * directly by n, m and p (same layout and limits as pfsp_load_instance) with
 * the same options, outcomes and counters as pfsp_solve, but calls no
 * cudaMalloc or cudaFree: its device scratch -- the instance tables and the
 * explorer pool -- is one static 8 MiB array per device, created when the
 * library loads and kept until the process exits.  Use it where allocating is
 * not allowed: a service that reserves its memory at start-up, an application
 * whose device memory belongs to another allocator, or a caller that cannot
 * afford the device synchronisation an allocation implies.
 *   - Every call looks up the array's device address on the current device
 *     (a query that allocates nothing); the first call on a device also loads
 *     the library's module there, and the array with it, so make that first
 *     call before any stream capture begins.
 *   - Every call shares the array and overwrites what the previous call left;
 *     calls that overlap on the GPU (other threads or streams) race and must
 *     be serialised by the caller.
 *   - The pool takes as many explorers per SM as fit in the array beside the
 *     tables (the largest pool first, down to one explorer per SM); only when
 *     the tables plus a one-explorer-per-SM pool exceed 8 MiB does the call
 *     fail with PFSP_ERR_UNSUPPORTED.  On a 152-SM GPU every instance the
 *     library accepts (n, m <= 64) fits: at n = 64 that pool takes 3.1 MB.
 *   - stats may be NULL; otherwise it receives the solve's counters.
 * Returns the same codes as pfsp_solve.
 */
int pfsp_solve_noalloc(int n, int m, const int32_t *p, const pfsp_options *opt, int32_t *best_cmax,
                       int32_t *best_perm, int *outcome, pfsp_stats_t *stats);

/*
 * pfsp_solve that also records every `stride`-th counted decomposition (per
 * explorer) into caller buffers: perm [capacity][n], d1 [capacity],
 * d2 [capacity] in the layout of pfsp_bound_batch; *count receives the number
 * of nodes recorded (at most capacity).  These are the solver's own traces
 * from which the ordering network's training rows are built.
 */
int pfsp_solve_trace(const pfsp_instance *inst, const pfsp_options *opt, int64_t capacity, int stride,
                     uint8_t *perm, uint8_t *d1, uint8_t *d2, int64_t *count, int32_t *best_cmax, int *outcome);

/*
 * Ordering network (not in the paper): a two-hidden-layer MLP (128 ReLU
 * units each, bf16 weights, fp32 accumulation, tensor-core kernels) that
 * reads a node's per-machine front, back and remaining work, each divided by
 * the instance's mean machine load (sum of p / m), and outputs one "descend
 * first" logit (column 0) and one logit per machine pair k < l (columns
 * 1..m(m-1)/2, in the order k = 0..m-2, l = k+1..m-1).  Inputs are padded to
 * D0 = 3m rounded up to 16 columns, outputs to O = 1 + m(m-1)/2 rounded up to
 * 16.  Parameters are one fp32 vector [W1 (D0 x 128) | b1 | W2 (128 x 128) |
 * b2 | W3 (128 x O) | b3], row-major.  2 <= m <= 20.
 */
/* New network for m machines, He-uniform weights from a SplitMix64 stream. */
int pfsp_mlp_create(int m, uint64_t seed, pfsp_mlp **out);
void pfsp_mlp_free(pfsp_mlp *mlp);
/* Input width, hidden width, output width, number of pairs, parameter count. */
int pfsp_mlp_shape(const pfsp_mlp *mlp, int *D0, int *H, int *O, int *P, int64_t *n_params);
int pfsp_mlp_get_params(const pfsp_mlp *mlp, float *out);
int pfsp_mlp_set_params(pfsp_mlp *mlp, const float *in);
/* Logits Y [rows][O] of inputs X [rows][D0] (host buffers). */
int pfsp_mlp_forward(const pfsp_mlp *mlp, int64_t rows, const float *X, float *Y);
/* Masked mean binary cross-entropy of logits against targets T with mask M
 * (both [rows][O]), and its gradient with respect to every parameter (host
 * buffer of n_params floats, parameter layout); the parameters are unchanged. */
int pfsp_mlp_loss_grad(const pfsp_mlp *mlp, int64_t rows, const float *X, const float *T, const float *M,
                       float *loss, float *grad);
/* Adam training (beta 0.9 / 0.999) on mini-batches of `batch` rows of a
 * SplitMix64-shuffled order per epoch; epoch_loss (NULL or epochs floats)
 * receives each epoch's mean batch loss. */
int pfsp_mlp_train(pfsp_mlp *mlp, int64_t rows, const float *X, const float *T, const float *M, int epochs,
                   int batch, float lr, uint64_t seed, float *epoch_loss);

/*
 * Training rows of the network from num_nodes nodes of `inst` (layout of
 * pfsp_bound_batch), computed on the GPU: per node 1 + 2n rows -- the parent
 * (features: front, back, remaining work per machine over the mean machine
 * load; targets on columns 1..P: the pair's two-machine term equals the LB2
 * of some child and exceeds its LB1), then the forward child of each job j
 * (row 1 + j) and the backward child (row 1 + n + j), whose column-0 target
 * is 1 for the child of least LB2 of its direction (ties: lowest job id).
 * X [rows][D0], T and M [rows][O] (host buffers, M = loss mask).
 */
int pfsp_mlp_rows(const pfsp_instance *inst, const pfsp_mlp *mlp, int64_t num_nodes, const uint8_t *perm,
                  const uint8_t *d1, const uint8_t *d2, float *X, float *T, float *M);

/*
 * Per-pair scores of the ordering network over num_nodes nodes of `inst`
 * (layout of pfsp_bound_batch), on the GPU: score[q] (q in the network's pair
 * order, m(m-1)/2 floats) is the mean over the nodes of the network's
 * probability that pair q gives the LB2 of a child, read from the parent
 * row's features.  num_nodes >= 1.
 */
int pfsp_mlp_pair_scores(const pfsp_instance *inst, const pfsp_mlp *mlp, int64_t num_nodes, const uint8_t *perm,
                         const uint8_t *d1, const uint8_t *d2, float *score);

/*
 * Learned pair order (not in the paper): pfsp_mlp_pair_scores over the given
 * nodes, pairs sorted by decreasing score (ties: lower index first), then
 * pfsp_set_pair_order.  order (NULL or m(m-1)/2 int32) receives the order.
 * The nodes are typically a short trace of the solver on this instance
 * (pfsp_solve_trace), so that the first 32-pair slot holds the pairs that
 * most often decide a child of the nodes the search visits.
 */
int pfsp_learn_pair_order(pfsp_instance *inst, const pfsp_mlp *mlp, int64_t num_nodes, const uint8_t *perm,
                          const uint8_t *d1, const uint8_t *d2, int32_t *order);

/*
 * Learned LB2 pair subset (not in the paper; an LB2 variant of Section 2.4):
 * the network's mean pair probability over the given nodes (perm NULL: the
 * 2n children of the root, job j first or last), and LB2 restricted to the
 * `keep` pairs of highest score through pfsp_set_lb2_pairs (all pairs when
 * keep >= m(m-1)/2).  With keep = 32 the sweep is a single 32-pair slot.  The
 * bound stays a valid lower bound, so solves stay exact.  pairs (NULL or
 * min(keep, m(m-1)/2) int32) receives the pairs kept, best first.
 */
int pfsp_learn_lb2_pairs(pfsp_instance *inst, const pfsp_mlp *mlp, int64_t num_nodes, const uint8_t *perm,
                         const uint8_t *d1, const uint8_t *d2, int keep, int32_t *pairs);

/*
 * Host heuristic (Section 4.2's heuristic threads run a local search from
 * diversified starting points; this is the search they run here): the
 * iterated greedy of Ruiz and Stuetzle (2007) on the instance p (n x m,
 * job-major, as pfsp_load_instance), from `start` (a permutation of 0..n-1,
 * or NULL: the NEH schedule), for `iterations` iterations with the random
 * choices of `seed` (the same inputs give the same result).  Each iteration
 * removes 4 random jobs, reinserts each at its best position, improves the
 * schedule by insertion local search and accepts it by a constant-temperature
 * annealing test.  best_perm (n int32) and *best_cmax receive the best
 * schedule seen, never worse than the start after its local search.  Host
 * code only: needs no GPU.
 * Errors: PFSP_ERR_INVALID (NULL output, n < 1, m < 1, iterations < 0, a
 * negative time, a start that is not a permutation), PFSP_ERR_UNSUPPORTED
 * (n > 64).
 */
int pfsp_iterated_greedy(const int32_t *p, int n, int m, const int32_t *start, int64_t iterations,
                         uint64_t seed, int32_t *best_perm, int32_t *best_cmax);

/*
 * Host beam search (the paper's heuristic threads also run the beam search of
 * Libralesso et al. on partial schedules of the exact search, prefix and
 * suffix unchanged, Section 4.2): from the node (prefix, suffix) of the
 * instance p (n x m, job-major), forward branching only, keeping at each
 * level the `width` partial schedules of least LB1 (Section 2.4; ties: the
 * smaller sum of the front on all machines, then generation order).  With a
 * width of at least the number of completions it enumerates them all and
 * returns the best.  best_perm (n int32, starting with prefix and ending with
 * suffix) and *best_cmax receive the best complete schedule found.  Host code
 * only: needs no GPU.
 * Errors: PFSP_ERR_INVALID (NULL output, n < 1, m < 1, width < 1, d1 + d2 > n,
 * prefix and suffix not distinct valid jobs, a negative time),
 * PFSP_ERR_UNSUPPORTED (n > 64).
 */
int pfsp_beam_search(const int32_t *p, int n, int m, const int32_t *prefix, int d1, const int32_t *suffix, int d2,
                     int width, int32_t *best_perm, int32_t *best_cmax);

/* Message of the last error in the calling thread ("" if none). */
const char *pfsp_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PFSP_H */
