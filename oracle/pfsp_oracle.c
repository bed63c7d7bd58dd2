/*
 * pfsp_oracle.c -- plain, sequential CPU oracle for the permutation flow-shop
 * branch-and-bound of Gmys, "Solving large permutation flow-shop scheduling
 * problems on GPU-accelerated supercomputers" (arXiv 2012.09511).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA path, and nothing in the product
 * calls it.
 *
 * Everything is int32 arithmetic (the paper's bounds are integer), written
 * straight from the definitions, one node and one child at a time, with no
 * incremental or algebraic shortcuts:
 *   - completion times: Eq. 1 (Section 2.1);
 *   - LB1: the four steps of Section 2.4 (front, remaining work, back,
 *     combination), with the back obtained by the reversibility property;
 *   - LB2: Section 2.4's two-machine bound over all m(m-1)/2 machine pairs,
 *     each pair solved by Johnson's rule extended to time lags (the reading
 *     of the silent passage is in the header of lb2_from_parts below), or
 *     over a given subset of the pairs (the paper's variants use between
 *     about m and m(m-1)/2 of them);
 *   - branching: forward/backward/dynamic branching and the MinMin rule of
 *     Section 2.3, and readings of the MinBranch and MinSum rules that
 *     Table 4 names;
 *   - search: depth-first (Section 2.5) with pruning of children whose bound
 *     is not below the incumbent;
 *   - factorial number system of Section 2.6;
 *   - brute force over n!, Johnson's rule for m = 2, and the NEH heuristic
 *     (not in the paper; used for the initial upper bound).
 *
 * Conventions: p is job-major, p[j*m + k] = time of job j on machine k,
 * jobs and machines 0-based.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_FWD 0
#define ORC_BWD 1
#define ORC_LB1 1
#define ORC_LB2 2
#define ORC_MINHT 4  /* kind / bound bit: the heads and tails refinement (refine_heads_tails) */

#define ORC_OPTIMAL 0
#define ORC_PROVEN_NO_BETTER 1
#define ORC_LIMIT_NODES 2

#define ORC_MAXN 64

static int32_t imax(int32_t a, int32_t b) { return a > b ? a : b; }
static int32_t imin(int32_t a, int32_t b) { return a < b ? a : b; }

/* ------------------------------------------------------------------ */
/* Eq. 1 (Section 2.1): C[pi(i),k] = max(C[pi(i),k-1], C[pi(i-1),k]) + p */
/* ------------------------------------------------------------------ */

/* Completion times on every machine of the last job of `seq` (length len),
 * started on an empty shop; C[k] = 0 for all k when len = 0. */
void orc_completion(int m, const int32_t *p, const int32_t *seq, int len, int32_t *C)
{
    for (int k = 0; k < m; ++k) C[k] = 0;
    for (int i = 0; i < len; ++i) {
        int j = seq[i];
        int32_t left = 0; /* C of this job on machine k-1; 0 before machine 0 */
        for (int k = 0; k < m; ++k) {
            C[k] = imax(C[k], left) + p[j * m + k];
            left = C[k];
        }
    }
}

/* Makespan C_max(pi) = C[pi(n), m] of a full permutation (Section 2.1). */
int32_t orc_makespan(int n, int m, const int32_t *p, const int32_t *perm)
{
    int32_t C[ORC_MAXN];
    orc_completion(m, p, perm, n, C);
    return C[m - 1];
}

/* ------------------------------------------------------------------ */
/* LB1, Section 2.4, steps 1-4                                          */
/* ------------------------------------------------------------------ */

/* Step 1: front[k] = completion time of sigma1's last job on machine k. */
void orc_front(int m, const int32_t *p, const int32_t *sigma1, int d1, int32_t *front)
{
    orc_completion(m, p, sigma1, d1, front);
}

/* Step 3: back[k] = least time from the start of sigma2 on machine k to the
 * end of all operations.  By the reversibility property, this is Eq. 1
 * applied to sigma2 taken last-job-first on the machines taken last-first. */
void orc_back(int m, const int32_t *p, const int32_t *sigma2, int d2, int32_t *back)
{
    for (int k = 0; k < m; ++k) back[k] = 0;
    for (int i = d2 - 1; i >= 0; --i) {
        int j = sigma2[i];
        int32_t right = 0; /* reversed-shop completion on machine k+1 */
        for (int k = m - 1; k >= 0; --k) {
            back[k] = imax(back[k], right) + p[j * m + k];
            right = back[k];
        }
    }
}

/* Step 2: remain[k] = sum of p[j][k] over unscheduled jobs j. */
void orc_remain(int n, int m, const int32_t *p, const uint8_t *unscheduled, int32_t *remain)
{
    for (int k = 0; k < m; ++k) remain[k] = 0;
    for (int j = 0; j < n; ++j)
        if (unscheduled[j])
            for (int k = 0; k < m; ++k) remain[k] += p[j * m + k];
}

/* Step 4: LB1 = max_k front[k] + remain[k] + back[k]. */
int32_t orc_lb1_combine(int m, const int32_t *front, const int32_t *remain, const int32_t *back)
{
    int32_t v = front[0] + remain[0] + back[0];
    for (int k = 1; k < m; ++k) v = imax(v, front[k] + remain[k] + back[k]);
    return v;
}

/* Unscheduled-job indicator of the node (sigma1, sigma2). */
static void node_unscheduled(int n, const int32_t *s1, int d1, const int32_t *s2, int d2, uint8_t *un)
{
    for (int j = 0; j < n; ++j) un[j] = 1;
    for (int i = 0; i < d1; ++i) un[s1[i]] = 0;
    for (int i = 0; i < d2; ++i) un[s2[i]] = 0;
}

/* The heads and tails refinement of LB1 (not in the paper, which leaves the
 * front of an empty sigma1 and the back of an empty sigma2 at zero; an
 * option, off by default).  With sigma1 empty, an unscheduled job j cannot
 * start on machine k before its own work on machines 0..k-1 is done, so
 * front[k] is raised to the least such work over the unscheduled jobs; with
 * sigma2 empty, back[k] is raised to the least work on machines k+1..m-1.
 * A node without unscheduled jobs is a complete schedule: nothing changes. */
static void refine_heads_tails(int n, int m, const int32_t *p, const uint8_t *un, int d1, int d2,
                               int32_t *front, int32_t *back)
{
    int any = 0;
    for (int j = 0; j < n; ++j) any |= un[j];
    if (!any) return;
    for (int k = 0; k < m; ++k) {
        int32_t head = INT32_MAX, tail = INT32_MAX;
        for (int j = 0; j < n; ++j) {
            if (!un[j]) continue;
            int32_t h = 0, t = 0;
            for (int q = 0; q < k; ++q) h += p[j * m + q];
            for (int q = k + 1; q < m; ++q) t += p[j * m + q];
            head = imin(head, h);
            tail = imin(tail, t);
        }
        if (d1 == 0) front[k] = head;
        if (d2 == 0) back[k] = tail;
    }
}

int32_t orc_lb1_minht(int n, int m, const int32_t *p, const int32_t *s1, int d1, const int32_t *s2, int d2)
{
    int32_t f[ORC_MAXN], r[ORC_MAXN], b[ORC_MAXN];
    uint8_t un[ORC_MAXN];
    node_unscheduled(n, s1, d1, s2, d2, un);
    orc_front(m, p, s1, d1, f);
    orc_remain(n, m, p, un, r);
    orc_back(m, p, s2, d2, b);
    refine_heads_tails(n, m, p, un, d1, d2, f, b);
    return orc_lb1_combine(m, f, r, b);
}

int32_t orc_lb1(int n, int m, const int32_t *p, const int32_t *s1, int d1, const int32_t *s2, int d2)
{
    int32_t f[ORC_MAXN], r[ORC_MAXN], b[ORC_MAXN];
    uint8_t un[ORC_MAXN];
    node_unscheduled(n, s1, d1, s2, d2, un);
    orc_front(m, p, s1, d1, f);
    orc_remain(n, m, p, un, r);
    orc_back(m, p, s2, d2, b);
    return orc_lb1_combine(m, f, r, b);
}

/* ------------------------------------------------------------------ */
/* Johnson's rule and LB2                                               */
/* ------------------------------------------------------------------ */

/* Johnson's rule for two machines (Section 2.1 cites it as the O(n log n)
 * exact method for m = 2), extended to time lags (Mitten): with first-machine
 * times x_j, second-machine times y_j and lags g_j, jobs with x_j <= y_j come
 * first in ascending x_j + g_j, then the others in descending y_j + g_j.
 * Ties go to the lower job id.  Writes the sequence of all n jobs. */
typedef struct { int32_t key; int32_t grp; int32_t job; } orc_jkey;

static int cmp_jkey(const void *a, const void *b)
{
    const orc_jkey *x = (const orc_jkey *)a, *y = (const orc_jkey *)b;
    if (x->grp != y->grp) return x->grp - y->grp;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return x->job - y->job;
}

void orc_johnson_lag_order(int n, const int32_t *x, const int32_t *y, const int32_t *g, int32_t *order)
{
    orc_jkey keys[ORC_MAXN];
    for (int j = 0; j < n; ++j) {
        keys[j].job = j;
        if (x[j] <= y[j]) { keys[j].grp = 0; keys[j].key = x[j] + g[j]; }
        else { keys[j].grp = 1; keys[j].key = -(y[j] + g[j]); } /* descending */
    }
    qsort(keys, (size_t)n, sizeof(orc_jkey), cmp_jkey);
    for (int t = 0; t < n; ++t) order[t] = keys[t].job;
}

/* Optimal two-machine makespan by Johnson's rule (m must be 2). */
int32_t orc_johnson(int n, const int32_t *p, int32_t *order_out)
{
    int32_t x[ORC_MAXN], y[ORC_MAXN], g[ORC_MAXN], ord[ORC_MAXN];
    for (int j = 0; j < n; ++j) { x[j] = p[j * 2]; y[j] = p[j * 2 + 1]; g[j] = 0; }
    orc_johnson_lag_order(n, x, y, g, ord);
    if (order_out) memcpy(order_out, ord, sizeof(int32_t) * (size_t)n);
    return orc_makespan(n, 2, p, ord);
}

/* Per-instance LB2 tables: for every machine pair k < l, the lag
 * g_j = sum_{k<q<l} p[j][q] of each job and the Johnson order of all jobs on
 * (p[j][k] + g_j, p[j][l] + g_j).  The paper calls these pre-sorted Johnson
 * schedules (Section 2.4). */
typedef struct {
    int n, m, npairs;
    int subset;          /* 1: only some pairs are used (LB2 over a subset) */
    const int32_t *p;
    int32_t *pk, *pl;    /* [pair] machine indices */
    int32_t *lag;        /* [pair][job] */
    int32_t *order;      /* [pair][position] -> job */
} orc_tables;

static void tables_init(orc_tables *T, int n, int m, const int32_t *p)
{
    T->n = n; T->m = m; T->p = p;
    T->npairs = m * (m - 1) / 2;
    int P = T->npairs > 0 ? T->npairs : 1;
    T->pk = (int32_t *)malloc(sizeof(int32_t) * (size_t)P);
    T->pl = (int32_t *)malloc(sizeof(int32_t) * (size_t)P);
    T->lag = (int32_t *)malloc(sizeof(int32_t) * (size_t)P * (size_t)n);
    T->order = (int32_t *)malloc(sizeof(int32_t) * (size_t)P * (size_t)n);
    int q = 0;
    for (int k = 0; k < m; ++k)
        for (int l = k + 1; l < m; ++l, ++q) {
            int32_t x[ORC_MAXN], y[ORC_MAXN];
            T->pk[q] = k; T->pl[q] = l;
            for (int j = 0; j < n; ++j) {
                int32_t g = 0;
                for (int r = k + 1; r < l; ++r) g += p[j * m + r];
                T->lag[q * n + j] = g;
                x[j] = p[j * m + k];
                y[j] = p[j * m + l];
            }
            orc_johnson_lag_order(n, x, y, T->lag + (size_t)q * n, T->order + (size_t)q * n);
        }
}

static void tables_free(orc_tables *T)
{
    free(T->pk); free(T->pl); free(T->lag); free(T->order);
}

/* Keep only the pairs listed (indices in the k < l lexicographic order used
 * above), in that order.  pairs == NULL keeps every pair. */
static void tables_select(orc_tables *T, const int32_t *pairs, int count)
{
    if (!pairs) return;
    int n = T->n;
    int32_t *pk = (int32_t *)malloc(sizeof(int32_t) * (size_t)(count > 0 ? count : 1));
    int32_t *pl = (int32_t *)malloc(sizeof(int32_t) * (size_t)(count > 0 ? count : 1));
    int32_t *lag = (int32_t *)malloc(sizeof(int32_t) * (size_t)(count > 0 ? count : 1) * (size_t)n);
    int32_t *ord = (int32_t *)malloc(sizeof(int32_t) * (size_t)(count > 0 ? count : 1) * (size_t)n);
    for (int i = 0; i < count; ++i) {
        int q = pairs[i];
        pk[i] = T->pk[q];
        pl[i] = T->pl[q];
        memcpy(lag + (size_t)i * n, T->lag + (size_t)q * n, sizeof(int32_t) * (size_t)n);
        memcpy(ord + (size_t)i * n, T->order + (size_t)q * n, sizeof(int32_t) * (size_t)n);
    }
    tables_free(T);
    T->pk = pk; T->pl = pl; T->lag = lag; T->order = ord;
    T->npairs = count;
    T->subset = 1;
}

/* LB2 of a node given its front, back and unscheduled set (Section 2.4).
 * Reading of the silent passage: for every pair k < l, the unscheduled jobs
 * are run through the two-machine problem with time lags in Johnson order,
 * machine k free from front[k] and machine l from front[l]:
 *     t0 += p[j][k];   t1 = max(t1, t0 + g_j) + p[j][l];
 * and the pair's value adds the tails: max(t0 + back[k], t1 + back[l]).
 * LB2 is the largest pair value.  With a single machine there is no pair and
 * LB2 is defined equal to LB1.  Over a subset of the pairs (the paper's LB2
 * uses between m and m(m-1)/2 of them), LB2 is the largest of LB1 and the
 * values of the pairs kept. */
static int32_t lb2_from_parts(const orc_tables *T, const int32_t *front, const int32_t *back,
                              const uint8_t *un)
{
    int n = T->n, m = T->m;
    const int32_t *p = T->p;
    int32_t lb1 = 0;
    if (T->npairs == 0 || T->subset) {
        int32_t r[ORC_MAXN];
        orc_remain(n, m, p, un, r);
        lb1 = orc_lb1_combine(m, front, r, back);
        if (T->npairs == 0) return lb1;
    }
    int32_t best = T->subset ? lb1 : 0;
    for (int q = 0; q < T->npairs; ++q) {
        int k = T->pk[q], l = T->pl[q];
        int32_t t0 = front[k], t1 = front[l];
        const int32_t *ord = T->order + (size_t)q * n;
        const int32_t *lag = T->lag + (size_t)q * n;
        for (int t = 0; t < n; ++t) {
            int j = ord[t];
            if (!un[j]) continue;
            t0 += p[j * m + k];
            t1 = imax(t1, t0 + lag[j]) + p[j * m + l];
        }
        int32_t v = imax(t0 + back[k], t1 + back[l]);
        if ((q == 0 && !T->subset) || v > best) best = v;
    }
    return best;
}

int32_t orc_lb2(int n, int m, const int32_t *p, const int32_t *s1, int d1, const int32_t *s2, int d2)
{
    orc_tables T;
    int32_t f[ORC_MAXN], b[ORC_MAXN];
    uint8_t un[ORC_MAXN];
    tables_init(&T, n, m, p);
    node_unscheduled(n, s1, d1, s2, d2, un);
    orc_front(m, p, s1, d1, f);
    orc_back(m, p, s2, d2, b);
    int32_t v = lb2_from_parts(&T, f, b, un);
    tables_free(&T);
    return v;
}

/* Value of the two-machine relaxation of pair (k, l) for one given order of
 * the unscheduled jobs (used by the tests to brute-force the best order). */
int32_t orc_pair_value(int n, int m, const int32_t *p, int k, int l, const int32_t *front,
                       const int32_t *back, const int32_t *seq, int len)
{
    int32_t t0 = front[k], t1 = front[l];
    for (int i = 0; i < len; ++i) {
        int j = seq[i];
        int32_t g = 0;
        for (int r = k + 1; r < l; ++r) g += p[j * m + r];
        t0 += p[j * m + k];
        t1 = imax(t1, t0 + g) + p[j * m + l];
    }
    (void)n;
    return imax(t0 + back[k], t1 + back[l]);
}

/* ------------------------------------------------------------------ */
/* Children of a node and dynamic branching (Section 2.3)               */
/* ------------------------------------------------------------------ */

/* Bounds of both children sets of the node [perm, d1, d2] (positions [0,d1)
 * hold sigma1, [n-d2, n) hold sigma2).  Each child is bounded from scratch:
 * forward child of j is (sigma1 j, sigma2), backward child is (sigma1, j sigma2).
 * Output layout [dir][job]; scheduled jobs get -1.  kind is a bit mask of
 * ORC_LB1 / ORC_LB2 / ORC_MINHT; a NULL output is skipped.  With ORC_MINHT,
 * LB1 takes the refined heads and tails and LB2 is the larger of that LB1 and
 * the pair values (which keep the plain ones). */
static void children_bounds_t(const orc_tables *T, int kind, const uint8_t *perm, int d1, int d2,
                              int32_t *lb1, int32_t *lb2)
{
    int n = T->n, m = T->m;
    const int32_t *p = T->p;
    int32_t s1[ORC_MAXN + 1], s2[ORC_MAXN + 1];
    int32_t f[ORC_MAXN], b[ORC_MAXN], r[ORC_MAXN];
    uint8_t un[ORC_MAXN];
    for (int i = 0; i < 2 * n; ++i) {
        if (lb1) lb1[i] = -1;
        if (lb2) lb2[i] = -1;
    }
    for (int pos = d1; pos < n - d2; ++pos) {
        int j = perm[pos];
        for (int dir = 0; dir < 2; ++dir) {
            int c1 = d1, c2 = d2;
            for (int i = 0; i < d1; ++i) s1[i] = perm[i];
            if (dir == ORC_FWD) {
                s1[c1++] = j;
                for (int i = 0; i < d2; ++i) s2[i] = perm[n - d2 + i];
            } else {
                s2[0] = j;
                for (int i = 0; i < d2; ++i) s2[i + 1] = perm[n - d2 + i];
                c2 = d2 + 1;
            }
            node_unscheduled(n, s1, c1, s2, c2, un);
            orc_front(m, p, s1, c1, f);
            orc_back(m, p, s2, c2, b);
            if (kind & ORC_MINHT) {
                int32_t fr[ORC_MAXN], br[ORC_MAXN];
                for (int k = 0; k < m; ++k) { fr[k] = f[k]; br[k] = b[k]; }
                refine_heads_tails(n, m, p, un, c1, c2, fr, br);
                orc_remain(n, m, p, un, r);
                int32_t v1 = orc_lb1_combine(m, fr, r, br);
                if (lb1 && (kind & ORC_LB1)) lb1[dir * n + j] = v1;
                if (lb2 && (kind & ORC_LB2)) lb2[dir * n + j] = imax(lb2_from_parts(T, f, b, un), v1);
                continue;
            }
            if (lb1 && (kind & ORC_LB1)) {
                orc_remain(n, m, p, un, r);
                lb1[dir * n + j] = orc_lb1_combine(m, f, r, b);
            }
            if (lb2 && (kind & ORC_LB2)) lb2[dir * n + j] = lb2_from_parts(T, f, b, un);
        }
    }
}

void orc_children_bounds(int n, int m, const int32_t *p, int kind, const uint8_t *perm, int d1, int d2,
                         int32_t *lb1, int32_t *lb2)
{
    orc_tables T;
    tables_init(&T, n, m, p);
    children_bounds_t(&T, kind, perm, d1, d2, lb1, lb2);
    tables_free(&T);
}

typedef struct {
    const orc_tables *T;
    int kind;
    int64_t lo, hi;
    const uint8_t *perm, *d1, *d2;
    int32_t *lb1, *lb2;
} batch_job;

static void *batch_worker(void *arg)
{
    batch_job *J = (batch_job *)arg;
    int n = J->T->n;
    for (int64_t i = J->lo; i < J->hi; ++i)
        children_bounds_t(J->T, J->kind, J->perm + i * n, J->d1[i], J->d2[i],
                          J->lb1 ? J->lb1 + i * 2 * n : NULL, J->lb2 ? J->lb2 + i * 2 * n : NULL);
    return NULL;
}

/* Children bounds of `count` nodes; the nodes are independent, so they are
 * split into `threads` contiguous ranges run on plain pthreads. */
void orc_children_bounds_batch_pairs(int n, int m, const int32_t *p, int kind, int64_t count,
                                     const uint8_t *perm, const uint8_t *d1, const uint8_t *d2,
                                     int32_t *lb1, int32_t *lb2, int threads, const int32_t *pairs,
                                     int npairs)
{
    orc_tables T;
    tables_init(&T, n, m, p);
    tables_select(&T, pairs, npairs);
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    pthread_t tid[256];
    batch_job jobs[256];
    for (int t = 0; t < threads; ++t) {
        jobs[t].T = &T; jobs[t].kind = kind;
        jobs[t].lo = count * t / threads; jobs[t].hi = count * (t + 1) / threads;
        jobs[t].perm = perm; jobs[t].d1 = d1; jobs[t].d2 = d2;
        jobs[t].lb1 = lb1; jobs[t].lb2 = lb2;
    }
    for (int t = 1; t < threads; ++t) pthread_create(&tid[t], NULL, batch_worker, &jobs[t]);
    batch_worker(&jobs[0]);
    for (int t = 1; t < threads; ++t) pthread_join(tid[t], NULL);
    tables_free(&T);
}

void orc_children_bounds_batch(int n, int m, const int32_t *p, int kind, int64_t count,
                               const uint8_t *perm, const uint8_t *d1, const uint8_t *d2,
                               int32_t *lb1, int32_t *lb2, int threads)
{
    orc_children_bounds_batch_pairs(n, m, p, kind, count, perm, d1, d2, lb1, lb2, threads, NULL, 0);
}

/* MinMin (Section 2.3): among both children sets, find the smallest bound;
 * choose the set where it occurs less often; on a tie the set with the larger
 * sum of bounds; on a further tie, forward.  With cap < INT32_MAX every value
 * is first replaced by min(value, cap) (the capped variant, which needs only
 * the bounds below the incumbent to be exact).  Returns ORC_FWD or ORC_BWD. */
int orc_minmin(int n, const int32_t *lbf, const int32_t *lbb, const uint8_t *un, int32_t cap)
{
    int32_t mu = INT32_MAX;
    for (int j = 0; j < n; ++j)
        if (un[j]) mu = imin(mu, imin(imin(lbf[j], cap), imin(lbb[j], cap)));
    int cf = 0, cb = 0;
    int64_t sf = 0, sb = 0;
    for (int j = 0; j < n; ++j) {
        if (!un[j]) continue;
        int32_t vf = imin(lbf[j], cap), vb = imin(lbb[j], cap);
        cf += (vf == mu);
        cb += (vb == mu);
        sf += vf;
        sb += vb;
    }
    if (cf != cb) return cf < cb ? ORC_FWD : ORC_BWD;
    if (sf != sb) return sf > sb ? ORC_FWD : ORC_BWD;
    return ORC_FWD;
}

/* The other dynamic branching rules that Table 4 names for earlier solvers
 * of the same problem (the paper names them without defining them; these
 * are this oracle's readings):
 *   MinBranch: choose the set with fewer children whose bound is below c
 *     (fewer subproblems to explore); on a tie the set with the larger sum
 *     of bounds; on a further tie, forward.  c is the solve's initial
 *     incumbent, a constant like the capped MinMin's: the intervals of
 *     Section 2.6 number the leaves of one fixed tree, so a node's decision
 *     may not depend on the incumbent as it improves.
 *   MinSum: choose the set whose children leave the smaller total gap
 *     sum(ub - LB) to the incumbent.  Both sets hold the same children count,
 *     so this is the set with the larger sum of bounds; on a tie, forward.
 * rule: 0 MinMin, 1 MinMin on min(LB, cap), 2 MinBranch below cap, 3 MinSum. */
int orc_branch_rule(int n, const int32_t *lbf, const int32_t *lbb, const uint8_t *un, int rule,
                    int32_t cap)
{
    if (rule == 0) return orc_minmin(n, lbf, lbb, un, INT32_MAX);
    if (rule == 1) return orc_minmin(n, lbf, lbb, un, cap);
    int kf = 0, kb = 0;
    int64_t sf = 0, sb = 0;
    for (int j = 0; j < n; ++j) {
        if (!un[j]) continue;
        kf += lbf[j] < cap;
        kb += lbb[j] < cap;
        sf += lbf[j];
        sb += lbb[j];
    }
    if (rule == 2 && kf != kb) return kf < kb ? ORC_FWD : ORC_BWD;
    if (sf != sb) return sf > sb ? ORC_FWD : ORC_BWD;
    return ORC_FWD;
}

/* ------------------------------------------------------------------ */
/* Depth-first branch-and-bound (Sections 2.2-2.5)                      */
/* ------------------------------------------------------------------ */

typedef struct {
    orc_tables T;
    int bound;          /* ORC_LB1 or ORC_LB2, with ORC_MINHT for the refined heads and tails */
    int rule;           /* branching rule, as orc_branch_rule's */
    int32_t cap;        /* the run's initial incumbent */
    int32_t ub;         /* incumbent: only makespans < ub are sought */
    int32_t best_perm[ORC_MAXN];
    int found;
    int64_t node_limit;
    int aborted;
    int64_t decomposed, bounded, leaves, pruned;
} orc_bb;

/* Decompose the node whose layout is perm = [sigma1 | unscheduled ascending |
 * sigma2]; children are visited in ascending job order (the order of the
 * IVM rows, which copy the remaining jobs in order, Section 2.5). */
static void bb_dfs(orc_bb *S, const int32_t *perm, int d1, int d2)
{
    int n = S->T.n;
    if (S->aborted) return;
    if (S->node_limit > 0 && S->decomposed >= S->node_limit) { S->aborted = 1; return; }
    S->decomposed++;
    int u = n - d1 - d2;
    uint8_t p8[ORC_MAXN], un[ORC_MAXN];
    int32_t lb1[2 * ORC_MAXN], lb2[2 * ORC_MAXN];
    for (int i = 0; i < n; ++i) p8[i] = (uint8_t)perm[i];
    children_bounds_t(&S->T, S->bound, p8, d1, d2, lb1, lb2);
    const int32_t *lb = (S->bound & ORC_LB2) ? lb2 : lb1;
    S->bounded += 2 * u;
    if (u == 1) S->leaves += 2;
    for (int j = 0; j < n; ++j) un[j] = 0;
    for (int i = d1; i < n - d2; ++i) un[perm[i]] = 1;
    int dir = orc_branch_rule(n, lb, lb + n, un, S->rule, S->cap);
    const int32_t *lbd = lb + dir * n;

    /* prune at bounding time against the current incumbent */
    uint8_t keep[ORC_MAXN];
    for (int i = d1; i < n - d2; ++i) {
        int j = perm[i];
        keep[i] = lbd[j] < S->ub;
        if (!keep[i]) S->pruned++;
    }
    for (int i = d1; i < n - d2; ++i) {
        if (!keep[i]) continue;
        int j = perm[i];
        if (lbd[j] >= S->ub) continue; /* incumbent improved since bounding */
        int32_t child[ORC_MAXN];
        int c = 0;
        for (int t = 0; t < d1; ++t) child[c++] = perm[t];
        if (dir == ORC_FWD) child[c++] = j;
        for (int t = d1; t < n - d2; ++t)
            if (perm[t] != j) child[c++] = perm[t];
        if (dir == ORC_BWD) child[c++] = j;
        for (int t = n - d2; t < n; ++t) child[c++] = perm[t];
        if (u == 1) {
            /* the child is a complete schedule; its bound is its makespan */
            S->ub = lbd[j];
            memcpy(S->best_perm, child, sizeof(int32_t) * (size_t)n);
            S->found = 1;
            continue;
        }
        bb_dfs(S, child, d1 + (dir == ORC_FWD), d2 + (dir == ORC_BWD));
        if (S->aborted) return;
    }
}

int32_t orc_neh(int n, int m, const int32_t *p, int32_t *perm_out);

/* Solve from the root with branching rule `rule` (0 MinMin, 1 capped MinMin,
 * 2 MinBranch, 3 MinSum; see orc_branch_rule).  init_ub is exclusive (only
 * makespans < init_ub are sought); INT32_MAX means "start from the NEH
 * schedule".  Returns the
 * outcome code; counters[0..3] = decomposed, bounded, leaves, pruned. */
int orc_bb_solve_pairs(int n, int m, const int32_t *p, int bound, int rule, int32_t init_ub,
                       int64_t node_limit, int32_t *best_cmax, int32_t *best_perm, int64_t *counters,
                       const int32_t *pairs, int npairs)
{
    orc_bb *S = (orc_bb *)calloc(1, sizeof(orc_bb));
    tables_init(&S->T, n, m, p);
    tables_select(&S->T, pairs, npairs);
    S->bound = bound;
    S->rule = rule;
    S->node_limit = node_limit;
    int from_neh = 0;
    if (init_ub == INT32_MAX) {
        S->ub = orc_neh(n, m, p, S->best_perm);
        from_neh = 1;
    } else {
        S->ub = init_ub;
    }
    S->cap = S->ub;
    int32_t root[ORC_MAXN];
    for (int j = 0; j < n; ++j) root[j] = j;
    bb_dfs(S, root, 0, 0);
    int outcome;
    if (S->aborted) outcome = ORC_LIMIT_NODES;
    else if (S->found || from_neh) outcome = ORC_OPTIMAL;
    else outcome = ORC_PROVEN_NO_BETTER;
    *best_cmax = S->ub;
    if (best_perm && (S->found || from_neh)) memcpy(best_perm, S->best_perm, sizeof(int32_t) * (size_t)n);
    if (counters) {
        counters[0] = S->decomposed; counters[1] = S->bounded;
        counters[2] = S->leaves; counters[3] = S->pruned;
    }
    tables_free(&S->T);
    free(S);
    return outcome;
}

int orc_bb_solve(int n, int m, const int32_t *p, int bound, int capped, int32_t init_ub,
                 int64_t node_limit, int32_t *best_cmax, int32_t *best_perm, int64_t *counters)
{
    return orc_bb_solve_pairs(n, m, p, bound, capped, init_ub, node_limit, best_cmax, best_perm, counters,
                              NULL, 0);
}

/* ------------------------------------------------------------------ */
/* Exact and heuristic references                                       */
/* ------------------------------------------------------------------ */

/* Minimum makespan over all n! permutations (lexicographic enumeration);
 * writes the first optimal permutation found. */
int32_t orc_brute_force(int n, int m, const int32_t *p, int32_t *best_perm)
{
    int32_t a[ORC_MAXN];
    for (int j = 0; j < n; ++j) a[j] = j;
    int32_t best = INT32_MAX;
    for (;;) {
        int32_t c = orc_makespan(n, m, p, a);
        if (c < best) {
            best = c;
            if (best_perm) memcpy(best_perm, a, sizeof(int32_t) * (size_t)n);
        }
        /* next lexicographic permutation */
        int i = n - 2;
        while (i >= 0 && a[i] >= a[i + 1]) --i;
        if (i < 0) break;
        int k = n - 1;
        while (a[k] <= a[i]) --k;
        int32_t t = a[i]; a[i] = a[k]; a[k] = t;
        for (int x = i + 1, y = n - 1; x < y; ++x, --y) { t = a[x]; a[x] = a[y]; a[y] = t; }
    }
    return best;
}

/* NEH (Nawaz, Enscore and Ham, 1983): jobs by decreasing total processing
 * time (ties: lower id first), each inserted at the position of least partial
 * makespan (ties: earliest position). */
int32_t orc_neh(int n, int m, const int32_t *p, int32_t *perm_out)
{
    int32_t order[ORC_MAXN], tot[ORC_MAXN];
    for (int j = 0; j < n; ++j) {
        order[j] = j;
        tot[j] = 0;
        for (int k = 0; k < m; ++k) tot[j] += p[j * m + k];
    }
    for (int a = 1; a < n; ++a) { /* stable insertion sort, decreasing total */
        int32_t x = order[a];
        int b = a - 1;
        while (b >= 0 && tot[order[b]] < tot[x]) { order[b + 1] = order[b]; --b; }
        order[b + 1] = x;
    }
    int32_t seq[ORC_MAXN], cand[ORC_MAXN], C[ORC_MAXN];
    int len = 0;
    for (int a = 0; a < n; ++a) {
        int j = order[a];
        int best_pos = 0;
        int32_t best_c = INT32_MAX;
        for (int pos = 0; pos <= len; ++pos) {
            int c = 0;
            for (int t = 0; t < pos; ++t) cand[c++] = seq[t];
            cand[c++] = j;
            for (int t = pos; t < len; ++t) cand[c++] = seq[t];
            orc_completion(m, p, cand, len + 1, C);
            if (C[m - 1] < best_c) { best_c = C[m - 1]; best_pos = pos; }
        }
        for (int t = len; t > best_pos; --t) seq[t] = seq[t - 1];
        seq[best_pos] = j;
        ++len;
    }
    if (perm_out) memcpy(perm_out, seq, sizeof(int32_t) * (size_t)n);
    return orc_makespan(n, m, p, seq);
}

/* ------------------------------------------------------------------ */
/* Factorial number system and work units (Section 2.6)                 */
/* ------------------------------------------------------------------ */

static uint64_t factorial(int k)
{
    uint64_t f = 1;
    for (int i = 2; i <= k; ++i) f *= (uint64_t)i;
    return f;
}

/* digits[i] (position i from the left, radix n - i, weight (n-1-i)!) of the
 * decimal leaf index x in [0, n!), n <= 20. */
void orc_factoradic_from_decimal(int n, uint64_t x, int32_t *digits)
{
    for (int i = 0; i < n; ++i) {
        uint64_t w = factorial(n - 1 - i);
        digits[i] = (int32_t)(x / w);
        x %= w;
    }
}

uint64_t orc_factoradic_to_decimal(int n, const int32_t *digits)
{
    uint64_t x = 0;
    for (int i = 0; i < n; ++i) x += (uint64_t)digits[i] * factorial(n - 1 - i);
    return x;
}

/* The interval [a, b) handed to a thief by work stealing: its right half
 * [floor((a + b) / 2), b) (Section 2.6). */
uint64_t orc_steal_midpoint(uint64_t a, uint64_t b) { return a + (b - a) / 2; }

/* IVM decoding (Section 2.5): the job selected at each level 0..I and the
 * branching type of each level give the subproblem (sigma1, sigma2); forward
 * levels append to sigma1, backward levels prepend to sigma2. */
void orc_ivm_decode(int level, const int32_t *jobs, const int32_t *dirs, int32_t *sigma1, int32_t *d1,
                    int32_t *sigma2, int32_t *d2)
{
    int a = 0, b = 0;
    int32_t back[ORC_MAXN];
    for (int i = 0; i <= level; ++i) {
        if (dirs[i] == ORC_FWD) sigma1[a++] = jobs[i];
        else back[b++] = jobs[i];
    }
    for (int i = 0; i < b; ++i) sigma2[i] = back[b - 1 - i];
    *d1 = a;
    *d2 = b;
}
