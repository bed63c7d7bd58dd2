// heuristic.cu -- host heuristic threads (Section 4.2): iterated greedy search
// from promoted explorer nodes, feeding improved incumbents to the explorer
// pool through host-mapped memory.  Host code only.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstring>

#include "heuristic.h"
#include "pfsp_internal.h"

namespace pfsp {

static double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// ---------------------------------------------------------------------------
// Iterated greedy (Ruiz and Stuetzle 2007).  Parameters are the ones that
// paper recommends: d = 4 jobs removed per iteration, temperature
// 0.4 * (total processing time) / (10 n m).
// ---------------------------------------------------------------------------
constexpr int kDestroy = 4;
constexpr double kTemperatureFactor = 0.4;

IteratedGreedy::IteratedGreedy(int n, int m, const int32_t *p, uint64_t seed)
    : n_(n), m_(m), p_(p), rng_(seed), e_((size_t)(n + 1) * m), q_((size_t)(n + 1) * m), order_(n) {
    long long tot = 0;
    for (int i = 0; i < n * m; ++i) tot += p[i];
    temperature_ = kTemperatureFactor * (double)tot / (10.0 * n * m);
}

// Completion time of the last job on the last machine (Eq. 1).
int IteratedGreedy::makespan(const int *seq, int len) {
    int *C = e_.data();
    std::fill(C, C + m_, 0);
    for (int i = 0; i < len; ++i) {
        const int32_t *pj = p_ + (size_t)seq[i] * m_;
        int prev = 0;
        for (int k = 0; k < m_; ++k) {
            C[k] = std::max(C[k], prev) + pj[k];
            prev = C[k];
        }
    }
    return len ? C[m_ - 1] : 0;
}

// Insert `job` into seq at the position of least makespan (the first such
// position), evaluating all k + 1 positions in O(k m) with Taillard's heads
// e (completion of seq[0..i] on each machine), tails q (longest path from the
// start of seq[i] on a machine to the end) and the inserted job's completion
// f at each position.  Returns the new makespan.
int IteratedGreedy::insert_best(std::vector<int> &seq, int job, int *pos_out) {
    const int k = (int)seq.size(), m = m_;
    int *e = e_.data(), *q = q_.data();
    for (int i = 0; i < k; ++i) {
        const int32_t *pj = p_ + (size_t)seq[i] * m;
        for (int l = 0; l < m; ++l) {
            int up = i ? e[(i - 1) * m + l] : 0;
            int left = l ? e[i * m + l - 1] : 0;
            e[i * m + l] = std::max(up, left) + pj[l];
        }
    }
    for (int i = k - 1; i >= 0; --i) {
        const int32_t *pj = p_ + (size_t)seq[i] * m;
        for (int l = m - 1; l >= 0; --l) {
            int down = i + 1 < k ? q[(i + 1) * m + l] : 0;
            int right = l + 1 < m ? q[i * m + l + 1] : 0;
            q[i * m + l] = std::max(down, right) + pj[l];
        }
    }
    const int32_t *pn = p_ + (size_t)job * m;
    int best = INT_MAX, bi = 0;
    for (int i = 0; i <= k; ++i) {
        int f = 0, c = 0;
        for (int l = 0; l < m; ++l) {
            f = std::max(f, i ? e[(i - 1) * m + l] : 0) + pn[l];
            c = std::max(c, f + (i < k ? q[i * m + l] : 0));
        }
        if (c < best) {
            best = c;
            bi = i;
        }
    }
    seq.insert(seq.begin() + bi, job);
    if (pos_out) *pos_out = bi;
    return best;
}

// Iterative improvement by insertion: each job, in a random order, is taken
// out and reinserted at its best position; a move is kept only if it lowers
// the makespan.  Repeats until a pass improves nothing.
int IteratedGreedy::local_search(std::vector<int> &seq, int c) {
    bool improved = true;
    while (improved) {
        improved = false;
        for (int i = 0; i < n_; ++i) order_[i] = i;
        for (int i = n_ - 1; i > 0; --i) std::swap(order_[i], order_[rng_.below(i + 1)]);
        for (int t = 0; t < n_; ++t) {
            const int job = order_[t];
            const int at = (int)(std::find(seq.begin(), seq.end(), job) - seq.begin());
            seq.erase(seq.begin() + at);
            int pos;
            const int c2 = insert_best(seq, job, &pos);
            if (c2 < c) {
                c = c2;
                improved = true;
            } else {
                seq.erase(seq.begin() + pos);
                seq.insert(seq.begin() + at, job);
            }
        }
    }
    return c;
}

void IteratedGreedy::reset(const int *seq) {
    cur_.assign(seq, seq + n_);
    cur_c_ = local_search(cur_, makespan(cur_.data(), n_));
    best_ = cur_;
    best_c_ = cur_c_;
}

int IteratedGreedy::run(int64_t iterations, const std::atomic<int> *stop) {
    const int d = std::min(kDestroy, std::max(1, n_ - 1));
    std::vector<int> s, removed;
    for (int64_t it = 0; it < iterations; ++it) {
        if (stop && stop->load(std::memory_order_relaxed)) break;
        s = cur_;
        removed.clear();
        for (int r = 0; r < d; ++r) {
            const int at = rng_.below((int)s.size());
            removed.push_back(s[at]);
            s.erase(s.begin() + at);
        }
        int c = 0;
        for (int job : removed) c = insert_best(s, job, nullptr);
        c = local_search(s, c);
        if (c < cur_c_) {
            cur_.swap(s);
            cur_c_ = c;
            if (c < best_c_) {
                best_ = cur_;
                best_c_ = c;
            }
        } else if (rng_.unit() <= std::exp(-(double)(c - cur_c_) / temperature_)) {
            cur_.swap(s);
            cur_c_ = c;
        }
    }
    return best_c_;
}

// ---------------------------------------------------------------------------
// Beam search between a fixed prefix and suffix
// ---------------------------------------------------------------------------
int beam_search(int n, int m, const int32_t *p, const int *seq, int d1, int d2, int width,
                std::vector<int> &best) {
    const int u = n - d1 - d2;
    // back of sigma2: Eq. 1 on the reversed suffix and machines
    std::vector<int> back(m, 0), front0(m, 0), rem0(m, 0);
    for (int i = n - 1; i >= n - d2; --i) {
        const int32_t *pj = p + (size_t)seq[i] * m;
        int right = 0;
        for (int k = m - 1; k >= 0; --k) {
            back[k] = std::max(back[k], right) + pj[k];
            right = back[k];
        }
    }
    for (int i = 0; i < d1; ++i) {
        const int32_t *pj = p + (size_t)seq[i] * m;
        int left = 0;
        for (int k = 0; k < m; ++k) {
            front0[k] = std::max(front0[k], left) + pj[k];
            left = front0[k];
        }
    }
    std::vector<int> mid(seq + d1, seq + (n - d2));
    for (int j : mid)
        for (int k = 0; k < m; ++k) rem0[k] += p[(size_t)j * m + k];
    // beam entries: front [m], remaining work [m], the jobs placed after sigma1
    struct Entry {
        std::vector<int> front, rem, placed;
        uint64_t used;
    };
    std::vector<Entry> beam(1, Entry{front0, rem0, {}, 0ull});
    struct Child {
        int lb, fsum, parent, job;
        bool operator<(const Child &o) const {
            if (lb != o.lb) return lb < o.lb;
            if (fsum != o.fsum) return fsum < o.fsum;
            if (parent != o.parent) return parent < o.parent;
            return job < o.job;
        }
    };
    std::vector<Child> kids;
    std::vector<int> f(m);
    for (int step = 0; step < u; ++step) {
        kids.clear();
        for (int b = 0; b < (int)beam.size(); ++b) {
            const Entry &e = beam[b];
            for (int t = 0; t < u; ++t) {
                const int j = mid[t];
                if ((e.used >> t) & 1ull) continue;
                const int32_t *pj = p + (size_t)j * m;
                int left = 0, lb = 0, fs = 0;
                for (int k = 0; k < m; ++k) {
                    f[k] = std::max(e.front[k], left) + pj[k];
                    left = f[k];
                    lb = std::max(lb, f[k] + e.rem[k] - pj[k] + back[k]);
                    fs += f[k];
                }
                kids.push_back(Child{lb, fs, b, t});
            }
        }
        const size_t keep = std::min<size_t>((size_t)width, kids.size());
        std::partial_sort(kids.begin(), kids.begin() + keep, kids.end());
        std::vector<Entry> next;
        next.reserve(keep);
        for (size_t q = 0; q < keep; ++q) {
            const Child &c = kids[q];
            const Entry &e = beam[c.parent];
            Entry x{e.front, e.rem, e.placed, e.used | (1ull << c.job)};
            const int j = mid[c.job];
            const int32_t *pj = p + (size_t)j * m;
            int left = 0;
            for (int k = 0; k < m; ++k) {
                x.front[k] = std::max(x.front[k], left) + pj[k];
                left = x.front[k];
                x.rem[k] -= pj[k];
            }
            x.placed.push_back(j);
            next.push_back(std::move(x));
        }
        beam.swap(next);
    }
    // complete schedules: makespan = max_k front_k + back_k
    int bc = INT_MAX, bi = 0;
    for (int b = 0; b < (int)beam.size(); ++b) {
        int c = 0;
        for (int k = 0; k < m; ++k) c = std::max(c, beam[b].front[k] + back[k]);
        if (c < bc) {
            bc = c;
            bi = b;
        }
    }
    best.assign(seq, seq + d1);
    best.insert(best.end(), beam[bi].placed.begin(), beam[bi].placed.end());
    best.insert(best.end(), seq + (n - d2), seq + n);
    return bc;
}

// ---------------------------------------------------------------------------
// Heuristic threads beside the explorer pool
// ---------------------------------------------------------------------------
constexpr double kSnapPeriod = 0.005;  // seconds between snapshot requests
constexpr double kSnapWait = 0.002;    // seconds to wait for the explorers' answers
constexpr int kSlice = 16;             // iterated-greedy iterations between offers
constexpr int kBeamMax = 256;          // widest beam a thread runs from one node

// Page-locked host memory mapped into the device's address space.
static bool alloc_mapped(size_t bytes, void **host, void **dev) {
    *host = *dev = nullptr;
    if (cudaHostAlloc(host, bytes, cudaHostAllocMapped) != cudaSuccess) return false;
    if (cudaHostGetDevicePointer(dev, *host, 0) != cudaSuccess) {
        cudaFreeHost(*host);
        *host = nullptr;
        return false;
    }
    memset(*host, 0, bytes);
    return true;
}

HeuristicPool::HeuristicPool(int n, int m, const int32_t *p, int threads, uint64_t seed, int kind)
    : n_(n), m_(m), threads_(threads), K_(0), p_(p, p + (size_t)n * m), seed_(seed), kind_(kind) {
    void *h, *d;
    if (!alloc_mapped(sizeof(CoopShared), &h, &d)) return;
    shared_ = (CoopShared *)h;
    dshared_ = (CoopShared *)d;
    shared_->host_ub = INT_MAX;
    shared_->dev_cmax = INT_MAX;
}

bool HeuristicPool::attach(int explorers) {
    void *h, *d;
    if (!alloc_mapped((size_t)explorers * sizeof(CoopSlot), &h, &d)) return false;
    slots_ = (CoopSlot *)h;
    dslots_ = (CoopSlot *)d;
    K_ = explorers;
    return true;
}

HeuristicPool::~HeuristicPool() {
    stop();
    if (slots_) cudaFreeHost(slots_);
    if (shared_) cudaFreeHost(shared_);
}

void HeuristicPool::start(int ub0, const std::vector<int> &start) {
    ub0_ = ub0;
    best_c_ = ub0;
    own_c_ = INT_MAX;
    best_ = start;
    shared_->host_ub = ub0;
    IteratedGreedy probe(n_, m_, p_.data(), 0);
    starts_.assign(1, Start{probe.makespan(start.data(), n_), start, 0, 0});
    last_snap_ = now_s();
    for (int t = 0; t < threads_; ++t) pool_.emplace_back(&HeuristicPool::worker, this, t);
}

void HeuristicPool::stop() {
    stop_.store(1);
    for (auto &t : pool_) t.join();
    pool_.clear();
}

int HeuristicPool::best(std::vector<int> *seq) {
    std::lock_guard<std::mutex> g(mu_);
    if (best_c_ >= ub0_) return INT_MAX;
    if (seq) *seq = best_;
    return best_c_;
}

// A schedule better than every one known so far becomes the incumbent: the
// explorers fold host_ub into theirs at their next limit check.
void HeuristicPool::offer(const std::vector<int> &seq, int c) {
    std::lock_guard<std::mutex> g(mu_);
    if (c < own_c_) own_c_ = c;
    if (c >= best_c_) return;
    best_c_ = c;
    best_ = seq;
    shared_->host_ub = c;
    improvements_.fetch_add(1);
}

void HeuristicPool::worker(int id) {
    IteratedGreedy ig(n_, m_, p_.data(), seed_ * 0x100000001b3ull + (uint64_t)id * 0x9e3779b97f4a7c15ull + 1);
    std::vector<int> s, b;
    const bool beam = kind_ == 1 || (kind_ == 2 && (id & 1));
    while (!stop_.load()) {
        int d1 = 0, d2 = 0;
        {
            std::lock_guard<std::mutex> g(mu_);
            if (starts_.empty()) {
                s = best_;
            } else {
                const Start &st = starts_[next_start_++ % starts_.size()];
                s = st.seq;
                d1 = st.d1;
                d2 = st.d2;
            }
        }
        if (beam) {
            // iterative beam search below this node: widths 1, 2, 4, ... kBeamMax
            for (int w = 1; w <= kBeamMax && !stop_.load(); w *= 2) {
                const int c = beam_search(n_, m_, p_.data(), s.data(), d1, d2, w, b);
                offer(b, c);
            }
            continue;
        }
        ig.reset(s.data());
        offer(ig.best_seq(), ig.best());
        // one slice from this start, offering the best after every few iterations
        for (int r = 0; r < 16 && !stop_.load(); ++r) {
            ig.run(kSlice, &stop_);
            offer(ig.best_seq(), ig.best());
        }
    }
}

void HeuristicPool::tick() {
    adopt_device_incumbent();
    const double t = now_s();
    if (!pending_) {
        if (t - last_snap_ < kSnapPeriod) return;
        req_ += 1;
        shared_->snap_req = req_;
        pending_ = true;
        req_time_ = t;
        return;
    }
    int answered = 0;
    for (int k = 0; k < K_; ++k) answered += slots_[k].seq == req_;
    if (answered < K_ && t - req_time_ < kSnapWait) return;
    collect();
    snapshots_ += 1;
    pending_ = false;
    last_snap_ = now_s();
}

// The explorers' incumbent schedule, when it is better than the threads' best,
// becomes their best too: promotions complete nodes in its order and the
// threads restart from it.  It is not counted as an improvement of theirs.
void HeuristicPool::adopt_device_incumbent() {
    const int c = shared_->dev_cmax;
    if (c == dev_seen_) return;
    dev_seen_ = c;
    std::atomic_thread_fence(std::memory_order_acquire);
    std::vector<int> seq(n_);
    std::vector<char> seen(n_, 0);
    for (int i = 0; i < n_; ++i) {
        const int j = shared_->dev_perm[i];
        if (j >= n_ || seen[j]) return;  // torn by a concurrent writer
        seen[j] = 1;
        seq[i] = j;
    }
    IteratedGreedy ev(n_, m_, p_.data(), 0);
    const int mk = ev.makespan(seq.data(), n_);
    std::lock_guard<std::mutex> g(mu_);
    if (mk >= best_c_) return;
    best_c_ = mk;
    best_ = seq;
    shared_->host_ub = mk;
}

// Promote the explorers' nodes to complete schedules: sigma1, then the
// unscheduled jobs in the order they have in the incumbent, then sigma2.  The
// best 2 x threads distinct schedules become the threads' starting points.
void HeuristicPool::collect() {
    std::atomic_thread_fence(std::memory_order_acquire);
    std::vector<int> inc;
    {
        std::lock_guard<std::mutex> g(mu_);
        inc = best_;
    }
    std::vector<int> rank(n_, 0);
    for (int i = 0; i < n_; ++i) rank[inc[i]] = i;
    IteratedGreedy ev(n_, m_, p_.data(), 0);
    std::vector<Start> cand;
    std::vector<int> seq(n_), mid;
    std::vector<char> seen(n_);
    for (int k = 0; k < K_; ++k) {
        const CoopSlot &sl = slots_[k];
        if (sl.seq != req_) continue;
        const int d1 = sl.d1, d2 = sl.d2;
        if (d1 + d2 > n_) continue;
        std::fill(seen.begin(), seen.end(), 0);
        bool ok = true;
        for (int i = 0; i < n_ && ok; ++i) {
            const int j = sl.perm[i];
            ok = j < n_ && !seen[j];
            if (ok) seen[j] = 1;
        }
        if (!ok) continue;  // an explorer that has not decomposed a node yet
        mid.assign(sl.perm + d1, sl.perm + (n_ - d2));
        std::sort(mid.begin(), mid.end(), [&](int x, int y) { return rank[x] < rank[y]; });
        for (int i = 0; i < d1; ++i) seq[i] = sl.perm[i];
        for (int i = 0; i < (int)mid.size(); ++i) seq[d1 + i] = mid[i];
        for (int i = n_ - d2; i < n_; ++i) seq[i] = sl.perm[i];
        cand.push_back(Start{ev.makespan(seq.data(), n_), seq, d1, d2});
        promoted_ += 1;
    }
    if (cand.empty()) return;
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    if ((int)cand.size() > 2 * threads_) cand.resize((size_t)2 * threads_);
    offer(cand[0].seq, cand[0].c);
    std::lock_guard<std::mutex> g(mu_);
    starts_ = std::move(cand);
}

}  // namespace pfsp

using namespace pfsp;

extern "C" int pfsp_iterated_greedy(const int32_t *p, int n, int m, const int32_t *start, int64_t iterations,
                                    uint64_t seed, int32_t *best_perm, int32_t *best_cmax) {
    if (!p || !best_perm || !best_cmax || n < 1 || m < 1 || iterations < 0)
        return set_error(PFSP_ERR_INVALID, "pfsp_iterated_greedy: bad argument");
    if (n > 64) return set_error(PFSP_ERR_UNSUPPORTED, "pfsp_iterated_greedy: n > 64");
    for (int i = 0; i < n * m; ++i)
        if (p[i] < 0) return set_error(PFSP_ERR_INVALID, "pfsp_iterated_greedy: negative processing time");
    std::vector<int> s(n);
    if (start) {
        std::vector<char> seen(n, 0);
        for (int i = 0; i < n; ++i) {
            if (start[i] < 0 || start[i] >= n || seen[start[i]])
                return set_error(PFSP_ERR_INVALID, "pfsp_iterated_greedy: start is not a permutation");
            seen[start[i]] = 1;
            s[i] = start[i];
        }
    } else {
        neh(n, m, p, s);
    }
    IteratedGreedy ig(n, m, p, seed);
    ig.reset(s.data());
    ig.run(iterations, nullptr);
    for (int i = 0; i < n; ++i) best_perm[i] = ig.best_seq()[i];
    *best_cmax = ig.best();
    return PFSP_OK;
}

extern "C" int pfsp_beam_search(const int32_t *p, int n, int m, const int32_t *prefix, int d1, const int32_t *suffix,
                                int d2, int width, int32_t *best_perm, int32_t *best_cmax) {
    if (!p || !best_perm || !best_cmax || n < 1 || m < 1 || width < 1 || d1 < 0 || d2 < 0 || d1 + d2 > n ||
        (d1 > 0 && !prefix) || (d2 > 0 && !suffix))
        return set_error(PFSP_ERR_INVALID, "pfsp_beam_search: bad argument");
    if (n > 64) return set_error(PFSP_ERR_UNSUPPORTED, "pfsp_beam_search: n > 64");
    for (int i = 0; i < n * m; ++i)
        if (p[i] < 0) return set_error(PFSP_ERR_INVALID, "pfsp_beam_search: negative processing time");
    std::vector<char> seen(n, 0);
    std::vector<int> seq(n);
    for (int i = 0; i < d1 + d2; ++i) {
        const int j = i < d1 ? prefix[i] : suffix[i - d1];
        if (j < 0 || j >= n || seen[j]) return set_error(PFSP_ERR_INVALID, "pfsp_beam_search: prefix and suffix must be distinct jobs");
        seen[j] = 1;
    }
    for (int i = 0; i < d1; ++i) seq[i] = prefix[i];
    for (int i = 0; i < d2; ++i) seq[n - d2 + i] = suffix[i];
    for (int j = 0, at = d1; j < n; ++j)
        if (!seen[j]) seq[at++] = j;
    std::vector<int> best;
    *best_cmax = beam_search(n, m, p, seq.data(), d1, d2, width, best);
    for (int i = 0; i < n; ++i) best_perm[i] = best[i];
    return PFSP_OK;
}
