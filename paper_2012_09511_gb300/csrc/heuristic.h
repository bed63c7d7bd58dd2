// heuristic.h -- host-side heuristic search that cooperates with the exact
// search (the paper's heuristic threads, Section 4.2): an iterated greedy
// over permutations (Ruiz and Stuetzle, "A simple and effective iterated
// greedy algorithm for the permutation flowshop scheduling problem", EJOR
// 2007), and the pool of host threads that runs it beside the explorer pool,
// exchanging incumbents with the explorers through host-mapped memory.
#pragma once

#include <stdint.h>

#include <atomic>
#include <mutex>
#include <thread>
#include <vector>

#include "solve_internal.h"

namespace pfsp {

// Counter-based generator (splitmix64, Steele, Lea and Flood 2014).
struct SplitMix {
    uint64_t s;
    explicit SplitMix(uint64_t seed) : s(seed) {}
    uint64_t next() {
        uint64_t z = (s += 0x9e3779b97f4a7c15ull);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        return z ^ (z >> 31);
    }
    int below(int k) { return (int)(next() % (uint64_t)k); }  // k > 0
    double unit() { return (double)(next() >> 11) * (1.0 / 9007199254740992.0); }
};

// Iterated greedy on one instance (p job-major, n x m).  Each iteration
// removes d random jobs, reinserts each at its best position (Taillard's
// O(k m) evaluation of all k + 1 insertion points), improves the result by
// insertion local search and accepts it if better, or worse with the
// probability of a constant-temperature simulated-annealing test.
class IteratedGreedy {
  public:
    IteratedGreedy(int n, int m, const int32_t *p, uint64_t seed);
    // start from seq (a permutation of 0..n-1); keeps the best seen
    void reset(const int *seq);
    // run `iterations` iterations or until *stop is set; returns the best makespan
    int run(int64_t iterations, const std::atomic<int> *stop);
    int best() const { return best_c_; }
    const std::vector<int> &best_seq() const { return best_; }
    int makespan(const int *seq, int len);

  private:
    int insert_best(std::vector<int> &seq, int job, int *pos_out);
    int local_search(std::vector<int> &seq, int c);

    int n_, m_;
    const int32_t *p_;
    SplitMix rng_;
    double temperature_;
    std::vector<int> cur_, best_;
    int cur_c_ = 0, best_c_ = 0;
    std::vector<int> e_, q_, f_, order_;
};

// Beam search over forward branching between a fixed prefix sigma1 (seq's
// first d1 jobs) and a fixed suffix sigma2 (its last d2 jobs): level by level,
// every partial schedule of the beam is extended by each unscheduled job and
// the `width` extensions of least LB1 (Section 2.4, the bound as the guide;
// ties: the smaller sum of the front, then the order of generation) are kept.
// The paper applies the beam search of Libralesso et al. to partial schedules
// of the exact search this way, prefix and suffix unchanged (Section 4.2).
// With a width of at least the number of completions it is exhaustive.
// Returns the best makespan and writes its schedule to best.
int beam_search(int n, int m, const int32_t *p, const int *seq, int d1, int d2, int width, std::vector<int> &best);

// A starting point of the threads: a complete schedule, its makespan, and the
// depths of the explorer node it was promoted from (0, 0 for the initial one).
struct Start {
    int c;
    std::vector<int> seq;
    int d1, d2;
    bool operator<(const Start &o) const { return c != o.c ? c < o.c : seq < o.seq; }
    bool operator==(const Start &o) const { return c == o.c && seq == o.seq; }
};

// The heuristic threads of one solve.  The calling thread drives snapshots
// (tick) while the explorer pool runs: the explorers' current nodes are
// promoted to complete schedules (unscheduled jobs in the incumbent's order),
// the best distinct ones feed a buffer of starting points, and each thread
// runs the iterated greedy from one of them for a slice of iterations.
class HeuristicPool {
  public:
    // kind: 0 iterated greedy, 1 beam search from the promoted nodes, 2 both (alternate threads)
    HeuristicPool(int n, int m, const int32_t *p, int threads, uint64_t seed, int kind = 0);
    ~HeuristicPool();
    bool ok() const { return shared_ != nullptr; }
    bool attach(int explorers);  // the explorers' snapshot slots, once their count is known
    CoopShared *device_shared() const { return dshared_; }
    CoopSlot *device_slots() const { return dslots_; }
    // ub0: exclusive incumbent of the solve; start: a schedule to begin from
    void start(int ub0, const std::vector<int> &start);
    void tick();  // called repeatedly by the host thread while the kernel runs
    void stop();
    int best(std::vector<int> *seq);  // best makespan below ub0 (INT32_MAX if none)
    int own_best() {  // best makespan the threads themselves found below ub0
        std::lock_guard<std::mutex> g(mu_);
        return own_c_ < ub0_ ? own_c_ : INT32_MAX;
    }
    uint64_t improvements() const { return improvements_.load(); }
    uint64_t promoted() const { return promoted_; }
    int snapshots() const { return snapshots_; }

  private:
    void worker(int id);
    void offer(const std::vector<int> &seq, int c);
    void collect();
    void adopt_device_incumbent();

    int n_, m_, threads_, K_;
    std::vector<int32_t> p_;
    uint64_t seed_;
    CoopShared *shared_ = nullptr, *dshared_ = nullptr;  // host-mapped
    CoopSlot *slots_ = nullptr, *dslots_ = nullptr;      // host-mapped
    std::vector<std::thread> pool_;
    std::atomic<int> stop_{0};
    std::mutex mu_;
    int best_c_ = 0;    // best makespan known: the threads' or the explorers'
    int own_c_ = 0;     // best makespan the threads found
    int dev_seen_ = INT32_MAX;
    std::vector<int> best_;
    std::vector<Start> starts_;  // best promoted schedules
    int kind_ = 0;
    uint64_t next_start_ = 0;
    std::atomic<uint64_t> improvements_{0};
    uint64_t promoted_ = 0;
    int snapshots_ = 0;
    int ub0_ = 0;
    int req_ = 0;
    bool pending_ = false;
    double last_snap_ = 0, req_time_ = 0;
};

}  // namespace pfsp
