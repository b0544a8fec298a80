// batch_split.h -- the size-class split of a batched fit (host code, no CUDA).
//
// The instances of a batch, ordered by n (largest first), are cut into runs
// ("size classes"); each run is scored by its own persistent pair launch with
// shared memory laid out for the run's largest n.  Model: a run starting at
// position p costs (its pair-rows) / rate[p], rate[p] the resident warps of
// the plan for the n at position p; a run may start only where rate > 0
// (where n changes).  S is the prefix sum of the pair-rows (S[0] = 0,
// S[B] = total).
#pragma once
#include <cstddef>
#include <limits>
#include <vector>

namespace l1l {

// Starts (positions in the n order) of the classes of the cheapest split into
// at most `maxk` runs; with fixed_k > 0, of the cheapest split into fixed_k
// runs (fewer when fewer starts are allowed).  Otherwise a run is added while
// the model puts it at least `gain` (fractionally) below the best with one run
// fewer.  The first start is always 0.  Dynamic programme over start
// positions, O(maxk B^2).
inline std::vector<size_t> best_split(const std::vector<double> &S,
                                      const std::vector<double> &rate, int maxk, int fixed_k,
                                      double gain) {
    const size_t B = rate.size();
    const double INF = std::numeric_limits<double>::infinity();
    // g[k][p]: least cost of positions [p, B) in k + 1 runs starting at p;
    // nxt[k][p]: where the second of them starts
    std::vector<std::vector<double>> g((size_t)maxk, std::vector<double>(B + 1, INF));
    std::vector<std::vector<size_t>> nxt((size_t)maxk, std::vector<size_t>(B + 1, B));
    for (size_t p = 0; p < B; ++p)
        if (rate[p] > 0.0) g[0][p] = (S[B] - S[p]) / rate[p];
    for (int k = 1; k < maxk; ++k)
        for (size_t p = 0; p < B; ++p) {
            if (rate[p] <= 0.0) continue;
            for (size_t q = p + 1; q < B; ++q) {
                if (g[(size_t)k - 1][q] == INF) continue;
                const double t = (S[q] - S[p]) / rate[p] + g[(size_t)k - 1][q];
                if (t < g[(size_t)k][p]) {
                    g[(size_t)k][p] = t;
                    nxt[(size_t)k][p] = q;
                }
            }
        }
    int k = 0;
    if (fixed_k > 0) {
        for (int kk = (fixed_k < maxk ? fixed_k : maxk) - 1; kk >= 0 && k == 0; --kk)
            if (g[(size_t)kk][0] < INF) k = kk;  // fewer when fewer starts are allowed
    } else {
        for (int kk = 1; kk < maxk; ++kk)
            if (g[(size_t)kk][0] < (1.0 - gain) * g[(size_t)k][0]) k = kk;
    }
    std::vector<size_t> starts;
    for (size_t p = 0; k >= 0; --k) {
        starts.push_back(p);
        p = k > 0 ? nxt[(size_t)k][p] : B;
    }
    return starts;
}

// Modelled cost of the runs beginning at `starts` (for tests).
inline double split_cost(const std::vector<double> &S, const std::vector<double> &rate,
                         const std::vector<size_t> &starts) {
    const size_t B = rate.size();
    double t = 0.0;
    for (size_t i = 0; i < starts.size(); ++i) {
        const size_t p = starts[i], q = i + 1 < starts.size() ? starts[i + 1] : B;
        if (rate[p] <= 0.0) return std::numeric_limits<double>::infinity();
        t += (S[q] - S[p]) / rate[p];
    }
    return t;
}

}  // namespace l1l
