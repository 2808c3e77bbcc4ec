// Host check of the ranker's training-batch planner (csrc/train_batches.h) on random pair
// graphs: the components equal those found by a breadth-first search, every epoch lists every
// pair exactly once, batches hold at most batch_pairs pairs, a component that fits a batch is
// never split, a larger one fills whole batches of its own except its last chunk, batches are
// filled greedily in the epoch's component order, and two epochs differ in order.
// Prints "ok <trials>" or the first violation (exit 1).
#include <cstdio>
#include <algorithm>
#include <cstdlib>
#include <queue>
#include <random>
#include <vector>

#include "train_batches.h"

using namespace cm;

#define CHECK(cond)                                                                     \
    do {                                                                                \
        if (!(cond)) {                                                                  \
            std::printf("trial %d: check failed: %s (line %d)\n", trial, #cond, __LINE__); \
            return 1;                                                                   \
        }                                                                               \
    } while (0)

int main(int argc, char** argv)
{
    const int trials = argc > 1 ? std::atoi(argv[1]) : 5000;
    std::mt19937_64 rng(1908);
    int eligible = 0, differ = 0;
    for (int trial = 0; trial < trials; ++trial) {
        const int32_t n = 1 + (int32_t)(rng() % 40);
        const int64_t np = (int64_t)(rng() % 80);
        // a few groups, pairs mostly inside a group (some across, to merge groups)
        const int ng = 1 + (int)(rng() % 6);
        std::vector<int32_t> grp((size_t)n);
        for (auto& x : grp) x = (int32_t)(rng() % ng);
        std::vector<int32_t> pairs((size_t)(2 * np));
        for (int64_t k = 0; k < np; ++k) {
            const int32_t a = (int32_t)(rng() % n);
            int32_t b = (int32_t)(rng() % n);
            if (rng() % 8 != 0)
                for (int t = 0; t < 50 && grp[b] != grp[a]; ++t) b = (int32_t)(rng() % n);
            pairs[2 * k] = a;
            pairs[2 * k + 1] = b;
        }
        const TrainComponents C = train_components(pairs.data(), np, n);
        // reference components by BFS over the pair graph
        std::vector<std::vector<int32_t>> adj((size_t)n);
        for (int64_t k = 0; k < np; ++k) {
            adj[pairs[2 * k]].push_back(pairs[2 * k + 1]);
            adj[pairs[2 * k + 1]].push_back(pairs[2 * k]);
        }
        std::vector<int32_t> bfs((size_t)n, -1);
        int32_t nb = 0;
        for (int32_t s = 0; s < n; ++s) {
            if (bfs[s] >= 0) continue;
            std::queue<int32_t> q;
            q.push(s);
            bfs[s] = nb;
            while (!q.empty()) {
                const int32_t x = q.front();
                q.pop();
                for (int32_t y : adj[x])
                    if (bfs[y] < 0) { bfs[y] = nb; q.push(y); }
            }
            ++nb;
        }
        const int64_t nc = (int64_t)C.off.size() - 1;
        CHECK(C.off[0] == 0 && C.off[nc] == np && (int64_t)C.pairs.size() == np);
        std::vector<int64_t> comp_of((size_t)np, -1);
        for (int64_t c = 0; c < nc; ++c) {
            CHECK(C.off[c + 1] > C.off[c]);
            for (int64_t i = C.off[c]; i < C.off[c + 1]; ++i) {
                const int64_t k = C.pairs[i];
                CHECK(k >= 0 && k < np && comp_of[k] < 0);
                comp_of[k] = c;
                if (i > C.off[c]) CHECK(C.pairs[i - 1] < k);           // list order kept
                // same component <=> same BFS component
                CHECK(bfs[pairs[2 * k]] == bfs[pairs[2 * C.pairs[C.off[c]]]]);
            }
        }
        for (int64_t k = 0; k < np; ++k)
            for (int64_t l = k + 1; l < np; ++l)
                CHECK((comp_of[k] == comp_of[l]) == (bfs[pairs[2 * k]] == bfs[pairs[2 * l]]));
        const int64_t bp = 1 + (int64_t)(rng() % 12);
        std::mt19937_64 g(rng());
        std::vector<int64_t> order, bounds, order2, bounds2;
        train_epoch_batches(C, bp, g, order, bounds);
        train_epoch_batches(C, bp, g, order2, bounds2);
        for (const auto* o : {&order, &order2}) {
            std::vector<int> seen((size_t)np, 0);
            for (int64_t k : *o) { CHECK(k >= 0 && k < np); ++seen[k]; }
            for (int64_t k = 0; k < np; ++k) CHECK(seen[k] == 1);
        }
        const int64_t nbt = (int64_t)bounds.size() - 1;
        CHECK(bounds[0] == 0 && bounds[nbt] == np);
        std::vector<int64_t> batch_of((size_t)np);
        for (int64_t b = 0; b < nbt; ++b) {
            CHECK(bounds[b + 1] > bounds[b] && bounds[b + 1] - bounds[b] <= bp);
            for (int64_t i = bounds[b]; i < bounds[b + 1]; ++i) batch_of[order[i]] = b;
        }
        for (int64_t c = 0; c < nc; ++c) {
            const int64_t sz = C.off[c + 1] - C.off[c];
            const int64_t first = batch_of[C.pairs[C.off[c]]];
            int64_t lo = first, hi = first;
            for (int64_t i = C.off[c]; i < C.off[c + 1]; ++i) {
                lo = std::min(lo, batch_of[C.pairs[i]]);
                hi = std::max(hi, batch_of[C.pairs[i]]);
            }
            if (sz <= bp) {
                CHECK(lo == hi);                                        // never split
            } else {
                // its pairs are contiguous in the epoch order and start a batch; every batch
                // but its last holds only this component and is full
                int64_t pos = np;
                for (int64_t i = 0; i < np; ++i)
                    if (comp_of[order[i]] == c) { pos = i; break; }
                CHECK(bounds[lo] == pos);
                for (int64_t i = pos; i < pos + sz; ++i) CHECK(comp_of[order[i]] == c);
                for (int64_t b = lo; b < hi; ++b) {
                    CHECK(bounds[b + 1] - bounds[b] == bp);
                    for (int64_t i = bounds[b]; i < bounds[b + 1]; ++i)
                        CHECK(comp_of[order[i]] == c);
                }
                for (int64_t i = bounds[lo]; i < bounds[lo + 1]; ++i) CHECK(comp_of[order[i]] == c);
            }
        }
        // greedy fill: a batch that ends before a small component could not have taken it
        for (int64_t b = 0; b + 1 < nbt; ++b) {
            const int64_t c = comp_of[order[bounds[b + 1]]];
            const int64_t sz = C.off[c + 1] - C.off[c];
            if (sz <= bp && comp_of[order[bounds[b + 1] - 1]] != c)
                CHECK((bounds[b + 1] - bounds[b]) + sz > bp);
        }
        // without grouping: one component, epochs are shuffled chunks of bp pairs
        {
            const TrainComponents O = train_one_component(np);
            std::vector<int64_t> o1, b1;
            train_epoch_batches(O, bp, g, o1, b1);
            CHECK((int64_t)o1.size() == np);
            for (size_t b = 0; b + 1 < b1.size(); ++b)
                CHECK(b1[b + 1] - b1[b] == std::min<int64_t>(bp, np - b1[b]));
            std::vector<int64_t> sorted = o1;
            std::sort(sorted.begin(), sorted.end());
            for (int64_t k = 0; k < np; ++k) CHECK(sorted[k] == k);
        }
        if (np >= 8 && nc >= 3) {
            ++eligible;
            differ += order != order2;
        }
    }
    const int trial = trials;
    CHECK(eligible > 0 && differ * 10 > eligible * 9);      // epochs reshuffle
    std::printf("ok %d\n", trials);
    return 0;
}
