// Host check of the int16x2 launch planner (csrc/plan.h): the tile choice for every query
// length 0..70,000 (both with and without a partner query), the CTA tasks of random subject
// lists, and the launch-bin order.  Prints the (mode, R) pairs the tile choice produces, one
// "tile <mode> <R>" line each, then "ok"; a violated check prints it and exits 1.
#include <cstdio>
#include <map>
#include <random>
#include <set>
#include <utility>
#include <vector>

#include "plan.h"

using namespace cm;

static int fails = 0;
#define CHECK(cond, ...)                                                \
    do {                                                                \
        if (!(cond)) {                                                  \
            std::printf("check failed: %s (line %d):", #cond, __LINE__); \
            std::printf(__VA_ARGS__);                                   \
            std::printf("\n");                                          \
            if (++fails > 10) return 1;                                 \
        }                                                               \
    } while (0)

int main()
{
    std::set<std::pair<int, int>> tiles;
    for (int hi = 0; hi < 2; ++hi)
        for (int64_t m = 0; m <= 70000; ++m) {
            const TileChoice t = choose_tile(m, hi != 0);
            tiles.insert({t.mode, t.R});
            const int64_t per = m > 0 ? (m + t.npass - 1) / t.npass : 0;
            CHECK(t.npass >= 1 && t.R >= 1 && t.R <= 32, " m=%lld hi=%d", (long long)m, hi);
            CHECK((int64_t)t.seg * t.R >= per, " m=%lld hi=%d (tile covers a pass)", (long long)m, hi);
            CHECK(m == 0 || (int64_t)t.seg * (t.R - 1) < per, " m=%lld hi=%d (no spare lane column)",
                  (long long)m, hi);
            CHECK((int64_t)t.seg * t.R * t.npass >= m, " m=%lld hi=%d", (long long)m, hi);
            if (hi) {
                CHECK(t.mode == (m <= kSeg16MaxCols ? kModeSeg16 : kModePair), " m=%lld", (long long)m);
                CHECK(t.spw == (t.mode == kModePair ? 1 : 2), " m=%lld", (long long)m);
                if (t.mode == kModePair) CHECK(t.seg * t.R <= 1024 && t.seg == 32, " m=%lld", (long long)m);
            } else {
                CHECK(t.mode == (m <= kTwo16MaxCols ? kModeTwo16 : kModeTwo), " m=%lld", (long long)m);
                CHECK(t.spw == (t.mode == kModeTwo16 ? 4 : 2), " m=%lld", (long long)m);
                if (t.mode == kModeTwo) CHECK(t.seg * t.R <= kTwoPassCols && t.seg == 32, " m=%lld",
                                              (long long)m);
            }
            if (t.mode == kModeSeg16 || t.mode == kModeTwo16) CHECK(t.seg == 16 && t.npass == 1, " m=%lld",
                                                                    (long long)m);
        }

    // tasks of random subject lists, with a row table and without (device-built lists)
    std::mt19937_64 rng(1908);
    for (int trial = 0; trial < 3000; ++trial) {
        const int32_t ns = (int32_t)(rng() % 300);
        std::vector<int64_t> srow(1, 0);
        for (int32_t s = 0; s < ns; ++s) srow.push_back(srow.back() + stream_rows((int64_t)(rng() % 3000)));
        const bool hi = rng() % 2;
        const int64_t m = (int64_t)(rng() % 9000);
        const int64_t target = 256 + (int64_t)(rng() % 200000);
        const TileChoice tc = choose_tile(m, hi);
        const int64_t tgt = std::max<int64_t>(target * tc.spw / tc.npass, 2048);
        for (int with_rows = 0; with_rows < 2; ++with_rows) {
            Plan P;
            add_tasks(P, 3, 7, ns, hi, m, with_rows ? srow.data() : nullptr, target, srow.back());
            CHECK(P.tasks.size() == P.task_R.size() && P.tasks.size() == P.keys.size(), " trial %d", trial);
            int32_t s = 0;
            for (size_t i = 0; i < P.tasks.size(); ++i) {
                const SwTask& t = P.tasks[i];
                CHECK(t.block == 3 && t.k == 7 && t.hi_valid == (hi ? 1 : 0), " trial %d", trial);
                CHECK(t.mode == tc.mode && t.npass == tc.npass, " trial %d", trial);
                CHECK(P.task_R[i] == tc.R * 4 + tc.mode, " trial %d", trial);
                CHECK(t.s0 == s && t.s1 > t.s0 && t.s1 <= ns, " trial %d task %zu", trial, i);
                if (with_rows) {
                    // each task reaches the row target, except the last; one subject fewer
                    // would not
                    const int64_t rows = srow[t.s1] - srow[t.s0];
                    CHECK(t.s1 == ns || rows >= tgt, " trial %d task %zu", trial, i);
                    CHECK(srow[t.s1 - 1] - srow[t.s0] < tgt, " trial %d task %zu", trial, i);
                }
                s = t.s1;
            }
            CHECK(s == ns, " trial %d (coverage)", trial);
        }
    }

    // launch-bin order: a permutation, bins descending, work descending inside a bin
    for (int trial = 0; trial < 300; ++trial) {
        Plan P;
        const int nq = 1 + (int)(rng() % 40);
        for (int q = 0; q < nq; ++q) {
            std::vector<int64_t> srow(1, 0);
            const int32_t ns = 1 + (int32_t)(rng() % 50);
            for (int32_t s = 0; s < ns; ++s) srow.push_back(srow.back() + stream_rows((int64_t)(rng() % 2000)));
            add_tasks(P, q, 2 * q, ns, rng() % 2, (int64_t)(rng() % 6000), srow.data(), 4096);
        }
        std::multiset<std::pair<int, int>> before;
        std::map<std::pair<int, int>, std::pair<int64_t, int>> key_of;   // (block, s0) -> key
        for (size_t i = 0; i < P.tasks.size(); ++i) {
            before.insert({P.tasks[i].block, P.tasks[i].s0});
            key_of[{P.tasks[i].block, P.tasks[i].s0}] = P.keys[i];
        }
        order_tasks(P);
        std::multiset<std::pair<int, int>> after;
        for (const SwTask& t : P.tasks) after.insert({t.block, t.s0});
        CHECK(before == after, " trial %d (permutation)", trial);
        for (size_t i = 0; i < P.tasks.size(); ++i) {
            const auto& k = key_of[{P.tasks[i].block, P.tasks[i].s0}];
            CHECK(P.task_R[i] == k.second, " trial %d (bin travels with its task)", trial);
            if (i + 1 < P.tasks.size()) {
                const auto& k2 = key_of[{P.tasks[i + 1].block, P.tasks[i + 1].s0}];
                CHECK(k.second > k2.second || (k.second == k2.second && k.first >= k2.first),
                      " trial %d (bins descending, work descending inside a bin)", trial);
            }
        }
    }
    if (fails) return 1;
    for (const auto& t : tiles) std::printf("tile %d %d\n", t.first, t.second);
    std::printf("ok\n");
    return 0;
}
