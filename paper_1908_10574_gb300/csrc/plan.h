// Host planner of the int16x2 Smith-Waterman launches: a pair block's queries, taken one or
// two at a time, get a register tile and launch mode (tile choice), their subjects are cut into
// CTA tasks of bounded work (add_tasks), and the tasks are grouped into one persistent launch
// per (tile, mode) bin, longest first (order_tasks).  Host code only; the host tests compile it
// on its own.
#pragma once

#include <algorithm>
#include <cstdint>
#include <utility>
#include <vector>

#include "cm_internal.h"

namespace cm {

struct Plan {
    std::vector<SwBlock> blocks;
    std::vector<int64_t> first_slot;     // per block, ascending
    std::vector<int32_t> ids;            // A ids then B ids
    std::vector<int64_t> srow;           // global row table over all B subjects (+1)
    std::vector<SwTask> tasks;           // grouped by R, cost descending inside a group
    std::vector<int> task_R;             // launch bin R * 4 + mode per task (parallel to tasks)
    std::vector<std::pair<int64_t, int>> keys;   // (cost, bin) per task, for ordering
    int64_t nslots = 0;
    int64_t cells = 0, cells_padded = 0, pairs = 0;
    int64_t max_warp_rows = 0;
    // Device-built subject lists: `ids` holds the A ids only; the B ids (n_sub of them) and the
    // row table (n_sub + 1 entries, total_rows rows) already sit in the B_IDS (after the A ids)
    // and B_SROW buffers; `srow` stays empty.
    bool dev_lists = false;
    int64_t n_sub = 0, total_rows = 0;
};

// Register tile and launch mode of a query (pair) whose longer query has m_hi residues.
struct TileChoice {
    int mode;      // SwMode
    int R;         // columns per lane per pass
    int npass;     // column passes
    int seg;       // lanes per query segment (32, or 16 in the segment modes)
    int spw;       // subject streams per warp
};

// A query without a partner runs in a single-query mode (two subject streams per 32-lane warp,
// or four over two 16-lane segments); a pair runs over 32 lanes or, when its longer query fits
// 16 lanes x 32 columns, in the 16-lane segment mode (R per lane twice that of a 32-lane tile,
// 16-column granularity).  32-lane pair tiles take passes of at most 1,024 columns (R 17..32
// above 512 residues); 32-lane single-query tiles passes of at most 512 (R 9..16), where the
// two-stream step still fits two rows into the register budget.
inline TileChoice choose_tile(int64_t m_hi, bool hi_valid)
{
    TileChoice t{};
    if (m_hi <= (hi_valid ? kSeg16MaxCols : kTwo16MaxCols)) {
        t.mode = hi_valid ? kModeSeg16 : kModeTwo16;
        t.seg = 16;
        t.R = (int)std::max<int64_t>(1, (m_hi + 15) / 16);
        t.npass = 1;
    } else if (hi_valid) {
        t.mode = kModePair;
        t.seg = 32;
        t.npass = (int)((m_hi + 1023) / 1024);
        const int64_t per = (m_hi + t.npass - 1) / t.npass;
        t.R = std::max(1, std::min(32, (int)((per + 31) / 32)));
    } else {
        t.mode = kModeTwo;
        t.seg = 32;
        t.npass = (int)((m_hi + kTwoPassCols - 1) / kTwoPassCols);
        const int64_t per = (m_hi + t.npass - 1) / t.npass;
        t.R = (int)((per + 31) / 32);
    }
    t.spw = t.mode == kModePair ? 1 : t.mode == kModeTwo16 ? 4 : 2;
    return t;
}

// Tasks of one query pair (k, k+1) or single query k against the block's subjects [0, ns), each
// holding about `target` rows per stream of its warps, divided by the query's column passes (a
// task streams its rows once per pass: sizing by rows x passes keeps the tasks of long queries
// as long as everyone else's).  With `srow` (the block's subject row table) the tasks split at
// subject boundaries by rows; without it (device-built lists) into equal subject counts,
// `rows_total` being the rows of all ns subjects.
inline void add_tasks(Plan& P, int32_t block, int32_t k, int32_t ns, bool hi_valid,
                      int64_t m_hi, const int64_t* srow, int64_t target, int64_t rows_total = 0)
{
    const TileChoice tc = choose_tile(m_hi, hi_valid);
    const int R = tc.R, np = tc.npass, mode = tc.mode, seg = tc.seg, spw = tc.spw;
    const bool single = mode == kModeTwo || mode == kModeTwo16;
    target = std::max<int64_t>(target * spw / np, 2048);
    const int64_t ntask = srow ? 0 : std::max<int64_t>(1, (rows_total + target - 1) / target);
    const int64_t per = srow ? 0 : (ns + ntask - 1) / ntask;
    int32_t s = 0;
    while (s < ns) {
        int32_t e;
        if (srow) {
            const int64_t want = srow[s] + target;
            e = (int32_t)(std::lower_bound(srow + s + 1, srow + ns + 1, want) - srow);
        } else {
            e = (int32_t)std::min<int64_t>(ns, s + per);
        }
        if (e > ns) e = ns;
        SwTask t{};
        t.block = block;
        t.k = k;
        t.s0 = s;
        t.s1 = e;
        t.npass = np;
        t.hi_valid = hi_valid ? 1 : 0;
        t.mode = mode;
        const int64_t rows = srow ? srow[e] - srow[s] : rows_total * (e - s) / std::max(ns, 1);
        P.cells_padded += rows * seg * R * np * (single ? 1 : 2);
        P.tasks.push_back(t);
        P.task_R.push_back(R * 4 + mode);         // launch bin: register tile and mode
        P.keys.push_back({rows * R * np / spw, R * 4 + mode});
        s = e;
    }
}

// Groups the tasks by launch bin (descending), most work first inside a bin, ties in the
// order the tasks were made.  (The keys are sorted with their task index, not through it, so
// the sort stays cache-friendly for the millions of tasks of a large merge.)
inline void order_tasks(Plan& P)
{
    struct Key {
        int64_t cost;
        int bin;
        size_t i;
    };
    std::vector<Key> k(P.tasks.size());
    for (size_t i = 0; i < k.size(); ++i) k[i] = {P.keys[i].first, P.keys[i].second, i};
    std::sort(k.begin(), k.end(), [](const Key& x, const Key& y) {
        if (x.bin != y.bin) return x.bin > y.bin;
        if (x.cost != y.cost) return x.cost > y.cost;
        return x.i < y.i;
    });
    std::vector<SwTask> t2(k.size());
    std::vector<int> r2(k.size());
    for (size_t i = 0; i < k.size(); ++i) { t2[i] = P.tasks[k[i].i]; r2[i] = P.task_R[k[i].i]; }
    P.tasks.swap(t2);
    P.task_R.swap(r2);
}

}  // namespace cm
