// Host check of the device-batch splitter (csrc/batches.h) on random block lists: the batches
// cover the unsplit slot layout in order, respect the slot limit, cut CROSS blocks only between
// query rows, fill each batch greedily, and the significant slots of the batches, renumbered,
// equal those of the whole list.  Prints "ok <trials>" or the first violation (exit 1).
#include <cstdio>
#include <cstdlib>
#include <random>
#include <utility>
#include <vector>

#include "batches.h"

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
    const int trials = argc > 1 ? std::atoi(argv[1]) : 20000;
    std::mt19937_64 rng(1908);
    for (int trial = 0; trial < trials; ++trial) {
        const int nb = (int)(rng() % 9);
        std::vector<BlockShape> bl((size_t)nb);
        for (auto& b : bl) {
            b.tri = rng() % 4 == 0;
            b.a_count = (int64_t)(rng() % 8);
            b.b_count = b.tri ? b.a_count : (int64_t)(rng() % 10);
        }
        std::vector<int64_t> base((size_t)nb + 1, 0);
        for (int b = 0; b < nb; ++b) base[b + 1] = base[b] + block_slots(bl[b]);
        const int64_t total = base[nb];
        const int64_t maxs = 1 + (int64_t)(rng() % 48);
        const auto batches = split_batches(bl, maxs);

        // coverage, order, row cuts, limit
        int64_t next = 0;
        std::vector<int64_t> rows_done((size_t)nb, 0);
        std::vector<int64_t> batch_slots;
        for (const auto& bt : batches) {
            CHECK(!bt.empty());
            int64_t s = 0;
            for (const auto& p : bt) {
                const BlockShape& B = bl[p.block];
                CHECK(p.slots > 0);
                CHECK(p.slot0 == next);
                if (B.tri) {
                    CHECK(p.row0 == 0 && p.rows == B.a_count && p.slots == block_slots(B));
                    CHECK(p.slot0 == base[p.block]);
                } else {
                    CHECK(p.row0 == rows_done[p.block]);
                    CHECK(p.rows >= 1 && p.slots == p.rows * B.b_count);
                    CHECK(p.slot0 == base[p.block] + p.row0 * B.b_count);
                    rows_done[p.block] += p.rows;
                }
                next += p.slots;
                s += p.slots;
            }
            const BlockPiece& p0 = bt[0];
            CHECK(s <= maxs || (bt.size() == 1 && (bl[p0.block].tri || p0.rows == 1)));
            batch_slots.push_back(s);
        }
        CHECK(next == total);
        for (int b = 0; b < nb; ++b)
            if (!bl[b].tri && block_slots(bl[b]) > 0) CHECK(rows_done[b] == bl[b].a_count);
        // greedy: the next batch's first row (or TRI block) did not fit into the previous one
        for (size_t i = 0; i + 1 < batches.size(); ++i) {
            const BlockPiece& p = batches[i + 1][0];
            const BlockShape& B = bl[p.block];
            const int64_t need = B.tri ? p.slots : B.b_count;
            CHECK(batch_slots[i] + need > maxs);
        }

        // renumbering: a batch's local slots enumerate its pieces' pairs in the order of the
        // unsplit layout (CROSS k * nb + s, TRI k (k - 1) / 2 + s)
        std::vector<int32_t> score((size_t)total);
        for (auto& v : score) v = (int32_t)(rng() % 100);
        const int32_t T = (int32_t)(rng() % 100);
        std::vector<std::pair<int64_t, int32_t>> direct, via;
        for (int64_t i = 0; i < total; ++i)
            if (score[i] > T) direct.push_back({i, score[i]});
        for (const auto& bt : batches) {
            std::vector<int64_t> sbase(bt.size() + 1, 0), global;
            for (size_t j = 0; j < bt.size(); ++j) {
                const BlockPiece& p = bt[j];
                const BlockShape& B = bl[p.block];
                sbase[j + 1] = sbase[j] + p.slots;
                if (B.tri) {
                    for (int64_t k = 1; k < B.a_count; ++k)
                        for (int64_t s = 0; s < k; ++s)
                            global.push_back(base[p.block] + k * (k - 1) / 2 + s);
                } else {
                    for (int64_t k = p.row0; k < p.row0 + p.rows; ++k)
                        for (int64_t s = 0; s < B.b_count; ++s)
                            global.push_back(base[p.block] + k * B.b_count + s);
                }
            }
            CHECK((int64_t)global.size() == sbase[bt.size()]);
            std::vector<std::pair<int64_t, int32_t>> part;
            for (int64_t l = 0; l < (int64_t)global.size(); ++l)
                if (score[global[l]] > T) part.push_back({l, score[global[l]]});
            append_batch_slots(bt, sbase, part, via);
        }
        CHECK(via == direct);
    }
    std::printf("ok %d\n", trials);
    return 0;
}
