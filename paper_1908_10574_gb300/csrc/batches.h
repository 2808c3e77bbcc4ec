// Host-only: cut a list of pair blocks into device batches of bounded slot count, so that a
// merge round whose rep x rep cross products exceed device memory runs as several batches
// whose results, concatenated, are those of the whole list.  Plain C++ (no CUDA), so the
// host tests compile it on its own.
#pragma once

#include <algorithm>
#include <cstdint>
#include <utility>
#include <vector>

namespace cm {

// Shape of a pair block: CROSS (every (A[k], B[s])) holds a_count * b_count slots in rows of
// b_count; TRI (pairs of A with s < k) holds a_count (a_count - 1) / 2 and is never split.
struct BlockShape {
    bool tri;
    int64_t a_count, b_count;
};

inline int64_t block_slots(const BlockShape& b)
{
    return b.tri ? b.a_count * (b.a_count - 1) / 2 : b.a_count * b.b_count;
}

// Query rows [row0, row0 + rows) of block `block`; their pairs are the slots
// [slot0, slot0 + slots) of the unsplit layout (blocks one after another in list order).
struct BlockPiece {
    int32_t block;
    int64_t row0, rows;
    int64_t slot0, slots;
};

// Batches of at most max_slots slots (max_slots >= 1).  Blocks keep their order and a CROSS
// block is cut between query rows, so every batch's pieces, concatenated in order, cover a
// contiguous slot range, and the batches cover [0, total) in order.  A CROSS row or a TRI
// block larger than max_slots forms a batch of its own.  Empty blocks yield no piece.
inline std::vector<std::vector<BlockPiece>> split_batches(const std::vector<BlockShape>& blocks,
                                                          int64_t max_slots)
{
    std::vector<std::vector<BlockPiece>> batches;
    std::vector<BlockPiece> cur;
    int64_t cur_slots = 0, gslot = 0;
    auto flush = [&]() {
        if (!cur.empty()) batches.push_back(cur);
        cur.clear();
        cur_slots = 0;
    };
    for (size_t b = 0; b < blocks.size(); ++b) {
        const BlockShape& B = blocks[b];
        const int64_t total = block_slots(B);
        if (total <= 0) continue;
        if (B.tri) {
            if (cur_slots > 0 && cur_slots + total > max_slots) flush();
            cur.push_back({(int32_t)b, 0, B.a_count, gslot, total});
            cur_slots += total;
        } else {
            const int64_t per_row = B.b_count;
            int64_t row = 0;
            while (row < B.a_count) {
                int64_t take = (max_slots - cur_slots) / per_row;
                if (take <= 0) {
                    if (cur_slots > 0) {
                        flush();
                        continue;
                    }
                    take = 1;                   // one row above the limit: a batch of its own
                }
                take = std::min(take, B.a_count - row);
                cur.push_back({(int32_t)b, row, take, gslot + row * per_row, take * per_row});
                cur_slots += take * per_row;
                row += take;
            }
        }
        gslot += total;
        if (cur_slots >= max_slots) flush();
    }
    flush();
    return batches;
}

// Appends the significant slots of one batch (`part`: batch-local slot and score, in slot
// order) to `out`, renumbered to the slots of the whole list.  sbase[j] is the batch-local
// first slot of piece j (the running sum of the pieces' slots).
inline void append_batch_slots(const std::vector<BlockPiece>& batch,
                               const std::vector<int64_t>& sbase,
                               const std::vector<std::pair<int64_t, int32_t>>& part,
                               std::vector<std::pair<int64_t, int32_t>>& out)
{
    size_t j = 0;
    for (const auto& e : part) {
        while (j + 1 < batch.size() && sbase[j + 1] <= e.first) ++j;
        out.push_back({batch[j].slot0 + (e.first - sbase[j]), e.second});
    }
}

}  // namespace cm
