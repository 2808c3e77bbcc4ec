// Host mocks shared by the driver harnesses: the ranked path's selection bitmap (from a keep
// predicate instead of ranker logits) and the two kept-list kernels, each written from its
// documented contract (csrc/cm_internal.h): per list, the subjects its op selects from the two
// bitmap rows, in bit order.
#pragma once

#include <cstdint>
#include <vector>

#include "ctx.h"

namespace mock {

inline int64_t rows_of(int64_t len)
{
    return len <= 0 ? cm::kRowGroup : (len + cm::kRowGroup - 1) / cm::kRowGroup * cm::kRowGroup;
}

inline uint32_t kept_word(const cm::KeptList& L, const uint32_t* bits, int64_t w)
{
    const uint32_t a = bits[L.row_a + w];
    if (L.op == cm::kKeepA) return a;
    const uint32_t b = bits[L.row_b + w];
    return L.op == cm::kKeepAnd ? (a & b) : L.op == cm::kKeepAOnly ? (a & ~b) : (b & ~a);
}

// keep(x, y) for the pair of sequence ids; bitmaps and rows live in host vectors standing in
// for device memory
struct Selection {
    bool (*keep)(int32_t, int32_t) = nullptr;
    std::vector<uint32_t> bits;
    std::vector<int32_t> rows;
};
inline Selection& selection()
{
    static Selection s;
    return s;
}

inline void select_pairs(const std::vector<int32_t>& rows, const std::vector<cm::SelTile>& tiles,
                         int64_t nwords, std::vector<uint32_t>& bitmap)
{
    bitmap.assign((size_t)nwords, 0u);
    for (const cm::SelTile& t : tiles)
        for (int32_t i = 0; i < t.na; ++i)
            for (int32_t j = 0; j < t.nb; ++j)
                if (selection().keep(rows[t.a + i], rows[t.b + j])) {
                    const int64_t col = t.j0 + j;
                    bitmap[t.bits + (int64_t)(t.i0 + i) * t.words + (col >> 5)] |= 1u << (col & 31);
                }
    selection().bits = bitmap;
    selection().rows = rows;
}

inline void kept_totals(const cm::KeptList* lists, int32_t nlists, const uint32_t* bits,
                        const int32_t* reps, const int64_t* off, int64_t* totals)
{
    for (int32_t l = 0; l < nlists; ++l) {
        int64_t rows = 0, res = 0;
        for (int64_t w = 0; w < lists[l].words; ++w)
            for (uint32_t x = kept_word(lists[l], bits, w); x; x &= x - 1) {
                const int32_t id = reps[lists[l].b0 + w * 32 + __builtin_ctz(x)];
                rows += rows_of(off[id + 1] - off[id]);
                res += off[id + 1] - off[id];
            }
        totals[2 * l] = rows;
        totals[2 * l + 1] = res;
    }
}

inline void kept_expand(const cm::KeptList* lists, int32_t nlists, const uint32_t* bits,
                        const int32_t* reps, const int64_t* off, int32_t* ids, int64_t* srow)
{
    for (int32_t l = 0; l < nlists; ++l) {
        int64_t gi = lists[l].g0, row = lists[l].rowbase;
        for (int64_t w = 0; w < lists[l].words; ++w)
            for (uint32_t x = kept_word(lists[l], bits, w); x; x &= x - 1) {
                const int32_t id = reps[lists[l].b0 + w * 32 + __builtin_ctz(x)];
                row += rows_of(off[id + 1] - off[id]);
                ids[gi] = id;
                srow[gi + 1] = row;
                ++gi;
            }
    }
}

}  // namespace mock
