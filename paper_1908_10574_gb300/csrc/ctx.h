// Host-side runtime shared by the C ABI entry points: the context, device buffers, input
// preparation, the planner (pair blocks -> length-binned CTA tasks) and plan execution.
#pragma once

#include <algorithm>
#include <cstdio>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "cm_internal.h"
#include "plan.h"

namespace cm {

struct DevBuf {
    void* p = nullptr;
    size_t cap = 0;
};

enum BufId {
    B_DB, B_RAW, B_OFF, B_BLOCKS, B_TASKS, B_IDS, B_STREAM, B_SROW, B_OUT, B_OMAP, B_BND,
    B_FLAGS, B_PREF, B_FIRST, B_PAIRS, B_CELLS, B_SCRATCH, B_CHUNK, B_POUT, B_SOUT, B_MAT,
    B_JOBS, B_RES, B_KEPT, B_KTOT, B_COUNT
};

}  // namespace cm

struct cm_ctx {
    int device = 0;
    int num_sms = 0;
    cudaStream_t own = nullptr;
    cudaStream_t stream = nullptr;
    std::string err;
    cm_stats stats{};
    int W = 16;                             // the autotuner's usual choice on GB300
    int rows_per_warp = 8192;
    int64_t max_batch_slots = (int64_t)1 << 32;   // slots of one rep-wave device batch
    int32_t wait_limit = 1 << 24;           // polls (~100 ns each) of a bounded device wait
    int32_t greedy_chunk = 2048;            // sequences per device batch of greedy_cluster
    int64_t chunk_pairs = (int64_t)1 << 24; // plain merges of >= 2x this many rep pairs score cs2
    int32_t rep_chunks = 16;                // ... in column ranges of >= chunk_pairs, at most this many
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaStream_t aux = nullptr;             // second stream: alternate length bins overlap tails
    cudaEvent_t fork = nullptr, join = nullptr;
    cm::DevBuf buf[cm::B_COUNT];
    void* ranker = nullptr;                 // learned ranker state (ranker.cu)
    void (*ranker_free)(void*) = nullptr;
    int sw16_occ[3][33][4] = {};            // CTAs per SM by (W = 4/8/16, R, mode); 0 = unknown
};

namespace cm {

int fail(cm_ctx* c, int code, const std::string& msg);

// NVTX range for the lifetime of a scope (a no-op unless a profiler is attached)
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// resident CTAs per SM of the int16x2 kernel (W, R, mode), queried once per context
inline int sw16_occupancy(cm_ctx* c, int R, int W, int mode)
{
    int& v = c->sw16_occ[W == 4 ? 0 : W == 8 ? 1 : 2][R][mode];
    if (v == 0) v = std::max(1, sw16_ctas_per_sm(R, W, mode));
    return v;
}

#define CUDA_TRY(call)                                                                      \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return ::cm::fail(c, e_ == cudaErrorMemoryAllocation ? CM_ERR_OOM : CM_ERR_CUDA, \
                              std::string(#call " failed: ") + cudaGetErrorString(e_));     \
    } while (0)

int ensure_bytes(cm_ctx* c, BufId id, size_t bytes, void** out);

template <class T>
int ensure(cm_ctx* c, BufId id, size_t count, T** out)
{
    void* p = nullptr;
    int r = ensure_bytes(c, id, count * sizeof(T), &p);
    *out = reinterpret_cast<T*>(p);
    return r;
}

// B_FLAGS layout (int32 words): [1] kernel bounds-check flag, [2..3] int32-rerun list count and
// ticket, [4..7] other kernels' tickets, [8 ..) one task ticket per (tile width, launch mode)
// bin of the int16x2 kernel.
constexpr int kTaskBins = 32 * 4;
constexpr int kFlagWords = 8 + kTaskBins;

#define ENSURE(id, n, ptr)                                                                  \
    do {                                                                                    \
        int r_ = ::cm::ensure(c, id, (size_t)(n), &(ptr));                                  \
        if (r_) return r_;                                                                  \
    } while (0)

struct Prepared {
    const uint8_t* db = nullptr;     // device residue codes
    const int64_t* off = nullptr;    // device offsets
    std::vector<int64_t> hoff;       // host offsets
    int16_t mat[kAlpha * kAlpha];    // [first][second], stride kAlpha
    int32_t alpha = 20;              // letters of the call's matrix (20, or 24 with CM_MATRIX24)
    int32_t g1 = 0, ge = 0;          // first-gap cost, extension cost
    int32_t beta = 0, sat_thr = 0;
    bool symmetric = true;
    int64_t maxlen = 0;
    int64_t len(int32_t i) const { return hoff[i + 1] - hoff[i]; }
};

int copy_in(cm_ctx* c, void* dst, const void* src, size_t bytes, bool dev);
int prepare(cm_ctx* c, const uint8_t* seqs, const int64_t* offsets, int32_t n_seqs,
            const int8_t* matrix, int32_t gap_open, int32_t gap_extend, uint32_t flags,
            Prepared& P);
// sequences only (no matrix / gaps): validation and device staging
int prepare_seqs(cm_ctx* c, const uint8_t* seqs, const int64_t* offsets, int32_t n_seqs,
                 uint32_t flags, Prepared& P);
int ranker_embed_device(cm_ctx* c, const Prepared& P, const int32_t* ids, int64_t n, float* V);
// one 128 x 128 tile of a pair-selection block: rows[a + i] x rows[b + j], i < na, j < nb
struct SelTile {
    int32_t block;
    int32_t i0, j0;        // offsets of the tile inside its block
    int32_t na, nb;        // valid rows / columns of the tile (<= 128)
    int32_t a, b;          // first A row / B row of the tile in the row list
    int32_t words;         // 32-bit words per bitmap row of the block
    int64_t bits;          // first bitmap word of the block
};
int ranker_unit_vectors(cm_ctx* c, const Prepared& P, int64_t n, void** U_out);
// sets bit (i, j) of each block's bitmap (row-major, `words` words per row) where the
// ranker logit of (A row i, B row j) reaches thr; `bitmap` holds nwords words on return
int ranker_select(cm_ctx* c, const void* U, const std::vector<int32_t>& rows,
                  const std::vector<SelTile>& tiles, float thr, int64_t nwords,
                  std::vector<uint32_t>& bitmap, const uint32_t** d_bits_out = nullptr,
                  const int32_t** d_rows_out = nullptr);
int ranker_alpha_beta(cm_ctx* c, float* ab);

int run_plan(cm_ctx* c, const Prepared& P, Plan& plan, int32_t* out, const int64_t* d_omap,
             uint32_t flags);

// A block request for score_blocks: queries A and subjects B are ranges of `ids`.
// kind kCross: every (A[k], B[s]); kind kTri (A must equal B): (A[k], A[s]), s < k.
// swap 0 scores the pair as (query, subject), swap 1 as (subject, query).
struct BlockReq {
    int32_t kind;
    int32_t swap;
    int64_t a_begin, a_count;
    int64_t b_begin, b_count;
};

// Scores every pair of every block; slot order: block after block, CROSS k*nb + s, TRI
// k(k-1)/2 + s.  base[b] = first slot of block b.  Results land in `scores` (host).
int score_blocks(cm_ctx* c, const Prepared& P, const std::vector<int32_t>& ids,
                 const std::vector<BlockReq>& req, std::vector<int32_t>& scores,
                 std::vector<int64_t>& base, uint32_t flags);

// As score_blocks, but only the slots whose score exceeds T come back: (slot, score) in slot
// order, compacted on the device (the full score array never leaves it).  Lists of more than
// the context's max_batch_slots slots run as several device batches cut between query rows
// (same result); *n_batches (may be null) receives the number of batches.
int score_blocks_sig(cm_ctx* c, const Prepared& P, const std::vector<int32_t>& ids,
                     const std::vector<BlockReq>& req, int32_t T,
                     std::vector<std::pair<int64_t, int32_t>>& sig, std::vector<int64_t>& base,
                     uint32_t flags, int64_t* n_batches = nullptr);

// (slot, score) of the device slots [0, nslots) of `out` whose score exceeds T, slot order.
int compact_sig(cm_ctx* c, const int32_t* out, int64_t nslots, int32_t T,
                std::vector<std::pair<int64_t, int32_t>>& sig);

// Exact int32 scores of host pairs (pairs[2k] = query: columns, pairs[2k + 1] = subject:
// rows) straight on the int32 kernels, with no int16 pass: pairs of >= kLongMinCols columns and
// >= kLongMinRows rows on whole CTAs (passes pipelined over the warps), the rest one warp each.
// Meant for pairs of two long sequences, for which the int16 pass runs one warp per pair and
// mostly marks the pair for rescoring anyway.  scores[k] = f(pair k).
int score_pairs_int32(cm_ctx* c, const Prepared& P, const std::vector<int32_t>& pairs,
                      std::vector<int32_t>& scores);

// Score and alignment cells (5 int32 per pair) of host pairs, on the device data of P.
int run_cells(cm_ctx* c, const Prepared& P, const int32_t* host_pairs, int64_t n_pairs,
              int32_t* host_cells);

}  // namespace cm
