// Internal declarations shared by the libcm CUDA sources (not part of the C ABI).
#pragma once

#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/cm.h"

namespace cm {

// ---- residue streams -------------------------------------------------------------------
// A block's subjects are concatenated into one byte stream, one byte per DP row:
// bits 0-4 residue code (0..23, 24 = pad row whose scores are all non-positive),
// bit 7 = first row of a subject, bit 6 = last row of a subject.  Every subject occupies a
// multiple of kRowGroup rows (pad rows follow it), so subjects start on group boundaries and a
// kernel step can cover up to kRowGroup rows; an empty subject is one group of pad rows, the
// first carrying both flags, so its score comes out 0.
constexpr uint8_t kFirst = 0x80;
constexpr uint8_t kLast = 0x40;
// Residue codes: ARNDCQEGHILKMFPSTWYV = 0..19, then B, Z, X, * = 20..23 (24-letter matrices,
// CM_MATRIX24); a 20 x 20 matrix sits in the top-left corner of the 24 x 24 one every kernel
// reads, and calls with it accept codes 0..19 only.
constexpr int kAlpha = 24;             // letters of the largest alphabet (matrix stride)
constexpr uint8_t kPadCode = 24;
constexpr int kProfRows = 25;          // 24 residues + pad row

// rows a subject of `len` residues occupies in a stream: a multiple of kRowGroup (at least
// one group), so subjects start on group boundaries and a kernel step can cover a group
constexpr int kRowGroup = 4;
inline int64_t stream_rows(int64_t len)
{
    return len <= 0 ? kRowGroup : (len + kRowGroup - 1) / kRowGroup * kRowGroup;
}

// longest sequence accepted: keeps every warp stream of the kernels below 2^31 rows
constexpr int64_t kMaxSeqLen = int64_t(1) << 28;

// ---- pair blocks -----------------------------------------------------------------------
// A block is a set of pairs between queries A (held in registers, one column per residue)
// and subjects B (streamed row by row).  CROSS: query k pairs with every subject s < nb.
// TRI: A == B sorted by length; query k pairs with subjects s < k.
enum BlockKind : int32_t { kCross = 0, kTri = 1 };

struct SwBlock {
    int32_t kind;       // BlockKind
    int32_t swap;       // 0: cell score M[q][x] (query = pair's first); 1: M[x][q]
    int32_t na, nb;     // |A|, |B|
    int64_t a_ids;      // offset of A's sequence ids in the id pool
    int64_t b_ids;      // offset of B's sequence ids in the id pool
    int64_t stream;     // byte offset of B's row stream in the stream pool
    int64_t srow;       // offset of B's row table (nb+1 entries) in the row pool
    int64_t out_base;   // output slot of the block's first pair
    int32_t k0;         // first query index covered (TRI: slot = tri(k) - tri(k0) + s)
    int32_t has_map;    // 1: slot -> user index through out_map[]
};

// Launch modes of the int16x2 kernel (see sw16_kernel): query pair over 32 lanes; single
// query with two subject streams in the word halves; query pair with two subject streams,
// one per 16-lane half-warp segment; single query with four subject streams (two 16-lane
// segments x two halves).  The 16-lane modes serve queries of at most kSeg16MaxCols.
enum SwMode : int32_t { kModePair = 0, kModeTwo = 1, kModeSeg16 = 2, kModeTwo16 = 3 };
constexpr int kSeg16MaxCols = 16 * 32;   // longest query tile of the 16-lane pair mode
constexpr int kTwo16MaxCols = 16 * 16;   // ... of the 16-lane single-query mode (registers)
constexpr int kTwoPassCols = 32 * 16;    // column pass of the 32-lane single-query mode

// One CTA task: query k (single-query modes) or the query pair (k, k+1) (pair modes, the two
// queries in the two 16-bit halves) of a block against subjects [s0, s1), whose rows are split
// over the CTA's subject streams.  `mode` is the SwMode of the launch the task belongs to.
struct SwTask {
    int32_t block;
    int32_t k;          // lo query index; hi = k+1 (if hi_valid)
    int32_t s0, s1;     // subjects covered (rows split over the CTA's streams)
    int32_t npass;      // column passes of SEG*R columns
    int32_t hi_valid;   // 0 when the lo query has no partner
    int32_t mode;
    int32_t pad;
};

struct SwArgs {
    const uint8_t* db;          // residue codes of all sequences
    const int64_t* off;         // n_seqs+1 offsets
    const SwBlock* blocks;
    const SwTask* tasks;
    int32_t ntasks;
    int32_t* task_counter;      // zeroed before launch
    const int32_t* ids;         // id pool
    const uint8_t* streams;     // stream pool
    const int64_t* srows;       // row pool
    int32_t* out;               // output slots (int32 scores, kSat = needs int32 rerun)
    const int64_t* out_map;     // slot -> user index (blocks with has_map)
    uint2* bnd;                 // multi-pass boundary columns, bnd_stride rows per warp
    int64_t bnd_stride;
    int32_t* err;               // set non-zero by a kernel's own bounds checks
    int16_t mat[kAlpha * kAlpha];   // substitution matrix, [first residue][second residue]
    int32_t gap_open;           // first-gap cost (already includes extend for BLAST mode)
    int32_t gap_extend;
    int32_t beta;               // int16 bias: stored = true + beta
    int32_t sat_thr;            // stored best >= sat_thr -> rerun in int32
    int32_t wait_limit;         // polls of a bounded device wait before it gives up (long pairs)
};

constexpr int32_t kSat = INT32_MIN;   // output slot marker: saturated in int16, rerun pending

// One pair for the int32 rerun / cells kernels.
struct PairRef {
    int32_t q, x;       // query (columns) and subject (rows) sequence ids
    int32_t swap;       // as SwBlock::swap
    int32_t pad;
    int64_t slot;       // output slot (final index)
};

// One job of the alignment-cells kernel: rows a[0..m), columns b[0..n) (both reversed when
// `reverse`), result = (best, first row, first column) in row-major order, 0-based.
struct CellJob {
    int32_t a, b;
    int32_t m, n;
    int32_t reverse;
    int32_t pad;
};

// One subject list of a ranked block, selected by bitmap rows of the ranker's pair selection:
// op 0 = row a, 1 = row a AND row b, 2 = row a AND NOT row b, 3 = row b AND NOT row a.  Bit i
// of a row selects subject reps[b0 + i].  The list's subjects become global subjects g0 ..,
// its stream rows start at rowbase.
enum KeptOp : int32_t { kKeepA = 0, kKeepAnd = 1, kKeepAOnly = 2, kKeepBOnly = 3 };
struct KeptList {
    int64_t row_a, row_b;   // word offsets of the two bitmap rows (row_b unused for kKeepA)
    int32_t words;          // words per row
    int32_t op;             // KeptOp
    int64_t b0;             // offset of the subject reps in `reps`
    int64_t g0;             // first global subject index of the list
    int64_t rowbase;        // first stream row of the list
};

// ---- launchers (sw16.cu) ---------------------------------------------------------------
int sw16_ctas_per_sm(int R, int W, int mode);
cudaError_t launch_sw16(int R, int W, int mode, int grid, const SwArgs& a, cudaStream_t st);
cudaError_t launch_sw32(int R, int grid, const SwArgs& a, const PairRef* pr, int32_t npairs,
                        int32_t* counter, cudaStream_t st);
int sw32_smem_bytes(int R);
int cells_wf_ctas_per_sm();
// long pairs on a whole CTA (longpair.cu): one CTA per SM, kLongSlots boundary slots per CTA
constexpr int kLongSlots = 8;
constexpr int64_t kLongMinCols = 2048, kLongMinRows = 512;
int long_pair_smem();
cudaError_t launch_long_sw32(int grid, const SwArgs& a, const PairRef* pr, int32_t npairs,
                             int32_t* counter, cudaStream_t st);
cudaError_t launch_long_cells(int grid, const SwArgs& a, const CellJob* jobs, int32_t njobs,
                              int32_t* counter, int32_t* res, cudaStream_t st);
cudaError_t launch_cells_wf(int grid, const SwArgs& a, const CellJob* jobs, int32_t njobs,
                            int32_t* counter, int32_t* res, cudaStream_t st);

// ---- pack.cu ---------------------------------------------------------------------------
// letters of the 20-letter alphabet (alpha 20) or also B, Z, X, * (alpha 24) -> codes
cudaError_t launch_ascii_to_codes(const uint8_t* in, uint8_t* out, int64_t n, int32_t alpha,
                                  int32_t* bad, cudaStream_t st);
cudaError_t launch_check_codes(const uint8_t* in, int64_t n, int32_t alpha, int32_t* bad,
                               cudaStream_t st);
cudaError_t launch_gather_stream(const uint8_t* db, const int64_t* off, const int32_t* ids,
                                 int32_t nb, const int64_t* srow, uint8_t* stream,
                                 cudaStream_t st);
cudaError_t launch_collect_saturated(const int32_t* out, int64_t nslots, const SwBlock* blocks,
                                     int32_t nblocks, const int64_t* block_first_slot,
                                     const int32_t* ids, const int64_t* out_map,
                                     PairRef* list, int32_t* count, int32_t cap,
                                     cudaStream_t st);
cudaError_t launch_compact_tri(const int32_t* out, int64_t nslots, int32_t k0,
                               const int32_t* order, int32_t T, int32_t* pairs_out,
                               int32_t* scores_out, int64_t* chunk_counts, int64_t nchunks,
                               int phase, cudaStream_t st);
cudaError_t launch_scan_chunks(int64_t* counts, int64_t nchunks, int64_t* total,
                               cudaStream_t st);
cudaError_t launch_compact_slots(const int32_t* out, int64_t nslots, int32_t T,
                                 int64_t* slots_out, int32_t* scores_out, int64_t* chunk_counts,
                                 int64_t nchunks, int phase, cudaStream_t st);
int64_t compact_chunks(int64_t nslots);
// per list: stream rows and residues of its subjects (totals[2*l], totals[2*l + 1])
cudaError_t launch_kept_totals(const KeptList* lists, int32_t nlists, const uint32_t* bits,
                               const int32_t* reps, const int64_t* off, int64_t* totals,
                               cudaStream_t st);
// per list: subject ids (ids[g0 + s]) and row table (srow[g0 + s + 1]) in bitmap order
cudaError_t launch_kept_expand(const KeptList* lists, int32_t nlists, const uint32_t* bits,
                               const int32_t* reps, const int64_t* off, int32_t* ids,
                               int64_t* srow, cudaStream_t st);

}  // namespace cm
