// Host harness for the library's host runtime: csrc/api.cu and csrc/cluster_merge.cu compiled as
// plain C++ and linked with host mocks of the kernel launchers and of the CUDA runtime.  The
// mock kernels compute a fake, deterministic similarity instead of Smith-Waterman (the planner,
// the launch bins, the int16 -> int32 rerun loop, the slot maps, compaction, the cells pipeline,
// the bounded batches and the ClusterMerge driver do not depend on what the scores mean) and
// check the launch contracts the real kernels rely on: a zeroed task ticket per launch, every
// task in its launch's (tile, mode) bin, each warp stream within the boundary stride, the row
// stream holding the block's subjects where the kernel reads them, long pairs only on the
// whole-CTA kernels; after every call the library's cell count must equal the cells the mock
// int16 kernel computed.  Device
// memory is host memory filled with garbage when allocated.
//
// fake score of the ordered pair (a, b): 0 if either is empty; else, with
// h = mix(u * 1000003 + v) (u, v = a, b, or min, max in symmetric mode) and t = h >> 32:
// h % 1000 < 550 -> t % 100; < 940 -> 101 + t % 300; else 30000 + t % 20000 (beyond int16
// with the bias, so those pairs take the int32 rerun); in sparse mode the bounds are 985 and
// 997.  Fake cells of (a, b): with
// h = mix(a * 7919 + b * 104729 + 17), residues of a left uncovered ua = (h & 1) ? (h >> 8) % 15
// : 15 + (h >> 8) % 40 and of b ub = (h & 2) ? (h >> 24) % 15 : 15 + (h >> 24) % 40, each split
// u / 2 before the alignment and the rest after it (capped at length - 1).
//
// Commands on stdin (tokens): "seqs n len..." | "sym 0|1" | "sparse 0|1" | "limit S" | "tuning W rows" |
// "score flags k a0 b0 ..." | "cells k a0 b0 ..." | "allpairs T part nparts capacity" |
// "cm T mT mU use_ranker min_pairs".  Each prints one result block or "error code message".
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <iostream>
#include <string>
#include <vector>

#include "ctx.h"
#include "mock_ranked.h"

using namespace cm;

namespace {

bool g_sym = false;
bool g_sparse = false;            // sparse mode: about 1.5 % of pairs above 100 instead of 45 %
std::vector<int64_t> g_off;       // host copy of the offsets (the fake similarity's lengths)
int g_dummy_handle[64];
int g_next_handle = 0;
int g_dummy_u;

uint64_t mix(uint64_t z)
{
    z += 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

int64_t len_of(int32_t x) { return g_off[x + 1] - g_off[x]; }

int32_t fake_score(int32_t a, int32_t b)
{
    if (len_of(a) == 0 || len_of(b) == 0) return 0;
    uint64_t u = (uint64_t)a, v = (uint64_t)b;
    if (g_sym && u > v) std::swap(u, v);
    const uint64_t h = mix(u * 1000003ULL + v), t = h >> 32, r = h % 1000;
    if (r < (g_sparse ? 985u : 550u)) return (int32_t)(t % 100);
    if (r < (g_sparse ? 997u : 940u)) return (int32_t)(101 + t % 300);
    return (int32_t)(30000 + t % 20000);
}

void fake_extent(int64_t L, uint64_t u, int64_t* s, int64_t* e)
{
    if ((int64_t)u > L - 1) u = (uint64_t)(L - 1);
    const int64_t left = (int64_t)u / 2, right = (int64_t)u - left;
    *s = 1 + left;
    *e = L - right;
}

// (score, i_start, i_end, j_start, j_end) of the ordered pair (a, b)
void fake_cells(int32_t a, int32_t b, int64_t c[5])
{
    c[0] = fake_score(a, b);
    if (c[0] <= 0) { c[1] = c[2] = c[3] = c[4] = 0; return; }
    const uint64_t h = mix((uint64_t)a * 7919ULL + (uint64_t)b * 104729ULL + 17);
    const uint64_t ua = (h & 1) ? (h >> 8) % 15 : 15 + (h >> 8) % 40;
    const uint64_t ub = (h & 2) ? (h >> 24) % 15 : 15 + (h >> 24) % 40;
    fake_extent(len_of(a), ua, &c[1], &c[2]);
    fake_extent(len_of(b), ub, &c[3], &c[4]);
}

int64_t tri(int64_t k) { return k * (k - 1) / 2; }
int64_t tri_row(int64_t v)          // k with tri(k) <= v < tri(k + 1)
{
    int64_t k = (int64_t)((1.0 + std::sqrt(1.0 + 8.0 * (double)v)) * 0.5);
    while (k > 0 && tri(k) > v) --k;
    while (tri(k + 1) <= v) ++k;
    return k;
}

int32_t first_of(int32_t q, int32_t x, int32_t swap) { return swap ? x : q; }
int32_t second_of(int32_t q, int32_t x, int32_t swap) { return swap ? q : x; }

bool contract_error(const SwArgs& a, const char* what)
{
    std::fprintf(stderr, "mock contract violated: %s\n", what);
    *a.err = 7;
    return false;
}

constexpr int64_t kMockChunk = 64;   // compaction chunk of the mock (small: many chunks)
int64_t g_cells_done = 0;            // cells of every slot the mock int16 kernel computed

}  // namespace

// ---- CUDA runtime -----------------------------------------------------------------------
extern "C" {
cudaError_t cudaSetDevice(int) { return cudaSuccess; }
cudaError_t cudaDeviceGetAttribute(int* v, cudaDeviceAttr, int)
{
    *v = 4;
    return cudaSuccess;
}
cudaError_t cudaGetDeviceProperties(cudaDeviceProp* p, int)
{
    std::memset(p, 0, sizeof(*p));
    std::strcpy(p->name, "mock");
    p->multiProcessorCount = 4;
    return cudaSuccess;
}
cudaError_t cudaStreamCreateWithFlags(cudaStream_t* s, unsigned int)
{
    *s = reinterpret_cast<cudaStream_t>(&g_dummy_handle[g_next_handle++ % 64]);
    return cudaSuccess;
}
cudaError_t cudaStreamDestroy(cudaStream_t) { return cudaSuccess; }
cudaError_t cudaStreamSynchronize(cudaStream_t) { return cudaSuccess; }
cudaError_t cudaStreamWaitEvent(cudaStream_t, cudaEvent_t, unsigned int) { return cudaSuccess; }
cudaError_t cudaEventCreate(cudaEvent_t* e)
{
    *e = reinterpret_cast<cudaEvent_t>(&g_dummy_handle[g_next_handle++ % 64]);
    return cudaSuccess;
}
cudaError_t cudaEventCreateWithFlags(cudaEvent_t* e, unsigned int) { return cudaEventCreate(e); }
cudaError_t cudaEventDestroy(cudaEvent_t) { return cudaSuccess; }
cudaError_t cudaEventRecord(cudaEvent_t, cudaStream_t) { return cudaSuccess; }
cudaError_t cudaEventElapsedTime(float* ms, cudaEvent_t, cudaEvent_t)
{
    *ms = 0.f;
    return cudaSuccess;
}
cudaError_t cudaMalloc(void** p, size_t n)
{
    *p = std::malloc(n ? n : 1);
    if (!*p) return cudaErrorMemoryAllocation;
    std::memset(*p, 0xCD, n);                   // device memory is not zeroed
    return cudaSuccess;
}
cudaError_t cudaFree(void* p)
{
    std::free(p);
    return cudaSuccess;
}
cudaError_t cudaMemcpy(void* d, const void* s, size_t n, cudaMemcpyKind)
{
    std::memmove(d, s, n);
    return cudaSuccess;
}
cudaError_t cudaMemcpyAsync(void* d, const void* s, size_t n, cudaMemcpyKind, cudaStream_t)
{
    std::memmove(d, s, n);
    return cudaSuccess;
}
cudaError_t cudaMemsetAsync(void* d, int v, size_t n, cudaStream_t)
{
    std::memset(d, v, n);
    return cudaSuccess;
}
cudaError_t cudaGetLastError(void) { return cudaSuccess; }
const char* cudaGetErrorString(cudaError_t) { return "mock"; }
}

// ---- kernel launchers ---------------------------------------------------------------------
namespace cm {

int sw16_ctas_per_sm(int, int, int) { return 1; }
int sw32_ctas_per_sm() { return 1; }
int cells_wf_ctas_per_sm() { return 1; }

cudaError_t launch_check_codes(const uint8_t* in, int64_t n, int32_t alpha, int32_t* bad, cudaStream_t)
{
    for (int64_t i = 0; i < n; ++i)
        if (in[i] >= alpha) *bad = 1;
    return cudaSuccess;
}

cudaError_t launch_ascii_to_codes(const uint8_t* in, uint8_t* out, int64_t n, int32_t alpha,
                                  int32_t* bad, cudaStream_t)
{
    const std::string A = std::string("ARNDCQEGHILKMFPSTWYVBZX*").substr(0, (size_t)alpha);
    for (int64_t i = 0; i < n; ++i) {
        const char ch = in[i] >= 'a' && in[i] <= 'z' ? (char)(in[i] - 32) : (char)in[i];
        const size_t p = A.find(ch);
        if (p == std::string::npos || !in[i]) { *bad = 1; out[i] = 0; } else out[i] = (uint8_t)p;
    }
    return cudaSuccess;
}

// subject s of the list occupies rows [srow[s], srow[s + 1]): its residues, then pad rows;
// the first row flagged kFirst, the last residue's row (row 0 when empty) kLast
cudaError_t launch_gather_stream(const uint8_t* db, const int64_t* off, const int32_t* ids,
                                 int32_t nb, const int64_t* srow, uint8_t* stream, cudaStream_t)
{
    for (int32_t s = 0; s < nb; ++s) {
        if (srow[s + 1] < srow[s]) return cudaErrorInvalidValue;
        const int64_t b = off[ids[s]], len = off[ids[s] + 1] - b;
        for (int64_t r = 0; r < srow[s + 1] - srow[s]; ++r) {
            uint8_t v = r < len ? db[b + r] : (uint8_t)kPadCode;
            if (r == 0) v |= kFirst;
            if (r == (len > 0 ? len - 1 : 0)) v |= kLast;
            stream[srow[s] + r] = v;
        }
    }
    return cudaSuccess;
}

// first s in [lo, hi] with v[s] >= key; then the nearer of it and its predecessor (the
// kernel's split of a task's rows over its warps' streams, at subject boundaries)
int32_t nearest_boundary(const int64_t* v, int32_t lo, int32_t hi, int64_t key)
{
    const int32_t s = (int32_t)(std::lower_bound(v + lo, v + hi + 1, key) - v);
    const int32_t t = s > hi ? hi : s;
    return (t > lo && key - v[t - 1] < v[t] - key) ? t - 1 : t;
}

cudaError_t launch_sw16(int R, int W, int mode, int grid, const SwArgs& a, cudaStream_t)
{
    if (grid < 1 || (W != 4 && W != 8 && W != 16)) return cudaErrorInvalidValue;
    if (*a.task_counter != 0) { contract_error(a, "task ticket not zeroed"); return cudaSuccess; }
    const int spw = mode == kModePair ? 1 : mode == kModeTwo16 ? 4 : 2;
    for (int32_t i = 0; i < a.ntasks; ++i) {
        const SwTask& t = a.tasks[i];
        const SwBlock& B = a.blocks[t.block];
        const int32_t qhi = a.ids[B.a_ids + t.k + (t.hi_valid ? 1 : 0)];
        const TileChoice tc = choose_tile(len_of(qhi), t.hi_valid != 0);
        if (t.mode != mode || tc.mode != mode || tc.R != R || tc.npass != t.npass) {
            contract_error(a, "task outside its launch bin");
            return cudaSuccess;
        }
        // every warp stream of a multi-pass task must fit the boundary buffer's stride
        const int64_t* srow = a.srows + B.srow;
        const int64_t R0 = srow[t.s0], R1 = srow[t.s1];
        int64_t nmax = 0;
        for (int w = 0; w < W; ++w) {
            int32_t prev = -1;
            for (int k = 0; k <= spw; ++k) {
                const int32_t b = nearest_boundary(srow, t.s0, t.s1,
                                                   R0 + (R1 - R0) * (w * spw + k) / (W * spw));
                if (prev >= 0) nmax = std::max(nmax, srow[b] - srow[prev]);
                prev = b;
            }
        }
        if (t.npass > 1 && (tc.seg == 16 || nmax > a.bnd_stride)) {
            contract_error(a, "warp stream longer than the boundary stride");
            return cudaSuccess;
        }
        // the rows the device kernel reads for subject s must be that subject's
        for (int32_t s = t.s0; s < t.s1; ++s) {
            const int32_t xid = a.ids[B.b_ids + s];
            const uint8_t* row = a.streams + B.stream + srow[s];
            const int64_t len = len_of(xid);
            bool ok = srow[s + 1] - srow[s] == stream_rows(len) && (row[0] & kFirst) &&
                      (row[len > 0 ? len - 1 : 0] & kLast);
            for (int64_t r = 0; ok && r < srow[s + 1] - srow[s]; ++r)
                ok = (row[r] & 31) == (r < len ? a.db[a.off[xid] + r] : (uint8_t)kPadCode);
            if (!ok) {
                contract_error(a, "row stream does not hold the block's subject");
                return cudaSuccess;
            }
        }
        for (int32_t q = t.k; q <= t.k + (t.hi_valid ? 1 : 0); ++q)
            for (int32_t s = t.s0; s < t.s1; ++s) {
                if (B.kind == kTri && s >= q) continue;
                int64_t slot = B.out_base + (B.kind == kTri ? tri(q) - tri(B.k0) + s
                                                            : (int64_t)(q - B.k0) * B.nb + s);
                if (B.has_map) slot = a.out_map[slot];
                const int32_t qid = a.ids[B.a_ids + q], xid = a.ids[B.b_ids + s];
                g_cells_done += len_of(qid) * len_of(xid);
                const int32_t f = fake_score(first_of(qid, xid, B.swap), second_of(qid, xid, B.swap));
                a.out[slot] = (a.sat_thr < 0 || f + a.beta >= a.sat_thr) ? kSat : f;
            }
    }
    *a.task_counter = a.ntasks;
    return cudaSuccess;
}

static cudaError_t rescore(const SwArgs& a, const PairRef* pr, int32_t n, int32_t* counter,
                           bool want_long)
{
    if (*counter != 0) { contract_error(a, "rerun ticket not zeroed"); return cudaSuccess; }
    for (int32_t i = 0; i < n; ++i) {
        const bool lng = len_of(pr[i].q) >= kLongMinCols && len_of(pr[i].x) >= kLongMinRows;
        if (lng != want_long) { contract_error(a, "pair on the wrong rerun kernel"); return cudaSuccess; }
        if (len_of(pr[i].x) > a.bnd_stride) { contract_error(a, "rerun subject longer than the stride"); return cudaSuccess; }
        a.out[pr[i].slot] = fake_score(first_of(pr[i].q, pr[i].x, pr[i].swap),
                                       second_of(pr[i].q, pr[i].x, pr[i].swap));
    }
    *counter = n;
    return cudaSuccess;
}

cudaError_t launch_sw32(int, int grid, const SwArgs& a, const PairRef* pr, int32_t n,
                        int32_t* counter, cudaStream_t)
{
    if (grid < 1) return cudaErrorInvalidValue;
    return rescore(a, pr, n, counter, false);
}

cudaError_t launch_long_sw32(int grid, const SwArgs& a, const PairRef* pr, int32_t n,
                             int32_t* counter, cudaStream_t)
{
    if (grid < 1) return cudaErrorInvalidValue;
    return rescore(a, pr, n, counter, true);
}

static cudaError_t cells_jobs(const SwArgs& a, const CellJob* jobs, int32_t n, int32_t* counter,
                              int32_t* res, bool want_long)
{
    if (*counter != 0) { contract_error(a, "cells ticket not zeroed"); return cudaSuccess; }
    for (int32_t i = 0; i < n; ++i) {
        const CellJob& J = jobs[i];
        const bool lng = J.n >= kLongMinCols && J.m >= kLongMinRows;
        if (lng != want_long) { contract_error(a, "job on the wrong cells kernel"); return cudaSuccess; }
        int64_t c[5];
        fake_cells(J.a, J.b, c);
        if (!J.reverse) {
            if (J.m != len_of(J.a) || J.n != len_of(J.b)) { contract_error(a, "forward job extent"); return cudaSuccess; }
            res[3 * i] = (int32_t)c[0];
            res[3 * i + 1] = c[0] > 0 ? (int32_t)(c[2] - 1) : 0;
            res[3 * i + 2] = c[0] > 0 ? (int32_t)(c[4] - 1) : 0;
        } else {
            if (J.m != c[2] || J.n != c[4]) { contract_error(a, "reverse job extent"); return cudaSuccess; }
            res[3 * i] = (int32_t)c[0];
            res[3 * i + 1] = (int32_t)(J.m - c[1]);
            res[3 * i + 2] = (int32_t)(J.n - c[3]);
        }
    }
    *counter = n;
    return cudaSuccess;
}

cudaError_t launch_cells_wf(int grid, const SwArgs& a, const CellJob* jobs, int32_t n,
                            int32_t* counter, int32_t* res, cudaStream_t)
{
    if (grid < 1) return cudaErrorInvalidValue;
    return cells_jobs(a, jobs, n, counter, res, false);
}

cudaError_t launch_long_cells(int grid, const SwArgs& a, const CellJob* jobs, int32_t n,
                              int32_t* counter, int32_t* res, cudaStream_t)
{
    if (grid < 1) return cudaErrorInvalidValue;
    return cells_jobs(a, jobs, n, counter, res, true);
}

cudaError_t launch_collect_saturated(const int32_t* out, int64_t nslots, const SwBlock* blocks,
                                     int32_t nblocks, const int64_t* first_slot,
                                     const int32_t* ids, const int64_t* out_map, PairRef* list,
                                     int32_t* count, int32_t cap, cudaStream_t)
{
    for (int64_t i = 0; i < nslots; ++i) {
        int32_t b = (int32_t)(std::upper_bound(first_slot, first_slot + nblocks, i) - first_slot) - 1;
        const SwBlock& B = blocks[b];
        const int64_t v = i - B.out_base;
        int64_t k, s;
        if (B.kind == kTri) {
            k = tri_row(v + tri(B.k0));
            s = v + tri(B.k0) - tri(k);
        } else {
            k = B.k0 + v / B.nb;
            s = v % B.nb;
        }
        const int64_t slot = B.has_map ? out_map[i] : i;
        if (out[slot] != kSat) continue;
        const int32_t c = (*count)++;
        if (c < cap) list[c] = PairRef{ids[B.a_ids + k], ids[B.b_ids + s], B.swap, 0, slot};
    }
    return cudaSuccess;
}

int64_t compact_chunks(int64_t nslots) { return (nslots + kMockChunk - 1) / kMockChunk; }

cudaError_t launch_scan_chunks(int64_t* counts, int64_t n, int64_t* total, cudaStream_t)
{
    int64_t run = 0;
    for (int64_t c = 0; c < n; ++c) {
        const int64_t v = counts[c];
        counts[c] = run;
        run += v;
    }
    *total = run;
    return cudaSuccess;
}

static void compact(const int32_t* out, int64_t nslots, int32_t k0, const int32_t* order, int32_t T,
                    int32_t* pairs_out, int64_t* slots_out, int32_t* scores_out,
                    int64_t* chunk_counts, int64_t nchunks, int phase)
{
    for (int64_t c = 0; c < nchunks; ++c) {
        int64_t pos = phase ? chunk_counts[c] : 0, cnt = 0;
        for (int64_t i = c * kMockChunk; i < std::min(nslots, (c + 1) * kMockChunk); ++i) {
            if (!(out[i] > T)) continue;
            ++cnt;
            if (!phase) continue;
            if (order) {
                const int64_t k = tri_row(i + tri(k0)), s = i + tri(k0) - tri(k);
                pairs_out[2 * pos] = std::min(order[k], order[s]);
                pairs_out[2 * pos + 1] = std::max(order[k], order[s]);
            } else {
                slots_out[pos] = i;
            }
            scores_out[pos++] = out[i];
        }
        if (!phase) chunk_counts[c] = cnt;
    }
}

cudaError_t launch_compact_tri(const int32_t* out, int64_t nslots, int32_t k0,
                               const int32_t* order, int32_t T, int32_t* pairs_out,
                               int32_t* scores_out, int64_t* chunk_counts, int64_t nchunks,
                               int phase, cudaStream_t)
{
    compact(out, nslots, k0, order, T, pairs_out, nullptr, scores_out, chunk_counts, nchunks, phase);
    return cudaSuccess;
}

cudaError_t launch_compact_slots(const int32_t* out, int64_t nslots, int32_t T, int64_t* slots_out,
                                 int32_t* scores_out, int64_t* chunk_counts, int64_t nchunks,
                                 int phase, cudaStream_t)
{
    compact(out, nslots, 0, nullptr, T, nullptr, slots_out, scores_out, chunk_counts, nchunks, phase);
    return cudaSuccess;
}

cudaError_t launch_kept_totals(const KeptList* lists, int32_t nlists, const uint32_t* bits,
                               const int32_t* reps, const int64_t* off, int64_t* totals,
                               cudaStream_t)
{
    mock::kept_totals(lists, nlists, bits, reps, off, totals);
    return cudaSuccess;
}

cudaError_t launch_kept_expand(const KeptList* lists, int32_t nlists, const uint32_t* bits,
                               const int32_t* reps, const int64_t* off, int32_t* ids,
                               int64_t* srow, cudaStream_t)
{
    mock::kept_expand(lists, nlists, bits, reps, off, ids, srow);
    return cudaSuccess;
}

// ---- the ranker's two calls from the driver ----------------------------------------------
int ranker_unit_vectors(cm_ctx*, const Prepared&, int64_t, void** U_out)
{
    *U_out = &g_dummy_u;
    return CM_OK;
}

int ranker_select(cm_ctx*, const void*, const std::vector<int32_t>& rows,
                  const std::vector<SelTile>& tiles, float, int64_t nwords,
                  std::vector<uint32_t>& bitmap, const uint32_t** d_bits_out,
                  const int32_t** d_rows_out)
{
    mock::select_pairs(rows, tiles, nwords, bitmap);
    if (d_bits_out) *d_bits_out = mock::selection().bits.data();
    if (d_rows_out) *d_rows_out = mock::selection().rows.data();
    return CM_OK;
}

}  // namespace cm

int main()
{
    cm_ctx* ctx = nullptr;
    if (cm_create(&ctx, 0) != CM_OK) {
        std::printf("error create\n");
        return 1;
    }
    mock::selection().keep = [](int32_t x, int32_t y) {
        const uint64_t u = (uint64_t)std::min(x, y), v = (uint64_t)std::max(x, y);
        return mix(u * 31 + v + 5) % 10 < 7;
    };
    std::vector<uint8_t> seqs;
    int8_t mat[400] = {};
    std::string cmd;
    while (std::cin >> cmd) {
        if (cmd == "seqs") {
            int32_t n;
            std::cin >> n;
            g_off.assign((size_t)n + 1, 0);
            seqs.clear();
            for (int32_t i = 0; i < n; ++i) {
                int64_t L;
                std::cin >> L;
                g_off[i + 1] = g_off[i] + L;
                for (int64_t j = 0; j < L; ++j) seqs.push_back((uint8_t)((i * 7 + j) % 20));
            }
            continue;
        }
        if (cmd == "sym") { int s; std::cin >> s; g_sym = s != 0; continue; }
        if (cmd == "sparse") { int s; std::cin >> s; g_sparse = s != 0; continue; }
        if (cmd == "limit") {
            long long s;
            std::cin >> s;
            const int r = cm_set_batch_limit(ctx, s);
            if (r) std::printf("error %d %s\n", r, cm_last_error(ctx));
            continue;
        }
        if (cmd == "tuning") {
            int w, r;
            std::cin >> w >> r;
            const int e = cm_set_tuning(ctx, w, r);
            if (e) std::printf("error %d %s\n", e, cm_last_error(ctx));
            continue;
        }
        const int32_t n = (int32_t)g_off.size() - 1;
        if (cmd == "score" || cmd == "cells") {
            unsigned flags = 0;
            if (cmd == "score") std::cin >> flags;
            long long k;
            std::cin >> k;
            std::vector<int32_t> p((size_t)(2 * k));
            for (auto& v : p) std::cin >> v;
            std::vector<int32_t> o((size_t)(cmd == "score" ? k : 5 * k));
            std::vector<uint8_t> in = seqs;
            if (flags & CM_ASCII)                      // the same residues as letters
                for (auto& ch : in) ch = (uint8_t)"arndcqeghilkmfpstwyv"[ch];
            const int r = cmd == "score"
                ? sw_score_batch(ctx, in.data(), g_off.data(), n, p.data(), k, mat, 11, 1, o.data(), flags)
                : sw_cells_batch(ctx, seqs.data(), g_off.data(), n, p.data(), k, mat, 11, 1, o.data(), 0);
            if (r) { std::printf("error %d %s\n", r, cm_last_error(ctx)); continue; }
            std::printf("%s %lld\n", cmd.c_str(), (long long)o.size());
            for (int32_t v : o) std::printf("%d\n", v);
        } else if (cmd == "allpairs") {
            int T;
            long long part, nparts, cap;
            std::cin >> T >> part >> nparts >> cap;
            std::vector<int32_t> po((size_t)(2 * cap + 2)), so((size_t)(cap + 1));
            int64_t found = 0;
            const int r = sw_allpairs(ctx, seqs.data(), g_off.data(), n, mat, 11, 1, T, part, nparts,
                                      po.data(), so.data(), cap, &found, 0);
            if (r) { std::printf("error %d %lld %s\n", r, (long long)found, cm_last_error(ctx)); continue; }
            std::printf("allpairs %lld\n", (long long)found);
            for (int64_t i = 0; i < found; ++i) std::printf("%d %d %d\n", po[2 * i], po[2 * i + 1], so[i]);
        } else if (cmd == "cm") {
            cm_params prm{};
            std::cin >> prm.T >> prm.mT >> prm.mU >> prm.use_ranker >> prm.ranker_min_pairs;
            cm_result* res = nullptr;
            const int r = cluster_merge(ctx, seqs.data(), g_off.data(), n, mat, 11, 1, &prm, &res, 0);
            if (r) { std::printf("error %d %s\n", r, cm_last_error(ctx)); continue; }
            std::printf("clusters %d\n", res->n_clusters);
            for (int32_t c = 0; c < res->n_clusters; ++c) {
                std::printf("%d %lld", res->reps[c], (long long)(res->cl_offsets[c + 1] - res->cl_offsets[c]));
                for (int64_t j = res->cl_offsets[c]; j < res->cl_offsets[c + 1]; ++j) std::printf(" %d", res->members[j]);
                std::printf("\n");
            }
            std::printf("pairs %lld\n", (long long)res->n_pairs);
            for (int64_t k = 0; k < res->n_pairs; ++k)
                std::printf("%d %d %d\n", res->pairs[2 * k], res->pairs[2 * k + 1], res->scores[k]);
            std::printf("stats %lld %lld %lld %lld %lld %lld %lld\n", (long long)res->rep_comparisons,
                        (long long)res->exchange_comparisons, (long long)res->intra_comparisons,
                        (long long)res->full_merges, (long long)res->exchanges, (long long)res->merges,
                        (long long)res->gpu_batches);
            cm_result_free(res);
        } else {
            std::printf("error unknown command %s\n", cmd.c_str());
            return 1;
        }
        // the library's cell count must be the cells its int16 launches computed
        cm_stats st{};
        cm_get_stats(ctx, &st);
        if (st.cells != g_cells_done)
            std::fprintf(stderr, "mock contract violated: cells counted %lld, computed %lld\n",
                         (long long)st.cells, (long long)g_cells_done);
        std::fflush(stdout);
    }
    cm_destroy(ctx);
    return 0;
}
