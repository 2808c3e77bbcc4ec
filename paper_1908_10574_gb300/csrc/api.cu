// C ABI of libcm: context, input validation, the host planner that turns pair lists into
// length-binned CTA tasks for the persistent int16x2 kernel, the int32 rerun of saturated
// pairs, and threshold compaction.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "batches.h"
#include "ctx.h"

namespace cm {
int sw32_ctas_per_sm();
}  // namespace cm

using namespace cm;

namespace cm {

int fail(cm_ctx* c, int code, const std::string& msg)
{
    if (c) c->err = msg;
    return code;
}

int ensure_bytes(cm_ctx* c, BufId id, size_t bytes_in, void** out)
{
    DevBuf& b = c->buf[id];
    const size_t bytes = std::max<size_t>(bytes_in, 16);
    if (bytes > b.cap) {
        if (b.p) {
            cudaStreamSynchronize(c->stream);
            cudaFree(b.p);
        }
        const size_t want = std::max(bytes, b.cap + b.cap / 2);
        b.p = nullptr;
        b.cap = 0;
        cudaError_t e = cudaMalloc(&b.p, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            b.p = nullptr;
            return fail(c, CM_ERR_OOM, "device allocation of " + std::to_string(want) +
                                           " bytes failed: " + cudaGetErrorString(e));
        }
        b.cap = want;
    }
    *out = b.p;
    return CM_OK;
}

int copy_in(cm_ctx* c, void* dst, const void* src, size_t bytes, bool dev)
{
    if (bytes == 0) return CM_OK;
    CUDA_TRY(cudaMemcpyAsync(dst, src, bytes, dev ? cudaMemcpyDeviceToDevice
                                                  : cudaMemcpyHostToDevice, c->stream));
    return CM_OK;
}

int prepare(cm_ctx* c, const uint8_t* seqs, const int64_t* offsets, int32_t n_seqs,
            const int8_t* matrix, int32_t gap_open, int32_t gap_extend, uint32_t flags,
            Prepared& P)
{
    const bool dev = (flags & CM_DEVICE_PTRS) != 0;
    if (!c) return CM_ERR_ARG;
    c->err.clear();
    if (!matrix) return fail(c, CM_ERR_ARG, "null matrix");
    // gaps
    const int64_t g1 = (flags & CM_GAP_BLAST) ? (int64_t)gap_open + gap_extend : gap_open;
    if (g1 < 1 || g1 > 1000 || gap_extend < 0 || gap_extend > g1)
        return fail(c, CM_ERR_ARG, "gap costs must satisfy 1 <= first-gap cost <= 1000 and "
                                   "0 <= gap_extend <= first-gap cost");
    P.g1 = (int32_t)g1;
    P.ge = gap_extend;
    // matrix: 20 x 20, or 24 x 24 over ARNDCQEGHILKMFPSTWYVBZX* with CM_MATRIX24; either sits
    // in the 24 x 24 table the kernels read (a 20 x 20 one in its top-left corner)
    const int A = (flags & CM_MATRIX24) ? kAlpha : 20;
    P.alpha = A;
    int8_t hm[kAlpha * kAlpha];
    if (dev) CUDA_TRY(cudaMemcpy(hm, matrix, (size_t)A * A, cudaMemcpyDeviceToHost));
    else std::memcpy(hm, matrix, (size_t)A * A);
    int mn = 0, mx = 0;
    for (int i = 0; i < kAlpha * kAlpha; ++i) P.mat[i] = 0;
    for (int x = 0; x < A; ++x)
        for (int y = 0; y < A; ++y) {
            const int8_t v = hm[x * A + y];
            P.mat[x * kAlpha + y] = v;
            mn = std::min<int>(mn, v);
            mx = std::max<int>(mx, v);
            if (v != hm[y * A + x]) P.symmetric = false;
        }
    P.beta = std::max<int32_t>(P.g1 + P.ge, -mn) + 1;
    P.sat_thr = 32767 - std::max(mx, 0);
    return prepare_seqs(c, seqs, offsets, n_seqs, flags, P);
}

int prepare_seqs(cm_ctx* c, const uint8_t* seqs, const int64_t* offsets, int32_t n_seqs,
                 uint32_t flags, Prepared& P)
{
    const bool dev = (flags & CM_DEVICE_PTRS) != 0;
    if (!c) return CM_ERR_ARG;
    c->err.clear();
    if (n_seqs < 0 || !offsets) return fail(c, CM_ERR_ARG, "null offsets or n_seqs < 0");
    // offsets
    P.hoff.resize((size_t)n_seqs + 1);
    if (dev) CUDA_TRY(cudaMemcpy(P.hoff.data(), offsets, sizeof(int64_t) * (n_seqs + 1),
                                 cudaMemcpyDeviceToHost));
    else std::memcpy(P.hoff.data(), offsets, sizeof(int64_t) * (n_seqs + 1));
    if (P.hoff[0] != 0) return fail(c, CM_ERR_ARG, "offsets[0] must be 0");
    for (int32_t i = 0; i < n_seqs; ++i) {
        const int64_t L = P.hoff[i + 1] - P.hoff[i];
        if (L < 0) return fail(c, CM_ERR_ARG, "offsets must be non-decreasing");
        if (L > kMaxSeqLen)
            return fail(c, CM_ERR_ARG, "a sequence is longer than 2^28 residues");
        P.maxlen = std::max(P.maxlen, L);
    }
    const int64_t total = P.hoff[n_seqs];
    if (total > 0 && !seqs) return fail(c, CM_ERR_ARG, "seqs is null");
    // residues
    int32_t* flags_d;
    ENSURE(B_FLAGS, kFlagWords, flags_d);
    CUDA_TRY(cudaMemsetAsync(flags_d, 0, kFlagWords * sizeof(int32_t), c->stream));
    uint8_t* db;
    if (flags & CM_ASCII) {
        ENSURE(B_DB, total, db);
        const uint8_t* src = seqs;
        if (!dev) {
            uint8_t* raw;
            ENSURE(B_RAW, total, raw);
            int r = copy_in(c, raw, seqs, total, false);
            if (r) return r;
            src = raw;
        }
        CUDA_TRY(launch_ascii_to_codes(src, db, total, P.alpha, flags_d, c->stream));
        P.db = db;
    } else if (dev) {
        P.db = seqs;
        CUDA_TRY(launch_check_codes(seqs, total, P.alpha, flags_d, c->stream));
    } else {
        ENSURE(B_DB, total, db);
        int r = copy_in(c, db, seqs, total, false);
        if (r) return r;
        CUDA_TRY(launch_check_codes(db, total, P.alpha, flags_d, c->stream));
        P.db = db;
    }
    if (dev) {
        P.off = offsets;
    } else {
        int64_t* off;
        ENSURE(B_OFF, n_seqs + 1, off);
        int r = copy_in(c, off, P.hoff.data(), sizeof(int64_t) * (n_seqs + 1), false);
        if (r) return r;
        P.off = off;
    }
    int32_t bad = 0;
    CUDA_TRY(cudaMemcpyAsync(&bad, flags_d, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (bad) return fail(c, CM_ERR_RESIDUE, (flags & CM_ASCII)
                                                ? "a letter outside the matrix's alphabet in seqs"
                                                : "a residue code outside the matrix's alphabet in seqs");
    return CM_OK;
}

// ---- execution --------------------------------------------------------------------------
int run_plan(cm_ctx* c, const Prepared& P, Plan& plan, int32_t* out, const int64_t* d_omap,
             uint32_t flags)
{
    const cudaStream_t st = c->stream;
    const int W = c->W;
    // upload
    SwBlock* d_blocks; SwTask* d_tasks; int32_t* d_ids; int64_t* d_srow; uint8_t* d_stream;
    int64_t* d_first; int32_t* d_flags;
    ENSURE(B_BLOCKS, plan.blocks.size(), d_blocks);
    ENSURE(B_TASKS, plan.tasks.size(), d_tasks);
    const int64_t nsub = plan.dev_lists ? plan.n_sub : (int64_t)plan.srow.size() - 1;
    const int64_t n_ids = plan.dev_lists ? (int64_t)plan.ids.size() + plan.n_sub
                                         : (int64_t)plan.ids.size();
    ENSURE(B_IDS, n_ids, d_ids);
    ENSURE(B_SROW, nsub + 1, d_srow);
    ENSURE(B_FIRST, plan.first_slot.size(), d_first);
    ENSURE(B_FLAGS, kFlagWords, d_flags);
    const int64_t nrows_total = plan.dev_lists ? plan.total_rows : plan.srow.back();
    ENSURE(B_STREAM, nrows_total + 64, d_stream);
    int r;
    if ((r = copy_in(c, d_blocks, plan.blocks.data(), plan.blocks.size() * sizeof(SwBlock), false))) return r;
    if ((r = copy_in(c, d_tasks, plan.tasks.data(), plan.tasks.size() * sizeof(SwTask), false))) return r;
    if ((r = copy_in(c, d_ids, plan.ids.data(), plan.ids.size() * sizeof(int32_t), false))) return r;
    if (!plan.dev_lists)
        if ((r = copy_in(c, d_srow, plan.srow.data(), plan.srow.size() * sizeof(int64_t), false))) return r;
    if ((r = copy_in(c, d_first, plan.first_slot.data(), plan.first_slot.size() * sizeof(int64_t), false))) return r;
    CUDA_TRY(cudaMemsetAsync(d_flags, 0, kFlagWords * sizeof(int32_t), st));
    // the B subjects of all blocks form one list in the id pool after the A ids
    const int64_t b_first = n_ids - nsub;
    CUDA_TRY(launch_gather_stream(P.db, P.off, d_ids + b_first, (int32_t)nsub, d_srow, d_stream, st));
    c->stats.launches += 1;

    SwArgs a{};
    a.db = P.db;
    a.off = P.off;
    a.blocks = d_blocks;
    a.ids = d_ids;
    a.streams = d_stream;
    a.srows = d_srow;
    a.out = out;
    a.out_map = d_omap;
    a.err = d_flags + 1;
    a.wait_limit = c->wait_limit;
    std::memcpy(a.mat, P.mat, sizeof(a.mat));
    a.gap_open = P.g1;
    a.gap_extend = P.ge;
    a.beta = P.beta;
    a.sat_thr = (flags & CM_FORCE_INT32) ? -1 : P.sat_thr;   // -1: every pair goes to int32

    // boundary buffer for multi-pass queries and for the int32 rerun
    // even, so the pair-mode records (16 bytes per two rows) stay 16-byte aligned
    const int64_t stride = (std::max<int64_t>(plan.max_warp_rows, P.maxlen) + 64 + 1) & ~(int64_t)1;
    int max_ctas = 0;
    for (int R = 1; R <= 32; ++R)
        for (int mode = 0; mode < 4; ++mode)
            max_ctas = std::max(max_ctas, c->num_sms * sw16_occupancy(c, R, W, mode));
    const int64_t nwarps = std::max<int64_t>(std::max<int64_t>((int64_t)max_ctas * W,
                                             (int64_t)c->num_sms * std::max(1, sw32_ctas_per_sm())),
                                             (int64_t)c->num_sms * kLongSlots);
    uint2* d_bnd;
    ENSURE(B_BND, 2 * nwarps * stride, d_bnd);     // one half per stream
    a.bnd_stride = stride;

    // One persistent launch per (register tile, mode) bin, longest tasks first within it.
    // Consecutive bins alternate between the context stream and the auxiliary stream, so the
    // next bin's CTAs take the SMs that the previous bin's CTAs leave as its queue drains
    // (launch tails overlap); each stream has its own half of the boundary buffer.
    CUDA_TRY(cudaEventRecord(c->ev[0], st));
    CUDA_TRY(cudaEventRecord(c->fork, st));
    CUDA_TRY(cudaStreamWaitEvent(c->aux, c->fork, 0));
    size_t i0 = 0;
    int bin = 0;
    cudaError_t le = cudaSuccess;
    while (i0 < plan.tasks.size() && le == cudaSuccess && bin < kTaskBins) {
        const int key = plan.task_R[i0];
        const int R = key / 4, mode = key % 4;
        size_t i1 = i0;
        while (i1 < plan.tasks.size() && plan.task_R[i1] == key) ++i1;
        a.tasks = d_tasks + i0;
        a.ntasks = (int32_t)(i1 - i0);
        a.task_counter = d_flags + 8 + bin;
        const int occ = sw16_occupancy(c, R, W, mode);
        const int grid = (int)std::min<int64_t>(a.ntasks, (int64_t)c->num_sms * occ);
        a.bnd = d_bnd + (bin & 1) * nwarps * stride;
        le = launch_sw16(R, W, mode, grid, a, (bin & 1) ? c->aux : st);
        c->stats.launches += 1;
        c->stats.sw16_launches += 1;
        i0 = i1;
        ++bin;
    }
    // join the auxiliary stream before any return, so no launch of this call outlives it
    CUDA_TRY(cudaEventRecord(c->join, c->aux));
    CUDA_TRY(cudaStreamWaitEvent(st, c->join, 0));
    CUDA_TRY(le);
    if (i0 < plan.tasks.size()) return fail(c, CM_ERR_INTERNAL, "more launch bins than task tickets");
    CUDA_TRY(cudaEventRecord(c->ev[1], st));
    a.bnd = d_bnd;

    // int32 rescoring of every pair the int16 pass marked as possibly saturated
    PairRef* d_pref;
    const int32_t cap = (int32_t)std::min<int64_t>(std::max<int64_t>(plan.nslots, 1), 1 << 20);
    ENSURE(B_PREF, cap, d_pref);
    for (int round = 0;; ++round) {
        CUDA_TRY(cudaMemsetAsync(d_flags + 2, 0, 4 * sizeof(int32_t), st));
        CUDA_TRY(launch_collect_saturated(out, plan.nslots, d_blocks, (int32_t)plan.blocks.size(),
                                          d_first, d_ids, d_omap, d_pref, d_flags + 2, cap, st));
        int32_t cnt = 0;
        CUDA_TRY(cudaMemcpyAsync(&cnt, d_flags + 2, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        c->stats.launches += 1;
        if (cnt == 0) break;
        const int32_t n = std::min(cnt, cap);
        c->stats.saturated += n;
        // Long pairs (many column passes) first, on whole CTAs; the rest longest first on one
        // warp each (the persistent warps claim them in order).
        std::vector<PairRef> lst((size_t)n);
        CUDA_TRY(cudaMemcpyAsync(lst.data(), d_pref, n * sizeof(PairRef), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        auto is_long = [&](const PairRef& x) {
            return P.len(x.q) >= kLongMinCols && P.len(x.x) >= kLongMinRows;
        };
        std::stable_sort(lst.begin(), lst.end(), [&](const PairRef& x, const PairRef& y) {
            const bool lx = is_long(x), ly = is_long(y);
            if (lx != ly) return lx;
            return P.len(x.q) * P.len(x.x) > P.len(y.q) * P.len(y.x);
        });
        if ((r = copy_in(c, d_pref, lst.data(), lst.size() * sizeof(PairRef), false))) return r;
        int32_t nlong = 0;
        while (nlong < n && is_long(lst[nlong])) ++nlong;
        if (nlong > 0) {
            CUDA_TRY(launch_long_sw32((int)std::min<int64_t>(nlong, c->num_sms), a, d_pref, nlong,
                                      d_flags + 5, st));
            c->stats.launches += 1;
        }
        if (n > nlong) {
            const int grid = (int)std::min<int64_t>(n - nlong, (int64_t)c->num_sms * std::max(1, sw32_ctas_per_sm()));
            CUDA_TRY(launch_sw32(16, grid, a, d_pref + nlong, n - nlong, d_flags + 3, st));
            c->stats.launches += 1;
        }
        // every full round rescored `cap` distinct slots (a rescored slot no longer holds the
        // saturation mark), so more rounds than slots / cap means no progress
        if ((int64_t)round * cap > plan.nslots)
            return fail(c, CM_ERR_INTERNAL, "int32 rerun did not converge");
    }
    int32_t kerr = 0;
    CUDA_TRY(cudaMemcpyAsync(&kerr, d_flags + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (kerr == 2) return fail(c, CM_ERR_TIMEOUT, "a long-pair pipeline wait gave up");
    if (kerr) return fail(c, CM_ERR_INTERNAL, "kernel bounds check fired (boundary buffer)");
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, c->ev[0], c->ev[1]));
    c->stats.sw16_ms += ms;
    c->stats.pairs += plan.pairs;
    c->stats.cells += plan.cells;
    c->stats.cells_padded += plan.cells_padded;
    return CM_OK;
}

namespace {

// Plan of a list of block requests (see score_blocks); returns the number of slots.
int64_t plan_blocks(cm_ctx* c, const Prepared& P, const std::vector<int32_t>& ids,
                    const std::vector<BlockReq>& req, Plan& plan, std::vector<int64_t>& base)
{
    base.assign(req.size() + 1, 0);
    int64_t slots = 0;
    std::vector<int32_t> a_ids, b_ids;
    plan.srow.push_back(0);
    const int64_t target = (int64_t)c->W * c->rows_per_warp;
    for (size_t bi = 0; bi < req.size(); ++bi) {
        const BlockReq& r = req[bi];
        base[bi] = slots;
        SwBlock B{};
        B.kind = r.kind;
        B.swap = r.swap;
        B.na = (int32_t)r.a_count;
        B.nb = (int32_t)r.b_count;
        B.stream = 0;
        B.srow = (int64_t)plan.srow.size() - 1;
        B.b_ids = (int64_t)b_ids.size();
        B.a_ids = (r.kind == kTri) ? -1 : (int64_t)a_ids.size();   // TRI: fixed up below
        B.out_base = slots;
        B.k0 = 0;
        B.has_map = 0;
        for (int64_t s = 0; s < r.b_count; ++s) {
            const int32_t id = ids[r.b_begin + s];
            b_ids.push_back(id);
            plan.srow.push_back(plan.srow.back() + stream_rows(P.len(id)));
        }
        if (r.kind != kTri)
            for (int64_t k = 0; k < r.a_count; ++k) a_ids.push_back(ids[r.a_begin + k]);
        const int64_t nslots = (r.kind == kTri) ? r.a_count * (r.a_count - 1) / 2
                                                : r.a_count * r.b_count;
        slots += nslots;
        plan.first_slot.push_back(B.out_base);
        plan.blocks.push_back(B);
        const int32_t bidx = (int32_t)plan.blocks.size() - 1;
        const int64_t* srow = plan.srow.data() + B.srow;
        // residues of the subjects before s, so a query's cells are one product
        std::vector<int64_t> pre((size_t)r.b_count + 1, 0);
        for (int64_t s = 0; s < r.b_count; ++s) pre[s + 1] = pre[s] + P.len(ids[r.b_begin + s]);
        for (int64_t k = 0; k < r.a_count; k += 2) {
            const bool hi = k + 1 < r.a_count;
            const int32_t qhi = ids[r.a_begin + (hi ? k + 1 : k)];
            int32_t ns = (int32_t)r.b_count;
            if (r.kind == kTri) ns = (int32_t)(hi ? k + 1 : k);
            for (int64_t q = k; q < k + (hi ? 2 : 1); ++q)
                plan.cells += P.len(ids[r.a_begin + q]) * pre[(r.kind == kTri) ? q : r.b_count];
            if (ns > 0) add_tasks(plan, bidx, (int32_t)k, ns, hi, P.len(qhi), srow, target);
        }
        if (nslots == 0) {   // keep first_slot strictly usable by the saturated-pair scan
            plan.first_slot.pop_back();
            plan.blocks.pop_back();
            plan.srow.resize(B.srow + 1);
            b_ids.resize(B.b_ids);
            if (r.kind != kTri) a_ids.resize(B.a_ids);
            plan.keys.erase(plan.keys.begin() + plan.tasks.size(), plan.keys.end());
        }
    }
    base[req.size()] = slots;
    if (slots == 0) return 0;
    for (auto& B : plan.blocks) {
        B.b_ids += (int64_t)a_ids.size();
        B.a_ids = (B.a_ids < 0) ? B.b_ids : B.a_ids;
    }
    plan.ids = a_ids;
    plan.ids.insert(plan.ids.end(), b_ids.begin(), b_ids.end());
    plan.nslots = slots;
    plan.pairs = slots;
    order_tasks(plan);
    int64_t maxlen_rows = 1;
    for (size_t s = 0; s + 1 < plan.srow.size(); ++s)
        maxlen_rows = std::max(maxlen_rows, plan.srow[s + 1] - plan.srow[s]);
    plan.max_warp_rows = 2 * c->rows_per_warp + 2 * maxlen_rows + 2 * target / c->W;
    return slots;
}

}  // namespace

int score_blocks(cm_ctx* c, const Prepared& P, const std::vector<int32_t>& ids,
                 const std::vector<BlockReq>& req, std::vector<int32_t>& scores,
                 std::vector<int64_t>& base, uint32_t flags)
{
    Plan plan;
    const int64_t slots = plan_blocks(c, P, ids, req, plan, base);
    scores.assign((size_t)slots, 0);
    if (slots == 0) return CM_OK;
    int32_t* out;
    ENSURE(B_OUT, slots, out);
    int r = run_plan(c, P, plan, out, nullptr, flags);
    if (r) return r;
    CUDA_TRY(cudaMemcpyAsync(scores.data(), out, slots * sizeof(int32_t), cudaMemcpyDeviceToHost,
                             c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return CM_OK;
}

int score_blocks_sig(cm_ctx* c, const Prepared& P, const std::vector<int32_t>& ids,
                     const std::vector<BlockReq>& req, int32_t T,
                     std::vector<std::pair<int64_t, int32_t>>& sig, std::vector<int64_t>& base,
                     uint32_t flags, int64_t* n_batches)
{
    if (n_batches) *n_batches = 1;
    std::vector<BlockShape> shape(req.size());
    int64_t total = 0;
    for (size_t b = 0; b < req.size(); ++b) {
        shape[b] = {req[b].kind == kTri, req[b].a_count, req[b].b_count};
        total += block_slots(shape[b]);
    }
    sig.clear();
    if (total <= c->max_batch_slots) {          // one device batch
        Plan plan;
        const int64_t slots = plan_blocks(c, P, ids, req, plan, base);
        if (slots == 0) return CM_OK;
        int32_t* out;
        ENSURE(B_OUT, slots, out);
        int r = run_plan(c, P, plan, out, nullptr, flags);
        if (r) return r;
        return compact_sig(c, out, slots, T, sig);
    }
    // Several batches, cut between query rows: each batch's significant slots are mapped back
    // to the slot numbering of the whole list, so the caller sees one batch's result.
    base.assign(req.size() + 1, 0);
    for (size_t b = 0; b < req.size(); ++b) base[b + 1] = base[b] + block_slots(shape[b]);
    const std::vector<std::vector<BlockPiece>> batches = split_batches(shape, c->max_batch_slots);
    if (n_batches) *n_batches = (int64_t)batches.size();
    for (const std::vector<BlockPiece>& batch : batches) {
        std::vector<BlockReq> sub;
        sub.reserve(batch.size());
        for (const BlockPiece& pc : batch) {
            BlockReq q = req[pc.block];
            if (q.kind != kTri) {
                q.a_begin += pc.row0;
                q.a_count = pc.rows;
            }
            sub.push_back(q);
        }
        Plan plan;
        std::vector<int64_t> sbase;
        const int64_t slots = plan_blocks(c, P, ids, sub, plan, sbase);
        if (slots == 0) continue;
        int32_t* out;
        ENSURE(B_OUT, slots, out);
        int r = run_plan(c, P, plan, out, nullptr, flags);
        if (r) return r;
        std::vector<std::pair<int64_t, int32_t>> part;
        if ((r = compact_sig(c, out, slots, T, part))) return r;
        append_batch_slots(batch, sbase, part, sig);
    }
    return CM_OK;
}

int compact_sig(cm_ctx* c, const int32_t* out, int64_t slots, int32_t T,
                std::vector<std::pair<int64_t, int32_t>>& sig)
{
    sig.clear();
    const cudaStream_t st = c->stream;
    const int64_t nch = compact_chunks(slots);
    int64_t* d_chunk;
    ENSURE(B_CHUNK, nch + 2, d_chunk);
    CUDA_TRY(launch_compact_slots(out, slots, T, nullptr, nullptr, d_chunk, nch, 0, st));
    CUDA_TRY(launch_scan_chunks(d_chunk, nch, d_chunk + nch, st));
    int64_t total = 0;
    CUDA_TRY(cudaMemcpyAsync(&total, d_chunk + nch, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    c->stats.launches += 2;
    if (total == 0) return CM_OK;
    int64_t* d_slots;
    int32_t* d_sc;
    ENSURE(B_POUT, total, d_slots);
    ENSURE(B_SOUT, total, d_sc);
    CUDA_TRY(launch_compact_slots(out, slots, T, d_slots, d_sc, d_chunk, nch, 1, st));
    c->stats.launches += 1;
    std::vector<int64_t> hs((size_t)total);
    std::vector<int32_t> hv((size_t)total);
    CUDA_TRY(cudaMemcpyAsync(hs.data(), d_slots, total * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(hv.data(), d_sc, total * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    sig.resize((size_t)total);
    for (int64_t k = 0; k < total; ++k) sig[k] = {hs[k], hv[k]};
    return CM_OK;
}

int score_pairs_int32(cm_ctx* c, const Prepared& P, const std::vector<int32_t>& pairs,
                      std::vector<int32_t>& scores)
{
    const int64_t n = (int64_t)pairs.size() / 2;
    scores.assign((size_t)n, 0);
    if (n == 0) return CM_OK;
    if (n >= ((int64_t)1 << 31)) return fail(c, CM_ERR_ARG, "too many pairs");
    const cudaStream_t st = c->stream;
    std::vector<PairRef> lst((size_t)n);
    for (int64_t k = 0; k < n; ++k) lst[k] = PairRef{pairs[2 * k], pairs[2 * k + 1], 0, 0, k};
    // long pairs first, for whole CTAs; the rest longest first on one warp each
    auto is_long = [&](const PairRef& x) {
        return P.len(x.q) >= kLongMinCols && P.len(x.x) >= kLongMinRows;
    };
    std::stable_sort(lst.begin(), lst.end(), [&](const PairRef& x, const PairRef& y) {
        const bool lx = is_long(x), ly = is_long(y);
        if (lx != ly) return lx;
        return P.len(x.q) * P.len(x.x) > P.len(y.q) * P.len(y.x);
    });
    int32_t nlong = 0;
    while (nlong < n && is_long(lst[nlong])) ++nlong;
    PairRef* d_pref;
    int32_t *d_out, *d_flags;
    uint2* d_bnd;
    ENSURE(B_PREF, n, d_pref);
    ENSURE(B_OUT, n, d_out);
    ENSURE(B_FLAGS, kFlagWords, d_flags);
    const int64_t stride = (P.maxlen + 64 + 1) & ~(int64_t)1;
    const int64_t nslot = std::max<int64_t>((int64_t)c->num_sms * kLongSlots,
                                            (int64_t)c->num_sms * std::max(1, sw32_ctas_per_sm()));
    ENSURE(B_BND, nslot * stride, d_bnd);
    int r = copy_in(c, d_pref, lst.data(), lst.size() * sizeof(PairRef), false);
    if (r) return r;
    CUDA_TRY(cudaMemsetAsync(d_flags, 0, kFlagWords * sizeof(int32_t), st));
    SwArgs a{};
    a.db = P.db;
    a.off = P.off;
    a.out = d_out;
    a.err = d_flags + 1;
    a.wait_limit = c->wait_limit;
    std::memcpy(a.mat, P.mat, sizeof(a.mat));
    a.gap_open = P.g1;
    a.gap_extend = P.ge;
    a.beta = P.beta;
    a.sat_thr = P.sat_thr;
    a.bnd = d_bnd;
    a.bnd_stride = stride;
    if (nlong > 0) {
        CUDA_TRY(launch_long_sw32((int)std::min<int64_t>(nlong, c->num_sms), a, d_pref, nlong,
                                  d_flags + 5, st));
        c->stats.launches += 1;
    }
    if (n > nlong) {
        const int grid = (int)std::min<int64_t>(n - nlong, (int64_t)c->num_sms * std::max(1, sw32_ctas_per_sm()));
        CUDA_TRY(launch_sw32(16, grid, a, d_pref + nlong, (int32_t)(n - nlong), d_flags + 3, st));
        c->stats.launches += 1;
    }
    int32_t kerr = 0;
    CUDA_TRY(cudaMemcpyAsync(scores.data(), d_out, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(&kerr, d_flags + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (kerr == 2) return fail(c, CM_ERR_TIMEOUT, "a long-pair pipeline wait gave up");
    if (kerr) return fail(c, CM_ERR_INTERNAL, "kernel bounds check fired (boundary buffer)");
    c->stats.pairs += n;
    return CM_OK;
}

int run_cells(cm_ctx* c, const Prepared& P, const int32_t* hp, int64_t n_pairs, int32_t* hcells)
{
    if (n_pairs == 0) return CM_OK;
    if (n_pairs >= ((int64_t)1 << 31)) return fail(c, CM_ERR_ARG, "n_pairs must be < 2^31");
    const cudaStream_t st = c->stream;
    // jobs longest first (the persistent warps claim them in order), pad = the pair's index
    // long jobs (many column passes) first, for whole CTAs; the rest longest first
    auto is_long = [](const CellJob& x) { return x.n >= kLongMinCols && x.m >= kLongMinRows; };
    auto lpt = [&](std::vector<CellJob>& v) {
        std::stable_sort(v.begin(), v.end(), [&](const CellJob& x, const CellJob& y) {
            const bool lx = is_long(x), ly = is_long(y);
            if (lx != ly) return lx;
            return (int64_t)x.m * x.n > (int64_t)y.m * y.n;
        });
    };
    std::vector<CellJob> jobs((size_t)n_pairs);
    for (int64_t k = 0; k < n_pairs; ++k) {
        const int32_t x = hp[2 * k], y = hp[2 * k + 1];
        jobs[k] = CellJob{x, y, (int32_t)P.len(x), (int32_t)P.len(y), 0, (int32_t)k};
    }
    lpt(jobs);
    CellJob* d_jobs;
    int32_t *d_res, *d_flags;
    uint2* d_bnd;
    ENSURE(B_JOBS, n_pairs, d_jobs);
    ENSURE(B_RES, 3 * n_pairs, d_res);
    ENSURE(B_FLAGS, kFlagWords, d_flags);
    const int occ = std::max(1, cells_wf_ctas_per_sm());
    const int grid = (int)std::min<int64_t>(n_pairs, (int64_t)c->num_sms * occ);
    const int64_t stride = P.maxlen + 64;
    ENSURE(B_BND, std::max<int64_t>(grid, (int64_t)c->num_sms * kLongSlots) * stride, d_bnd);
    SwArgs a{};
    a.db = P.db;
    a.off = P.off;
    a.bnd = d_bnd;
    a.bnd_stride = stride;
    a.err = d_flags + 1;
    a.wait_limit = c->wait_limit;
    std::memcpy(a.mat, P.mat, sizeof(a.mat));
    a.gap_open = P.g1;
    a.gap_extend = P.ge;
    std::vector<int32_t> fwd((size_t)n_pairs * 3);
    for (int dir = 0; dir < 2; ++dir) {
        int r = copy_in(c, d_jobs, jobs.data(), jobs.size() * sizeof(CellJob), false);
        if (r) return r;
        CUDA_TRY(cudaMemsetAsync(d_flags, 0, kFlagWords * sizeof(int32_t), st));
        int32_t nlong = 0;
        while (nlong < (int32_t)jobs.size() && is_long(jobs[nlong])) ++nlong;
        if (nlong > 0) {
            CUDA_TRY(launch_long_cells((int)std::min<int64_t>(nlong, c->num_sms), a, d_jobs, nlong,
                                       d_flags + 6, d_res, st));
            c->stats.launches += 1;
        }
        const int32_t nshort = (int32_t)jobs.size() - nlong;
        if (nshort > 0) {
            CUDA_TRY(launch_cells_wf((int)std::min<int64_t>(grid, nshort), a, d_jobs + nlong, nshort,
                                     d_flags + 4, d_res + 3 * (int64_t)nlong, st));
            c->stats.launches += 1;
        }
        std::vector<int32_t> res(jobs.size() * 3);
        int32_t kerr = 0;
        CUDA_TRY(cudaMemcpyAsync(res.data(), d_res, res.size() * sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaMemcpyAsync(&kerr, d_flags + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        if (kerr == 2) return fail(c, CM_ERR_TIMEOUT, "a long-pair pipeline wait gave up");
        if (kerr) return fail(c, CM_ERR_INTERNAL, "cells kernel bounds check fired");
        if (dir == 0) {
            fwd = res;
            std::vector<CellJob> rev;
            for (size_t q = 0; q < jobs.size(); ++q) {
                const int64_t k = jobs[q].pad;
                int32_t* cl = hcells + 5 * k;
                cl[0] = fwd[3 * q];
                cl[1] = cl[2] = cl[3] = cl[4] = 0;
                if (fwd[3 * q] > 0)
                    rev.push_back(CellJob{jobs[q].a, jobs[q].b, fwd[3 * q + 1] + 1,
                                          fwd[3 * q + 2] + 1, 1, (int32_t)k});
            }
            if (rev.empty()) break;
            lpt(rev);
            jobs.swap(rev);
        } else {
            for (size_t q = 0; q < jobs.size(); ++q) {
                const int64_t k = jobs[q].pad;
                int32_t* cl = hcells + 5 * k;
                const int32_t ie = jobs[q].m, je = jobs[q].n;
                cl[1] = ie - (res[3 * q + 1] + 1) + 1;
                cl[2] = ie;
                cl[3] = je - (res[3 * q + 2] + 1) + 1;
                cl[4] = je;
            }
        }
    }
    return CM_OK;
}

// Plan of part `part` of `n_parts` (about equal cell counts) of the all-against-all triangle:
// one TRI block over the sequences in length order (ties by index), so that every pair's
// query is the longer sequence.  L receives that order, k0 the first query row of the part.
void allpairs_plan(cm_ctx* c, const Prepared& P, int32_t n_seqs, int64_t part, int64_t n_parts,
                   std::vector<int32_t>& L, int32_t& k0_out, Plan& plan)
{
    L.resize((size_t)n_seqs);
    std::iota(L.begin(), L.end(), 0);
    std::stable_sort(L.begin(), L.end(), [&](int32_t x, int32_t y) {
        return P.hoff[x + 1] - P.hoff[x] < P.hoff[y + 1] - P.hoff[y];
    });
    plan.srow.resize((size_t)n_seqs + 1);
    plan.srow[0] = 0;
    for (int32_t s = 0; s < n_seqs; ++s)
        plan.srow[s + 1] = plan.srow[s] + stream_rows(P.hoff[L[s] + 1] - P.hoff[L[s]]);
    // parts: equal shares of cells, boundaries on even k
    std::vector<double> cum((size_t)n_seqs + 1, 0.0);
    int64_t residues = 0;
    for (int32_t k = 0; k < n_seqs; ++k) {
        const int64_t mk = P.hoff[L[k] + 1] - P.hoff[L[k]];
        cum[k + 1] = cum[k] + (double)mk * (double)residues;
        residues += mk;
    }
    auto kb = [&](int64_t p) -> int32_t {
        if (p <= 0) return 0;
        if (p >= n_parts) return n_seqs;
        const double want = cum[n_seqs] * (double)p / (double)n_parts;
        int32_t k = (int32_t)(std::lower_bound(cum.begin(), cum.end(), want) - cum.begin());
        k &= ~1;
        return std::min(k, n_seqs);
    };
    const int32_t k0 = kb(part), k1 = kb(part + 1);
    SwBlock B{};
    B.kind = kTri;
    B.swap = 0;
    B.na = n_seqs;
    B.nb = n_seqs;
    B.a_ids = 0;
    B.b_ids = 0;
    B.stream = 0;
    B.srow = 0;
    B.out_base = 0;
    B.k0 = k0;
    B.has_map = 0;
    plan.blocks.push_back(B);
    plan.first_slot.push_back(0);
    plan.ids = L;
    auto tri = [](int64_t k) { return k * (k - 1) / 2; };
    plan.nslots = tri(k1) - tri(k0);
    plan.pairs = plan.nslots;
    const int64_t target = (int64_t)c->W * c->rows_per_warp;
    for (int32_t k = k0; k < k1; k += 2) {
        const bool hi = (k + 1 < k1);
        const int32_t ns = hi ? k + 1 : k;
        const int64_t m_hi = P.hoff[L[hi ? k + 1 : k] + 1] - P.hoff[L[hi ? k + 1 : k]];
        if (ns > 0) add_tasks(plan, 0, k, ns, hi, m_hi, plan.srow.data(), target);
    }
    {   // cells = sum over pairs of len(a) * len(b)
        int64_t acc = 0, pre = 0;
        for (int32_t k = 0; k < k1; ++k) {
            const int64_t mk = P.hoff[L[k] + 1] - P.hoff[L[k]];
            if (k >= k0) acc += mk * pre;
            pre += mk;
        }
        plan.cells = acc;
    }
    order_tasks(plan);
    int64_t maxlen_rows = 1;
    for (int32_t s = 0; s < n_seqs; ++s)
        maxlen_rows = std::max(maxlen_rows, plan.srow[s + 1] - plan.srow[s]);
    plan.max_warp_rows = 2 * c->rows_per_warp + 2 * maxlen_rows + 2 * target / c->W;

    k0_out = k0;
}

}  // namespace cm

// =========================================================================================
extern "C" {

int cm_create(cm_ctx** out, int device)
{
    if (!out) return CM_ERR_ARG;
    *out = nullptr;
    cm_ctx* c = new (std::nothrow) cm_ctx();
    if (!c) return CM_ERR_OOM;
    c->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->own, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking);
    for (int i = 0; i < 4 && e == cudaSuccess; ++i) e = cudaEventCreate(&c->ev[i]);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->join, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        cudaGetLastError();
        c->stream = nullptr;
        cm_destroy(c);
        cudaGetLastError();
        return CM_ERR_CUDA;
    }
    c->stream = c->own;
    *out = c;
    return CM_OK;
}

void cm_destroy(cm_ctx* c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (auto& b : c->buf)
        if (b.p) cudaFree(b.p);
    if (c->ranker && c->ranker_free) c->ranker_free(c->ranker);
    for (auto& e : c->ev)
        if (e) cudaEventDestroy(e);
    if (c->fork) cudaEventDestroy(c->fork);
    if (c->join) cudaEventDestroy(c->join);
    if (c->aux) cudaStreamDestroy(c->aux);
    if (c->own) cudaStreamDestroy(c->own);
    delete c;
}

const char* cm_last_error(const cm_ctx* c) { return c ? c->err.c_str() : "null context"; }

int cm_set_stream(cm_ctx* c, void* s)
{
    if (!c) return CM_ERR_ARG;
    c->stream = s ? reinterpret_cast<cudaStream_t>(s) : c->own;
    return CM_OK;
}

int cm_set_tuning(cm_ctx* c, int32_t warps, int32_t rows)
{
    if (!c) return CM_ERR_ARG;
    if (warps && warps != 4 && warps != 8 && warps != 16)
        return fail(c, CM_ERR_ARG, "warps_per_cta must be 4, 8 or 16");
    if (rows && (rows < 256 || rows > 65536))
        return fail(c, CM_ERR_ARG, "rows_per_warp must be in [256, 65536]");
    if (warps) c->W = warps;
    if (rows) c->rows_per_warp = rows;
    return CM_OK;
}

int cm_set_batch_limit(cm_ctx* c, int64_t max_slots)
{
    if (!c) return CM_ERR_ARG;
    if (max_slots != 0 && max_slots < 1024)
        return fail(c, CM_ERR_ARG, "max_slots must be 0 or >= 1024");
    c->max_batch_slots = max_slots ? max_slots : ((int64_t)1 << 32);
    return CM_OK;
}

int cm_set_wait_limit(cm_ctx* c, int32_t polls)
{
    if (!c) return CM_ERR_ARG;
    if (polls < 0) return fail(c, CM_ERR_ARG, "polls must be >= 0 (0 restores the default)");
    c->wait_limit = polls ? polls : (1 << 24);
    return CM_OK;
}

int cm_get_stats(const cm_ctx* c, cm_stats* out)
{
    if (!c || !out) return CM_ERR_ARG;
    *out = c->stats;
    return CM_OK;
}

int cm_reset_stats(cm_ctx* c)
{
    if (!c) return CM_ERR_ARG;
    c->stats = cm_stats{};
    return CM_OK;
}

int sw_score_batch(cm_ctx* c, const uint8_t* seqs, const int64_t* offsets, int32_t n_seqs,
                   const int32_t* pairs, int64_t n_pairs, const int8_t* matrix,
                   int32_t gap_open, int32_t gap_extend, int32_t* scores_out, uint32_t flags)
{
    if (!c) return CM_ERR_ARG;
    NvtxRange range("sw_score_batch");
    CUDA_TRY(cudaSetDevice(c->device));
    if (n_pairs < 0 || (n_pairs > 0 && (!pairs || !scores_out)))
        return fail(c, CM_ERR_ARG, "bad pairs / scores_out");
    if (n_pairs >= (int64_t)1 << 31) return fail(c, CM_ERR_ARG, "n_pairs must be < 2^31");
    Prepared P;
    int r = prepare(c, seqs, offsets, n_seqs, matrix, gap_open, gap_extend, flags, P);
    if (r) return r;
    if (n_pairs == 0) return CM_OK;
    const bool dev = (flags & CM_DEVICE_PTRS) != 0;
    std::vector<int32_t> hp((size_t)n_pairs * 2);
    if (dev) CUDA_TRY(cudaMemcpy(hp.data(), pairs, hp.size() * 4, cudaMemcpyDeviceToHost));
    else std::memcpy(hp.data(), pairs, hp.size() * 4);
    for (int64_t k = 0; k < 2 * n_pairs; ++k)
        if (hp[k] < 0 || hp[k] >= n_seqs) return fail(c, CM_ERR_ARG, "pair index out of range");

    // group pairs by their first sequence: one CROSS block {a} x {b...} per distinct a
    std::vector<int64_t> ord((size_t)n_pairs);
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int64_t x, int64_t y) {
        return hp[2 * x] < hp[2 * y];
    });
    Plan plan;
    std::vector<int32_t> a_ids, b_ids;
    std::vector<int64_t> omap((size_t)n_pairs);
    plan.srow.push_back(0);
    const int64_t target = (int64_t)c->W * c->rows_per_warp;
    int64_t slot = 0;
    for (size_t g0 = 0; g0 < ord.size();) {
        size_t g1 = g0;
        const int32_t a = hp[2 * ord[g0]];
        while (g1 < ord.size() && hp[2 * ord[g1]] == a) ++g1;
        SwBlock B{};
        B.kind = kCross;
        B.swap = 0;
        B.na = 1;
        B.nb = (int32_t)(g1 - g0);
        B.a_ids = (int64_t)a_ids.size();
        B.b_ids = (int64_t)b_ids.size();       // fixed up below (after the A ids)
        B.stream = 0;
        B.srow = (int64_t)plan.srow.size() - 1;
        B.out_base = slot;
        B.k0 = 0;
        B.has_map = 1;
        a_ids.push_back(a);
        const int64_t ma = P.hoff[a + 1] - P.hoff[a];
        for (size_t g = g0; g < g1; ++g) {
            const int32_t b = hp[2 * ord[g] + 1];
            const int64_t mb = P.hoff[b + 1] - P.hoff[b];
            b_ids.push_back(b);
            plan.srow.push_back(plan.srow.back() + stream_rows(mb));
            omap[(size_t)slot++] = ord[g];
            plan.cells += ma * mb;
        }
        plan.first_slot.push_back(B.out_base);
        plan.blocks.push_back(B);
        add_tasks(plan, (int32_t)plan.blocks.size() - 1, 0, B.nb, false, ma,
                  plan.srow.data() + B.srow, target);
        g0 = g1;
    }
    for (auto& B : plan.blocks) B.b_ids += (int64_t)a_ids.size();
    plan.ids = a_ids;
    plan.ids.insert(plan.ids.end(), b_ids.begin(), b_ids.end());
    plan.nslots = n_pairs;
    plan.pairs = n_pairs;
    order_tasks(plan);
    int64_t maxlen_rows = 0;
    for (size_t s = 0; s + 1 < plan.srow.size(); ++s)
        maxlen_rows = std::max(maxlen_rows, plan.srow[s + 1] - plan.srow[s]);
    plan.max_warp_rows = 2 * c->rows_per_warp + 2 * maxlen_rows + 2 * target / c->W;

    int64_t* d_omap;
    ENSURE(B_OMAP, n_pairs, d_omap);
    if ((r = copy_in(c, d_omap, omap.data(), omap.size() * sizeof(int64_t), false))) return r;
    int32_t* out = scores_out;
    if (!dev) ENSURE(B_OUT, n_pairs, out);
    if ((r = run_plan(c, P, plan, out, d_omap, flags))) return r;
    if (!dev) {
        CUDA_TRY(cudaMemcpyAsync(scores_out, out, n_pairs * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                 c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
    }
    return CM_OK;
}

int sw_cells_batch(cm_ctx* c, const uint8_t* seqs, const int64_t* offsets, int32_t n_seqs,
                   const int32_t* pairs, int64_t n_pairs, const int8_t* matrix,
                   int32_t gap_open, int32_t gap_extend, int32_t* cells_out, uint32_t flags)
{
    if (!c) return CM_ERR_ARG;
    CUDA_TRY(cudaSetDevice(c->device));
    if (n_pairs < 0 || (n_pairs > 0 && (!pairs || !cells_out)))
        return fail(c, CM_ERR_ARG, "bad pairs / cells_out");
    Prepared P;
    int r = prepare(c, seqs, offsets, n_seqs, matrix, gap_open, gap_extend, flags, P);
    if (r) return r;
    if (n_pairs == 0) return CM_OK;
    const bool dev = (flags & CM_DEVICE_PTRS) != 0;
    std::vector<int32_t> hp((size_t)n_pairs * 2);
    if (dev) CUDA_TRY(cudaMemcpy(hp.data(), pairs, hp.size() * 4, cudaMemcpyDeviceToHost));
    else std::memcpy(hp.data(), pairs, hp.size() * 4);
    int64_t maxb = 0;
    for (int64_t k = 0; k < n_pairs; ++k) {
        if (hp[2 * k] < 0 || hp[2 * k] >= n_seqs || hp[2 * k + 1] < 0 || hp[2 * k + 1] >= n_seqs)
            return fail(c, CM_ERR_ARG, "pair index out of range");
        const int32_t b = hp[2 * k + 1];
        maxb = std::max(maxb, P.hoff[b + 1] - P.hoff[b]);
    }
    (void)maxb;
    std::vector<int32_t> hc((size_t)n_pairs * 5);
    if ((r = run_cells(c, P, hp.data(), n_pairs, hc.data()))) return r;
    CUDA_TRY(cudaMemcpyAsync(cells_out, hc.data(), hc.size() * sizeof(int32_t),
                             dev ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return CM_OK;
}

int cm_autotune(cm_ctx* c, const uint8_t* seqs, const int64_t* offsets, int32_t n_seqs,
                const int8_t* matrix, int32_t gap_open, int32_t gap_extend, int32_t sample_seqs,
                const char* cache_path, int32_t* warps_out, int32_t* rows_out, uint32_t flags)
{
    if (!c) return CM_ERR_ARG;
    CUDA_TRY(cudaSetDevice(c->device));
    Prepared P;
    int r = prepare(c, seqs, offsets, n_seqs, matrix, gap_open, gap_extend, flags, P);
    if (r) return r;
    if (n_seqs < 2) return fail(c, CM_ERR_ARG, "autotune needs at least 2 sequences");
    // length profile of the set: median length bucket (powers of two)
    std::vector<int64_t> lens((size_t)n_seqs);
    for (int32_t i = 0; i < n_seqs; ++i) lens[i] = P.len(i);
    std::vector<int64_t> sl = lens;
    std::nth_element(sl.begin(), sl.begin() + sl.size() / 2, sl.end());
    int bucket = 0;
    while (bucket < 30 && ((int64_t)1 << bucket) < sl[sl.size() / 2]) ++bucket;
    cudaDeviceProp prop;
    CUDA_TRY(cudaGetDeviceProperties(&prop, c->device));
    char key[sizeof(prop.name) + 32];          // name, SM count and bucket always fit
    std::snprintf(key, sizeof(key), "%s|%d|%d", prop.name, prop.multiProcessorCount, bucket);
    for (char* q = key; *q; ++q)
        if (*q == ' ') *q = '_';
    if (cache_path) {
        FILE* f = std::fopen(cache_path, "r");
        if (f) {
            char k2[256];
            int w = 0, rw = 0;
            while (std::fscanf(f, "%255s %d %d", k2, &w, &rw) == 3) {
                if (std::strcmp(k2, key) == 0 && cm_set_tuning(c, w, rw) == CM_OK) {
                    std::fclose(f);
                    if (warps_out) *warps_out = c->W;
                    if (rows_out) *rows_out = c->rows_per_warp;
                    return CM_OK;
                }
            }
            std::fclose(f);
        }
    }
    // timing sample: the middle part of the caller's own all-against-all, so that query
    // lengths and subject-stream lengths are those of the real workload
    (void)sample_seqs;
    std::vector<int32_t> Lord;
    Plan plan0;
    int32_t k0 = 0;
    const int64_t nparts = std::max<int64_t>(1, std::min<int64_t>(256, n_seqs / 4));
    allpairs_plan(c, P, n_seqs, nparts / 2, nparts, Lord, k0, plan0);
    if (plan0.tasks.empty()) return fail(c, CM_ERR_ARG, "autotune sample is empty");
    int32_t* d_out;
    ENSURE(B_OUT, plan0.nslots, d_out);
    const int Ws[3] = {4, 8, 16};
    const int Rs[4] = {4096, 8192, 16384, 32768};
    const int W0 = c->W, R0 = c->rows_per_warp;
    double best_rate = -1.0;
    int bw = W0, brw = R0;
    for (int wi = 0; wi < 3; ++wi)
        for (int ri = 0; ri < 4; ++ri) {
            c->W = Ws[wi];
            c->rows_per_warp = Rs[ri];
            double ms = 0.0;
            int64_t cells = 0;
            Plan plan;
            allpairs_plan(c, P, n_seqs, nparts / 2, nparts, Lord, k0, plan);
            for (int rep = 0; rep < 2; ++rep) {       // first run warms up, second is timed
                const double ms0 = c->stats.sw16_ms;
                const int64_t c0 = c->stats.cells;
                r = run_plan(c, P, plan, d_out, nullptr, flags);
                if (r) { c->W = W0; c->rows_per_warp = R0; return r; }
                ms = c->stats.sw16_ms - ms0;
                cells = c->stats.cells - c0;
            }
            const double rate = ms > 0 ? (double)cells / ms : 0.0;
            if (rate > best_rate) { best_rate = rate; bw = Ws[wi]; brw = Rs[ri]; }
        }
    c->W = bw;
    c->rows_per_warp = brw;
    if (cache_path) {
        FILE* f = std::fopen(cache_path, "a");
        if (f) {
            std::fprintf(f, "%s %d %d\n", key, bw, brw);
            std::fclose(f);
        }
    }
    if (warps_out) *warps_out = bw;
    if (rows_out) *rows_out = brw;
    return CM_OK;
}

int sw_allpairs(cm_ctx* c, const uint8_t* seqs, const int64_t* offsets, int32_t n_seqs,
                const int8_t* matrix, int32_t gap_open, int32_t gap_extend, int32_t T,
                int64_t part, int64_t n_parts, int32_t* pairs_out, int32_t* scores_out,
                int64_t capacity, int64_t* n_found, uint32_t flags)
{
    if (!c) return CM_ERR_ARG;
    NvtxRange range("sw_allpairs");
    CUDA_TRY(cudaSetDevice(c->device));
    if (!n_found || n_parts < 1 || part < 0 || part >= n_parts || capacity < 0 ||
        (capacity > 0 && (!pairs_out || !scores_out)))
        return fail(c, CM_ERR_ARG, "bad part / capacity / output arguments");
    *n_found = 0;
    Prepared P;
    int r = prepare(c, seqs, offsets, n_seqs, matrix, gap_open, gap_extend, flags, P);
    if (r) return r;
    if (!P.symmetric) return fail(c, CM_ERR_ARG, "sw_allpairs needs a symmetric matrix");
    const bool dev = (flags & CM_DEVICE_PTRS) != 0;
    CUDA_TRY(cudaEventRecord(c->ev[2], c->stream));
    std::vector<int32_t> L;
    Plan plan;
    int32_t k0 = 0;
    allpairs_plan(c, P, n_seqs, part, n_parts, L, k0, plan);
    int32_t* out;
    ENSURE(B_OUT, plan.nslots, out);
    if (!plan.tasks.empty())
        if ((r = run_plan(c, P, plan, out, nullptr, flags))) return r;

    // compaction of f > T (deterministic order: slot order)
    const int64_t nch = compact_chunks(plan.nslots);
    int64_t* d_chunk;
    ENSURE(B_CHUNK, nch + 2, d_chunk);
    int32_t* d_order;
    ENSURE(B_IDS, plan.ids.size(), d_order);   // already uploaded by run_plan (same pool)
    if (plan.tasks.empty())
        if ((r = copy_in(c, d_order, L.data(), L.size() * 4, false))) return r;
    CUDA_TRY(launch_compact_tri(out, plan.nslots, k0, d_order, T, nullptr, nullptr, d_chunk, nch,
                                0, c->stream));
    CUDA_TRY(launch_scan_chunks(d_chunk, nch, d_chunk + nch, c->stream));
    int64_t total = 0;
    CUDA_TRY(cudaMemcpyAsync(&total, d_chunk + nch, sizeof(int64_t), cudaMemcpyDeviceToHost,
                             c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    c->stats.launches += 2;
    *n_found = total;
    if (total > capacity) return fail(c, CM_ERR_CAPACITY, "capacity too small for the significant pairs");
    int32_t *po = pairs_out, *so = scores_out;
    if (!dev) {
        ENSURE(B_POUT, 2 * std::max<int64_t>(total, 1), po);
        ENSURE(B_SOUT, std::max<int64_t>(total, 1), so);
    }
    CUDA_TRY(launch_compact_tri(out, plan.nslots, k0, d_order, T, po, so, d_chunk, nch, 1,
                                c->stream));
    c->stats.launches += 1;
    if (!dev && total > 0) {
        CUDA_TRY(cudaMemcpyAsync(pairs_out, po, 2 * total * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                 c->stream));
        CUDA_TRY(cudaMemcpyAsync(scores_out, so, total * sizeof(int32_t), cudaMemcpyDeviceToHost,
                                 c->stream));
    }
    CUDA_TRY(cudaEventRecord(c->ev[3], c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, c->ev[2], c->ev[3]));
    c->stats.total_ms += ms;
    return CM_OK;
}

}  // extern "C"
