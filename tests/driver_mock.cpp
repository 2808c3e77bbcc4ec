// Host harness for the ClusterMerge driver (csrc/cluster_merge.cu, compiled here as plain C++):
// every function the driver calls into the device layer is replaced by a host mock that
// computes the documented result from a given similarity: f(x, y) = M[x][y], and the
// alignment of (x, y) covering residues 1..cov[x][y] of x and 1..cov[y][x] of y.  The ranked
// path's selection bitmap comes from a given keep[x][y].  The mocks also check that every
// output slot of a plan is written exactly once.
//
// Input (stdin, whitespace separated): K instances, each
//   n T mT mU use_ranker ranker_min_pairs merge_mode algorithm (0 cluster_merge, 1 greedy,
//   2 cluster_merge_resume stopping after every round; argv[1] = the state file)
//   len[n]  M[n*n]  cov[n*n]  keep[n*n]
// Output per instance: "clusters C" then C lines "rep size members...", "pairs P" then P lines
// "i j s", then "stats rep exchange intra full_merges exchanges merges", or "error code msg".
#include <cstdio>
#include <cstring>
#include <iostream>
#include <map>
#include <string>
#include <vector>

#include "ctx.h"
#include "mock_ranked.h"

using namespace cm;

namespace {

struct Instance {
    int32_t n = 0;
    std::vector<int64_t> len, off;
    std::vector<int32_t> M, cov;
    std::vector<char> keep;
    int32_t at(const std::vector<int32_t>& A, int32_t x, int32_t y) const
    {
        return A[(size_t)x * n + y];
    }
};

const Instance* g = nullptr;
std::map<int, std::vector<char>> g_buf;             // mock device buffers by BufId
int g_dummy;

int64_t tri(int64_t k) { return k * (k - 1) / 2; }

int32_t pair_score(int32_t x, int32_t y, int32_t swap)
{
    return swap ? g->at(g->M, y, x) : g->at(g->M, x, y);
}

// slot layout of score_blocks: blocks in order, CROSS k * nb + s, TRI k (k - 1) / 2 + s
void all_scores(const std::vector<int32_t>& ids, const std::vector<BlockReq>& req,
                std::vector<int32_t>& scores, std::vector<int64_t>& base)
{
    base.assign(req.size() + 1, 0);
    scores.clear();
    for (size_t b = 0; b < req.size(); ++b) {
        const BlockReq& r = req[b];
        if (r.kind == kTri) {
            for (int64_t k = 1; k < r.a_count; ++k)
                for (int64_t s = 0; s < k; ++s)
                    scores.push_back(pair_score(ids[r.a_begin + k], ids[r.a_begin + s], r.swap));
        } else {
            for (int64_t k = 0; k < r.a_count; ++k)
                for (int64_t s = 0; s < r.b_count; ++s)
                    scores.push_back(pair_score(ids[r.a_begin + k], ids[r.b_begin + s], r.swap));
        }
        base[b + 1] = (int64_t)scores.size();
    }
}

}  // namespace

// ---- CUDA runtime calls the driver makes directly -------------------------------------
extern "C" {
cudaError_t cudaSetDevice(int) { return cudaSuccess; }
cudaError_t cudaStreamSynchronize(cudaStream_t) { return cudaSuccess; }
cudaError_t cudaMemcpyAsync(void* d, const void* s, size_t n, cudaMemcpyKind, cudaStream_t)
{
    std::memcpy(d, s, n);
    return cudaSuccess;
}
cudaError_t cudaMemsetAsync(void* d, int v, size_t n, cudaStream_t)
{
    std::memset(d, v, n);
    return cudaSuccess;
}
const char* cudaGetErrorString(cudaError_t) { return "mock"; }
}

// ---- the device layer --------------------------------------------------------------------
namespace cm {

int fail(cm_ctx* c, int code, const std::string& msg)
{
    if (c) c->err = msg;
    return code;
}

int ensure_bytes(cm_ctx*, BufId id, size_t bytes, void** out)
{
    std::vector<char>& b = g_buf[id];
    if (b.size() < bytes + 16) b.resize(bytes + 16);
    *out = b.data();
    return CM_OK;
}

int copy_in(cm_ctx*, void* dst, const void* src, size_t bytes, bool)
{
    if (bytes) std::memcpy(dst, src, bytes);
    return CM_OK;
}

int prepare(cm_ctx* c, const uint8_t*, const int64_t* offsets, int32_t n_seqs, const int8_t*,
            int32_t, int32_t, uint32_t, Prepared& P)
{
    c->err.clear();
    P.hoff.assign(offsets, offsets + n_seqs + 1);
    P.off = P.hoff.data();                      // the mocks read offsets on the host
    P.symmetric = true;
    for (int32_t i = 0; i < n_seqs; ++i) P.maxlen = std::max(P.maxlen, P.len(i));
    return CM_OK;
}

int score_blocks(cm_ctx*, const Prepared&, const std::vector<int32_t>& ids,
                 const std::vector<BlockReq>& req, std::vector<int32_t>& scores,
                 std::vector<int64_t>& base, uint32_t)
{
    all_scores(ids, req, scores, base);
    return CM_OK;
}

int score_blocks_sig(cm_ctx*, const Prepared&, const std::vector<int32_t>& ids,
                     const std::vector<BlockReq>& req, int32_t T,
                     std::vector<std::pair<int64_t, int32_t>>& sig, std::vector<int64_t>& base,
                     uint32_t, int64_t* n_batches)
{
    std::vector<int32_t> s;
    all_scores(ids, req, s, base);
    sig.clear();
    for (size_t i = 0; i < s.size(); ++i)
        if (s[i] > T) sig.push_back({(int64_t)i, s[i]});
    if (n_batches) *n_batches = 1;
    return CM_OK;
}

int compact_sig(cm_ctx*, const int32_t* out, int64_t slots, int32_t T,
                std::vector<std::pair<int64_t, int32_t>>& sig)
{
    sig.clear();
    for (int64_t i = 0; i < slots; ++i)
        if (out[i] > T) sig.push_back({i, out[i]});
    return CM_OK;
}

// the persistent kernel's work: every task's queries against its subjects, into the block slots
int run_plan(cm_ctx* c, const Prepared&, Plan& plan, int32_t* out, const int64_t* omap, uint32_t)
{
    std::vector<int32_t> pool = plan.ids;
    if (plan.dev_lists) {
        const int32_t* d = reinterpret_cast<const int32_t*>(g_buf[B_IDS].data());
        pool.assign(d, d + plan.ids.size() + plan.n_sub);
        for (size_t i = 0; i < plan.ids.size(); ++i) pool[i] = plan.ids[i];
    }
    std::vector<int> written((size_t)plan.nslots, 0);
    for (const SwTask& t : plan.tasks) {
        const SwBlock& B = plan.blocks[t.block];
        for (int32_t q = t.k; q <= t.k + (t.hi_valid ? 1 : 0); ++q)
            for (int32_t s = t.s0; s < t.s1; ++s) {
                if (B.kind == kTri && s >= q) continue;
                int64_t slot = B.out_base + (B.kind == kTri ? tri(q) - tri(B.k0) + s
                                                            : (int64_t)(q - B.k0) * B.nb + s);
                if (B.has_map) slot = omap[slot];
                if (slot < 0 || slot >= plan.nslots) return fail(c, CM_ERR_INTERNAL, "mock: slot out of range");
                out[slot] = pair_score(pool[B.a_ids + q], pool[B.b_ids + s], B.swap);
                ++written[slot];
            }
    }
    for (int64_t i = 0; i < plan.nslots; ++i)
        if (written[i] != 1) return fail(c, CM_ERR_INTERNAL, "mock: slot written " +
                                         std::to_string(written[i]) + " times");
    return CM_OK;
}

int g_int32_pairs = 0;                               // pairs scored by score_pairs_int32

int score_pairs_int32(cm_ctx*, const Prepared&, const std::vector<int32_t>& pairs,
                      std::vector<int32_t>& scores)
{
    scores.resize(pairs.size() / 2);
    for (size_t k = 0; k < scores.size(); ++k) scores[k] = pair_score(pairs[2 * k], pairs[2 * k + 1], 0);
    g_int32_pairs += (int)scores.size();
    return CM_OK;
}

int run_cells(cm_ctx*, const Prepared&, const int32_t* hp, int64_t n_pairs, int32_t* hcells)
{
    for (int64_t k = 0; k < n_pairs; ++k) {
        const int32_t x = hp[2 * k], y = hp[2 * k + 1];
        int32_t* cl = hcells + 5 * k;
        cl[0] = g->at(g->M, x, y);
        cl[1] = 1;
        cl[2] = g->at(g->cov, x, y);
        cl[3] = 1;
        cl[4] = g->at(g->cov, y, x);
        if (cl[0] <= 0) cl[1] = cl[2] = cl[3] = cl[4] = 0;
    }
    return CM_OK;
}

int ranker_unit_vectors(cm_ctx*, const Prepared&, int64_t, void** U_out)
{
    *U_out = &g_dummy;
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

}  // namespace cm

int main(int argc, char** argv)
{
    const char* state_path = argc > 1 ? argv[1] : "driver_mock.state";
    int K = 0;
    std::cin >> K;
    for (int inst = 0; inst < K; ++inst) {
        Instance I;
        int32_t T, mT, mU, use_ranker, min_pairs;
        int merge_mode = 0, algorithm = 0;
        std::cin >> I.n >> T >> mT >> mU >> use_ranker >> min_pairs >> merge_mode >> algorithm;
        const size_t nn = (size_t)I.n * I.n;
        I.len.resize(I.n);
        I.off.assign(I.n + 1, 0);
        for (int32_t i = 0; i < I.n; ++i) {
            std::cin >> I.len[i];
            I.off[i + 1] = I.off[i] + I.len[i];
        }
        I.M.resize(nn);
        I.cov.resize(nn);
        I.keep.resize(nn);
        for (auto& v : I.M) std::cin >> v;
        for (auto& v : I.cov) std::cin >> v;
        for (auto& v : I.keep) { int b; std::cin >> b; v = (char)b; }
        g = &I;
        g_buf.clear();
        mock::selection().keep = [](int32_t x, int32_t y) { return g->keep[(size_t)x * g->n + y] != 0; };
        cm_ctx ctx;
        ctx.greedy_chunk = 1 + (int32_t)((I.n * 7 + T) % 9);     // several chunks per instance
        ctx.chunk_pairs = 1 + (I.n * 3 + mU) % 7;                // rep waves in column ranges
        ctx.rep_chunks = 2 + (I.n + mT) % 4;
        cm_params prm{};
        prm.T = T;
        prm.mT = mT;
        prm.mU = mU;
        prm.use_ranker = use_ranker;
        prm.prune_logit = 0.f;
        prm.ranker_min_pairs = min_pairs;
        prm.merge_mode = merge_mode;
        int8_t mat[400] = {};
        uint8_t dummy = 0;
        cm_result* res = nullptr;
        int r = 0;
        if (algorithm == 1) {
            r = greedy_cluster(&ctx, &dummy, I.off.data(), I.n, mat, 11, 1, &prm, &res, 0);
        } else if (algorithm == 2) {
            // checkpointed run: stop after every round, resume from the state file
            std::remove(state_path);
            int calls = 0;
            do {
                r = cluster_merge_resume(&ctx, &dummy, I.off.data(), I.n, mat, 11, 1, &prm,
                                         state_path, 1e-12, &res, 0);
                ++calls;
            } while (r == CM_STOPPED && calls < 64);
            if (r == CM_OK && calls > 1) {
                // a truncated checkpoint is refused, and so is one of another problem
                {
                    FILE* f = std::fopen(state_path, "rb");
                    std::vector<char> bytes;
                    if (f) {
                        int ch;
                        while ((ch = std::fgetc(f)) != EOF) bytes.push_back((char)ch);
                        std::fclose(f);
                    }
                    const std::string cut = std::string(state_path) + ".cut";
                    FILE* g2 = std::fopen(cut.c_str(), "wb");
                    if (g2) {
                        std::fwrite(bytes.data(), 1, bytes.size() / 2, g2);
                        std::fclose(g2);
                    }
                    cm_result* res3 = nullptr;
                    const int r3 = cluster_merge_resume(&ctx, &dummy, I.off.data(), I.n, mat, 11, 1,
                                                        &prm, cut.c_str(), 0.0, &res3, 0);
                    std::remove(cut.c_str());
                    if (r3 != CM_ERR_ARG || res3) {
                        std::printf("error %d truncated checkpoint accepted\n", r3);
                        cm_result_free(res3);
                        cm_result_free(res);
                        continue;
                    }
                }
                cm_params other = prm;
                other.T += 1;
                cm_result* res2 = nullptr;
                const int r2 = cluster_merge_resume(&ctx, &dummy, I.off.data(), I.n, mat, 11, 1,
                                                    &other, state_path, 0.0, &res2, 0);
                if (r2 != CM_ERR_ARG || res2) {
                    std::printf("error %d foreign checkpoint accepted\n", r2);
                    cm_result_free(res);
                    continue;
                }
            }
            if (r == CM_OK) std::fprintf(stderr, "resumed %d\n", calls);
        } else {
            r = cluster_merge(&ctx, &dummy, I.off.data(), I.n, mat, 11, 1, &prm, &res, 0);
        }
        if (r) {
            std::printf("error %d %s\n", r, ctx.err.c_str());
            continue;
        }
        std::printf("clusters %d\n", res->n_clusters);
        for (int32_t k = 0; k < res->n_clusters; ++k) {
            std::printf("%d %lld", res->reps[k], (long long)(res->cl_offsets[k + 1] - res->cl_offsets[k]));
            for (int64_t j = res->cl_offsets[k]; j < res->cl_offsets[k + 1]; ++j)
                std::printf(" %d", res->members[j]);
            std::printf("\n");
        }
        std::printf("pairs %lld\n", (long long)res->n_pairs);
        for (int64_t k = 0; k < res->n_pairs; ++k)
            std::printf("%d %d %d\n", res->pairs[2 * k], res->pairs[2 * k + 1], res->scores[k]);
        std::printf("stats %lld %lld %lld %lld %lld %lld\n", (long long)res->rep_comparisons,
                    (long long)res->exchange_comparisons, (long long)res->intra_comparisons,
                    (long long)res->full_merges, (long long)res->exchanges, (long long)res->merges);
        cm_result_free(res);
    }
    std::fprintf(stderr, "int32 pairs %d\n", g_int32_pairs);
    return 0;
}
