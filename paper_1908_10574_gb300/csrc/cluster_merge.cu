// ClusterMerge driver: Algorithm 2 (BottomUpMerge) over Algorithm 1 (Merge) with the protein
// transitivity test of Sec. 4, then the intra-cluster all-against-all of Sec. 6.1, with every
// alignment scored on the GPU in device batches.
//
// Determinism.  Algorithm 2's FIFO fixes which sets each merge combines, independently of the
// data, so the merges form a DAG; merges whose inputs are ready form one round and are
// independent (the paper's tree-level parallelism, Sec. 5).  Inside a merge, Algorithm 1 is
// sequential, but
//   * its control flow (which cluster pairs are compared, which ones fully merge, which ones
//     exchange) depends only on the representatives' scores and alignment cells, and a
//     cluster's representative never changes, so every rep x rep score of a merge can be
//     computed up front (one CROSS block per merge) and the control flow replayed on the host;
//   * membership changes only by appends, so the (member, rep) scores an exchange needs are
//     requested for the members known so far; a replay that finds every score it needs is the
//     exact sequential result.  A few such waves resolve a round.
// The result (clusters, member order, similar pairs, logical comparison counts) equals the
// plain sequential algorithm's; speculation only adds alignments that are never looked at.
#include <algorithm>
#include <cstdio>
#include <string>
#include <cmath>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <numeric>
#include <unordered_map>
#include <unordered_set>

#include "ctx.h"

namespace cm {
namespace {

struct Cluster {
    int32_t rep;
    std::vector<int32_t> objs;           // insertion order, rep first
    std::unordered_set<int32_t> mem;
    void add(int32_t x)
    {
        if (mem.insert(x).second) objs.push_back(x);
    }
};

struct Merge {
    int32_t left, right, out;
};

enum EvKind : int32_t { kAbsorbInto2 = 0, kAbsorbInto1 = 1, kExchange = 2 };

struct Event {
    int32_t kind, i1, i2, s;
};

inline uint64_t key2(int32_t a, int32_t b) { return ((uint64_t)(uint32_t)a << 32) | (uint32_t)b; }

// Longest sequence streamed as a subject (one warp's rows); longer ones are made queries.
constexpr int64_t kLongSubject = 4096;

// a rep x rep pair of a merge with s > T: cs1 index, cs2 index, score
struct SigPair {
    int32_t i1, i2, s;
    bool operator<(const SigPair& o) const { return i1 != o.i1 ? i1 < o.i1 : i2 < o.i2; }
};

inline double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Driver {
    cm_ctx* c;
    const Prepared& P;
    cm_params prm;
    uint32_t flags;
    std::vector<Cluster> arena;                      // all clusters ever created
    std::vector<std::vector<int32_t>> sets;          // set id -> cluster indices
    std::unordered_map<uint64_t, int32_t> memo;      // (member, rep) -> score
    int64_t rep_cmp = 0, exch_cmp = 0, full_merges = 0, exchanges = 0, scored = 0;
    int64_t cells_pairs = 0, batches = 0, rounds = 0, merges = 0, waves = 0;
    double t_rep = 0, t_cells = 0, t_exch = 0, t_intra = 0, t_rank = 0;
    void* U = nullptr;                               // ranker unit vectors (device), or null
    int64_t selected = 0;

    Driver(cm_ctx* c_, const Prepared& P_, const cm_params& p, uint32_t f)
        : c(c_), P(P_), prm(p), flags(f) {}

    std::vector<int32_t> by_length(std::vector<int32_t> v) const
    {
        std::stable_sort(v.begin(), v.end(),
                         [&](int32_t x, int32_t y) { return P.len(x) < P.len(y); });
        return v;
    }

    int run_round(const std::vector<Merge>& ms);
    bool partial_mode() const { return prm.merge_mode == CM_MERGE_PARTIAL; }
    int score_ranked(const std::vector<Merge>& ms, const std::vector<char>& ranked,
                     const std::vector<uint32_t>& bitmap, const std::vector<int64_t>& bitbase,
                     const std::vector<int64_t>& words, const std::vector<int64_t>& repb0,
                     const uint32_t* d_bits, const int32_t* d_reps,
                     std::vector<std::vector<SigPair>>& sigm);
    int finish(std::vector<int32_t>& final_set, cm_result* res);
    int run_greedy(int32_t n, int32_t chunk, std::vector<int32_t>& final_set);

    // One merge's events as independent partial merges (CM_MERGE_PARTIAL): every event reads
    // the cs2 cluster as the merge began; additions to cs2 clusters are applied after all
    // events, in event (cs1) order.  Scores not in the memo are requested, as in the
    // sequential replay.
    void replay_partial(const std::vector<int32_t>& cs1, const std::vector<int32_t>& cs2,
                        const std::vector<Event>& evs,
                        std::unordered_map<int32_t, std::vector<int32_t>>& need,
                        std::unordered_set<uint64_t>& needed, int64_t& lookups)
    {
        std::unordered_map<int32_t, std::vector<int32_t>> view, added;   // by cs2 index
        for (const Event& ev : evs)
            if (!view.count(ev.i2)) view[ev.i2] = arena[cs2[ev.i2]].objs;
        auto score_of = [&](int32_t x, int32_t rep, int32_t self_rep, int32_t s, int32_t* out) {
            if (x == self_rep) { *out = s; return true; }
            ++lookups;
            auto it = memo.find(key2(x, rep));
            if (it == memo.end()) {
                if (needed.insert(key2(x, rep)).second) need[rep].push_back(x);
                return false;
            }
            *out = it->second;
            return true;
        };
        for (const Event& ev : evs) {
            Cluster& c1 = arena[cs1[ev.i1]];
            const std::vector<int32_t>& v2 = view[ev.i2];
            std::vector<int32_t>& add2 = added[ev.i2];
            const int32_t rep2 = arena[cs2[ev.i2]].rep;
            if (ev.kind == kAbsorbInto2) {
                add2.insert(add2.end(), c1.objs.begin(), c1.objs.end());
            } else if (ev.kind == kAbsorbInto1) {
                for (int32_t x : v2) c1.add(x);
            } else {
                // the partial merge's own copy of c2, then ExchangeSimilar on it
                std::unordered_set<int32_t> vmem(v2.begin(), v2.end());
                const std::vector<int32_t> s1 = c1.objs;
                for (int32_t x : s1) {
                    if (vmem.count(x)) continue;
                    int32_t sm;
                    if (!score_of(x, rep2, c1.rep, ev.s, &sm)) continue;
                    if (sm > prm.T) {
                        vmem.insert(x);
                        add2.push_back(x);
                    }
                }
                for (int32_t x : v2) {
                    if (c1.mem.count(x)) continue;
                    int32_t sm;
                    if (!score_of(x, c1.rep, rep2, ev.s, &sm)) continue;
                    if (sm > prm.T) c1.add(x);
                }
            }
        }
        std::vector<int32_t> touched;
        for (const auto& kv : added) touched.push_back(kv.first);
        std::sort(touched.begin(), touched.end());
        for (int32_t i2 : touched)
            for (int32_t x : added[i2]) arena[cs2[i2]].add(x);
    }
};

int Driver::run_round(const std::vector<Merge>& ms)
{
    const size_t nm = ms.size();
    char label[64];
    std::snprintf(label, sizeof(label), "cm round %lld (%zu merges)", (long long)rounds, nm);
    NvtxRange range(label);
    // ---- wave 1: rep x rep scores.  Every merge's full cross product is one CROSS block
    // (queries = cs1 reps by length).  With the ranker, merges whose cross product has at
    // least ranker_min_pairs pairs align only the pairs whose ranker logit reaches
    // prune_logit (one single-query block per cs1 rep); Algorithm 1 still visits cs2 in set
    // order, so the ranker changes which pairs are aligned, never the order of the loop. ----
    std::vector<int64_t> base;
    std::vector<char> ranked(nm, 0);
    double t0 = now_s();
    int r;
    std::vector<uint32_t> bitmap;
    std::vector<int64_t> bitbase(nm, 0), words(nm, 0), repb0(nm, 0);
    const uint32_t* d_bits = nullptr;
    const int32_t* d_reps = nullptr;
    if (U) {
        std::vector<int32_t> rows;
        std::vector<SelTile> tiles;
        int64_t nwords = 0;
        for (size_t m = 0; m < nm; ++m) {
            const auto& cs1 = sets[ms[m].left];
            const auto& cs2 = sets[ms[m].right];
            if ((int64_t)cs1.size() * (int64_t)cs2.size() < (int64_t)prm.ranker_min_pairs) continue;
            ranked[m] = 1;
            words[m] = ((int64_t)cs2.size() + 31) / 32;
            bitbase[m] = nwords;
            nwords += words[m] * (int64_t)cs1.size();
            const int32_t a0 = (int32_t)rows.size();
            for (int32_t ci : cs1) rows.push_back(arena[ci].rep);
            const int32_t b0 = (int32_t)rows.size();
            repb0[m] = b0;
            for (int32_t ci : cs2) rows.push_back(arena[ci].rep);
            for (int32_t i0 = 0; i0 < (int32_t)cs1.size(); i0 += 128)
                for (int32_t j0 = 0; j0 < (int32_t)cs2.size(); j0 += 128) {
                    SelTile t{};
                    t.block = (int32_t)m;
                    t.i0 = i0;
                    t.j0 = j0;
                    t.na = std::min<int32_t>(128, (int32_t)cs1.size() - i0);
                    t.nb = std::min<int32_t>(128, (int32_t)cs2.size() - j0);
                    t.a = a0 + i0;
                    t.b = b0 + j0;
                    t.words = (int32_t)words[m];
                    t.bits = bitbase[m];
                    tiles.push_back(t);
                }
        }
        if (!tiles.empty()) {
            const double tr = now_s();
            r = ranker_select(c, U, rows, tiles, prm.prune_logit, nwords, bitmap, &d_bits, &d_reps);
            if (r) return r;
            t_rank += now_s() - tr;
            ++batches;
        }
    }
    // Plain merges: queries = cs1 reps (length order) against the cs2 reps in set order.  A
    // subject is one warp's stream and cannot be split, so cs2 reps longer than kLongSubject
    // become queries of a second block against the cs1 reps instead (f is symmetric here).
    std::vector<std::vector<int32_t>> qorder(nm), sorder(nm);   // block rows / subjects -> index
    std::vector<std::vector<int32_t>> lorder(nm);                 // long cs2 reps (queries)
    for (size_t m = 0; m < nm; ++m) {
        const auto& cs1 = sets[ms[m].left];
        const auto& cs2 = sets[ms[m].right];
        if (ranked[m]) continue;
        auto by_len = [&](const std::vector<int32_t>& cs, std::vector<int32_t>& order) {
            std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
                return P.len(arena[cs[x]].rep) < P.len(arena[cs[y]].rep);
            });
        };
        std::vector<int32_t>& order = qorder[m];
        order.resize(cs1.size());
        std::iota(order.begin(), order.end(), 0);
        by_len(cs1, order);
        for (int32_t i2 = 0; i2 < (int32_t)cs2.size(); ++i2)
            (P.len(arena[cs2[i2]].rep) > kLongSubject ? lorder[m] : sorder[m]).push_back(i2);
        by_len(cs2, lorder[m]);
    }
    // only the pairs with s > T can act in Algorithm 1 (every other visit is a `continue`),
    // so only they come back from the device.  A plain merge of at least 2 chunk_pairs rep
    // pairs scores cs2 in column ranges of at least chunk_pairs pairs (at most rep_chunks
    // ranges): after each range the replay restricted to the columns scored so far is exact
    // (a cs2 cluster an earlier row merged was merged at a column already scored), so the rows
    // that broke are known and the later ranges skip them -- Algorithm 1 never visits the
    // rest of a row after its cluster is absorbed.
    std::vector<std::vector<SigPair>> sigm(nm);       // per merge: (i1, i2, s), s > T
    std::vector<int32_t> cp;                          // candidate full merges: rep pairs
    std::vector<std::vector<std::pair<uint64_t, int64_t>>> cidx(nm);   // (i1, i2) -> cp index / 2
    std::vector<std::unordered_set<uint64_t>> have_cells(nm);
    std::vector<int32_t> cells;
    auto add_cells = [&](bool only_chunked, const std::vector<int32_t>& nchunks) -> int {
        const size_t first = cp.size() / 2;
        for (size_t m = 0; m < nm; ++m) {
            if (only_chunked && nchunks[m] < 2) continue;
            const auto& cs1 = sets[ms[m].left];
            const auto& cs2 = sets[ms[m].right];
            for (const SigPair& e : sigm[m])
                if (e.s > prm.mT && have_cells[m].insert(key2(e.i1, e.i2)).second) {
                    cidx[m].push_back({key2(e.i1, e.i2), (int64_t)cp.size() / 2});
                    cp.push_back(arena[cs1[e.i1]].rep);
                    cp.push_back(arena[cs2[e.i2]].rep);
                }
        }
        const size_t nnew = cp.size() / 2 - first;
        if (nnew == 0) return CM_OK;
        cells.resize(cp.size() / 2 * 5);
        const double tc0 = now_s();
        const int rc = run_cells(c, P, cp.data() + 2 * first, (int64_t)nnew, cells.data() + 5 * first);
        if (rc) return rc;
        t_cells += now_s() - tc0;
        cells_pairs += (int64_t)nnew;
        ++batches;
        return CM_OK;
    };
    auto transit = [&](size_t m, const std::unordered_map<uint64_t, int64_t>& cmap, int32_t i1,
                       int32_t i2, bool* t21, bool* t12) {
        const auto& cs1 = sets[ms[m].left];
        const auto& cs2 = sets[ms[m].right];
        const int32_t* cl = &cells[cmap.at(key2(i1, i2)) * 5];
        const int64_t la = P.len(arena[cs1[i1]].rep), lb = P.len(arena[cs2[i2]].rep);
        const int64_t ua = cl[0] ? la - (cl[2] - cl[1] + 1) : la;
        const int64_t ub = cl[0] ? lb - (cl[4] - cl[3] + 1) : lb;
        *t21 = ua < prm.mU;
        *t12 = ub < prm.mU;
    };
    std::vector<int32_t> nchunks(nm, 1);
    int32_t max_chunks = 1;
    for (size_t m = 0; m < nm; ++m) {
        const int64_t pairs = (int64_t)sets[ms[m].left].size() * (int64_t)sets[ms[m].right].size();
        if (!ranked[m] && pairs >= 2 * c->chunk_pairs && sets[ms[m].right].size() > 1) {
            // ranges of at least chunk_pairs pairs, at most rep_chunks of them
            nchunks[m] = (int32_t)std::min<int64_t>(
                std::min<int64_t>(std::max(1, c->rep_chunks), pairs / c->chunk_pairs),
                (int64_t)sets[ms[m].right].size());
            max_chunks = std::max(max_chunks, nchunks[m]);
        }
    }
    std::vector<std::vector<char>> dead(nm);
    for (size_t m = 0; m < nm; ++m) dead[m].assign(sets[ms[m].left].size(), 0);
    for (int32_t k = 0; k < max_chunks; ++k) {
        // blocks of range k of every merge (all of cs2 for an unchunked merge at k = 0)
        std::vector<int32_t> kids;
        std::vector<BlockReq> kreq;
        std::vector<std::vector<int32_t>> rowsel, colsel;   // per block: row and column indices
        std::vector<std::pair<int32_t, int32_t>> kown;      // per block: (merge, transposed)
        for (size_t m = 0; m < nm; ++m) {
            if (ranked[m] || k >= nchunks[m]) continue;
            const int64_t n2 = (int64_t)sets[ms[m].right].size();
            const int32_t lo = (int32_t)(n2 * k / nchunks[m]), hi = (int32_t)(n2 * (k + 1) / nchunks[m]);
            std::vector<int32_t> rows_alive;
            for (int32_t i1 : qorder[m]) if (!dead[m][i1]) rows_alive.push_back(i1);
            if (rows_alive.empty()) continue;
            std::vector<int32_t> sc, lc;
            for (int32_t i2 : sorder[m]) if (i2 >= lo && i2 < hi) sc.push_back(i2);
            for (int32_t i2 : lorder[m]) if (i2 >= lo && i2 < hi) lc.push_back(i2);
            const auto& cs1 = sets[ms[m].left];
            const auto& cs2 = sets[ms[m].right];
            if (!sc.empty()) {
                BlockReq b{};
                b.kind = kCross;
                b.swap = 0;                                  // pair (rep1, rep2)
                b.a_begin = (int64_t)kids.size();
                b.a_count = (int64_t)rows_alive.size();
                for (int32_t i1 : rows_alive) kids.push_back(arena[cs1[i1]].rep);
                b.b_begin = (int64_t)kids.size();
                b.b_count = (int64_t)sc.size();
                for (int32_t i2 : sc) kids.push_back(arena[cs2[i2]].rep);
                kreq.push_back(b);
                rowsel.push_back(rows_alive);
                colsel.push_back(sc);
                kown.push_back({(int32_t)m, 0});
            }
            if (!lc.empty()) {
                BlockReq b{};
                b.kind = kCross;
                b.swap = 1;                                  // pair (rep1, rep2) = (subject, query)
                b.a_begin = (int64_t)kids.size();
                b.a_count = (int64_t)lc.size();
                for (int32_t i2 : lc) kids.push_back(arena[cs2[i2]].rep);
                b.b_begin = (int64_t)kids.size();
                b.b_count = (int64_t)rows_alive.size();
                for (int32_t i1 : rows_alive) kids.push_back(arena[cs1[i1]].rep);
                kreq.push_back(b);
                rowsel.push_back(rows_alive);
                colsel.push_back(lc);
                kown.push_back({(int32_t)m, 1});
            }
        }
        if (!kreq.empty()) {
            std::vector<std::pair<int64_t, int32_t>> sig;
            int64_t dev_batches = 1;
            r = score_blocks_sig(c, P, kids, kreq, prm.T, sig, base, flags, &dev_batches);
            if (r) return r;
            batches += std::max<int64_t>(dev_batches - 1, 0) + (k > 0 ? 1 : 0);
            for (const BlockReq& b : kreq) scored += b.a_count * b.b_count;
            size_t bi = 0;
            for (const auto& e : sig) {
                while (bi + 1 < kreq.size() && base[bi + 1] <= e.first) ++bi;
                const size_t m = (size_t)kown[bi].first;
                const int64_t local = e.first - base[bi];
                const int64_t nb = kreq[bi].b_count;
                if (kown[bi].second == 0)
                    sigm[m].push_back({rowsel[bi][local / nb], colsel[bi][local % nb], e.second});
                else
                    sigm[m].push_back({rowsel[bi][local % nb], colsel[bi][local / nb], e.second});
            }
        }
        if (k + 1 >= max_chunks) break;
        // the rows of the chunked merges that break within the columns scored so far
        for (size_t m = 0; m < nm; ++m)
            if (nchunks[m] > 1) std::sort(sigm[m].begin(), sigm[m].end());
        r = add_cells(true, nchunks);
        if (r) return r;
        for (size_t m = 0; m < nm; ++m) {
            if (nchunks[m] < 2 || k + 1 >= nchunks[m]) continue;
            const int64_t n2 = (int64_t)sets[ms[m].right].size();
            const int32_t hi = (int32_t)(n2 * (k + 1) / nchunks[m]);
            std::unordered_map<uint64_t, int64_t> cmap(cidx[m].begin(), cidx[m].end());
            std::vector<char> merged2((size_t)n2, 0);
            for (size_t q = 0; q < sigm[m].size();) {
                const int32_t i1 = sigm[m][q].i1;
                size_t q1 = q;
                while (q1 < sigm[m].size() && sigm[m][q1].i1 == i1) ++q1;
                for (; q < q1; ++q) {
                    const SigPair& e = sigm[m][q];
                    if (e.i2 >= hi) continue;
                    if (merged2[e.i2] && !partial_mode()) continue;
                    if (e.s <= prm.mT) continue;
                    bool t21, t12;
                    transit(m, cmap, i1, e.i2, &t21, &t12);
                    if (t21) { dead[m][i1] = 1; break; }
                    if (t12) merged2[e.i2] = 1;
                }
                q = q1;
            }
        }
    }
    if (d_bits) {
        r = score_ranked(ms, ranked, bitmap, bitbase, words, repb0, d_bits, d_reps, sigm);
        if (r) return r;
    }
    for (size_t m = 0; m < nm; ++m) std::sort(sigm[m].begin(), sigm[m].end());
    t_rep += now_s() - t0;
    ++batches;

    // ---- wave 2: alignment cells of every candidate full merge (s > mT and s > T) not yet
    // computed by a chunked merge's break search ----
    r = add_cells(false, nchunks);
    if (r) return r;

    // ---- Algorithm 1 control flow per merge -> event list ----
    // Visits are counted as Algorithm 1 makes them: i1's loop over cs2 (the plain merge) or
    // over its selected candidates (a ranked merge), up to the break, skipping c2 already
    // merged when i1's loop starts; the cs2 merged during i1's own loop were visited first.
    // With partial merges (CM_MERGE_PARTIAL) every cs1 cluster's loop sees cs2 as the merge
    // began: it visits the cs2 clusters other loops merged, and the counts do not discount them.
    const bool partial = prm.merge_mode == CM_MERGE_PARTIAL;
    std::vector<std::vector<Event>> events(nm);
    std::vector<std::vector<int32_t>> out_sets(nm);
    for (size_t m = 0; m < nm; ++m) {
        const auto& cs1 = sets[ms[m].left];
        const auto& cs2 = sets[ms[m].right];
        std::unordered_map<uint64_t, int64_t> cmap(cidx[m].begin(), cidx[m].end());
        std::vector<char> merged1(cs1.size(), 0), merged2(cs2.size(), 0);
        std::vector<int32_t> merged_before;               // sorted cs2 indices merged so far
        std::vector<uint32_t> merged_bits(ranked[m] ? (size_t)words[m] : 0, 0u);   // same, as bits
        const std::vector<SigPair>& sg = sigm[m];
        size_t p = 0;
        for (int32_t i1 = 0; i1 < (int32_t)cs1.size(); ++i1) {
            size_t p_end = p;
            while (p_end < sg.size() && sg[p_end].i1 == i1) ++p_end;
            int64_t end = (int64_t)cs2.size();            // visited range [0, end)
            std::vector<int32_t> newly;
            for (size_t q = p; q < p_end; ++q) {
                const int32_t i2 = sg[q].i2;
                if (merged2[i2] && !partial) continue;
                const int32_t s = sg[q].s;
                bool t21 = false, t12 = false;
                if (s > prm.mT) {
                    const int32_t* cl = &cells[cmap.at(key2(i1, i2)) * 5];
                    const int64_t la = P.len(arena[cs1[i1]].rep), lb = P.len(arena[cs2[i2]].rep);
                    const int64_t ua = cl[0] ? la - (cl[2] - cl[1] + 1) : la;
                    const int64_t ub = cl[0] ? lb - (cl[4] - cl[3] + 1) : lb;
                    t21 = ua < prm.mU;
                    t12 = ub < prm.mU;
                }
                if (t21) {
                    events[m].push_back({kAbsorbInto2, i1, i2, s});
                    merged1[i1] = 1;
                    ++full_merges;
                    end = (int64_t)i2 + 1;
                    break;
                } else if (t12) {
                    events[m].push_back({kAbsorbInto1, i1, i2, s});
                    merged2[i2] = 1;
                    newly.push_back(i2);
                    ++full_merges;
                } else {
                    events[m].push_back({kExchange, i1, i2, s});
                    ++exchanges;
                }
            }
            const int64_t before = partial ? 0 :
                                   std::lower_bound(merged_before.begin(), merged_before.end(),
                                                    (int32_t)std::min<int64_t>(end, INT32_MAX)) -
                                   merged_before.begin();
            if (!ranked[m]) {
                rep_cmp += end - before;
            } else {
                // selected cs2 below the break, less those merged before i1's loop started
                const uint32_t* row = bitmap.data() + bitbase[m] + (int64_t)i1 * words[m];
                int64_t vis = 0;
                for (int64_t w = 0; w * 32 < end; ++w) {
                    uint32_t x = partial ? row[w] : row[w] & ~merged_bits[w];
                    if ((w + 1) * 32 > end) x &= (1u << (end - w * 32)) - 1u;
                    vis += __builtin_popcount(x);
                }
                rep_cmp += vis;
            }
            for (int32_t i2 : newly) {
                merged_before.insert(std::upper_bound(merged_before.begin(), merged_before.end(), i2), i2);
                if (ranked[m]) merged_bits[i2 >> 5] |= 1u << (i2 & 31);
            }
            p = p_end;
        }
        for (size_t i1 = 0; i1 < cs1.size(); ++i1)
            if (!merged1[i1]) out_sets[m].push_back(cs1[i1]);
        for (size_t i2 = 0; i2 < cs2.size(); ++i2)
            if (!merged2[i2]) out_sets[m].push_back(cs2[i2]);
    }

    // ---- membership: replay the events until no (member, rep) score is missing ----
    std::vector<int32_t> involved;
    for (size_t m = 0; m < nm; ++m) {
        if (events[m].empty()) continue;
        for (int32_t ci : sets[ms[m].left]) involved.push_back(ci);
        for (int32_t ci : sets[ms[m].right]) involved.push_back(ci);
    }
    std::vector<std::vector<int32_t>> snap(involved.size());
    for (size_t i = 0; i < involved.size(); ++i) snap[i] = arena[involved[i]].objs;
    // A wave resolves at least the first event of each merge that still misses a score (the
    // state before that event is already exact), so a merge needs at most its event count
    // plus one waves; more than that means no progress.
    size_t max_events = 0;
    for (size_t m = 0; m < nm; ++m) max_events = std::max(max_events, events[m].size());
    for (int64_t wave = 0;; ++wave) {
        if (wave > 0) {
            for (size_t i = 0; i < involved.size(); ++i) {
                Cluster& cl = arena[involved[i]];
                cl.objs = snap[i];
                cl.mem.clear();
                cl.mem.insert(cl.objs.begin(), cl.objs.end());
            }
        }
        std::unordered_map<int32_t, std::vector<int32_t>> need;   // rep -> members to score
        std::unordered_set<uint64_t> needed;
        int64_t lookups = 0;
        for (size_t m = 0; m < nm; ++m) {
            const auto& cs1 = sets[ms[m].left];
            const auto& cs2 = sets[ms[m].right];
            if (partial) {
                replay_partial(cs1, cs2, events[m], need, needed, lookups);
                continue;
            }
            for (const Event& ev : events[m]) {
                Cluster& c1 = arena[cs1[ev.i1]];
                Cluster& c2 = arena[cs2[ev.i2]];
                if (ev.kind == kAbsorbInto2) {
                    const std::vector<int32_t> o = c1.objs;
                    for (int32_t x : o) c2.add(x);
                } else if (ev.kind == kAbsorbInto1) {
                    const std::vector<int32_t> o = c2.objs;
                    for (int32_t x : o) c1.add(x);
                } else {
                    const std::vector<int32_t> s1 = c1.objs, s2 = c2.objs;
                    for (int pass = 0; pass < 2; ++pass) {
                        const std::vector<int32_t>& snapv = pass ? s2 : s1;
                        Cluster& self = pass ? c2 : c1;
                        Cluster& other = pass ? c1 : c2;
                        for (int32_t x : snapv) {
                            if (other.mem.count(x)) continue;
                            int32_t sm;
                            if (x == self.rep) {
                                sm = ev.s;
                            } else {
                                ++lookups;
                                auto it = memo.find(key2(x, other.rep));
                                if (it == memo.end()) {
                                    if (needed.insert(key2(x, other.rep)).second)
                                        need[other.rep].push_back(x);
                                    continue;
                                }
                                sm = it->second;
                            }
                            if (sm > prm.T) other.add(x);
                        }
                    }
                }
            }
        }
        if (need.empty()) {
            exch_cmp += lookups;
            waves += wave + 1;
            break;
        }
        // score the missing (member, rep) pairs: one block per rep, pair = (member, rep)
        std::vector<int32_t> eids;
        std::vector<BlockReq> ereq;
        std::vector<int32_t> reps;
        for (auto& kv : need) reps.push_back(kv.first);
        std::sort(reps.begin(), reps.end());
        std::vector<std::pair<int32_t, int32_t>> eown;    // block -> (rep, -1) or (rep, long member)
        for (int32_t rp : reps) {
            auto& mv = need[rp];
            std::vector<int32_t> shortm;
            for (int32_t x : mv) {
                if (P.len(x) > kLongSubject) {              // a long member is a query (see wave 1)
                    BlockReq b{};
                    b.kind = kCross;
                    b.swap = 0;                             // pair (member, rep)
                    b.a_begin = (int64_t)eids.size();
                    b.a_count = 1;
                    eids.push_back(x);
                    b.b_begin = (int64_t)eids.size();
                    b.b_count = 1;
                    eids.push_back(rp);
                    ereq.push_back(b);
                    eown.push_back({rp, x});
                } else {
                    shortm.push_back(x);
                }
            }
            if (shortm.empty()) continue;
            BlockReq b{};
            b.kind = kCross;
            b.swap = 1;
            b.a_begin = (int64_t)eids.size();
            b.a_count = 1;
            eids.push_back(rp);
            b.b_begin = (int64_t)eids.size();
            b.b_count = (int64_t)shortm.size();
            eids.insert(eids.end(), shortm.begin(), shortm.end());
            ereq.push_back(b);
            eown.push_back({rp, -1});
        }
        std::vector<int32_t> ES;
        std::vector<int64_t> ebase;
        t0 = now_s();
        r = score_blocks(c, P, eids, ereq, ES, ebase, flags);
        if (r) return r;
        t_exch += now_s() - t0;
        scored += (int64_t)ES.size();
        ++batches;
        for (size_t b = 0; b < ereq.size(); ++b) {
            const int32_t rp = eown[b].first;
            if (eown[b].second >= 0) {
                memo[key2(eown[b].second, rp)] = ES[ebase[b]];
                continue;
            }
            for (int64_t s = 0; s < ereq[b].b_count; ++s)
                memo[key2(eids[ereq[b].b_begin + s], rp)] = ES[ebase[b] + s];
        }
        if (wave > (int64_t)max_events)
            return fail(c, CM_ERR_INTERNAL, "exchange replay did not converge");
    }
    for (size_t m = 0; m < nm; ++m) sets[ms[m].out] = std::move(out_sets[m]);
    merges += (int64_t)nm;
    return CM_OK;
}

// Rep x rep scores of the ranked merges, planned on the device from the selection bitmap.
// The cs1 reps of a merge are paired in length order; for a pair (a, b) the subjects both
// select form one pair-mode block (both queries over one shared stream), those only a or
// only b selects form single-query blocks, and an unpaired rep runs alone.  The subject
// lists, their row tables and streams are expanded on the device; the host handles per-list
// counts only.  Lists run in chunks of at most kRankedChunkRows stream rows.  Only the pairs
// with s > T come back, appended to sigm[m] as (i1, i2, s).
int Driver::score_ranked(const std::vector<Merge>& ms, const std::vector<char>& ranked,
                         const std::vector<uint32_t>& bitmap, const std::vector<int64_t>& bitbase,
                         const std::vector<int64_t>& words, const std::vector<int64_t>& repb0,
                         const uint32_t* d_bits, const int32_t* d_reps,
                         std::vector<std::vector<SigPair>>& sigm)
{
    NvtxRange range("cm ranked rep wave");
    constexpr int64_t kRankedChunkRows = (int64_t)8 << 30;
    struct LMeta { int32_t m, a, b, op; int64_t count; };
    std::vector<KeptList> lists;
    std::vector<LMeta> meta;
    auto derived = [&](const LMeta& L, int64_t w) -> uint32_t {
        const uint32_t x = bitmap[bitbase[L.m] + (int64_t)L.a * words[L.m] + w];
        if (L.op == kKeepA) return x;
        const uint32_t y = bitmap[bitbase[L.m] + (int64_t)L.b * words[L.m] + w];
        return L.op == kKeepAnd ? (x & y) : L.op == kKeepAOnly ? (x & ~y) : (y & ~x);
    };
    for (size_t m = 0; m < ms.size(); ++m) {
        if (!ranked[m]) continue;
        const auto& cs1 = sets[ms[m].left];
        std::vector<int32_t> order(cs1.size());
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
            return P.len(arena[cs1[x]].rep) < P.len(arena[cs1[y]].rep);
        });
        auto add = [&](int32_t a, int32_t b, int32_t op) {
            LMeta L{(int32_t)m, a, b, op, 0};
            for (int64_t w = 0; w < words[m]; ++w) L.count += __builtin_popcount(derived(L, w));
            selected += L.count * (op == kKeepAnd ? 2 : 1);
            if (L.count == 0) return;
            KeptList K{};
            K.row_a = bitbase[m] + (int64_t)a * words[m];
            K.row_b = b >= 0 ? bitbase[m] + (int64_t)b * words[m] : K.row_a;
            K.words = (int32_t)words[m];
            K.op = op;
            K.b0 = repb0[m];
            lists.push_back(K);
            meta.push_back(L);
        };
        size_t t = 0;
        for (; t + 1 < order.size(); t += 2) {
            add(order[t], order[t + 1], kKeepAnd);
            add(order[t], order[t + 1], kKeepAOnly);
            add(order[t], order[t + 1], kKeepBOnly);
        }
        if (t < order.size()) add(order[t], -1, kKeepA);
    }
    if (lists.empty()) return CM_OK;
    const int32_t nl = (int32_t)lists.size();
    const cudaStream_t st = c->stream;
    KeptList* d_lists;
    int64_t* d_tot;
    ENSURE(B_KEPT, nl, d_lists);
    ENSURE(B_KTOT, 2 * (int64_t)nl, d_tot);
    int r;
    if ((r = copy_in(c, d_lists, lists.data(), lists.size() * sizeof(KeptList), false))) return r;
    CUDA_TRY(launch_kept_totals(d_lists, nl, d_bits, d_reps, P.off, d_tot, st));
    std::vector<int64_t> tot(2 * (size_t)nl);
    CUDA_TRY(cudaMemcpyAsync(tot.data(), d_tot, tot.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    c->stats.launches += 1;
    const int64_t target = (int64_t)c->W * c->rows_per_warp;
    for (int32_t l0 = 0; l0 < nl;) {
        int32_t l1 = l0;
        int64_t rows = 0;
        while (l1 < nl && (l1 == l0 || rows + tot[2 * l1] <= kRankedChunkRows)) rows += tot[2 * l1++];
        Plan plan;
        plan.dev_lists = true;
        plan.total_rows = rows;
        std::vector<int64_t> first;
        int64_t g = 0, rowbase = 0, slots = 0;
        for (int32_t l = l0; l < l1; ++l) {
            const LMeta& L = meta[l];
            const auto& cs1 = sets[ms[L.m].left];
            KeptList& K = lists[l];
            K.g0 = g;
            K.rowbase = rowbase;
            const bool pair = L.op == kKeepAnd;
            const int32_t qa = arena[cs1[L.op == kKeepBOnly ? L.b : L.a]].rep;
            const int32_t qb = pair ? arena[cs1[L.b]].rep : qa;
            SwBlock B{};
            B.kind = kCross;
            B.swap = 0;
            B.na = pair ? 2 : 1;
            B.nb = (int32_t)L.count;
            B.a_ids = (int64_t)plan.ids.size();
            plan.ids.push_back(qa);
            if (pair) plan.ids.push_back(qb);
            B.b_ids = -1;                                  // fixed up below (after the A ids)
            B.stream = 0;
            B.srow = g;
            B.out_base = slots;
            B.k0 = 0;
            B.has_map = 0;
            plan.blocks.push_back(B);
            plan.first_slot.push_back(slots);
            first.push_back(slots);
            add_tasks(plan, (int32_t)plan.blocks.size() - 1, 0, (int32_t)L.count, pair, P.len(qb),
                      nullptr, target, tot[2 * l]);
            plan.cells += (P.len(qa) + (pair ? P.len(qb) : 0)) * tot[2 * l + 1];
            slots += (int64_t)B.na * L.count;
            g += L.count;
            rowbase += tot[2 * l];
        }
        const int64_t nA = (int64_t)plan.ids.size();
        for (auto& B : plan.blocks) B.b_ids = nA + B.srow;
        plan.n_sub = g;
        plan.nslots = plan.pairs = slots;
        order_tasks(plan);
        plan.max_warp_rows = 2 * c->rows_per_warp + 2 * stream_rows(P.maxlen) + 2 * target / c->W;
        int32_t* d_ids;
        int64_t* d_srow;
        ENSURE(B_IDS, nA + g, d_ids);
        ENSURE(B_SROW, g + 1, d_srow);
        if ((r = copy_in(c, d_lists, lists.data() + l0, (size_t)(l1 - l0) * sizeof(KeptList), false))) return r;
        CUDA_TRY(cudaMemsetAsync(d_srow, 0, sizeof(int64_t), st));
        CUDA_TRY(launch_kept_expand(d_lists, l1 - l0, d_bits, d_reps, P.off, d_ids + nA, d_srow, st));
        c->stats.launches += 1;
        int32_t* out;
        ENSURE(B_OUT, slots, out);
        if ((r = run_plan(c, P, plan, out, nullptr, flags))) return r;
        std::vector<std::pair<int64_t, int32_t>> sig;
        if ((r = compact_sig(c, out, slots, prm.T, sig))) return r;
        scored += slots;
        // `sig` is in slot order, so the ranks of one list row ascend: one forward scan of the
        // list's bitmap words per (list, query row) finds the subject of every significant slot
        int32_t cur_l = -1;
        int64_t cur_k = -1, cur_w = 0, before = 0;     // set bits in words [0, cur_w)
        for (const auto& e : sig) {
            const int32_t l = l0 + (int32_t)(std::upper_bound(first.begin(), first.end(), e.first) -
                                             first.begin()) - 1;
            const LMeta& L = meta[l];
            const int64_t local = e.first - first[l - l0];
            const int64_t k = local / L.count, rank = local % L.count;
            if (l != cur_l || k != cur_k) {
                cur_l = l;
                cur_k = k;
                cur_w = 0;
                before = 0;
            }
            uint32_t x = derived(L, cur_w);
            while (rank >= before + __builtin_popcount(x)) {
                before += __builtin_popcount(x);
                x = derived(L, ++cur_w);
            }
            for (int64_t q = before; q < rank; ++q) x &= x - 1;
            const int32_t i1 = (L.op == kKeepBOnly || (L.op == kKeepAnd && k == 1)) ? L.b : L.a;
            sigm[L.m].push_back({i1, (int32_t)(cur_w * 32 + __builtin_ctz(x)), e.second});
        }
        ++batches;
        l0 = l1;
    }
    return CM_OK;
}

int Driver::finish(std::vector<int32_t>& final_set, cm_result* res)
{
    NvtxRange range("cm intra-cluster pairs");
    // intra-cluster all-against-all: one TRI block per cluster (members in length order).  A
    // cluster with two or more members longer than kLongSubject splits: TRI over its short
    // members, a CROSS block of the long members (queries) against the short ones, and the
    // long x long pairs straight on the int32 whole-CTA kernels (in a TRI block each of them
    // is one warp's stream over dozens of column passes while the CTA's other warps wait,
    // and such pairs of one family exceed the int16 range and are rescored anyway).
    std::vector<int32_t> ids, ll;
    std::vector<BlockReq> req;
    auto add_block = [&](int32_t kind, const int32_t* a, int64_t na, const int32_t* b, int64_t nb) {
        BlockReq blk{};
        blk.kind = kind;
        blk.swap = 0;
        blk.a_begin = (int64_t)ids.size();
        blk.a_count = na;
        ids.insert(ids.end(), a, a + na);
        if (kind == kTri) {
            blk.b_begin = blk.a_begin;
            blk.b_count = na;
        } else {
            blk.b_begin = (int64_t)ids.size();
            blk.b_count = nb;
            ids.insert(ids.end(), b, b + nb);
        }
        req.push_back(blk);
    };
    for (int32_t ci : final_set) {
        const Cluster& cl = arena[ci];
        if (cl.objs.size() < 2) continue;
        std::vector<int32_t> mem = by_length(cl.objs);
        const int64_t n = (int64_t)mem.size();
        int64_t p = n;                                   // first member longer than kLongSubject
        while (p > 0 && P.len(mem[p - 1]) > kLongSubject) --p;
        if (n - p < 2) {
            add_block(kTri, mem.data(), n, nullptr, 0);
            continue;
        }
        if (p >= 2) add_block(kTri, mem.data(), p, nullptr, 0);
        if (p >= 1) add_block(kCross, mem.data() + p, n - p, mem.data(), p);
        for (int64_t k = p + 1; k < n; ++k)
            for (int64_t s2 = p; s2 < k; ++s2) {
                ll.push_back(mem[k]);
                ll.push_back(mem[s2]);
            }
    }
    std::vector<int32_t> S, SL;
    std::vector<int64_t> base;
    const double t0 = now_s();
    int r = req.empty() ? CM_OK : score_blocks(c, P, ids, req, S, base, flags);
    if (r) return r;
    r = score_pairs_int32(c, P, ll, SL);
    if (r) return r;
    t_intra += now_s() - t0;
    scored += (int64_t)S.size() + (int64_t)SL.size();
    ++batches;
    std::vector<uint64_t> all;
    std::vector<std::pair<uint64_t, int32_t>> sig;
    all.reserve(S.size() + SL.size());
    auto visit = [&](int32_t x, int32_t y, int32_t score) {
        const int32_t i = std::min(x, y), j = std::max(x, y);
        all.push_back(key2(i, j));
        if (score > prm.T) sig.push_back({key2(i, j), score});
    };
    for (size_t b = 0; b < req.size(); ++b) {
        const int32_t* A = ids.data() + req[b].a_begin;
        const int64_t na = req[b].a_count;
        int64_t slot = base[b];
        if (req[b].kind == kTri) {
            for (int64_t k = 1; k < na; ++k)
                for (int64_t s2 = 0; s2 < k; ++s2, ++slot) visit(A[k], A[s2], S[slot]);
        } else {
            const int32_t* B = ids.data() + req[b].b_begin;
            const int64_t nb = req[b].b_count;
            for (int64_t k = 0; k < na; ++k)
                for (int64_t s2 = 0; s2 < nb; ++s2, ++slot) visit(A[k], B[s2], S[slot]);
        }
    }
    for (size_t k = 0; k < SL.size(); ++k) visit(ll[2 * k], ll[2 * k + 1], SL[k]);
    std::sort(all.begin(), all.end());
    const int64_t intra = std::unique(all.begin(), all.end()) - all.begin();
    std::sort(sig.begin(), sig.end());
    sig.erase(std::unique(sig.begin(), sig.end(),
                          [](const std::pair<uint64_t, int32_t>& x,
                             const std::pair<uint64_t, int32_t>& y) { return x.first == y.first; }),
              sig.end());

    // result arrays (library-owned, freed by cm_result_free)
    res->n_clusters = (int32_t)final_set.size();
    int64_t total = 0;
    for (int32_t ci : final_set) total += (int64_t)arena[ci].objs.size();
    res->reps = (int32_t*)std::malloc(sizeof(int32_t) * std::max<size_t>(final_set.size(), 1));
    res->cl_offsets = (int64_t*)std::malloc(sizeof(int64_t) * (final_set.size() + 1));
    res->members = (int32_t*)std::malloc(sizeof(int32_t) * std::max<int64_t>(total, 1));
    res->n_pairs = (int64_t)sig.size();
    res->pairs = (int32_t*)std::malloc(sizeof(int32_t) * 2 * std::max<size_t>(sig.size(), 1));
    res->scores = (int32_t*)std::malloc(sizeof(int32_t) * std::max<size_t>(sig.size(), 1));
    if (!res->reps || !res->cl_offsets || !res->members || !res->pairs || !res->scores)
        return fail(c, CM_ERR_OOM, "host allocation of the result failed");
    int64_t pos = 0;
    res->cl_offsets[0] = 0;
    for (size_t k = 0; k < final_set.size(); ++k) {
        const Cluster& cl = arena[final_set[k]];
        res->reps[k] = cl.rep;
        std::memcpy(res->members + pos, cl.objs.data(), cl.objs.size() * sizeof(int32_t));
        pos += (int64_t)cl.objs.size();
        res->cl_offsets[k + 1] = pos;
    }
    for (size_t k = 0; k < sig.size(); ++k) {
        res->pairs[2 * k] = (int32_t)(sig[k].first >> 32);
        res->pairs[2 * k + 1] = (int32_t)(sig[k].first & 0xffffffffu);
        res->scores[k] = sig[k].second;
    }
    res->rep_comparisons = rep_cmp;
    res->exchange_comparisons = exch_cmp;
    res->intra_comparisons = intra;
    res->comparisons_scored = scored;
    res->cells_pairs = cells_pairs;
    res->full_merges = full_merges;
    res->exchanges = exchanges;
    res->merges = merges;
    res->rounds = rounds;
    res->gpu_batches = batches;
    res->exchange_waves = waves;
    res->t_rep = t_rep;
    res->t_cells = t_cells;
    res->t_exchange = t_exch;
    res->t_intra = t_intra;
    res->t_rank = t_rank;
    res->ranker_selected = selected;
    return CM_OK;
}

// Incremental greedy clustering (the comparison method of Sec. 2, after Wittwer et al.): each
// sequence in input order is compared with every representative in creation order, joins the
// cluster of every one with s > T, and starts a new cluster unless some representative
// represents it (s > mT and fewer than mU of its residues outside the alignment, the Sec. 4
// test with the sequence in the absorbed role).  Sequences are taken in chunks: one device
// batch scores the chunk against the representatives before it (CROSS) and against itself
// (TRI, speculative: any earlier chunk member may become a representative), a second the
// alignment cells of every pair above mT; the host then replays the chunk in input order.
int Driver::run_greedy(int32_t n, int32_t chunk, std::vector<int32_t>& final_set)
{
    NvtxRange range("cm greedy");
    arena.clear();
    std::vector<int32_t> cluster_of((size_t)std::max(n, 1), -1);   // representative -> cluster
    for (int32_t x0 = 0; x0 < n; x0 += chunk) {
        const int32_t x1 = std::min<int32_t>(n, x0 + chunk);
        const int32_t nr = (int32_t)arena.size();
        std::vector<int32_t> ids;
        std::vector<BlockReq> req;
        std::vector<int32_t> members((size_t)(x1 - x0));
        std::iota(members.begin(), members.end(), x0);
        members = by_length(members);
        BlockReq tri{};
        tri.kind = kTri;
        tri.a_begin = tri.b_begin = 0;
        tri.a_count = tri.b_count = (int64_t)members.size();
        ids.insert(ids.end(), members.begin(), members.end());
        req.push_back(tri);
        std::vector<int32_t> short_reps, long_reps;
        for (int32_t k = 0; k < nr; ++k)
            (P.len(arena[k].rep) > kLongSubject ? long_reps : short_reps).push_back(arena[k].rep);
        if (!short_reps.empty()) {                        // chunk (queries) x reps (subjects)
            BlockReq b{};
            b.kind = kCross;
            b.a_begin = 0;
            b.a_count = (int64_t)members.size();
            b.b_begin = (int64_t)ids.size();
            b.b_count = (int64_t)short_reps.size();
            ids.insert(ids.end(), short_reps.begin(), short_reps.end());
            req.push_back(b);
        }
        if (!long_reps.empty()) {                         // long reps (queries) x chunk
            BlockReq b{};
            b.kind = kCross;
            b.swap = 1;
            b.a_begin = (int64_t)ids.size();
            b.a_count = (int64_t)long_reps.size();
            ids.insert(ids.end(), long_reps.begin(), long_reps.end());
            b.b_begin = 0;
            b.b_count = (int64_t)members.size();
            req.push_back(b);
        }
        std::vector<std::pair<int64_t, int32_t>> sig;
        std::vector<int64_t> base;
        double t0 = now_s();
        int r = score_blocks_sig(c, P, ids, req, prm.T, sig, base, flags);
        if (r) return r;
        t_rep += now_s() - t0;
        ++batches;
        for (const BlockReq& b : req)
            scored += b.kind == kTri ? b.a_count * (b.a_count - 1) / 2 : b.a_count * b.b_count;
        // similar pairs (x, y, s) of the chunk: y a representative before it or an earlier
        // chunk member
        std::vector<SigPair> simp;
        size_t q = 0;
        for (size_t bi = 0; bi < req.size(); ++bi) {
            const BlockReq& b = req[bi];
            const int64_t end = bi + 1 < req.size() ? base[bi + 1] : INT64_MAX;
            for (; q < sig.size() && sig[q].first < end; ++q) {
                const int64_t loc = sig[q].first - base[bi];
                int32_t u, v;
                if (b.kind == kTri) {
                    int64_t k = (int64_t)((1.0 + std::sqrt(1.0 + 8.0 * (double)loc)) / 2.0);
                    while (k * (k - 1) / 2 > loc) --k;
                    while ((k + 1) * k / 2 <= loc) ++k;
                    u = ids[b.a_begin + k];
                    v = ids[b.a_begin + (loc - k * (k - 1) / 2)];
                    if (u < v) std::swap(u, v);             // (later, earlier) in input order
                } else {
                    const int32_t qa = ids[b.a_begin + loc / b.b_count];
                    const int32_t sb = ids[b.b_begin + loc % b.b_count];
                    u = b.swap ? sb : qa;                   // the chunk member
                    v = b.swap ? qa : sb;                   // the representative
                }
                simp.push_back({u, v, sig[q].second});
            }
        }
        // alignment cells of every candidate representation (s > mT), pair (x, y)
        std::vector<int32_t> cp;
        for (const SigPair& e : simp)
            if (e.s > prm.mT) { cp.push_back(e.i1); cp.push_back(e.i2); }
        std::vector<int32_t> cells(cp.size() / 2 * 5);
        std::unordered_map<uint64_t, int64_t> cidx;
        if (!cp.empty()) {
            t0 = now_s();
            r = run_cells(c, P, cp.data(), (int64_t)cp.size() / 2, cells.data());
            if (r) return r;
            t_cells += now_s() - t0;
            cells_pairs += (int64_t)cp.size() / 2;
            for (size_t k = 0; k < cp.size() / 2; ++k)
                cidx[key2(cp[2 * k], cp[2 * k + 1])] = (int64_t)k;
        }
        // replay in input order; a sequence's candidates in its representatives' creation
        // order (those before the chunk first, by cluster; then chunk members by input order)
        std::sort(simp.begin(), simp.end(), [&](const SigPair& a, const SigPair& b) {
            if (a.i1 != b.i1) return a.i1 < b.i1;
            const bool ea = a.i2 < x0, eb = b.i2 < x0;
            if (ea != eb) return ea;
            return ea ? cluster_of[a.i2] < cluster_of[b.i2] : a.i2 < b.i2;
        });
        size_t p = 0;
        int32_t chunk_reps = 0;
        for (int32_t x = x0; x < x1; ++x) {
            rep_cmp += nr + chunk_reps;
            bool represented = false;
            for (; p < simp.size() && simp[p].i1 == x; ++p) {
                const SigPair& e = simp[p];
                const int32_t cl = cluster_of[e.i2];
                if (cl < 0) continue;                       // not a representative
                arena[cl].objs.push_back(x);
                if (e.s > prm.mT) {
                    const int32_t* ce = &cells[cidx.at(key2(x, e.i2)) * 5];
                    const int64_t lx = P.len(x);
                    const int64_t ux = ce[0] ? lx - (ce[2] - ce[1] + 1) : lx;
                    if (ux < prm.mU) represented = true;
                }
            }
            if (!represented) {
                Cluster nc;
                nc.rep = x;
                nc.objs = {x};
                cluster_of[x] = (int32_t)arena.size();
                arena.push_back(std::move(nc));
                ++chunk_reps;
            } else {
                ++full_merges;
            }
        }
        ++rounds;
    }
    final_set.resize(arena.size());
    std::iota(final_set.begin(), final_set.end(), 0);
    return CM_OK;
}

// ---- round-state checkpoints: Algorithm 2's schedule position plus the cluster arena ----
// File: "CMRS", version, a fingerprint of the problem (sequence lengths, matrix, gaps,
// params), the rounds completed, the driver's counters and timers, the seconds of earlier
// calls, then every set a later round reads: set id, its clusters (rep, members in order).
// The score memo is not kept: a resumed run rescores what it needs, with the same results.
constexpr uint32_t kStateMagic = 0x53524d43u;      // "CMRS"
constexpr uint32_t kStateVersion = 1;

uint64_t fnv(uint64_t h, const void* p, size_t n)
{
    const uint8_t* b = static_cast<const uint8_t*>(p);
    for (size_t i = 0; i < n; ++i) { h ^= b[i]; h *= 1099511628211ull; }
    return h;
}

uint64_t fingerprint(const Prepared& P, int32_t n, const cm_params& prm, uint32_t flags)
{
    uint64_t h = 14695981039346656037ull;
    h = fnv(h, &n, sizeof(n));
    h = fnv(h, P.hoff.data(), P.hoff.size() * sizeof(int64_t));
    h = fnv(h, P.mat, sizeof(P.mat));
    h = fnv(h, &P.g1, sizeof(P.g1));
    h = fnv(h, &P.ge, sizeof(P.ge));
    const int32_t pv[6] = {prm.T, prm.mT, prm.mU, prm.use_ranker, prm.ranker_min_pairs,
                           prm.merge_mode};
    h = fnv(h, pv, sizeof(pv));
    h = fnv(h, &prm.prune_logit, sizeof(prm.prune_logit));
    h = fnv(h, &flags, sizeof(flags));
    return h;
}

struct StateFile {
    FILE* f = nullptr;
    bool ok = true;
    ~StateFile() { if (f) std::fclose(f); }
    template <class T> void put(const T& v) { ok = ok && std::fwrite(&v, sizeof(T), 1, f) == 1; }
    template <class T> void get(T& v) { ok = ok && std::fread(&v, sizeof(T), 1, f) == 1; }
    void put_vec(const std::vector<int32_t>& v)
    {
        put((uint64_t)v.size());
        ok = ok && (v.empty() || std::fwrite(v.data(), sizeof(int32_t), v.size(), f) == v.size());
    }
    void get_vec(std::vector<int32_t>& v, uint64_t limit)
    {
        uint64_t k = 0;
        get(k);
        if (!ok || k > limit) { ok = false; return; }
        v.resize((size_t)k);
        ok = ok && (k == 0 || std::fread(v.data(), sizeof(int32_t), (size_t)k, f) == k);
    }
};

}  // namespace
}  // namespace cm

using namespace cm;

extern "C" {

static int run_cluster_merge(cm_ctx* c, const uint8_t* seqs, const int64_t* offsets,
                             int32_t n_seqs, const int8_t* matrix, int32_t gap_open,
                             int32_t gap_extend, const cm_params* params, const char* state_path,
                             double budget_seconds, cm_result** out, uint32_t flags)
{
    if (!c) return CM_ERR_ARG;
    NvtxRange range("cluster_merge");
    if (!out || !params) return fail(c, CM_ERR_ARG, "null params / out");
    *out = nullptr;
    CUDA_TRY(cudaSetDevice(c->device));
    const auto t0 = std::chrono::steady_clock::now();
    Prepared P;
    int r = prepare(c, seqs, offsets, n_seqs, matrix, gap_open, gap_extend, flags, P);
    if (r) return r;
    if (!P.symmetric)
        return fail(c, CM_ERR_ARG, "cluster_merge needs a symmetric substitution matrix");
    if (params->merge_mode != CM_MERGE_SEQUENTIAL && params->merge_mode != CM_MERGE_PARTIAL)
        return fail(c, CM_ERR_ARG, "merge_mode must be CM_MERGE_SEQUENTIAL or CM_MERGE_PARTIAL");
    const uint32_t dflags = flags & CM_FORCE_INT32;     // device data is resident from here on
    Driver D(c, P, *params, dflags);

    // Algorithm 2: FIFO of singleton sets -> merge DAG -> dependency rounds
    D.sets.resize((size_t)std::max(1, 2 * n_seqs));
    std::deque<int32_t> q;
    std::vector<int32_t> round_of((size_t)std::max(1, 2 * n_seqs), 0);
    std::vector<std::vector<Merge>> rounds;
    for (int32_t e = 0; e < n_seqs; ++e) q.push_back(e);
    int32_t next = n_seqs;
    while (q.size() > 1) {
        const int32_t a = q.front(); q.pop_front();
        const int32_t b = q.front(); q.pop_front();
        const int32_t o = next++;
        const int32_t rd = 1 + std::max(round_of[a], round_of[b]);
        round_of[o] = rd;
        if ((int32_t)rounds.size() < rd) rounds.resize(rd);
        rounds[rd - 1].push_back({a, b, o});
        q.push_back(o);
    }

    const uint64_t fp = fingerprint(P, n_seqs, *params, dflags);
    size_t first_round = 0;
    double earlier_seconds = 0;
    bool resumed = false;
    if (state_path) {
        StateFile F;
        F.f = std::fopen(state_path, "rb");
        if (F.f) {
            uint32_t magic = 0, version = 0;
            uint64_t fp_file = 0, nsets = 0;
            int64_t done = 0;
            F.get(magic);
            F.get(version);
            F.get(fp_file);
            if (!F.ok || magic != kStateMagic || version != kStateVersion)
                return fail(c, CM_ERR_ARG, "state file is not a ClusterMerge checkpoint");
            if (fp_file != fp)
                return fail(c, CM_ERR_ARG, "state file belongs to another problem or parameters");
            F.get(done);
            int64_t* cnt[] = {&D.rep_cmp, &D.exch_cmp, &D.full_merges, &D.exchanges, &D.scored,
                              &D.cells_pairs, &D.batches, &D.merges, &D.waves, &D.selected};
            for (int64_t* x : cnt) F.get(*x);
            double* tm[] = {&D.t_rep, &D.t_cells, &D.t_exch, &D.t_intra, &D.t_rank,
                            &earlier_seconds};
            for (double* x : tm) F.get(*x);
            F.get(nsets);
            if (!F.ok || done < 0 || done > (int64_t)rounds.size() || nsets > D.sets.size())
                return fail(c, CM_ERR_ARG, "state file is truncated or inconsistent");
            for (uint64_t k = 0; k < nsets && F.ok; ++k) {
                int32_t sid = -1;
                uint64_t ncl = 0;
                F.get(sid);
                F.get(ncl);
                if (!F.ok || sid < 0 || (size_t)sid >= D.sets.size() || ncl > (uint64_t)n_seqs) {
                    F.ok = false;
                    break;
                }
                for (uint64_t i = 0; i < ncl && F.ok; ++i) {
                    Cluster cl;
                    F.get(cl.rep);
                    F.get_vec(cl.objs, (uint64_t)n_seqs);
                    if (!F.ok || cl.objs.empty() || cl.objs[0] != cl.rep) { F.ok = false; break; }
                    for (int32_t x : cl.objs) {
                        if (x < 0 || x >= n_seqs || !cl.mem.insert(x).second) F.ok = false;
                    }
                    D.sets[sid].push_back((int32_t)D.arena.size());
                    D.arena.push_back(std::move(cl));
                }
            }
            // every set a remaining round reads must have come back (and hold a cluster)
            for (size_t j = (size_t)done; j < rounds.size() && F.ok; ++j)
                for (const Merge& m : rounds[j])
                    for (int32_t sid : {m.left, m.right})
                        if (round_of[sid] <= (int32_t)done && D.sets[sid].empty()) F.ok = false;
            if (!F.ok) return fail(c, CM_ERR_ARG, "state file is truncated or inconsistent");
            first_round = (size_t)done;
            D.rounds = done;
            resumed = true;
        }
    }
    if (!resumed) {
        D.arena.resize((size_t)n_seqs);
        for (int32_t e = 0; e < n_seqs; ++e) {
            D.arena[e].rep = e;
            D.arena[e].objs = {e};
            D.arena[e].mem = {e};
            D.sets[e] = {e};
        }
    }
    if (params->use_ranker) {
        const double tr = now_s();
        r = ranker_unit_vectors(c, P, n_seqs, &D.U);
        if (r) return r;
        D.t_rank += now_s() - tr;
    }
    auto elapsed = [&]() {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    };
    for (size_t k = first_round; k < rounds.size(); ++k) {
        r = D.run_round(rounds[k]);
        if (r) return r;
        ++D.rounds;
        if (state_path && budget_seconds > 0 && k + 1 < rounds.size() &&
            elapsed() >= budget_seconds) {
            // the sets later rounds read: inputs of rounds k+1.. made by rounds <= k or leaves
            std::vector<int32_t> live;
            for (size_t j = k + 1; j < rounds.size(); ++j)
                for (const Merge& m : rounds[j])
                    for (int32_t sid : {m.left, m.right})
                        if (sid < n_seqs || round_of[sid] <= (int32_t)(k + 1)) live.push_back(sid);
            std::sort(live.begin(), live.end());
            live.erase(std::unique(live.begin(), live.end()), live.end());
            const std::string tmp = std::string(state_path) + ".tmp";
            {
                StateFile F;
                F.f = std::fopen(tmp.c_str(), "wb");
                if (!F.f) return fail(c, CM_ERR_ARG, "cannot write the state file");
                F.put(kStateMagic);
                F.put(kStateVersion);
                F.put(fp);
                F.put((int64_t)(k + 1));
                for (int64_t x : {D.rep_cmp, D.exch_cmp, D.full_merges, D.exchanges, D.scored,
                                  D.cells_pairs, D.batches, D.merges, D.waves, D.selected})
                    F.put(x);
                for (double x : {D.t_rep, D.t_cells, D.t_exch, D.t_intra, D.t_rank,
                                 earlier_seconds + elapsed()})
                    F.put(x);
                F.put((uint64_t)live.size());
                for (int32_t sid : live) {
                    F.put(sid);
                    F.put((uint64_t)D.sets[sid].size());
                    for (int32_t ci : D.sets[sid]) {
                        F.put(D.arena[ci].rep);
                        F.put_vec(D.arena[ci].objs);
                    }
                }
                if (!F.ok || std::fflush(F.f) != 0)
                    return fail(c, CM_ERR_ARG, "cannot write the state file");
            }
            if (std::rename(tmp.c_str(), state_path) != 0)
                return fail(c, CM_ERR_ARG, "cannot write the state file");
            return CM_STOPPED;
        }
    }
    cm_result* res = (cm_result*)std::calloc(1, sizeof(cm_result));
    if (!res) return fail(c, CM_ERR_OOM, "host allocation failed");
    res->n_seqs = n_seqs;
    std::vector<int32_t> final_set;
    if (!q.empty()) final_set = D.sets[q.front()];
    r = D.finish(final_set, res);
    if (r) { cm_result_free(res); return r; }
    res->seconds = earlier_seconds + elapsed();
    *out = res;
    return CM_OK;
}

int cluster_merge(cm_ctx* c, const uint8_t* seqs, const int64_t* offsets, int32_t n_seqs,
                  const int8_t* matrix, int32_t gap_open, int32_t gap_extend,
                  const cm_params* params, cm_result** out, uint32_t flags)
{
    return run_cluster_merge(c, seqs, offsets, n_seqs, matrix, gap_open, gap_extend, params,
                             nullptr, 0.0, out, flags);
}

int cluster_merge_resume(cm_ctx* c, const uint8_t* seqs, const int64_t* offsets,
                         int32_t n_seqs, const int8_t* matrix, int32_t gap_open,
                         int32_t gap_extend, const cm_params* params, const char* state_path,
                         double budget_seconds, cm_result** out, uint32_t flags)
{
    if (!state_path) return c ? fail(c, CM_ERR_ARG, "null state path") : CM_ERR_ARG;
    return run_cluster_merge(c, seqs, offsets, n_seqs, matrix, gap_open, gap_extend, params,
                             state_path, budget_seconds, out, flags);
}

int greedy_cluster(cm_ctx* c, const uint8_t* seqs, const int64_t* offsets, int32_t n_seqs,
                   const int8_t* matrix, int32_t gap_open, int32_t gap_extend,
                   const cm_params* params, cm_result** out, uint32_t flags)
{
    if (!c) return CM_ERR_ARG;
    NvtxRange range("greedy_cluster");
    if (!out || !params) return fail(c, CM_ERR_ARG, "null params / out");
    *out = nullptr;
    CUDA_TRY(cudaSetDevice(c->device));
    const auto t0 = std::chrono::steady_clock::now();
    Prepared P;
    int r = prepare(c, seqs, offsets, n_seqs, matrix, gap_open, gap_extend, flags, P);
    if (r) return r;
    if (!P.symmetric)
        return fail(c, CM_ERR_ARG, "greedy_cluster needs a symmetric substitution matrix");
    if (params->use_ranker || params->merge_mode)
        return fail(c, CM_ERR_ARG, "greedy_cluster takes neither the ranker nor a merge mode");
    cm_result* res = (cm_result*)std::calloc(1, sizeof(cm_result));
    if (!res) return fail(c, CM_ERR_OOM, "host allocation failed");
    res->n_seqs = n_seqs;
    Driver D(c, P, *params, flags & CM_FORCE_INT32);
    std::vector<int32_t> final_set;
    r = D.run_greedy(n_seqs, std::max(1, c->greedy_chunk), final_set);
    if (!r) r = D.finish(final_set, res);
    if (r) { cm_result_free(res); return r; }
    res->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = res;
    return CM_OK;
}

void cm_result_free(cm_result* r)
{
    if (!r) return;
    std::free(r->reps);
    std::free(r->cl_offsets);
    std::free(r->members);
    std::free(r->pairs);
    std::free(r->scores);
    std::free(r);
}

}  // extern "C"
