// Host-only: mini-batches of the ranker's training pairs that can reuse each sequence embedding
// as often as the pair list allows.  A training step embeds every distinct sequence of its batch
// (forward and backward through the convolutions), while the loss is a sum over pairs, so
// the step's cost follows the distinct sequences and its supervision follows the pairs.  On
// request the pairs are grouped by the connected components of the pair graph (sequences as
// nodes): a batch holds whole components, as many as fit in `batch_pairs` pairs, and a
// component with more pairs is cut into chunks of `batch_pairs`.  Pairs drawn within groups
// of sequences (training sets built that way) thus train one group per step with every pair
// of it.  Otherwise all pairs form one component and every epoch is shuffled chunks of
// batch_pairs pairs (grouping small components of an arbitrary pair list can make batches of
// one label only).  Every epoch shuffles the component order and the pairs inside each
// component.  Plain C++ (no CUDA), so the host tests compile it on its own.
#pragma once

#include <algorithm>
#include <cstdint>
#include <numeric>
#include <random>
#include <vector>

namespace cm {

struct TrainComponents {
    std::vector<int64_t> off;     // components' slices of `pairs` (n_components + 1)
    std::vector<int64_t> pairs;   // pair indices grouped by component
};

// All pairs as one component (list order): epochs are then shuffled chunks of batch_pairs.
inline TrainComponents train_one_component(int64_t n_pairs)
{
    TrainComponents C;
    C.off = {0, n_pairs};
    C.pairs.resize((size_t)n_pairs);
    std::iota(C.pairs.begin(), C.pairs.end(), 0);
    if (n_pairs == 0) C.off.assign(1, 0);
    return C;
}

// Components of the graph whose nodes are sequences 0..n_seqs-1 and whose edges are the
// pairs (pairs[2k], pairs[2k+1]); pairs must index [0, n_seqs).  Component order: by the
// smallest pair index they hold; pairs keep their list order inside a component.
inline TrainComponents train_components(const int32_t* pairs, int64_t n_pairs, int32_t n_seqs)
{
    std::vector<int32_t> parent((size_t)n_seqs);
    std::iota(parent.begin(), parent.end(), 0);
    auto find = [&](int32_t x) {
        while (parent[x] != x) {
            parent[x] = parent[parent[x]];
            x = parent[x];
        }
        return x;
    };
    for (int64_t k = 0; k < n_pairs; ++k) {
        const int32_t a = find(pairs[2 * k]), b = find(pairs[2 * k + 1]);
        if (a != b) parent[std::max(a, b)] = std::min(a, b);
    }
    // number the roots by first appearance in pair order
    std::vector<int32_t> id((size_t)n_seqs, -1);
    std::vector<int64_t> comp_of((size_t)n_pairs);
    int64_t nc = 0;
    for (int64_t k = 0; k < n_pairs; ++k) {
        const int32_t r = find(pairs[2 * k]);
        if (id[r] < 0) id[r] = (int32_t)nc++;
        comp_of[k] = id[r];
    }
    TrainComponents C;
    C.off.assign((size_t)nc + 1, 0);
    for (int64_t k = 0; k < n_pairs; ++k) ++C.off[comp_of[k] + 1];
    for (int64_t c = 0; c < nc; ++c) C.off[c + 1] += C.off[c];
    C.pairs.resize((size_t)n_pairs);
    std::vector<int64_t> fill(C.off.begin(), C.off.end() - 1);
    for (int64_t k = 0; k < n_pairs; ++k) C.pairs[fill[comp_of[k]]++] = k;
    return C;
}

// One epoch's batches: `order` receives the pair indices of every batch one after another,
// `bounds` the batch boundaries in `order` (n_batches + 1, starting at 0).  Consumes `g`.
inline void train_epoch_batches(const TrainComponents& C, int64_t batch_pairs,
                                std::mt19937_64& g, std::vector<int64_t>& order,
                                std::vector<int64_t>& bounds)
{
    const int64_t nc = (int64_t)C.off.size() - 1;
    std::vector<int64_t> perm((size_t)nc);
    std::iota(perm.begin(), perm.end(), 0);
    std::shuffle(perm.begin(), perm.end(), g);
    order.clear();
    bounds.assign(1, 0);
    int64_t open = 0;                       // pairs in the batch being filled
    for (int64_t c : perm) {
        const int64_t b = C.off[c], e = C.off[c + 1], n = e - b;
        const size_t at = order.size();
        order.insert(order.end(), C.pairs.begin() + b, C.pairs.begin() + e);
        std::shuffle(order.begin() + (int64_t)at, order.end(), g);
        if (n <= batch_pairs) {
            if (open + n > batch_pairs) {   // close the batch before this component
                bounds.push_back((int64_t)at);
                open = 0;
            }
            open += n;
            continue;
        }
        // a component larger than a batch: close the open batch, then chunks of batch_pairs
        if (open > 0) bounds.push_back((int64_t)at);
        int64_t s = (int64_t)at;
        while ((int64_t)order.size() - s > batch_pairs) {
            s += batch_pairs;
            bounds.push_back(s);
        }
        open = (int64_t)order.size() - s;
    }
    if (open > 0) bounds.push_back((int64_t)order.size());
}

}  // namespace cm
