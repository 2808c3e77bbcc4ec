"""The benchmark's learned-path record (bench.train_ranker) and the default line's ClusterMerge
comparison (bench.cm_comparison) on the CPU with a stand-in context: the training pairs, the
held-out split, the pruning threshold, the algorithmic convolution work it reports (3 x the
forward FLOPs per residue of every protein in the training pairs, per epoch) and the keys of
the comparison record -- no GPU call is made."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_1908_10574_gb300 import synth  # noqa: E402


class StandInContext:
    """Records the calls; scores pairs of one family above T, others below; logits = score."""

    def __init__(self, family):
        self.family = family
        self.trained = None

    def sw_score_batch(self, seqs, offsets, pairs, matrix, go, ge):
        same = self.family[pairs[:, 0]] == self.family[pairs[:, 1]]
        return np.where(same, bench.T_SIG + 50, bench.T_SIG - 50).astype(np.int32)

    def ranker_init(self, seed):
        pass

    def ranker_standardize(self, seqs, offsets, max_sample=0):
        pass

    def ranker_train(self, seqs, offsets, pairs, y, epochs, batch_pairs, lr, seed, flags):
        self.trained = (len(pairs), epochs, flags)
        return 0.5

    def ranker_logits(self, seqs, offsets, pairs):
        same = self.family[pairs[:, 0]] == self.family[pairs[:, 1]]
        return np.where(same, 2.0, -2.0).astype(np.float32) + 0.01 * np.arange(len(pairs))


def test_training_work_accounting():
    ss = synth.proteome(600, family_size=6, singleton_frac=0.2, stream=9)
    ctx = StandInContext(ss.family)
    info = bench.train_ranker(ctx, 600, 4000, 3, 0.999, train_set=ss, group=64)
    n_train = info["train_pairs"]
    assert ctx.trained[0] == n_train and ctx.trained[1] == 3
    assert n_train + info["heldout_pairs"] >= 4000 * 0.9
    # the same pairs again (same seed) -> the residues of the proteins they touch, per epoch
    rng = np.random.default_rng(13)
    pairs, _ = bench.grouped_training_pairs(ss.family, 4000, 64, rng)
    used = np.unique(pairs[:n_train].reshape(-1))
    flops = 3.0 * bench.RANKER_FWD_FLOPS_PER_ROW * float(ss.lengths[used].sum()) * 3
    assert info["train_tflops"] > 0
    assert abs(info["train_tflops"] * info["train_seconds"] * 1e12 - flops) <= 1e-6 * flops
    assert bench.RANKER_FWD_FLOPS_PER_ROW == 2 * 9 * (32 * 128 + 128 * 128 + 128 * 128)
    assert 0 < info["train_frac_of_bf16_sustained"] < info["train_tflops"]
    # separable stand-in logits: every held-out negative is pruned at a 99.9 % keep
    assert info["heldout_auc"] == 1.0 and info["heldout_negatives_kept"] == 0.0


class StandInMerge(StandInContext):
    """Adds ClusterMerge and the all-against-all: similar pairs = the within-family pairs."""

    def _family_pairs(self):
        fp = bench.family_pairs(self.family)
        return np.concatenate([fp, np.full((len(fp), 1), bench.T_SIG + 50)], 1).astype(np.int64)

    def cluster_merge(self, seqs, offsets, matrix, go, ge, T, mT, mU, use_ranker=False,
                      prune_logit=0.0, ranker_min_pairs=0):
        keys = ("rep_comparisons", "exchange_comparisons", "intra_comparisons",
                "comparisons_scored", "full_merges", "exchanges", "rounds", "t_rep", "t_cells",
                "t_exchange", "t_intra", "t_rank", "ranker_selected")
        return {"pairs": self._family_pairs(), "clusters": [(0, [0])],
                "stats": {k: 1 for k in keys}}

    def sw_allpairs(self, seqs, offsets, matrix, go, ge, T, part, parts, capacity=0):
        p = self._family_pairs()
        return p[part::parts, :2].astype(np.int32), p[part::parts, 2].astype(np.int32)


def test_comparison_record_on_the_cpu():
    """The default bench line's ClusterMerge comparison, end to end on the stand-in: every
    key of the record is present and the learned entry carries the training work."""
    out = bench.cm_comparison(StandInMerge(synth.proteome(300, family_size=8, singleton_frac=0.2,
                                                          stream=3).family), n_seqs=300)
    assert out["plain"]["recall"] == 1.0 and out["truth_pairs"] > 0
    (lr,) = out["learned"]
    assert lr["recall"] == 1.0 and lr["train_tflops"] > 0
    assert 0 < lr["train_frac_of_bf16_sustained"] < 1e6
    assert lr["seconds_total"] >= lr["seconds_merge"] > 0
