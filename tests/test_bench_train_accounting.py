"""The benchmark's learned-path record (bench.train_ranker) on the CPU with a stand-in context:
the training pairs, the held-out split, the pruning threshold and the algorithmic convolution
work it reports (3 x the forward FLOPs per residue of every protein in the training pairs, per
epoch) -- no GPU call is made."""
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
