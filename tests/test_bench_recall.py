"""Recall bookkeeping of the benchmark's ClusterMerge runs (CPU): within-family pairs, recall
restricted to a protein sample (numbering of the sample's all-against-all), and recall over a
pair stratum."""
import importlib.util
import os

import numpy as np

import oracle
from paper_1908_10574_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
bench = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(bench)


def test_family_pairs():
    fam = np.array([2, 0, 2, 1, 0, 2, 7])
    got = sorted(map(tuple, bench.family_pairs(fam).tolist()))
    assert got == [(0, 2), (0, 5), (1, 4), (2, 5)]
    assert len(bench.family_pairs(np.arange(5))) == 0
    f = synth.proteome(400, family_size=8, singleton_frac=0.2, stream=2).family
    p = bench.family_pairs(f)
    assert (p[:, 0] < p[:, 1]).all() and (f[p[:, 0]] == f[p[:, 1]]).all()
    _, counts = np.unique(f, return_counts=True)
    assert len(p) == int((counts * (counts - 1) // 2).sum())


def test_subset_recall_hand_case():
    subset = np.array([1, 3, 4, 7])
    truth_sub = np.array([[0, 1], [3, 2], [1, 2]])          # global (1,3), (4,7), (3,4)
    found = np.array([[1, 3], [3, 4], [0, 1], [2, 9]])
    r, nt, nf = bench.subset_recall(found, subset, truth_sub)
    assert (nt, nf) == (3, 2) and abs(r - 2 / 3) < 1e-12


def test_subset_recall_matches_set_arithmetic():
    rng = np.random.default_rng(5)
    for _ in range(50):
        n = 60
        subset = np.sort(rng.choice(n, size=int(rng.integers(2, 30)), replace=False))
        a = rng.integers(0, n, size=(200, 2))
        found = np.sort(a[a[:, 0] != a[:, 1]], axis=1)
        b = rng.integers(0, len(subset), size=(40, 2))
        truth_sub = b[b[:, 0] != b[:, 1]]
        pos = {int(g): k for k, g in enumerate(subset)}
        fs = {(min(pos[i], pos[j]), max(pos[i], pos[j])) for i, j in found.tolist()
              if i in pos and j in pos}
        ts = {(min(i, j), max(i, j)) for i, j in truth_sub.tolist()}
        r, nt, nf = bench.subset_recall(found, subset, truth_sub)
        assert nt == len(ts) and nf == len(fs)
        assert abs(r - len(fs & ts) / max(len(ts), 1)) < 1e-12


def test_subset_recall_with_the_oracle_all_against_all():
    """A sample's own all-against-all (in sample numbering) is the full truth restricted to the
    sample: reporting every similar pair of the full set gives recall 1 on any sample."""
    ss = synth.small_families()
    truth, _ = oracle.all_pairs(ss.seqs, ss.offsets, synth.BLOSUM62, 11, 1, T=60)
    subset = np.sort(np.random.default_rng(3).choice(len(ss), size=70, replace=False))
    sub = ss.subset(subset)
    truth_sub, _ = oracle.all_pairs(sub.seqs, sub.offsets, synth.BLOSUM62, 11, 1, T=60)
    r, nt, nf = bench.subset_recall(truth[:, :2], subset, truth_sub[:, :2])
    inside = np.isin(truth[:, 0], subset) & np.isin(truth[:, 1], subset)
    assert r == 1.0 and nt == nf == int(inside.sum()) and nt > 0


def test_stratum_recall():
    truth = np.array([[1, 2], [5, 3], [0, 9]])
    found = np.array([[2, 1], [3, 5], [4, 6]])
    assert abs(bench.stratum_recall(found, truth, 10) - 2 / 3) < 1e-12
    assert bench.stratum_recall(found, np.zeros((0, 2)), 10) == 1.0
