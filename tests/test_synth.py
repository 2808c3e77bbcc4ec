"""The synthetic inputs match their stated recipe (CPU only): proteome-shaped sets, families,
and the long-tail tandem repeats (the matrix is pinned with the oracle's tests)."""
import numpy as np

import oracle
from paper_1908_10574_gb300 import synth


def test_proteome_shape_and_determinism():
    ss = synth.proteome(20000, 10)
    L = ss.lengths
    assert len(ss) == 20000
    assert L.min() >= 1 and L.max() <= 5000 + 500          # clip 30-5000 on roots, members +-indels
    assert 300 < np.median(L) < 420                          # lognormal median 350 (roots)
    fam, counts = np.unique(ss.family, return_counts=True)
    assert len(fam) == 2000 and (counts == 10).all()
    again = synth.proteome(20000, 10)
    assert np.array_equal(again.seqs, ss.seqs) and np.array_equal(again.offsets, ss.offsets)
    assert int(ss.seqs.max()) <= 19


def test_proteome_with_singletons():
    ss = synth.proteome(5000, family_size=8, singleton_frac=0.2, stream=7)
    _, counts = np.unique(ss.family, return_counts=True)
    assert (counts == 1).sum() == 1000
    assert (counts == 8).sum() == 500


def test_small_families_recipe():
    ss = synth.small_families()
    _, counts = np.unique(ss.family, return_counts=True)
    assert len(ss) == 200 and len(counts) == 20 and (counts == 10).all()
    assert ss.lengths.min() >= 40 and ss.lengths.max() <= 340   # roots 50-300, 5 % indels


def test_long_tail_motif_families():
    base = synth.proteome(20, family_size=10, stream=9)
    ss = synth.long_tail(base, 4, 2, stream=9, lo=3000, hi=4000)
    L = ss.lengths
    assert len(ss) == 24 and ((L[20:] >= 3000) & (L[20:] <= 4000)).all()
    assert np.array_equal(ss.seqs[:base.offsets[-1]], base.seqs)
    f = ss.family[20:]
    assert f[0] == f[2] and f[1] == f[3] and f[0] != f[1]
    same = oracle.sw_score(ss[20], ss[22], synth.BLOSUM62, 11, 1)
    cross = oracle.sw_score(ss[20], ss[21], synth.BLOSUM62, 11, 1)
    assert same > 10000 and cross < 500              # a whole-length alignment vs chance
