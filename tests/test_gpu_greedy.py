"""GPU incremental greedy clustering (greedy_cluster: the paper's comparison method, run on
the same kernels) against the oracle's greedy clustering: clusters with their member order,
similar pairs and the comparison counts must be identical -- on the small families set (one
device batch of sequences) and on 2,300 short proteins (two batches, so the speculative
scoring of a batch against itself decides representatives created inside it)."""
import numpy as np
import pytest

import oracle
from oracle.greedy import greedy_cluster as oracle_greedy
import paper_1908_10574_gb300 as cm
from paper_1908_10574_gb300 import synth

pytestmark = pytest.mark.gpu
S62 = synth.BLOSUM62


def _matrix(ss):
    _, scores = oracle.all_pairs(ss.seqs, ss.offsets, S62, 11, 1, T=-1)
    n = len(ss)
    M = np.zeros((n, n), np.int64)
    M[np.triu_indices(n, 1)] = scores
    return M + M.T


def _check(got, want):
    assert got["clusters"] == want["clusters"]
    assert got["pairs"].tolist() == want["pairs"].tolist()
    st, ws = got["stats"], want["stats"]
    assert st["rep_comparisons"] == ws["rep"]
    assert st["intra_comparisons"] == ws["intra"]
    assert st["full_merges"] == ws["full_merges"]


@pytest.mark.parametrize("T,mT,mU", [(60, 83, 15), (100, 138, 15), (60, 10 ** 9, 15)])
def test_greedy_small_families_matches_oracle(T, mT, mU):
    ss = synth.small_families()
    ctx = cm.Context(0)
    got = ctx.greedy_cluster(ss.seqs, ss.offsets, S62, 11, 1, T, mT, mU)
    want = oracle_greedy(ss.seqs, ss.offsets, S62, 11, 1, T=T, mT=mT, mU=mU,
                         score_matrix=_matrix(ss))
    _check(got, want)


def test_greedy_two_batches_matches_oracle_and_truth():
    rng = np.random.default_rng(1908)
    ss = synth.families(230, 10, rng.integers(50, 151, size=230), stream=41)
    assert len(ss) > 2048
    M = _matrix(ss)
    ctx = cm.Context(0)
    got = ctx.greedy_cluster(ss.seqs, ss.offsets, S62, 11, 1, 60, 83, 15)
    want = oracle_greedy(ss.seqs, ss.offsets, S62, 11, 1, T=60, mT=83, mU=15, score_matrix=M)
    _check(got, want)
    assert got["stats"]["rounds"] == 2
    truth = np.argwhere(np.triu(M > 60, 1))
    tset = set(map(tuple, truth.tolist()))
    assert all((int(i), int(j)) in tset for i, j, _ in got["pairs"])
    assert oracle.recall(got["pairs"], truth) > 0.95
