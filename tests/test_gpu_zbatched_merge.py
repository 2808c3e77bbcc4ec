"""GPU ClusterMerge with the representative wave cut into small device batches
(cm_set_batch_limit): rounds whose rep x rep cross products exceed the limit run as several
batches cut between query rows, and clusters, similar pairs and comparison counts must still
equal those of the oracle's sequential Algorithms 1 and 2 exactly.  (A 1M-protein proteome's
top merges exceed device memory as one batch; the limit here is set low so that small inputs
take the same path.)"""
import numpy as np
import pytest

import oracle
import paper_1908_10574_gb300 as cm
from paper_1908_10574_gb300 import synth

pytestmark = pytest.mark.gpu
S62 = synth.BLOSUM62


def _oracle_cm(ss, T, mT, mU):
    _, scores = oracle.all_pairs(ss.seqs, ss.offsets, S62, 11, 1, T=T)
    n = len(ss)
    M = np.zeros((n, n), np.int64)
    M[np.triu_indices(n, 1)] = scores
    M = M + M.T
    return oracle.cluster_merge(ss.seqs, ss.offsets, S62, 11, 1, T=T, mT=mT, mU=mU,
                                score_matrix=M)


def _check(got, want):
    assert got["clusters"] == want["clusters"]
    assert got["pairs"].tolist() == want["pairs"].tolist()
    st, ws = got["stats"], want["stats"]
    assert st["rep_comparisons"] == ws["rep"]
    assert st["exchange_comparisons"] == ws["exchange"]
    assert st["intra_comparisons"] == ws["intra"]
    assert st["full_merges"] == ws["full_merges"]
    assert st["exchanges"] == ws["exchanges"]
    assert st["merges"] == ws["merges"]


@pytest.fixture(scope="module")
def case():
    full = synth.proteome(5000, family_size=8, singleton_frac=0.2, stream=7)
    ss = full.subset(np.arange(600))
    return ss, _oracle_cm(ss, 100, 138, 15)


@pytest.mark.parametrize("limit", [1024, 5000])
def test_batched_rep_wave_matches_oracle(case, limit):
    ss, want = case
    ctx = cm.Context(0)
    one = ctx.cluster_merge(ss.seqs, ss.offsets, S62, 11, 1, 100, 138, 15)
    _check(one, want)
    ctx.set_batch_limit(limit)
    got = ctx.cluster_merge(ss.seqs, ss.offsets, S62, 11, 1, 100, 138, 15)
    _check(got, want)
    # the larger rounds' cross products exceed the limit and ran as several device batches
    assert got["stats"]["gpu_batches"] > one["stats"]["gpu_batches"]
    assert got["stats"]["comparisons_scored"] == one["stats"]["comparisons_scored"]


@pytest.fixture(scope="module")
def case2k():
    """2,000 proteins of the 100k benchmark set (same recipe and stream): 200 whole families of
    8 and 400 singletons, in the set's order."""
    full = synth.proteome(100000, family_size=8, singleton_frac=0.2, stream=3)
    fam, counts = np.unique(full.family, return_counts=True)
    rng = np.random.default_rng(1908)
    fams = rng.choice(fam[counts == 8], 200, replace=False)
    singles = rng.choice(fam[counts == 1], 400, replace=False)
    ids = np.flatnonzero(np.isin(full.family, np.concatenate([fams, singles])))
    assert len(ids) == 2000
    ss = full.subset(ids)
    return ss, _oracle_cm(ss, 100, 138, 15)


@pytest.mark.parametrize("limit", [0, 1 << 16])
def test_2k_subset_of_the_100k_set_exact(case2k, limit):
    """Clusters, similar pairs and comparison counts equal the oracle's on the 2k subset, with
    whole rounds in one device batch and in batches of 65,536 slots."""
    ss, want = case2k
    ctx = cm.Context(0)
    ctx.set_batch_limit(limit)
    got = ctx.cluster_merge(ss.seqs, ss.offsets, S62, 11, 1, 100, 138, 15)
    _check(got, want)


def test_batch_limit_argument_checks():
    ctx = cm.Context(0)
    with pytest.raises(cm.CMError):
        ctx.set_batch_limit(1000)
    ctx.set_batch_limit(0)


def test_partial_merges_on_the_2k_subset(case2k):
    """Independent partial merges (CM_MERGE_PARTIAL, Sec. 5) on the 2k subset: clusters,
    similar pairs and counts equal the oracle's partial-merge Algorithm 2, every pair found
    is in the all-against-all truth, and recall is within 0.1 % of the sequential merge's."""
    ss, want_seq = case2k
    _, scores = oracle.all_pairs(ss.seqs, ss.offsets, S62, 11, 1, T=100)
    n = len(ss)
    M = np.zeros((n, n), np.int64)
    M[np.triu_indices(n, 1)] = scores
    M = M + M.T
    want = oracle.cluster_merge(ss.seqs, ss.offsets, S62, 11, 1, T=100, mT=138, mU=15,
                                score_matrix=M, partial=True)
    ctx = cm.Context(0)
    got = ctx.cluster_merge(ss.seqs, ss.offsets, S62, 11, 1, 100, 138, 15,
                            merge_mode=cm.CM_MERGE_PARTIAL)
    _check(got, want)
    truth, _ = oracle.all_pairs(ss.seqs, ss.offsets, S62, 11, 1, T=100)
    tset = {(int(i), int(j)) for i, j, _ in truth}
    assert all((int(i), int(j)) in tset for i, j, _ in got["pairs"])
    r_par = oracle.recall(got["pairs"], truth)
    r_seq = oracle.recall(want_seq["pairs"], truth)
    assert abs(r_par - r_seq) <= 1e-3, (r_par, r_seq)
    # partial merges visit the clusters other partial merges fully merged
    assert got["stats"]["rep_comparisons"] >= want_seq["stats"]["rep"]
    with pytest.raises(cm.CMError):
        ctx.cluster_merge(ss.seqs, ss.offsets, S62, 11, 1, 100, 138, 15, merge_mode=2)
