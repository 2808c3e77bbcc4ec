"""Host logic of the GPU ClusterMerge driver against the oracle's Algorithms 1 and 2 (CPU).

csrc/cluster_merge.cu holds no kernels: it plans device batches and replays Algorithm 1 over
what they return.  Here it is compiled with the host compiler and linked with
tests/driver_mock.cpp, which replaces every device-layer call with a host mock of its
documented result: scores, alignment cells and the ranked path's selection bitmap come from a
random similarity instance, so the replay, the exact visit counts, the exchange waves, the
transposed blocks of long representatives and the device-planned lists of ranked merges are
checked on hundreds of random merge trees, including ones the GPU tests never reach.  The
oracle runs Algorithm 2 with the same similarity (`score`, `transitive` and the pruning hook
`keep`); clusters with their member order, similar pairs and all comparison counts must be
identical, for sequential merges, for independent partial merges (CM_MERGE_PARTIAL, the
oracle's merge_partial) and for the incremental greedy clustering (greedy_cluster, the
oracle's greedy)."""
import importlib
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

ocm = importlib.import_module("oracle.cluster_merge")   # the module (the package re-exports a function of that name)
ogr = importlib.import_module("oracle.greedy")

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1908_10574_gb300", "csrc")


def _cuda_include():
    for base in (os.environ.get("CUDA_HOME"), os.environ.get("CUDA_PATH"),
                 os.path.dirname(os.path.dirname(shutil.which("nvcc") or "")), "/usr/local/cuda"):
        if base and os.path.exists(os.path.join(base, "include", "cuda_runtime.h")):
            return os.path.join(base, "include")
    return None


def _instance(rng):
    n = int(rng.choice([0, 1, 2, 3, 5, 8, 13, 21, 34, 55, 70]))
    T = int(rng.choice([60, 100]))
    mT = T + int(rng.choice([10, 38, 80]))
    mU = int(rng.choice([5, 15, 40]))
    L = np.exp(rng.normal(np.log(300), 0.7, size=n)).astype(np.int64).clip(1, 3000)
    long_ = rng.random(n) < 0.08                       # longer than a stream subject
    L[long_] = rng.integers(4097, 6500, size=int(long_.sum()))
    L[rng.random(n) < 0.04] = 0                        # empty proteins
    fam = rng.integers(0, max(1, n // 3), size=n)
    M = rng.integers(0, T + 1, size=(n, n))             # unrelated: not similar
    same = fam[:, None] == fam[None, :]
    hi = T + 1 + rng.integers(0, mT - T + 60, size=(n, n))
    M = np.where(same & (rng.random((n, n)) < 0.85), hi, M)
    M = np.where(~same & (rng.random((n, n)) < 0.03), T + 1 + rng.integers(0, 40, size=(n, n)), M)
    M = np.triu(M, 1)
    M = M + M.T
    zero = L == 0
    M[zero, :] = 0
    M[:, zero] = 0
    # residues of x covered by the alignment of (x, y): often within mU of the whole
    # length, otherwise well short of it
    short = rng.integers(0, mU, size=(n, n))
    far = rng.integers(mU, mU + 200, size=(n, n))
    unc = np.where(rng.random((n, n)) < 0.6, short, far)
    cov = np.clip(L[:, None] - unc, 0, L[:, None])
    cov = np.maximum(cov, (L[:, None] > 0).astype(np.int64))
    keep = rng.random((n, n)) < 0.7
    keep = np.triu(keep, 1)
    keep = keep | keep.T
    use_ranker = int(rng.random() < 0.5)
    min_pairs = int(rng.choice([0, 1, 4, 30]))
    partial = int(rng.random() < 0.4)
    greedy = int(rng.random() < 0.25)
    if greedy:
        use_ranker = partial = 0
    resume = int(not greedy and rng.random() < 0.3)
    return dict(n=n, T=T, mT=mT, mU=mU, use_ranker=use_ranker, min_pairs=min_pairs, L=L, M=M,
                cov=cov, keep=keep, partial=partial, greedy=greedy, resume=resume)


def _serialise(insts):
    out = [str(len(insts))]
    for d in insts:
        out.append("%d %d %d %d %d %d %d %d" % (d["n"], d["T"], d["mT"], d["mU"], d["use_ranker"],
                                               d["min_pairs"], d["partial"],
                                               2 if d["resume"] else d["greedy"]))
        for key in ("L", "M", "cov", "keep"):
            out.append(" ".join(str(int(v)) for v in np.asarray(d[key]).reshape(-1)))
    return "\n".join(out) + "\n"


def _parse(text, k):
    tok = text.split()
    pos = 0
    res = []
    for _ in range(k):
        if tok[pos] == "error":
            raise AssertionError("driver error: " + " ".join(tok[pos:pos + 12]))
        assert tok[pos] == "clusters"
        nc = int(tok[pos + 1])
        pos += 2
        clusters = []
        for _ in range(nc):
            rep, size = int(tok[pos]), int(tok[pos + 1])
            clusters.append((rep, [int(x) for x in tok[pos + 2:pos + 2 + size]]))
            pos += 2 + size
        assert tok[pos] == "pairs"
        npairs = int(tok[pos + 1])
        pos += 2
        pairs = [tuple(int(x) for x in tok[pos + 3 * i:pos + 3 * i + 3]) for i in range(npairs)]
        pos += 3 * npairs
        assert tok[pos] == "stats"
        stats = [int(x) for x in tok[pos + 1:pos + 7]]
        pos += 7
        res.append((clusters, pairs, stats))
    return res


def _oracle(d):
    M, cov, L, keep = d["M"], d["cov"], d["L"], d["keep"]
    T, mT, mU = d["T"], d["mT"], d["mU"]

    def score(x, y):
        return int(M[x, y])

    def transitive(r1, r2, s):
        if not s > mT:
            return False, False
        return int(L[r1] - cov[r1, r2]) < mU, int(L[r2] - cov[r2, r1]) < mU

    kf = (lambda a, b: bool(keep[a, b])) if d["use_ranker"] else None
    if d["greedy"]:
        final, stats = ogr.greedy(d["n"], score, lambda x, r: int(L[x] - cov[x, r]), T, mT, mU)
    else:
        final, stats = ocm.bottom_up_merge(d["n"], score, transitive, T, keep=kf,
                                           min_pairs=d["min_pairs"], partial=bool(d["partial"]))
    pairs = ocm.intra_cluster_pairs(final, score, T, stats)
    clusters = [(c.rep, list(c.objs)) for c in final]
    return clusters, [tuple(map(int, p)) for p in pairs.tolist()], \
        [stats["rep"], stats["exchange"], stats["intra"], stats["full_merges"],
         stats["exchanges"], stats["merges"]]


@pytest.mark.skipif(shutil.which("g++") is None or _cuda_include() is None,
                    reason="no host C++ compiler or CUDA headers")
def test_driver_replay_matches_oracle(tmp_path):
    exe = str(tmp_path / "driver_mock")
    subprocess.run(["g++", "-std=c++17", "-O1", "-Wall", "-Werror", "-I", CSRC, "-I",
                    _cuda_include(), "-x", "c++", os.path.join(CSRC, "cluster_merge.cu"),
                    "-x", "c++", os.path.join(HERE, "driver_mock.cpp"), "-o", exe], check=True)
    rng = np.random.default_rng(1908)
    insts = [_instance(rng) for _ in range(400)]
    out = subprocess.run([exe, str(tmp_path / "cm.state")], input=_serialise(insts),
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    got = _parse(out.stdout, len(insts))
    exercised = {"ranked": 0, "full": 0, "exchange": 0, "long": 0, "partial": 0, "greedy": 0,
                 "resumed": sum(int(x) > 2 for x in re.findall(r"resumed (\d+)", out.stderr)),
                 "long x long": int(re.findall(r"int32 pairs (\d+)", out.stderr)[-1])}
    for d, g in zip(insts, got):
        want = _oracle(d)
        assert g[0] == want[0], ("clusters", d["n"], d["use_ranker"])
        assert g[1] == want[1], ("pairs", d["n"])
        assert g[2] == want[2], ("stats", g[2], want[2])
        exercised["ranked"] += d["use_ranker"] and d["n"] > 2
        exercised["full"] += want[2][3] > 0
        exercised["exchange"] += want[2][4] > 0
        exercised["long"] += bool((d["L"] > 4096).any())
        exercised["partial"] += d["partial"] and want[2][3] > 0 and want[2][4] > 0
        exercised["greedy"] += d["greedy"] and want[2][3] > 0 and d["n"] > 8
    assert min(exercised.values()) >= 20, exercised
