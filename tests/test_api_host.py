"""Host runtime of the C ABI on the CPU: csrc/api.cu and csrc/cluster_merge.cu compiled with the
host compiler and linked with tests/api_mock.cpp, which mocks the kernel launchers and the CUDA
runtime with a fake deterministic similarity (see that file for its definition, restated in
`_score` and `_cells` below).  Everything above the kernels runs for real: input validation,
pair grouping and slot maps of sw_score_batch, the planner and launch bins, the int16 -> int32
rerun loop (saturated fake scores), the two-phase compaction, the all-against-all parts, the
two-pass cells pipeline, the bounded rep-wave batches, and ClusterMerge end to end (plain and
ranked).  Scores and cells must equal the fake similarity's; ClusterMerge must equal the
oracle's Algorithms 1 and 2 on that similarity."""
import importlib
import os
import shutil
import subprocess

import numpy as np
import pytest

ocm = importlib.import_module("oracle.cluster_merge")

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1908_10574_gb300", "csrc")
M64 = (1 << 64) - 1
CM_DEVICE_PTRS, CM_ASCII, CM_FORCE_INT32 = 0x1, 0x2, 0x8


def _cuda_include():
    for base in (os.environ.get("CUDA_HOME"), os.environ.get("CUDA_PATH"),
                 os.path.dirname(os.path.dirname(shutil.which("nvcc") or "")), "/usr/local/cuda"):
        if base and os.path.exists(os.path.join(base, "include", "cuda_runtime.h")):
            return os.path.join(base, "include")
    return None


def _mix(z):
    z = (z + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def _score(a, b, L, sym, sparse=False):
    a, b = int(a), int(b)
    if L[a] == 0 or L[b] == 0:
        return 0
    u, v = (min(a, b), max(a, b)) if sym else (a, b)
    h = _mix(u * 1000003 + v)
    t, r = h >> 32, h % 1000
    if r < (985 if sparse else 550):
        return t % 100
    if r < (997 if sparse else 940):
        return 101 + t % 300
    return 30000 + t % 20000


def _extent(L, u):
    u = min(u, L - 1)
    left = u // 2
    return 1 + left, L - (u - left)


def _cells(a, b, L, sym, sparse=False):
    a, b = int(a), int(b)
    s = _score(a, b, L, sym, sparse)
    if s <= 0:
        return (0, 0, 0, 0, 0)
    h = _mix(a * 7919 + b * 104729 + 17)
    ua = (h >> 8) % 15 if h & 1 else 15 + (h >> 8) % 40
    ub = (h >> 24) % 15 if h & 2 else 15 + (h >> 24) % 40
    i0, i1 = _extent(int(L[a]), ua)
    j0, j1 = _extent(int(L[b]), ub)
    return (s, i0, i1, j0, j1)


def _keep(x, y):
    u, v = min(int(x), int(y)), max(int(x), int(y))
    return _mix(u * 31 + v + 5) % 10 < 7


def _lengths(rng, n):
    L = np.exp(rng.normal(np.log(300), 0.8, size=n)).astype(np.int64).clip(1, 2000)
    pick = rng.random(n)
    L[pick < 0.10] = rng.integers(2048, 9000, size=int((pick < 0.10).sum()))   # long pairs
    L[(pick >= 0.10) & (pick < 0.14)] = 0                                         # empty
    return L


class Harness:
    def __init__(self, exe):
        self.exe = exe
        self.cmds = []
        self.checks = []

    def add(self, text, check):
        self.cmds.append(text)
        self.checks.append(check)

    def run(self):
        out = subprocess.run([self.exe], input="\n".join(self.cmds) + "\n", capture_output=True,
                             text=True, timeout=600)
        assert out.returncode == 0, out.stdout[-1000:] + out.stderr[-2000:]
        assert "mock contract violated" not in out.stderr, out.stderr[-2000:]
        lines = out.stdout.splitlines()
        pos = 0
        for check in self.checks:
            if check is None:
                continue
            pos = check(lines, pos)
        assert pos == len(lines), lines[pos:pos + 5]


def _expect_values(kind, want):
    def check(lines, pos):
        assert lines[pos] == "%s %d" % (kind, len(want)), lines[pos]
        got = [int(x) for x in lines[pos + 1:pos + 1 + len(want)]]
        assert got == list(want), kind
        return pos + 1 + len(want)
    return check


def _expect_error(code):
    def check(lines, pos):
        assert lines[pos].startswith("error %d" % code), lines[pos]
        return pos + 1
    return check


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    if shutil.which("g++") is None or _cuda_include() is None:
        pytest.skip("no host C++ compiler or CUDA headers")
    path = str(tmp_path_factory.mktemp("api") / "api_mock")
    subprocess.run(["g++", "-std=c++17", "-O1", "-Wall", "-Werror", "-I", CSRC, "-I",
                    _cuda_include(), "-I", HERE, "-x", "c++", os.path.join(CSRC, "api.cu"),
                    "-x", "c++", os.path.join(CSRC, "cluster_merge.cu"), "-x", "c++",
                    os.path.join(HERE, "api_mock.cpp"), "-o", path], check=True)
    return path


def test_score_batch_cells_and_rerun(exe):
    """Pair lists of every shape (shared first sequences, repeats, self pairs, empty and long
    sequences) under several scheduler tunings, with and without forcing the int32 path."""
    rng = np.random.default_rng(11)
    H = Harness(exe)
    for trial in range(12):
        n = int(rng.integers(2, 90))
        L = _lengths(rng, n)
        H.add("seqs %d %s" % (n, " ".join(map(str, L))), None)
        H.add("sym 0", None)
        w, rows = [(16, 8192), (4, 256), (8, 65536), (16, 2048)][trial % 4]
        H.add("tuning %d %d" % (w, rows), None)
        k = int(rng.integers(1, 400))
        firsts = rng.integers(0, n, size=max(1, k // 7))
        p = np.stack([rng.choice(firsts, size=k), rng.integers(0, n, size=k)], axis=1)
        flat = " ".join(map(str, p.reshape(-1)))
        want = [_score(a, b, L, False) for a, b in p]
        H.add("score 0 %d %s" % (k, flat), _expect_values("score", want))
        H.add("score %d %d %s" % (CM_FORCE_INT32, k, flat), _expect_values("score", want))
        extra = [CM_DEVICE_PTRS, CM_ASCII, CM_ASCII | CM_DEVICE_PTRS][trial % 3]
        H.add("score %d %d %s" % (extra, k, flat), _expect_values("score", want))
        wc = [v for a, b in p for v in _cells(a, b, L, False)]
        H.add("cells %d %s" % (k, flat), _expect_values("cells", wc))
    H.add("score 0 1 0 %d" % 10 ** 6, _expect_error(-1))       # pair index out of range
    H.run()


def test_argument_errors(exe):
    """Invalid arguments come back as CM_ERR_ARG (-1) with nothing computed, and the context
    stays usable."""
    H = Harness(exe)
    L = [40, 300, 0, 2500]
    H.add("seqs 4 %s" % " ".join(map(str, L)), None)
    H.add("sym 1", None)
    H.add("allpairs 50 3 3 100", _expect_error(-1))             # part >= n_parts
    H.add("allpairs 50 -1 3 100", _expect_error(-1))
    H.add("cells 1 0 4", _expect_error(-1))                     # pair index out of range
    H.add("score 0 1 -1 0", _expect_error(-1))
    H.add("tuning 12 0", _expect_error(-1))                      # warps must be 4, 8 or 16
    H.add("tuning 0 100", _expect_error(-1))                     # rows below 256
    H.add("limit 1000", _expect_error(-1))                       # below 1,024 slots
    H.add("score 0 2 0 1 3 1", _expect_values("score", [_score(0, 1, L, True),
                                                         _score(3, 1, L, True)]))
    H.run()


def test_allpairs_parts(exe):
    rng = np.random.default_rng(12)
    H = Harness(exe)
    for trial in range(6):
        n = int(rng.integers(2, 120))
        L = _lengths(rng, n)
        T = int(rng.choice([50, 100, 300]))
        truth = sorted((i, j, _score(i, j, L, True)) for i in range(n) for j in range(i + 1, n)
                       if _score(i, j, L, True) > T)
        H.add("seqs %d %s" % (n, " ".join(map(str, L))), None)
        H.add("sym 1", None)
        nparts = int(rng.choice([1, 3, 7]))
        got = []

        def part_check(lines, pos, got=got):
            assert lines[pos].startswith("allpairs "), lines[pos]
            k = int(lines[pos].split()[1])
            got.extend(tuple(map(int, l.split())) for l in lines[pos + 1:pos + 1 + k])
            return pos + 1 + k
        for part in range(nparts):
            H.add("allpairs %d %d %d %d" % (T, part, nparts, 100000), part_check)

        def union_check(lines, pos, got=got, truth=truth):
            assert sorted(got) == truth
            return pos
        H.checks[-1] = (lambda f1, f2: (lambda lines, pos: f2(lines, f1(lines, pos))))(
            H.checks[-1], union_check)
        if truth:
            H.add("allpairs %d 0 1 0" % T, _expect_error(-6))        # capacity too small
    H.run()


def _oracle_cm(L, T, mT, mU, use_ranker, min_pairs, sparse):
    n = len(L)

    def score(x, y):
        return _score(x, y, L, True, sparse)

    def transitive(r1, r2, s):
        if not s > mT:
            return False, False
        c = _cells(r1, r2, L, True, sparse)
        return int(L[r1]) - (c[2] - c[1] + 1) < mU, int(L[r2]) - (c[4] - c[3] + 1) < mU

    final, stats = ocm.bottom_up_merge(n, score, transitive, T,
                                       keep=_keep if use_ranker else None, min_pairs=min_pairs)
    pairs = ocm.intra_cluster_pairs(final, score, T, stats)
    return ([(c.rep, list(c.objs)) for c in final], [tuple(map(int, p)) for p in pairs.tolist()],
            [stats["rep"], stats["exchange"], stats["intra"], stats["full_merges"],
             stats["exchanges"], stats["merges"]])


def _expect_cm(want, batches=None):
    def check(lines, pos):
        assert lines[pos].startswith("clusters "), lines[pos]
        nc = int(lines[pos].split()[1])
        clusters = []
        for l in lines[pos + 1:pos + 1 + nc]:
            v = list(map(int, l.split()))
            clusters.append((v[0], v[2:]))
        pos += 1 + nc
        npairs = int(lines[pos].split()[1])
        pairs = [tuple(map(int, l.split())) for l in lines[pos + 1:pos + 1 + npairs]]
        pos += 1 + npairs
        stats = list(map(int, lines[pos].split()[1:]))
        assert clusters == want[0]
        assert pairs == want[1]
        assert stats[:6] == want[2], (stats, want[2])
        if batches is not None:
            batches.append(stats[6])
        return pos + 1
    return check


def test_cluster_merge_plain_ranked_and_batched(exe):
    """ClusterMerge through the whole host runtime, with the default device batch and with
    rep waves cut into batches of 1,024 and 3,000 slots; results must not change and the
    small limits must add device batches."""
    rng = np.random.default_rng(13)
    H = Harness(exe)
    counts = []
    for trial in range(10):
        big = trial >= 6                      # large, sparser sets: rounds above the limits
        n = int(rng.integers(250, 330)) if big else int(rng.integers(3, 110))
        L = _lengths(rng, n)
        T = int(rng.choice([100, 300]))
        mT, mU = T + 38, 15
        use_ranker = trial % 2
        min_pairs = int(rng.choice([0, 16]))
        want = _oracle_cm(L, T, mT, mU, use_ranker, min_pairs, big)
        H.add("seqs %d %s" % (n, " ".join(map(str, L))), None)
        H.add("sym 1", None)
        H.add("sparse %d" % big, None)
        nb = []
        for limit in (0, 1024, 3000):
            H.add("limit %d" % limit, None)
            H.add("cm %d %d %d %d %d" % (T, mT, mU, use_ranker, min_pairs), _expect_cm(want, nb))

        def more_batches(lines, pos, nb=nb):
            assert nb[1] >= nb[0] and nb[2] >= nb[0]
            counts.append(nb)
            return pos
        H.add("limit 0", more_batches)
    H.run()
    assert sum(nb[1] > nb[0] for nb in counts) >= 2, counts     # the small limits split rounds
