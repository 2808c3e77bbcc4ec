"""Seeded synthetic protein inputs shared by the CUDA path, the oracle and the tests.

This module holds inputs only: the 20-letter alphabet, the BLOSUM62 substitution matrix
(Henikoff & Henikoff 1992, as the paper's related-work section names it) and a background
residue distribution, plus generators for proteome-shaped sequence sets.  It performs none of
the method's arithmetic (no alignment, no clustering), so both the CUDA path and the CPU oracle
may import it without sharing any computation.

Workload recipes (the paper's OMA / QfO datasets are not available; these stand in for them):

* families: a random root is drawn from the background distribution; each member is derived
  from the root independently with a per-residue 30 % substitution (to a different residue,
  drawn from the background) and a per-position 5 % single-residue indel (insertion or
  deletion, 50/50).  This mimics homologous proteins (Sec. 4 of the paper).
* lengths: uniform 50-300 for the small case; lognormal (median 350, sigma 0.6, clipped to
  30-5000) for the proteome-shaped cases.
"""
from __future__ import annotations

import numpy as np

#: residue letters in the order used for residue codes 0..19 (NCBI matrix order)
ALPHABET = "ARNDCQEGHILKMFPSTWYV"

#: BLOSUM62, rows/columns in ALPHABET order (published NCBI table, integer half-bit units)
BLOSUM62 = np.array([
    # A   R   N   D   C   Q   E   G   H   I   L   K   M   F   P   S   T   W   Y   V
    [ 4, -1, -2, -2,  0, -1, -1,  0, -2, -1, -1, -1, -1, -2, -1,  1,  0, -3, -2,  0],  # A
    [-1,  5,  0, -2, -3,  1,  0, -2,  0, -3, -2,  2, -1, -3, -2, -1, -1, -3, -2, -3],  # R
    [-2,  0,  6,  1, -3,  0,  0,  0,  1, -3, -3,  0, -2, -3, -2,  1,  0, -4, -2, -3],  # N
    [-2, -2,  1,  6, -3,  0,  2, -1, -1, -3, -4, -1, -3, -3, -1,  0, -1, -4, -3, -3],  # D
    [ 0, -3, -3, -3,  9, -3, -4, -3, -3, -1, -1, -3, -1, -2, -3, -1, -1, -2, -2, -1],  # C
    [-1,  1,  0,  0, -3,  5,  2, -2,  0, -3, -2,  1,  0, -3, -1,  0, -1, -2, -1, -2],  # Q
    [-1,  0,  0,  2, -4,  2,  5, -2,  0, -3, -3,  1, -2, -3, -1,  0, -1, -3, -2, -2],  # E
    [ 0, -2,  0, -1, -3, -2, -2,  6, -2, -4, -4, -2, -3, -3, -2,  0, -2, -2, -3, -3],  # G
    [-2,  0,  1, -1, -3,  0,  0, -2,  8, -3, -3, -1, -2, -1, -2, -1, -2, -2,  2, -3],  # H
    [-1, -3, -3, -3, -1, -3, -3, -4, -3,  4,  2, -3,  1,  0, -3, -2, -1, -3, -1,  3],  # I
    [-1, -2, -3, -4, -1, -2, -3, -4, -3,  2,  4, -2,  2,  0, -3, -2, -1, -2, -1,  1],  # L
    [-1,  2,  0, -1, -3,  1,  1, -2, -1, -3, -2,  5, -1, -3, -1,  0, -1, -3, -2, -2],  # K
    [-1, -1, -2, -3, -1,  0, -2, -3, -2,  1,  2, -1,  5,  0, -2, -1, -1, -1, -1,  1],  # M
    [-2, -3, -3, -3, -2, -3, -3, -3, -1,  0,  0, -3,  0,  6, -4, -2, -2,  1,  3, -1],  # F
    [-1, -2, -2, -1, -3, -1, -1, -2, -2, -3, -3, -1, -2, -4,  7, -1, -1, -4, -3, -2],  # P
    [ 1, -1,  1,  0, -1,  0,  0,  0, -1, -2, -2,  0, -1, -2, -1,  4,  1, -3, -2, -2],  # S
    [ 0, -1,  0, -1, -1, -1, -1, -2, -2, -1, -1, -1, -1, -2, -1,  1,  5, -2, -2,  0],  # T
    [-3, -3, -4, -4, -2, -2, -3, -2, -2, -3, -2, -3, -1,  1, -4, -3, -2, 11,  2, -3],  # W
    [-2, -2, -2, -3, -2, -1, -2, -3,  2, -1, -1, -2, -1,  3, -3, -2, -2,  2,  7, -1],  # Y
    [ 0, -3, -3, -3, -1, -2, -2, -3, -3,  3,  1, -2,  1, -1, -2, -2,  0, -3, -1,  4],  # V
], dtype=np.int8)

#: the 24-letter alphabet of the published 24 x 24 tables: B = D or N, Z = E or Q, X = any,
#: * = stop (residue codes 20..23)
ALPHABET24 = ALPHABET + "BZX*"

#: BLOSUM62 over ALPHABET24 (published NCBI table: the 20 x 20 block above plus B, Z, X, *)
BLOSUM62_24 = np.zeros((24, 24), dtype=np.int8)
BLOSUM62_24[:20, :20] = BLOSUM62
_B62_EXTRA = {
    "B": [-2, -1, 3, 4, -3, 0, 1, -1, 0, -3, -4, 0, -3, -3, -2, 0, -1, -4, -3, -3, 4, 1, -1, -4],
    "Z": [-1, 0, 0, 1, -3, 3, 4, -2, 0, -3, -3, 1, -1, -3, -1, 0, -1, -3, -2, -2, 1, 4, -1, -4],
    "X": [0, -1, -1, -1, -2, -1, -1, -1, -1, -1, -1, -1, -1, -1, -2, 0, 0, -2, -1, -1, -1, -1, -1, -4],
    "*": [-4] * 23 + [1],
}
for _k, _row in enumerate("BZX*"):
    BLOSUM62_24[20 + _k, :] = _B62_EXTRA[_row]
    BLOSUM62_24[:, 20 + _k] = _B62_EXTRA[_row]

#: PAM250 (Dayhoff et al. 1978, the matrix the paper clusters with, Sec. 4) over ALPHABET24,
#: rows/columns in the layout of the published NCBI table
PAM250_24 = np.array([
    # A   R   N   D   C   Q   E   G   H   I   L   K   M   F   P   S   T   W   Y   V   B   Z   X   *
    [ 2, -2,  0,  0, -2,  0,  0,  1, -1, -1, -2, -1, -1, -3,  1,  1,  1, -6, -3,  0,  0,  0,  0, -8],  # A
    [-2,  6,  0, -1, -4,  1, -1, -3,  2, -2, -3,  3,  0, -4,  0,  0, -1,  2, -4, -2, -1,  0, -1, -8],  # R
    [ 0,  0,  2,  2, -4,  1,  1,  0,  2, -2, -3,  1, -2, -3,  0,  1,  0, -4, -2, -2,  2,  1,  0, -8],  # N
    [ 0, -1,  2,  4, -5,  2,  3,  1,  1, -2, -4,  0, -3, -6, -1,  0,  0, -7, -4, -2,  3,  3, -1, -8],  # D
    [-2, -4, -4, -5, 12, -5, -5, -3, -3, -2, -6, -5, -5, -4, -3,  0, -2, -8,  0, -2, -4, -5, -3, -8],  # C
    [ 0,  1,  1,  2, -5,  4,  2, -1,  3, -2, -2,  1, -1, -5,  0, -1, -1, -5, -4, -2,  1,  3, -1, -8],  # Q
    [ 0, -1,  1,  3, -5,  2,  4,  0,  1, -2, -3,  0, -2, -5, -1,  0,  0, -7, -4, -2,  3,  3, -1, -8],  # E
    [ 1, -3,  0,  1, -3, -1,  0,  5, -2, -3, -4, -2, -3, -5,  0,  1,  0, -7, -5, -1,  0,  0, -1, -8],  # G
    [-1,  2,  2,  1, -3,  3,  1, -2,  6, -2, -2,  0, -2, -2,  0, -1, -1, -3,  0, -2,  1,  2, -1, -8],  # H
    [-1, -2, -2, -2, -2, -2, -2, -3, -2,  5,  2, -2,  2,  1, -2, -1,  0, -5, -1,  4, -2, -2, -1, -8],  # I
    [-2, -3, -3, -4, -6, -2, -3, -4, -2,  2,  6, -3,  4,  2, -3, -3, -2, -2, -1,  2, -3, -3, -1, -8],  # L
    [-1,  3,  1,  0, -5,  1,  0, -2,  0, -2, -3,  5,  0, -5, -1,  0,  0, -3, -4, -2,  1,  0, -1, -8],  # K
    [-1,  0, -2, -3, -5, -1, -2, -3, -2,  2,  4,  0,  6,  0, -2, -2, -1, -4, -2,  2, -2, -2, -1, -8],  # M
    [-3, -4, -3, -6, -4, -5, -5, -5, -2,  1,  2, -5,  0,  9, -5, -3, -3,  0,  7, -1, -4, -5, -2, -8],  # F
    [ 1,  0,  0, -1, -3,  0, -1,  0,  0, -2, -3, -1, -2, -5,  6,  1,  0, -6, -5, -1, -1,  0, -1, -8],  # P
    [ 1,  0,  1,  0,  0, -1,  0,  1, -1, -1, -3,  0, -2, -3,  1,  2,  1, -2, -3, -1,  0,  0,  0, -8],  # S
    [ 1, -1,  0,  0, -2, -1,  0,  0, -1,  0, -2,  0, -1, -3,  0,  1,  3, -5, -3,  0,  0, -1,  0, -8],  # T
    [-6,  2, -4, -7, -8, -5, -7, -7, -3, -5, -2, -3, -4,  0, -6, -2, -5, 17,  0, -6, -5, -6, -4, -8],  # W
    [-3, -4, -2, -4,  0, -4, -4, -5,  0, -1, -1, -4, -2,  7, -5, -3, -3,  0, 10, -2, -3, -4, -2, -8],  # Y
    [ 0, -2, -2, -2, -2, -2, -2, -1, -2,  4,  2, -2,  2, -1, -1, -1,  0, -6, -2,  4, -2, -2, -1, -8],  # V
    [ 0, -1,  2,  3, -4,  1,  3,  0,  1, -2, -3,  1, -2, -4, -1,  0,  0, -5, -3, -2,  3,  2, -1, -8],  # B
    [ 0,  0,  1,  3, -5,  3,  3,  0,  2, -2, -3,  0, -2, -5,  0,  0, -1, -6, -4, -2,  2,  3, -1, -8],  # Z
    [ 0, -1,  0, -1, -3, -1, -1, -1, -1, -1, -1, -1, -1, -2, -1,  0,  0, -4, -2, -1, -1, -1, -1, -8],  # X
    [-8, -8, -8, -8, -8, -8, -8, -8, -8, -8, -8, -8, -8, -8, -8, -8, -8, -8, -8, -8, -8, -8, -8,  1],  # *
], dtype=np.int8)

#: PAM250 restricted to the 20 amino acids (ALPHABET order)
PAM250 = np.ascontiguousarray(PAM250_24[:20, :20])

#: Background amino-acid frequencies (Robinson & Robinson 1991), ALPHABET order, normalised.
_BG_RAW = np.array([0.07805, 0.05129, 0.04487, 0.05364, 0.01925, 0.04264, 0.06295, 0.07377,
                    0.02199, 0.05142, 0.09019, 0.05744, 0.02243, 0.03856, 0.05203, 0.07120,
                    0.05841, 0.01330, 0.03216, 0.06441])
BACKGROUND = _BG_RAW / _BG_RAW.sum()

#: default affine gap penalties (gap of k residues costs GAP_OPEN + (k-1)*GAP_EXTEND)
GAP_OPEN = 11
GAP_EXTEND = 1

SEED = 1908

_CODE = np.full(256, 255, dtype=np.uint8)
for _i, _c in enumerate(ALPHABET24):
    _CODE[ord(_c)] = _i
    _CODE[ord(_c.lower())] = _i


def encode(s: str, alphabet24: bool = False) -> np.ndarray:
    """Map an amino-acid string to residue codes 0..19 (0..23 with alphabet24: B, Z, X, *
    too); raises on any other letter."""
    a = _CODE[np.frombuffer(s.encode("ascii"), dtype=np.uint8)]
    if (a == 255).any() or (not alphabet24 and (a >= 20).any()):
        raise ValueError("letter outside the alphabet in %r" % s[:40])
    return a


def decode(codes) -> str:
    return "".join(ALPHABET24[int(c)] for c in codes)


class SeqSet:
    """Sequences as one concatenated uint8 code array plus int64 offsets (n+1)."""

    def __init__(self, seqs, offsets, family=None):
        self.seqs = np.ascontiguousarray(seqs, dtype=np.uint8)
        self.offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        self.family = None if family is None else np.asarray(family, dtype=np.int32)

    @classmethod
    def from_list(cls, arrays, family=None):
        lens = np.array([len(a) for a in arrays], dtype=np.int64)
        off = np.zeros(len(arrays) + 1, dtype=np.int64)
        np.cumsum(lens, out=off[1:])
        cat = np.concatenate([np.asarray(a, dtype=np.uint8) for a in arrays]) if arrays else \
            np.zeros(0, dtype=np.uint8)
        return cls(cat, off, family)

    def __len__(self):
        return len(self.offsets) - 1

    @property
    def lengths(self):
        return np.diff(self.offsets)

    def __getitem__(self, i):
        return self.seqs[self.offsets[i]:self.offsets[i + 1]]

    def subset(self, ids):
        ids = np.asarray(ids)
        return SeqSet.from_list([self[int(i)] for i in ids],
                                None if self.family is None else self.family[ids])


def _rng(stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([SEED, stream])))


def random_seq(rng, n):
    return rng.choice(20, size=n, p=BACKGROUND).astype(np.uint8)


def mutate(rng, root, sub_rate=0.30, indel_rate=0.05):
    """Member derived from root: per-residue substitution to a different residue, then
    per-position single-residue indels (insertion or deletion with equal probability)."""
    out = []
    for r in root:
        if rng.random() < indel_rate:
            if rng.random() < 0.5:          # deletion of this position
                continue
            out.append(int(random_seq(rng, 1)[0]))   # insertion before this position
        if rng.random() < sub_rate:
            p = BACKGROUND.copy()
            p[r] = 0.0
            p /= p.sum()
            out.append(int(rng.choice(20, p=p)))
        else:
            out.append(int(r))
    if not out:
        out.append(int(root[0]))
    return np.array(out, dtype=np.uint8)


def _mutate_fast(rng, root, sub_rate=0.30, indel_rate=0.05):
    """Vectorised form of `mutate` with the same model (used for the large sets)."""
    n = len(root)
    ev = rng.random(n) < indel_rate
    ins = rng.random(n) < 0.5
    sub = rng.random(n) < sub_rate
    base = root.copy()
    idx = np.nonzero(sub)[0]
    if len(idx):
        # substitute to a different residue drawn from the background
        cand = random_seq(rng, len(idx))
        same = cand == base[idx]
        while same.any():
            cand[same] = random_seq(rng, int(same.sum()))
            same = cand == base[idx]
        base[idx] = cand
    keep = ~(ev & ~ins)            # deletion events drop the residue
    insert_here = ev & ins         # insertion events add a residue before it
    counts = insert_here.astype(np.int64) + keep
    start = np.cumsum(counts) - counts
    out = np.empty(int(counts.sum()), dtype=np.uint8)
    out[start[insert_here]] = random_seq(rng, int(insert_here.sum()))
    out[start[keep] + insert_here[keep]] = base[keep]
    if len(out) == 0:
        out = root[:1].copy()
    return out


def lognormal_lengths(rng, n, median=350.0, sigma=0.6, lo=30, hi=5000):
    return np.clip(np.round(rng.lognormal(np.log(median), sigma, size=n)), lo, hi).astype(np.int64)


def families(n_families, members, root_lengths, stream, singletons=0, singleton_lengths=None,
             fast=True):
    """Planted families plus optional unrelated singletons, shuffled with a seeded permutation."""
    rng = _rng(stream)
    seqs, fam = [], []
    mut = _mutate_fast if fast else mutate
    for f in range(n_families):
        root = random_seq(rng, int(root_lengths[f]))
        for _ in range(members):
            seqs.append(mut(rng, root))
            fam.append(f)
    for s in range(singletons):
        seqs.append(random_seq(rng, int(singleton_lengths[s])))
        fam.append(n_families + s)
    perm = rng.permutation(len(seqs))
    return SeqSet.from_list([seqs[i] for i in perm], np.array(fam, dtype=np.int32)[perm])


def small_families(stream=1):
    """200 proteins: 20 families of 10, root length uniform 50-300 (the small all-pairs case)."""
    rng = _rng(100 + stream)
    return families(20, 10, rng.integers(50, 301, size=20), stream)


def proteome(n_seqs=20000, family_size=10, singleton_frac=0.0, stream=2):
    """Proteome-shaped set: lognormal lengths (median 350, sigma 0.6, clip 30-5000),
    planted families of `family_size`, plus a fraction of unrelated singletons."""
    rng = _rng(200 + stream)
    n_single = int(round(n_seqs * singleton_frac))
    n_fam = (n_seqs - n_single) // family_size
    return families(n_fam, family_size, lognormal_lengths(rng, n_fam), stream,
                    singletons=n_single, singleton_lengths=lognormal_lengths(rng, n_single))


def tandem_repeat(rng, length, motif_len=40, sub_rate=0.05, motif=None):
    """Long self-similar sequence: copies of one motif (random unless given), each copy with
    5 % substitutions."""
    if motif is None:
        motif = random_seq(rng, motif_len)
    motif_len = len(motif)
    reps = []
    while sum(len(r) for r in reps) < length:
        c = motif.copy()
        m = rng.random(motif_len) < sub_rate
        c[m] = random_seq(rng, int(m.sum()))
        reps.append(c)
    return np.concatenate(reps)[:length]


def long_tail(base, n_long, n_motifs, stream=5, lo=10000, hi=35000, motif_len=40):
    """`base` plus `n_long` long tandem repeats of lengths uniform [lo, hi], in `n_motifs`
    families that share a 40-residue motif (members of one family align over their whole
    length with scores far above the int16 range).  The long sequences are appended after
    base's; family labels continue base's."""
    rng = _rng(500 + stream)
    motifs = [random_seq(rng, motif_len) for _ in range(n_motifs)]
    longs = [tandem_repeat(rng, int(rng.integers(lo, hi + 1)), motif=motifs[i % n_motifs])
             for i in range(n_long)]
    fam0 = int(base.family.max()) + 1 if base.family is not None and len(base) else 0
    fam = None if base.family is None else np.concatenate(
        [base.family, fam0 + np.arange(n_long, dtype=np.int32) % n_motifs])
    return SeqSet.from_list([base[i] for i in range(len(base))] + longs, fam)


def random_pairs(n_seqs, n_pairs, stream=3):
    rng = _rng(300 + stream)
    a = rng.integers(0, n_seqs, size=n_pairs)
    b = rng.integers(0, n_seqs, size=n_pairs)
    return np.stack([a, b], axis=1).astype(np.int32)


def random_codes(n, stream=4, alphabet=20):
    rng = _rng(400 + stream)
    return rng.integers(0, alphabet, size=n).astype(np.uint8)
