"""Pins for the float64 ranker oracle: central finite differences of the numpy forward
against the autograd gradient, closed forms for degenerate weights, symmetry, and the
independence of a sequence's vector from the rest of the batch."""
import numpy as np

from oracle import ranker as R
from paper_1908_10574_gb300 import synth


def _toy():
    rng = np.random.default_rng(0)
    seqs = [synth.random_seq(rng, L) for L in (5, 1, 12, 9)]
    ss = synth.SeqSet.from_list(seqs)
    pairs = np.array([[0, 2], [1, 3], [2, 3], [0, 0]], np.int32)
    labels = np.array([1, 0, 1, 0], np.float64)
    return ss, pairs, labels


def test_gradient_matches_central_differences():
    ss, pairs, labels = _toy()
    p = R.init_params(1)
    lo, g = R.loss_grad(ss.seqs, ss.offsets, p, pairs, labels)
    assert abs(lo - R.loss(ss.seqs, ss.offsets, p, pairs, labels)) < 1e-12
    rng = np.random.default_rng(2)
    offs = [0, 640, 640 + 9 * 32 * 128, 640 + 9 * 32 * 128 + 128]
    idx = np.concatenate([rng.integers(0, R.num_params(), 40),
                          [R.num_params() - 1, R.num_params() - 2]] + [[o + 3] for o in offs])
    h = 1e-6
    for i in idx:
        d = np.zeros_like(p)
        d[i] = h
        fd = (R.loss(ss.seqs, ss.offsets, p + d, pairs, labels) -
              R.loss(ss.seqs, ss.offsets, p - d, pairs, labels)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_zero_weights_closed_form():
    ss, pairs, labels = _toy()
    p = R.init_params(3)
    P = R.unpack(p)
    for k in ("W1", "W2", "W3"):
        P[k][...] = 0.0
    # every row of Z3 equals b3 (Z2 = relu(b2) does not reach it through zero weights)
    V = R.embed(ss.seqs, ss.offsets, p)
    for i in range(len(ss)):
        assert np.allclose(V[i], P["b3"])
    z = R.logits(ss.seqs, ss.offsets, p, pairs)
    b = P["b3"]
    assert np.allclose(z, float(P["alpha"]) * (b @ b) / (b @ b + R.COS_EPS) + float(P["beta"]))


def test_single_tap_identity_network():
    """Only the centre tap of every layer is the identity (W1 maps 32 channels into the first
    32 of 128): the network reduces to relu(relu(E[code])) per residue, averaged."""
    ss, _, _ = _toy()
    p = R.init_params(4)
    P = R.unpack(p)
    for k in ("W1", "W2", "W3"):
        P[k][...] = 0.0
    P["W1"][4][:, :32] = np.eye(32)
    P["W2"][4] = np.eye(128)
    P["W3"][4] = np.eye(128)
    for k in ("b1", "b2", "b3"):
        P[k][...] = 0.0
    V = R.embed(ss.seqs, ss.offsets, p)
    for i in range(len(ss)):
        codes = ss[i]
        want = np.zeros(128)
        want[:32] = np.maximum(P["E"][codes], 0).mean(axis=0)
        assert np.allclose(V[i], want)


def test_symmetry_and_batch_isolation():
    ss, pairs, _ = _toy()
    p = R.init_params(5)
    z1 = R.logits(ss.seqs, ss.offsets, p, pairs)
    z2 = R.logits(ss.seqs, ss.offsets, p, pairs[:, ::-1])
    assert np.allclose(z1, z2)
    V = R.embed(ss.seqs, ss.offsets, p)
    alone = R.embed(ss.subset([2]).seqs, ss.subset([2]).offsets, p)
    assert np.allclose(V[2], alone[0])
