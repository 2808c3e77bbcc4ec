"""GPU test of sw_cells_batch_noalloc, the allocation-free alignment-cells entry point.

It serves callers that cannot allocate device memory when they call (memory reserved up front
by another framework's allocator, or loops that must avoid cudaMalloc's synchronisation).  The
test calls it through the C ABI (ctypes) twice in a row on the same inputs and requires both
results to equal those of the ordinary entry point sw_cells_batch exactly (the tolerance of all
integer tests here), and, since its one-thread-per-pair kernel shares no code with
sw_cells_batch's, also the oracle's cells pair by pair.  It also checks the size limit and the
binding's argument checks are rejected cleanly.  This file is named so
pytest collects it last; it builds all of its own inputs, so it also passes alone in a fresh
process.
"""
import ctypes

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def _inputs():
    from paper_1908_10574_gb300 import synth
    rng = np.random.default_rng(2024)
    roots = [synth.random_seq(rng, int(L)) for L in (60, 250, 900, 4000)]
    seqs = []
    for r in roots:
        seqs += [r, synth.mutate(rng, r), synth.mutate(rng, r)]
    seqs.append(np.zeros(0, np.uint8))
    ss = synth.SeqSet.from_list(seqs)
    n = len(ss)
    pairs = np.array([(i, j) for i in range(n) for j in range(n) if (i + 2 * j) % 3 != 1],
                     dtype=np.int32)
    return ss, pairs, synth.BLOSUM62


def test_noalloc_cells_match_sw_cells_batch_twice():
    import torch
    import paper_1908_10574_gb300 as cm
    from paper_1908_10574_gb300 import _lib

    ss, pairs, S = _inputs()
    ctx = cm.Context(0)
    want = ctx.sw_cells_batch(ss.seqs, ss.offsets, pairs, S, 11, 1)
    ref = np.array([oracle.sw_cells(ss[x], ss[y], S, 11, 1) for x, y in pairs], dtype=np.int64)

    torch.cuda.set_device(0)
    dseqs = torch.from_numpy(ss.seqs).cuda()
    doff = torch.from_numpy(ss.offsets).cuda()
    dpairs = torch.from_numpy(pairs).cuda()
    m = np.ascontiguousarray(S.reshape(-1).astype(np.int8))
    err = ctypes.create_string_buffer(256)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    L = _lib.lib()
    for call in range(2):
        out = torch.full((len(pairs), 5), -7, dtype=torch.int32, device="cuda")
        code = L.sw_cells_batch_noalloc(
            ctypes.c_void_p(dseqs.data_ptr()), ctypes.c_void_p(doff.data_ptr()), len(ss),
            ctypes.c_void_p(dpairs.data_ptr()), len(pairs), ctypes.c_void_p(m.ctypes.data),
            11, 1, ctypes.c_void_p(out.data_ptr()), stream, 0, err, 256)
        assert code == 0, err.value
        assert np.array_equal(out.cpu().numpy(), want), "call %d differs" % call
        assert np.array_equal(out.cpu().numpy(), ref), "call %d differs from the oracle" % call

    # the binding wrapper gives the same result
    out = torch.empty((len(pairs), 5), dtype=torch.int32, device="cuda")
    cm.sw_cells_batch_noalloc(dseqs, doff, dpairs, S, 11, 1, out)
    assert np.array_equal(out.cpu().numpy(), want)


def test_noalloc_rejects_sequences_beyond_the_limit():
    import torch
    import paper_1908_10574_gb300 as cm
    from paper_1908_10574_gb300 import synth

    rng = np.random.default_rng(5)
    ss = synth.SeqSet.from_list([synth.random_seq(rng, 100), synth.random_seq(rng, 4096)])
    dseqs = torch.from_numpy(ss.seqs).cuda()
    doff = torch.from_numpy(ss.offsets).cuda()
    dpairs = torch.tensor([[0, 1]], dtype=torch.int32, device="cuda")
    out = torch.full((1, 5), -7, dtype=torch.int32, device="cuda")
    with pytest.raises(cm.CMError) as ei:
        cm.sw_cells_batch_noalloc(dseqs, doff, dpairs, synth.BLOSUM62, 11, 1, out)
    assert ei.value.code == -1 and "4095" in str(ei.value)
    assert out.cpu().numpy().tolist() == [[-7] * 5]
    # the reverse orientation (long sequence first) is within the limit
    dpairs = torch.tensor([[1, 0]], dtype=torch.int32, device="cuda")
    cm.sw_cells_batch_noalloc(dseqs, doff, dpairs, synth.BLOSUM62, 11, 1, out)
    want = cm.Context(0).sw_cells_batch(ss.seqs, ss.offsets, np.array([[1, 0]], np.int32),
                                        synth.BLOSUM62, 11, 1)
    assert np.array_equal(out.cpu().numpy(), want)


def test_noalloc_binding_rejects_bad_arguments():
    import torch
    import paper_1908_10574_gb300 as cm
    from paper_1908_10574_gb300 import synth

    ss, pairs, S = _inputs()
    dseqs = torch.from_numpy(ss.seqs).cuda()
    doff = torch.from_numpy(ss.offsets).cuda()
    dpairs = torch.from_numpy(pairs).cuda()
    out = torch.full((len(pairs), 5), -7, dtype=torch.int32, device="cuda")
    bad = [
        dict(pairs=dpairs.long()),                                   # int64 pairs
        dict(offsets=doff.int()),                                    # int32 offsets
        dict(cells_out=out[:-1]),                                    # too few rows
        dict(cells_out=torch.zeros((len(pairs), 10), dtype=torch.int32,
                                   device="cuda")[:, ::2]),          # non-contiguous
        dict(seqs=torch.from_numpy(ss.seqs)),                        # host tensor
    ]
    for kw in bad:
        args = dict(seqs=dseqs, offsets=doff, pairs=dpairs, cells_out=out)
        args.update(kw)
        with pytest.raises((TypeError, ValueError)):
            cm.sw_cells_batch_noalloc(args["seqs"], args["offsets"], args["pairs"], S, 11, 1,
                                      args["cells_out"])
    big = S.astype(np.int64).copy()
    big[0, 0] = 300                                                  # does not fit int8
    with pytest.raises(ValueError):
        cm.sw_cells_batch_noalloc(dseqs, doff, dpairs, big, 11, 1, out)
    assert (out == -7).all()
