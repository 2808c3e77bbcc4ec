#!/usr/bin/env python
"""Benchmark: Smith-Waterman GCUPS (bit-exact) on the all-against-all of 20,000 synthetic
proteins (lognormal lengths, median 350, sigma 0.6, clipped 30-5000; 2,000 planted families of
10; BLOSUM62, gap open 11 / extend 1; significant pairs f > T = 100).

A step is one part (1/16 of the cells) of the all-against-all triangle through sw_allpairs:
packing, the int16x2 DPX kernel, the int32 rerun of saturated pairs and threshold compaction.
`value` times steps on device-resident inputs (CUDA events on the library's stream, L2 flushed
between steps); `e2e` times the same steps through the C ABI with pinned host buffers (the
sequences go host->device and the significant pairs device->host inside every step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank scores its own parts (weak scaling, no collective on the
data path); rank 0 prints one JSON line.  `--impl reference` times the CPU oracle (scalar int64
Gotoh on the host cores) on a bounded sample of the same workload.  The roofline object reports
the SW kernel against the DPX-pipe peak at the sampled SM clock (the DPX issue rate is measured
in the same run by cm_dpx_rate), and its DRAM traffic per launch from an ncu capture scaled by
cells.

At N = 1 the line also carries `cluster_merge` (skip with --no-cm), the metric's second half:
ClusterMerge of 100,000 proteome-shaped proteins, the plain merge against the learned path
timed end to end (labelling 1M training pairs with the GPU SW path, training the ranker on the
set, calibrating its pruning threshold on held-out pairs, the ranked merge), both recalls
against the GPU all-against-all of the set, with its own SM-clock record.  It adds about four
minutes.

ClusterMerge experiments (`--workload cm`): plain merge of a proteome-shaped set
(`--cm-seqs`, default 100,000; `--family-size`, `--singleton-frac`; `--long-tail K` adds K long
tandem repeats); `--ranker [--transductive]` trains the learned ranker and runs the ranked merge
too; `--recall` scores the GPU all-against-all for recall (`--recall-sample F`: of a random
fraction F of the proteins only); `--recall-families` adds recall over every within-family pair
with s > T; `--batch-slots` bounds one device batch of the rep wave; `--ranker-untrained Q` runs
the ranked path with untrained weights (profiling).  The 1M-protein long-tail configuration:

  python bench.py --workload cm --cm-seqs 1000000 --family-size 10 --singleton-frac 0 \
      --long-tail 1000 --recall --recall-sample 0.01 --recall-families [--ranker --transductive]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1908_10574_gb300 import synth  # noqa: E402

METRIC = "SW GCUPS (bit-exact)"
N_SEQS = 20000
FAMILY = 10
T_SIG = 100
M_T, M_U = 138, 15
GAP_OPEN, GAP_EXT = 11, 1
PARTS_PER_GPU = 16
OPS_PER_PACKED_CELL = 4.5    # DPX/ALU-pipe operations of the kernel's cell update, 2 cells each
OPS_PER_PACKED_CELL_PLAIN = 7.0   # the plain per-cell count (E 2, F 2, H 2, running max 1)


def workload_desc(n_parts):
    return ("all-against-all Smith-Waterman of %d synthetic proteins (lognormal lengths median "
            "350 sigma 0.6 clipped 30-5000, %d planted families of %d, 30%% substitution + 5%% "
            "indel members), BLOSUM62 gap 11/1, significant pairs f > %d; one step = 1/%d of "
            "the triangle's cells" % (N_SEQS, N_SEQS // FAMILY, FAMILY, T_SIG, n_parts))


def make_set():
    return synth.proteome(N_SEQS, FAMILY)


def total_cells(ss):
    L = ss.lengths.astype(np.float64)
    return int((L.sum() ** 2 - (L ** 2).sum()) / 2)


# DRAM bytes per cell of the int16 kernel, from one ncu capture of the small case
# (`--steps 1 --warmup 0 --parts-per-gpu 512 --part-offset 50 --no-e2e --no-cpu-baseline --no-cm
# --warps 16 --rows 8192`, `-k regex:sw16_kernel -c 1`): 6,448,640 bytes read and 0 written for
# 64,034,019,251 cells in 11.71 ms; sequence rows are re-read from L2, not HBM.
DRAM_BYTES_PER_CELL = 6448640 / 64034019251


def part_sequence(n_parts, count, offset=0):
    return [((3 + 5 * (i + offset)) % n_parts) for i in range(count)]


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index, directory):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join(directory, "clocks_rank%d.csv" % device_index)

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "samples": len(sm), "reasons": sorted(reasons)}


def cpu_baseline(ss, target_s=10.0):
    """The oracle as it stands (scalar Gotoh in C, all host cores) on a bounded random sample
    of the same workload's pairs."""
    import oracle
    rng = np.random.default_rng(77)
    n = len(ss)
    cores = os.cpu_count() or 1
    L = ss.lengths.astype(np.int64)

    def sample(k):
        i = rng.integers(0, n, size=k)
        j = rng.integers(0, n - 1, size=k)
        j = np.where(j >= i, j + 1, j)
        return np.stack([np.minimum(i, j), np.maximum(i, j)], 1).astype(np.int32)

    p = sample(2000)
    t0 = time.perf_counter()
    oracle.sw_batch(ss.seqs, ss.offsets, p, synth.BLOSUM62, GAP_OPEN, GAP_EXT, threads=cores)
    dt = time.perf_counter() - t0
    rate = (L[p[:, 0]] * L[p[:, 1]]).sum() / max(dt, 1e-6)
    k = int(min(max(2000, target_s * rate / (L.mean() ** 2)), 2_000_000))
    p = sample(k)
    cells = int((L[p[:, 0]] * L[p[:, 1]]).sum())
    t0 = time.perf_counter()
    oracle.sw_batch(ss.seqs, ss.offsets, p, synth.BLOSUM62, GAP_OPEN, GAP_EXT, threads=cores)
    dt = time.perf_counter() - t0
    return {"value": cells / dt / 1e9, "unit": "GCUPS", "cores": cores, "kind": "oracle",
            "sample": "%d uniformly random pairs of the all-against-all (%.3g cells), scalar "
                      "int64 Gotoh on %d POSIX threads, %.1f s" % (k, cells, cores, dt)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl"
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(world, x, device):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def run_reference(args, world, rank):
    if rank != 0:
        return
    ss = make_set()
    import oracle
    cores = os.cpu_count() or 1
    L = ss.lengths.astype(np.int64)
    rng = np.random.default_rng(5)
    n = len(ss)
    per_step = 4000     # pairs per step: a bounded sample of the workload (~seconds of CPU)
    cells_t, time_t = 0, 0.0
    for step in range(args.warmup + args.steps):
        i = rng.integers(0, n, size=per_step)
        j = rng.integers(0, n - 1, size=per_step)
        j = np.where(j >= i, j + 1, j)
        p = np.stack([np.minimum(i, j), np.maximum(i, j)], 1).astype(np.int32)
        t0 = time.perf_counter()
        oracle.sw_batch(ss.seqs, ss.offsets, p, synth.BLOSUM62, GAP_OPEN, GAP_EXT, threads=cores)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            cells_t += int((L[p[:, 0]] * L[p[:, 1]]).sum())
            time_t += dt
    v = cells_t / time_t / 1e9
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "GCUPS",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": time_t * 1e3 / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
           "config": {"workload": workload_desc(PARTS_PER_GPU), "n_seqs": N_SEQS},
           "cpu_baseline": {"value": v, "unit": "GCUPS", "cores": cores, "kind": "oracle",
                            "sample": "%d uniformly random pairs per step of the same "
                                      "all-against-all, scalar int64 Gotoh on %d threads"
                                      % (per_step, cores)},
           "e2e": {"value": v, "unit": "GCUPS", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def subset_recall(found, subset, truth_sub):
    """Recall of similar pairs restricted to a sequence subset: `found` holds the (i, j) global
    ids of the pairs a merge reported, `subset` the sorted global ids of the sample and
    `truth_sub` the all-against-all similar pairs of the sample in sample numbering.  Returns
    (recall, truth pairs, found pairs inside the sample)."""
    subset = np.asarray(subset, dtype=np.int64)
    found = np.asarray(found, dtype=np.int64).reshape(-1, 2)
    a = np.searchsorted(subset, found[:, 0])
    b = np.searchsorted(subset, found[:, 1])
    a_in = (a < len(subset)) & (subset[np.minimum(a, len(subset) - 1)] == found[:, 0])
    b_in = (b < len(subset)) & (subset[np.minimum(b, len(subset) - 1)] == found[:, 1])
    keep = a_in & b_in
    fs = set(zip(np.minimum(a, b)[keep].tolist(), np.maximum(a, b)[keep].tolist()))
    t = np.asarray(truth_sub, dtype=np.int64).reshape(-1, 2)
    ts = set(zip(t.min(axis=1).tolist(), t.max(axis=1).tolist()))
    return len(fs & ts) / max(len(ts), 1), len(ts), len(fs)


def progress(phase, info):
    """One JSON line per finished phase of a long ClusterMerge run, on stderr (the result line
    on stdout stays the only one there)."""
    print(json.dumps({"phase": phase, **info}), file=sys.stderr, flush=True)


def family_pairs(family):
    """Every (i, j), i < j, of two proteins with the same planted family label."""
    family = np.asarray(family)
    order = np.argsort(family, kind="stable")
    bounds = np.flatnonzero(np.diff(family[order])) + 1
    out = []
    for g in np.split(order, bounds):
        if len(g) > 1:
            g = np.sort(g)
            i, j = np.triu_indices(len(g), 1)
            out.append(np.stack([g[i], g[j]], axis=1))
    return np.concatenate(out).astype(np.int32) if out else np.zeros((0, 2), np.int32)


def stratum_recall(found, truth, n):
    """Fraction of the pairs of `truth` (any order within a pair) that `found` contains."""
    def keys(p):
        p = np.asarray(p, dtype=np.int64).reshape(-1, 2)
        return p.min(axis=1) * n + p.max(axis=1)
    t = keys(truth)
    return float(np.isin(t, keys(found)).mean()) if len(t) else 1.0


# algorithmic FLOPs of the ranker per residue row embedded: three 9-tap convolutions
# (32 -> 128, 128 -> 128, 128 -> 128 channels), 2 FLOPs per multiply-add; training runs the
# forward, the data-gradient and the weight-gradient contraction of each (3x the forward)
RANKER_FWD_FLOPS_PER_ROW = 2 * 9 * (32 * 128 + 128 * 128 + 128 * 128)


def measured_peak(key, fallback):
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)[key]), "measured"
    except (OSError, KeyError, ValueError):
        return fallback, "fallback"


def run_train(args):
    """--workload train: one training run of the learned ranker (the learned path's cost) on a
    synthetic proteome, as a bench line against the bf16 tensor-core roofline.  Pairs are drawn
    inside groups of --train-group proteins (grouped_training_pairs) and labelled by the GPU SW
    path before the timed region; the timed region is cm_ranker_train for --epochs epochs."""
    import torch
    import paper_1908_10574_gb300 as cm

    torch.cuda.set_device(0)
    ctx = cm.Context(0)
    tr = synth.proteome(args.train_seqs, family_size=8, singleton_frac=0.2, stream=3)
    rng = np.random.default_rng(13)
    group = max(args.train_group, 2)
    pairs, _ = grouped_training_pairs(tr.family, args.train_pairs, group, rng)
    y = (ctx.sw_score_batch(tr.seqs, tr.offsets, pairs, synth.BLOSUM62, GAP_OPEN, GAP_EXT) >
         T_SIG).astype(np.float32)
    batch_pairs = int(1.5 * len(pairs) * group / max(len(tr), 1)) + 64
    flags = cm.CM_TRAIN_COMPONENTS | cm.CM_TRAIN_COSINE
    ctx.ranker_init(13)
    ctx.ranker_standardize(tr.seqs, tr.offsets, max_sample=2048)
    warm = pairs[: max(1, len(pairs) // 20)]
    ctx.ranker_train(tr.seqs, tr.offsets, warm, y[: len(warm)], epochs=1, batch_pairs=batch_pairs,
                     lr=args.lr, seed=13, flags=flags)
    ctx.ranker_init(13)
    ctx.ranker_standardize(tr.seqs, tr.offsets, max_sample=2048)
    torch.cuda.synchronize()
    clk = ClockSampler(0, args.clocks_dir)
    clk.start()
    ctx.reset_stats()
    t0 = time.perf_counter()
    loss = ctx.ranker_train(tr.seqs, tr.offsets, pairs, y, epochs=args.epochs,
                            batch_pairs=batch_pairs, lr=args.lr, seed=13, flags=flags)
    dt = time.perf_counter() - t0
    clocks = clk.stop()
    st = ctx.stats()
    used = np.unique(pairs.reshape(-1))
    rows = float(tr.lengths[used].astype(np.float64).sum()) * args.epochs
    flops = 3.0 * RANKER_FWD_FLOPS_PER_ROW * rows
    achieved = flops / dt / 1e12
    peak, basis = measured_peak("bf16_tflops_sustained", 1700.0)
    print(json.dumps({
        "metric": "ranker training throughput (bf16 tensor-core convolutions)",
        "value": achieved, "unit": "TFLOP/s", "higher_is_better": True, "n_gpus": 1,
        "dtype": "bf16", "data": "synthetic",
        "config": {"workload": "ranker training on %d synthetic proteins (lognormal lengths "
                               "median 350), %d grouped pairs (groups of %d), %d epoch(s), "
                               "whole components per step, cosine learning rate"
                               % (len(tr), len(pairs), group, args.epochs)},
        "train_seconds": dt, "epochs": args.epochs, "residue_rows": rows,
        "algorithmic_tflop": flops / 1e12, "last_batch_loss": loss,
        "gpu_launches": st["launches"],
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None,
                     "peak_basis": "bf16 dense, sustained (%s)" % basis,
                     "achieved_basis": "3 x %d FLOPs per residue row embedded per epoch over "
                                       "the wall time of cm_ranker_train (host and device)"
                                       % RANKER_FWD_FLOPS_PER_ROW},
        "clocks": clocks}))


def run_cluster_merge(args):
    """ClusterMerge end to end on a proteome-shaped set (default: 100,000 proteins, 80,000 in
    10,000 families of 8 plus 20,000 singletons); recall against the GPU all-against-all when
    --recall, of the whole set or (--recall-sample F) of a random fraction F of its proteins."""
    import torch
    import paper_1908_10574_gb300 as cm
    ss = synth.proteome(args.cm_seqs, family_size=args.family_size,
                        singleton_frac=args.singleton_frac, stream=3)
    if args.long_tail:
        ss = synth.long_tail(ss, args.long_tail, args.long_motifs)
    n = len(ss)
    ctx = cm.Context(0)
    if args.batch_slots:
        ctx.set_batch_limit(args.batch_slots)
    T, mT, mU = T_SIG, M_T, M_U
    ranker = None
    if args.ranker:
        ranker = train_ranker(ctx, args.train_seqs, args.train_pairs, args.epochs, args.keep,
                              lr=args.lr, train_set=ss if args.transductive else None,
                              group=args.train_group)
        progress("ranker training", ranker)
    elif args.ranker_untrained is not None:
        # profiling the ranked path without training: standardised random weights, pruning at
        # a quantile of random-pair logits (the pruning is not meaningful, the work is)
        ctx.ranker_init(13)
        ctx.ranker_standardize(ss.seqs, ss.offsets, max_sample=2048)
        z = ctx.ranker_logits(ss.seqs, ss.offsets, synth.random_pairs(len(ss), 20000, stream=21))
        ranker = {"untrained": True, "prune_logit": float(np.quantile(z, args.ranker_untrained))}
    clk = ClockSampler(0, args.clocks_dir)
    clk.start()
    t0 = time.perf_counter()
    res = ctx.cluster_merge(ss.seqs, ss.offsets, synth.BLOSUM62, GAP_OPEN, GAP_EXT, T, mT, mU,
                            state_path=args.cm_state, budget_seconds=args.cm_budget)
    dt = time.perf_counter() - t0
    clocks = clk.stop()
    if res is None:
        # stopped at a round boundary past --cm-budget; the state is in --cm-state
        print(json.dumps({"metric": "ClusterMerge seconds", "stopped": True,
                          "state": args.cm_state, "seconds_this_call": dt, "clocks": clocks}),
              flush=True)
        return
    if args.cm_state:
        dt = res["stats"]["seconds"]                  # every call of the checkpointed run
    progress("plain merge", {"seconds": dt, "clusters": len(res["clusters"]),
                             "similar_pairs": len(res["pairs"]), "stats": res["stats"],
                             "clocks": clocks})
    ranked = None
    if ranker is not None:
        t1 = time.perf_counter()
        ranked = ctx.cluster_merge(ss.seqs, ss.offsets, synth.BLOSUM62, GAP_OPEN, GAP_EXT, T, mT,
                                   mU, use_ranker=True, prune_logit=ranker["prune_logit"],
                                   ranker_min_pairs=args.min_pairs)
        ranker["ranker_min_pairs"] = args.min_pairs
        ranker["cluster_merge_seconds"] = time.perf_counter() - t1
        ranker["stats"] = ranked["stats"]
        progress("ranked merge", {"seconds": ranker["cluster_merge_seconds"],
                                  "similar_pairs": len(ranked["pairs"]), "stats": ranked["stats"]})
        ranker["clusters"] = len(ranked["clusters"])
        ranker["similar_pairs"] = len(ranked["pairs"])
    out = {"metric": "ClusterMerge seconds", "value": dt, "unit": "s", "n_gpus": 1, "clocks": clocks,
           "higher_is_better": False, "data": "synthetic", "dtype": "int16",
           "config": {"workload": "ClusterMerge of %d synthetic proteins (lognormal lengths, "
                                  "families of %d + %d%% singletons%s), BLOSUM62 11/1, T=%d, mT=%d, "
                                  "mU=%d" % (n, args.family_size, round(100 * args.singleton_frac),
                                             (", + %d tandem repeats of 10,000-35,000 residues in "
                                              "%d motif families" % (args.long_tail, args.long_motifs))
                                             if args.long_tail else "", T, mT, mU)},
           "clusters": len(res["clusters"]), "similar_pairs": len(res["pairs"]),
           "stats": res["stats"], "ranker": ranker}
    if args.recall and args.recall_sample > 0:
        # the all-against-all of a random sample of the proteins (a 1M set's whole
        # all-against-all is ~9e16 cells); recall counts the sample's pairs only
        t1 = time.perf_counter()
        rng = np.random.default_rng(1908)
        m = max(2, int(round(args.recall_sample * n)))
        subset = np.sort(rng.choice(n, size=m, replace=False))
        sub = ss.subset(subset)
        tp = []
        parts = max(1, int(total_cells(sub) / 2e12))
        for part in range(parts):
            p, s = ctx.sw_allpairs(sub.seqs, sub.offsets, synth.BLOSUM62, GAP_OPEN, GAP_EXT, T,
                                   part, parts, capacity=1 << 22)
            tp.append(p.astype(np.int64))
        truth_sub = np.concatenate(tp) if tp else np.zeros((0, 2), np.int64)
        r, nt, nf = subset_recall(res["pairs"][:, :2], subset, truth_sub)
        out["all_pairs_seconds"] = time.perf_counter() - t1
        out["recall_sample"] = {"fraction": args.recall_sample, "proteins": m,
                                "truth_pairs": nt, "found_pairs": nf}
        out["recall"] = r
        if ranked is not None:
            ranker["recall"] = subset_recall(ranked["pairs"][:, :2], subset, truth_sub)[0]
        progress("sample recall", {"recall": r, "recall_sample": out["recall_sample"],
                                   "seconds": out["all_pairs_seconds"]})
    elif args.recall:
        t1 = time.perf_counter()
        truth = set()
        parts = max(1, int(total_cells(ss) / 2e12))
        for part in range(parts):
            p, s = ctx.sw_allpairs(ss.seqs, ss.offsets, synth.BLOSUM62, GAP_OPEN, GAP_EXT, T,
                                   part, parts, capacity=1 << 22)
            truth.update(zip(p[:, 0].tolist(), p[:, 1].tolist()))
        found = set(zip(res["pairs"][:, 0].tolist(), res["pairs"][:, 1].tolist()))
        out["all_pairs_seconds"] = time.perf_counter() - t1
        out["truth_pairs"] = len(truth)
        out["recall"] = len(found & truth) / max(len(truth), 1)
        if ranked is not None:
            fr = set(zip(ranked["pairs"][:, 0].tolist(), ranked["pairs"][:, 1].tolist()))
            ranker["recall"] = len(fr & truth) / max(len(truth), 1)
    if args.recall_families:
        # recall over the planted homologs: every within-family pair scored exactly, those
        # with s > T the truth of this stratum (millions of pairs at 1M proteins)
        t1 = time.perf_counter()
        fp = family_pairs(ss.family)
        sc = ctx.sw_score_batch(ss.seqs, ss.offsets, fp, synth.BLOSUM62, GAP_OPEN, GAP_EXT)
        truth_f = fp[sc > T]
        out["family_recall"] = {"within_family_pairs": int(len(fp)),
                                "similar": int(len(truth_f)),
                                "recall": stratum_recall(res["pairs"][:, :2], truth_f, n),
                                "seconds": time.perf_counter() - t1}
        if ranked is not None:
            ranker["family_recall"] = stratum_recall(ranked["pairs"][:, :2], truth_f, n)
        progress("family recall", out["family_recall"])
    out["comparisons_fraction"] = (res["stats"]["rep_comparisons"] +
                                   res["stats"]["exchange_comparisons"] +
                                   res["stats"]["intra_comparisons"]) / max(n * (n - 1) / 2, 1)
    print(json.dumps(out), flush=True)


# the learned-ranker recipe of the ClusterMerge comparison (training pairs drawn inside groups
# of this many proteins, epochs, peak Adam learning rate with warmup and cosine decay, held-out
# positives kept by the pruning)
CM_RECIPE = {"group": 128, "epochs": 20, "lr": 1e-3, "cosine": True, "keep": 0.9995}


def cm_comparison(ctx, n_seqs=100000, recipes=(CM_RECIPE,), clocks_dir=None, device=0):
    """ClusterMerge of a proteome-shaped set (80 % in families of 8, 20 % singletons, lognormal
    lengths): the plain merge, then for each learned-ranker recipe the whole learned path --
    labelling 1M training pairs with the GPU SW path, training on the set itself, calibrating
    the pruning threshold on held-out pairs, and the ranked merge -- each timed end to end;
    recall of both against the GPU all-against-all of the set (Sec. 6.1), plus recall over the
    planted within-family pairs.  Returns a dict with its own SM-clock record."""
    ss = synth.proteome(n_seqs, family_size=8, singleton_frac=0.2, stream=3)
    n = len(ss)
    T, mT, mU = T_SIG, M_T, M_U
    clk = ClockSampler(device, clocks_dir or tempfile.gettempdir())
    clk.path = clk.path.replace(".csv", "_cm.csv")
    clk.start()
    t0 = time.perf_counter()
    plain = ctx.cluster_merge(ss.seqs, ss.offsets, synth.BLOSUM62, GAP_OPEN, GAP_EXT, T, mT, mU)
    t_plain = time.perf_counter() - t0
    progress("plain merge", {"seconds": t_plain})
    learned = []
    for rc in recipes:
        t0 = time.perf_counter()
        info = train_ranker(ctx, n, 1000000, rc["epochs"], rc["keep"], lr=rc["lr"], train_set=ss,
                            group=rc["group"], cosine=rc.get("cosine", False),
                            seed=rc.get("seed", 13))
        t_train = time.perf_counter() - t0
        t0 = time.perf_counter()
        ranked = ctx.cluster_merge(ss.seqs, ss.offsets, synth.BLOSUM62, GAP_OPEN, GAP_EXT, T, mT,
                                   mU, use_ranker=True, prune_logit=info["prune_logit"],
                                   ranker_min_pairs=100000)
        t_merge = time.perf_counter() - t0
        learned.append((rc, info, t_train, t_merge, ranked))
        progress("learned path", {"recipe": rc, "train_seconds": t_train, "merge_seconds": t_merge})
    t0 = time.perf_counter()
    truth = set()
    parts = max(1, int(total_cells(ss) / 2e12))
    for part in range(parts):
        p, _ = ctx.sw_allpairs(ss.seqs, ss.offsets, synth.BLOSUM62, GAP_OPEN, GAP_EXT, T, part,
                               parts, capacity=1 << 22)
        truth.update(zip(p[:, 0].tolist(), p[:, 1].tolist()))
    t_truth = time.perf_counter() - t0
    clocks = clk.stop()
    fp = family_pairs(ss.family)
    sc = ctx.sw_score_batch(ss.seqs, ss.offsets, fp, synth.BLOSUM62, GAP_OPEN, GAP_EXT)
    truth_f = fp[sc > T]

    def recall(res):
        found = set(zip(res["pairs"][:, 0].tolist(), res["pairs"][:, 1].tolist()))
        return len(found & truth) / max(len(truth), 1)

    def merge_stats(res):
        st = res["stats"]
        return {k: st[k] for k in ("rep_comparisons", "exchange_comparisons", "intra_comparisons",
                                   "comparisons_scored", "full_merges", "exchanges", "rounds",
                                   "t_rep", "t_cells", "t_exchange", "t_intra", "t_rank")}

    out = {"workload": "ClusterMerge of %d synthetic proteins (80%% in 10,000 families of 8, 20%% "
                       "singletons; lognormal lengths median 350 sigma 0.6 clipped 30-5000), "
                       "BLOSUM62 11/1, T=%d, mT=%d, mU=%d" % (n, T, mT, mU),
           "truth_pairs": len(truth), "all_pairs_seconds": t_truth,
           "plain": {"seconds": t_plain, "recall": recall(plain),
                     "family_recall": stratum_recall(plain["pairs"][:, :2], truth_f, n),
                     "similar_pairs": len(plain["pairs"]), "clusters": len(plain["clusters"]),
                     **merge_stats(plain)},
           "learned": [], "clocks": clocks}
    for rc, info, t_train, t_merge, ranked in learned:
        out["learned"].append({
            "recipe": rc, "seconds_total": t_train + t_merge, "seconds_merge": t_merge,
            "seconds_training_path": t_train, "label_seconds": info["label_seconds"],
            "train_seconds": info["train_seconds"], "train_tflops": info["train_tflops"],
            "train_frac_of_bf16_sustained": info["train_frac_of_bf16_sustained"],
            "heldout_auc": info["heldout_auc"],
            "heldout_negatives_kept": info["heldout_negatives_kept"],
            "recall": recall(ranked),
            "family_recall": stratum_recall(ranked["pairs"][:, :2], truth_f, n),
            "ranker_selected": ranked["stats"]["ranker_selected"],
            "vs_plain_end_to_end": t_plain / (t_train + t_merge),
            "vs_plain_merge_only": t_plain / t_merge, **merge_stats(ranked)})
    return out


def grouped_training_pairs(family, n_pairs, group, rng):
    """Training pairs drawn inside groups of about `group` proteins: the planted families
    (singletons count as families of one) are dealt whole, in random order, into consecutive
    groups; each group gets a share of the pairs proportional to its size, half of them two
    distinct members of one of its families (within-family), half two distinct proteins of
    the group drawn uniformly (random).  Returns (pairs (n, 2) int32, group id per pair)."""
    family = np.asarray(family)
    order = np.argsort(family, kind="stable")
    bounds = np.flatnonzero(np.diff(family[order])) + 1
    fstart = np.concatenate([[0], bounds])
    fsize = np.diff(np.concatenate([fstart, [len(order)]]))
    fperm = rng.permutation(len(fsize))
    # members laid out family by family in the dealt order; groups cut at family boundaries
    members = np.concatenate([order[fstart[f]:fstart[f] + fsize[f]] for f in fperm])
    sizes = fsize[fperm]
    cum = np.cumsum(sizes)
    gid_fam = np.zeros(len(sizes), np.int64)
    g, acc = 0, 0
    for i, sz in enumerate(sizes):                  # a group closes once it holds `group`
        gid_fam[i] = g
        acc += sz
        if acc >= group:
            g, acc = g + 1, 0
    ngroups = int(gid_fam[-1]) + 1
    fam_off = cum - sizes                            # first member position of each family
    first = np.searchsorted(gid_fam, np.arange(ngroups), side="left")
    last = np.searchsorted(gid_fam, np.arange(ngroups), side="right") - 1
    gstart = fam_off[first]
    gend = cum[last]
    gsize = gend - gstart
    n = len(family)
    # a group of one protein (a trailing singleton) has no pair to draw
    k = np.where(gsize >= 2, np.maximum(2, np.round(n_pairs * gsize / n).astype(np.int64)), 0)
    multi = np.flatnonzero(sizes > 1)
    mg = gid_fam[multi]
    mcount = np.bincount(mg, minlength=ngroups)
    mfirst = np.searchsorted(mg, np.arange(ngroups), side="left")
    kpos = np.where(mcount > 0, k // 2, 0)
    # within-family pairs: a multi-member family of the group, two distinct members of it
    pg = np.repeat(np.arange(ngroups), kpos)
    fam = multi[mfirst[pg] + rng.integers(0, np.maximum(mcount[pg], 1))]
    a = rng.integers(0, sizes[fam])
    b = rng.integers(0, sizes[fam] - 1)
    b = np.where(b >= a, b + 1, b)
    pos = np.stack([members[fam_off[fam] + a], members[fam_off[fam] + b]], 1)
    # random pairs: two distinct proteins of the group
    kneg = k - kpos
    ng = np.repeat(np.arange(ngroups), kneg)
    a = rng.integers(0, gsize[ng])
    b = rng.integers(0, gsize[ng] - 1)
    b = np.where(b >= a, b + 1, b)
    neg = np.stack([members[gstart[ng] + a], members[gstart[ng] + b]], 1)
    pairs = np.concatenate([pos, neg]).astype(np.int32)
    gids = np.concatenate([pg, ng])
    perm = rng.permutation(len(pairs))[:n_pairs]
    return pairs[perm], gids[perm]


def train_ranker(ctx, n_train_seqs, n_pairs, epochs, keep, seed=13, lr=1e-3, train_set=None,
                 group=512, cosine=False):
    """Train the ranker on a synthetic proteome (an independent one, or `train_set` itself):
    pairs drawn inside groups of about `group` proteins, half within-family and half random
    (grouped_training_pairs), labelled [SW score > T] by the GPU path; 10 % held out to
    calibrate the pruning threshold so that a fraction `keep` of held-out positives survives.
    Each training step takes one group with all of its pairs (CM_TRAIN_COMPONENTS: the library
    batches whole components of the pair graph), so every protein is embedded once per epoch."""
    import paper_1908_10574_gb300 as cm
    tr = train_set if train_set is not None else \
        synth.proteome(n_train_seqs, family_size=8, singleton_frac=0.2, stream=seed)
    rng = np.random.default_rng(seed)
    if group > 0:
        pairs, _ = grouped_training_pairs(tr.family, n_pairs, group, rng)
    else:
        # pairs over the whole set: half within-family, half uniformly random
        fam = tr.family
        order = np.argsort(fam, kind="stable")
        bounds = np.flatnonzero(np.diff(fam[order])) + 1
        groups = [g for g in np.split(order, bounds) if len(g) > 1]
        gi = rng.integers(0, len(groups), size=n_pairs // 2)
        pos = np.array([rng.choice(groups[g], 2, replace=False) for g in gi])
        neg = rng.integers(0, len(tr), size=(n_pairs - len(pos), 2))
        pairs = np.concatenate([pos, neg]).astype(np.int32)
        pairs = pairs[rng.permutation(len(pairs))]
    t0 = time.perf_counter()
    sc = ctx.sw_score_batch(tr.seqs, tr.offsets, pairs, synth.BLOSUM62, GAP_OPEN, GAP_EXT)
    t_label = time.perf_counter() - t0
    y = (sc > T_SIG).astype(np.float32)
    cut = int(0.9 * len(pairs))
    batch_pairs = int(1.5 * n_pairs * group / max(len(tr), 1)) + 64 if group > 0 else 256
    t0 = time.perf_counter()
    ctx.ranker_init(seed)
    ctx.ranker_standardize(tr.seqs, tr.offsets, max_sample=2048)
    loss = ctx.ranker_train(tr.seqs, tr.offsets, pairs[:cut], y[:cut], epochs=epochs,
                            batch_pairs=batch_pairs, lr=lr, seed=seed,
                            flags=(cm.CM_TRAIN_COMPONENTS if group > 0 else 0) |
                                  (cm.CM_TRAIN_COSINE if cosine else 0))
    t_train = time.perf_counter() - t0
    # algorithmic convolution work of the training run: with whole components per step every
    # protein of the training pairs is embedded once per epoch (3 x the forward per row)
    tflops = None
    if group > 0:
        rows = float(tr.lengths[np.unique(pairs[:cut].reshape(-1))].astype(np.float64).sum())
        tflops = 3.0 * RANKER_FWD_FLOPS_PER_ROW * rows * epochs / max(t_train, 1e-9) / 1e12
    z = ctx.ranker_logits(tr.seqs, tr.offsets, pairs[cut:])
    yh = y[cut:]
    thr = float(np.quantile(z[yh == 1], 1.0 - keep))
    zo = np.argsort(z)
    ranks = np.empty(len(z))
    ranks[zo] = np.arange(1, len(z) + 1)
    npos = yh.sum()
    auc = float((ranks[yh == 1].sum() - npos * (npos + 1) / 2) / (npos * (len(yh) - npos)))
    return {"train_seqs": len(tr), "transductive": train_set is not None,
            "train_pairs": int(cut), "heldout_pairs": int(len(pairs) - cut),
            "group": group, "batch_pairs": batch_pairs, "cosine": cosine,
            "positives": float(y.mean()), "epochs": epochs, "lr": lr, "last_batch_loss": loss,
            "label_seconds": t_label, "train_seconds": t_train, "heldout_auc": auc,
            "train_tflops": tflops,
            "train_frac_of_bf16_sustained": (tflops / measured_peak("bf16_tflops_sustained", 1700.0)[0]
                                             if tflops is not None else None),
            "prune_logit": thr, "keep_heldout_positives": keep,
            "heldout_negatives_kept": float((z[yh == 0] >= thr).mean())}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="allpairs", choices=["allpairs", "cm", "train"],
                    help="allpairs: SW GCUPS (default); cm: ClusterMerge seconds; train: ranker "
                         "training TFLOP/s")
    ap.add_argument("--cm-seqs", type=int, default=100000)
    ap.add_argument("--recall", action="store_true")
    ap.add_argument("--recall-sample", type=float, default=0.0, metavar="F",
                    help="cm: measure recall on the all-against-all of a random fraction F of "
                         "the proteins (0: the whole set)")
    ap.add_argument("--recall-families", action="store_true",
                    help="cm: recall over every within-family pair with s > T (planted homologs)")
    ap.add_argument("--family-size", type=int, default=8, help="cm: proteins per family")
    ap.add_argument("--singleton-frac", type=float, default=0.2,
                    help="cm: fraction of proteins outside any family")
    ap.add_argument("--cm-state", default=None, metavar="PATH",
                    help="cm: checkpointed merge (cluster_merge_resume): resume from PATH if it "
                         "holds a state, save the state there when stopping")
    ap.add_argument("--cm-budget", type=float, default=0.0, metavar="S",
                    help="cm with --cm-state: stop at the first round boundary after S seconds")
    ap.add_argument("--batch-slots", type=int, default=0,
                    help="cm: pair slots of one device batch of the rep wave (0: library default)")
    ap.add_argument("--long-tail", type=int, default=0,
                    help="cm: add this many long tandem repeats (the long-tail workload)")
    ap.add_argument("--long-motifs", type=int, default=10)
    ap.add_argument("--ranker", action="store_true", help="cm: also run the learned-ranker merge")
    ap.add_argument("--ranker-untrained", type=float, default=None, metavar="Q",
                    help="cm: run the ranked merge with untrained (standardised) weights, pruning "
                         "at the Q-quantile of random-pair logits (profiling the ranked path)")
    ap.add_argument("--train-seqs", type=int, default=100000)
    ap.add_argument("--train-pairs", type=int, default=1000000)
    ap.add_argument("--epochs", type=int, default=10)
    ap.add_argument("--keep", type=float, default=0.9995)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--train-group", type=int, default=512,
                    help="cm: training pairs are drawn inside groups of this many proteins "
                         "(0: over the whole set, trained in shuffled batches of 256 pairs)")
    ap.add_argument("--transductive", action="store_true",
                    help="cm: train the ranker on the set being clustered (as the 100k setup)")
    ap.add_argument("--min-pairs", type=int, default=100000,
                    help="cm: merges with fewer rep x rep pairs stay unpruned")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cm", action="store_true",
                    help="skip the ClusterMerge plain-vs-learned comparison of the default run")
    ap.add_argument("--clocks-dir", default=tempfile.gettempdir(),
                    help="where the SM-clock samples of the timed region are written")
    ap.add_argument("--parts-per-gpu", type=int, default=PARTS_PER_GPU,
                    help="split of the triangle; a larger value gives shorter steps (profiling)")
    ap.add_argument("--part-offset", type=int, default=0,
                    help="start the part sequence further along (profiling a given length range)")
    ap.add_argument("--warps", type=int, default=0)
    ap.add_argument("--rows", type=int, default=0)
    args = ap.parse_args()
    if args.workload == "cm":
        run_cluster_merge(args)
        return
    if args.workload == "train":
        run_train(args)
        return
    world, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch
    import paper_1908_10574_gb300 as cm

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ctx = cm.Context(local)
    ss = make_set()
    tuning = {"source": "autotune"}
    if args.warps or args.rows:
        ctx.set_tuning(args.warps, args.rows)
        tuning.update(source="command line", warps_per_cta=args.warps, rows_per_warp=args.rows)
    else:
        t0 = time.perf_counter()
        w, r = ctx.autotune(ss.seqs, ss.offsets, synth.BLOSUM62, GAP_OPEN, GAP_EXT, sample_seqs=3000)
        tuning.update(warps_per_cta=w, rows_per_warp=r,
                      autotune_seconds=round(time.perf_counter() - t0, 2))
    dpx_rate = ctx.dpx_rate()
    ctx.reset_stats()
    n_parts = args.parts_per_gpu * world
    seq = part_sequence(n_parts, (args.warmup + args.steps) * world, args.part_offset)
    my_parts = seq[rank::world]
    d_seqs = torch.from_numpy(ss.seqs).to(dev)
    d_off = torch.from_numpy(ss.offsets).to(dev)
    d_mat = torch.from_numpy(synth.BLOSUM62.reshape(-1).copy()).to(dev)
    cap = 1 << 21
    d_pairs = torch.empty((cap, 2), dtype=torch.int32, device=dev)
    d_scores = torch.empty(cap, dtype=torch.int32, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step(part):
        return ctx.sw_allpairs(d_seqs, d_off, d_mat, GAP_OPEN, GAP_EXT, T_SIG, part, n_parts,
                               capacity=cap, pairs_out=d_pairs, scores_out=d_scores)

    for i in range(args.warmup):
        step(my_parts[i])
    torch.cuda.synchronize()
    ctx.reset_stats()
    if args.steps < 1:
        return
    clk = ClockSampler(local, args.clocks_dir)
    clk.start()
    barrier(world)
    torch.cuda.synchronize()
    ms_total = 0.0
    found = 0
    for i in range(args.steps):
        flush.zero_()                                  # L2 flush between timed steps
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        p, s = step(my_parts[args.warmup + i])
        e1.record()
        e1.synchronize()
        ms_total += e0.elapsed_time(e1)
        found += len(s)
    torch.cuda.synchronize()
    barrier(world)
    clocks = clk.stop()
    st = ctx.stats()
    ms_max = max_over_ranks(world, ms_total, dev)
    cells_all = sum_over_ranks(world, float(st["cells"]), dev)
    value = cells_all / (ms_max * 1e-3) / 1e9

    # roofline of the dominant kernel (int16x2 DPX Smith-Waterman), from the library's own
    # CUDA events around its launches on this stream
    props = torch.cuda.get_device_properties(local)
    n_sm = props.multi_processor_count
    clk_mhz = clocks["sm_mhz"] if clocks else None
    achieved = st["cells"] / (st["sw16_ms"] * 1e-3) / 1e9 if st["sw16_ms"] > 0 else None
    # the DPX issue rate measured on this GPU in this run (cm_dpx_rate), lane-ops / clk / SM
    rate = dpx_rate
    peak = n_sm * (clk_mhz * 1e6) * rate * 2.0 / OPS_PER_PACKED_CELL / 1e9 if clk_mhz else None
    peak7 = n_sm * (clk_mhz * 1e6) * rate * 2.0 / OPS_PER_PACKED_CELL_PLAIN / 1e9 if clk_mhz else None
    cells_per_launch = st["cells"] / max(st["sw16_launches"], 1)
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "GCUPS",
            "frac": (achieved / peak) if (achieved and peak) else None,
            "traffic": DRAM_BYTES_PER_CELL * cells_per_launch,
            "traffic_basis": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch of the "
                             "small case (part 253 of 512: sw16_kernel<22,16,0>, 6.40e10 cells, "
                             "6.45 MB read, 0 written), scaled by cells per launch",
            "kernel": "sw16_kernel (int16x2 DPX wavefront)",
            "peak_basis": "%d SMs x median SM clock under load x %.2f DPX lane-ops per clk per SM "
                          "(measured in this run by cm_dpx_rate) x 2 cells per %.1f ops (the "
                          "kernel's cell update)" % (n_sm, rate, OPS_PER_PACKED_CELL),
            "dpx_lane_ops_per_clk_per_sm": rate,
            "frac_7op": (achieved / peak7) if (achieved and peak7) else None,
            "peak_7op": peak7,
            "sw16_ms_per_launch": st["sw16_ms"] / max(st["sw16_launches"], 1),
            "cells_per_launch": st["cells"] / max(st["sw16_launches"], 1),
            "padded_cell_fraction": (st["cells"] / st["cells_padded"]) if st["cells_padded"] else None}

    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(a).pin_memory().numpy()
        h_seqs, h_off, h_mat = pin(ss.seqs), pin(ss.offsets), pin(synth.BLOSUM62.reshape(-1).copy())
        h_pairs = pin(np.empty((cap, 2), np.int32))
        h_scores = pin(np.empty(cap, np.int32))
        ctx.reset_stats()
        barrier(world)
        t0 = time.perf_counter()
        nf = 0
        for i in range(args.steps):
            p, s = ctx.sw_allpairs(h_seqs, h_off, h_mat, GAP_OPEN, GAP_EXT, T_SIG,
                                   my_parts[args.warmup + i], n_parts, capacity=cap,
                                   pairs_out=h_pairs, scores_out=h_scores)
            nf += len(s)
        dt = time.perf_counter() - t0
        dt = max_over_ranks(world, dt, dev)
        cells_e = sum_over_ranks(world, float(ctx.stats()["cells"]), dev)
        e2e = {"value": cells_e / dt / 1e9, "unit": "GCUPS",
               "h2d_bytes_per_step": int(ss.seqs.nbytes + ss.offsets.nbytes + 400),
               "d2h_bytes_per_step": int(nf * 12 / args.steps)}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(ss)

    # the headline's second half: ClusterMerge at 100k proteins, plain vs learned (training
    # included), recall against the GPU all-against-all; one GPU only
    cmcmp = None
    if world == 1 and not args.no_cm:
        cmcmp = cm_comparison(ctx, args.cm_seqs, clocks_dir=args.clocks_dir, device=local)

    if rank == 0:
        out = {"metric": METRIC, "value": value, "unit": "GCUPS", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "int16", "data": "synthetic",
               "config": {"workload": workload_desc(n_parts), "n_seqs": N_SEQS,
                          "families": N_SEQS // FAMILY, "cells_all_pairs": total_cells(ss),
                          "cells_timed": int(cells_all), "significant_pairs_timed": found,
                          "parts_timed": my_parts[args.warmup:], "n_parts": n_parts,
                          "l2": "flushed between timed steps (256 MiB write)",
                          "tuning": tuning},
               "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
               "gpu_launches": int(st["launches"]), "clocks": clocks,
               "cluster_merge": cmcmp}
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
