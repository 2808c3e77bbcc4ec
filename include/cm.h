/*
 * cm.h -- C ABI of the GB300 batched Smith-Waterman / ClusterMerge library (libcm.so).
 *
 * What is computed (Byma et al., "Parallel and Scalable Precise Clustering for Homologous
 * Protein Discovery", PPoPP'20):
 *   - the similarity f of two proteins is their Smith-Waterman local-alignment score under a
 *     substitution matrix with gaps (Sec. 4); this library uses the affine (Gotoh) gap model,
 *     a gap of k residues costing gap_open + (k-1)*gap_extend (CM_GAP_BLAST: open + k*extend);
 *   - a pair (i, j) is significant when f(i, j) > T (Sec. 3);
 *   - ClusterMerge builds a precise clustering by bottom-up cluster-set merges (Algorithm 1
 *     Merge, Algorithm 2 BottomUpMerge) with the protein transitivity test of Sec. 4 (score >
 *     mT and fewer than mU uncovered residues), then aligns all pairs inside each final
 *     cluster (Sec. 6.1).
 *
 * Conventions for every entry point
 *   - Return value: CM_OK (0) or a negative CM_ERR_* code; cm_last_error() describes the last
 *     error on that context.  On error no output array has been written.
 *   - Sequences: `seqs` is one concatenated array of residue codes 0..19 in the order
 *     ARNDCQEGHILKMFPSTWYV (or ASCII letters with CM_ASCII); sequence i is
 *     seqs[offsets[i] .. offsets[i+1]), offsets has n_seqs+1 non-decreasing int64 entries
 *     starting at 0.  Sequences may be empty (their scores are 0); one longer than 2^28
 *     residues is rejected with CM_ERR_ARG.  Device scratch grows with the longest sequence
 *     of a call (one boundary column per resident warp, 40-160 KB per residue on 152 SMs: a
 *     few GB at 35,000 residues); a call whose scratch does not fit the device fails with
 *     CM_ERR_OOM before any output is written.
 *   - Matrix: 400 int8 entries, row-major, matrix[x*20 + y] = score of residue x of the
 *     pair's FIRST sequence against residue y of its SECOND sequence.  Entries must lie in
 *     [-1000, 1000]; it need not be symmetric.  With CM_MATRIX24 the matrix has 576 entries
 *     (matrix[x*24 + y]) over the 24 letters ARNDCQEGHILKMFPSTWYVBZX* (B = D or N, Z = E or Q,
 *     X = any, * = stop; the layout of the published 24 x 24 tables), residue codes may be
 *     0..23 and CM_ASCII also accepts B, Z, X and *.  The learned ranker embeds codes 20..23
 *     as zero vectors.
 *   - Gaps: 1 <= first-gap cost (gap_open, or gap_open+gap_extend with CM_GAP_BLAST) <= 1000,
 *     0 <= gap_extend <= first-gap cost.
 *   - Pointers: host memory by default; with CM_DEVICE_PTRS every array argument is device
 *     memory on the context's device and all work is ordered on the context's stream
 *     (cm_set_stream); the call still returns after the results are written.
 *   - Ownership: the caller owns every input and output array; the library never keeps a
 *     pointer to them after returning.  cm_result objects are owned by the library and freed
 *     with cm_result_free().
 *   - Thread safety: a context may be used by one host thread at a time.
 */
#ifndef CM_H
#define CM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---- */
#define CM_OK              0
#define CM_ERR_ARG        -1   /* invalid argument (null pointer, bad size, bad offsets) */
#define CM_ERR_RESIDUE    -2   /* residue code >= 20, or non-amino-acid letter with CM_ASCII */
#define CM_ERR_OOM        -3   /* device or host allocation failed */
#define CM_ERR_CUDA       -4   /* a CUDA call failed; message in cm_last_error() */
#define CM_ERR_TIMEOUT    -5   /* a bounded device wait gave up (a long pair's pass pipeline) */
#define CM_ERR_CAPACITY   -6   /* output capacity too small; *n_found holds the needed size */
#define CM_ERR_INTERNAL   -7   /* a kernel's own bounds check fired (a library bug) */
#define CM_STOPPED         1   /* cluster_merge_resume stopped at a round boundary, state saved */

/* ---- flags ---- */
#define CM_DEVICE_PTRS    0x1u  /* all array arguments are device pointers */
#define CM_ASCII          0x2u  /* seqs holds ASCII letters (upper or lower case) */
#define CM_GAP_BLAST      0x4u  /* gap of k residues costs open + k*extend */
#define CM_FORCE_INT32    0x8u  /* score every pair on the int32 path (no int16x2 first pass) */
#define CM_MATRIX24       0x40u /* 24 x 24 matrix over ARNDCQEGHILKMFPSTWYVBZX* (codes 0..23) */
#define CM_TRAIN_COMPONENTS 0x10u /* cm_ranker_train: batches hold whole components of the pair graph */
#define CM_TRAIN_COSINE   0x20u /* cm_ranker_train: learning rate warms up over the first 2 % of the
                                   steps, then follows a half cosine from lr down to 0 */

typedef struct cm_ctx cm_ctx;

/* Create a context on CUDA device `device`: a stream, device scratch grown on demand, and
 * the scheduler's tuning state.  *out is set to NULL on failure. */
int cm_create(cm_ctx **out, int device);

/* Release the context and every device buffer it owns.  NULL is ignored. */
void cm_destroy(cm_ctx *ctx);

/* Message of the last error on this context ("" if none).  Valid until the next call on it. */
const char *cm_last_error(const cm_ctx *ctx);

/* Order all further device work of this context on `cuda_stream` (a cudaStream_t on the
 * context's device; NULL selects the context's own stream). */
int cm_set_stream(cm_ctx *ctx, void *cuda_stream);

/* Scheduler tuning of the int16x2 kernel: warps per CTA (4, 8 or 16) and target rows per
 * warp stream (256 .. 65536).  0 keeps the current value.  The autotuner sets these. */
int cm_set_tuning(cm_ctx *ctx, int32_t warps_per_cta, int32_t rows_per_warp);

/* Upper bound on the pair slots (4 bytes of device memory each, plus the subjects' row
 * streams) of one device batch of ClusterMerge's representative wave (Algorithm 2 rounds,
 * Sec. 5's merges of large sets).  A round whose rep x rep cross products exceed it runs as
 * several batches, cut between query rows, with the same results.  max_slots >= 1024;
 * 0 restores the default of 2^32. */
int cm_set_batch_limit(cm_ctx *ctx, int64_t max_slots);

/* Bound on the one device wait of the library: a pass of the whole-CTA long-pair kernels
 * (int32 rescoring and alignment cells of pairs of >= 2,048 x 512 residues) waits for the
 * rows its predecessor pass has written.  Such a wait always ends in a correct run; after
 * `polls` polls of ~100 ns each it gives up instead, the call returns CM_ERR_TIMEOUT with
 * nothing written, and the context stays usable.  0 restores the default of 2^24 polls
 * (~1.7 s).  A small value exists to exercise that error path. */
int cm_set_wait_limit(cm_ctx *ctx, int32_t polls);

/* Autotuner: scores the all-against-all of a length-stratified sample of `sample_seqs` of the
 * given sequences (0 = 3000) under every CTA width (4, 8, 16 warps) and warp-stream length
 * (4096 .. 32768 rows), keeps the fastest (CUDA-event time of the int16x2 kernel per cell) as
 * the context's tuning and reports it.  With cache_path (may be NULL) the choice is looked up
 * first and appended after measuring, keyed by GPU name, SM count and median length bucket. */
int cm_autotune(cm_ctx *ctx, const uint8_t *seqs, const int64_t *offsets, int32_t n_seqs,
                const int8_t *matrix, int32_t gap_open, int32_t gap_extend, int32_t sample_seqs,
                const char *cache_path, int32_t *warps_out, int32_t *rows_out, uint32_t flags);

/* Issue rate of the packed 16-bit DPX max-add instructions the Smith-Waterman cell update is
 * built from, measured on this GPU: one CTA of 1,024 threads per SM runs independent chains
 * of __viaddmax_s16x2 / __vimax3_s16x2 (3:1) timed with each SM's clock64.  Writes
 * lane-operations per clock per SM (the roofline denominator of the int16x2 kernel: peak
 * cells/s = SMs x clock x rate x 2 cells / operations per packed cell).  No paper counterpart:
 * a measurement of the hardware. */
int cm_dpx_rate(cm_ctx *ctx, double *lane_ops_per_clk_per_sm);

/* Counters of the work done since cm_create or the last cm_reset_stats. */
typedef struct {
    int64_t pairs;              /* pairs scored */
    int64_t cells;              /* sum of len(a)*len(b) over the pairs scored */
    int64_t cells_padded;       /* cells actually computed by the int16x2 kernel (padding incl.) */
    int64_t saturated;          /* pairs rerun on the int32 path after int16 saturation */
    int64_t launches;           /* kernel launches */
    int64_t sw16_launches;      /* launches of the int16x2 Smith-Waterman kernel */
    double  sw16_ms;            /* device time of those launches (CUDA events on the stream) */
    double  total_ms;           /* device time of whole calls (CUDA events on the stream) */
} cm_stats;
int cm_get_stats(const cm_ctx *ctx, cm_stats *out);
int cm_reset_stats(cm_ctx *ctx);

/* sw_score_batch -- similarity f (Sec. 4) of every pair in a list.
 *   pairs:      2*n_pairs int32 sequence indices; pair k is (pairs[2k], pairs[2k+1]) and is
 *               scored with the matrix indexed [first][second].
 *   scores_out: n_pairs int32, the Smith-Waterman (Gotoh) local-alignment score of each pair,
 *               exact (int16x2 pass; pairs that could overflow int16 are rerun in int32).
 * Pairs sharing their first sequence are scored together against that sequence's query
 * profile, so listing the sequence with many partners first is fastest. */
int sw_score_batch(cm_ctx *ctx, const uint8_t *seqs, const int64_t *offsets, int32_t n_seqs,
                   const int32_t *pairs, int64_t n_pairs, const int8_t *matrix,
                   int32_t gap_open, int32_t gap_extend, int32_t *scores_out, uint32_t flags);

/* sw_cells_batch -- score plus the cells of one optimal local alignment per pair, the
 * quantity the protein transitivity test needs (Sec. 4: residues uA, uD left uncovered).
 *   cells_out: 5*n_pairs int32: score, i_start, i_end, j_start, j_end (1-based, inclusive,
 *              i over the first sequence).  The end cell is the first cell in row-major order
 *              (i, then j) whose score equals the optimum; the start is the first row-major
 *              cell of the same recurrence run on the reversed prefixes a[i_end..1],
 *              b[j_end..1] (the optimal alignment ending there that spans the fewest residues
 *              of a, then of b).  All four cells are 0 when the score is 0. */
int sw_cells_batch(cm_ctx *ctx, const uint8_t *seqs, const int64_t *offsets, int32_t n_seqs,
                   const int32_t *pairs, int64_t n_pairs, const int8_t *matrix,
                   int32_t gap_open, int32_t gap_extend, int32_t *cells_out, uint32_t flags);

/* sw_allpairs -- the all-against-all comparison (Sec. 1, Sec. 6.1): every pair i < j of the
 * set is aligned and the significant pairs f(i, j) > T (Sec. 3) are returned.
 *   part, n_parts: the triangle of pairs is split into n_parts parts of about equal cell
 *               count (pairs grouped by the longer sequence); this call scores part `part`
 *               (0 <= part < n_parts).  The union over all parts is the full result.
 *   pairs_out:  2*capacity int32 (i, j) with i < j;  scores_out: capacity int32.
 *   n_found:    number of significant pairs of this part (host pointer, always host).
 * If *n_found > capacity nothing is written and CM_ERR_CAPACITY is returned.  Output order
 * is deterministic: by (longer sequence, shorter sequence) in length order (ties by index). */
int sw_allpairs(cm_ctx *ctx, const uint8_t *seqs, const int64_t *offsets, int32_t n_seqs,
                const int8_t *matrix, int32_t gap_open, int32_t gap_extend, int32_t T,
                int64_t part, int64_t n_parts, int32_t *pairs_out, int32_t *scores_out,
                int64_t capacity, int64_t *n_found, uint32_t flags);

/* sw_align_batch -- one optimal local alignment per pair, for re-aligning the similar pairs a
 * clustering reports (Sec. 6.1), as run-length operations.
 *   cells_out:   5*n_pairs int32 as sw_cells_batch (score, i_start, i_end, j_start, j_end).
 *   ops_offsets: n_pairs+1 int64; the runs of pair k are ops_out[ops_offsets[k] ..
 *                ops_offsets[k+1]), none when its score is 0.
 *   ops_out:     ops_capacity int32 runs, each (length << 2) | op from the alignment's start to
 *                its end: op 0 = M (a residue of the first sequence aligned with one of the
 *                second), 1 = I (a residue of the first sequence against a gap), 2 = D (a
 *                residue of the second sequence against a gap).
 *   n_ops:       total runs (host pointer, always host).
 * The alignment spans exactly the cells: a[i_start..i_end] against b[j_start..j_end].  Inside
 * that span it is the global affine alignment of the two substrings (same gap costs), which
 * scores the local optimum; among equal-scoring ones the traceback from the end takes an
 * aligned pair first, then I, then D, and a gap's opening before its extension.  If
 * *n_ops > ops_capacity nothing is written and CM_ERR_CAPACITY is returned.  One GPU thread
 * aligns one pair (a p x q byte matrix of choices per pair in device scratch): meant for the
 * similar pairs of a clustering, not for all-against-all. */
int sw_align_batch(cm_ctx *ctx, const uint8_t *seqs, const int64_t *offsets, int32_t n_seqs,
                   const int32_t *pairs, int64_t n_pairs, const int8_t *matrix,
                   int32_t gap_open, int32_t gap_extend, int32_t *cells_out,
                   int64_t *ops_offsets, int32_t *ops_out, int64_t ops_capacity,
                   int64_t *n_ops, uint32_t flags);

/* ---- ClusterMerge (Algorithm 1 Merge, Algorithm 2 BottomUpMerge, Sec. 4 transitivity) ---- */
typedef struct {
    int32_t T;      /* significance: a pair is similar when its score > T (Sec. 3) */
    int32_t mT;     /* full-merge threshold: representatives' score > mT (Sec. 4) */
    int32_t mU;     /* full merge needs fewer than mU uncovered residues in the absorbed rep */
    int32_t use_ranker;    /* 1: the learned ranker orders and prunes rep x rep comparisons */
    float prune_logit;     /* with the ranker: rep pairs whose logit is below this are not
                              aligned (treated as dissimilar); Algorithm 1 still visits the
                              kept pairs in set order */
    int32_t ranker_min_pairs;  /* only merges with |cs1|*|cs2| >= this use the ranker */
    int32_t merge_mode;    /* CM_MERGE_SEQUENTIAL (0) or CM_MERGE_PARTIAL (1), below */
    int32_t reserved;      /* must be 0 */
} cm_params;

/* merge_mode.  CM_MERGE_SEQUENTIAL: Algorithm 1 exactly, Set 1's clusters one after another.
 * CM_MERGE_PARTIAL: every set merge runs as independent partial merges (Sec. 5), as the
 * distributed runtime's workers do: each cluster of Set 1 runs Algorithm 1's inner loop
 * against Set 2 as it stood when the merge began (it does not see what the other partial
 * merges did: clusters they fully merged are still visited, members they added are not
 * seen); then the additions to every Set-2 cluster are applied in Set-1 order without
 * duplicates, and the merged set keeps the clusters of both sets that no partial merge fully
 * merged (members added to a fully merged Set-2 cluster go with it).  Deterministic; it does
 * a little more work than the sequential merge and its recall differs slightly. */
#define CM_MERGE_SEQUENTIAL 0
#define CM_MERGE_PARTIAL    1

typedef struct {
    int32_t n_seqs;
    int32_t n_clusters;
    int32_t *reps;             /* n_clusters representatives (final set order) */
    int64_t *cl_offsets;       /* n_clusters+1 offsets into members */
    int32_t *members;          /* members of every cluster, insertion order, rep first */
    int64_t n_pairs;           /* similar pairs found: i < j, score > T, sorted by (i, j) */
    int32_t *pairs;            /* 2*n_pairs */
    int32_t *scores;           /* n_pairs */
    int64_t rep_comparisons;       /* representative comparisons of Algorithm 1 */
    int64_t exchange_comparisons;  /* member-vs-representative comparisons of ExchangeSimilar */
    int64_t intra_comparisons;     /* distinct intra-cluster pairs aligned (Sec. 6.1) */
    int64_t comparisons_scored;    /* alignments run on the GPU (speculation and duplicates incl.) */
    int64_t cells_pairs;           /* alignments re-run for their cells (candidate full merges) */
    int64_t full_merges, exchanges, merges, rounds, gpu_batches, exchange_waves;
    double seconds;                /* wall time of the call */
    double t_rep, t_cells, t_exchange, t_intra;   /* wall time of the device batches by kind */
    double t_rank;                 /* ranker inference and pair selection */
    int64_t ranker_selected;       /* rep pairs the ranker kept */
} cm_result;

/* cluster_merge -- precise clustering of a protein set (Sec. 3-4) followed by the
 * intra-cluster all-against-all (Sec. 6.1).  Deterministic: without the ranker, clusters,
 * member order, similar pairs and the three logical comparison counts equal those of the
 * plain sequential Algorithms 1 and 2 (FIFO in input order); with it, the same algorithm runs
 * on the ranker's pruned and ordered representative comparisons.  The matrix must be
 * symmetric.  *out is owned by the library; release it with cm_result_free. */
int cluster_merge(cm_ctx *ctx, const uint8_t *seqs, const int64_t *offsets, int32_t n_seqs,
                  const int8_t *matrix, int32_t gap_open, int32_t gap_extend,
                  const cm_params *params, cm_result **out, uint32_t flags);
void cm_result_free(cm_result *result);

/* cluster_merge_resume -- cluster_merge with round-state checkpoints (the position in
 * Algorithm 2's merge schedule plus the clusters of every set a later round reads).  If
 * `state_path` names a checkpoint, the run resumes after its last completed round; a
 * checkpoint of another problem (sequence lengths, matrix, gaps, params or flags differ) is
 * rejected with CM_ERR_ARG -- the caller must pass the same residues, which are not
 * fingerprinted.  With budget_seconds > 0 the call stops after the first completed round at
 * which budget_seconds have passed since it began (unless no round is left), writes the
 * checkpoint to `state_path` (through a temporary file renamed over it) and returns CM_STOPPED
 * with *out = NULL; call again to continue.  Otherwise, or once every round is done, it
 * finishes as cluster_merge and returns CM_OK; result->seconds then sums the wall time of
 * every call of the run.  The result equals cluster_merge's (clusters, member order, pairs and
 * the logical comparison counts); comparisons_scored may grow, since scores cached in one call
 * are recomputed in the next.  With the ranker, the context must hold the same ranker weights
 * in every call (cm_ranker_load).  Errors as cluster_merge, plus CM_ERR_ARG for an unreadable,
 * truncated or foreign state file or one that cannot be written. */
int cluster_merge_resume(cm_ctx *ctx, const uint8_t *seqs, const int64_t *offsets,
                         int32_t n_seqs, const int8_t *matrix, int32_t gap_open,
                         int32_t gap_extend, const cm_params *params, const char *state_path,
                         double budget_seconds, cm_result **out, uint32_t flags);

/* greedy_cluster -- incremental greedy clustering, the comparison method of Sec. 2 (after
 * Wittwer et al.), on the same kernels: sequences in input order are compared with every
 * cluster representative in creation order; a sequence joins the cluster of every
 * representative with score > T, and becomes the representative of a new cluster unless
 * some representative represents it (score > mT and fewer than mU of its residues outside
 * their optimal local alignment, the Sec. 4 test).  Then the intra-cluster all-against-all
 * (Sec. 6.1), as cluster_merge.  params: T, mT, mU; use_ranker and merge_mode must be 0.
 * Result as cluster_merge: clusters in creation order (members in joining order, rep
 * first), rep_comparisons = the comparisons with representatives, full_merges = sequences
 * represented by an existing cluster, rounds = device batches of sequences (2,048 each, the
 * chunk scored against the representatives before it and, speculatively, against itself). */
int greedy_cluster(cm_ctx *ctx, const uint8_t *seqs, const int64_t *offsets, int32_t n_seqs,
                   const int8_t *matrix, int32_t gap_open, int32_t gap_extend,
                   const cm_params *params, cm_result **out, uint32_t flags);

/* ---- learned representative ranker (orders and prunes rep x rep comparisons) ----
 * The paper has no learned component; this network only decides which representative pairs
 * are aligned (and in which order) inside Algorithm 1 — the exact Smith-Waterman score alone
 * decides similarity.  Model: residue embedding (20 x 32) -> conv1d 32->128 (width
 * 9) + ReLU -> conv1d 128->128 + ReLU -> conv1d 128->128 -> mean over the sequence -> v (128-d);
 * logit(a, b) = alpha * cos(v_a, v_b) + beta, cos = <a,b> / sqrt((|a|^2+1e-6)(|b|^2+1e-6)),
 * trained with binary cross-entropy on labels
 * [score(a, b) > T].  Parameters are one flat float array of cm_ranker_num_params() values in
 * the order E[20][32], W1[9][32][128], b1[128], W2[9][128][128], b2[128], W3[9][128][128],
 * b3[128], alpha, beta (W[k][c][n]: tap k, input channel c, output channel n).  Sequence and
 * pair arguments follow the conventions above (host pointers; CM_ASCII accepted). */
int64_t cm_ranker_num_params(void);
int cm_ranker_init(cm_ctx *ctx, uint64_t seed);
int cm_ranker_set_params(cm_ctx *ctx, const float *params, int64_t n);
/* data-dependent init: rescale W3, b3 so every channel of v has zero mean and unit variance
 * over an evenly spaced sample of at most max_sample of the sequences */
int cm_ranker_standardize(cm_ctx *ctx, const uint8_t *seqs, const int64_t *offsets,
                          int32_t n_seqs, int32_t max_sample, uint32_t flags);
int cm_ranker_get_params(cm_ctx *ctx, float *params, int64_t n);
/* Save the parameters to a file / load them from one: 8 bytes "CMRANK01", the parameter count
 * as a little-endian int64, then the parameters as little-endian float32, in the order above.
 * Errors: CM_ERR_ARG for a null path, an unreadable or unwritable file, or a file whose tag or
 * count does not match (nothing is loaded then); saving needs parameters to be set. */
int cm_ranker_save(cm_ctx *ctx, const char *path);
int cm_ranker_load(cm_ctx *ctx, const char *path);
/* mean BCE loss of the pairs and its gradient w.r.t. every parameter (grad may be NULL) */
int cm_ranker_loss_grad(cm_ctx *ctx, const uint8_t *seqs, const int64_t *offsets, int32_t n_seqs,
                        const int32_t *pairs, const float *labels, int64_t n_pairs,
                        float *loss, float *grad, uint32_t flags);
/* Adam (beta1 0.9, beta2 0.999, eps 1e-8) over mini-batches of at most batch_pairs pairs,
 * reshuffled every epoch (seeded by `seed`); the loss of a step is the mean BCE over its pairs.
 * Each step embeds every distinct sequence of its batch once.  By default a batch is a chunk
 * of the shuffled pair list.  With CM_TRAIN_COMPONENTS in flags a batch holds whole connected
 * components of the pair graph (sequences as nodes, pairs as edges), as many as fit, and a
 * component with more pairs is cut into chunks of batch_pairs: pairs drawn within groups of
 * sequences then train one group per step with all of its pairs, each sequence embedded once
 * per epoch.  The component order and the pairs inside each component are shuffled. */
int cm_ranker_train(cm_ctx *ctx, const uint8_t *seqs, const int64_t *offsets, int32_t n_seqs,
                    const int32_t *pairs, const float *labels, int64_t n_pairs, int32_t epochs,
                    int32_t batch_pairs, float lr, uint64_t seed, float *last_loss,
                    uint32_t flags);
/* v of every sequence: out is n_seqs x 128 floats (device memory with CM_DEVICE_PTRS) */
int cm_ranker_embed(cm_ctx *ctx, const uint8_t *seqs, const int64_t *offsets, int32_t n_seqs,
                    float *out, uint32_t flags);
/* logits of pairs (n_pairs floats, host) */
int cm_ranker_logits(cm_ctx *ctx, const uint8_t *seqs, const int64_t *offsets, int32_t n_seqs,
                     const int32_t *pairs, int64_t n_pairs, float *out, uint32_t flags);

/* sw_cells_batch_noalloc -- the same results as sw_cells_batch, for callers that cannot
 * allocate device memory when they call (for example a service whose GPU memory is reserved
 * up front by another framework's caching allocator, or a latency-bound loop that must avoid
 * the device synchronisation cudaMalloc/cudaFree can cause).  The paper has no counterpart:
 * this is a deployment variant of the alignment-cells pass.
 *   seqs, offsets, pairs, cells_out: DEVICE pointers on the current CUDA device (no context);
 *   matrix: HOST pointer (400 int8, as above); cuda_stream: the stream to run on (NULL = the
 *   legacy default stream); flags: 0 or CM_GAP_BLAST; err_msg/err_len: optional caller buffer
 *   that receives a message on error (may be NULL).
 * It calls no cudaMalloc, cudaFree or other allocating routine: the per-pair DP rows use one
 * fixed 32 MiB array compiled into the library, which every GPU that loads the library keeps
 * until the process exits.  Limit: the second sequence of every pair must have at most 4095
 * residues; larger pairs are rejected with CM_ERR_ARG before anything is written.  Pair
 * indices, offset order and residue codes are checked on the device before any output is
 * written, but the length of the `seqs` allocation is not passed: offsets[n_seqs] must not
 * exceed it (the caller's guarantee).  Every call looks up that array's device address on the
 * current device (cudaGetSymbolAddress; the first lookup on a device may load the library's
 * device code), so make the first call on a device before any stream capture.  All calls
 * share the array: calls whose work overlaps on the GPU (other streams or threads) race and
 * must be serialised by the caller.  The call returns after the results are written. */
int sw_cells_batch_noalloc(const uint8_t *seqs, const int64_t *offsets, int32_t n_seqs,
                           const int32_t *pairs, int64_t n_pairs, const int8_t *matrix,
                           int32_t gap_open, int32_t gap_extend, int32_t *cells_out,
                           void *cuda_stream, uint32_t flags, char *err_msg, int32_t err_len);

#ifdef __cplusplus
}
#endif

#endif /* CM_H */
