/*
 * Oracle: plain scalar Smith-Waterman local alignment with affine gaps (Gotoh), int64.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
 * leg may load this library.  It shares no code, header or table with the CUDA path.
 *
 * The paper's similarity f is the Smith-Waterman score (Sec. 4, "Protein Sequence
 * Clustering"): a weighted sum of matches, mismatches and gaps under a substitution matrix.
 * It names neither the gap model nor its constants; this oracle takes the affine (Gotoh)
 * model with two conventions:
 *   gap_mode 0: a gap of k residues costs o + (k-1)*e
 *   gap_mode 1: a gap of k residues costs o + k*e            (BLAST-style)
 *
 * Recurrences over a (rows i = 1..m) and b (columns j = 1..n), S[x*24+y] = score(x, y) (a
 * 24 x 24 table over ARNDCQEGHILKMFPSTWYVBZX*; 20-letter matrices fill its top-left corner):
 *   E(i,j) = max(E(i,j-1) - e, H(i,j-1) - g1)     horizontal gap, g1 = cost of a 1-gap
 *   F(i,j) = max(F(i-1,j) - e, H(i-1,j) - g1)     vertical gap
 *   H(i,j) = max(0, H(i-1,j-1) + S(a_i, b_j), E(i,j), F(i,j))
 *   H(0,.) = H(.,0) = 0,  E(i,0) = F(0,j) = -infinity
 * score = max over all cells of H.  End cell = first (i, j) in row-major order (i, then j)
 * with H = score.  Start cell: the same DP on the reversed prefixes a[i_e..1], b[j_e..1];
 * the first cell (i', j') in row-major order with H' = score gives i_s = i_e - i' + 1,
 * j_s = j_e - j' + 1.  When score == 0 all four cell indices are 0.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define NEG_INF (INT64_MIN / 4)

static int64_t max64(int64_t x, int64_t y) { return x > y ? x : y; }

/* Forward DP over a[0..m) x b[0..n) with optional reversal of both inputs.
 * Returns the best score; writes the first row-major cell (1-based) reaching it. */
static int64_t gotoh(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n, int reverse,
                     const int32_t *S, int64_t o, int64_t e, int gap_mode,
                     int64_t *best_i, int64_t *best_j)
{
    int64_t g1 = (gap_mode == 0) ? o : o + e;
    int64_t *Hprev = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t *Hcur = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t *F = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n + 1));
    int64_t best = 0, bi = 0, bj = 0;
    for (int64_t j = 0; j <= n; j++) { Hprev[j] = 0; F[j] = NEG_INF; }
    for (int64_t i = 1; i <= m; i++) {
        uint8_t ai = reverse ? a[m - i] : a[i - 1];
        int64_t E = NEG_INF;
        Hcur[0] = 0;
        for (int64_t j = 1; j <= n; j++) {
            uint8_t bj_res = reverse ? b[n - j] : b[j - 1];
            E = max64(E - e, Hcur[j - 1] - g1);
            F[j] = max64(F[j] - e, Hprev[j] - g1);
            int64_t h = Hprev[j - 1] + (int64_t)S[ai * 24 + bj_res];
            h = max64(h, E);
            h = max64(h, F[j]);
            h = max64(h, 0);
            Hcur[j] = h;
            if (h > best) { best = h; bi = i; bj = j; }
        }
        int64_t *t = Hprev; Hprev = Hcur; Hcur = t;
    }
    free(Hprev); free(Hcur); free(F);
    *best_i = bi; *best_j = bj;
    return best;
}

int64_t cm_oracle_sw(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                     const int32_t *S, int64_t o, int64_t e, int gap_mode)
{
    int64_t bi, bj;
    return gotoh(a, m, b, n, 0, S, o, e, gap_mode, &bi, &bj);
}

/* Score plus end and start cells (1-based, inclusive).  out[0..4] = score, i_s, i_e, j_s, j_e */
void cm_oracle_sw_cells(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                        const int32_t *S, int64_t o, int64_t e, int gap_mode, int64_t *out)
{
    int64_t ie, je, ri, rj;
    int64_t best = gotoh(a, m, b, n, 0, S, o, e, gap_mode, &ie, &je);
    out[0] = best;
    if (best == 0) { out[1] = out[2] = out[3] = out[4] = 0; return; }
    /* reversed prefixes a[ie..1], b[je..1] */
    int64_t best2 = gotoh(a, ie, b, je, 1, S, o, e, gap_mode, &ri, &rj);
    (void)best2;
    out[1] = ie - ri + 1;
    out[2] = ie;
    out[3] = je - rj + 1;
    out[4] = je;
}

/* One optimal local alignment as run-length operations (the alignment biologists re-inspect
 * for the similar pairs, Sec. 6.1).  The alignment spans exactly the cells of
 * cm_oracle_sw_cells: a[i_s..i_e] against b[j_s..j_e].  Inside that rectangle it is a global
 * affine alignment of the two substrings (Gotoh recurrences; it scores the local optimum,
 * since a global alignment of the span is a local alignment and the optimal local alignment
 * is a global alignment of its span):
 *   H(0,0) = 0;  H(0,j) = E(0,j) = -(g1 + (j-1)e);  H(i,0) = F(i,0) = -(g1 + (i-1)e)
 *   E(i,j) = max(H(i,j-1) - g1, E(i,j-1) - e)    gap in a: b_j against '-'   (op D)
 *   F(i,j) = max(H(i-1,j) - g1, F(i-1,j) - e)    gap in b: a_i against '-'   (op I)
 *   H(i,j) = max(H(i-1,j-1) + S(a_i, b_j), F(i,j), E(i,j))                 (op M)
 * Traceback from (p, q) in H.  Ties: H takes the aligned pair first, then F, then E; F and E
 * take opening (from H) before extending.  Output: ops[k] = (run length << 2) | op, op 0 = M,
 * 1 = I, 2 = D, from the start of the alignment to its end.  Returns the number of runs
 * (0 when the score is 0), or -1 if max_ops is too small.  cells as cm_oracle_sw_cells. */
int64_t cm_oracle_sw_align(const uint8_t *a, int64_t m, const uint8_t *b, int64_t n,
                           const int32_t *S, int64_t o, int64_t e, int gap_mode,
                           int64_t *cells, int32_t *ops, int64_t max_ops)
{
    (void)m; (void)n;
    cm_oracle_sw_cells(a, m, b, n, S, o, e, gap_mode, cells);
    if (cells[0] == 0) return 0;
    const int64_t g1 = (gap_mode == 0) ? o : o + e;
    const uint8_t *A = a + cells[1] - 1, *B = b + cells[3] - 1;
    const int64_t p = cells[2] - cells[1] + 1, q = cells[4] - cells[3] + 1;
    const size_t W = (size_t)(q + 1), cnt = (size_t)(p + 1) * W;
    int64_t *H = (int64_t *)malloc(sizeof(int64_t) * cnt);
    int64_t *E = (int64_t *)malloc(sizeof(int64_t) * cnt);
    int64_t *F = (int64_t *)malloc(sizeof(int64_t) * cnt);
    H[0] = 0; E[0] = F[0] = NEG_INF;
    for (int64_t j = 1; j <= q; j++) { H[j] = E[j] = -(g1 + (j - 1) * e); F[j] = NEG_INF; }
    for (int64_t i = 1; i <= p; i++) {
        H[i * W] = F[i * W] = -(g1 + (i - 1) * e);
        E[i * W] = NEG_INF;
        for (int64_t j = 1; j <= q; j++) {
            E[i * W + j] = max64(H[i * W + j - 1] - g1, E[i * W + j - 1] - e);
            F[i * W + j] = max64(H[(i - 1) * W + j] - g1, F[(i - 1) * W + j] - e);
            int64_t h = H[(i - 1) * W + j - 1] + (int64_t)S[A[i - 1] * 24 + B[j - 1]];
            h = max64(h, F[i * W + j]);
            h = max64(h, E[i * W + j]);
            H[i * W + j] = h;
        }
    }
    /* reversed op sequence, one op per column of the alignment */
    int8_t *rev = (int8_t *)malloc((size_t)(p + q));
    int64_t len = 0, i = p, j = q;
    int state = 0;                      /* 0 = H, 1 = F, 2 = E */
    while (i > 0 || j > 0) {
        if (i == 0) { rev[len++] = 2; j--; continue; }
        if (j == 0) { rev[len++] = 1; i--; continue; }
        if (state == 0) {
            if (H[i * W + j] == H[(i - 1) * W + j - 1] + (int64_t)S[A[i - 1] * 24 + B[j - 1]]) {
                rev[len++] = 0; i--; j--;
            } else if (H[i * W + j] == F[i * W + j]) {
                state = 1;
            } else {
                state = 2;
            }
        } else if (state == 1) {
            rev[len++] = 1;
            state = (F[i * W + j] == H[(i - 1) * W + j] - g1) ? 0 : 1;
            i--;
        } else {
            rev[len++] = 2;
            state = (E[i * W + j] == H[i * W + j - 1] - g1) ? 0 : 2;
            j--;
        }
    }
    int64_t nruns = 0;
    for (int64_t k = len - 1; k >= 0; ) {
        int64_t r = 1;
        while (k - r >= 0 && rev[k - r] == rev[k]) r++;
        if (nruns >= max_ops) { nruns = -1; break; }
        ops[nruns++] = (int32_t)((r << 2) | rev[k]);
        k -= r;
    }
    free(H); free(E); free(F); free(rev);
    return nruns;
}

typedef struct {
    const uint8_t *seqs; const int64_t *off; const int32_t *pairs; int64_t npairs;
    const int32_t *S; int64_t o, e; int gap_mode; int64_t *out; int tid, nthreads;
} job_t;

static void *batch_worker(void *p)
{
    job_t *J = (job_t *)p;
    for (int64_t k = J->tid; k < J->npairs; k += J->nthreads) {
        int32_t x = J->pairs[2 * k], y = J->pairs[2 * k + 1];
        J->out[k] = cm_oracle_sw(J->seqs + J->off[x], J->off[x + 1] - J->off[x],
                                 J->seqs + J->off[y], J->off[y + 1] - J->off[y],
                                 J->S, J->o, J->e, J->gap_mode);
    }
    return NULL;
}

/* Scores of pairs (pairs[2k], pairs[2k+1]) = (a, b), nthreads POSIX threads over pairs. */
int cm_oracle_sw_batch(const uint8_t *seqs, const int64_t *off, const int32_t *pairs,
                       int64_t npairs, const int32_t *S, int64_t o, int64_t e, int gap_mode,
                       int64_t *out, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nthreads);
    job_t *jobs = (job_t *)malloc(sizeof(job_t) * (size_t)nthreads);
    for (int t = 0; t < nthreads; t++) {
        job_t J = {seqs, off, pairs, npairs, S, o, e, gap_mode, out, t, nthreads};
        jobs[t] = J;
        pthread_create(&th[t], NULL, batch_worker, &jobs[t]);
    }
    for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
    free(th); free(jobs);
    return 0;
}
