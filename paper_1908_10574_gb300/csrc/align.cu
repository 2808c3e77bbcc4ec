// sw_align_batch: one optimal local alignment per pair as run-length operations, for the
// similar pairs a clustering reports (Sec. 6.1: the pairs are re-aligned for inspection).
//
// The alignment cells (score, start and end cell, csrc/api.cu run_cells) fix the span of the
// alignment: a[i_s..i_e] against b[j_s..j_e].  Inside that rectangle the alignment is the
// global affine (Gotoh) alignment of the two substrings, which scores the local optimum:
//   H(0,0) = 0;  H(0,j) = E(0,j) = -(g1 + (j-1)e);  H(i,0) = F(i,0) = -(g1 + (i-1)e)
//   E(i,j) = max(H(i,j-1) - g1, E(i,j-1) - e)     b_j against a gap      (op D)
//   F(i,j) = max(H(i-1,j) - g1, F(i-1,j) - e)     a_i against a gap      (op I)
//   H(i,j) = max(H(i-1,j-1) + S(a_i, b_j), F(i,j), E(i,j))              (op M)
// The fill keeps one H row and one F row and stores, per cell, which term won (ties: the
// aligned pair, then F, then E; a gap's opening before its extension) in one byte; the
// traceback walks those bytes back from (p, q) and writes the runs.  One thread per pair:
// the work is a few similar pairs per cluster, and each thread's rectangle lives in its own
// slice of a scratch buffer (direction bytes, two int32 rows, the runs), so pairs are cut
// into rounds whose slices fit the scratch budget.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "ctx.h"

namespace cm {
namespace {

struct AlnMatrix {
    int16_t v[kAlpha * kAlpha];
};

struct AlnJob {
    int32_t a, b;        // sequence ids (a: first sequence of the pair)
    int32_t i0, j0;      // 0-based first residue of the span in a and b
    int32_t p, q;        // span lengths
    int32_t score;       // expected global score of the span (the local optimum)
    int32_t pad;
    int64_t dir;         // byte offset of the p x q direction bytes in the scratch
    int64_t rows;        // byte offset of the two (q + 1) int32 rows
    int64_t ops;         // byte offset of the (p + q) int32 runs
};

constexpr int32_t kAlnNeg = -(1 << 29);
constexpr uint8_t kSrcF = 1, kSrcE = 2, kFOpen = 4, kEOpen = 8;

__global__ void __launch_bounds__(128) align_kernel(const uint8_t* __restrict__ db,
                                                    const int64_t* __restrict__ off,
                                                    const AlnJob* __restrict__ jobs,
                                                    int32_t njobs, const AlnMatrix mat_in,
                                                    int32_t g1, int32_t ge,
                                                    uint8_t* __restrict__ scratch,
                                                    int32_t* __restrict__ nops,
                                                    int32_t* __restrict__ err)
{
    __shared__ int16_t mat[kAlpha * kAlpha];
    for (int i = threadIdx.x; i < kAlpha * kAlpha; i += blockDim.x) mat[i] = mat_in.v[i];
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= njobs) return;
    const AlnJob J = jobs[t];
    const uint8_t* A = db + off[J.a] + J.i0;
    const uint8_t* B = db + off[J.b] + J.j0;
    const int p = J.p, q = J.q;
    uint8_t* D = scratch + J.dir;
    int32_t* Hrow = reinterpret_cast<int32_t*>(scratch + J.rows);
    int32_t* Frow = Hrow + (q + 1);
    int32_t* out = reinterpret_cast<int32_t*>(scratch + J.ops);

    Hrow[0] = 0;
    for (int j = 1; j <= q; ++j) {
        Hrow[j] = -(g1 + (j - 1) * ge);
        Frow[j] = kAlnNeg;
    }
    for (int i = 1; i <= p; ++i) {
        const int16_t* srow = mat + A[i - 1] * kAlpha;
        int32_t diag = Hrow[0];                   // H(i-1, 0)
        int32_t hleft = -(g1 + (i - 1) * ge);     // H(i, 0)
        Hrow[0] = hleft;
        int32_t E = kAlnNeg;
        uint8_t* drow = D + (int64_t)(i - 1) * q;
        for (int j = 1; j <= q; ++j) {
            const int32_t hup = Hrow[j];
            const int32_t eo = hleft - g1, ee = E - ge;
            const bool e_open = eo >= ee;
            E = e_open ? eo : ee;
            const int32_t fo = hup - g1, fe = Frow[j] - ge;
            const bool f_open = fo >= fe;
            const int32_t F = f_open ? fo : fe;
            Frow[j] = F;
            const int32_t dg = diag + srow[B[j - 1]];
            int32_t h;
            uint8_t d;
            if (dg >= F && dg >= E) { h = dg; d = 0; }
            else if (F >= E) { h = F; d = kSrcF; }
            else { h = E; d = kSrcE; }
            drow[j - 1] = d | (f_open ? kFOpen : 0) | (e_open ? kEOpen : 0);
            diag = hup;
            Hrow[j] = h;
            hleft = h;
        }
    }
    if (Hrow[q] != J.score) atomicExch(err, 1);   // the span's global score is the optimum
    // traceback: runs from the end, reversed at the end
    int i = p, j = q, state = 0, n = 0, cur = -1, run = 0;
    auto emit = [&](int op) {
        if (op == cur) { ++run; return; }
        if (run) out[n++] = (run << 2) | cur;
        cur = op;
        run = 1;
    };
    while (i > 0 || j > 0) {
        if (i == 0) { emit(2); --j; continue; }
        if (j == 0) { emit(1); --i; continue; }
        const uint8_t d = D[(int64_t)(i - 1) * q + (j - 1)];
        if (state == 0) {
            const int src = d & 3;
            if (src == 0) { emit(0); --i; --j; }
            else state = src;                     // 1: F, 2: E
        } else if (state == 1) {
            emit(1);
            state = (d & kFOpen) ? 0 : 1;
            --i;
        } else {
            emit(2);
            state = (d & kEOpen) ? 0 : 2;
            --j;
        }
    }
    if (run) out[n++] = (run << 2) | cur;
    for (int k = 0; k < n / 2; ++k) {
        const int32_t x = out[k];
        out[k] = out[n - 1 - k];
        out[n - 1 - k] = x;
    }
    nops[t] = n;
}

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

}  // namespace
}  // namespace cm

using namespace cm;

extern "C" int sw_align_batch(cm_ctx* c, const uint8_t* seqs, const int64_t* offsets,
                              int32_t n_seqs, const int32_t* pairs, int64_t n_pairs,
                              const int8_t* matrix, int32_t gap_open, int32_t gap_extend,
                              int32_t* cells_out, int64_t* ops_offsets, int32_t* ops_out,
                              int64_t ops_capacity, int64_t* n_ops, uint32_t flags)
{
    if (!c) return CM_ERR_ARG;
    CUDA_TRY(cudaSetDevice(c->device));
    if (n_pairs < 0 || !n_ops || ops_capacity < 0 ||
        (n_pairs > 0 && (!pairs || !cells_out || !ops_offsets)) || (ops_capacity > 0 && !ops_out))
        return fail(c, CM_ERR_ARG, "bad pairs, outputs or capacity");
    NvtxRange nv("sw_align_batch");
    Prepared P;
    int r = prepare(c, seqs, offsets, n_seqs, matrix, gap_open, gap_extend, flags, P);
    if (r) return r;
    const bool dev = (flags & CM_DEVICE_PTRS) != 0;
    const cudaMemcpyKind out_kind = dev ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
    *n_ops = 0;
    if (n_pairs == 0) {
        const int64_t zero = 0;
        CUDA_TRY(cudaMemcpyAsync(ops_offsets, &zero, 8, out_kind, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        return CM_OK;
    }
    std::vector<int32_t> hp((size_t)n_pairs * 2);
    if (dev) CUDA_TRY(cudaMemcpy(hp.data(), pairs, hp.size() * 4, cudaMemcpyDeviceToHost));
    else std::memcpy(hp.data(), pairs, hp.size() * 4);
    for (int64_t k = 0; k < 2 * n_pairs; ++k)
        if (hp[k] < 0 || hp[k] >= n_seqs) return fail(c, CM_ERR_ARG, "pair index out of range");
    std::vector<int32_t> hc((size_t)n_pairs * 5);
    if ((r = run_cells(c, P, hp.data(), n_pairs, hc.data()))) return r;

    // jobs: pairs with a non-empty alignment, in rounds whose scratch slices fit the budget
    std::vector<AlnJob> jobs;
    std::vector<int64_t> job_pair;
    for (int64_t k = 0; k < n_pairs; ++k) {
        const int32_t* cl = &hc[5 * k];
        if (cl[0] == 0) continue;
        AlnJob J{};
        J.a = hp[2 * k];
        J.b = hp[2 * k + 1];
        J.i0 = cl[1] - 1;
        J.j0 = cl[3] - 1;
        J.p = cl[2] - cl[1] + 1;
        J.q = cl[4] - cl[3] + 1;
        J.score = cl[0];
        jobs.push_back(J);
        job_pair.push_back(k);
    }
    const int64_t budget = (int64_t)1 << 30;
    std::vector<int32_t> counts(jobs.size(), 0);
    std::vector<std::vector<int32_t>> runs(jobs.size());
    size_t j0 = 0;
    int64_t rounds = 0;
    while (j0 < jobs.size()) {
        size_t j1 = j0;
        int64_t bytes = 0;
        while (j1 < jobs.size()) {
            AlnJob& J = jobs[j1];
            const int64_t need = round_up((int64_t)J.p * J.q, 16) + round_up(8 * ((int64_t)J.q + 1), 16) +
                                 round_up(4 * ((int64_t)J.p + J.q), 16);
            if (j1 > j0 && bytes + need > budget) break;
            J.dir = bytes;
            J.rows = J.dir + round_up((int64_t)J.p * J.q, 16);
            J.ops = J.rows + round_up(8 * ((int64_t)J.q + 1), 16);
            bytes += need;
            ++j1;
        }
        const int32_t nj = (int32_t)(j1 - j0);
        uint8_t* d_scr;
        AlnJob* d_jobs;
        int32_t* d_cnt;
        ENSURE(B_SCRATCH, (size_t)bytes, d_scr);
        ENSURE(B_JOBS, (size_t)nj, d_jobs);
        ENSURE(B_FLAGS, kFlagWords + (size_t)nj, d_cnt);
        if ((r = copy_in(c, d_jobs, jobs.data() + j0, (size_t)nj * sizeof(AlnJob), false))) return r;
        CUDA_TRY(cudaMemsetAsync(d_cnt, 0, sizeof(int32_t) * 8, c->stream));
        AlnMatrix M;
        std::memcpy(M.v, P.mat, sizeof(M.v));
        align_kernel<<<(unsigned)((nj + 127) / 128), 128, 0, c->stream>>>(
            P.db, P.off, d_jobs, nj, M, P.g1, P.ge, d_scr, d_cnt + 8, d_cnt + 1);
        CUDA_TRY(cudaGetLastError());
        c->stats.launches += 1;
        int32_t kerr = 0;
        CUDA_TRY(cudaMemcpyAsync(&kerr, d_cnt + 1, 4, cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaMemcpyAsync(counts.data() + j0, d_cnt + 8, (size_t)nj * 4,
                                 cudaMemcpyDeviceToHost, c->stream));
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        if (kerr) return fail(c, CM_ERR_INTERNAL, "alignment span does not reach the local optimum");
        for (size_t t = j0; t < j1; ++t) {
            runs[t].resize((size_t)counts[t]);
            if (counts[t])
                CUDA_TRY(cudaMemcpyAsync(runs[t].data(), d_scr + jobs[t].ops, (size_t)counts[t] * 4,
                                         cudaMemcpyDeviceToHost, c->stream));
        }
        CUDA_TRY(cudaStreamSynchronize(c->stream));
        j0 = j1;
        ++rounds;
    }
    // offsets per pair (pairs without an alignment have no runs)
    std::vector<int64_t> hoff((size_t)n_pairs + 1, 0);
    std::vector<int32_t> per_pair((size_t)n_pairs, 0);
    for (size_t t = 0; t < jobs.size(); ++t) per_pair[job_pair[t]] = counts[t];
    for (int64_t k = 0; k < n_pairs; ++k) hoff[k + 1] = hoff[k] + per_pair[k];
    *n_ops = hoff[n_pairs];
    if (hoff[n_pairs] > ops_capacity)
        return fail(c, CM_ERR_CAPACITY, "ops_capacity too small; *n_ops holds the needed size");
    std::vector<int32_t> flat((size_t)hoff[n_pairs]);
    for (size_t t = 0; t < jobs.size(); ++t)
        std::copy(runs[t].begin(), runs[t].end(), flat.begin() + hoff[job_pair[t]]);
    CUDA_TRY(cudaMemcpyAsync(cells_out, hc.data(), hc.size() * 4, out_kind, c->stream));
    CUDA_TRY(cudaMemcpyAsync(ops_offsets, hoff.data(), hoff.size() * 8, out_kind, c->stream));
    if (!flat.empty())
        CUDA_TRY(cudaMemcpyAsync(ops_out, flat.data(), flat.size() * 4, out_kind, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return CM_OK;
}
