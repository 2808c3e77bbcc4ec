// Score plus the cells of one optimal local alignment per pair: the extent the protein
// transitivity test needs (Sec. 4: uncovered residues uA, uD of the two representatives).
// One thread per pair, int32, plain row-by-row Gotoh recurrence with the previous row kept in
// a column-interleaved global scratch (coalesced across the threads of a warp).  Only the
// candidate representative pairs whose score exceeds the full-merge threshold come here.
#include "cm_internal.h"

namespace cm {

namespace {

constexpr int32_t kNeg = -(1 << 28);

// Forward recurrence over a[0..m) x b[0..n) (optionally both reversed).  Returns the best
// score and the first row-major cell (1-based) that reaches it.
__device__ int32_t gotoh_cells(const uint8_t* a, int64_t m, const uint8_t* b, int64_t n,
                               bool rev, const int16_t* mat, int32_t g1, int32_t ge,
                               int32_t* H, int32_t* F, int64_t stride, int32_t* bi,
                               int32_t* bj)
{
    for (int64_t j = 0; j <= n; ++j) { H[j * stride] = 0; F[j * stride] = kNeg; }
    int32_t best = 0, ii = 0, jj = 0;
    for (int64_t i = 1; i <= m; ++i) {
        const int ai = rev ? a[m - i] : a[i - 1];
        const int16_t* row = mat + ai * 20;
        int32_t E = kNeg, hleft = 0, hdiag = 0;
        for (int64_t j = 1; j <= n; ++j) {
            const int32_t hup = H[j * stride];
            E = max(E - ge, hleft - g1);
            const int32_t f = max(F[j * stride] - ge, hup - g1);
            F[j * stride] = f;
            const int bj_res = rev ? b[n - j] : b[j - 1];
            int32_t h = max(max(hdiag + row[bj_res], 0), max(E, f));
            hdiag = hup;
            H[j * stride] = h;
            hleft = h;
            if (h > best) { best = h; ii = (int32_t)i; jj = (int32_t)j; }
        }
    }
    *bi = ii;
    *bj = jj;
    return best;
}

__global__ void cells_kernel(const uint8_t* __restrict__ db, const int64_t* __restrict__ off,
                             const int32_t* __restrict__ pairs, int64_t npairs,
                             const int16_t* __restrict__ gmat, int32_t g1, int32_t ge,
                             int32_t* __restrict__ cells, int32_t* scratch, int64_t cols,
                             int32_t nthreads)
{
    __shared__ int16_t mat[400];
    for (int i = threadIdx.x; i < 400; i += blockDim.x) mat[i] = gmat[i];
    __syncthreads();
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (tid >= nthreads) return;
    int32_t* H = scratch + tid;
    int32_t* F = scratch + (int64_t)nthreads * cols + tid;
    for (int64_t p = tid; p < npairs; p += nthreads) {
        const int32_t x = pairs[2 * p], y = pairs[2 * p + 1];
        const uint8_t* a = db + off[x];
        const uint8_t* b = db + off[y];
        const int64_t m = off[x + 1] - off[x], n = off[y + 1] - off[y];
        int32_t* c = cells + 5 * p;
        if (n + 1 > cols) {               // scratch too short: report, never overrun
            c[0] = -1; c[1] = c[2] = c[3] = c[4] = 0;
            continue;
        }
        int32_t ie, je, ri, rj;
        const int32_t best = gotoh_cells(a, m, b, n, false, mat, g1, ge, H, F, nthreads, &ie, &je);
        c[0] = best;
        if (best == 0) { c[1] = c[2] = c[3] = c[4] = 0; continue; }
        gotoh_cells(a, ie, b, je, true, mat, g1, ge, H, F, nthreads, &ri, &rj);
        c[1] = ie - ri + 1;
        c[2] = ie;
        c[3] = je - rj + 1;
        c[4] = je;
    }
}

}  // namespace

cudaError_t launch_cells(const uint8_t* db, const int64_t* off, const int32_t* pairs,
                         int64_t npairs, const int16_t* mat, int32_t g1, int32_t ge,
                         int32_t* cells_out, int32_t* scratch, int64_t scratch_cols,
                         int32_t nthreads, cudaStream_t st)
{
    if (npairs == 0) return cudaSuccess;
    const int threads = 128;
    const int grid = (nthreads + threads - 1) / threads;
    cells_kernel<<<grid, threads, 0, st>>>(db, off, pairs, npairs, mat, g1, ge, cells_out,
                                           scratch, scratch_cols, nthreads);
    return cudaGetLastError();
}

}  // namespace cm
