// sw_cells_batch_noalloc: an allocation-free variant of sw_cells_batch.
//
// Who needs it: callers that cannot allocate device memory at call time.  Examples are a
// service whose GPU memory was reserved up front by another framework's caching allocator
// (a fresh cudaMalloc would fail or fragment that pool), and a latency-bound loop that must
// not pay the device-wide synchronisation cudaMalloc / cudaFree can cause.  Such callers
// pass device inputs and outputs; the per-pair DP rows live in one fixed array compiled into
// this library instead of a context's grow-on-demand buffers.
//
// The scratch below is a file-scope __device__ array.  In host code its name is only a
// host-side stand-in, never a device address, so every call looks up the real address with
// cudaGetSymbolAddress (with the caller's device current) and passes that pointer to the
// kernels.  The address is not cached: after a cudaDeviceReset the module is loaded again and
// the array may move, and a lookup allocates nothing.  Every GPU that loads the library holds
// the array until the process exits.  All calls on a device share it, so two calls whose work
// overlaps on the GPU race; the array keeps the last call's contents, and the status words at
// its end are cleared at the start of every call.
#include <algorithm>
#include <cstdio>
#include <cstring>

#include "cm_internal.h"

namespace {

constexpr int kNaThreads = 1024;                 // pairs in flight (one thread each)
constexpr int kNaCols = 4096;                    // DP row length: second sequence <= 4095
constexpr size_t kNaRowWords = 2ull * kNaThreads * kNaCols;   // H and F rows: 32 MiB
constexpr size_t kNaStatusWords = 64;            // status words after the rows
constexpr int32_t kNaNeg = -(1 << 28);

static __device__ __align__(256) int32_t g_na_scratch[kNaRowWords + kNaStatusWords];

struct NaMatrix {
    int16_t v[400];
};

void na_message(char* buf, int32_t len, const char* msg)
{
    if (buf && len > 0) {
        std::strncpy(buf, msg, (size_t)len - 1);
        buf[len - 1] = '\0';
    }
}

// status[0]: pair index out of range or bad offsets; status[1]: second sequence too long;
// status[2]: residue code >= 20
__global__ void na_check_kernel(const uint8_t* __restrict__ seqs, const int64_t* __restrict__ off,
                                int32_t n_seqs, const int32_t* __restrict__ pairs, int64_t npairs,
                                int32_t* status)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npairs;
         p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t x = pairs[2 * p], y = pairs[2 * p + 1];
        if (x < 0 || x >= n_seqs || y < 0 || y >= n_seqs) { atomicExch(status + 0, 1); continue; }
        const int64_t xb = off[x], xe = off[x + 1], yb = off[y], ye = off[y + 1];
        if (xb < 0 || xe < xb || yb < 0 || ye < yb) { atomicExch(status + 0, 1); continue; }
        if (ye - yb > kNaCols - 1) { atomicExch(status + 1, 1); continue; }
        for (int64_t i = xb; i < xe; ++i)
            if (seqs[i] >= 20) { atomicExch(status + 2, 1); break; }
        for (int64_t i = yb; i < ye; ++i)
            if (seqs[i] >= 20) { atomicExch(status + 2, 1); break; }
    }
}

__device__ int32_t na_gotoh(const uint8_t* a, int64_t m, const uint8_t* b, int64_t n, bool rev,
                            const int16_t* mat, int32_t g1, int32_t ge, int32_t* H, int32_t* F,
                            int32_t* bi, int32_t* bj)
{
    for (int64_t j = 0; j <= n; ++j) { H[j * kNaThreads] = 0; F[j * kNaThreads] = kNaNeg; }
    int32_t best = 0, ii = 0, jj = 0;
    for (int64_t i = 1; i <= m; ++i) {
        const int16_t* row = mat + (rev ? a[m - i] : a[i - 1]) * 20;
        int32_t E = kNaNeg, hleft = 0, hdiag = 0;
        for (int64_t j = 1; j <= n; ++j) {
            const int32_t hup = H[j * kNaThreads];
            E = max(E - ge, hleft - g1);
            const int32_t f = max(F[j * kNaThreads] - ge, hup - g1);
            F[j * kNaThreads] = f;
            const int32_t h = max(max(hdiag + row[rev ? b[n - j] : b[j - 1]], 0), max(E, f));
            hdiag = hup;
            H[j * kNaThreads] = h;
            hleft = h;
            if (h > best) { best = h; ii = (int32_t)i; jj = (int32_t)j; }
        }
    }
    *bi = ii;
    *bj = jj;
    return best;
}

// one thread per pair; thread t keeps its H and F rows in columns t of the scratch rows
__global__ void __launch_bounds__(128) na_cells_kernel(const uint8_t* __restrict__ seqs,
                                                     const int64_t* __restrict__ off,
                                                     const int32_t* __restrict__ pairs,
                                                     int64_t npairs, const NaMatrix mat_in,
                                                     int32_t g1, int32_t ge,
                                                     int32_t* __restrict__ cells,
                                                     int32_t* scratch)
{
    __shared__ int16_t mat[400];
    for (int i = threadIdx.x; i < 400; i += blockDim.x) mat[i] = mat_in.v[i];
    __syncthreads();
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= kNaThreads) return;
    int32_t* H = scratch + t;
    int32_t* F = scratch + (size_t)kNaThreads * kNaCols + t;
    for (int64_t p = t; p < npairs; p += kNaThreads) {
        const int32_t x = pairs[2 * p], y = pairs[2 * p + 1];
        const uint8_t* a = seqs + off[x];
        const uint8_t* b = seqs + off[y];
        const int64_t m = off[x + 1] - off[x], n = off[y + 1] - off[y];
        int32_t* c = cells + 5 * p;
        int32_t ie, je, ri, rj;
        const int32_t best = na_gotoh(a, m, b, n, false, mat, g1, ge, H, F, &ie, &je);
        c[0] = best;
        if (best == 0) { c[1] = c[2] = c[3] = c[4] = 0; continue; }
        na_gotoh(a, ie, b, je, true, mat, g1, ge, H, F, &ri, &rj);
        c[1] = ie - ri + 1;
        c[2] = ie;
        c[3] = je - rj + 1;
        c[4] = je;
    }
}

}  // namespace

extern "C" int sw_cells_batch_noalloc(const uint8_t* seqs, const int64_t* offsets,
                                      int32_t n_seqs, const int32_t* pairs, int64_t n_pairs,
                                      const int8_t* matrix, int32_t gap_open,
                                      int32_t gap_extend, int32_t* cells_out, void* cuda_stream,
                                      uint32_t flags, char* err_msg, int32_t err_len)
{
    na_message(err_msg, err_len, "");
    if (flags & ~(uint32_t)CM_GAP_BLAST) {
        na_message(err_msg, err_len, "only CM_GAP_BLAST is accepted (inputs are device pointers)");
        return CM_ERR_ARG;
    }
    if (n_seqs < 0 || n_pairs < 0 || n_pairs >= ((int64_t)1 << 31) || !offsets || !matrix ||
        (n_pairs > 0 && (!seqs || !pairs || !cells_out))) {
        na_message(err_msg, err_len, "null pointer or size out of range (n_pairs < 2^31)");
        return CM_ERR_ARG;
    }
    const int64_t g1 = (flags & CM_GAP_BLAST) ? (int64_t)gap_open + gap_extend : gap_open;
    if (g1 < 1 || g1 > 1000 || gap_extend < 0 || gap_extend > g1) {
        na_message(err_msg, err_len, "gap costs must satisfy 1 <= first-gap cost <= 1000 and "
                                     "0 <= gap_extend <= first-gap cost");
        return CM_ERR_ARG;
    }
    NaMatrix M;
    for (int i = 0; i < 400; ++i) {
        if (matrix[i] < -1000 || matrix[i] > 1000) {
            na_message(err_msg, err_len, "matrix entries must lie in [-1000, 1000]");
            return CM_ERR_ARG;
        }
        M.v[i] = matrix[i];
    }
    if (n_pairs == 0) return CM_OK;

    // the array's device address on the current device, looked up on every call
    int32_t* scratch = nullptr;
    {
        void* p = nullptr;
        const cudaError_t le = cudaGetSymbolAddress(&p, g_na_scratch);
        if (le != cudaSuccess || !p) {
            cudaGetLastError();
            na_message(err_msg, err_len, "cudaGetSymbolAddress of the scratch array failed "
                                         "(no usable current CUDA device?)");
            return CM_ERR_CUDA;
        }
        scratch = static_cast<int32_t*>(p);
    }
    int32_t* status = scratch + kNaRowWords;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);

    cudaError_t e = cudaMemsetAsync(status, 0, kNaStatusWords * sizeof(int32_t), st);
    if (e == cudaSuccess) {
        const int64_t blocks = std::min<int64_t>((n_pairs + 255) / 256, 4096);
        na_check_kernel<<<(unsigned)blocks, 256, 0, st>>>(seqs, offsets, n_seqs, pairs, n_pairs,
                                                           status);
        e = cudaGetLastError();
    }
    int32_t hs[3] = {0, 0, 0};
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs, status, sizeof(hs), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        na_message(err_msg, err_len, cudaGetErrorString(e));
        return CM_ERR_CUDA;
    }
    if (hs[0]) {
        na_message(err_msg, err_len, "pair index out of range or offsets not non-decreasing");
        return CM_ERR_ARG;
    }
    if (hs[1]) {
        na_message(err_msg, err_len, "a pair's second sequence is longer than 4095 residues, "
                                     "the fixed scratch limit of this entry point");
        return CM_ERR_ARG;
    }
    if (hs[2]) {
        na_message(err_msg, err_len, "residue code >= 20 in a paired sequence");
        return CM_ERR_RESIDUE;
    }
    na_cells_kernel<<<kNaThreads / 128, 128, 0, st>>>(seqs, offsets, pairs, n_pairs, M,
                                                      (int32_t)g1, gap_extend, cells_out,
                                                      scratch);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        na_message(err_msg, err_len, cudaGetErrorString(e));
        return CM_ERR_CUDA;
    }
    return CM_OK;
}
