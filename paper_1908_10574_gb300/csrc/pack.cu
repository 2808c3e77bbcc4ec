// Packing (residue validation, per-block row streams), saturated-pair collection and
// threshold compaction of significant pairs f > T (Sec. 3).
#include "cm_internal.h"

namespace cm {

namespace {

__device__ __forceinline__ int64_t tri(int64_t k) { return k * (k - 1) / 2; }

// k with tri(k) <= v < tri(k+1)
__device__ __forceinline__ int64_t tri_row(int64_t v)
{
    int64_t k = (int64_t)((1.0 + sqrt(1.0 + 8.0 * (double)v)) * 0.5);
    while (tri(k) > v) --k;
    while (tri(k + 1) <= v) ++k;
    return k;
}

__global__ void ascii_kernel(const uint8_t* __restrict__ in, uint8_t* __restrict__ out,
                             int64_t n, int32_t alpha, int32_t* bad)
{
    // ARNDCQEGHILKMFPSTWYV -> 0..19 (and with alpha 24: B, Z, X, * -> 20..23), letters
    // case-insensitive; anything else flags `bad`
    __shared__ uint8_t lut[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) lut[i] = 255;
    __syncthreads();
    if (threadIdx.x < alpha) {
        const char* A = "ARNDCQEGHILKMFPSTWYVBZX*";
        const uint8_t ch = (uint8_t)A[threadIdx.x];
        lut[ch] = (uint8_t)threadIdx.x;
        if (ch >= 'A' && ch <= 'Z') lut[ch + 32] = (uint8_t)threadIdx.x;
    }
    __syncthreads();
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t c = lut[in[i]];
        if (c == 255) atomicExch(bad, 1);
        out[i] = (c == 255) ? 0 : c;
    }
}

__global__ void check_kernel(const uint8_t* __restrict__ in, int64_t n, int32_t alpha,
                             int32_t* bad)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (in[i] >= alpha) atomicExch(bad, 1);
}

// one warp per subject: copy its residues into the block stream with first/last flags
__global__ void gather_kernel(const uint8_t* __restrict__ db, const int64_t* __restrict__ off,
                              const int32_t* __restrict__ ids, int32_t nb,
                              const int64_t* __restrict__ srow, uint8_t* __restrict__ stream)
{
    const int lane = threadIdx.x & 31;
    for (int64_t s = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; s < nb;
         s += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int32_t id = ids[s];
        const int64_t b = off[id], len = off[id + 1] - b;
        uint8_t* dst = stream + srow[s];
        const int64_t rows = srow[s + 1] - srow[s];        // len rounded up to the row group
        for (int64_t r = lane; r < rows; r += 32) {
            // codes above kPadCode never reach a stream (the SW kernels index profile rows
            // by the low five bits without a clamp); validated input has none anyway
            uint8_t v = (r < len) ? (uint8_t)min((int)db[b + r], (int)kPadCode) : kPadCode;
            if (r == 0) v |= kFirst;
            if (r == (len > 0 ? len - 1 : 0)) v |= kLast;
            dst[r] = v;
        }
    }
}

__global__ void collect_kernel(const int32_t* __restrict__ out, int64_t nslots,
                               const SwBlock* __restrict__ blocks, int32_t nblocks,
                               const int64_t* __restrict__ first_slot,
                               const int32_t* __restrict__ ids,
                               const int64_t* __restrict__ out_map, PairRef* list,
                               int32_t* count, int32_t cap)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nslots;
         i += (int64_t)gridDim.x * blockDim.x) {
        // block containing slot i (first_slot ascending, first_slot[0] == 0)
        int32_t lo = 0, hi = nblocks - 1;
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (first_slot[mid] <= i) lo = mid; else hi = mid - 1;
        }
        const SwBlock B = blocks[lo];
        const int64_t v = i - B.out_base;
        int64_t k, s;
        if (B.kind == kTri) {
            k = tri_row(v + tri(B.k0));
            s = v + tri(B.k0) - tri(k);
        } else {
            k = B.k0 + v / B.nb;
            s = v % B.nb;
        }
        const int64_t slot = B.has_map ? out_map[i] : i;
        if (out[slot] != kSat) continue;
        const int32_t c = atomicAdd(count, 1);
        if (c < cap) {
            PairRef p;
            p.q = ids[B.a_ids + k];
            p.x = ids[B.b_ids + s];
            p.swap = B.swap;
            p.pad = 0;
            p.slot = slot;
            list[c] = p;
        }
    }
}

// Deterministic compaction of the slots [0, nslots) whose score exceeds T, in slot order.
// TRI: the slots are the pairs (k, s), s < k, of the length order `order`, numbered
// tri(k) - tri(k0) + s, written as (min, max) sequence ids to pairs_out.  Otherwise the slot
// index itself goes to slots_out.  Chunk = 256 threads x 32 slots; phase 0 counts per chunk,
// phase 1 (after an exclusive scan of the counts) writes.
constexpr int kCT = 256, kPer = 32, kChunk = kCT * kPer;

template <bool TRI>
__global__ void compact_kernel(const int32_t* __restrict__ out, int64_t nslots, int32_t k0,
                               const int32_t* __restrict__ order, int32_t T,
                               int32_t* __restrict__ pairs_out, int64_t* __restrict__ slots_out,
                               int32_t* __restrict__ scores_out, int64_t* chunk_counts, int phase)
{
    __shared__ int64_t s_warp[kCT / 32];
    const int64_t base = (int64_t)blockIdx.x * kChunk + (int64_t)threadIdx.x * kPer;
    int64_t c = 0;
    for (int u = 0; u < kPer; ++u) {
        const int64_t i = base + u;
        if (i < nslots && out[i] > T) ++c;
    }
    // block exclusive scan of c
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t incl = c;
    for (int d = 1; d < 32; d <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    int64_t wbase = 0, total = 0;
    for (int w = 0; w < kCT / 32; ++w) {
        if (w < warp) wbase += s_warp[w];
        total += s_warp[w];
    }
    if (phase == 0) {
        if (threadIdx.x == 0) chunk_counts[blockIdx.x] = total;
        return;
    }
    int64_t pos = chunk_counts[blockIdx.x] + wbase + incl - c;   // chunk_counts now exclusive
    if (c == 0) return;
    const int64_t t0 = TRI ? tri(k0) : 0;
    for (int u = 0; u < kPer; ++u) {
        const int64_t i = base + u;
        if (i < nslots && out[i] > T) {
            if (TRI) {
                const int64_t k = tri_row(i + t0);
                const int64_t s = i + t0 - tri(k);
                const int32_t a = order[k], b = order[s];
                pairs_out[2 * pos] = min(a, b);
                pairs_out[2 * pos + 1] = max(a, b);
            } else {
                slots_out[pos] = i;
            }
            scores_out[pos] = out[i];
            ++pos;
        }
    }
}

__global__ void scan_kernel(int64_t* counts, int64_t n, int64_t* total)
{
    // single block, sequential chunks of the block size
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b = 0; b < n; b += blockDim.x) {
        const int64_t i = b + threadIdx.x;
        const int64_t v = (i < n) ? counts[i] : 0;
        // inclusive scan over the block
        __shared__ int64_t buf[1024];
        buf[threadIdx.x] = v;
        __syncthreads();
        for (int d = 1; d < (int)blockDim.x; d <<= 1) {
            const int64_t y = (threadIdx.x >= (unsigned)d) ? buf[threadIdx.x - d] : 0;
            __syncthreads();
            buf[threadIdx.x] += y;
            __syncthreads();
        }
        if (i < n) counts[i] = carry + buf[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += buf[threadIdx.x];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

// ---- ranked subject lists: one warp per list, 32 bitmap words per iteration, bit order ----
__device__ __forceinline__ uint32_t kept_word(const KeptList& L, const uint32_t* bits, int64_t w)
{
    const uint32_t a = bits[L.row_a + w];
    if (L.op == kKeepA) return a;
    const uint32_t b = bits[L.row_b + w];
    return L.op == kKeepAnd ? (a & b) : L.op == kKeepAOnly ? (a & ~b) : (b & ~a);
}

__device__ __forceinline__ int64_t rows_of(int64_t len)
{
    return len <= 0 ? kRowGroup : (len + kRowGroup - 1) / kRowGroup * kRowGroup;
}

__global__ void kept_totals_kernel(const KeptList* __restrict__ lists, int32_t nlists,
                                   const uint32_t* __restrict__ bits,
                                   const int32_t* __restrict__ reps,
                                   const int64_t* __restrict__ off, int64_t* __restrict__ totals)
{
    const int lane = threadIdx.x & 31;
    const int64_t l = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (l >= nlists) return;
    const KeptList L = lists[l];
    int64_t rows = 0, res = 0;
    for (int64_t w = lane; w < L.words; w += 32) {
        for (uint32_t x = kept_word(L, bits, w); x; x &= x - 1) {
            const int32_t id = reps[L.b0 + w * 32 + __ffs(x) - 1];
            const int64_t len = off[id + 1] - off[id];
            rows += rows_of(len);
            res += len;
        }
    }
    for (int d = 16; d > 0; d >>= 1) {
        rows += __shfl_xor_sync(0xffffffffu, rows, d);
        res += __shfl_xor_sync(0xffffffffu, res, d);
    }
    if (lane == 0) { totals[2 * l] = rows; totals[2 * l + 1] = res; }
}

__global__ void kept_expand_kernel(const KeptList* __restrict__ lists, int32_t nlists,
                                   const uint32_t* __restrict__ bits,
                                   const int32_t* __restrict__ reps,
                                   const int64_t* __restrict__ off, int32_t* __restrict__ ids,
                                   int64_t* __restrict__ srow)
{
    const int lane = threadIdx.x & 31;
    const int64_t l = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (l >= nlists) return;
    const KeptList L = lists[l];
    int64_t g = L.g0, row = L.rowbase;          // next subject index and its first row
    for (int64_t w0 = 0; w0 < L.words; w0 += 32) {
        const int64_t w = w0 + lane;
        const uint32_t x0 = (w < L.words) ? kept_word(L, bits, w) : 0u;
        // rows of this lane's selected subjects, then an exclusive scan over the lanes
        int64_t myrows = 0;
        for (uint32_t x = x0; x; x &= x - 1) {
            const int32_t id = reps[L.b0 + w * 32 + __ffs(x) - 1];
            myrows += rows_of(off[id + 1] - off[id]);
        }
        int32_t cnt = __popc(x0);
        int64_t rincl = myrows;
        int32_t cincl = cnt;
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t ry = __shfl_up_sync(0xffffffffu, rincl, d);
            const int32_t cy = __shfl_up_sync(0xffffffffu, cincl, d);
            if (lane >= d) { rincl += ry; cincl += cy; }
        }
        int64_t gi = g + cincl - cnt, ri = row + rincl - myrows;
        for (uint32_t x = x0; x; x &= x - 1) {
            const int32_t id = reps[L.b0 + w * 32 + __ffs(x) - 1];
            ri += rows_of(off[id + 1] - off[id]);
            ids[gi] = id;
            srow[gi + 1] = ri;
            ++gi;
        }
        g += __shfl_sync(0xffffffffu, cincl, 31);
        row += __shfl_sync(0xffffffffu, rincl, 31);
    }
}

int grid_for(int64_t n, int threads)
{
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > 65535) g = 65535;
    return (int)g;
}

}  // namespace

cudaError_t launch_ascii_to_codes(const uint8_t* in, uint8_t* out, int64_t n, int32_t alpha,
                                  int32_t* bad, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    ascii_kernel<<<grid_for(n, 256), 256, 0, st>>>(in, out, n, alpha, bad);
    return cudaGetLastError();
}

cudaError_t launch_check_codes(const uint8_t* in, int64_t n, int32_t alpha, int32_t* bad,
                               cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    check_kernel<<<grid_for(n, 256), 256, 0, st>>>(in, n, alpha, bad);
    return cudaGetLastError();
}

cudaError_t launch_gather_stream(const uint8_t* db, const int64_t* off, const int32_t* ids,
                                 int32_t nb, const int64_t* srow, uint8_t* stream,
                                 cudaStream_t st)
{
    if (nb == 0) return cudaSuccess;
    gather_kernel<<<grid_for((int64_t)nb * 32, 256), 256, 0, st>>>(db, off, ids, nb, srow,
                                                                     stream);
    return cudaGetLastError();
}

cudaError_t launch_collect_saturated(const int32_t* out, int64_t nslots, const SwBlock* blocks,
                                     int32_t nblocks, const int64_t* first_slot,
                                     const int32_t* ids, const int64_t* out_map,
                                     PairRef* list, int32_t* count, int32_t cap,
                                     cudaStream_t st)
{
    if (nslots == 0) return cudaSuccess;
    collect_kernel<<<grid_for(nslots, 256), 256, 0, st>>>(out, nslots, blocks, nblocks,
                                                           first_slot, ids, out_map, list,
                                                           count, cap);
    return cudaGetLastError();
}

cudaError_t launch_compact_tri(const int32_t* out, int64_t nslots, int32_t k0,
                               const int32_t* order, int32_t T, int32_t* pairs_out,
                               int32_t* scores_out, int64_t* chunk_counts, int64_t nchunks,
                               int phase, cudaStream_t st)
{
    if (nchunks == 0) return cudaSuccess;
    compact_kernel<true><<<(unsigned)nchunks, kCT, 0, st>>>(out, nslots, k0, order, T, pairs_out,
                                                            nullptr, scores_out, chunk_counts,
                                                            phase);
    return cudaGetLastError();
}

cudaError_t launch_compact_slots(const int32_t* out, int64_t nslots, int32_t T,
                                 int64_t* slots_out, int32_t* scores_out, int64_t* chunk_counts,
                                 int64_t nchunks, int phase, cudaStream_t st)
{
    if (nchunks == 0) return cudaSuccess;
    compact_kernel<false><<<(unsigned)nchunks, kCT, 0, st>>>(out, nslots, 0, nullptr, T, nullptr,
                                                             slots_out, scores_out, chunk_counts,
                                                             phase);
    return cudaGetLastError();
}

cudaError_t launch_scan_chunks(int64_t* counts, int64_t nchunks, int64_t* total,
                               cudaStream_t st)
{
    scan_kernel<<<1, 1024, 0, st>>>(counts, nchunks, total);
    return cudaGetLastError();
}

int64_t compact_chunks(int64_t nslots) { return (nslots + kChunk - 1) / kChunk; }

cudaError_t launch_kept_totals(const KeptList* lists, int32_t nlists, const uint32_t* bits,
                               const int32_t* reps, const int64_t* off, int64_t* totals,
                               cudaStream_t st)
{
    if (nlists == 0) return cudaSuccess;
    kept_totals_kernel<<<(unsigned)(((int64_t)nlists * 32 + 255) / 256), 256, 0, st>>>(
        lists, nlists, bits, reps, off, totals);
    return cudaGetLastError();
}

cudaError_t launch_kept_expand(const KeptList* lists, int32_t nlists, const uint32_t* bits,
                               const int32_t* reps, const int64_t* off, int32_t* ids,
                               int64_t* srow, cudaStream_t st)
{
    if (nlists == 0) return cudaSuccess;
    kept_expand_kernel<<<(unsigned)(((int64_t)nlists * 32 + 255) / 256), 256, 0, st>>>(
        lists, nlists, bits, reps, off, ids, srow);
    return cudaGetLastError();
}

}  // namespace cm
