// Long pairs on a whole CTA: the int32 rescoring and the alignment-cells pass of pairs whose
// query spans many column passes (tandem repeats of 10,000-35,000 residues).  One warp per
// pair would run the passes one after another; here the CTA's LW warps run them as a
// pipeline: warp w takes passes w, w + LW, w + 2 LW, ...; pass p reads the boundary column
// (H - o and E of its left neighbour column for every row) that pass p - 1 writes, trailing it
// by at least 32 row groups (the wavefront of dp32.cuh: four rows per step).  The boundary of
// pass p lives in global slot (p mod LW) of the CTA; a warp publishes how many rows of its
// current pass are written in shared memory (tagged with the pass), after a block fence.
// Waits only point from pass p to pass p - 1 (never backwards), and the warps of a CTA are
// co-resident, so the pipeline always advances; every wait is still bounded
// (SwArgs::wait_limit polls of ~100 ns) and sets the error flag (2) when it gives up.  Slot
// p mod LW is rewritten by pass p + LW, which trails its reader (pass p + 1) by at least
// 32 (LW - 1) row groups through the chain of waits, so a row is never overwritten before it
// has been read.
#include "sw16_kernel.cuh"

namespace cm {
namespace {

constexpr int kLW = 8;                 // warps per CTA (passes in flight)
constexpr int kLR = 8;                 // columns per lane: 256-column passes

// the job in a form common to both uses: rows stream sequence `ra` (m residues), the columns
// hold `cb` (n residues); either may be read back to front (cells reverse pass)
struct LongJob {
    const uint8_t* ra;
    const uint8_t* cb;
    int64_t m, n;
    int32_t reverse;
    int32_t swap;            // 0: score S[col residue][row residue]; 1: S[row][col] (int32 rerun)
};

template <bool CELLS>
__global__ void __launch_bounds__(kLW * 32, 1)
long_pair_kernel(const __grid_constant__ SwArgs a, const PairRef* __restrict__ pr,
                 const CellJob* __restrict__ jobs, int32_t njobs, int32_t* counter,
                 int32_t* __restrict__ res)
{
    using G = Geo<kLR>;
    constexpr int LS = kLR;                                   // dense rows: 2-way conflicts only
    constexpr int ROWW = 32 * LS;
    extern __shared__ __align__(16) uint8_t smem[];
    __shared__ int16_t s_mat[kAlpha * kAlpha];
    __shared__ volatile int32_t s_pass[kLW];                 // pass whose boundary is in slot w
    __shared__ volatile int32_t s_prog[kLW];                 // rows of it written so far
    __shared__ int s_job;
    __shared__ int32_t s_best[kLW], s_row[kLW], s_col[kLW];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int32_t* prof = reinterpret_cast<int32_t*>(smem) + (size_t)warp * kProfRows * ROWW;
    uint8_t* qres = smem + (size_t)kLW * kProfRows * ROWW * 4 + (size_t)warp * G::COLS;
    for (int i = tid; i < kAlpha * kAlpha; i += kLW * 32) s_mat[i] = a.mat[i];
    const int o = a.gap_open, ge = a.gap_extend;
    int2* slots = reinterpret_cast<int2*>(a.bnd + (int64_t)blockIdx.x * kLW * a.bnd_stride);

    for (;;) {
        __syncthreads();
        if (tid == 0) s_job = *reinterpret_cast<volatile int32_t*>(a.err) ? njobs : atomicAdd(counter, 1);
        if (tid < kLW) { s_pass[tid] = -1 - kLW; s_prog[tid] = 0; }
        __syncthreads();
        const int p_job = s_job;
        if (p_job >= njobs) break;
        LongJob J;
        int64_t out_idx;
        if (CELLS) {
            const CellJob C = jobs[p_job];
            J = LongJob{a.db + a.off[C.a], a.db + a.off[C.b], C.m, C.n, C.reverse, 0};
            out_idx = p_job;
        } else {
            const PairRef P = pr[p_job];
            // rows: subject x, columns: query q (as the one-warp rescoring kernel)
            J = LongJob{a.db + a.off[P.x], a.db + a.off[P.q], a.off[P.x + 1] - a.off[P.x],
                        a.off[P.q + 1] - a.off[P.q], 0, P.swap};
            out_idx = P.slot;
        }
        int64_t m = J.m;
        const int64_t n = J.n;
        const int npass = (int)((n + G::COLS - 1) / G::COLS);
        if (m > a.bnd_stride || m >= ((int64_t)1 << 30)) {     // boundary slots too short
            if (tid == 0) atomicExch(a.err, 1);
            m = 0;
        }
        int32_t gbest = 0, grow = -1, gcol = -1;                // this warp's passes
        bool gave_up = false;
        for (int pass = warp; pass < npass && m > 0 && !gave_up; pass += kLW) {
            const int64_t c0 = (int64_t)pass * G::COLS;
            // this warp's slot takes pass `pass`: reset its progress, then publish the pass
            if (lane == 0) {
                s_prog[warp] = 0;
                __threadfence_block();
                s_pass[warp] = pass;
            }
            for (int c = lane; c < G::COLS; c += 32) {
                const int64_t cc = c0 + c;
                qres[c] = (cc < n) ? (J.reverse ? J.cb[n - 1 - cc] : J.cb[cc]) : kPadCode;
            }
            __syncwarp();
            for (int i = lane; i < kProfRows * G::COLS; i += 32) {
                const int x = i / G::COLS, c = i - x * G::COLS;
                const int ln = c / kLR, k = c - ln * kLR;
                const int q = qres[c];
                int32_t s = kSpad;                // +o: the DP keeps H - o as its diagonal input
                if (x != kPadCode && q != kPadCode)
                    s = ((CELLS || J.swap) ? s_mat[x * kAlpha + q] : s_mat[q * kAlpha + x]) + o;
                prof[x * ROWW + ln * LS + k] = s;
            }
            __syncwarp();
            const int src = (warp + kLW - 1) % kLW;               // slot of pass - 1
            // rows [0, need) of pass - 1's boundary written: lane 0 polls, bounded
            auto wait = [&](int32_t need) {
                int ok = 1;
                if (lane == 0) {
                    int spins = 0;
                    for (;;) {
                        const int32_t ps = s_pass[src];
                        if (ps > pass - 1 || (ps == pass - 1 && s_prog[src] >= need)) break;
                        if (++spins > a.wait_limit) { ok = 0; break; }
                        __nanosleep(100);
                    }
                    __threadfence_block();
                }
                return __shfl_sync(kFull, ok, 0) != 0;
            };
            auto publish = [&](int32_t rows) {
                __threadfence_block();
                s_prog[warp] = rows;
            };
            D32Best r;
            if (!dp32_pass<kLR, LS, CELLS>(prof + lane * LS, J.ra, m, J.reverse != 0, o, ge,
                                           pass > 0 ? slots + (int64_t)src * a.bnd_stride : nullptr,
                                           pass + 1 < npass ? slots + (int64_t)warp * a.bnd_stride : nullptr,
                                           (int32_t)c0 + lane * kLR, wait, publish, r)) {
                if (lane == 0) atomicExch(a.err, 2);
                gave_up = true;
                break;
            }
            if (CELLS) {
                if (first_max(r.b, r.r, r.c, gbest, grow, gcol)) { gbest = r.b; grow = r.r; gcol = r.c; }
            } else {
                gbest = max(gbest, r.b);
            }
        }
        // combine the warps' passes: largest score, then smallest row, then smallest column
        if (lane == 0) { s_best[warp] = gbest; s_row[warp] = grow; s_col[warp] = gcol; }
        __syncthreads();
        if (tid == 0) {
            int32_t b = 0, rw = -1, cl = -1;
            for (int w = 0; w < kLW; ++w)
                if (first_max(s_best[w], s_row[w], s_col[w], b, rw, cl)) { b = s_best[w]; rw = s_row[w]; cl = s_col[w]; }
            if (CELLS) {
                res[3 * out_idx] = b;
                res[3 * out_idx + 1] = b > 0 ? rw : -1;
                res[3 * out_idx + 2] = b > 0 ? cl : -1;
            } else {
                a.out[out_idx] = b;
            }
        }
    }
}

constexpr int long_smem_bytes() { return kLW * (kProfRows * 32 * kLR * 4 + 32 * kLR); }

}  // namespace

int long_pair_smem() { return long_smem_bytes(); }

cudaError_t launch_long_sw32(int grid, const SwArgs& a, const PairRef* pr, int32_t npairs,
                             int32_t* counter, cudaStream_t st)
{
    if (npairs == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(long_pair_kernel<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         long_smem_bytes());
    if (e != cudaSuccess) return e;
    long_pair_kernel<false><<<grid, kLW * 32, long_smem_bytes(), st>>>(a, pr, nullptr, npairs,
                                                                       counter, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_long_cells(int grid, const SwArgs& a, const CellJob* jobs, int32_t njobs,
                              int32_t* counter, int32_t* res, cudaStream_t st)
{
    if (njobs == 0) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(long_pair_kernel<true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         long_smem_bytes());
    if (e != cudaSuccess) return e;
    long_pair_kernel<true><<<grid, kLW * 32, long_smem_bytes(), st>>>(a, nullptr, jobs, njobs,
                                                                      counter, res);
    return cudaGetLastError();
}

}  // namespace cm
