// Long pairs on a whole CTA: the int32 rescoring and the alignment-cells pass of pairs whose
// query spans many column passes (tandem repeats of 10,000-35,000 residues).  One warp per
// pair would run the passes one after another; here the CTA's LW warps run them as a
// pipeline: warp w takes passes w, w + LW, w + 2 LW, ...; pass p reads the boundary column
// (H, E of its left neighbour column for every row) that pass p - 1 writes, trailing it by at
// least 32 rows.  The boundary of pass p lives in global slot (p mod LW) of the CTA; a warp
// publishes how many rows of its current pass are written in shared memory (tagged with the
// pass), after a block fence.  Waits only point from pass p to pass p - 1 (never backwards),
// and the warps of a CTA are co-resident, so the pipeline always advances; every wait is still
// bounded (SwArgs::wait_limit polls of ~100 ns) and sets the error flag (2) when it gives up.
// Slot p mod LW is rewritten by pass p + LW, which trails its reader (pass p + 1) by at least
// 32 (LW - 1) rows through the chain of waits, so a row is never overwritten before it has
// been read.
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
        if (m > a.bnd_stride) {                                 // boundary slots too short
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
                int32_t s = kSpad;
                if (x != kPadCode && q != kPadCode)
                    s = (CELLS || J.swap) ? s_mat[x * kAlpha + q] : s_mat[q * kAlpha + x];
                prof[x * ROWW + ln * LS + k] = s;
            }
            __syncwarp();
            const int src = (warp + kLW - 1) % kLW;               // slot of pass - 1
            const int2* in = slots + (int64_t)src * a.bnd_stride;
            int2* outb = slots + (int64_t)warp * a.bnd_stride;
            const bool has_out = pass + 1 < npass;
            int32_t hp[kLR], fp[kLR];
#pragma unroll
            for (int k = 0; k < kLR; ++k) { hp[k] = 0; fp[k] = -o; }
            int32_t out_h = 0, out_e = -o, diag0 = 0, best = 0, out_acc = 0;
            int32_t lbest = 0, lrow = -1, lcol = -1;
            uint32_t cur = kPadCode, prev = kPadCode;
            int32_t bh = 0, be = -o;
            const int32_t* plane = prof + lane * LS;
            const int32_t col0 = (int32_t)c0 + lane * kLR;
            for (int64_t t = 0; t < m + 31; ++t) {
                const int j = (int)(t & 31);
                if (j == 0) {
                    if (pass > 0) {                              // rows [t, t + 32) of pass - 1
                        const int32_t need = (int32_t)((t + 32 < m) ? t + 32 : m);
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
                        ok = __shfl_sync(kFull, ok, 0);
                        if (!ok) {
                            if (lane == 0) atomicExch(a.err, 2);
                            gave_up = true;
                            break;
                        }
                    }
                    prev = cur;
                    const int64_t r = t + lane;
                    cur = (r < m) ? (uint32_t)(J.reverse ? J.ra[m - 1 - r] : J.ra[r]) : (uint32_t)kPadCode;
                    if (pass > 0) {
                        if (r < m) { const int2 v = __ldcg(in + r); bh = v.x; be = v.y; }
                        else { bh = 0; be = -o; }
                    }
                }
                const uint32_t rv = __shfl_sync(kFull, (lane <= j) ? cur : prev, (j - lane) & 31);
                int32_t hl = __shfl_up_sync(kFull, out_h, 1);
                int32_t el = __shfl_up_sync(kFull, out_e, 1);
                int32_t ai = __shfl_up_sync(kFull, out_acc, 1);
                if (pass > 0) {
                    const int32_t x = __shfl_sync(kFull, bh, j), y = __shfl_sync(kFull, be, j);
                    if (lane == 0) { hl = x; el = y; }
                } else if (lane == 0) {
                    hl = 0; el = -o;
                }
                if (lane == 0) ai = 0;
                int32_t dg = diag0;
                diag0 = hl;
                const int32_t row = (int32_t)(t - lane);
                const int32_t* prow = plane + (int)min(rv & 31u, (uint32_t)kPadCode) * ROWW;
                int32_t h = hl, e = el;
#pragma unroll
                for (int j4 = 0; j4 < kLR / 4; ++j4) {
                    const int4 sv = *reinterpret_cast<const int4*>(prow + 4 * j4);
                    const int32_t s4[4] = {sv.x, sv.y, sv.z, sv.w};
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int k = 4 * j4 + u;
                        e = __viaddmax_s32(h, -o, e - ge);
                        const int32_t f = __viaddmax_s32(hp[k], -o, fp[k] - ge);
                        fp[k] = f;
                        const int32_t d = __viaddmax_s32(dg, s4[u], 0);
                        dg = hp[k];
                        h = __vimax3_s32(d, e, f);
                        hp[k] = h;
                        if (CELLS) {
                            if (h > lbest) { lbest = h; lrow = row; lcol = col0 + k; }
                        } else {
                            best = max(best, h);
                        }
                    }
                }
                out_h = h;
                out_e = e;
                if (!CELLS) {
                    out_acc = max(ai, best);
                    if (lane == 31 && t - 31 == m - 1) gbest = max(gbest, out_acc);
                }
                if (has_out && t >= 31) {
                    if (lane == 31) __stcg(outb + (t - 31), make_int2(out_h, out_e));
                    if (j == 31 && lane == 31) {                // publish rows [0, t - 30)
                        __threadfence_block();
                        s_prog[warp] = (int32_t)(t - 30);
                    }
                }
            }
            if (gave_up) break;
            if (has_out && lane == 31) {
                __threadfence_block();
                s_prog[warp] = (int32_t)m;
            }
            if (CELLS) {
                // pad rows / columns stay below the maximum over real cells
                for (int d = 16; d >= 1; d >>= 1) {
                    const int32_t ob = __shfl_xor_sync(kFull, lbest, d);
                    const int32_t orw = __shfl_xor_sync(kFull, lrow, d);
                    const int32_t oc = __shfl_xor_sync(kFull, lcol, d);
                    const bool better = ob > lbest ||
                                        (ob == lbest && (orw < lrow || (orw == lrow && oc < lcol)));
                    if (better) { lbest = ob; lrow = orw; lcol = oc; }
                }
                const bool better = lbest > gbest ||
                                    (lbest == gbest && lbest > 0 &&
                                     (lrow < grow || (lrow == grow && lcol < gcol)));
                if (better) { gbest = lbest; grow = lrow; gcol = lcol; }
            }
        }
        // combine the warps' passes: largest score, then smallest row, then smallest column
        if (!CELLS) gbest = __shfl_sync(kFull, gbest, 31);
        if (lane == 0) { s_best[warp] = gbest; s_row[warp] = grow; s_col[warp] = gcol; }
        __syncthreads();
        if (tid == 0) {
            int32_t b = 0, rw = -1, cl = -1;
            for (int w = 0; w < kLW; ++w) {
                const int32_t ob = s_best[w], orw = s_row[w], oc = s_col[w];
                const bool better = ob > b || (ob == b && ob > 0 && (orw < rw || (orw == rw && oc < cl)));
                if (better) { b = ob; rw = orw; cl = oc; }
            }
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
