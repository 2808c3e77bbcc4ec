// int32 Smith-Waterman wavefront of one warp over one column pass: the exact rescoring of pairs
// whose int16 scores saturated, and the alignment-cells pass (score plus the first row-major
// cell reaching it).  Same recurrences as the int16 kernel (Sec. 4's f: affine-gap local
// alignment score), on plain 32-bit integers, so no score range limit.
//
// Mapping.  Lane l holds R consecutive columns of the pass (profile segment `plane`, LS words
// per lane in a profile row).  Each step covers kD32Rows consecutive rows (a row group): at
// step t lane l works on row group t - l, receiving H - o and E of its left neighbour's last
// column for the group's rows by warp shuffles; inside the lane row q trails row q - 1 by one
// column, so the group's rows are independent dependency chains.  The DP keeps H - o (the
// value both gap types open from) and the profile carries S + o:
//   E = max(E - e, (H - o)_left),  F = max(F - e, (H - o)_up),
//   D = max((H - o)_diag + (S + o), 0),  H = max(D, E, F),  then H - o once.
// A multi-pass matrix hands a boundary column from pass to pass: (H - o, E) of the pass's last
// column for every row.
#pragma once
#include <cstdint>

#include "cm_internal.h"

namespace cm {
namespace {

constexpr int kD32Rows = 4;

// first maximum in row-major order: larger score, then smaller row, then smaller column
__device__ __forceinline__ bool first_max(int32_t b, int32_t r, int32_t c, int32_t b0, int32_t r0,
                                          int32_t c0)
{
    return b > b0 || (b == b0 && b > 0 && (r < r0 || (r == r0 && c < c0)));
}

struct D32Best {
    int32_t b, r, c;     // score; its first (row, column) in row-major order (CELLS), else -1
};

// One column pass over rows ra[0..m) (read back to front when `reverse`; m < 2^30).  `bin`:
// boundary column of the previous pass (nullptr on the first pass: the matrix's left edge);
// `bout`: where this pass writes its own (nullptr on the last pass).  Before the warp reads the
// boundary rows [.., need) it calls wait(need) (warp-uniform; false gives up and the pass
// returns false); lane 31 calls publish(rows) after the first `rows` boundary rows are
// written.  col0 = the first column of this lane.  CELLS: every row class q (rows = q mod
// kD32Rows) keeps its own first maximum with strict > (its rows come in order, a row's columns
// in order), and the classes, then the lanes, are merged with the row-major tie-break; cells of
// pad rows or pad columns stay below the maximum over real cells.  Returns the warp's result
// in `out` on every lane.
template <int R, int LS, bool CELLS, class Wait, class Publish>
__device__ __forceinline__ bool dp32_pass(const int32_t* __restrict__ plane,
                                          const uint8_t* __restrict__ ra, int64_t m, bool reverse,
                                          int o, int ge, const int2* bin, int2* bout, int32_t col0,
                                          Wait&& wait, Publish&& publish, D32Best& out)
{
    static_assert(R % 4 == 0, "profile rows are read as 16-byte vectors");
    constexpr int NR = kD32Rows;
    constexpr int ROWW = 32 * LS;
    constexpr uint32_t kAll = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int32_t ngrp = (int32_t)((m + NR - 1) / NR);
    int32_t hp[R], fp[R];                                 // H - o and F of the row above
#pragma unroll
    for (int k = 0; k < R; ++k) { hp[k] = -o; fp[k] = -o; }
    int32_t oh[NR], oe[NR], bh[NR], be[NR];               // last column; boundary rows
#pragma unroll
    for (int q = 0; q < NR; ++q) { oh[q] = -o; oe[q] = -o; bh[q] = -o; be[q] = -o; }
    int32_t diag0 = -o, best = 0, out_acc = 0, result = 0;
    int32_t lbest[NR], lrow[NR], lcol[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) { lbest[q] = 0; lrow[q] = -1; lcol[q] = -1; }
    // rows before the first (lane l runs l of them while the wavefront fills) are pad rows
    constexpr uint32_t kPadRows = (uint32_t)kPadCode * 0x01010101u;
    uint32_t cur = kPadRows, prev = kPadRows;

    for (int32_t t = 0; t < ngrp + 31; ++t) {
        const int j = t & 31;
        if (j == 0) {
            if (bin != nullptr) {                         // row groups [t, t + 32) of the boundary
                const int64_t need = (int64_t)(t + 32) * NR;
                if (!wait((int32_t)(need < m ? need : m))) return false;
            }
            prev = cur;
            cur = 0;
            const int64_t g = (int64_t)(t + lane) * NR;   // first row of this lane's next group
#pragma unroll
            for (int q = 0; q < NR; ++q) {
                const int64_t r = g + q;
                const uint32_t x = (r < m) ? (uint32_t)(reverse ? ra[m - 1 - r] : ra[r])
                                           : (uint32_t)kPadCode;
                cur |= min(x, (uint32_t)kPadCode) << (8 * q);
                if (bin != nullptr) {
                    if (r < m) { const int2 v = __ldcg(bin + r); bh[q] = v.x; be[q] = v.y; }
                    else { bh[q] = -o; be[q] = -o; }
                }
            }
        }
        const uint32_t rv = __shfl_sync(kAll, (lane <= j) ? cur : prev, (j - lane) & 31);
        int32_t hL[NR], eL[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            hL[q] = __shfl_up_sync(kAll, oh[q], 1);
            eL[q] = __shfl_up_sync(kAll, oe[q], 1);
        }
        int32_t ai = __shfl_up_sync(kAll, out_acc, 1);
        if (bin != nullptr) {
#pragma unroll
            for (int q = 0; q < NR; ++q) {
                const int32_t x = __shfl_sync(kAll, bh[q], j), y = __shfl_sync(kAll, be[q], j);
                if (lane == 0) { hL[q] = x; eL[q] = y; }
            }
        } else if (lane == 0) {
#pragma unroll
            for (int q = 0; q < NR; ++q) { hL[q] = -o; eL[q] = -o; }
        }
        if (lane == 0) ai = 0;
        int32_t dg[NR], h[NR], e[NR];
        dg[0] = diag0;
#pragma unroll
        for (int q = 1; q < NR; ++q) dg[q] = hL[q - 1];
        diag0 = hL[NR - 1];
        const int32_t row0 = (t - lane) * NR;
        const int32_t* prow[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            prow[q] = plane + (int)((rv >> (8 * q)) & 0xffu) * ROWW;
            h[q] = hL[q];
            e[q] = eL[q];
        }
        int32_t sq[NR][4];
#pragma unroll
        for (int k = 0; k < R + NR - 1; ++k) {
#pragma unroll
            for (int q = 0; q < NR; ++q) {
                const int c = k - q;
                if (c < 0 || c >= R) continue;
                if ((c & 3) == 0) {
                    const int4 sv = *reinterpret_cast<const int4*>(prow[q] + c);
                    sq[q][0] = sv.x; sq[q][1] = sv.y; sq[q][2] = sv.z; sq[q][3] = sv.w;
                }
                e[q] = __viaddmax_s32(e[q], -ge, h[q]);
                const int32_t f = __viaddmax_s32(fp[c], -ge, hp[c]);
                const int32_t d = __viaddmax_s32(dg[q], sq[q][c & 3], 0);
                dg[q] = hp[c];
                const int32_t hh = __vimax3_s32(d, e[q], f);
                if (CELLS) {
                    if (hh > lbest[q]) { lbest[q] = hh; lrow[q] = row0 + q; lcol[q] = col0 + c; }
                } else {
                    best = max(best, hh);
                }
                h[q] = hh - o;
                hp[c] = h[q];
                fp[c] = f;
            }
        }
#pragma unroll
        for (int q = 0; q < NR; ++q) { oh[q] = h[q]; oe[q] = e[q]; }
        if (!CELLS) {
            out_acc = max(ai, best);
            if (lane == 31 && t - 31 == ngrp - 1) result = out_acc;
        }
        if (bout != nullptr && t >= 31 && lane == 31) {
            const int64_t g = (int64_t)(t - 31) * NR;
#pragma unroll
            for (int q = 0; q < NR; ++q)
                if (g + q < m) __stcg(bout + g + q, make_int2(oh[q], oe[q]));
            if (j == 31) {                                // rows [0, NR (t - 30)) are written
                const int64_t done = (int64_t)(t - 30) * NR;
                publish((int32_t)(done < m ? done : m));
            }
        }
    }
    if (bout != nullptr && lane == 31) publish((int32_t)m);
    if (CELLS) {
        int32_t b = lbest[0], rw = lrow[0], cl = lcol[0];
#pragma unroll
        for (int q = 1; q < NR; ++q)
            if (first_max(lbest[q], lrow[q], lcol[q], b, rw, cl)) { b = lbest[q]; rw = lrow[q]; cl = lcol[q]; }
        for (int d = 16; d >= 1; d >>= 1) {
            const int32_t ob = __shfl_xor_sync(kAll, b, d);
            const int32_t orw = __shfl_xor_sync(kAll, rw, d);
            const int32_t oc = __shfl_xor_sync(kAll, cl, d);
            if (first_max(ob, orw, oc, b, rw, cl)) { b = ob; rw = orw; cl = oc; }
        }
        out = D32Best{b, b > 0 ? rw : -1, b > 0 ? cl : -1};
    } else {
        out = D32Best{__shfl_sync(kAll, result, 31), -1, -1};
    }
    return true;
}

}  // namespace
}  // namespace cm
