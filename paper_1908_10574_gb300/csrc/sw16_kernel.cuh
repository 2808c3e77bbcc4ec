// Batched Smith-Waterman (Gotoh affine gaps) on sm_103a: the similarity f of the paper's
// protein clustering (Sec. 4), scored for many pairs at once.
//
// Recurrences (a gap of k residues costs o + (k-1)e; H >= 0 makes the alignment local):
//   E(r,c) = max(E(r,c-1) - e, H(r,c-1) - o)
//   F(r,c) = max(F(r-1,c) - e, H(r-1,c) - o)
//   H(r,c) = max(0, H(r-1,c-1) + S(q_c, x_r), E(r,c), F(r,c)),   score = max H
//
// Mapping.  A warp owns 32*R query columns (lane l holds columns l*R .. l*R+R-1 in
// registers) and streams subject rows through an anti-diagonal wavefront: at step t lane l
// computes row t-l of its columns, receiving H and E of its left neighbour's last column for
// the same row by one warp shuffle.  Many subjects are concatenated in one row stream (first
// and last rows flagged), so the fill/drain of the wavefront is paid once per stream, not once
// per pair.  The two 16-bit halves of every register carry two different queries that share
// the subject stream, so each packed DPX instruction advances two cells.
//
// Packed-int16 formulation.  Every stored value carries a bias beta >= o+e (stored = true +
// beta), which keeps each half within [beta-o, 32767].  The DP keeps H - o, the value both gap
// types open from, and the profile carries S + o, so the diagonal term reads H - o as well:
// per packed column 3 viaddmax (E, F, diagonal), 1 vimax3 (H) and 1/2 vimax3 (running
// maximum, every two columns) on the ALU pipe, plus one plain 32-bit subtract for H - o on
// the IADD path (H >= beta > o in both halves, so it never borrows across them).  If a stored
// best reaches 32767 - max(S), some cell may have overflowed int16; that pair is marked and
// rescored on the int32 path, so every score returned is exact.
#pragma once
#include <algorithm>

#include "cm_internal.h"
#include "dp32.cuh"

namespace cm {

namespace {

constexpr uint32_t kFull = 0xffffffffu;
constexpr int kSpad = -1024;   // profile entry of pad rows / pad columns (any value <= 0 works)

// Words per lane in a profile row: R rounded up to a multiple of 4 (16-byte loads), plus 4
// more when that is an even number of 16-byte units, so that the eight lanes of a quarter
// warp always read eight distinct 16-byte bank groups whatever residues they look up.
__host__ __device__ constexpr int lane_stride(int R)
{
    return (((R + 3) / 4) & 1) ? (R + 3) / 4 * 4 : (R + 3) / 4 * 4 + 4;
}

// Tile geometry: SEG lanes (32, or 16 for a half-warp segment) of R columns each.
template <int R, int SEG = 32>
struct Geo {
    static constexpr int LS = lane_stride(R);       // 32-bit words per lane in a profile row
    static constexpr int ROWW = SEG * LS;           // words per profile row (multiple of 64 B)
    static constexpr int PROF_WORDS = kProfRows * ROWW;
    static constexpr int COLS = SEG * R;            // query columns per pass
};

__device__ __forceinline__ uint32_t pack2(int lo, int hi)
{
    return (uint32_t)(uint16_t)(int16_t)lo | ((uint32_t)(uint16_t)(int16_t)hi << 16);
}

__device__ __forceinline__ int64_t tri(int64_t k) { return k * (k - 1) / 2; }

__device__ __forceinline__ int32_t lower_bound64(const int64_t* v, int32_t lo, int32_t hi,
                                                 int64_t key)
{
    // first index s in [lo, hi] with v[s] >= key (v strictly increasing)
    while (lo < hi) {
        const int32_t mid = (lo + hi) >> 1;
        if (v[mid] < key) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// subject boundary in [lo, hi] nearest to row `key` (ties to the later one): stream splits
// land within half a subject of their target, so the warps of a task finish closer together
__device__ __forceinline__ int32_t nearest_boundary(const int64_t* v, int32_t lo, int32_t hi,
                                                    int64_t key)
{
    const int32_t s = lower_bound64(v, lo, hi, key);
    return (s > lo && key - v[s - 1] < v[s] - key) ? s - 1 : s;
}

__device__ __forceinline__ int64_t slot_of(const SwBlock& B, int32_t k, int32_t s)
{
    const int64_t base = (B.kind == kTri) ? (tri(k) - tri(B.k0)) : (int64_t)(k - B.k0) * B.nb;
    return B.out_base + base + s;
}

__device__ __forceinline__ void store_score(const SwArgs& a, const SwBlock& B, int32_t k,
                                            int32_t s, int32_t stored, int pass)
{
    int64_t slot = slot_of(B, k, s);
    if (B.has_map) slot = a.out_map[slot];
    const int32_t val = (stored >= a.sat_thr) ? kSat : stored - a.beta;
    if (pass == 0) {
        a.out[slot] = val;
    } else {
        const int32_t old = a.out[slot];
        if (old != kSat) a.out[slot] = (val == kSat) ? kSat : max(old, val);
    }
}

// One wavefront segment of SEG lanes (a whole warp, or a half-warp when SEG = 16) against the
// profile tile of this pass.  Every subject starts on a row that is a multiple of kRowGroup.
//   pair (TWO = false): the two 16-bit halves are two queries; one subject stream `lo` of
//     n_lo rows feeds both.
//   single query (TWO = true): both halves hold the same query; the lo half runs stream `lo`
//     (n_lo rows), the hi half stream `hi` (n_hi rows).  The profile then carries the score in
//     its low half only, and the packed score word of a column is hi_row * 2^16 + lo_row (one
//     multiply-add on the FMA pipe).
// A step covers NR consecutive rows of each stream; row q of the step trails row q-1 by one
// column inside the lane, so the NR rows form independent dependency chains and the step's
// fixed costs (shuffles, residue and flag handling) are shared by NR rows.  The segment's
// last lane writes one score per finished subject per half.  All lanes of the warp run
// `nrows_max` rows (the warp's longest stream); shorter streams step through pad rows
// meanwhile.  Multi-pass tiles (boundary columns in `bnd`) use SEG = 32 only.
// Rows per step: four (a row group) in the pair modes.  The single-query modes carry a second
// subject stream (a second residue-row lookup per row) and fit four rows into the register
// budget only for narrow tiles: four up to 7 columns per lane in 16-lane segments, two up
// to 16 columns, one above (the host keeps single-query tiles at <= 16 columns per lane).
template <int R, int SEG, bool TWO>
struct RowsPerStep {
    static constexpr int value = !TWO ? 4 : (SEG == 16 && R <= 7) ? 4 : (R <= 16 ? 2 : 1);
};

template <int NR> struct RowWord;
template <> struct RowWord<1> { typedef uint8_t type; };
template <> struct RowWord<2> { typedef uint16_t type; };
template <> struct RowWord<4> { typedef uint32_t type; };

// load the profile words of columns [c, c + 4) of one row (fewer at the tile's right edge;
// the lane's row segment always holds whole 16-byte units)
template <int R>
__device__ __forceinline__ void load_cols(const uint32_t* p, int c, uint32_t (&v)[4])
{
    if (c + 3 <= R) {
        const uint4 x = *reinterpret_cast<const uint4*>(p + c);
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    } else if (c + 2 == R) {
        const uint2 x = *reinterpret_cast<const uint2*>(p + c);
        v[0] = x.x; v[1] = x.y;
    } else {
        v[0] = p[c];
    }
}

template <int R, int SEG, bool TWO>
__device__ __forceinline__ void warp_dp16(const SwArgs& a, const SwBlock& B,
                                          const uint32_t* __restrict__ prof,
                                          const uint8_t* __restrict__ st_lo, int64_t n_lo,
                                          const uint8_t* __restrict__ st_hi, int64_t n_hi,
                                          int64_t nrows_max, int pass, int npass,
                                          uint2* __restrict__ bnd, int32_t s_lo0, int32_t s_hi0,
                                          int32_t k_lo, int32_t ns_lo, int32_t ns_hi,
                                          bool hi_valid)
{
    using G = Geo<R, SEG>;
    constexpr int NR = RowsPerStep<R, SEG, TWO>::value;
    typedef typename RowWord<NR>::type word_t;
    const int lane = threadIdx.x & (SEG - 1);    // lane within the segment
    const int o = a.gap_open, ge = a.gap_extend, beta = a.beta;
    const uint32_t BETA2 = (uint32_t)beta * 0x10001u;
    const uint32_t BMO2 = (uint32_t)(beta - o) * 0x10001u;   // H - o of an empty prefix; E, F floor
    const uint32_t O2 = (uint32_t)o * 0x10001u;
    const uint32_t NEGE = pack2(-ge, -ge);
    const uint32_t PADW = (kPadCode * 0x01010101u) >> (32 - 8 * NR);   // kPadCode in every byte
    // boundary records of one step: (H - o, E) of the last column of each of its rows, as
    // uint4 pairs of rows (one uint2 when a step has one row)
    constexpr int NB = (NR >= 2) ? NR / 2 : 1;
    uint4* bnd4 = reinterpret_cast<uint4*>(bnd);
    const uint32_t CODEMASK = 0x1f1f1f1fu >> (32 - 8 * NR);           // residue code bits
    uint32_t LASTBITS = 0;
#pragma unroll
    for (int q = 0; q < NR; ++q) LASTBITS |= (uint32_t)kLast << (8 * q);

    // hp[c] holds H - o of the row above (the value both E and F start a gap from, and the
    // diagonal of column c+1 against a profile that carries +o); fp[c] holds F.
    uint32_t hp[R], fp[R];
#pragma unroll
    for (int k = 0; k < R; ++k) { hp[k] = BMO2; fp[k] = BMO2; }
    uint32_t best = BETA2, out_acc = BETA2;
    uint32_t oh[NR], oe[NR];                      // last column of each row: H - o and E
#pragma unroll
    for (int q = 0; q < NR; ++q) { oh[q] = BMO2; oe[q] = BMO2; }
    uint32_t diag0 = BMO2;                        // left H - o of the previous step's last row
    uint32_t cur = PADW, prev = PADW, cur2 = PADW, prev2 = PADW;
    uint4 bv[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) bv[q] = make_uint4(BMO2, BMO2, BMO2, BMO2);
    int32_t s_lo = s_lo0, s_hi = s_hi0;
    const uint32_t* plane = prof + lane * G::LS;
    const int nsup = (int)(n_lo / NR);            // a warp stream holds < 2^31 rows
    const int nsup2 = TWO ? (int)(n_hi / NR) : 0;
    const int nsup_max = (int)(nrows_max / NR);
    const int nsteps = nsup_max + SEG - 1;
    const word_t* stw = reinterpret_cast<const word_t*>(st_lo);
    const word_t* stw2 = reinterpret_cast<const word_t*>(st_hi);

    for (int t = 0; t < nsteps; ++t) {
        const int j = t & (SEG - 1);
        if (j == 0) {
            const int u = t + lane;
            prev = cur;
            cur = (u < nsup) ? (uint32_t)stw[u] : PADW;
            if (TWO) {
                prev2 = cur2;
                cur2 = (u < nsup2) ? (uint32_t)stw2[u] : PADW;
            }
            if (SEG == 32 && pass > 0) {
                if constexpr (NR >= 2) {
#pragma unroll
                    for (int q = 0; q < NB; ++q)
                        bv[q] = (u < nsup_max) ? bnd4[u * NB + q] : make_uint4(BMO2, BMO2, BMO2, BMO2);
                } else {
                    const uint2 v = (u < nsup_max) ? bnd[u] : make_uint2(BMO2, BMO2);
                    bv[0] = make_uint4(v.x, v.y, BMO2, BMO2);
                }
            }
        }
        const int src = (j - lane) & (SEG - 1);
        const uint32_t rv = __shfl_sync(kFull, (lane <= j) ? cur : prev, src, SEG);
        const uint32_t rw = TWO ? __shfl_sync(kFull, (lane <= j) ? cur2 : prev2, src, SEG) : 0u;
        uint32_t hL[NR], eL[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            hL[q] = __shfl_up_sync(kFull, oh[q], 1, SEG);
            eL[q] = __shfl_up_sync(kFull, oe[q], 1, SEG);
        }
        uint32_t ai = __shfl_up_sync(kFull, out_acc, 1, SEG);
        if (SEG == 32 && pass > 0) {
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                const uint32_t x0 = __shfl_sync(kFull, bv[q].x, j), x1 = __shfl_sync(kFull, bv[q].y, j);
                if (lane == 0) { hL[2 * q] = x0; eL[2 * q] = x1; }
                if constexpr (NR >= 2) {
                    const uint32_t x2 = __shfl_sync(kFull, bv[q].z, j), x3 = __shfl_sync(kFull, bv[q].w, j);
                    if (lane == 0) { hL[2 * q + 1] = x2; eL[2 * q + 1] = x3; }
                }
            }
        } else if (lane == 0) {
#pragma unroll
            for (int q = 0; q < NR; ++q) { hL[q] = BMO2; eL[q] = BMO2; }
        }
        if (lane == 0) ai = BETA2;
        uint32_t dg[NR], h[NR], e[NR];
        dg[0] = diag0;
#pragma unroll
        for (int q = 1; q < NR; ++q) dg[q] = hL[q - 1];
        diag0 = hL[NR - 1];
        if (!TWO) {
            if (rv & kFirst) {                    // a subject starts at the step's first row
#pragma unroll
                for (int k = 0; k < R; ++k) { hp[k] = BMO2; fp[k] = BMO2; }
                best = BETA2;
                dg[0] = BMO2;
            }
        } else if ((rv | rw) & kFirst) {          // per half: whose stream starts a subject
            const uint32_t keep = ((rv & kFirst) ? 0u : 0x0000ffffu) | ((rw & kFirst) ? 0u : 0xffff0000u);
#pragma unroll
            for (int k = 0; k < R; ++k) {
                hp[k] = (hp[k] & keep) | (BMO2 & ~keep);
                fp[k] = (fp[k] & keep) | (BMO2 & ~keep);
            }
            best = (best & keep) | (BETA2 & ~keep);
            dg[0] = (dg[0] & keep) | (BMO2 & ~keep);
        }
        // profile row of each residue: one mask takes the flags off all NR bytes, one byte
        // permute moves a code to the low byte (the stream writer keeps codes <= kPadCode)
        const uint32_t rc = rv & CODEMASK, rc2 = TWO ? (rw & CODEMASK) : 0u;
        const uint32_t* prow[NR];
        const uint32_t* prow2[NR];
#pragma unroll
        for (int q = 0; q < NR; ++q) {
            prow[q] = plane + __byte_perm(rc, 0u, 0x4440u | q) * G::ROWW;
            if (TWO) prow2[q] = plane + __byte_perm(rc2, 0u, 0x4440u | q) * G::ROWW;
            h[q] = hL[q];
            e[q] = eL[q];
        }
        uint32_t sq[NR][4];
        uint32_t pend = 0;
        bool has_pend = false;
        // Row q trails row q-1 by one column.  Per packed cell: E = max(E - e, (H - o)_left),
        // F = max(F - e, (H - o)_up), D = max((H - o)_diag + (S + o), beta), H = max(D, E, F),
        // then H - o once for the neighbours (plain 32-bit subtract: H >= beta >= o + e, so
        // neither half borrows).
#pragma unroll
        for (int k = 0; k < R + NR - 1; ++k) {
#pragma unroll
            for (int q = 0; q < NR; ++q) {
                const int c = k - q;
                if (c < 0 || c >= R) continue;
                if ((c & 3) == 0) {               // next (up to) four profile columns of row q
                    load_cols<R>(prow[q], c, sq[q]);
                    if (TWO) {
                        uint32_t v2[4];
                        load_cols<R>(prow2[q], c, v2);
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (c + u < R) sq[q][u] = v2[u] * 0x10000u + sq[q][u];
                    }
                }
                e[q] = __viaddmax_s16x2(e[q], NEGE, h[q]);
                const uint32_t f = __viaddmax_s16x2(fp[c], NEGE, hp[c]);
                const uint32_t d = __viaddmax_s16x2(dg[q], sq[q][c & 3], BETA2);
                dg[q] = hp[c];
                const uint32_t hh = __vimax3_s16x2(d, e[q], f);
                if (has_pend) { best = __vimax3_s16x2(best, pend, hh); has_pend = false; }
                else { pend = hh; has_pend = true; }
                h[q] = hh - O2;
                hp[c] = h[q];
                fp[c] = f;
            }
        }
        if (has_pend) best = __vmaxs2(best, pend);
#pragma unroll
        for (int q = 0; q < NR; ++q) { oh[q] = h[q]; oe[q] = e[q]; }
        out_acc = __vmaxs2(ai, best);
        if (lane == SEG - 1) {
            const int32_t lo = (int32_t)(int16_t)(out_acc & 0xffffu);
            const int32_t hi = (int32_t)(int16_t)(out_acc >> 16);
            if (!TWO) {
                if (rv & LASTBITS) {
                    const int32_t s = s_lo++;
                    if (s < ns_lo) store_score(a, B, k_lo, s, lo, pass);
                    if (hi_valid && s < ns_hi) store_score(a, B, k_lo + 1, s, hi, pass);
                }
            } else {
                if (rv & LASTBITS) {
                    const int32_t s = s_lo++;
                    if (s < ns_lo) store_score(a, B, k_lo, s, lo, pass);
                }
                if (rw & LASTBITS) {
                    const int32_t s = s_hi++;
                    if (s < ns_lo) store_score(a, B, k_lo, s, hi, pass);
                }
            }
        }
        if (SEG == 32 && lane == 31 && pass + 1 < npass && t >= 31) {
            if constexpr (NR >= 2) {
#pragma unroll
                for (int q = 0; q < NB; ++q)
                    bnd4[(t - 31) * NB + q] = make_uint4(oh[2 * q], oe[2 * q], oh[2 * q + 1], oe[2 * q + 1]);
            } else {
                bnd[t - 31] = make_uint2(oh[0], oe[0]);
            }
        }
    }
}

// Persistent int16x2 kernel.  MODE kModePair: a query pair (two 16-bit halves) per task, one
// subject stream per warp over 32 lanes.  kModeTwo: one query, two subject streams in the two
// halves of each warp.  kModeSeg16: a query pair, two subject streams per warp, one per
// half-warp segment of 16 lanes.  kModeTwo16: one query, four subject streams per warp (two
// 16-lane segments x two halves).  The 16-lane modes serve short queries (16 lanes x R).
template <int R, int W, int MODE>
__global__ void __launch_bounds__(W * 32, 16 / W)
sw16_kernel(const __grid_constant__ SwArgs a)
{
    constexpr bool TWO = (MODE == kModeTwo || MODE == kModeTwo16);
    constexpr int SEG = (MODE == kModeSeg16 || MODE == kModeTwo16) ? 16 : 32;
    constexpr int SPW = (MODE == kModePair) ? 1 : (MODE == kModeTwo16) ? 4 : 2;   // streams per warp
    using G = Geo<R, SEG>;
    extern __shared__ __align__(16) uint8_t smem[];
    uint32_t* prof = reinterpret_cast<uint32_t*>(smem);
    uint8_t* qres = smem + (size_t)G::PROF_WORDS * 4;          // [2][COLS]
    __shared__ int16_t s_mat[kAlpha * kAlpha];
    __shared__ int s_task[2];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int i = tid; i < kAlpha * kAlpha; i += W * 32) s_mat[i] = a.mat[i];
    if (tid == 0) s_task[0] = atomicAdd(a.task_counter, 1);
    __syncthreads();

    uint2* bnd = a.bnd + ((int64_t)blockIdx.x * W + warp) * a.bnd_stride;
    for (int it = 0;; ++it) {
        const int ti = s_task[it & 1];
        if (ti >= a.ntasks) break;
        if (tid == 0) s_task[(it + 1) & 1] = atomicAdd(a.task_counter, 1);

        const SwTask T = a.tasks[ti];
        const SwBlock B = a.blocks[T.block];
        const int32_t* A_ids = a.ids + B.a_ids;
        const int32_t q_lo = A_ids[T.k];
        const int32_t q_hi = (!TWO && T.hi_valid) ? A_ids[T.k + 1] : q_lo;
        const int64_t qoff_lo = a.off[q_lo], m_lo = a.off[q_lo + 1] - qoff_lo;
        const int64_t qoff_hi = a.off[q_hi];
        const int64_t m_hi = (!TWO && T.hi_valid) ? a.off[q_hi + 1] - qoff_hi : 0;
        const int32_t ns_lo = (B.kind == kTri) ? T.k : B.nb;
        const int32_t ns_hi = (B.kind == kTri) ? T.k + 1 : B.nb;
        const int64_t* srow = a.srows + B.srow;

        // rows of this task split over the CTA's streams at subject boundaries
        constexpr int NS = W * SPW;
        const int64_t R0 = srow[T.s0], R1 = srow[T.s1];
        int32_t sb[SPW + 1];
        int64_t nmax = 0;
#pragma unroll
        for (int i = 0; i <= SPW; ++i) {
            sb[i] = nearest_boundary(srow, T.s0, T.s1, R0 + (R1 - R0) * (warp * SPW + i) / NS);
            if (i > 0) nmax = max(nmax, srow[sb[i]] - srow[sb[i - 1]]);
        }
        // this lane's streams: index of the lo stream among the warp's SPW
        const int seg = (SEG == 16) ? (lane >> 4) : 0;
        const int i_lo = TWO ? 2 * seg : seg;
        const int32_t slo0 = sb[i_lo], slo1 = sb[i_lo + 1];
        const int32_t shi0 = TWO ? sb[i_lo + 1] : slo1, shi1 = TWO ? sb[i_lo + 2] : slo1;
        int64_t n_lo = srow[slo1] - srow[slo0];
        int64_t n_hi = srow[shi1] - srow[shi0];
        if (T.npass > 1 && (SEG == 16 || nmax > a.bnd_stride)) {
            if (lane == 0) atomicExch(a.err, 1);      // boundary buffer too small: refuse
            n_lo = n_hi = nmax = 0;
        }
        const uint8_t* st_lo = a.streams + B.stream + srow[slo0];
        const uint8_t* st_hi = a.streams + B.stream + srow[shi0];

        for (int pass = 0; pass < T.npass; ++pass) {
            const int64_t c0 = (int64_t)pass * G::COLS;
            for (int c = tid; c < G::COLS; c += W * 32) {
                qres[c] = (c0 + c < m_lo) ? a.db[qoff_lo + c0 + c] : kPadCode;
                qres[G::COLS + c] = (c0 + c < m_hi) ? a.db[qoff_hi + c0 + c] : kPadCode;
            }
            __syncthreads();
            for (int i = tid; i < kProfRows * G::COLS; i += W * 32) {
                const int x = i / G::COLS, c = i - x * G::COLS;
                const int ln = c / R, k = c - ln * R;
                const int ql = qres[c], qh = qres[G::COLS + c];
                int sl = kSpad, sh = TWO ? 0 : kSpad;
                if (x != kPadCode) {          // +o: the DP keeps H - o as its diagonal input
                    if (ql != kPadCode) sl = (B.swap ? s_mat[x * kAlpha + ql] : s_mat[ql * kAlpha + x]) + a.gap_open;
                    if (!TWO && qh != kPadCode) sh = (B.swap ? s_mat[x * kAlpha + qh] : s_mat[qh * kAlpha + x]) + a.gap_open;
                }
                prof[x * G::ROWW + ln * G::LS + k] = pack2(sl, sh);
            }
            __syncthreads();
            if (nmax > 0)
                warp_dp16<R, SEG, TWO>(a, B, prof, st_lo, n_lo, st_hi, n_hi, nmax, pass, T.npass,
                                       bnd, slo0, shi0, T.k, ns_lo, ns_hi, T.hi_valid != 0);
            __syncthreads();
        }
    }
}

// ---- int32 rescoring of pairs flagged by the int16 pass: one warp per pair -----------------
// Rows stream the subject x, columns hold the query q in passes of 32 R columns; the passes of
// a pair run one after another on the warp, the boundary column kept in the warp's own slot
// of `bnd` (read ahead of where the same pass writes it).
template <int R>
__global__ void __launch_bounds__(32) sw32_kernel(const __grid_constant__ SwArgs a,
                                                 const PairRef* __restrict__ pr,
                                                 int32_t npairs, int32_t* counter)
{
    using G = Geo<R>;
    extern __shared__ __align__(16) uint8_t smem[];
    int32_t* prof = reinterpret_cast<int32_t*>(smem);
    uint8_t* qres = smem + (size_t)G::PROF_WORDS * 4;
    __shared__ int16_t s_mat[kAlpha * kAlpha];
    const int lane = threadIdx.x;
    for (int i = lane; i < kAlpha * kAlpha; i += 32) s_mat[i] = a.mat[i];
    __syncwarp();
    const int o = a.gap_open, ge = a.gap_extend;
    int2* bnd = reinterpret_cast<int2*>(a.bnd + (int64_t)blockIdx.x * a.bnd_stride);
    auto no_wait = [](int32_t) { return true; };
    auto no_publish = [](int32_t) {};

    for (;;) {
        int p = 0;
        if (lane == 0) p = atomicAdd(counter, 1);
        p = __shfl_sync(kFull, p, 0);
        if (p >= npairs) break;
        const PairRef P = pr[p];
        const int64_t qoff = a.off[P.q], m = a.off[P.q + 1] - qoff;
        const int64_t xoff = a.off[P.x];
        int64_t n = a.off[P.x + 1] - xoff;
        const int npass = (m <= G::COLS) ? 1 : (int)((m + G::COLS - 1) / G::COLS);
        if ((npass > 1 && n > a.bnd_stride) || n >= ((int64_t)1 << 30)) {
            if (lane == 0) atomicExch(a.err, 1);
            n = 0;
        }
        int32_t result = 0;
        for (int pass = 0; pass < npass && n > 0; ++pass) {
            const int64_t c0 = (int64_t)pass * G::COLS;
            __syncwarp();
            for (int c = lane; c < G::COLS; c += 32)
                qres[c] = (c0 + c < m) ? a.db[qoff + c0 + c] : kPadCode;
            __syncwarp();
            for (int i = lane; i < kProfRows * G::COLS; i += 32) {
                const int x = i / G::COLS, c = i - x * G::COLS;
                const int ln = c / R, k = c - ln * R;
                const int q = qres[c];
                int s = kSpad;                    // +o: the DP keeps H - o as its diagonal input
                if (x != kPadCode && q != kPadCode)
                    s = (P.swap ? s_mat[x * kAlpha + q] : s_mat[q * kAlpha + x]) + o;
                prof[x * G::ROWW + ln * G::LS + k] = s;
            }
            __syncwarp();
            D32Best r;
            dp32_pass<R, G::LS, false>(prof + lane * G::LS, a.db + xoff, n, false, o, ge,
                                       pass > 0 ? bnd : nullptr,
                                       pass + 1 < npass ? bnd : nullptr,
                                       (int32_t)c0 + lane * R, no_wait, no_publish, r);
            result = max(result, r.b);
        }
        if (lane == 0) a.out[P.slot] = result;
    }
}

// ---- alignment cells: score plus the first row-major cell reaching it, one warp per job ----
// Rows stream the job's first sequence a[0..m) (reversed when J.reverse), columns hold its
// second sequence b[0..n) (reversed likewise); cell scores are matrix[a residue][b residue].
// The passes keep the largest score, then the smallest row, then the smallest column.
template <int R>
__global__ void __launch_bounds__(32) cells_wf_kernel(const __grid_constant__ SwArgs a,
                                                     const CellJob* __restrict__ jobs,
                                                     int32_t njobs, int32_t* counter,
                                                     int32_t* __restrict__ res)
{
    using G = Geo<R>;
    extern __shared__ __align__(16) uint8_t smem[];
    int32_t* prof = reinterpret_cast<int32_t*>(smem);
    uint8_t* qres = smem + (size_t)G::PROF_WORDS * 4;
    __shared__ int16_t s_mat[kAlpha * kAlpha];
    const int lane = threadIdx.x;
    for (int i = lane; i < kAlpha * kAlpha; i += 32) s_mat[i] = a.mat[i];
    __syncwarp();
    const int o = a.gap_open, ge = a.gap_extend;
    int2* bnd = reinterpret_cast<int2*>(a.bnd + (int64_t)blockIdx.x * a.bnd_stride);
    auto no_wait = [](int32_t) { return true; };
    auto no_publish = [](int32_t) {};

    for (;;) {
        int p = 0;
        if (lane == 0) p = atomicAdd(counter, 1);
        p = __shfl_sync(kFull, p, 0);
        if (p >= njobs) break;
        const CellJob J = jobs[p];
        const uint8_t* ra = a.db + a.off[J.a];
        const uint8_t* cb = a.db + a.off[J.b];
        int64_t m = J.m;
        const int64_t n = J.n;
        const int npass = (n <= G::COLS) ? 1 : (int)((n + G::COLS - 1) / G::COLS);
        if ((npass > 1 && m > a.bnd_stride) || m >= ((int64_t)1 << 30)) {
            if (lane == 0) atomicExch(a.err, 1);
            m = 0;
        }
        int32_t gbest = 0, grow = -1, gcol = -1;
        for (int pass = 0; pass < npass && m > 0 && n > 0; ++pass) {
            const int64_t c0 = (int64_t)pass * G::COLS;
            __syncwarp();
            for (int c = lane; c < G::COLS; c += 32) {
                const int64_t cc = c0 + c;
                qres[c] = (cc < n) ? (J.reverse ? cb[n - 1 - cc] : cb[cc]) : kPadCode;
            }
            __syncwarp();
            for (int i = lane; i < kProfRows * G::COLS; i += 32) {
                const int x = i / G::COLS, c = i - x * G::COLS;
                const int ln = c / R, k = c - ln * R;
                const int q = qres[c];
                prof[x * G::ROWW + ln * G::LS + k] =
                    (x != kPadCode && q != kPadCode) ? s_mat[x * kAlpha + q] + o : kSpad;
            }
            __syncwarp();
            D32Best r;
            dp32_pass<R, G::LS, true>(prof + lane * G::LS, ra, m, J.reverse != 0, o, ge,
                                      pass > 0 ? bnd : nullptr, pass + 1 < npass ? bnd : nullptr,
                                      (int32_t)c0 + lane * R, no_wait, no_publish, r);
            if (first_max(r.b, r.r, r.c, gbest, grow, gcol)) { gbest = r.b; grow = r.r; gcol = r.c; }
        }
        if (lane == 0) {
            res[3 * (int64_t)p] = gbest;
            res[3 * (int64_t)p + 1] = gbest > 0 ? grow : -1;
            res[3 * (int64_t)p + 2] = gbest > 0 ? gcol : -1;
        }
    }
}

}  // namespace
}  // namespace cm
