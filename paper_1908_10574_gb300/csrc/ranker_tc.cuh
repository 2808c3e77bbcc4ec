// The ranker's width-9 convolutions as implicit GEMMs on the 5th-generation tensor cores
// (tcgen05.mma, BF16 operands, FP32 accumulator in tensor memory).  Rows are the residues of
// a batch's concatenated sequences (with zero gap rows between them), channels are contiguous.
//
// conv_tc_kernel<CIN, NOUT, EPI>: out[r, n] = sum_t sum_c X[r + t - 4, c] * Wk[n, t*CIN + c]
//   (forward: Wk[n, t*CIN + c] = W[t][c][n]; backward-data: X = dY, Wk[c, t*128 + n] =
//   W[8-t][c][n]).  A tile is 128 rows x NOUT channels: K runs over the 9 taps x CIN channels
//   in stages of BK channels; a stage's A tile is the 128 rows starting at r0 + t - 4, loaded
//   by TMA straight from the activation matrix (rows before 0 or past the end come back as
//   zeros), and its B tile the matching BK columns of Wk.  Persistent: one CTA per SM walks
//   the tiles; one thread streams the stages of every tile through a deep mbarrier ring,
//   one thread issues the MMAs of a tile into one of two TMEM accumulators, and four warps
//   read the other accumulator back and apply the epilogue meanwhile (details below).
// wgrad_tc_kernel<CIN>: part[chunk][m = t*CIN + c][n] = sum over the chunk's rows r of
//   X[r + t - 4, c] * dY[r, n] -- a GEMM whose K runs over rows.  Both operands are read
//   MN-major (channels contiguous, one row per K index), so the tap shift stays on the row
//   coordinate of the TMA load.  One CTA = 128 values of m (one tap of 128 channels, or four
//   taps of 32) x 128 n, over `rows_per_chunk` rows in stages of 64 (about one CTA per SM,
//   each a long K loop through a 6-stage ring).
#pragma once

#include <cuda_bf16.h>

#include "tc_gemm.cuh"

namespace cm {

// Epilogues of conv_tc_kernel (rows whose rowseq is negative are gap rows and give zeros):
//   kEpiRelu   out = bf16(relu(acc + bias))
//   kEpiPool   v[seq] += (acc + bias) / len(seq) for every real row (mean pooling; the
//              pre-pooling activations are never stored).  The sums are kept in 64-bit fixed
//              point (units of 2^-32) so that the atomic adds commute: v does not depend on
//              the order in which CTAs finish, and neither do the ranker's logits.
//   kEpiGate   out = bf16(gate > 0 ? acc : 0), and colsum[n] += the column sums of those
//              values (the bias gradient of the layer below)
//   kEpiEmbed  dE[code][c] += acc for every real row (the embedding table's gradient; dX0 is
//              never stored)
enum Epi : int { kEpiRelu = 0, kEpiPool = 1, kEpiGate = 2, kEpiEmbed = 3 };

struct ConvEpi {
    const float* bias;          // Relu, Pool
    const int32_t* rowseq;      // every mode: sequence index of a row, < 0 for gap rows
    const __nv_bfloat16* gate;  // Gate
    __nv_bfloat16* out;         // Relu, Gate
    const int32_t* slen;        // Pool: rows of every sequence
    const uint8_t* codes;       // Embed: residue code of every row
    float* acc;                 // Gate: column sums; Embed: dE (20 x NOUT)
    unsigned long long* acc64;  // Pool: v (ns x NOUT) in units of 2^-32
};

constexpr double kPoolScale = 4294967296.0;   // 2^32: fixed-point unit of the pooled sums

__device__ __forceinline__ void add_fixed(unsigned long long* p, float v)
{
    atomicAdd(p, (unsigned long long)__double2ll_rn((double)v * kPoolScale));
}

namespace tc {

constexpr int kTcRows = 128;        // rows (M) per CTA

// Column sums of a warp's 32 x 32 tile (lane = row, v[0..31] = columns): a transposing
// reduction (halve the columns a lane keeps at every step, adding the partner lane's copy of
// them), 31 shuffles in all; afterwards lane c holds the sum of column c.  Overwrites v.
__device__ __forceinline__ float warp_colsum32(float* v, int lane)
{
#pragma unroll
    for (int s = 16; s >= 1; s >>= 1) {
        const bool up = (lane & s) != 0;
#pragma unroll
        for (int k = 0; k < s; ++k) {
            const float keep = up ? v[k + s] : v[k];
            const float give = up ? v[k] : v[k + s];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, give, s);
        }
    }
    return v[0];
}

// ---- persistent convolution kernel ------------------------------------------------------
// One CTA per SM walks the 128-row tiles blockIdx.x, blockIdx.x + gridDim.x, ...  Warp 0
// (one thread) streams the A / B stages of every tile through a ring of STAGES shared-memory
// stages, across tile boundaries; warp 1 (one thread) issues the MMAs of a tile into one of
// two TMEM accumulators (tile i uses buffer i & 1) and commits it; warps 2-9 read a finished
// accumulator back (warp w owns TMEM lanes 32 (w % 4) .., warps w and w + 4 one half of the
// columns each) and apply the epilogue while the MMAs of the next tile run, then release the
// buffer.  Barriers: full / empty per stage
// (TMA bytes landed / MMAs done reading), tfull / tempty per accumulator (MMAs done /
// epilogue done reading).  Every wait is bounded; a role that gives up sets the error word
// and stops, the others then give up at their next wait, and the teardown waits (bounded) for
// the copies and MMAs still in flight before the tensor memory is freed.
constexpr int kConvEpiWarps = 8;    // two per TMEM lane quadrant, each half of the columns
constexpr int kConvThreads = 64 + 32 * kConvEpiWarps;
constexpr int kConvStageBudget = 192 * 1024;

template <int CIN, int NOUT>
struct ConvCfg {
    static constexpr int BK = (CIN == 32) ? 32 : 64;       // channels per stage = swizzle row
    static constexpr int KB_PER_TAP = CIN / BK;
    static constexpr int NKB = 9 * KB_PER_TAP;
    // AREUSE (128-byte swizzle): a tile's A rows r0 - 4 .. r0 + 131 are loaded once per block
    // of BK channels, and tap t reads them from row t on (the descriptor start moves by whole
    // 128-byte rows; the swizzle follows the address, so the shifted view stays valid);
    // otherwise every stage carries its own 128-row A tile
    static constexpr bool AREUSE = (BK == 64);
    static constexpr int AROWS = AREUSE ? kTcRows + 8 : kTcRows;
    static constexpr int A_BOX_BYTES = AROWS * BK * 2;     // one channel block of a tile
    static constexpr int A_TILE_BYTES = KB_PER_TAP * A_BOX_BYTES;
    static constexpr int A_SLOTS_BYTES = AREUSE ? 2 * A_TILE_BYTES : 0;   // two tiles in flight
    static constexpr int A_BYTES = kTcRows * BK * 2;       // A of a stage (no reuse)
    static constexpr int B_BYTES = NOUT * BK * 2;
    static constexpr int STAGE_BYTES = (AREUSE ? 0 : A_BYTES) + B_BYTES;
    static constexpr int STAGES_FIT = (kConvStageBudget - A_SLOTS_BYTES) / STAGE_BYTES;
    static constexpr int STAGES = STAGES_FIT < 8 ? STAGES_FIT : 8;
    static constexpr uint32_t SWZ = (BK == 64) ? kSwizzle128 : kSwizzle64;
    static constexpr uint32_t SBO = 8 * BK * 2;
    static constexpr uint32_t TMEM_COLS = 2 * NOUT < 32 ? 32 : 2 * NOUT;   // two accumulators
    // the embedding-gradient epilogue's scratch: per epilogue warp a 32 x 33 transpose tile
    // and private bins of 20 codes x NOUT channels
    static constexpr int EMB_FLOATS = 4 * (32 * 33 + 20 * NOUT);
    static constexpr int SMEM = A_SLOTS_BYTES + STAGES * STAGE_BYTES + 1024;
    static_assert(A_BOX_BYTES % 1024 == 0 && STAGE_BYTES % 1024 == 0, "1024-byte aligned tiles");
};

// Epilogue of one accumulator: this thread's row r of the tile (TMEM lane 32 q + lane).
// Embed: lane = channel after a transpose through shared memory, adding into the warp's own
// bins (no atomics); Gate: column sums per warp into s_red (shared atomics, one per column).
template <int CIN, int NOUT, int EPI>
__device__ __forceinline__ void conv_epilogue(uint32_t tacc, int q, int lane, int j0, int j1,
                                              int64_t r0, int64_t R, const ConvEpi& ep,
                                              float* s_red, float* emb)
{
    const int64_t r = r0 + q * 32 + lane;
    const bool in = r < R;
    const int32_t seq = in ? ep.rowseq[r] : -1;
    const bool real = seq >= 0;
    // Pool: a warp whose real rows all belong to one sequence reduces its 32 rows first
    int32_t lead = -1;
    bool one_seq = false;
    float inv_len = 0.f;
    if (EPI == kEpiPool) {
        lead = __reduce_max_sync(0xffffffffu, seq);
        one_seq = __all_sync(0xffffffffu, seq < 0 || seq == lead);
        if (real) inv_len = 1.f / (float)ep.slen[seq];
    }
    // Embed: rows of letters outside the 20 embedded ones (zero embedding) add nothing
    int code = real ? (EPI == kEpiEmbed ? (int)ep.codes[r] : 0) : 0;
    const bool binned = EPI == kEpiEmbed && real && code < 20;
    if (!binned) code = 0;
#pragma unroll 1
    for (int j = j0; j < j1; ++j) {
        float v[32];
        tmem_ld32(tacc + ((uint32_t)(q * 32) << 16) + (uint32_t)(j * 32), v);
        const int n0 = j * 32;
        if (EPI == kEpiEmbed) {
            // transpose the warp's 32 rows x 32 channels, then lane c adds channel c of every
            // row into bin[code of the row][c] of this warp
            float* tile = emb;                                   // [32][33]
            float* bins = emb + 32 * 33;                         // [20][NOUT]
#pragma unroll
            for (int c = 0; c < 32; ++c) tile[c * 33 + lane] = binned ? v[c] : 0.f;
            __syncwarp();
#pragma unroll 4
            for (int rr = 0; rr < 32; ++rr) {
                const int cd = __shfl_sync(0xffffffffu, code, rr);
                bins[cd * NOUT + n0 + lane] += tile[lane * 33 + rr];
            }
            __syncwarp();
            continue;
        }
        if (EPI == kEpiPool) {
#pragma unroll
            for (int t = 0; t < 32; ++t) v[t] = real ? (v[t] + ep.bias[n0 + t]) * inv_len : 0.f;
            if (one_seq) {
                const float t = warp_colsum32(v, lane);
                if (lead >= 0) add_fixed(ep.acc64 + (int64_t)lead * NOUT + n0 + lane, t);
            } else if (real) {
#pragma unroll
                for (int t = 0; t < 32; ++t) add_fixed(ep.acc64 + (int64_t)seq * NOUT + n0 + t, v[t]);
            }
            continue;
        }
        if (EPI == kEpiRelu) {
#pragma unroll
            for (int t = 0; t < 32; ++t) v[t] = fmaxf(v[t] + ep.bias[n0 + t], 0.f);
        } else if (EPI == kEpiGate && in) {
            const uint4* g4 = reinterpret_cast<const uint4*>(ep.gate + r * NOUT + n0);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const uint4 gw = g4[t];
                const uint32_t w[4] = {gw.x, gw.y, gw.z, gw.w};
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const __nv_bfloat162 gz = *reinterpret_cast<const __nv_bfloat162*>(&w[h]);
                    if (!(__bfloat162float(gz.x) > 0.f)) v[8 * t + 2 * h] = 0.f;
                    if (!(__bfloat162float(gz.y) > 0.f)) v[8 * t + 2 * h + 1] = 0.f;
                }
            }
        }
#pragma unroll
        for (int t = 0; t < 32; ++t) v[t] = real ? v[t] : 0.f;
        if (in) {
            uint4* o = reinterpret_cast<uint4*>(ep.out + r * NOUT + n0);
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                uint32_t w[4];
#pragma unroll
                for (int h = 0; h < 4; ++h) {
                    const __nv_bfloat162 pr = __floats2bfloat162_rn(v[8 * t + 2 * h], v[8 * t + 2 * h + 1]);
                    w[h] = *reinterpret_cast<const uint32_t*>(&pr);
                }
                o[t] = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        if (EPI == kEpiGate && ep.acc) {
            const float t = warp_colsum32(v, lane);
            atomicAdd(s_red + n0 + lane, t);
        }
    }
}

template <int CIN, int NOUT, int EPI>
__global__ void __launch_bounds__(kConvThreads, 1)
conv_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               int64_t R, const ConvEpi ep, int32_t* err)
{
    using C = ConvCfg<CIN, NOUT>;
    constexpr int S = C::STAGES;
    constexpr uint32_t IDESC = idesc_bf16_f32(kTcRows, NOUT, false, false);
    // column chunks of 32 per epilogue warp pair; with one chunk only the first four warps
    constexpr int NCH = NOUT / 32;
    constexpr int kEpiActive = NCH >= 2 ? kConvEpiWarps : 4;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full[S], empty[S], afull[2], aempty[2], tfull[2], tempty[2], done;
    __shared__ uint32_t tmem_slot;
    __shared__ int32_t s_issued, s_consumed, s_aissued, s_aconsumed, s_abort;
    __shared__ float s_red[EPI == kEpiGate ? NOUT : 1];
    __shared__ float s_emb[EPI == kEpiEmbed ? C::EMB_FLOATS : 1];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t ntiles = (R + kTcRows - 1) / kTcRows;
    if (EPI == kEpiGate)
        for (int i = threadIdx.x; i < NOUT; i += kConvThreads) s_red[i] = 0.f;
    if (EPI == kEpiEmbed)
        for (int i = threadIdx.x; i < C::EMB_FLOATS; i += kConvThreads) s_emb[i] = 0.f;

    if (threadIdx.x == 0) {
        prefetch_tmap(&tmA);
        prefetch_tmap(&tmB);
        for (int s = 0; s < S; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], kEpiActive);
            mbar_init(&afull[b], 1);
            mbar_init(&aempty[b], 1);
        }
        mbar_init(&done, 1);
        fence_mbar_init();
        s_issued = 0;
        s_consumed = 0;
        s_aissued = 0;
        s_aconsumed = 0;
        s_abort = *reinterpret_cast<volatile int32_t*>(err);   // an earlier launch gave up
    }
    __syncthreads();
    if (s_abort) return;
    if (warp == 1) tmem_alloc(&tmem_slot, C::TMEM_COLS);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_slot;

    uint8_t* bring = smem + C::A_SLOTS_BYTES;                // B (or A + B) stages
    if (warp == 0) {
        if (lane == 0) {
            int it = 0, i = 0;
            bool ok = true;
            for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++i) {
                const int64_t r0 = tile * kTcRows;
                if constexpr (C::AREUSE) {
                    const int a = i & 1;
                    if (i >= 2 && !mbar_wait(&aempty[a], ((i / 2) - 1) & 1, err)) break;
                    uint8_t* as = smem + a * C::A_TILE_BYTES;
                    mbar_expect_tx(&afull[a], C::A_TILE_BYTES);
                    for (int cb = 0; cb < C::KB_PER_TAP; ++cb)
                        tma_load_2d(as + cb * C::A_BOX_BYTES, &tmA, cb * C::BK, (int32_t)(r0 - 4),
                                    &afull[a]);
                }
                for (int kb = 0; kb < C::NKB; ++kb, ++it) {
                    const int s = it % S;
                    if (it >= S && !mbar_wait(&empty[s], ((it / S) - 1) & 1, err)) { ok = false; break; }
                    const int tap = kb / C::KB_PER_TAP, c0 = (kb % C::KB_PER_TAP) * C::BK;
                    uint8_t* st = bring + s * C::STAGE_BYTES;
                    mbar_expect_tx(&full[s], C::STAGE_BYTES);
                    if constexpr (!C::AREUSE) {
                        tma_load_2d(st, &tmA, c0, (int32_t)(r0 + tap - 4), &full[s]);
                        tma_load_2d(st + C::A_BYTES, &tmB, tap * CIN + c0, 0, &full[s]);
                    } else {
                        tma_load_2d(st, &tmB, tap * CIN + c0, 0, &full[s]);
                    }
                }
            }
            s_issued = it;
            s_aissued = i;
        }
    } else if (warp == 1) {
        if (lane == 0) {
            int it = 0, i = 0;
            bool ok = true;
            for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++i) {
                const int b = i & 1;
                if (i >= 2 && !mbar_wait(&tempty[b], ((i / 2) - 1) & 1, err)) break;
                if constexpr (C::AREUSE) {
                    if (!mbar_wait(&afull[i & 1], (i / 2) & 1, err)) break;
                }
                fence_after_sync();
                const uint32_t acc = tmem + (uint32_t)(b * NOUT);
                const uint8_t* as = smem + (i & 1) * C::A_TILE_BYTES;
                for (int kb = 0; kb < C::NKB; ++kb, ++it) {
                    const int s = it % S;
                    if (!mbar_wait(&full[s], (it / S) & 1, err)) { ok = false; break; }
                    fence_after_sync();
                    const uint8_t* st = bring + s * C::STAGE_BYTES;
                    const int tap = kb / C::KB_PER_TAP, cb = kb % C::KB_PER_TAP;
                    const uint8_t* a = C::AREUSE ? as + cb * C::A_BOX_BYTES + tap * (C::BK * 2) : st;
                    const uint8_t* bb = C::AREUSE ? st : st + C::A_BYTES;
#pragma unroll
                    for (int k = 0; k < C::BK / 16; ++k)
                        mma_bf16(acc, smem_desc(a + 32 * k, 16, C::SBO, C::SWZ),
                                 smem_desc(bb + 32 * k, 16, C::SBO, C::SWZ), IDESC, (kb | k) != 0);
                    mma_commit(&empty[s]);
                }
                if (!ok) break;
                if constexpr (C::AREUSE) mma_commit(&aempty[i & 1]);
                mma_commit(&tfull[b]);
            }
            s_consumed = it;
            s_aconsumed = i;
            mma_commit(&done);            // arrives once every MMA issued above has completed
        }
    } else if (warp - 2 < kEpiActive) {
        const int ew = warp - 2;
        const int q = warp & 3;           // TMEM lane quadrant of this warp
        const int half = kEpiActive == 8 ? ew / 4 : 0;
        const int j0 = kEpiActive == 8 ? half * (NCH / 2) : 0;
        const int j1 = kEpiActive == 8 ? (half + 1) * (NCH / 2) : NCH;
        float* emb = s_emb + (EPI == kEpiEmbed ? ew * (32 * 33 + 20 * NOUT) : 0);
        int i = 0;
        for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++i) {
            const int b = i & 1;
            const bool ok = mbar_wait(&tfull[b], (i / 2) & 1, err);
            if (!__all_sync(0xffffffffu, ok)) break;      // warp-uniform: tcgen05.ld is warp-wide
            fence_after_sync();
            conv_epilogue<CIN, NOUT, EPI>(tmem + (uint32_t)(b * NOUT), q, lane, j0, j1,
                                          tile * kTcRows, R, ep, s_red, emb);
            fence_before_sync();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n"
                                        ::"r"(smem_addr(&tempty[b])) : "memory");
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        // MMAs issued but not awaited by an epilogue, and loads issued but never consumed
        // (only after a wait gave up): let them finish before the memory goes away
        mbar_wait(&done, 0, err);
        for (int it = s_consumed; it < s_issued; ++it)
            mbar_wait(&full[it % S], (it / S) & 1, err);
        if (C::AREUSE)
            for (int i = s_aconsumed; i < s_aissued; ++i)
                mbar_wait(&afull[i & 1], (i / 2) & 1, err);
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (EPI == kEpiGate && ep.acc)
        for (int i = threadIdx.x; i < NOUT; i += kConvThreads)
            if (s_red[i] != 0.f) atomicAdd(ep.acc + i, s_red[i]);
    if (EPI == kEpiEmbed) {
        const int per = 32 * 33 + 20 * NOUT;
        for (int i = threadIdx.x; i < 20 * NOUT; i += kConvThreads) {
            float t = 0.f;
#pragma unroll
            for (int w = 0; w < 4; ++w) t += s_emb[w * per + 32 * 33 + i];
            if (t != 0.f) atomicAdd(ep.acc + i, t);
        }
    }
    if (warp == 1) tmem_free(tmem, C::TMEM_COLS);
}

template <int CIN>
struct WgradCfg {
    static constexpr int CW = (CIN == 32) ? 32 : 64;        // channels per swizzle row of A
    static constexpr int A_BOXES = 128 / CW;                // boxes making up M = 128
    static constexpr int BKR = 64;                          // rows (K) per stage
    static constexpr int A_BYTES = 128 * BKR * 2;
    static constexpr int B_BYTES = 128 * BKR * 2;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    static constexpr uint32_t A_SWZ = (CW == 64) ? kSwizzle128 : kSwizzle64;
    static constexpr uint32_t A_ROW = CW * 2;               // bytes per K row of one A box
    static constexpr int STAGES = 6;                       // one CTA per SM, a deep ring
    static constexpr int SMEM = STAGES * STAGE_BYTES + 1024;
    static constexpr int MTILES = (9 * CIN + 127) / 128;
};

template <int CIN>
__global__ void __launch_bounds__(128, 1)
wgrad_tc_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmD,
                int64_t rows_per_chunk, float* __restrict__ part, int MPAD, int32_t* err)
{
    using C = WgradCfg<CIN>;
    constexpr uint32_t IDESC = idesc_bf16_f32(128, 128, true, true);
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full[C::STAGES], empty[C::STAGES], done;
    __shared__ uint32_t tmem_slot;
    __shared__ int32_t s_issued, s_consumed, s_abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mtile = blockIdx.x;
    const int64_t chunk = blockIdx.y;
    const int64_t rbeg = chunk * rows_per_chunk;
    const int nkb = (int)(rows_per_chunk / C::BKR);
    // taps held by this m-tile's A boxes (a box past the last tap is not loaded)
    const int nbox = (CIN == 32) ? min(C::A_BOXES, 9 - 4 * mtile) : C::A_BOXES;
    const uint32_t stage_tx = (uint32_t)(nbox * (C::A_BYTES / C::A_BOXES) + C::B_BYTES);

    if (threadIdx.x == 0) {
        prefetch_tmap(&tmX);
        prefetch_tmap(&tmD);
        for (int s = 0; s < C::STAGES; ++s) { mbar_init(&full[s], 1); mbar_init(&empty[s], 1); }
        mbar_init(&done, 1);
        fence_mbar_init();
        s_issued = 0;
        s_consumed = 0;
        s_abort = *reinterpret_cast<volatile int32_t*>(err);
    }
    __syncthreads();
    if (s_abort) return;
    if (warp == 2) tmem_alloc(&tmem_slot, 128);
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_slot;

    if (warp == 0 && lane == 0) {
        int kb = 0;
        for (; kb < nkb; ++kb) {
            const int s = kb % C::STAGES;
            if (kb >= C::STAGES && !mbar_wait(&empty[s], ((kb / C::STAGES) - 1) & 1, err)) break;
            const int64_t rr = rbeg + (int64_t)kb * C::BKR;
            uint8_t* st = smem + s * C::STAGE_BYTES;
            mbar_expect_tx(&full[s], stage_tx);
            for (int q = 0; q < nbox; ++q) {
                // CIN = 128: tap = mtile, channel half q; CIN = 32: tap 4 mtile + q
                const int tap = (CIN == 32) ? 4 * mtile + q : mtile;
                const int c0 = (CIN == 32) ? 0 : q * 64;
                tma_load_2d(st + q * (C::A_BYTES / C::A_BOXES), &tmX, c0,
                            (int32_t)(rr + tap - 4), &full[s]);
            }
            tma_load_2d(st + C::A_BYTES, &tmD, 0, (int32_t)rr, &full[s]);
            tma_load_2d(st + C::A_BYTES + C::B_BYTES / 2, &tmD, 64, (int32_t)rr, &full[s]);
        }
        s_issued = kb;
    } else if (warp == 1 && lane == 0) {
        int kb = 0;
        for (; kb < nkb; ++kb) {
            const int s = kb % C::STAGES;
            if (!mbar_wait(&full[s], (kb / C::STAGES) & 1, err)) break;
            fence_after_sync();
            const uint8_t* a = smem + s * C::STAGE_BYTES;
            const uint8_t* b = a + C::A_BYTES;
#pragma unroll
            for (int k = 0; k < C::BKR / 16; ++k)
                mma_bf16(tmem,
                         smem_desc(a + 16 * k * C::A_ROW, C::A_BYTES / C::A_BOXES, 8 * C::A_ROW,
                                   C::A_SWZ),
                         smem_desc(b + 16 * k * 128, C::B_BYTES / 2, 1024, kSwizzle128), IDESC,
                         (kb | k) != 0);
            mma_commit(&empty[s]);
        }
        s_consumed = kb;
        mma_commit(&done);
    }
    __syncwarp();
    const bool ok = mbar_wait(&done, 0, err);
    fence_after_sync();
    // warp-uniform: the TMEM loads below are warp-wide instructions
    if (__all_sync(0xffffffffu, ok && *reinterpret_cast<volatile int32_t*>(err) == 0)) {
        const int m = mtile * 128 + warp * 32 + lane;
        float* dst = part + (chunk * (int64_t)MPAD + m) * 128;
#pragma unroll 1
        for (int j = 0; j < 4; ++j) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(j * 32), v);
            float4* o = reinterpret_cast<float4*>(dst + j * 32);
#pragma unroll
            for (int q = 0; q < 8; ++q)
                o[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        }
    }
    fence_before_sync();
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int kb = s_consumed; kb < s_issued; ++kb)
            mbar_wait(&full[kb % C::STAGES], (kb / C::STAGES) & 1, err);
    }
    __syncthreads();
    if (warp == 2) tmem_free(tmem, 128);
}

}  // namespace tc
}  // namespace cm
