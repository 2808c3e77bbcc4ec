// Learned representative ranker: a small 1-D convolutional sequence embedding whose dot
// products order and prune the representative comparisons of ClusterMerge; the exact
// Smith-Waterman score alone decides similarity.
//
// Network (per sequence of length L, rows = residues):
//   X0 = E[code]                       (20 x 32 embedding)
//   Z1 = relu(conv9(X0; W1 32->128) + b1)
//   Z2 = relu(conv9(Z1; W2 128->128) + b2)
//   Z3 = conv9(Z2; W3 128->128) + b3
//   v  = mean over the L rows of Z3     (128-d)
//   logit(a, b) = alpha * cos(v_a, v_b) + beta,  loss = BCE(sigmoid(logit), [score > T])
// cm_ranker_standardize rescales W3, b3 so that every output channel of v has zero mean and
// unit variance over a sample of the data (a data-dependent initialisation; without it the
// pooled vectors share one large common component and the cosine hardly separates pairs).
// conv9 is a width-9 "same" convolution.  A batch concatenates its sequences with kGap = 4
// zero rows before, between and after them, so no output row ever reads another sequence.
//
// The convolutions run as implicit GEMMs on the 5th-generation tensor cores (tcgen05.mma,
// BF16 operands staged by TMA, FP32 accumulators in tensor memory; csrc/ranker_tc.cuh):
//   forward      C[r, n]        = sum_k sum_c X[r+k-4, c] * W[k][c][n]
//   backward dX  C[r, c]        = sum_k sum_n dY[r+k-4, n] * W[8-k][c][n]   (flipped weights)
//   backward dW  C[(k, c), n]   = sum_r X[r+k-4, c] * dY[r, n]             (split over rows)
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <random>

#include <cuda_bf16.h>

#include "ctx.h"
#include "ranker_tc.cuh"
#include "train_batches.h"

namespace cm {

typedef __nv_bfloat16 bf16;

constexpr int kGap = 4;
constexpr int kEmb = 32, kCh = 128, kTaps = 9;
// flat fp32 parameter vector layout
constexpr int64_t kOffE = 0;
constexpr int64_t kOffW1 = kOffE + 20 * kEmb;
constexpr int64_t kOffB1 = kOffW1 + (int64_t)kTaps * kEmb * kCh;
constexpr int64_t kOffW2 = kOffB1 + kCh;
constexpr int64_t kOffB2 = kOffW2 + (int64_t)kTaps * kCh * kCh;
constexpr int64_t kOffW3 = kOffB2 + kCh;
constexpr int64_t kOffB3 = kOffW3 + (int64_t)kTaps * kCh * kCh;
constexpr int64_t kOffAlpha = kOffB3 + kCh;
constexpr int64_t kOffBeta = kOffAlpha + 1;
constexpr int64_t kNumParams = kOffBeta + 1;

namespace {

// ---------------------------------------------------------------------------------------
// PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool valid)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)),
                 "l"(src), "r"(valid ? 16 : 0));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_wait0() { asm volatile("cp.async.wait_group 0;\n" ::); }

// sum the per-chunk partials into the gradient vector (first M rows of the padded tile)
__global__ void reduce_parts_kernel(const float* __restrict__ part, int64_t nchunks, int MPAD,
                                    int M, float* __restrict__ grad)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= (int64_t)M * kCh) return;
    float s = 0.f;
    for (int64_t c = 0; c < nchunks; ++c) s += part[c * (int64_t)MPAD * kCh + i];
    grad[i] += s;
}

__global__ void embed_fwd_kernel(const uint8_t* __restrict__ codes, int64_t R,
                                 const bf16* __restrict__ E, bf16* __restrict__ X0)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= R * kEmb) return;
    const int64_t r = i / kEmb;
    const int c = (int)(i % kEmb);
    const uint8_t code = codes[r];
    X0[i] = (code < 20) ? E[code * kEmb + c] : __float2bfloat16(0.f);
}

// pooled vectors from their 64-bit fixed-point sums (units of 2^-32)
__global__ void fixed_to_float_kernel(const unsigned long long* __restrict__ in, int64_t n,
                                      float* __restrict__ out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)((double)(long long)in[i] / kPoolScale);
}

// dY3[r] = dv[s] / len(s) for the real rows r of sequence s, 0 for gap rows (the gradient of
// the mean pooling); one thread per 8 channels of a row
__global__ void pool_bwd_kernel(const float* __restrict__ dv, const int32_t* __restrict__ rowseq,
                                const int32_t* __restrict__ slen, int64_t R, bf16* __restrict__ dZ)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= R * (kCh / 8)) return;
    const int64_t r = i / (kCh / 8);
    const int c0 = (int)(i % (kCh / 8)) * 8;
    const int32_t s = rowseq[r];
    uint32_t w[4] = {0u, 0u, 0u, 0u};
    if (s >= 0) {
        const float inv = 1.f / (float)slen[s];
        const float4 a = *reinterpret_cast<const float4*>(dv + (int64_t)s * kCh + c0);
        const float4 b = *reinterpret_cast<const float4*>(dv + (int64_t)s * kCh + c0 + 4);
        const float f[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const __nv_bfloat162 p = __floats2bfloat162_rn(f[2 * h] * inv, f[2 * h + 1] * inv);
            w[h] = *reinterpret_cast<const uint32_t*>(&p);
        }
    }
    *reinterpret_cast<uint4*>(dZ + r * kCh + c0) = make_uint4(w[0], w[1], w[2], w[3]);
}

// db3[n] += sum over the batch's non-empty sequences of dv[s][n]
// the last layer's bias gradient: the sum over the batch's (non-empty) sequences of dv; one
// block of kDvGroups x kCh threads, group g summing sequences g, g + kDvGroups, ..., then the
// groups' partial sums in a fixed order (deterministic)
constexpr int kDvGroups = 8;

__global__ void __launch_bounds__(kDvGroups * kCh)
dv_sum_kernel(const float* __restrict__ dv, const int32_t* __restrict__ slen, int64_t ns,
              float* __restrict__ db)
{
    __shared__ float part[kDvGroups][kCh];
    const int n = threadIdx.x % kCh, g = threadIdx.x / kCh;
    float t = 0.f;
    for (int64_t s = g; s < ns; s += kDvGroups)
        if (slen[s] > 0) t += dv[s * kCh + n];
    part[g][n] = t;
    __syncthreads();
    if (g == 0) {
        float u = 0.f;
#pragma unroll
        for (int k = 0; k < kDvGroups; ++k) u += part[k][n];
        db[n] += u;
    }
}

// one warp per pair: logit = alpha * cos(v_a, v_b) + beta, the loss and the gradients of v,
// alpha and beta; cos = <a, b> / sqrt((|a|^2 + eps)(|b|^2 + eps))
constexpr float kCosEps = 1e-6f;

__global__ void head_kernel(const float* __restrict__ v, const int32_t* __restrict__ pidx,
                            const float* __restrict__ y, int32_t npairs, const float* __restrict__ ab,
                            float* __restrict__ logits, float* __restrict__ dv,
                            float* __restrict__ gab, float* __restrict__ loss, int backward)
{
    const int lane = threadIdx.x & 31;
    const int64_t p = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (p >= npairs) return;
    const int32_t ia = pidx[2 * p], ib = pidx[2 * p + 1];
    const float* va = v + (int64_t)ia * kCh;
    const float* vb = v + (int64_t)ib * kCh;
    float d = 0.f, na = 0.f, nb = 0.f;
    for (int n = lane; n < kCh; n += 32) {
        d += va[n] * vb[n];
        na += va[n] * va[n];
        nb += vb[n] * vb[n];
    }
    for (int o = 16; o; o >>= 1) {
        d += __shfl_xor_sync(0xffffffffu, d, o);
        na += __shfl_xor_sync(0xffffffffu, na, o);
        nb += __shfl_xor_sync(0xffffffffu, nb, o);
    }
    const float qa = na + kCosEps, qb = nb + kCosEps;
    const float inv = rsqrtf(qa * qb);
    const float cs = d * inv;
    const float alpha = ab[0], beta = ab[1];
    const float z = alpha * cs + beta;
    if (lane == 0 && logits) logits[p] = z;
    if (!backward) return;
    const float yy = y[p];
    const float pr = 1.f / (1.f + expf(-z));
    const float l = fmaxf(z, 0.f) - z * yy + log1pf(expf(-fabsf(z)));   // stable BCE
    const float gz = (pr - yy) / (float)npairs;
    if (lane == 0) {
        atomicAdd(loss, l / (float)npairs);
        atomicAdd(&gab[0], gz * cs);
        atomicAdd(&gab[1], gz);
    }
    // d cos / d a = b * inv - cos * a / qa   (and symmetrically for b)
    const float ga = gz * alpha;
    for (int n = lane; n < kCh; n += 32) {
        atomicAdd(&dv[(int64_t)ia * kCh + n], ga * (vb[n] * inv - cs * va[n] / qa));
        atomicAdd(&dv[(int64_t)ib * kCh + n], ga * (va[n] * inv - cs * vb[n] / qb));
    }
}

__global__ void gather_rows_kernel(const uint8_t* __restrict__ db, const int64_t* __restrict__ off,
                                   const int32_t* __restrict__ sid, const int64_t* __restrict__ srow,
                                   const int32_t* __restrict__ slen, int32_t nseq,
                                   uint8_t* __restrict__ codes, int32_t* __restrict__ rowseq)
{
    const int s = blockIdx.x;
    if (s >= nseq) return;
    const uint8_t* src = db + off[sid[s]];
    const int64_t r0 = srow[s];
    for (int i = threadIdx.x; i < slen[s]; i += blockDim.x) {
        codes[r0 + i] = src[i];
        rowseq[r0 + i] = s;
    }
}

// bf16 copies of one conv layer's weight W[k][c][n] (cin inputs) as the two K-major GEMM
// operands: forward WF[n][k*cin + c] = W[k][c][n]; backward-data WB[c][k*128 + n] = W[8-k][c][n]
__device__ __forceinline__ void store_weight_operands(int64_t i, int cin, bf16 b, bf16* WF,
                                                      bf16* WB)
{
    const int k = (int)(i / ((int64_t)cin * kCh));
    const int c = (int)((i / kCh) % cin);
    const int n = (int)(i % kCh);
    WF[(int64_t)n * kTaps * cin + k * cin + c] = b;
    WB[(int64_t)c * kTaps * kCh + (kTaps - 1 - k) * kCh + n] = b;
}

struct Bf16Copies {
    bf16 *E, *W1, *W1T, *W2, *W2T, *W3, *W3T;
};

// Adam step on every parameter, then the bf16 operand copies of the embedding and conv weights
__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, int64_t n, float lr,
                            float b1, float b2, float eps, float bc1, float bc2, Bf16Copies out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    w[i] = wi;
    const bf16 b = __float2bfloat16(wi);
    if (i < kOffW1) out.E[i - kOffE] = b;
    else if (i < kOffB1) store_weight_operands(i - kOffW1, kEmb, b, out.W1, out.W1T);
    else if (i >= kOffW2 && i < kOffB2) store_weight_operands(i - kOffW2, kCh, b, out.W2, out.W2T);
    else if (i >= kOffW3 && i < kOffB3) store_weight_operands(i - kOffW3, kCh, b, out.W3, out.W3T);
}

// bf16 GEMM operands of a conv layer's W[k][c][n] (see store_weight_operands)
__global__ void cast_weights_kernel(const float* __restrict__ W, int cin, bf16* __restrict__ WF,
                                    bf16* __restrict__ WB)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < (int64_t)kTaps * cin * kCh) store_weight_operands(i, cin, __float2bfloat16(W[i]), WF, WB);
}

__global__ void cast_kernel(const float* __restrict__ x, bf16* __restrict__ y, int64_t n)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) y[i] = __float2bfloat16(x[i]);
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// U[i] = bf16(v_i / sqrt(|v_i|^2 + eps)), so that alpha * <U_a, U_b> + beta is the logit
__global__ void unit_rows_kernel(const float* __restrict__ V, int64_t n, bf16* __restrict__ U)
{
    const int lane = threadIdx.x & 31;
    const int64_t i = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (i >= n) return;
    float q = 0.f;
    for (int c = lane; c < kCh; c += 32) q += V[i * kCh + c] * V[i * kCh + c];
    for (int o = 16; o; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    const float inv = rsqrtf(q + kCosEps);
    for (int c = lane; c < kCh; c += 32) U[i * kCh + c] = __float2bfloat16(V[i * kCh + c] * inv);
}

// Pair selection: for every tile (128 A rows x 128 B rows of a block) the logits
// alpha * <U_a, U_b> + beta on the tensor cores (tcgen05.mma, M = N = 128, K = 128 in eight
// steps of 16, FP32 accumulator in TMEM) and the bits of the pairs at or above `thr`.  The
// rows are gathered by index with cp.async into the 128-byte-swizzled K-major layout the MMA
// reads (16-byte chunk c of row r at chunk position c ^ (r & 7), two 64-channel halves of
// 16 KB per operand), made visible to the tensor core's proxy by a proxy fence.  Tiles start
// at multiples of 128 columns, so every thread (one A row) ORs whole bitmap words.
__global__ void __launch_bounds__(128) pairsel_tc_kernel(const bf16* __restrict__ U,
                                                         const int32_t* __restrict__ rows,
                                                         const SelTile* __restrict__ tiles,
                                                         const float* __restrict__ ab, float thr,
                                                         uint32_t* __restrict__ bitmap,
                                                         int32_t* err)
{
    constexpr uint32_t IDESC = tc::idesc_bf16_f32(128, 128, false, false);
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = reinterpret_cast<uint8_t*>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    uint8_t* sA = smem;                   // [2 halves][128 rows][128 B]
    uint8_t* sB = smem + 32768;
    __shared__ __align__(8) uint64_t done;
    __shared__ uint32_t tmem_slot;
    const SelTile T = tiles[blockIdx.x];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (tid == 0) {
        tc::mbar_init(&done, 1);
        tc::fence_mbar_init();
    }
    if (warp == 2) tc::tmem_alloc(&tmem_slot, 128);
    // gather: 128 rows x 16 chunks of 16 bytes per operand
    for (int id = tid; id < 128 * 16; id += 128) {
        const int i = id >> 4, c16 = id & 15, h = c16 >> 3, c = c16 & 7;
        const uint32_t dst = (uint32_t)(h * 16384 + i * 128 + ((c ^ (i & 7)) << 4));
        const bool oka = i < T.na, okb = i < T.nb;
        const int32_t ra = oka ? rows[T.a + i] : 0, rb = okb ? rows[T.b + i] : 0;
        cp_async16(sA + dst, U + (int64_t)ra * kCh + c16 * 8, oka);
        cp_async16(sB + dst, U + (int64_t)rb * kCh + c16 * 8, okb);
    }
    cp_commit();
    cp_wait0();
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_slot;
    if (tid == 32) {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int off = (k >> 2) * 16384 + (k & 3) * 32;
            tc::mma_bf16(tmem, tc::smem_desc(sA + off, 16, 1024, tc::kSwizzle128),
                         tc::smem_desc(sB + off, 16, 1024, tc::kSwizzle128), IDESC, k != 0);
        }
        tc::mma_commit(&done);
    }
    __syncwarp();
    const bool ok = tc::mbar_wait(&done, 0, err);
    tc::fence_after_sync();
    if (__all_sync(0xffffffffu, ok)) {
        const float alpha = ab[0], beta = ab[1];
        const int i = warp * 32 + lane;
#pragma unroll 1
        for (int ch = 0; ch < 4; ++ch) {
            float v[32];
            tc::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(ch * 32), v);
            uint32_t mask = 0;
#pragma unroll
            for (int q = 0; q < 32; ++q)
                if (ch * 32 + q < T.nb && alpha * v[q] + beta >= thr) mask |= 1u << q;
            if (i < T.na && mask)
                atomicOr(&bitmap[T.bits + (int64_t)(T.i0 + i) * T.words + ((T.j0 + ch * 32) >> 5)], mask);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 2) tc::tmem_free(tmem, 128);
}

constexpr int kPairselSmem = 65536 + 1024;

}  // namespace

// ---------------------------------------------------------------------------------------
// Host side
struct Ranker {
    float* params = nullptr;      // fp32 master (kNumParams)
    float* grad = nullptr;
    float* m = nullptr;
    float* v = nullptr;
    bf16* E = nullptr;
    bf16* W1 = nullptr; bf16* W1T = nullptr;   // forward / backward-data GEMM operands
    bf16* W2 = nullptr; bf16* W2T = nullptr;
    bf16* W3 = nullptr; bf16* W3T = nullptr;
    int32_t* tc_err = nullptr;                  // error word of the tensor-core kernels
    int64_t step = 0;
    bool ready = false;
    // activation buffers (grown on demand)
    DevBuf act[24];
};

enum ActId { A_CODES, A_ROWSEQ, A_X0, A_Z1, A_Z2, A_DZ, A_DY2, A_PART, A_V, A_DV,
             A_SEQ, A_PIDX, A_Y, A_LOGIT, A_EP_SID, A_EP_SROW, A_EP_SLEN, A_EP_PIDX, A_EP_Y,
             A_V64 };

namespace {

int act_ensure(cm_ctx* c, Ranker* K, int id, size_t bytes, void** out)
{
    DevBuf& b = K->act[id];
    if (bytes < 256) bytes = 256;
    if (bytes > b.cap) {
        if (b.p) { cudaStreamSynchronize(c->stream); cudaFree(b.p); }
        const size_t want = std::max(bytes, b.cap + b.cap / 2);
        b.p = nullptr;
        b.cap = 0;
        cudaError_t e = cudaMalloc(&b.p, want);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(c, CM_ERR_OOM, "ranker activation allocation failed");
        }
        b.cap = want;
    }
    *out = b.p;
    return CM_OK;
}

#define AENSURE(id, bytes, ptr)                                                             \
    do {                                                                                    \
        void* p_;                                                                           \
        int r_ = act_ensure(c, K, id, (size_t)(bytes), &p_);                                \
        if (r_) return r_;                                                                  \
        ptr = reinterpret_cast<decltype(ptr)>(p_);                                          \
    } while (0)

void ranker_free(void* p)
{
    Ranker* K = static_cast<Ranker*>(p);
    if (!K) return;
    cudaFree(K->params); cudaFree(K->grad); cudaFree(K->m); cudaFree(K->v);
    cudaFree(K->E); cudaFree(K->W1); cudaFree(K->W1T); cudaFree(K->W2); cudaFree(K->W2T);
    cudaFree(K->W3); cudaFree(K->W3T); cudaFree(K->tc_err);
    for (auto& b : K->act) if (b.p) cudaFree(b.p);
    delete K;
}

int get_ranker(cm_ctx* c, Ranker** out)
{
    if (!c->ranker) {
        Ranker* K = new (std::nothrow) Ranker();
        if (!K) return fail(c, CM_ERR_OOM, "host allocation failed");
        const size_t nb = kNumParams * sizeof(float);
        const size_t w1 = (size_t)kTaps * kEmb * kCh * sizeof(bf16);
        const size_t w2 = (size_t)kTaps * kCh * kCh * sizeof(bf16);
        const std::pair<void**, size_t> bufs[] = {
            {(void**)&K->params, nb}, {(void**)&K->grad, nb}, {(void**)&K->m, nb},
            {(void**)&K->v, nb}, {(void**)&K->E, 20 * kEmb * sizeof(bf16)},
            {(void**)&K->W1, w1}, {(void**)&K->W1T, w1}, {(void**)&K->W2, w2},
            {(void**)&K->W2T, w2}, {(void**)&K->W3, w2}, {(void**)&K->W3T, w2},
            {(void**)&K->tc_err, 256}};
        cudaError_t e = cudaSuccess;
        for (const auto& b : bufs)
            if (e == cudaSuccess) e = cudaMalloc(b.first, b.second);
        if (e != cudaSuccess) {
            // no half-built ranker stays on the context: a later call starts over
            cudaGetLastError();
            ranker_free(K);
            return fail(c, CM_ERR_OOM, std::string("device allocation of the ranker failed: ") +
                                           cudaGetErrorString(e));
        }
        e = cudaMemset(K->tc_err, 0, 256);
        if (e != cudaSuccess) {
            ranker_free(K);
            return fail(c, CM_ERR_CUDA, std::string("cudaMemset failed: ") + cudaGetErrorString(e));
        }
        c->ranker = K;
        c->ranker_free = ranker_free;
    }
    *out = static_cast<Ranker*>(c->ranker);
    return CM_OK;
}

int refresh_bf16(cm_ctx* c, Ranker* K)
{
    const cudaStream_t st = c->stream;
    cast_kernel<<<blocks_for(20 * kEmb, 256), 256, 0, st>>>(K->params + kOffE, K->E, 20 * kEmb);
    cast_weights_kernel<<<blocks_for((int64_t)kTaps * kEmb * kCh, 256), 256, 0, st>>>(
        K->params + kOffW1, kEmb, K->W1, K->W1T);
    cast_weights_kernel<<<blocks_for((int64_t)kTaps * kCh * kCh, 256), 256, 0, st>>>(
        K->params + kOffW2, kCh, K->W2, K->W2T);
    cast_weights_kernel<<<blocks_for((int64_t)kTaps * kCh * kCh, 256), 256, 0, st>>>(
        K->params + kOffW3, kCh, K->W3, K->W3T);
    CUDA_TRY(cudaGetLastError());
    c->stats.launches += 4;
    return CM_OK;
}

// A batch of distinct sequences laid out as rows with kGap zero rows around each.
struct Batch {
    std::vector<int32_t> sid;     // sequence ids
    std::vector<int64_t> srow;    // first row of each sequence
    std::vector<int32_t> slen;
    int64_t R = 0;
};

void layout(const Prepared& P, const int32_t* ids, int64_t n, Batch& B)
{
    B.sid.assign(ids, ids + n);
    B.srow.resize((size_t)n);
    B.slen.resize((size_t)n);
    int64_t r = kGap;
    for (int64_t i = 0; i < n; ++i) {
        B.srow[i] = r;
        B.slen[i] = (int32_t)P.len(ids[i]);
        r += B.slen[i] + kGap;
    }
    B.R = r;
}

// One tensor-core convolution launch (csrc/ranker_tc.cuh): X is R x CIN bf16, Wk the layer's
// NOUT x 9*CIN K-major operand; tensor maps are encoded on the host for these buffers.
template <int CIN, int NOUT, int EPI>
int conv_tc(cm_ctx* c, Ranker* K, const bf16* X, int64_t R, const bf16* Wk, const ConvEpi& ep)
{
    using C = tc::ConvCfg<CIN, NOUT>;
    const int64_t tiles = blocks_for(R, tc::kTcRows);
    if (tiles == 0) return CM_OK;
    CUtensorMap ta, tb;
    CUDA_TRY(tc::make_tmap_bf16(&ta, X, CIN, (uint64_t)R, C::BK, C::AROWS));
    CUDA_TRY(tc::make_tmap_bf16(&tb, Wk, kTaps * CIN, NOUT, C::BK, NOUT));
    auto kern = tc::conv_tc_kernel<CIN, NOUT, EPI>;
    CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    // persistent: one CTA per SM over the 128-row tiles
    const int grid = (int)std::min<int64_t>(tiles, std::max(1, c->num_sms));
    kern<<<grid, tc::kConvThreads, C::SMEM, c->stream>>>(ta, tb, R, ep, K->tc_err);
    CUDA_TRY(cudaGetLastError());
    c->stats.launches += 1;
    return CM_OK;
}

// the tensor-core kernels' error word (a bounded wait gave up): reported and cleared
int check_tc(cm_ctx* c, Ranker* K)
{
    int32_t e = 0;
    CUDA_TRY(cudaMemcpyAsync(&e, K->tc_err, 4, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (e) {
        CUDA_TRY(cudaMemsetAsync(K->tc_err, 0, 4, c->stream));
        return fail(c, CM_ERR_TIMEOUT, "a tensor-core GEMM's bounded wait gave up");
    }
    return CM_OK;
}

// forward over a batch whose layout (sequence ids, first rows, lengths; R rows) is on the
// device; leaves X0, Z1, Z2, Z3 and the pooled vectors V on the device
int forward_dev(cm_ctx* c, const Prepared& P, Ranker* K, const int32_t* d_sid,
                const int64_t* d_srow, const int32_t* d_slen, int64_t ns, int64_t R, float** V_out)
{
    const cudaStream_t st = c->stream;
    uint8_t* codes; int32_t* rowseq; bf16 *X0, *Z1, *Z2; float* V; unsigned long long* V64;
    AENSURE(A_CODES, R, codes);
    AENSURE(A_ROWSEQ, R * 4, rowseq);
    AENSURE(A_X0, R * kEmb * 2, X0);
    AENSURE(A_Z1, R * kCh * 2, Z1);
    AENSURE(A_Z2, R * kCh * 2, Z2);
    AENSURE(A_V, ns * kCh * 4, V);
    AENSURE(A_V64, ns * kCh * 8, V64);
    int r;
    CUDA_TRY(cudaMemsetAsync(codes, 0xff, R, st));
    CUDA_TRY(cudaMemsetAsync(rowseq, 0xff, R * 4, st));
    CUDA_TRY(cudaMemsetAsync(V64, 0, ns * kCh * 8, st));
    gather_rows_kernel<<<(unsigned)ns, 128, 0, st>>>(P.db, P.off, d_sid, d_srow, d_slen, (int32_t)ns,
                                                     codes, rowseq);
    embed_fwd_kernel<<<blocks_for(R * kEmb, 256), 256, 0, st>>>(codes, R, K->E, X0);
    CUDA_TRY(cudaGetLastError());
    c->stats.launches += 2;
    ConvEpi ep{};
    ep.rowseq = rowseq;
    ep.bias = K->params + kOffB1;
    ep.out = Z1;
    if ((r = conv_tc<kEmb, kCh, kEpiRelu>(c, K, X0, R, K->W1, ep))) return r;
    ep.bias = K->params + kOffB2;
    ep.out = Z2;
    if ((r = conv_tc<kCh, kCh, kEpiRelu>(c, K, Z1, R, K->W2, ep))) return r;
    // layer 3 is pooled in its epilogue: v = mean over a sequence's rows of conv(Z2) + b3
    ep.bias = K->params + kOffB3;
    ep.out = nullptr;
    ep.slen = d_slen;
    ep.acc64 = V64;
    if ((r = conv_tc<kCh, kCh, kEpiPool>(c, K, Z2, R, K->W3, ep))) return r;
    fixed_to_float_kernel<<<blocks_for(ns * kCh, 256), 256, 0, st>>>(V64, ns * kCh, V);
    CUDA_TRY(cudaGetLastError());
    c->stats.launches += 1;
    *V_out = V;
    return CM_OK;
}

// forward over a batch laid out on the host
int forward(cm_ctx* c, const Prepared& P, Ranker* K, const Batch& B, float** V_out)
{
    const int64_t ns = (int64_t)B.sid.size();
    int32_t* seqinfo;
    AENSURE(A_SEQ, ns * 16 + 64, seqinfo);
    int32_t* d_sid = seqinfo;
    int64_t* d_srow = reinterpret_cast<int64_t*>(seqinfo + ((ns + 1) & ~1LL));
    int32_t* d_slen = reinterpret_cast<int32_t*>(d_srow + ns);
    int r;
    if ((r = copy_in(c, d_sid, B.sid.data(), ns * 4, false))) return r;
    if ((r = copy_in(c, d_srow, B.srow.data(), ns * 8, false))) return r;
    if ((r = copy_in(c, d_slen, B.slen.data(), ns * 4, false))) return r;
    return forward_dev(c, P, K, d_sid, d_srow, d_slen, ns, B.R, V_out);
}

// weight gradient of a conv layer on the tensor cores: the rows are cut into chunks so that
// the grid (m-tiles x chunks) fills about two CTAs per SM; the chunks' partial tiles are
// summed in a second kernel (deterministic)
template <int CIN>
int wgrad(cm_ctx* c, Ranker* K, const bf16* X, const bf16* dY, int64_t R, float* dW)
{
    using C = tc::WgradCfg<CIN>;
    const int M = kTaps * CIN;
    const int mtiles = C::MTILES, MPAD = mtiles * 128;
    // chunks of rows: about one CTA per SM over all m-tiles (each CTA a long K loop)
    const int64_t want = std::max<int64_t>(1, (int64_t)c->num_sms / mtiles);
    const int64_t steps = (R + C::BKR - 1) / C::BKR;
    const int64_t rpc = ((steps + want - 1) / want) * C::BKR;
    const int64_t nch = (R + rpc - 1) / rpc;
    float* part;
    AENSURE(A_PART, nch * MPAD * kCh * 4, part);
    CUtensorMap tx, td;
    CUDA_TRY(tc::make_tmap_bf16(&tx, X, CIN, (uint64_t)R, C::CW, C::BKR));
    CUDA_TRY(tc::make_tmap_bf16(&td, dY, kCh, (uint64_t)R, 64, C::BKR));
    auto kern = tc::wgrad_tc_kernel<CIN>;
    CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
    kern<<<dim3(mtiles, (unsigned)nch), 128, C::SMEM, c->stream>>>(tx, td, rpc, part, MPAD,
                                                                   K->tc_err);
    reduce_parts_kernel<<<blocks_for((int64_t)M * kCh, 256), 256, 0, c->stream>>>(part, nch, MPAD, M, dW);
    CUDA_TRY(cudaGetLastError());
    c->stats.launches += 2;
    return CM_OK;
}

// Training batches packed for the device: per batch its distinct sequences (in order of first
// appearance) with their first rows and lengths (rows relative to the batch, kGap zero rows
// around each), the pairs as indices into that list, and the labels.
struct Packed {
    std::vector<int32_t> sid, slen, pidx;
    std::vector<int64_t> srow;
    std::vector<float> y;
    std::vector<int64_t> seq_off{0}, pair_off{0}, rows;
    std::vector<int32_t> stamp, local;   // per sequence: last batch that listed it, its index
};

void pack_batch(const Prepared& P, int32_t n_seqs, const int32_t* pairs, const float* labels,
                const int64_t* idx, int64_t n, Packed& B)
{
    if ((int64_t)B.stamp.size() != n_seqs) {
        B.stamp.assign((size_t)n_seqs, -1);
        B.local.assign((size_t)n_seqs, 0);
    }
    const int32_t bid = (int32_t)B.rows.size();
    const size_t s0 = B.sid.size();
    int64_t r = kGap;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t k = idx ? idx[i] : i;
        for (int h = 0; h < 2; ++h) {
            const int32_t q = pairs[2 * k + h];
            if (B.stamp[q] != bid) {
                B.stamp[q] = bid;
                B.local[q] = (int32_t)(B.sid.size() - s0);
                B.sid.push_back(q);
                B.srow.push_back(r);
                B.slen.push_back((int32_t)P.len(q));
                r += P.len(q) + kGap;
            }
            B.pidx.push_back(B.local[q]);
        }
        B.y.push_back(labels[k]);
    }
    B.rows.push_back(r);
    B.seq_off.push_back((int64_t)B.sid.size());
    B.pair_off.push_back((int64_t)B.y.size());
}

// upload every packed batch's arrays (one copy each)
struct PackedDev {
    int32_t *sid, *slen, *pidx;
    int64_t* srow;
    float* y;
};

int upload_packed(cm_ctx* c, Ranker* K, const Packed& B, PackedDev& D)
{
    const int64_t ns = (int64_t)B.sid.size(), np = (int64_t)B.y.size();
    AENSURE(A_EP_SID, ns * 4, D.sid);
    AENSURE(A_EP_SLEN, ns * 4, D.slen);
    AENSURE(A_EP_SROW, ns * 8, D.srow);
    AENSURE(A_EP_PIDX, np * 8, D.pidx);
    AENSURE(A_EP_Y, np * 4 + 64, D.y);
    int r;
    if ((r = copy_in(c, D.sid, B.sid.data(), ns * 4, false))) return r;
    if ((r = copy_in(c, D.slen, B.slen.data(), ns * 4, false))) return r;
    if ((r = copy_in(c, D.srow, B.srow.data(), ns * 8, false))) return r;
    if ((r = copy_in(c, D.pidx, B.pidx.data(), np * 8, false))) return r;
    return copy_in(c, D.y, B.y.data(), np * 4, false);
}

// loss and gradient (accumulated into K->grad, which the caller zeroes) of packed batch b
int loss_grad_packed(cm_ctx* c, const Prepared& P, Ranker* K, const Packed& B, const PackedDev& D,
                     size_t b, float* loss_out)
{
    const cudaStream_t st = c->stream;
    const int64_t so = B.seq_off[b], ns = B.seq_off[b + 1] - so;
    const int64_t po = B.pair_off[b], npairs = B.pair_off[b + 1] - po;
    const int64_t R = B.rows[b];
    const int32_t* d_slen = D.slen + so;
    float* V;
    int r = forward_dev(c, P, K, D.sid + so, D.srow + so, d_slen, ns, R, &V);
    if (r) return r;
    const int32_t* d_pidx = D.pidx + 2 * po;
    const float* d_y = D.y + po;
    float *dv, *d_loss;
    AENSURE(A_DV, ns * kCh * 4, dv);
    AENSURE(A_LOGIT, 64, d_loss);
    CUDA_TRY(cudaMemsetAsync(dv, 0, ns * kCh * 4, st));
    CUDA_TRY(cudaMemsetAsync(d_loss, 0, 4, st));
    head_kernel<<<blocks_for(npairs * 32, 256), 256, 0, st>>>(V, d_pidx, d_y, (int32_t)npairs,
                                                              K->params + kOffAlpha, nullptr, dv,
                                                              K->grad + kOffAlpha, d_loss, 1);
    uint8_t* codes = (uint8_t*)K->act[A_CODES].p;
    int32_t* rowseq = (int32_t*)K->act[A_ROWSEQ].p;
    bf16* X0 = (bf16*)K->act[A_X0].p;
    bf16* Z1 = (bf16*)K->act[A_Z1].p;
    bf16* Z2 = (bf16*)K->act[A_Z2].p;
    bf16 *dZ, *dY2;
    AENSURE(A_DZ, R * kCh * 2, dZ);
    AENSURE(A_DY2, R * kCh * 2, dY2);
    pool_bwd_kernel<<<blocks_for(R * (kCh / 8), 256), 256, 0, st>>>(dv, rowseq, d_slen, R, dZ);  // dY3
    // b3's gradient: every real row of a sequence carries dv / len, so the rows sum to dv
    dv_sum_kernel<<<1, kDvGroups * kCh, 0, st>>>(dv, d_slen, ns, K->grad + kOffB3);
    c->stats.launches += 2;
    ConvEpi ep{};
    ep.rowseq = rowseq;
    // layer 3 (linear): W3's gradient, then dY2 = gate(Z2) * conv^T(dY3) with b2's gradient
    if ((r = wgrad<kCh>(c, K, Z2, dZ, R, K->grad + kOffW3))) return r;
    ep.gate = Z2;
    ep.out = dY2;
    ep.acc = K->grad + kOffB2;
    if ((r = conv_tc<kCh, kCh, kEpiGate>(c, K, dZ, R, K->W3T, ep))) return r;
    // layer 2: W2's gradient, then dY1 = gate(Z1) * conv^T(dY2) with b1's gradient
    if ((r = wgrad<kCh>(c, K, Z1, dY2, R, K->grad + kOffW2))) return r;
    ep.gate = Z1;
    ep.out = dZ;
    ep.acc = K->grad + kOffB1;
    if ((r = conv_tc<kCh, kCh, kEpiGate>(c, K, dY2, R, K->W2T, ep))) return r;
    // layer 1: W1's gradient, then the embedding table's gradient from conv^T(dY1)
    if ((r = wgrad<kEmb>(c, K, X0, dZ, R, K->grad + kOffW1))) return r;
    ep.gate = nullptr;
    ep.out = nullptr;
    ep.codes = codes;
    ep.acc = K->grad + kOffE;
    if ((r = conv_tc<kCh, kEmb, kEpiEmbed>(c, K, dZ, R, K->W1T, ep))) return r;
    if (loss_out) {
        CUDA_TRY(cudaMemcpyAsync(loss_out, d_loss, 4, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        if ((r = check_tc(c, K))) return r;
    }
    return CM_OK;
}

}  // namespace

// pooled 128-d vectors of `n` sequences (host ids) into device memory V (n x 128, fp32)
int ranker_embed_device(cm_ctx* c, const Prepared& P, const int32_t* ids, int64_t n, float* V)
{
    Ranker* K;
    int r = get_ranker(c, &K);
    if (r) return r;
    if (!K->ready) return fail(c, CM_ERR_ARG, "ranker has no parameters (init, train or load first)");
    const int64_t max_rows = (int64_t)1 << 22;   // activation budget per chunk
    int64_t i = 0;
    while (i < n) {
        int64_t j = i, rows = kGap;
        while (j < n && (j == i || rows + P.len(ids[j]) + kGap <= max_rows)) {
            rows += P.len(ids[j]) + kGap;
            ++j;
        }
        Batch B;
        layout(P, ids + i, j - i, B);
        float* Vc;
        if ((r = forward(c, P, K, B, &Vc))) return r;
        CUDA_TRY(cudaMemcpyAsync(V + i * kCh, Vc, (j - i) * kCh * 4, cudaMemcpyDeviceToDevice,
                                 c->stream));
        i = j;
    }
    return check_tc(c, K);
}

int ranker_alpha_beta(cm_ctx* c, float* ab)
{
    Ranker* K;
    int r = get_ranker(c, &K);
    if (r) return r;
    CUDA_TRY(cudaMemcpy(ab, K->params + kOffAlpha, 8, cudaMemcpyDeviceToHost));
    return CM_OK;
}

// Bitmaps of the (A row, B row) pairs of every tile whose ranker logit reaches thr.
int ranker_select(cm_ctx* c, const void* Uv, const std::vector<int32_t>& rows,
                  const std::vector<SelTile>& tiles, float thr, int64_t nwords,
                  std::vector<uint32_t>& bitmap, const uint32_t** d_bits_out,
                  const int32_t** d_rows_out)
{
    const bf16* U = static_cast<const bf16*>(Uv);
    bitmap.assign((size_t)nwords, 0u);
    if (tiles.empty()) return CM_OK;
    Ranker* K;
    int r = get_ranker(c, &K);
    if (r) return r;
    int32_t* d_rows;
    SelTile* d_tiles;
    uint32_t* d_bits;
    AENSURE(A_PIDX, rows.size() * 4, d_rows);
    AENSURE(A_Y, tiles.size() * sizeof(SelTile), d_tiles);
    AENSURE(A_LOGIT, nwords * 4, d_bits);
    if ((r = copy_in(c, d_rows, rows.data(), rows.size() * 4, false))) return r;
    if ((r = copy_in(c, d_tiles, tiles.data(), tiles.size() * sizeof(SelTile), false))) return r;
    CUDA_TRY(cudaMemsetAsync(d_bits, 0, nwords * 4, c->stream));
    CUDA_TRY(cudaFuncSetAttribute(pairsel_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kPairselSmem));
    for (size_t t0 = 0; t0 < tiles.size(); t0 += 65535) {
        const unsigned nt = (unsigned)std::min<size_t>(65535, tiles.size() - t0);
        pairsel_tc_kernel<<<nt, 128, kPairselSmem, c->stream>>>(U, d_rows, d_tiles + t0,
                                                                K->params + kOffAlpha, thr,
                                                                d_bits, K->tc_err);
        c->stats.launches += 1;
    }
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(bitmap.data(), d_bits, nwords * 4, cudaMemcpyDeviceToHost, c->stream));
    if ((r = check_tc(c, K))) return r;
    if (d_bits_out) *d_bits_out = d_bits;
    if (d_rows_out) *d_rows_out = d_rows;
    return CM_OK;
}

// unit rows U (bf16, n x 128) of the ranker vectors of all n sequences, in device memory
int ranker_unit_vectors(cm_ctx* c, const Prepared& P, int64_t n, void** U_out)
{
    Ranker* K;
    int r = get_ranker(c, &K);
    if (r) return r;
    float* V;
    bf16* U;
    void* pv;
    if ((r = ensure_bytes(c, B_RES, (size_t)n * kCh * 4, &pv))) return r;
    V = static_cast<float*>(pv);
    std::vector<int32_t> ids((size_t)n);
    std::iota(ids.begin(), ids.end(), 0);
    if ((r = ranker_embed_device(c, P, ids.data(), n, V))) return r;
    if ((r = ensure_bytes(c, B_SCRATCH, (size_t)n * kCh * 2, &pv))) return r;
    U = static_cast<bf16*>(pv);
    unit_rows_kernel<<<blocks_for(n * 32, 256), 256, 0, c->stream>>>(V, n, U);
    CUDA_TRY(cudaGetLastError());
    c->stats.launches += 1;
    *U_out = U;
    return CM_OK;
}


}  // namespace cm

using namespace cm;

namespace {

int set_params_host(cm_ctx* c, Ranker* K, const float* h)
{
    CUDA_TRY(cudaMemcpyAsync(K->params, h, kNumParams * 4, cudaMemcpyHostToDevice, c->stream));
    CUDA_TRY(cudaMemsetAsync(K->m, 0, kNumParams * 4, c->stream));
    CUDA_TRY(cudaMemsetAsync(K->v, 0, kNumParams * 4, c->stream));
    K->step = 0;
    int r = refresh_bf16(c, K);
    if (r) return r;
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    K->ready = true;
    return CM_OK;
}

}  // namespace

extern "C" {

int64_t cm_ranker_num_params(void) { return kNumParams; }

int cm_ranker_init(cm_ctx* c, uint64_t seed)
{
    if (!c) return CM_ERR_ARG;
    CUDA_TRY(cudaSetDevice(c->device));
    Ranker* K;
    int r = get_ranker(c, &K);
    if (r) return r;
    std::vector<float> h((size_t)kNumParams, 0.f);
    std::mt19937_64 g(seed);
    std::normal_distribution<float> nd(0.f, 1.f);
    auto fill = [&](int64_t off, int64_t n, float sd) {
        for (int64_t i = 0; i < n; ++i) h[off + i] = nd(g) * sd;
    };
    fill(kOffE, 20 * kEmb, 1.0f);
    fill(kOffW1, (int64_t)kTaps * kEmb * kCh, std::sqrt(2.f / (kTaps * kEmb)));
    fill(kOffW2, (int64_t)kTaps * kCh * kCh, std::sqrt(2.f / (kTaps * kCh)));
    fill(kOffW3, (int64_t)kTaps * kCh * kCh, std::sqrt(1.f / (kTaps * kCh)));
    h[kOffAlpha] = 10.f;
    h[kOffBeta] = -2.f;
    return set_params_host(c, K, h.data());
}

int cm_ranker_set_params(cm_ctx* c, const float* params, int64_t n)
{
    if (!c || !params || n != kNumParams) return c ? fail(c, CM_ERR_ARG, "expected cm_ranker_num_params() floats") : CM_ERR_ARG;
    CUDA_TRY(cudaSetDevice(c->device));
    Ranker* K;
    int r = get_ranker(c, &K);
    if (r) return r;
    return set_params_host(c, K, params);
}

int cm_ranker_get_params(cm_ctx* c, float* params, int64_t n)
{
    if (!c || !params || n != kNumParams) return c ? fail(c, CM_ERR_ARG, "expected cm_ranker_num_params() floats") : CM_ERR_ARG;
    Ranker* K;
    int r = get_ranker(c, &K);
    if (r) return r;
    if (!K->ready) return fail(c, CM_ERR_ARG, "ranker has no parameters");
    CUDA_TRY(cudaMemcpy(params, K->params, kNumParams * 4, cudaMemcpyDeviceToHost));
    return CM_OK;
}

// file layout: tag, parameter count, parameters (all little-endian, as the host stores them:
// the supported hosts, x86-64 and Arm64, are little-endian)
static const char kRankerTag[8] = {'C', 'M', 'R', 'A', 'N', 'K', '0', '1'};

int cm_ranker_save(cm_ctx* c, const char* path)
{
    if (!c) return CM_ERR_ARG;
    if (!path) return fail(c, CM_ERR_ARG, "null path");
    std::vector<float> h((size_t)kNumParams);
    int r = cm_ranker_get_params(c, h.data(), kNumParams);
    if (r) return r;
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(c, CM_ERR_ARG, std::string("cannot write ") + path);
    const int64_t n = kNumParams;
    const bool ok = std::fwrite(kRankerTag, 1, 8, f) == 8 && std::fwrite(&n, 8, 1, f) == 1 &&
                    std::fwrite(h.data(), 4, h.size(), f) == h.size();
    if (std::fclose(f) != 0 || !ok) return fail(c, CM_ERR_ARG, std::string("write failed: ") + path);
    return CM_OK;
}

int cm_ranker_load(cm_ctx* c, const char* path)
{
    if (!c) return CM_ERR_ARG;
    if (!path) return fail(c, CM_ERR_ARG, "null path");
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(c, CM_ERR_ARG, std::string("cannot read ") + path);
    char tag[8];
    int64_t n = 0;
    std::vector<float> h((size_t)kNumParams);
    bool ok = std::fread(tag, 1, 8, f) == 8 && std::memcmp(tag, kRankerTag, 8) == 0 &&
              std::fread(&n, 8, 1, f) == 1 && n == kNumParams &&
              std::fread(h.data(), 4, h.size(), f) == h.size();
    char extra;
    ok = ok && std::fread(&extra, 1, 1, f) == 0;      // nothing after the parameters
    std::fclose(f);
    if (!ok) return fail(c, CM_ERR_ARG, std::string("not a ranker parameter file: ") + path);
    return cm_ranker_set_params(c, h.data(), kNumParams);
}

int cm_ranker_loss_grad(cm_ctx* c, const uint8_t* seqs, const int64_t* offsets, int32_t n_seqs,
                        const int32_t* pairs, const float* labels, int64_t n_pairs,
                        float* loss, float* grad, uint32_t flags)
{
    if (!c) return CM_ERR_ARG;
    CUDA_TRY(cudaSetDevice(c->device));
    if (flags & CM_DEVICE_PTRS) return fail(c, CM_ERR_ARG, "host pointers only");
    if (n_pairs < 1 || !pairs || !labels || !loss) return fail(c, CM_ERR_ARG, "bad pairs");
    Prepared P;
    int r = prepare_seqs(c, seqs, offsets, n_seqs, flags, P);
    if (r) return r;
    for (int64_t k = 0; k < 2 * n_pairs; ++k)
        if (pairs[k] < 0 || pairs[k] >= n_seqs) return fail(c, CM_ERR_ARG, "pair index out of range");
    Ranker* K;
    if ((r = get_ranker(c, &K))) return r;
    if (!K->ready) return fail(c, CM_ERR_ARG, "ranker has no parameters");
    CUDA_TRY(cudaMemsetAsync(K->grad, 0, kNumParams * 4, c->stream));
    Packed B;
    pack_batch(P, n_seqs, pairs, labels, nullptr, n_pairs, B);
    PackedDev D;
    if ((r = upload_packed(c, K, B, D))) return r;
    if ((r = loss_grad_packed(c, P, K, B, D, 0, loss))) return r;
    if (grad) CUDA_TRY(cudaMemcpy(grad, K->grad, kNumParams * 4, cudaMemcpyDeviceToHost));
    return CM_OK;
}

int cm_ranker_train(cm_ctx* c, const uint8_t* seqs, const int64_t* offsets, int32_t n_seqs,
                    const int32_t* pairs, const float* labels, int64_t n_pairs, int32_t epochs,
                    int32_t batch_pairs, float lr, uint64_t seed, float* last_loss, uint32_t flags)
{
    if (!c) return CM_ERR_ARG;
    CUDA_TRY(cudaSetDevice(c->device));
    if (flags & CM_DEVICE_PTRS) return fail(c, CM_ERR_ARG, "host pointers only");
    if (n_pairs < 1 || !pairs || !labels || epochs < 1 || batch_pairs < 1 || !(lr > 0.f))
        return fail(c, CM_ERR_ARG, "bad training arguments");
    Prepared P;
    int r = prepare_seqs(c, seqs, offsets, n_seqs, flags, P);
    if (r) return r;
    for (int64_t k = 0; k < 2 * n_pairs; ++k)
        if (pairs[k] < 0 || pairs[k] >= n_seqs) return fail(c, CM_ERR_ARG, "pair index out of range");
    Ranker* K;
    if ((r = get_ranker(c, &K))) return r;
    if (!K->ready) return fail(c, CM_ERR_ARG, "ranker has no parameters (call cm_ranker_init)");
    // mini-batches (csrc/train_batches.h): shuffled chunks, or with CM_TRAIN_COMPONENTS whole
    // components of the pair graph; a step embeds each distinct sequence of its batch once
    const TrainComponents comps = (flags & CM_TRAIN_COMPONENTS)
                                      ? train_components(pairs, n_pairs, n_seqs)
                                      : train_one_component(n_pairs);
    std::mt19937_64 g(seed);
    std::vector<int64_t> order, bounds;
    float loss = 0.f;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const Bf16Copies copies{K->E, K->W1, K->W1T, K->W2, K->W2T, K->W3, K->W3T};
    int64_t total_steps = 0, t_step = 0;      // for CM_TRAIN_COSINE (batches per epoch are fixed)
    for (int ep = 0; ep < epochs; ++ep) {
        // the whole epoch's batches go to the device in one copy per array
        train_epoch_batches(comps, batch_pairs, g, order, bounds);
        const int64_t nb = (int64_t)bounds.size() - 1;
        if (ep == 0) total_steps = nb * (int64_t)epochs;
        Packed B;
        for (int64_t bi = 0; bi < nb; ++bi)
            pack_batch(P, n_seqs, pairs, labels, order.data() + bounds[bi],
                       bounds[bi + 1] - bounds[bi], B);
        PackedDev D;
        if ((r = upload_packed(c, K, B, D))) return r;
        for (int64_t bi = 0; bi < nb; ++bi) {
            CUDA_TRY(cudaMemsetAsync(K->grad, 0, kNumParams * 4, c->stream));
            const bool last = (ep == epochs - 1) && (bi == nb - 1);
            if ((r = loss_grad_packed(c, P, K, B, D, (size_t)bi, last ? &loss : nullptr))) return r;
            ++K->step;
            const float bc1 = 1.f - std::pow(b1, (float)K->step), bc2 = 1.f - std::pow(b2, (float)K->step);
            float lr_t = lr;
            if (flags & CM_TRAIN_COSINE) {
                const double T_ = (double)std::max<int64_t>(total_steps, 1);
                const double warm = std::min(1.0, (double)(t_step + 1) / std::max(1.0, 0.02 * T_));
                lr_t = (float)(lr * warm * 0.5 * (1.0 + std::cos(3.141592653589793 * (double)t_step / T_)));
            }
            ++t_step;
            adam_kernel<<<blocks_for(kNumParams, 256), 256, 0, c->stream>>>(
                K->params, K->grad, K->m, K->v, kNumParams, lr_t, b1, b2, eps, bc1, bc2, copies);
            CUDA_TRY(cudaGetLastError());
            c->stats.launches += 1;
        }
    }
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    if ((r = check_tc(c, K))) return r;
    if (last_loss) *last_loss = loss;
    return CM_OK;
}

int cm_ranker_standardize(cm_ctx* c, const uint8_t* seqs, const int64_t* offsets,
                          int32_t n_seqs, int32_t max_sample, uint32_t flags)
{
    if (!c) return CM_ERR_ARG;
    CUDA_TRY(cudaSetDevice(c->device));
    if (flags & CM_DEVICE_PTRS) return fail(c, CM_ERR_ARG, "host pointers only");
    if (n_seqs < 2 || max_sample < 2) return fail(c, CM_ERR_ARG, "need at least 2 sequences");
    Prepared P;
    int r = prepare_seqs(c, seqs, offsets, n_seqs, flags, P);
    if (r) return r;
    Ranker* K;
    if ((r = get_ranker(c, &K))) return r;
    if (!K->ready) return fail(c, CM_ERR_ARG, "ranker has no parameters");
    // evenly spaced sample of the set
    const int64_t ns = std::min<int64_t>(n_seqs, max_sample);
    std::vector<int32_t> ids((size_t)ns);
    for (int64_t i = 0; i < ns; ++i) ids[i] = (int32_t)(i * (int64_t)n_seqs / ns);
    void* pv;
    if ((r = ensure_bytes(c, B_RES, (size_t)ns * kCh * 4, &pv))) return r;
    if ((r = ranker_embed_device(c, P, ids.data(), ns, static_cast<float*>(pv)))) return r;
    std::vector<float> V((size_t)ns * kCh);
    CUDA_TRY(cudaMemcpyAsync(V.data(), pv, V.size() * 4, cudaMemcpyDeviceToHost, c->stream));
    std::vector<float> h((size_t)kNumParams);
    CUDA_TRY(cudaMemcpyAsync(h.data(), K->params, kNumParams * 4, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    for (int n = 0; n < kCh; ++n) {
        double mu = 0, sq = 0;
        for (int64_t i = 0; i < ns; ++i) mu += V[i * kCh + n];
        mu /= (double)ns;
        for (int64_t i = 0; i < ns; ++i) sq += (V[i * kCh + n] - mu) * (V[i * kCh + n] - mu);
        const double sd = std::sqrt(sq / (double)(ns - 1)) + 1e-6;
        for (int64_t q = 0; q < (int64_t)kTaps * kCh; ++q) h[kOffW3 + q * kCh + n] /= (float)sd;
        h[kOffB3 + n] = (float)((h[kOffB3 + n] - mu) / sd);
    }
    return set_params_host(c, K, h.data());
}

int cm_ranker_logits(cm_ctx* c, const uint8_t* seqs, const int64_t* offsets, int32_t n_seqs,
                     const int32_t* pairs, int64_t n_pairs, float* out, uint32_t flags)
{
    if (!c) return CM_ERR_ARG;
    CUDA_TRY(cudaSetDevice(c->device));
    if (flags & CM_DEVICE_PTRS) return fail(c, CM_ERR_ARG, "host pointers only");
    if (n_pairs < 0 || (n_pairs > 0 && (!pairs || !out))) return fail(c, CM_ERR_ARG, "bad pairs");
    Prepared P;
    int r = prepare_seqs(c, seqs, offsets, n_seqs, flags, P);
    if (r) return r;
    if (n_pairs == 0) return CM_OK;
    for (int64_t k = 0; k < 2 * n_pairs; ++k)
        if (pairs[k] < 0 || pairs[k] >= n_seqs) return fail(c, CM_ERR_ARG, "pair index out of range");
    Ranker* K;
    if ((r = get_ranker(c, &K))) return r;
    if (!K->ready) return fail(c, CM_ERR_ARG, "ranker has no parameters");
    std::vector<int32_t> uniq(pairs, pairs + 2 * n_pairs);
    std::sort(uniq.begin(), uniq.end());
    uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
    std::vector<int32_t> pidx((size_t)n_pairs * 2);
    for (int64_t i = 0; i < 2 * n_pairs; ++i)
        pidx[i] = (int32_t)(std::lower_bound(uniq.begin(), uniq.end(), pairs[i]) - uniq.begin());
    const int64_t ns = (int64_t)uniq.size();
    void* pv;
    if ((r = ensure_bytes(c, B_RES, (size_t)ns * kCh * 4, &pv))) return r;
    float* V = static_cast<float*>(pv);
    if ((r = ranker_embed_device(c, P, uniq.data(), ns, V))) return r;
    int32_t* d_pidx;
    float* d_logit;
    AENSURE(A_PIDX, n_pairs * 8, d_pidx);
    AENSURE(A_LOGIT, n_pairs * 4, d_logit);
    if ((r = copy_in(c, d_pidx, pidx.data(), n_pairs * 8, false))) return r;
    head_kernel<<<blocks_for(n_pairs * 32, 256), 256, 0, c->stream>>>(
        V, d_pidx, nullptr, (int32_t)n_pairs, K->params + kOffAlpha, d_logit, nullptr, nullptr,
        nullptr, 0);
    CUDA_TRY(cudaGetLastError());
    c->stats.launches += 1;
    CUDA_TRY(cudaMemcpyAsync(out, d_logit, n_pairs * 4, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return CM_OK;
}

int cm_ranker_embed(cm_ctx* c, const uint8_t* seqs, const int64_t* offsets, int32_t n_seqs,
                    float* out, uint32_t flags)
{
    if (!c) return CM_ERR_ARG;
    CUDA_TRY(cudaSetDevice(c->device));
    if (!out && n_seqs > 0) return fail(c, CM_ERR_ARG, "null out");
    Prepared P;
    int r = prepare_seqs(c, seqs, offsets, n_seqs, flags, P);
    if (r) return r;
    if (n_seqs == 0) return CM_OK;
    std::vector<int32_t> ids((size_t)n_seqs);
    std::iota(ids.begin(), ids.end(), 0);
    float* V = out;
    const bool dev = (flags & CM_DEVICE_PTRS) != 0;
    if (!dev) {
        void* p;
        if ((r = ensure_bytes(c, B_RES, (size_t)n_seqs * kCh * 4, &p))) return r;
        V = static_cast<float*>(p);
    }
    if ((r = ranker_embed_device(c, P, ids.data(), n_seqs, V))) return r;
    if (!dev) CUDA_TRY(cudaMemcpyAsync(out, V, (size_t)n_seqs * kCh * 4, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    return CM_OK;
}

}  // extern "C"
