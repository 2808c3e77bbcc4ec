// Instantiations of the int16x2 Smith-Waterman kernel for CTAs of 8 warps (one translation
// unit per CTA width keeps the parallel build short).
#include "sw16_kernel.cuh"

namespace cm {
namespace {

template <int R, bool TWO>
cudaError_t launch_one(int grid, const SwArgs& a, cudaStream_t st)
{
    const int smem = Geo<R>::PROF_WORDS * 4 + 2 * Geo<R>::COLS;
    cudaError_t e = cudaFuncSetAttribute(sw16_kernel<R, 8, TWO>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    sw16_kernel<R, 8, TWO><<<grid, 8 * 32, smem, st>>>(a);
    return cudaGetLastError();
}

template <int R>
int occ_one()
{
    const int smem = Geo<R>::PROF_WORDS * 4 + 2 * Geo<R>::COLS;
    int n = 1 << 30;
    for (int two = 0; two < 2; ++two) {
        auto f = two ? sw16_kernel<R, 8, true> : sw16_kernel<R, 8, false>;
        if (cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) !=
            cudaSuccess)
            return 1;
        int m = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, f, 8 * 32, smem) != cudaSuccess)
            return 1;
        n = std::min(n, m);
    }
    return n;
}

}  // namespace

#define CM_R_CASES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) \
                      X(14) X(15) X(16) X(17) X(18) X(19) X(20) X(21) X(22) X(23) X(24) \
                      X(25) X(26) X(27) X(28) X(29) X(30) X(31) X(32)

cudaError_t launch_sw16_w8(int R, bool two, int grid, const SwArgs& a, cudaStream_t st)
{
    switch (R) {
#define CM_CASE(r) case r: return two ? launch_one<r, true>(grid, a, st) : launch_one<r, false>(grid, a, st);
    CM_R_CASES(CM_CASE)
#undef CM_CASE
    default: return cudaErrorInvalidValue;
    }
}

int sw16_occ_w8(int R)
{
    switch (R) {
#define CM_CASE(r) case r: return occ_one<r>();
    CM_R_CASES(CM_CASE)
#undef CM_CASE
    default: return 1;
    }
}

}  // namespace cm
