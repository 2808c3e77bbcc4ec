// Instantiations of the int16x2 Smith-Waterman kernel for one CTA width (CM_W) and one launch
// mode (CM_MODE), every register tile width R = 1..32.  Each (width, mode) pair is its own
// translation unit so the build runs them in parallel; the including file defines CM_W,
// CM_MODE, CM_LAUNCH and CM_OCC.
#include "sw16_kernel.cuh"

namespace cm {
namespace {

template <int R>
constexpr int inst_smem()
{
    using G = Geo<R, (CM_MODE == kModeSeg16 || CM_MODE == kModeTwo16) ? 16 : 32>;
    return G::PROF_WORDS * 4 + 2 * G::COLS;
}

template <int R>
cudaError_t inst_launch(int grid, const SwArgs& a, cudaStream_t st)
{
    cudaError_t e = cudaFuncSetAttribute(sw16_kernel<R, CM_W, CM_MODE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         inst_smem<R>());
    if (e != cudaSuccess) return e;
    sw16_kernel<R, CM_W, CM_MODE><<<grid, CM_W * 32, inst_smem<R>(), st>>>(a);
    return cudaGetLastError();
}

template <int R>
int inst_occ()
{
    if (cudaFuncSetAttribute(sw16_kernel<R, CM_W, CM_MODE>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, inst_smem<R>()) !=
        cudaSuccess)
        return 1;
    int m = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&m, sw16_kernel<R, CM_W, CM_MODE>,
                                                      CM_W * 32, inst_smem<R>()) != cudaSuccess)
        return 1;
    return m;
}

}  // namespace

// The tile widths each mode can be given: the 32-lane pair mode runs tiles wider than 16
// lanes x 32 columns (R = 17..32); the single-query modes keep <= 16 columns per lane, over 16
// lanes up to 256 residues (R = 1..16) and over 32 lanes in passes above (R = 9..16).
#if CM_MODE == 0
#define CM_R_CASES(X) X(17) X(18) X(19) X(20) X(21) X(22) X(23) X(24) \
                      X(25) X(26) X(27) X(28) X(29) X(30) X(31) X(32)
#elif CM_MODE == 1
#define CM_R_CASES(X) X(9) X(10) X(11) X(12) X(13) X(14) X(15) X(16)
#elif CM_MODE == 3
#define CM_R_CASES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) \
                      X(14) X(15) X(16)
#else
#define CM_R_CASES(X) X(1) X(2) X(3) X(4) X(5) X(6) X(7) X(8) X(9) X(10) X(11) X(12) X(13) \
                      X(14) X(15) X(16) X(17) X(18) X(19) X(20) X(21) X(22) X(23) X(24) \
                      X(25) X(26) X(27) X(28) X(29) X(30) X(31) X(32)
#endif

cudaError_t CM_LAUNCH(int R, int grid, const SwArgs& a, cudaStream_t st)
{
    switch (R) {
#define CM_CASE(r) case r: return inst_launch<r>(grid, a, st);
    CM_R_CASES(CM_CASE)
#undef CM_CASE
    default: return cudaErrorInvalidValue;
    }
}

int CM_OCC(int R)
{
    switch (R) {
#define CM_CASE(r) case r: return inst_occ<r>();
    CM_R_CASES(CM_CASE)
#undef CM_CASE
    default: return 1;
    }
}

}  // namespace cm
