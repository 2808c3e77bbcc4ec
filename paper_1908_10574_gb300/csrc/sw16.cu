// Launchers of the Smith-Waterman kernels (templates in sw16_kernel.cuh): the int16x2 kernel
// dispatch by CTA width, the int32 rescoring kernel and the alignment-cells kernel.
#include "sw16_kernel.cuh"

namespace cm {

#define CM_DECL(w, m)                                                                     \
    cudaError_t launch_sw16_w##w##_m##m(int R, int grid, const SwArgs& a, cudaStream_t st); \
    int sw16_occ_w##w##_m##m(int R);
CM_DECL(4, 0) CM_DECL(4, 1) CM_DECL(4, 2) CM_DECL(4, 3)
CM_DECL(8, 0) CM_DECL(8, 1) CM_DECL(8, 2) CM_DECL(8, 3)
CM_DECL(16, 0) CM_DECL(16, 1) CM_DECL(16, 2) CM_DECL(16, 3)
#undef CM_DECL

int sw16_ctas_per_sm(int R, int W, int mode)
{
#define CM_OCC_CASE(w)                                                                   \
    case w:                                                                              \
        return mode == kModePair ? sw16_occ_w##w##_m0(R)                                 \
               : mode == kModeTwo ? sw16_occ_w##w##_m1(R)                                \
               : mode == kModeSeg16 ? sw16_occ_w##w##_m2(R) : sw16_occ_w##w##_m3(R);
    switch (W) {
    CM_OCC_CASE(4)
    CM_OCC_CASE(8)
    CM_OCC_CASE(16)
    default: return 1;
    }
#undef CM_OCC_CASE
}

int sw32_ctas_per_sm()
{
    const int smem = sw32_smem_bytes(16);
    if (cudaFuncSetAttribute(sw32_kernel<16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem) != cudaSuccess)
        return 1;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sw32_kernel<16>, 32, smem) !=
        cudaSuccess)
        return 1;
    return n;
}

cudaError_t launch_sw16(int R, int W, int mode, int grid, const SwArgs& a, cudaStream_t st)
{
#define CM_LAUNCH_CASE(w)                                                                \
    case w:                                                                              \
        return mode == kModePair ? launch_sw16_w##w##_m0(R, grid, a, st)                 \
               : mode == kModeTwo ? launch_sw16_w##w##_m1(R, grid, a, st)                \
               : mode == kModeSeg16 ? launch_sw16_w##w##_m2(R, grid, a, st)              \
                                    : launch_sw16_w##w##_m3(R, grid, a, st);
    switch (W) {
    CM_LAUNCH_CASE(4)
    CM_LAUNCH_CASE(8)
    CM_LAUNCH_CASE(16)
    default: return cudaErrorInvalidValue;
    }
#undef CM_LAUNCH_CASE
}

int sw32_smem_bytes(int R)
{
    const int LS = lane_stride(R);
    return kProfRows * 32 * LS * 4 + 32 * R;
}

cudaError_t launch_sw32(int R, int grid, const SwArgs& a, const PairRef* pr, int32_t npairs,
                        int32_t* counter, cudaStream_t st)
{
    if (R != 16) return cudaErrorInvalidValue;
    const int smem = sw32_smem_bytes(16);
    cudaError_t e = cudaFuncSetAttribute(sw32_kernel<16>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    sw32_kernel<16><<<grid, 32, smem, st>>>(a, pr, npairs, counter);
    return cudaGetLastError();
}

}  // namespace cm

namespace cm {

int cells_wf_smem_bytes() { return kProfRows * 32 * lane_stride(8) * 4 + 32 * 8; }

int cells_wf_ctas_per_sm()
{
    const int smem = cells_wf_smem_bytes();
    if (cudaFuncSetAttribute(cells_wf_kernel<8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem) != cudaSuccess)
        return 1;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, cells_wf_kernel<8>, 32, smem) !=
        cudaSuccess)
        return 1;
    return n;
}

cudaError_t launch_cells_wf(int grid, const SwArgs& a, const CellJob* jobs, int32_t njobs,
                            int32_t* counter, int32_t* res, cudaStream_t st)
{
    const int smem = cells_wf_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(cells_wf_kernel<8>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    cells_wf_kernel<8><<<grid, 32, smem, st>>>(a, jobs, njobs, counter, res);
    return cudaGetLastError();
}

}  // namespace cm
