// Launchers of the Smith-Waterman kernels (templates in sw16_kernel.cuh): the int16x2 kernel
// dispatch by CTA width, the int32 rescoring kernel and the alignment-cells kernel.
#include "sw16_kernel.cuh"

namespace cm {

cudaError_t launch_sw16_w4(int R, bool two, int grid, const SwArgs& a, cudaStream_t st);
cudaError_t launch_sw16_w8(int R, bool two, int grid, const SwArgs& a, cudaStream_t st);
cudaError_t launch_sw16_w16(int R, bool two, int grid, const SwArgs& a, cudaStream_t st);
int sw16_occ_w4(int R);
int sw16_occ_w8(int R);
int sw16_occ_w16(int R);

int sw16_ctas_per_sm(int R, int W)
{
    switch (W) {
    case 4: return sw16_occ_w4(R);
    case 8: return sw16_occ_w8(R);
    case 16: return sw16_occ_w16(R);
    default: return 1;
    }
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

int sw16_smem_bytes(int R)
{
    const int LS = lane_stride(R);
    return kProfRows * 32 * LS * 4 + 2 * 32 * R;
}

cudaError_t launch_sw16(int R, int W, bool two, int grid, const SwArgs& a, cudaStream_t st)
{
    switch (W) {
    case 4: return launch_sw16_w4(R, two, grid, a, st);
    case 8: return launch_sw16_w8(R, two, grid, a, st);
    case 16: return launch_sw16_w16(R, two, grid, a, st);
    default: return cudaErrorInvalidValue;
    }
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
