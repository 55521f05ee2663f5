// Instantiations of the fused PCG sweep (see sweep_kernel.cuh).
#include "sweep_kernel.cuh"

namespace rwk {

cudaError_t sweep_launch_f32_u16(int tile, const SweepArgs& a, int grid, cudaStream_t s) {
    switch (tile) {
    case 1:
        k_sweep<float, uint16_t, 32, 16, 512><<<grid, 512, sweep_planes_bytes<float>(720), s>>>(a);
        return cudaGetLastError();
    case 2:
        k_sweep<float, uint16_t, 64, 8, 512><<<grid, 512, sweep_planes_bytes<float>(816), s>>>(a);
        return cudaGetLastError();
    case 7:
        k_sweep<float, uint16_t, 32, 8, 256><<<grid, 256, sweep_planes_bytes<float>(432), s>>>(a);
        return cudaGetLastError();
    default:
        return cudaErrorInvalidValue;
    }
}

cudaError_t sweep_prepare_f32_u16(int tile) {
    switch (tile) {
    case 1:
        return cudaFuncSetAttribute(k_sweep<float, uint16_t, 32, 16, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    sweep_planes_bytes<float>(720));
    case 2:
        return cudaFuncSetAttribute(k_sweep<float, uint16_t, 64, 8, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    sweep_planes_bytes<float>(816));
    case 7:
        return cudaFuncSetAttribute(k_sweep<float, uint16_t, 32, 8, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    sweep_planes_bytes<float>(432));
    default:
        return cudaErrorInvalidValue;
    }
}

int sweep_occupancy_f32_u16(int tile) {
    int n = 0;
    switch (tile) {
    case 1:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<float, uint16_t, 32, 16, 512>, 512,
                                                      sweep_planes_bytes<float>(720));
        break;
    case 2:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<float, uint16_t, 64, 8, 512>, 512,
                                                      sweep_planes_bytes<float>(816));
        break;
    case 7:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<float, uint16_t, 32, 8, 256>, 256,
                                                      sweep_planes_bytes<float>(432));
        break;
    default:
        break;
    }
    return n;
}

}  // namespace rwk
