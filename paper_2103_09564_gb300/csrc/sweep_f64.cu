// Instantiations of the fused PCG sweep (see sweep_kernel.cuh).
#include "sweep_kernel.cuh"

namespace rwk {

cudaError_t sweep_launch_d64_u16(int tile, const SweepArgs& a, int grid, cudaStream_t s) {
    switch (tile) {
    case 3:
        k_sweep<double, uint16_t, 40, 8, 320><<<grid, 320, sweep_planes_bytes<double>(528), s>>>(a);
        return cudaGetLastError();
    case 7:
        k_sweep<double, uint16_t, 32, 8, 256><<<grid, 256, sweep_planes_bytes<double>(432), s>>>(a);
        return cudaGetLastError();
    default:
        return cudaErrorInvalidValue;
    }
}

cudaError_t sweep_prepare_d64_u16(int tile) {
    switch (tile) {
    case 3:
        return cudaFuncSetAttribute(k_sweep<double, uint16_t, 40, 8, 320>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    sweep_planes_bytes<double>(528));
    case 7:
        return cudaFuncSetAttribute(k_sweep<double, uint16_t, 32, 8, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    sweep_planes_bytes<double>(432));
    default:
        return cudaErrorInvalidValue;
    }
}

cudaError_t sweep_launch_d64_f32(int tile, const SweepArgs& a, int grid, cudaStream_t s) {
    switch (tile) {
    case 3:
        k_sweep<double, float, 40, 8, 320><<<grid, 320, sweep_planes_bytes<double>(528), s>>>(a);
        return cudaGetLastError();
    case 7:
        k_sweep<double, float, 32, 8, 256><<<grid, 256, sweep_planes_bytes<double>(432), s>>>(a);
        return cudaGetLastError();
    default:
        return cudaErrorInvalidValue;
    }
}

cudaError_t sweep_prepare_d64_f32(int tile) {
    switch (tile) {
    case 3:
        return cudaFuncSetAttribute(k_sweep<double, float, 40, 8, 320>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    sweep_planes_bytes<double>(528));
    case 7:
        return cudaFuncSetAttribute(k_sweep<double, float, 32, 8, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    sweep_planes_bytes<double>(432));
    default:
        return cudaErrorInvalidValue;
    }
}

int sweep_occupancy_d64_u16(int tile) {
    int n = 0;
    switch (tile) {
    case 3:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<double, uint16_t, 40, 8, 320>, 320,
                                                      sweep_planes_bytes<double>(528));
        break;
    case 7:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<double, uint16_t, 32, 8, 256>, 256,
                                                      sweep_planes_bytes<double>(432));
        break;
    default:
        break;
    }
    return n;
}

int sweep_occupancy_d64_f32(int tile) {
    int n = 0;
    switch (tile) {
    case 3:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<double, float, 40, 8, 320>, 320,
                                                      sweep_planes_bytes<double>(528));
        break;
    case 7:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<double, float, 32, 8, 256>, 256,
                                                      sweep_planes_bytes<double>(432));
        break;
    default:
        break;
    }
    return n;
}

}  // namespace rwk
