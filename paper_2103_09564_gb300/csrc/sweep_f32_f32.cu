// Instantiations of the fused PCG sweep (see sweep_kernel.cuh).
#include "sweep_kernel.cuh"

namespace rwk {

cudaError_t sweep_launch_f32_f32(int tile, const SweepArgs& a, int grid, cudaStream_t s) {
    switch (tile) {
    case 1:
        k_sweep<float, float, 32, 16, 512><<<grid, 512, sweep_planes_bytes<float>(720), s>>>(a);
        return cudaGetLastError();
    case 2:
        k_sweep<float, float, 64, 8, 512><<<grid, 512, sweep_planes_bytes<float>(816), s>>>(a);
        return cudaGetLastError();
    case 3:
        k_sweep<float, float, 40, 8, 320><<<grid, 320, sweep_planes_bytes<float>(528), s>>>(a);
        return cudaGetLastError();
    case 4:
        k_sweep<float, float, 40, 20, 800><<<grid, 800, sweep_planes_bytes<float>(1056), s>>>(a);
        return cudaGetLastError();
    case 5:
        k_sweep<float, float, 80, 8, 640><<<grid, 640, sweep_planes_bytes<float>(1008), s>>>(a);
        return cudaGetLastError();
    case 6:
        k_sweep<float, float, 80, 16, 640><<<grid, 640, sweep_planes_bytes<float>(1680), s>>>(a);
        return cudaGetLastError();
    case 7:
        k_sweep<float, float, 32, 8, 256><<<grid, 256, sweep_planes_bytes<float>(432), s>>>(a);
        return cudaGetLastError();
    default:
        return cudaErrorInvalidValue;
    }
}

cudaError_t sweep_prepare_f32_f32(int tile) {
    switch (tile) {
    case 1:
        return cudaFuncSetAttribute(k_sweep<float, float, 32, 16, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    sweep_planes_bytes<float>(720));
    case 2:
        return cudaFuncSetAttribute(k_sweep<float, float, 64, 8, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    sweep_planes_bytes<float>(816));
    case 3:
        return cudaFuncSetAttribute(k_sweep<float, float, 40, 8, 320>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    sweep_planes_bytes<float>(528));
    case 4:
        return cudaFuncSetAttribute(k_sweep<float, float, 40, 20, 800>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    sweep_planes_bytes<float>(1056));
    case 5:
        return cudaFuncSetAttribute(k_sweep<float, float, 80, 8, 640>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    sweep_planes_bytes<float>(1008));
    case 6:
        return cudaFuncSetAttribute(k_sweep<float, float, 80, 16, 640>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    sweep_planes_bytes<float>(1680));
    case 7:
        return cudaFuncSetAttribute(k_sweep<float, float, 32, 8, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    sweep_planes_bytes<float>(432));
    default:
        return cudaErrorInvalidValue;
    }
}

int sweep_occupancy_f32_f32(int tile) {
    int n = 0;
    switch (tile) {
    case 1:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<float, float, 32, 16, 512>, 512,
                                                      sweep_planes_bytes<float>(720));
        break;
    case 2:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<float, float, 64, 8, 512>, 512,
                                                      sweep_planes_bytes<float>(816));
        break;
    case 3:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<float, float, 40, 8, 320>, 320,
                                                      sweep_planes_bytes<float>(528));
        break;
    case 4:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<float, float, 40, 20, 800>, 800,
                                                      sweep_planes_bytes<float>(1056));
        break;
    case 5:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<float, float, 80, 8, 640>, 640,
                                                      sweep_planes_bytes<float>(1008));
        break;
    case 6:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<float, float, 80, 16, 640>, 640,
                                                      sweep_planes_bytes<float>(1680));
        break;
    case 7:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep<float, float, 32, 8, 256>, 256,
                                                      sweep_planes_bytes<float>(432));
        break;
    default:
        break;
    }
    return n;
}

}  // namespace rwk
