// Instantiations of the padded-layout FP32 sweep (see sweep4_kernel.cuh).
#include "sweep4_kernel.cuh"

namespace rwk {

cudaError_t sweep4_launch(int tile, const SweepArgs& a, int grid, cudaStream_t s) {
    switch (tile) {
    case 14:
        k_sweep4<32, 12, 288, 2, 4><<<grid, 288, sweep4_smem_bytes<32, 12, 4>(), s>>>(a);
        return cudaGetLastError();
    case 15:
        k_sweep4<32, 12, 288, 4, 8><<<grid, 288, sweep4_smem_bytes<32, 12, 8>(), s>>>(a);
        return cudaGetLastError();
    case 16:
        k_sweep4<32, 28, 576, 2, 4><<<grid, 576, sweep4_smem_bytes<32, 28, 4>(), s>>>(a);
        return cudaGetLastError();
    case 17:
        k_sweep4<40, 20, 352, 2, 4><<<grid, 352, sweep4_smem_bytes<40, 20, 4>(), s>>>(a);
        return cudaGetLastError();
    case 18:
        k_sweep4<40, 8, 352, 3, 8><<<grid, 352, sweep4_smem_bytes<40, 8, 8>(), s>>>(a);
        return cudaGetLastError();
    case 19:
        k_sweep4<32, 20, 288, 2, 4><<<grid, 288, sweep4_smem_bytes<32, 20, 4>(), s>>>(a);
        return cudaGetLastError();
    default:
        return cudaErrorInvalidValue;
    }
}

cudaError_t sweep4_prepare(int tile) {
    switch (tile) {
    case 14:
        return cudaFuncSetAttribute(k_sweep4<32, 12, 288, 2, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sweep4_smem_bytes<32, 12, 4>());
    case 15:
        return cudaFuncSetAttribute(k_sweep4<32, 12, 288, 4, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sweep4_smem_bytes<32, 12, 8>());
    case 16:
        return cudaFuncSetAttribute(k_sweep4<32, 28, 576, 2, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sweep4_smem_bytes<32, 28, 4>());
    case 17:
        return cudaFuncSetAttribute(k_sweep4<40, 20, 352, 2, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sweep4_smem_bytes<40, 20, 4>());
    case 18:
        return cudaFuncSetAttribute(k_sweep4<40, 8, 352, 3, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sweep4_smem_bytes<40, 8, 8>());
    case 19:
        return cudaFuncSetAttribute(k_sweep4<32, 20, 288, 2, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sweep4_smem_bytes<32, 20, 4>());
    default:
        return cudaErrorInvalidValue;
    }
}

int sweep4_occupancy(int tile) {
    int n = 0;
    switch (tile) {
    case 14:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep4<32, 12, 288, 2, 4>, 288, sweep4_smem_bytes<32, 12, 4>());
        break;
    case 15:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep4<32, 12, 288, 4, 8>, 288, sweep4_smem_bytes<32, 12, 8>());
        break;
    case 16:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep4<32, 28, 576, 2, 4>, 576, sweep4_smem_bytes<32, 28, 4>());
        break;
    case 17:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep4<40, 20, 352, 2, 4>, 352, sweep4_smem_bytes<40, 20, 4>());
        break;
    case 18:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep4<40, 8, 352, 3, 8>, 352, sweep4_smem_bytes<40, 8, 8>());
        break;
    case 19:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep4<32, 20, 288, 2, 4>, 288, sweep4_smem_bytes<32, 20, 4>());
        break;
    default:
        break;
    }
    return n;
}

size_t sweep4_smem(int tile) {
    switch (tile) {
    case 14:
        return sweep4_smem_bytes<32, 12, 4>();
    case 15:
        return sweep4_smem_bytes<32, 12, 8>();
    case 16:
        return sweep4_smem_bytes<32, 28, 4>();
    case 17:
        return sweep4_smem_bytes<40, 20, 4>();
    case 18:
        return sweep4_smem_bytes<40, 8, 8>();
    case 19:
        return sweep4_smem_bytes<32, 20, 4>();
    default:
        return 0;
    }
}

}  // namespace rwk
