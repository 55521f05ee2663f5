// Instantiations of the warp-row FP32 sweep (see sweep3_kernel.cuh).
#include "sweep3_kernel.cuh"

namespace rwk {

cudaError_t sweep3_launch(int tile, const SweepArgs& a, int grid, cudaStream_t s) {
    switch (tile) {
    case 10:
        k_sweep3<28, 16, 3><<<grid, 512, sweep3_smem_bytes<28, 3>(), s>>>(a);
        return cudaGetLastError();
    case 11:
        k_sweep3<12, 8, 3><<<grid, 256, sweep3_smem_bytes<12, 3>(), s>>>(a);
        return cudaGetLastError();
    case 12:
        k_sweep3<20, 8, 3><<<grid, 256, sweep3_smem_bytes<20, 3>(), s>>>(a);
        return cudaGetLastError();
    case 13:
        k_sweep3<28, 8, 2><<<grid, 256, sweep3_smem_bytes<28, 2>(), s>>>(a);
        return cudaGetLastError();
    default:
        return cudaErrorInvalidValue;
    }
}

cudaError_t sweep3_prepare(int tile) {
    switch (tile) {
    case 10:
        return cudaFuncSetAttribute(k_sweep3<28, 16, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sweep3_smem_bytes<28, 3>());
    case 11:
        return cudaFuncSetAttribute(k_sweep3<12, 8, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sweep3_smem_bytes<12, 3>());
    case 12:
        return cudaFuncSetAttribute(k_sweep3<20, 8, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sweep3_smem_bytes<20, 3>());
    case 13:
        return cudaFuncSetAttribute(k_sweep3<28, 8, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sweep3_smem_bytes<28, 2>());
    default:
        return cudaErrorInvalidValue;
    }
}

int sweep3_occupancy(int tile) {
    int n = 0;
    switch (tile) {
    case 10:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep3<28, 16, 3>, 512, sweep3_smem_bytes<28, 3>());
        break;
    case 11:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep3<12, 8, 3>, 256, sweep3_smem_bytes<12, 3>());
        break;
    case 12:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep3<20, 8, 3>, 256, sweep3_smem_bytes<20, 3>());
        break;
    case 13:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep3<28, 8, 2>, 256, sweep3_smem_bytes<28, 2>());
        break;
    default:
        break;
    }
    return n;
}

size_t sweep3_smem(int tile) {
    switch (tile) {
    case 10:
        return sweep3_smem_bytes<28, 3>();
    case 11:
        return sweep3_smem_bytes<12, 3>();
    case 12:
        return sweep3_smem_bytes<20, 3>();
    case 13:
        return sweep3_smem_bytes<28, 2>();
    default:
        return 0;
    }
}

}  // namespace rwk
