// Instantiations of the pipelined FP32 sweep (see sweep2_kernel.cuh).
#include "sweep2_kernel.cuh"

namespace rwk {

cudaError_t sweep2_launch(int tile, const SweepArgs& a, int grid, cudaStream_t s) {
    switch (tile) {
    case 1:
        k_sweep2<32, 16, 512, 3><<<grid, 512, sweep2_smem_bytes<32, 16, 3>(), s>>>(a);
        return cudaGetLastError();
    case 2:
        k_sweep2<64, 8, 512, 3><<<grid, 512, sweep2_smem_bytes<64, 8, 3>(), s>>>(a);
        return cudaGetLastError();
    case 3:
        k_sweep2<40, 8, 320, 3><<<grid, 320, sweep2_smem_bytes<40, 8, 3>(), s>>>(a);
        return cudaGetLastError();
    case 4:
        k_sweep2<40, 20, 800, 2><<<grid, 800, sweep2_smem_bytes<40, 20, 2>(), s>>>(a);
        return cudaGetLastError();
    case 5:
        k_sweep2<80, 8, 640, 2><<<grid, 640, sweep2_smem_bytes<80, 8, 2>(), s>>>(a);
        return cudaGetLastError();
    case 6:
        k_sweep2<80, 16, 640, 2><<<grid, 640, sweep2_smem_bytes<80, 16, 2>(), s>>>(a);
        return cudaGetLastError();
    case 7:
        k_sweep2<32, 8, 256, 3><<<grid, 256, sweep2_smem_bytes<32, 8, 3>(), s>>>(a);
        return cudaGetLastError();
    case 8:
        k_sweep2<32, 32, 1024, 2><<<grid, 1024, sweep2_smem_bytes<32, 32, 2>(), s>>>(a);
        return cudaGetLastError();
    case 9:
        k_sweep2<64, 16, 1024, 2><<<grid, 1024, sweep2_smem_bytes<64, 16, 2>(), s>>>(a);
        return cudaGetLastError();
    default:
        return cudaErrorInvalidValue;
    }
}

cudaError_t sweep2_prepare(int tile) {
    switch (tile) {
    case 1:
        return cudaFuncSetAttribute(k_sweep2<32, 16, 512, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sweep2_smem_bytes<32, 16, 3>());
    case 2:
        return cudaFuncSetAttribute(k_sweep2<64, 8, 512, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sweep2_smem_bytes<64, 8, 3>());
    case 3:
        return cudaFuncSetAttribute(k_sweep2<40, 8, 320, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sweep2_smem_bytes<40, 8, 3>());
    case 4:
        return cudaFuncSetAttribute(k_sweep2<40, 20, 800, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sweep2_smem_bytes<40, 20, 2>());
    case 5:
        return cudaFuncSetAttribute(k_sweep2<80, 8, 640, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sweep2_smem_bytes<80, 8, 2>());
    case 6:
        return cudaFuncSetAttribute(k_sweep2<80, 16, 640, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sweep2_smem_bytes<80, 16, 2>());
    case 7:
        return cudaFuncSetAttribute(k_sweep2<32, 8, 256, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sweep2_smem_bytes<32, 8, 3>());
    case 8:
        return cudaFuncSetAttribute(k_sweep2<32, 32, 1024, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sweep2_smem_bytes<32, 32, 2>());
    case 9:
        return cudaFuncSetAttribute(k_sweep2<64, 16, 1024, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)sweep2_smem_bytes<64, 16, 2>());
    default:
        return cudaErrorInvalidValue;
    }
}

int sweep2_occupancy(int tile) {
    int n = 0;
    switch (tile) {
    case 1:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep2<32, 16, 512, 3>, 512,
                                                      sweep2_smem_bytes<32, 16, 3>());
        break;
    case 2:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep2<64, 8, 512, 3>, 512,
                                                      sweep2_smem_bytes<64, 8, 3>());
        break;
    case 3:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep2<40, 8, 320, 3>, 320,
                                                      sweep2_smem_bytes<40, 8, 3>());
        break;
    case 4:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep2<40, 20, 800, 2>, 800,
                                                      sweep2_smem_bytes<40, 20, 2>());
        break;
    case 5:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep2<80, 8, 640, 2>, 640,
                                                      sweep2_smem_bytes<80, 8, 2>());
        break;
    case 6:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep2<80, 16, 640, 2>, 640,
                                                      sweep2_smem_bytes<80, 16, 2>());
        break;
    case 7:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep2<32, 8, 256, 3>, 256,
                                                      sweep2_smem_bytes<32, 8, 3>());
        break;
    case 8:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep2<32, 32, 1024, 2>, 1024,
                                                      sweep2_smem_bytes<32, 32, 2>());
        break;
    case 9:
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep2<64, 16, 1024, 2>, 1024,
                                                      sweep2_smem_bytes<64, 16, 2>());
        break;
    default:
        break;
    }
    return n;
}

size_t sweep2_smem(int tile) {
    switch (tile) {
    case 1:
        return sweep2_smem_bytes<32, 16, 3>();
    case 2:
        return sweep2_smem_bytes<64, 8, 3>();
    case 3:
        return sweep2_smem_bytes<40, 8, 3>();
    case 4:
        return sweep2_smem_bytes<40, 20, 2>();
    case 5:
        return sweep2_smem_bytes<80, 8, 2>();
    case 6:
        return sweep2_smem_bytes<80, 16, 2>();
    case 7:
        return sweep2_smem_bytes<32, 8, 3>();
    case 8:
        return sweep2_smem_bytes<32, 32, 2>();
    case 9:
        return sweep2_smem_bytes<64, 16, 2>();
    default:
        return 0;
    }
}

}  // namespace rwk
