// Instantiation of the pipelined FP32 sweep (see sweep2_kernel.cuh) for the
// one tile it serves: 32 x 8, for boxes narrower than one strip-kernel tile
// (the autotuner's choice below 25 voxels in x) and the fixed tile of the
// allocation-free solve.
#include "sweep2_kernel.cuh"

namespace rwk {

namespace {
constexpr int kTX = 32, kTY = 8, kNT = 256, kD = 3;
constexpr size_t kSmem = sweep2_smem_bytes<kTX, kTY, kD>();
}  // namespace

cudaError_t sweep2_launch(int tile, const SweepArgs& a, int grid, cudaStream_t s) {
    if (tile != TILE_32x8) return cudaErrorInvalidValue;
    k_sweep2<kTX, kTY, kNT, kD><<<grid, kNT, kSmem, s>>>(a);
    return cudaGetLastError();
}

cudaError_t sweep2_prepare(int tile) {
    if (tile != TILE_32x8) return cudaErrorInvalidValue;
    return cudaFuncSetAttribute(k_sweep2<kTX, kTY, kNT, kD>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
}

int sweep2_occupancy(int tile) {
    if (tile != TILE_32x8) return 0;
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep2<kTX, kTY, kNT, kD>, kNT, kSmem);
    return n;
}

size_t sweep2_smem(int tile) { return tile == TILE_32x8 ? kSmem : 0; }

}  // namespace rwk
