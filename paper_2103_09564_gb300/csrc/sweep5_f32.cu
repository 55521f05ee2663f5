// Instantiations of the register-blocked FP32 sweep (see sweep5_kernel.cuh).
#include "sweep5_kernel.cuh"

namespace rwk {

namespace {

// tile id -> (TX, TY, threads, planes ahead, minimum resident CTAs)
#define RW_STRIP_TILES(X)      \
    X(20, 64, 11, 256, 2, 2)   \
    X(21, 32, 22, 256, 2, 2)   \
    X(22, 32, 20, 256, 2, 2)   \
    X(23, 64, 8, 224, 2, 2)    \
    X(24, 40, 20, 288, 2, 2)   \
    X(25, 40, 8, 160, 2, 3)

template <int TX, int TY, int NT, int D, int MB>
cudaError_t launch_one(const SweepArgs& a, int grid, cudaStream_t s) {
    k_sweep5<TX, TY, NT, D, MB><<<grid, NT, sweep5_smem_bytes<TX, TY, D>(), s>>>(a);
    return cudaGetLastError();
}

template <int TX, int TY, int NT, int D, int MB>
cudaError_t prepare_one() {
    return cudaFuncSetAttribute(k_sweep5<TX, TY, NT, D, MB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sweep5_smem_bytes<TX, TY, D>());
}

template <int TX, int TY, int NT, int D, int MB>
int occupancy_one() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep5<TX, TY, NT, D, MB>, NT, sweep5_smem_bytes<TX, TY, D>());
    return n;
}

}  // namespace

cudaError_t sweep5_launch(int tile, const SweepArgs& a, int grid, cudaStream_t s) {
    switch (tile) {
#define X(id, tx, ty, nt, d, mb) \
    case id:                     \
        return launch_one<tx, ty, nt, d, mb>(a, grid, s);
        RW_STRIP_TILES(X)
#undef X
    default:
        return cudaErrorInvalidValue;
    }
}

cudaError_t sweep5_prepare(int tile) {
    switch (tile) {
#define X(id, tx, ty, nt, d, mb) \
    case id:                     \
        return prepare_one<tx, ty, nt, d, mb>();
        RW_STRIP_TILES(X)
#undef X
    default:
        return cudaErrorInvalidValue;
    }
}

int sweep5_occupancy(int tile) {
    switch (tile) {
#define X(id, tx, ty, nt, d, mb) \
    case id:                     \
        return occupancy_one<tx, ty, nt, d, mb>();
        RW_STRIP_TILES(X)
#undef X
    default:
        return 0;
    }
}

size_t sweep5_smem(int tile) {
    switch (tile) {
#define X(id, tx, ty, nt, d, mb) \
    case id:                     \
        return sweep5_smem_bytes<tx, ty, d>();
        RW_STRIP_TILES(X)
#undef X
    default:
        return 0;
    }
}

}  // namespace rwk
