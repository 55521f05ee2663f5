// Instantiations of the register-blocked FP32 sweep (see sweep5_kernel.cuh).
#include "sweep5_kernel.cuh"

namespace rwk {

namespace {

// tile id -> (TX, TY, voxels per strip, threads, planes ahead, minimum resident
// CTAs, p_k and u' exchanged through the ring slots)
#define RW_STRIP_TILES(X)                \
    X(20, 64, 11, 4, 256, 2, 2, false)   \
    X(21, 32, 22, 4, 256, 2, 2, false)   \
    X(22, 32, 20, 4, 256, 2, 2, false)   \
    X(23, 64, 8, 4, 224, 2, 2, false)    \
    X(24, 40, 20, 4, 288, 2, 2, false)   \
    X(25, 40, 8, 4, 160, 2, 3, false)    \
    X(31, 32, 20, 4, 256, 3, 2, false)   \
    X(32, 64, 8, 4, 224, 3, 2, false)    \
    X(33, 32, 22, 4, 256, 1, 2, false)   \
    X(34, 64, 8, 4, 224, 1, 3, false)    \
    X(35, 64, 14, 4, 320, 1, 2, false)   \
    X(36, 64, 14, 4, 320, 2, 2, true)    \
    X(37, 64, 14, 4, 320, 1, 2, true)    \
    X(38, 64, 11, 4, 256, 2, 2, true)    \
    X(39, 64, 11, 4, 256, 3, 2, true)    \
    X(40, 32, 22, 4, 256, 2, 2, true)    \
    X(41, 32, 20, 4, 256, 3, 2, true)    \
    X(42, 64, 13, 4, 288, 3, 2, true)    \
    X(43, 64, 12, 4, 288, 3, 2, true)    \
    X(44, 40, 20, 4, 288, 2, 2, true)    \
    X(45, 40, 20, 4, 288, 3, 2, true)    \
    X(46, 40, 8, 4, 160, 2, 3, true)

template <int TX, int TY, int V, int NT, int D, int MB, bool R>
cudaError_t launch_one(const SweepArgs& a, int grid, cudaStream_t s) {
    k_sweep5<TX, TY, V, NT, D, MB, false, R><<<grid, NT, sweep5_smem_bytes<TX, TY, V, D, R>(), s>>>(a);
    return cudaGetLastError();
}

template <int TX, int TY, int V, int NT, int D, int MB, bool R>
cudaError_t prepare_one() {
    return cudaFuncSetAttribute(k_sweep5<TX, TY, V, NT, D, MB, false, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sweep5_smem_bytes<TX, TY, V, D, R>());
}

template <int TX, int TY, int V, int NT, int D, int MB, bool R>
int occupancy_one() {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep5<TX, TY, V, NT, D, MB, false, R>, NT,
                                                  sweep5_smem_bytes<TX, TY, V, D, R>());
    return n;
}

template <int TX, int TY, int V, int NT, int D, int MB, bool R = false>
cudaError_t launch_loop_one(const SweepArgs& a, int grid, cudaStream_t s) {
    auto fn = k_sweep5<TX, TY, V, NT, D, MB, true, R>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sweep5_smem_bytes<TX, TY, V, D, R>());
    if (e != cudaSuccess) return e;
    SweepArgs arg = a;
    void* args[] = {&arg};
    return cudaLaunchCooperativeKernel((const void*)fn, dim3(grid), dim3(NT), args,
                                       sweep5_smem_bytes<TX, TY, V, D, R>(), s);
}

template <int TX, int TY, int V, int NT, int D, int MB, bool R = false>
int occupancy_loop_one() {
    int n = 0;
    cudaFuncSetAttribute(k_sweep5<TX, TY, V, NT, D, MB, true, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sweep5_smem_bytes<TX, TY, V, D, R>());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_sweep5<TX, TY, V, NT, D, MB, true, R>, NT,
                                                  sweep5_smem_bytes<TX, TY, V, D, R>());
    return n;
}

}  // namespace

// Looped (multi-iteration, cooperative) strip sweep: the brick tiles only.
cudaError_t sweep5_launch_loop(int tile, const SweepArgs& a, int grid, cudaStream_t s) {
    switch (tile) {
    case 24:
        return launch_loop_one<40, 20, 4, 288, 2, 2>(a, grid, s);
    case 25:
        return launch_loop_one<40, 8, 4, 160, 2, 3>(a, grid, s);
    case 44:
        return launch_loop_one<40, 20, 4, 288, 2, 2, true>(a, grid, s);
    case 45:
        return launch_loop_one<40, 20, 4, 288, 3, 2, true>(a, grid, s);
    case 46:
        return launch_loop_one<40, 8, 4, 160, 2, 3, true>(a, grid, s);
    default:
        return cudaErrorInvalidValue;
    }
}

int sweep5_occupancy_loop(int tile) {
    switch (tile) {
    case 24:
        return occupancy_loop_one<40, 20, 4, 288, 2, 2>();
    case 25:
        return occupancy_loop_one<40, 8, 4, 160, 2, 3>();
    case 44:
        return occupancy_loop_one<40, 20, 4, 288, 2, 2, true>();
    case 45:
        return occupancy_loop_one<40, 20, 4, 288, 3, 2, true>();
    case 46:
        return occupancy_loop_one<40, 8, 4, 160, 2, 3, true>();
    default:
        return 0;
    }
}

cudaError_t sweep5_launch(int tile, const SweepArgs& a, int grid, cudaStream_t s) {
    switch (tile) {
#define X(id, tx, ty, v, nt, d, mb, r) \
    case id:                           \
        return launch_one<tx, ty, v, nt, d, mb, r>(a, grid, s);
        RW_STRIP_TILES(X)
#undef X
    default:
        return cudaErrorInvalidValue;
    }
}

cudaError_t sweep5_prepare(int tile) {
    switch (tile) {
#define X(id, tx, ty, v, nt, d, mb, r) \
    case id:                           \
        return prepare_one<tx, ty, v, nt, d, mb, r>();
        RW_STRIP_TILES(X)
#undef X
    default:
        return cudaErrorInvalidValue;
    }
}

int sweep5_occupancy(int tile) {
    switch (tile) {
#define X(id, tx, ty, v, nt, d, mb, r) \
    case id:                           \
        return occupancy_one<tx, ty, v, nt, d, mb, r>();
        RW_STRIP_TILES(X)
#undef X
    default:
        return 0;
    }
}

size_t sweep5_smem(int tile) {
    switch (tile) {
#define X(id, tx, ty, v, nt, d, mb, r) \
    case id:                           \
        return sweep5_smem_bytes<tx, ty, v, d, r>();
        RW_STRIP_TILES(X)
#undef X
    default:
        return 0;
    }
}

}  // namespace rwk
