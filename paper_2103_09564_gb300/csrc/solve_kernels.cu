// Set-up, residual and bookkeeping kernels of the PCG solve (Sec. III-B
// system, Jacobi-PCG as in Sec. V), plus the sweep dispatcher.
//
// Precision scheme (mixed): the solution is held in FP64 (x_hi).  Each
// refinement round computes the true residual r = b - A x_hi with FP64 edge
// weights, starts the FP32 PCG on the correction system A delta = r
// (delta = 0, u = D^-1 r, p = 0), and adds delta to x_hi when the round
// ends.  In RW_FP64 mode the sweeps iterate on x_hi directly.
#include "rw_internal.h"
#include "sweep_kernel.cuh"

namespace rwk {

cudaError_t sweep2_launch(int tile, const SweepArgs& a, int grid, cudaStream_t s);
cudaError_t sweep2_prepare(int tile);
int sweep2_occupancy(int tile);
size_t sweep2_smem(int tile);
cudaError_t sweep5_launch(int tile, const SweepArgs& a, int grid, cudaStream_t s);
cudaError_t sweep5_prepare(int tile);
int sweep5_occupancy(int tile);
size_t sweep5_smem(int tile);
cudaError_t sweep_launch_d64_u16(int tile, const SweepArgs& a, int grid, cudaStream_t s);
cudaError_t sweep_launch_d64_f32(int tile, const SweepArgs& a, int grid, cudaStream_t s);
cudaError_t sweep_prepare_d64_u16(int tile);
cudaError_t sweep_prepare_d64_f32(int tile);
int sweep_occupancy_d64_u16(int tile);
int sweep_occupancy_d64_f32(int tile);

cudaError_t sweep_prepare(int fp64, int gtype, int tile);

// Resident CTAs per SM of an instantiated sweep (0 when the combination is
// not compiled); opts the kernel in to its dynamic shared memory first.
int sweep_occupancy(int fp64, int gtype, int tile) {
    static int cache[2][2][N_TILES];
    static bool init = false;
    if (!init) {
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b)
                for (int c = 0; c < N_TILES; ++c) cache[a][b][c] = -1;
        init = true;
    }
    if (!tile_compiled(fp64, tile)) return 0;
    int& slot = cache[fp64 ? 1 : 0][gtype == G_U16 ? 0 : 1][tile];
    if (slot >= 0) return slot;
    if (sweep_prepare(fp64, gtype, tile) != cudaSuccess) {
        cudaGetLastError();
        slot = 0;
        return 0;
    }
    if (fp64) slot = gtype == G_U16 ? sweep_occupancy_d64_u16(tile) : sweep_occupancy_d64_f32(tile);
    else slot = tile >= TILE_STRIP_FIRST ? sweep5_occupancy(tile) : sweep2_occupancy(tile);
    return slot;
}


void tile_dims(int tile, int* tx, int* ty) {
    static const int T[N_TILES][2] = {{0, 0},   {32, 16}, {64, 8},  {40, 8},  {40, 20}, {80, 8},  {80, 16},
                                      {32, 8},  {32, 32}, {64, 16}, {28, 28}, {28, 12}, {28, 20}, {28, 28},
                                      {32, 12}, {32, 12}, {32, 28}, {40, 20}, {40, 8},  {32, 20},
                                      {64, 11}, {32, 22}, {32, 20}, {64, 8},  {40, 20}, {40, 8},
                                      {32, 20}, {64, 11}, {32, 12}, {40, 20}, {40, 8},  {32, 20},
                                      {64, 8},  {32, 22}, {64, 8},  {64, 14}, {64, 14}, {64, 14},
                                      {64, 11}, {64, 11}, {32, 22}, {32, 20}, {64, 13}, {64, 12},
                                      {40, 20}, {40, 20}, {40, 8}};
    if (tile < 1 || tile >= N_TILES) tile = 1;
    *tx = T[tile][0];
    *ty = T[tile][1];
}

int sweep_threads(int tile) {
    static const int N[N_TILES] = {0,   512, 512, 320, 800, 640, 640, 256, 1024, 1024,
                                   512, 256, 256, 256, 288, 288, 576, 352, 352, 288,
                                   256, 256, 256, 224, 288, 160, 416, 480, 288, 512, 256, 256, 224, 256, 224,
                                   320, 320, 320, 256, 256, 256, 256, 288, 288, 288, 288, 160};
    return (tile >= 1 && tile < N_TILES) ? N[tile] : 0;
}

// FP64 sweeps use the generic kernel (sweep_kernel.cuh); FP32 sweeps the
// strip kernel (sweep5_kernel.cuh), or for narrow boxes the pipelined one
// (sweep2_kernel.cuh), which reads packed g|code words.
size_t sweep_smem_bytes(int fp64, int tile) {
    int tx, ty;
    tile_dims(tile, &tx, &ty);
    const int r2 = (tx + 4) * (ty + 4);
    if (fp64) return (size_t)sweep_planes_bytes<double>(r2);
    return tile >= TILE_STRIP_FIRST ? sweep5_smem(tile) : sweep2_smem(tile);
}

cudaError_t launch_sweep(int fp64, int gtype, int tile, const SweepArgs& a, int grid, cudaStream_t s) {
    if (fp64) return gtype == G_U16 ? sweep_launch_d64_u16(tile, a, grid, s) : sweep_launch_d64_f32(tile, a, grid, s);
    return tile >= TILE_STRIP_FIRST ? sweep5_launch(tile, a, grid, s) : sweep2_launch(tile, a, grid, s);
}

cudaError_t sweep_prepare(int fp64, int gtype, int tile) {
    if (fp64) return gtype == G_U16 ? sweep_prepare_d64_u16(tile) : sweep_prepare_d64_f32(tile);
    return tile >= TILE_STRIP_FIRST ? sweep5_prepare(tile) : sweep2_prepare(tile);
}

// ---------------------------------------------------------------------------
__device__ __forceinline__ double gdbl(const void* g, int gtype, int64_t i) {
    return gtype == G_U16 ? (double)static_cast<const uint16_t*>(g)[i] / 65535.0
                          : (double)static_cast<const float*>(g)[i];
}

// Intensity as the weights see it: g, or sqrt(g) for Poisson weights.
__device__ __forceinline__ double gdbl_w(const ResidArgs& a, int64_t i) {
    const double g = gdbl(a.g, a.gtype, i);
    return a.sqrt_g ? sqrt(g) : g;
}

__device__ __forceinline__ bool box_extent(const Boxes& bx, int box, int* ex, int* ey, int* ez) {
    if (bx.ext) {
        *ex = bx.ext[3 * box];
        *ey = bx.ext[3 * box + 1];
        *ez = bx.ext[3 * box + 2];
    } else {
        *ex = bx.nx;
        *ey = bx.ny;
        *ez = bx.nz;
    }
    return true;
}

// x_hi: seeds take their value, free voxels the initial guess, others 0.
__global__ void k_init_x(const ResidArgs a) {
    const int box = blockIdx.y;
    const int64_t nvox = (int64_t)a.bx.nx * a.bx.ny * a.bx.nz;
    const int64_t li = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= nvox) return;
    int ex, ey, ez;
    box_extent(a.bx, box, &ex, &ey, &ez);
    int x, y, z;
    vox_xyz(li, a.bx.nx, a.bx.ny, nvox, &x, &y, &z);
    const int64_t i = (int64_t)box * nvox + li;
    double v = 0.0;
    if (x < ex && y < ey && z < ez) {
        const uint8_t c = a.code[i];
        if (c == SEED) v = a.value ? (double)a.value[i] : 0.0;
        else if (c == FREE) v = a.x0 ? (double)a.x0[i] : 0.0;
    }
    static_cast<double*>(a.x)[i] = v;
}

// FP64 residual r = b - A x_hi = rhs - sum_j w_ij (x_i - x_j) on free voxels
// (x_j = seed value on seeds), with b = rhs + sum over seeded neighbours of
// w_ij m_j.  Writes u = r / d (T), p = 0 and, in mixed mode, delta = 0; per
// block partial sums of ||b||^2, ||r||^2, #seeds, #free.
template <typename T>
__global__ void __launch_bounds__(256) k_residual(const ResidArgs a, float* delta) {
    const int box = blockIdx.y;
    // a box that did not iterate since its last residual keeps it (and its
    // zero correction); k_box_reduce skips it the same way
    if (a.only_moved && !a.sc[box].moved) return;
    const int nx = a.bx.nx, ny = a.bx.ny, nz = a.bx.nz;
    const int64_t nvox = (int64_t)nx * ny * nz;
    // up to 4 voxels per thread, a grid stride apart (blocks_per_box blocks
    // per box): the FP64 reductions below are amortised over them
    const int64_t li0 = (int64_t)blockIdx.x * 256 + threadIdx.x;
    const int64_t stride = (int64_t)a.blocks_per_box * 256;
    double bb = 0, rr = 0;
    int ns = 0, nf = 0;
    for (int rep = 0; rep < 4; ++rep) {
        const int64_t li = li0 + rep * stride;
        if (li >= nvox) break;
        int ex, ey, ez;
        box_extent(a.bx, box, &ex, &ey, &ez);
        int x, y, z;
        vox_xyz(li, nx, ny, nvox, &x, &y, &z);
        // (u, p, delta follow a.pad; x_hi, g and the code the caller layout)
        const int64_t base = (int64_t)box * nvox;
        const int64_t i = base + li;
        const double* xh = static_cast<const double*>(a.x);
        T uo = 0;
        if (x < ex && y < ey && z < ez) {
            const uint8_t c = a.code[i];
            if (c == SEED) ++ns;
            if (c == FREE) {
                ++nf;
                const double gi = gdbl_w(a, i), xi = xh[i];
                const double rh = a.rhs ? (double)a.rhs[i] : 0.0;
                // s (the operator applied to x) in FP64; the diagonal d and the
                // right-hand side b in T: d only scales u (stored in T), b only
                // enters ||b||, the reference of the relative stopping test
                double s = 0;
                T d = 0, b = (T)rh;
                const int nbx[6] = {x - 1, x + 1, x, x, x, x};
                const int nby[6] = {y, y, y - 1, y + 1, y, y};
                const int nbz[6] = {z, z, z, z, z - 1, z + 1};
#pragma unroll
                for (int k = 0; k < 6; ++k) {
                    if (nbx[k] < 0 || nbx[k] >= ex || nby[k] < 0 || nby[k] >= ey || nbz[k] < 0 || nbz[k] >= ez) continue;
                    const int64_t j = base + ((int64_t)nbz[k] * ny + nby[k]) * nx + nbx[k];
                    const uint8_t cj = a.code[j];
                    if (cj == ABSENT) continue;
                    double w;
                    if (a.w3) {
                        // the forward edge of the lower voxel of the pair
                        const int64_t ntot = (int64_t)a.bx.nbox * nvox;
                        w = a.w3[(int64_t)(k >> 1) * ntot + ((k & 1) ? i : j)];
                    } else {
                        w = weight64(gi - gdbl_w(a, j), a.mbeta, a.wmin);
                    }
                    const double xj = xh[j];
                    d += (T)w;
                    s += w * (xi - xj);
                    if (cj == SEED) b += (T)w * (T)xj;
                }
                const double r = rh - s;
                bb += (double)b * (double)b;
                rr += r * r;
                // u is stored in T: for FP32 the quotient of the rounded
                // operands is as accurate as the stored value
                if constexpr (sizeof(T) == 4) uo = d > 0.0f ? (float)r / d : 0.0f;
                else uo = d > 0.0 ? (T)(r / d) : (T)0;
            }
        }
        const int64_t v = vec_index(a.pad, a.bx, box, x, y, z);
        static_cast<T*>(a.u)[v] = uo;
        if (!a.keep_p) static_cast<T*>(a.p)[v] = (T)0;
        else if (a.sc[box].par == 1) static_cast<T*>(a.p)[v] = static_cast<const T*>(a.p_other)[v];
        if (delta) delta[v] = 0.0f;
    }
    __shared__ double red[4][8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        bb += __shfl_down_sync(0xffffffffu, bb, o);
        rr += __shfl_down_sync(0xffffffffu, rr, o);
    }
    ns = __reduce_add_sync(0xffffffffu, ns);
    nf = __reduce_add_sync(0xffffffffu, nf);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][wid] = bb;
        red[1][wid] = rr;
        red[2][wid] = ns;
        red[3][wid] = nf;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double s = 0;
        for (int k = 0; k < 8; ++k) s += red[threadIdx.x][k];
        a.part[((int64_t)box * a.blocks_per_box + blockIdx.x) * 4 + threadIdx.x] = s;
    }
}

// Forward FP64 weights of every voxel: the same function (weight64), on the
// same operands up to an exact sign, as the residual's own evaluation and the
// FP64 sweeps'.
__global__ void k_weights64(const ResidArgs a, double* w3) {
    const int box = blockIdx.y;
    const int nx = a.bx.nx, ny = a.bx.ny, nz = a.bx.nz;
    const int64_t nvox = (int64_t)nx * ny * nz, ntot = (int64_t)a.bx.nbox * nvox;
    const int64_t li = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= nvox) return;
    int ex, ey, ez;
    box_extent(a.bx, box, &ex, &ey, &ez);
    int x, y, z;
    vox_xyz(li, nx, ny, nvox, &x, &y, &z);
    const int64_t i = (int64_t)box * nvox + li;
    double wv[3] = {0.0, 0.0, 0.0};
    if (x < ex && y < ey && z < ez && a.code[i] != ABSENT) {
        const double gi = gdbl_w(a, i);
        const bool in[3] = {x + 1 < ex, y + 1 < ey, z + 1 < ez};
        const int64_t st[3] = {1, nx, (int64_t)nx * ny};
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            if (!in[k]) continue;
            const int64_t j = i + st[k];
            if (a.code[j] == ABSENT) continue;
            wv[k] = weight64(gi - gdbl_w(a, j), a.mbeta, a.wmin);
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) w3[k * ntot + i] = wv[k];
}

cudaError_t launch_weights64(const ResidArgs& a, double* w3, cudaStream_t s) {
    const int64_t nvox = (int64_t)a.bx.nx * a.bx.ny * a.bx.nz;
    dim3 grid((unsigned)((nvox + 255) / 256), (unsigned)a.bx.nbox);
    k_weights64<<<grid, 256, 0, s>>>(a, w3);
    return cudaGetLastError();
}

cudaError_t launch_init_x(int fp64, const ResidArgs& a, cudaStream_t s) {
    (void)fp64;
    const int64_t nvox = (int64_t)a.bx.nx * a.bx.ny * a.bx.nz;
    dim3 grid((unsigned)((nvox + 255) / 256), (unsigned)a.bx.nbox);
    k_init_x<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_residual(int fp64, const ResidArgs& a, float* delta, cudaStream_t s) {
    dim3 grid((unsigned)a.blocks_per_box, (unsigned)a.bx.nbox);
    if (fp64) k_residual<double><<<grid, 256, 0, s>>>(a, nullptr);
    else k_residual<float><<<grid, 256, 0, s>>>(a, delta);
    return cudaGetLastError();
}

__global__ void k_box_reduce(const double* part, int bpb, BoxScalars* sc, int first, int only_moved) {
    __shared__ double red[4][256];
    const int box = blockIdx.x;
    if (only_moved && !sc[box].moved) return;
    double v[4] = {0, 0, 0, 0};
    for (int k = threadIdx.x; k < bpb; k += 256)
        for (int j = 0; j < 4; ++j) v[j] += part[((int64_t)box * bpb + k) * 4 + j];
    for (int j = 0; j < 4; ++j) red[j][threadIdx.x] = v[j];
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if (threadIdx.x < st)
            for (int j = 0; j < 4; ++j) red[j][threadIdx.x] += red[j][threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        BoxScalars* S = sc + box;
        if (first) {
            S->bb = red[0][0];
            S->nseed = (int)red[2][0];
            S->nfree = (int)red[3][0];
        }
        S->rr_true = red[1][0];
    }
}

cudaError_t launch_box_reduce(const double* part, int blocks_per_box, int nbox, BoxScalars* sc, int first,
                              cudaStream_t s, int only_moved) {
    k_box_reduce<<<nbox, 256, 0, s>>>(part, blocks_per_box, sc, first, only_moved);
    return cudaGetLastError();
}

// Decide which systems iterate in this refinement round and set their inner target:
// stop the round at ||r|| <= max(tol ||b||, eps_inner ||r_round_start||).
__global__ void k_start_round(BoxScalars* sc, int nbox, int round, double tol, double eps_inner, int max_iter,
                              int restart, int* n_active) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    BoxScalars* S = sc + b;
    if (round == 0) {
        S->iters = 0;
        S->max_iter = max_iter;
        S->status = 0;
        S->dbeta = 0.0;
    }
    if (!(S->bb > 0.0)) S->rr_true = 0.0;
    const double tgt = tol * tol * S->bb;
    const bool need = S->nseed > 0 && S->nfree > 0 && S->bb > 0.0 && S->rr_true > tgt && S->iters < max_iter;
    S->counter = 0u;
    S->moved = need ? 1 : 0;
    // the residual that precedes every round wrote u (and the kept p) into
    // buffer 0: the record must point there, for the sweeps that read the
    // system's own parity (the cluster-resident solver)
    S->par = 0;
    if (need) {
        S->active = 1;
        // continue the Krylov process across the residual replacement when
        // possible (reliable update); restart on the first round, after a
        // precision switch, or after a breakdown
        if (restart || round == 0 || S->status == 5 || !(S->gam > 0.0)) {
            S->phase = 0;
            S->status = 0;
        } else {
            S->phase = 2;
        }
        S->alpha = 0.0;
        S->beta = 0.0;
        S->tol2 = fmax(tgt, eps_inner * eps_inner * S->rr_true);
        atomicAdd(n_active, 1);
    } else {
        S->active = 0;
    }
}

cudaError_t launch_start_round(BoxScalars* sc, int nbox, int round, double tol, double eps_inner, int max_iter,
                               int restart, int* n_active, cudaStream_t s) {
    k_start_round<<<(nbox + 127) / 128, 128, 0, s>>>(sc, nbox, round, tol, eps_inner, max_iter, restart, n_active);
    return cudaGetLastError();
}

// A system whose right-hand side is zero has x_U = 0.
__global__ void k_zero_homog(const Boxes bx, const uint8_t* code, const BoxScalars* sc, double* x) {
    const int box = blockIdx.y;
    const int64_t nvox = (int64_t)bx.nx * bx.ny * bx.nz;
    const int64_t li = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= nvox) return;
    const BoxScalars* S = sc + box;
    if (!(S->bb == 0.0) || S->nseed == 0) return;
    const int64_t i = (int64_t)box * nvox + li;
    if (code[i] == FREE) x[i] = 0.0;
}

cudaError_t launch_zero_homog(int fp64, const Boxes& bx, const uint8_t* code, const BoxScalars* sc, void* x,
                              cudaStream_t s) {
    (void)fp64;
    const int64_t nvox = (int64_t)bx.nx * bx.ny * bx.nz;
    dim3 grid((unsigned)((nvox + 255) / 256), (unsigned)bx.nbox);
    k_zero_homog<<<grid, 256, 0, s>>>(bx, code, sc, static_cast<double*>(x));
    return cudaGetLastError();
}

// Ordered compaction of the active systems: one CTA scans the box records in
// chunks of its size (ballot within a warp, warp counts through shared memory).
__global__ void __launch_bounds__(1024) k_compact_active(const BoxScalars* sc, int nbox, int* list, int* nlist) {
    __shared__ int wsum[32];
    __shared__ int base;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (int c = 0; c < nbox; c += blockDim.x) {
        const int b = c + threadIdx.x;
        const bool on = b < nbox && sc[b].active;
        const unsigned m = __ballot_sync(0xffffffffu, on);
        if (lane == 0) wsum[warp] = __popc(m);
        __syncthreads();
        int off = base;
        for (int k = 0; k < warp; ++k) off += wsum[k];
        if (on) list[off + __popc(m & ((1u << lane) - 1u))] = b;
        __syncthreads();
        if (threadIdx.x == 0) {
            int tot = 0;
            for (int k = 0; k < nwarp; ++k) tot += wsum[k];
            base += tot;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *nlist = base;
}

cudaError_t launch_compact_active(const BoxScalars* sc, int nbox, int* list, int* nlist, cudaStream_t s) {
    k_compact_active<<<1, 1024, 0, s>>>(sc, nbox, list, nlist);
    return cudaGetLastError();
}

// x_hi += delta on free voxels (end of a mixed-precision round).
__global__ void k_accumulate(const Boxes bx, const Pad pad, const uint8_t* code, const float* delta, double* x) {
    const int box = blockIdx.y;
    const int64_t nvox = (int64_t)bx.nx * bx.ny * bx.nz;
    const int64_t li = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= nvox) return;
    const int64_t i = (int64_t)box * nvox + li;
    if (code[i] != FREE) return;
    int xx, yy, zz;
    vox_xyz(li, bx.nx, bx.ny, nvox, &xx, &yy, &zz);
    x[i] += (double)delta[vec_index(pad, bx, box, xx, yy, zz)];
}

cudaError_t launch_accumulate(const Boxes& bx, const Pad& pad, const uint8_t* code, const float* delta, double* x,
                              cudaStream_t s) {
    const int64_t nvox = (int64_t)bx.nx * bx.ny * bx.nz;
    dim3 grid((unsigned)((nvox + 255) / 256), (unsigned)bx.nbox);
    k_accumulate<<<grid, 256, 0, s>>>(bx, pad, code, delta, x);
    return cudaGetLastError();
}

// gc = (bits of FP32 g with the two low bits cleared) | code', where
// code' = 1 free, 2 seed, 0 absent (also for voxels beyond the box extent),
// so that zero-filled halo words read as absent voxels.
// fmt 0: FP32 g with the code in its two lowest mantissa bits (0 absent,
// 1 free, 2 seed); fmt 1: +g free, -g seed, NaN absent (g >= 0).
__global__ void k_pack_gc(const Boxes bx, const Pad pad, const void* g, int gtype, const uint8_t* code,
                          uint32_t* gc, int fmt, int sqrt_g) {
    const int box = blockIdx.y;
    const int64_t nvox = (int64_t)bx.nx * bx.ny * bx.nz;
    const int64_t li = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= nvox) return;
    int ex, ey, ez;
    box_extent(bx, box, &ex, &ey, &ez);
    int x, y, z;
    vox_xyz(li, bx.nx, bx.ny, nvox, &x, &y, &z);
    const int64_t i = (int64_t)box * nvox + li;
    uint32_t w = fmt ? GC_ABSENT : 0u;
    if (x < ex && y < ey && z < ez) {
        const uint8_t c = code[i];
        float gv = gtype == G_U16 ? (float)static_cast<const uint16_t*>(g)[i] * (1.0f / 65535.0f)
                                  : static_cast<const float*>(g)[i];
        if (sqrt_g) gv = sqrtf(gv);
        if (fmt) {
            const uint32_t gb = __float_as_uint(fabsf(gv));
            w = c == FREE ? gb : (c == SEED ? (gb | 0x80000000u) : GC_ABSENT);
        } else {
            const uint32_t cc = c == FREE ? 1u : (c == SEED ? 2u : 0u);
            w = cc ? ((__float_as_uint(gv) & ~3u) | cc) : 0u;
        }
    }
    gc[vec_index(pad, bx, box, x, y, z)] = w;
}

cudaError_t launch_pack_gc(const Boxes& bx, const Pad& pad, const void* g, int gtype, const uint8_t* code,
                           uint32_t* gc, cudaStream_t s, int fmt, int sqrt_g) {
    const int64_t nvox = (int64_t)bx.nx * bx.ny * bx.nz;
    dim3 grid((unsigned)((nvox + 255) / 256), (unsigned)bx.nbox);
    k_pack_gc<<<grid, 256, 0, s>>>(bx, pad, g, gtype, code, gc, fmt, sqrt_g);
    return cudaGetLastError();
}

__global__ void k_fill_u32(uint32_t* p, int64_t n, uint32_t v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

cudaError_t launch_fill_u32(uint32_t* p, int64_t n, uint32_t v, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, 65536);
    k_fill_u32<<<(unsigned)blocks, 256, 0, s>>>(p, n, v);
    return cudaGetLastError();
}

__global__ void k_copy_out(int64_t n, const double* x, float* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (float)x[i];
}

cudaError_t launch_copy_out(int fp64, const Boxes& bx, const void* x, float* out, cudaStream_t s) {
    (void)fp64;
    const int64_t n = (int64_t)bx.nbox * bx.nx * bx.ny * bx.nz;
    k_copy_out<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, static_cast<const double*>(x), out);
    return cudaGetLastError();
}

}  // namespace rwk
