// Internal declarations shared by the CUDA translation units of librw.so.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rwk {

enum : uint8_t { FREE = 0, SEED = 1, ABSENT = 2 };

// Per-system PCG state that lives on the device (one per box).
struct BoxScalars {
    double gam;      // gamma_k = (r_k, u_k) of the last sweep
    double alpha;    // alpha for the next sweep
    double beta;     // beta for the next sweep
    double rr;       // ||r||^2 (recursive)
    double bb;       // ||b||^2
    double tol2;     // the round stops when rr <= tol2
    double rr_true;  // FP64 ||b - A x||^2 of the last residual sweep
    double dbeta;    // adjoint: dl/dbeta
    double alpha_keep;  // alpha_k kept across a residual replacement (phase 2)
    int iters;       // regular sweeps completed (all rounds)
    int max_iter;
    int active;      // 1 while the box iterates
    int phase;       // next sweep: 0 restart (p = u), 1 regular, 2 inner products of a replaced residual
    int par;         // buffer (0/1) holding the system's latest u and p
    int nseed;
    int nfree;
    unsigned counter;  // arrival counter of the last-block reduction
    int status;      // 0 ok, 5 breakdown (restart next round)
    int moved;       // 1 when the box iterates in the current refinement round (its x changes)
};

// A batch of equally sized boxes: box b covers [0,nx) x [0,ny) x [0,nz) in
// its own storage; voxels at or beyond ext[b] are absent.
struct Boxes {
    int nbox;
    int nx, ny, nz;
    const int* ext;  // device [nbox][3] (x, y, z) or nullptr = full box
};

// TMA descriptors of the strip sweep's streamed arrays (u_in, p_in, g words,
// delta), encoded by the host for the launch's buffers and tile.
struct StripMaps {
    CUtensorMap u, p, g, x;
    CUtensorMap ua, pa;  // u and p of the other parity (the looped sweep's odd iterations)
};

struct SweepArgs {
    Boxes bx;
    int ntx, nty, nzc, zc;  // tiles per box: x, y, z-chunks; chunk depth
    const void* g;          // intensities (uint16 unorm or float), FP64 sweep
    const uint8_t* code;    // seed codes, FP64 sweep
    const uint32_t* gc;     // packed FP32 g | code (0 absent, 1 free, 2 seed), FP32 sweep
    void* x;                // iterate (T)
    const void* u_in;       // u_k   (T)
    const void* p_in;       // p_k-1 (T)
    void* u_out;            // u_k+1 (T)
    void* p_out;            // p_k   (T)
    BoxScalars* sc;
    double* partials;       // [list position or box][tiles][6]
    int* n_active;
    const int* list = nullptr;   // optional: the systems to sweep (ascending box indices), else all
    const int* nlist = nullptr;  // length of `list` (device), read by every launch
    int parity;             // index of the (u, p) buffers this launch reads
    int px, py, pz;         // box dims of the streamed vectors (k_sweep5: Pad of the strip layout)
    float c2f;              // -beta * log2(e), FP32 weights
    float wminf;
    double mbeta;           // -beta, FP64 weights
    double wmin;
    int* err = nullptr;     // set to 1 by a strip sweep whose load or grid wait ran out
    int loop_iters = 1;     // looped strip sweep: PCG iterations per launch
    int loop_stop = 0;      // looped strip sweep: stop once at most this many systems are active
    unsigned* gsync = nullptr;  // looped strip sweep: {arrivals, generation, go[2], iterations done}
    int barrier_extra = 0;      // looped strip sweep: arrivals its grid barrier expects beyond the grid
                                // (0; 1 only under the host's fault injection, so that every wait runs out)
    int sqrt_g = 0;         // Poisson weights: FP64 sweep reads sqrt(g) (the g words are packed so)
    StripMaps tm;           // k_sweep5 only
};

enum GType { G_U16 = 0, G_F32 = 1 };
// Sweep tiles.  The ids are part of the ABI (RW_TILE_* in rw_api.h); ids
// missing here are not assigned.
enum TileId {
    TILE_40x8 = 3,   // FP64 sweep (k_sweep)
    TILE_32x8 = 7,   // FP64 sweep, and the FP32 k_sweep2 for boxes narrower than a strip tile
    // FP32 strip kernel (k_sweep5, strips of 4 voxels), its own layout (Pad)
    TILE_S64x11 = 20, TILE_S32x22 = 21, TILE_S32x20 = 22, TILE_S64x8 = 23, TILE_S40x20 = 24, TILE_S40x8 = 25,
    TILE_S32x20_D3 = 31, TILE_S64x8_D3 = 32, TILE_S32x22_D1 = 33, TILE_S64x8_D1 = 34, TILE_S64x14_D1 = 35,
    // strips whose p_k and u' are exchanged through the TMA ring slots
    TILE_R64x14_D2 = 36, TILE_R64x14_D1 = 37, TILE_R64x11_D2 = 38, TILE_R64x11_D3 = 39, TILE_R32x22_D2 = 40,
    TILE_R32x20_D3 = 41, TILE_R64x13_D3 = 42, TILE_R64x12_D3 = 43,
    // brick tiles (40-voxel boxes) with the ring exchange
    TILE_R40x20_D2 = 44, TILE_R40x20_D3 = 45, TILE_R40x8_D2 = 46 };
constexpr int N_TILES = 47;
constexpr int TILE_RING_FIRST = TILE_R64x14_D2;  // k_sweep5 with the ring exchange
constexpr int TILE_STRIP_FIRST = TILE_S64x11;    // tiles from here on: k_sweep5, the strip layout
// Whether a tile id names a compiled sweep of this precision.
inline bool tile_compiled(int fp64, int tile) {
    if (fp64) return tile == TILE_40x8 || tile == TILE_32x8;
    return tile == TILE_32x8 || (tile >= TILE_S64x11 && tile <= TILE_S40x8) ||
           (tile >= TILE_S32x20_D3 && tile < N_TILES);
}
// the strip width of k_sweep5 (4), else 2
inline int tile_margin(int tile) { return tile >= TILE_STRIP_FIRST ? 4 : 2; }

// Sweep launchers (sweep_*.cu).  Return cudaErrorInvalidValue for a
// combination that is not instantiated.
// Looped strip sweep (cooperative launch, up to a.loop_iters iterations; brick
// tiles only: cudaErrorInvalidValue otherwise) and its resident CTAs per SM.
cudaError_t sweep5_launch_loop(int tile, const SweepArgs& a, int grid, cudaStream_t s);
int sweep5_occupancy_loop(int tile);
cudaError_t launch_sweep(int fp64, int gtype, int tile, const SweepArgs& a, int grid, cudaStream_t s);

// Cluster-resident PCG (cluster_kernel.cu): one thread-block cluster per
// system, the system's FP32 state in the shared memory of its CTAs across the
// iterations of a launch.  Systems of at most kClusterMaxDim voxels per axis
// and at least as many z planes as CTAs per cluster, in the strip kernels'
// layout.
constexpr int kClusterMaxDim = 40;
constexpr int kClusterSize = 16;
// The cluster-resident solver takes over once the active systems are at most
// kClusterTurns per resident cluster (the clusters take the systems in turn):
// an iteration of a 40^3 system there costs about 5.6 us, a looped batched
// iteration of n such systems about 14 + 0.43 n us.
constexpr int kClusterTurns = 4;
struct ClusterArgs {
    float* u[2];              // u and p buffers by parity (BoxScalars::par)
    float* p[2];
    float* x;                 // FP32 correction delta
    const uint32_t* gc;       // signed g words (+g free, -g seed, NaN absent)
    int px, py, pz;           // box dims of the streamed vectors (the strip kernel's layout)
    int nx, ny, nz;           // box dims
    int rs, rows;             // shared-memory row stride (floats, cluster_row_stride) and own rows per CTA (cluster_rows)
    BoxScalars* sc;
    const int* list;          // compacted active systems, or nullptr (all, skipping inactive)
    const int* nlist;
    int nbox;
    int* n_active;            // decremented once per system that stops
    int* done;                // max over systems of the iterations run in the launch
    int loop_iters;           // iteration budget per system and launch
    float c2f, wminf;         // weight parameters (as SweepArgs)
};
int cluster_row_stride(int nx);
int cluster_rows(int ny, int nz, int cl);
size_t cluster_smem_bytes(int nx, int ny, int nz, int cl);
int cluster_max_active(int nx, int ny, int nz, int cl);
cudaError_t launch_brick_cluster(const ClusterArgs& a, int nclusters, int cl, cudaStream_t s);
size_t sweep_smem_bytes(int fp64, int tile);
void tile_dims(int tile, int* tx, int* ty);
int sweep_threads(int tile);
cudaError_t sweep_prepare(int fp64, int gtype, int tile);  // opt-in dynamic smem
int sweep_occupancy(int fp64, int gtype, int tile);         // resident CTAs per SM (0: not instantiated)

// Layout of the vectors streamed by k_sweep5 (px != 0): a box is [pz][py][px]
// and user voxel (x, y, z) sits at (x + mx, y + my, z + mz).  The strip
// kernel's layout has no margins (its TMA loads fill everything outside the
// box: zeros for u, p and delta, NaN -- absent -- for the g words) and px = nx
// rounded up to a multiple of 4 (16-byte rows; the extra columns are absent
// voxels).  px = 0: the unpadded caller layout.
struct Pad {
    int px, py, pz;
    int mx, my, mz;
};

__host__ __device__ __forceinline__ int64_t vec_index(const Pad& pd, const Boxes& bx, int box, int x, int y,
                                                      int z) {
    if (pd.px == 0) return (((int64_t)box * bx.nz + z) * bx.ny + y) * bx.nx + x;
    return (((int64_t)box * pd.pz + (z + pd.mz)) * pd.py + (y + pd.my)) * pd.px + (x + pd.mx);
}

// (x, y, z) of the linear index li of an nx * ny * nz box: 32-bit division
// when the box has fewer than 2^31 voxels, 64-bit otherwise.
__host__ __device__ __forceinline__ void vox_xyz(int64_t li, int nx, int ny, int64_t nvox, int* x, int* y, int* z) {
    if (nvox <= 0x7fffffff) {
        const uint32_t l = (uint32_t)li, q = l / (uint32_t)nx;
        *x = (int)(l - q * (uint32_t)nx);
        *y = (int)(q % (uint32_t)ny);
        *z = (int)(q / (uint32_t)ny);
    } else {
        *x = (int)(li % nx);
        *y = (int)((li / nx) % ny);
        *z = (int)(li / ((int64_t)nx * ny));
    }
}

// Residual / initial guess (solve_kernels.cu).
struct ResidArgs {
    Boxes bx;
    const void* g;
    int gtype;
    const uint8_t* code;
    const float* value;    // seed values (nullable)
    const float* x0;       // initial guess (nullable)
    const float* rhs;      // extra right-hand side on free voxels (nullable)
    void* x;               // FP64 solution x_hi
    void* u;               // out: u = D^-1 r  (T), buffer 0
    void* p;               // p buffer 0 (T): zeroed, or kept (keep_p)
    void* p_other;         // p buffer 1 (T): source when a system's latest p is there
    const BoxScalars* sc;  // for keep_p: which buffer holds each system's p
    int keep_p;            // 1: residual replacement keeps the search direction
    Pad pad;               // layout of u, p and delta
    double* part;          // [nbox][blocks][4]: bb, rr, nseed, nfree
    int blocks_per_box;
    double mbeta, wmin;
    // optional FP64 forward edge weights (+x, +y, +z planes of nbox*nvox
    // each, caller layout) from launch_weights64; null: computed in place
    const double* w3 = nullptr;
    int sqrt_g = 0;  // Poisson weights: the Gaussian form on sqrt(g) (mbeta is then -beta/2)
    int only_moved = 0;  // 1: skip the boxes that did not iterate in the last round (their residual stands)
};
cudaError_t launch_init_x(int fp64, const ResidArgs& a, cudaStream_t s);
// FP64 edge weights, each edge once (its lower voxel's forward edge), for the
// residual rounds of one solve: w3 holds 3 * nbox * nvox doubles.
cudaError_t launch_weights64(const ResidArgs& a, double* w3, cudaStream_t s);
// fp64 = 0: also clears the FP32 correction vector `delta`.
cudaError_t launch_residual(int fp64, const ResidArgs& a, float* delta, cudaStream_t s);
cudaError_t launch_accumulate(const Boxes& bx, const Pad& pad, const uint8_t* code, const float* delta, double* x,
                              cudaStream_t s);
// only_moved = 1: only the boxes that iterated in the last round (BoxScalars::moved)
cudaError_t launch_box_reduce(const double* part, int blocks_per_box, int nbox, BoxScalars* sc, int first,
                              cudaStream_t s, int only_moved = 0);
cudaError_t launch_start_round(BoxScalars* sc, int nbox, int round, double tol, double eps_inner, int max_iter,
                               int restart, int* n_active, cudaStream_t s);
cudaError_t launch_zero_homog(int fp64, const Boxes& bx, const uint8_t* code, const BoxScalars* sc, void* x,
                              cudaStream_t s);
cudaError_t launch_copy_out(int fp64, const Boxes& bx, const void* x, float* out, cudaStream_t s);
// list <- the active systems in ascending order, *nlist <- their number (one CTA).
cudaError_t launch_compact_active(const BoxScalars* sc, int nbox, int* list, int* nlist, cudaStream_t s);
// Pack g and the seed code of every voxel into one word for the FP32 sweep:
// fmt 0 (k_sweep2/3/4): code in the two lowest mantissa bits; fmt 1
// (k_sweep5): +g free, -g seed, GC_ABSENT (a NaN) absent.
constexpr uint32_t GC_ABSENT = 0xffc00000u;
cudaError_t launch_pack_gc(const Boxes& bx, const Pad& pad, const void* g, int gtype, const uint8_t* code,
                           uint32_t* gc, cudaStream_t s, int fmt = 0, int sqrt_g = 0);
cudaError_t launch_fill_u32(uint32_t* p, int64_t n, uint32_t v, cudaStream_t s);

// Normalisation / quantisation (hier_kernels.cu).
cudaError_t launch_quantize(const void* v, int dtype, int64_t n, float lo, float hi, int normalize, int storage,
                            void* out, cudaStream_t s);

// Adjoint (adjoint_kernels.cu).
struct AdjArgs {
    Boxes bx;
    const void* g;
    int gtype;
    const uint8_t* code;
    const float* x;      // forward solution
    const double* lam;   // adjoint solution (FP64)
    float* dg;           // nullable
    double* part;        // [nbox][blocks] dbeta partials
    int blocks_per_box;
    double beta, wmin;
};
cudaError_t launch_adjoint(const AdjArgs& a, cudaStream_t s);
cudaError_t launch_adjoint_reduce(const double* part, int blocks_per_box, int nbox, double* dbeta, cudaStream_t s);

// Hierarchy (hier_kernels.cu).
cudaError_t launch_downsample_u16(const uint16_t* fine, int nx, int ny, int nz, float* coarse, cudaStream_t s);
cudaError_t launch_downsample_f32(const float* fine, int nx, int ny, int nz, float* coarse, cudaStream_t s);
cudaError_t launch_leaf_to_f32(const uint16_t* q, int64_t n, float* out, cudaStream_t s);

struct BrickJob {      // one active node of level k
    int bx, by, bz;    // brick index
    int rx0, ry0, rz0; // clipped neighbourhood origin (level voxels)
    int ex, ey, ez;    // clipped neighbourhood extent
    int faces;         // bit f set: face f (x0,x1,y0,y1,z0,z1) lies inside the level volume -> border seeds
    int pad;
};
struct LabelVox {      // a rasterised label voxel at level k
    int x, y, z;
    float value;
    int flags;         // 1: conflict, 2: conflict involves an added label
};
struct GatherArgs {
    Boxes bx;                  // pool boxes (E^3 padded)
    const BrickJob* jobs;
    const float* gf;           // level intensities (FP32) or nullptr when gq used
    const uint16_t* gq;        // leaf unorm16 (leaf level) or nullptr
    int lx, ly, lz;            // level dims
    const float* parent;       // filled level k-1 (nullptr at the root)
    int px, py, pz;            // parent dims
    const float* init;         // initial guess field at level k (nullptr: use the upsample / 0)
    float* g_out;              // pool intensities (FP32)
    uint8_t* code_out;
    double* x_out;             // pool FP64 iterate
};
cudaError_t launch_gather(const GatherArgs& a, cudaStream_t s);
cudaError_t launch_apply_labels(const Boxes& bx, const BrickJob* jobs, const LabelVox* lab, int nlab,
                                uint8_t* code, double* x, int* box_flags, cudaStream_t s);
struct ContractArgs {
    Boxes bx;
    const BrickJob* jobs;
    int s;                 // brick size
    const double* x;       // pool solution (FP64)
    float* field;          // level k field (written on the brick box unless stats_only or skip[box])
    const float* old;      // old level k field (nullable) for max |new - old|; may equal field when stats_only
    int lx, ly, lz;
    float* stats;          // [nbox][3]: min, max, maxdiff
    int stats_only = 0;    // 1: statistics only, the field is not written
    const int* skip = nullptr;  // per box, nonzero: nothing is written (nullable)
};
cudaError_t launch_contract(const ContractArgs& a, cudaStream_t s);
struct FillArgs {
    float* field;
    int lx, ly, lz;
    const float* parent;    // level k-1 filled field (nullptr at root)
    int px, py, pz;
    const uint8_t* status;  // per brick: 0 = write the upsampled parent, otherwise keep (in place)
    int nbx, nby, nbz, s;
};
cudaError_t launch_fill(const FillArgs& a, cudaStream_t s);
// Class fields of one level for the multi-class argmax.
struct ClassFields {
    const float* P[8];
    int n;
};
// Argmax over the bricks in `nodes` (linear brick indices of a level of
// lx x ly x lz voxels in bricks of s, nbx x nby bricks per plane), outputs in
// the level's layout.
cudaError_t launch_argmax_nodes(const ClassFields& f, int lx, int ly, int lz, int s, int nbx, int nby,
                                const int64_t* nodes, int64_t n_nodes, uint8_t* labels, float* prob, cudaStream_t st);
cudaError_t launch_argmax(const ClassFields& f, int lx, int ly, const int64_t box[6], uint8_t* labels, float* prob,
                          cudaStream_t s);
cudaError_t launch_brick_io(float* field, int lx, int ly, int lz, int s, int nbx, int nby, const int64_t* nodes,
                            int64_t n, float* packed, int to_packed, cudaStream_t st);
cudaError_t launch_read_box(const float* field, int lx, int ly, int lz, const int64_t box[6], float* out,
                            cudaStream_t s);

}  // namespace rwk
