/* rw_api.h — C ABI of the GB300 hierarchical random walker library (librw.so).
 *
 * The method is the random walker of Sec. III-B of "Hierarchical Random Walker
 * Segmentation for Large Volumetric Biomedical Images" (Drees, Eilers, Jiang,
 * arXiv 2103.09564) and its hierarchical form H / H_p (Sec. IV, Eqs. 1-3).
 *
 * Conventions shared by every entry point
 * - Arrays are dense, x fastest: element (x, y, z) of volume b is at
 *   ((b * dims[2] + z) * dims[1] + y) * dims[0] + x.
 * - Pointers may be device pointers (used in place) or host pointers (the
 *   library copies them through its workspace); the kind is detected with
 *   cudaPointerGetAttributes.  Caller-owned memory is never freed or kept.
 * - Opaque handles (rw_pyramid, rw_tree) are owned by the library and freed
 *   by the matching *_free call.
 * - Every call runs on `stream` (a cudaStream_t, NULL = legacy default
 *   stream) and synchronises it before returning, so outputs and rw_stats are
 *   valid on return.  Device-side conditions (non-convergence) are reported
 *   through the status of the same call.
 * - Errors: a non-RW_OK status; rw_last_error() returns a thread-local text.
 *   RW_ERR_NOT_CONVERGED still writes the best iterate.
 * - The library keeps one internal device workspace (grown with cudaMalloc,
 *   released by rw_release_workspace); calls are serialised by a mutex.
 */
#ifndef RW_API_H
#define RW_API_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum rw_status {
    RW_OK = 0,
    RW_ERR_INVALID_ARG = 1,    /* bad pointer, size, dtype or option */
    RW_ERR_NO_SEEDS = 2,       /* a system without any seed has no unique solution */
    RW_ERR_NOT_CONVERGED = 3,  /* max_iter reached before the tolerance */
    RW_ERR_TIMEOUT = 4,        /* a bounded wait inside a sweep kernel (a TMA load, a grid barrier)
                                  ran out: the kernel stopped waiting, flagged it and returned */
    RW_ERR_OOM = 5,            /* device allocation failed */
    RW_ERR_CUDA = 6,           /* a CUDA runtime call failed */
    RW_ERR_UNIMPLEMENTED = 7
} rw_status;

typedef enum rw_dtype { RW_U16 = 0, RW_F32 = 1 } rw_dtype;

/* How intensities are stored on the device after normalisation.
 * UNORM16: q = round_half_even(g * 65535) (2 B/voxel, the default; weights
 * then see g = q / 65535).  F32: g kept as FP32 (needed for gradients). */
typedef enum rw_storage { RW_STORE_UNORM16 = 0, RW_STORE_F32 = 1 } rw_storage;

/* RW_MIXED: FP32 vectors and stencil, FP64 reductions and FP64-residual
 * iterative refinement.  RW_FP64: every vector and weight in FP64. */
typedef enum rw_precision { RW_MIXED = 0, RW_FP64 = 1 } rw_precision;

/* Seed codes of rw_seed_mask.code. */
enum { RW_CODE_FREE = 0, RW_CODE_SEED = 1, RW_CODE_ABSENT = 2 };

/* Node flags returned by rw_tree_node_stats (one int32 per brick). */
enum {
    RW_NODE_SOLVED = 1, RW_NODE_PRUNABLE = 2, RW_NODE_HOM = 4, RW_NODE_DT = 8,
    RW_NODE_CFL = 16, RW_NODE_SIMILAR = 32, RW_NODE_REUSED = 64, RW_NODE_CFL_ADDED = 128,
    RW_NODE_NO_SEEDS = 256,
    /* the node's values changed in the pass: re-solved and not similar, or
     * absent and filled from a parent footprint that changed (every node of a
     * full refinement) */
    RW_NODE_CHANGED = 512
};

/* Intensity volume.  Normalisation (a reading: the paper applies
 * w = exp(-beta (n[p]-n[q])^2) to intensities without fixing their scale):
 *   normalize = 1: g = clamp((v - lo) / (hi - lo), 0, 1) in FP32;
 *   normalize = 0: F32 input is used as g (clamped to [0, 1]), U16 input is
 *   taken as unorm16. */
typedef struct rw_volume {
    const void* data;    /* [batch][z][y][x] */
    int32_t dtype;       /* rw_dtype */
    int32_t storage;     /* rw_storage */
    int64_t dims[3];     /* x, y, z of one volume */
    int64_t batch;       /* independent volumes, >= 1 (0 is read as 1) */
    float lo, hi;        /* normalisation window */
    int32_t normalize;
    int32_t reserved;
} rw_volume;

/* Dense seeds for the plain solve, same shape as the volume.
 * code: RW_CODE_FREE (unknown), RW_CODE_SEED (Dirichlet value from `value`),
 * RW_CODE_ABSENT (not a vertex).  value: seed values in [0, 1]; it may be
 * NULL when all seeds are background (0). */
typedef struct rw_seed_mask {
    const uint8_t* code;
    const float* value;
} rw_seed_mask;

/* Label points (Sec. IV-A: labels are 3-D points with a value in [0, 1]).
 * HOST memory.  xyz: n x 3 leaf-voxel coordinates (x, y, z); voxel i spans
 * [i, i + 1).  At level k a label falls into voxel floor(q / 2^(K-k)); a
 * voxel holding labels of different values is a conflict (unseeded).
 * cls (nullable): the class of each label in a multi-class labelling (one
 * tree per class, class c's labels with value 1, the others 0).  With it, a
 * voxel holding labels of different classes is a conflict as well, so that
 * every class tree leaves the same voxels unseeded and the class
 * probabilities sum to one (Sec. III-B). */
typedef struct rw_labels {
    const double* xyz;
    const float* value;
    int64_t n;
    const int32_t* cls;
} rw_labels;

typedef struct rw_opts {
    float beta;            /* Gaussian weight parameter (Sec. III-B), default 130 */
    float w_min;           /* lower clamp of the weights, default 1e-30 */
    double tol;            /* stop when ||b - A x||_2 <= tol ||b||_2, default 1e-8 */
    int32_t max_iter;      /* PCG iteration cap per system, default 20000 */
    int32_t precision;     /* rw_precision, default RW_MIXED */
    int32_t refine_rounds; /* FP64-residual refinement rounds (RW_MIXED), default 4 */
    int32_t brick_size;    /* s (Sec. IV-A), default 32 */
    float expand;          /* e (Sec. IV-B), default 1.25 */
    float t_hom;           /* Sec. IV-D1, default 0.3 */
    float t_bin;           /* Sec. IV-D1, default 0.01 */
    float t_inc;           /* Sec. IV-E, default 0.01 */
    int32_t prune_hom;     /* enable hom pruning, default 1 */
    int32_t prune_dt;      /* enable dt pruning, default 1 */
    int32_t iters_per_graph; /* PCG sweeps per captured CUDA graph (even) with a fixed tile, default 32;
                                the autotuner sizes graphs to about 4 ms of sweeps (8-32) */
    int32_t tile;          /* sweep tile: 0 = autotuned choice, else an RW_TILE_* value */
    int32_t batch_bricks;  /* 1: one batched launch per level (default); 0: bricks one by one */
    int32_t max_batch;     /* bricks per batched launch, default 8192 */
    int32_t weight;        /* rw_weight: edge weight function, default RW_WEIGHT_GAUSSIAN */
    int32_t leaf_field;    /* rw_leaf_field: where a tree keeps its leaf-level field, default
                              RW_LEAF_AS_PYRAMID (placement only: results are identical) */
} rw_opts;

/* Edge weight functions (Sec. III-B / III-C).
 *   RW_WEIGHT_GAUSSIAN: w = max(exp(-beta (g_p - g_q)^2), w_min).
 *   RW_WEIGHT_POISSON:  the weight for Poisson noise of the paper's case
 *     study, w = exp(-(sqrt(n_p) - sqrt(n_q))^2 / 2) on raw counts n; here
 *     n = beta * g (beta = the count that g = 1 stands for, e.g. the window's
 *     hi with lo = 0), i.e. w = max(exp(-(beta / 2) (sqrt(g_p) - sqrt(g_q))^2),
 *     w_min).  Forward solves only (rw_solve, the hierarchy); rw_solve_adjoint
 *     and rw_solve_noalloc return RW_ERR_UNIMPLEMENTED. */
typedef enum { RW_WEIGHT_GAUSSIAN = 0, RW_WEIGHT_POISSON = 1 } rw_weight;

/* Sweep tiles (rw_opts.tile).  Any other value, or a tile of the other
 * precision, is rejected with RW_ERR_INVALID_ARG. */
enum { RW_TILE_AUTO = 0,
       /* FP64 sweeps (RW_FP64 and the FP64 fallback); 32x8 is also the FP32
        * tile for boxes narrower than 25 voxels in x */
       RW_TILE_40x8 = 3, RW_TILE_32x8 = 7,
       /* FP32 register-blocked strips of 4 voxels:
        * 2 planes in flight, 3 (_D3) or 1 (_D1; s64x14_d1: 320 threads) */
       RW_TILE_S64x11 = 20, RW_TILE_S32x22 = 21, RW_TILE_S32x20 = 22, RW_TILE_S64x8 = 23,
       RW_TILE_S40x20 = 24, RW_TILE_S40x8 = 25,
       RW_TILE_S32x20_D3 = 31, RW_TILE_S64x8_D3 = 32, RW_TILE_S32x22_D1 = 33, RW_TILE_S64x8_D1 = 34,
       RW_TILE_S64x14_D1 = 35,
       /* strips of 4 whose p_k and u' are exchanged through the load ring (_D: planes ahead) */
       RW_TILE_R64x14_D2 = 36, RW_TILE_R64x14_D1 = 37, RW_TILE_R64x11_D2 = 38, RW_TILE_R64x11_D3 = 39,
       RW_TILE_R32x22_D2 = 40, RW_TILE_R32x20_D3 = 41, RW_TILE_R64x13_D3 = 42, RW_TILE_R64x12_D3 = 43,
       RW_TILE_R40x20_D2 = 44, RW_TILE_R40x20_D3 = 45, RW_TILE_R40x8_D2 = 46 };

typedef struct rw_stats {
    int32_t iters;          /* max PCG iterations over the systems of the call */
    int32_t refine_rounds;  /* FP64-residual rounds run */
    double rel_resid;       /* max over systems of the final FP64 ||b - A x|| / ||b|| */
    int64_t voxel_iters;    /* sum over systems of free voxels x iterations */
    int64_t free_voxels;    /* sum of free voxels */
    int64_t bricks_active;  /* nodes processed by the call */
    int64_t bricks_solved;
    int64_t bricks_pruned;
    int64_t bricks_reused;
    int64_t bricks_conflict;
    int64_t sweeps;         /* fused PCG sweep kernels launched */
    double ms;              /* wall time of the call */
    double ms_solve;        /* time inside the PCG loops */
    double ms_sweeps;       /* device time of the fused sweeps (CUDA events on the library stream) */
    int64_t launches;       /* kernels launched by the call */
    int32_t tile;           /* sweep tile used last (RW_TILE_*) */
    int32_t iters_per_graph;/* sweeps per CUDA graph used last */
    int64_t not_converged;  /* systems left above tol (bricks keep their best iterate) */
    int64_t fp64_fallbacks; /* solves that finished with FP64 sweeps */
} rw_stats;

typedef struct rw_pyramid rw_pyramid;
typedef struct rw_tree rw_tree;

/* Limits of rw_solve_noalloc (its scratch is a fixed device array). */
#define RW_NOALLOC_MAX_VOXELS 262144  /* voxels over the whole batch (64^3) */
#define RW_NOALLOC_MAX_BATCH 64

void rw_opts_default(rw_opts* opts);
const char* rw_last_error(void);
const char* rw_version(void);
/* Frees the internal workspace (cached device buffers). */
rw_status rw_release_workspace(void);

/* Plain random walker, Sec. III-B: for each of `vol->batch` volumes solve
 *   L_U x_U = -B^T x_M   (Dirichlet problem, 6-connected graph,
 *   w_pq = max(exp(-beta (g_p - g_q)^2), w_min))
 * by matrix-free Jacobi-PCG.  x0: optional initial guess (NULL = 0) on free
 * voxels, same layout as the volume.  x_out: full result (seeds carry their
 * value, absent voxels 0), float32, same layout.  Returns RW_ERR_NO_SEEDS if
 * a volume has no seed.  A volume whose right-hand side is 0 gets x_U = 0. */
rw_status rw_solve(const rw_volume* vol, const rw_seed_mask* seeds, const rw_opts* opts,
                   const float* x0, float* x_out, rw_stats* stats, void* stream);

/* rw_solve for callers that cannot allocate device memory.  The paper has no
 * counterpart: this is a deployment variant of the plain solve above.
 * Some callers must not call cudaMalloc/cudaFree while they run — an
 * interactive labelling loop with a latency budget (both calls can
 * synchronise the whole device), a plug-in inside a host application that
 * owns the GPU memory budget, a service that fixes its footprint at start-up.
 * This entry point allocates nothing: its scratch is one file-scope device
 * array of about 12.1 MB that every GPU loading the library keeps until the
 * process exits.  Same arguments and results as rw_solve, with these
 * differences:
 *  - every array must be device memory of the current device, or managed
 *    memory (no host staging); anything else is RW_ERR_INVALID_ARG;
 *  - at most RW_NOALLOC_MAX_VOXELS voxels in total and RW_NOALLOC_MAX_BATCH
 *    volumes; larger inputs are rejected with RW_ERR_INVALID_ARG;
 *  - opts->precision must be RW_MIXED and vol->storage RW_STORE_UNORM16; a
 *    system that FP32 sweeps cannot resolve returns RW_ERR_NOT_CONVERGED
 *    (rw_solve would finish it with FP64 sweeps);
 *  - work runs on `stream` itself (no internal stream, CUDA graph or timing
 *    event); the call synchronises the stream before it returns, and also
 *    between sweeps, where it reads the count of active systems on the host.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, once per device); make that first call before any
 * stream capture.  All calls share the array and each call clears what must
 * start at zero: calls that overlap on the GPU (from several streams or
 * threads) race and must be serialised by the caller. */
rw_status rw_solve_noalloc(const rw_volume* vol, const rw_seed_mask* seeds, const rw_opts* opts,
                           const float* x0, float* x_out, rw_stats* stats, void* stream);

/* Adjoint of rw_solve (not in the paper; gradient of a loss l(x)): solves
 * L_U lambda = (dl/dx)_U with the same PCG (L_U is symmetric) and returns
 *   dl/dg_i    = sum over edges e at i of dl/dw_e * dw_e/dg_i,
 *   dl/dbeta   = sum over edges of dl/dw_e * dw_e/dbeta,
 * with dl/dw_pq = -(lambda_p - lambda_q)(x_p - x_q) (lambda = 0 on seeds).
 * x: the solution from rw_solve.  dloss_dg (nullable): float32 like the
 * volume (gradient w.r.t. the normalised intensity g).  dloss_dbeta
 * (nullable): `batch` doubles. */
rw_status rw_solve_adjoint(const rw_volume* vol, const rw_seed_mask* seeds, const rw_opts* opts,
                           const float* x, const float* dloss_dx, float* dloss_dg,
                           double* dloss_dbeta, rw_stats* stats, void* stream);

/* LOD pyramid, Sec. III-A: leaf = normalised unorm16 volume; each coarser
 * level is the 2x2x2 mean (existing children only at odd borders, Sec. IV-A)
 * with ceil-halved dims, until every dim is <= brick_size (the root). */
rw_status rw_build_pyramid(const rw_volume* vol, int32_t brick_size, rw_pyramid** out, void* stream);

/* Placement of a tree's level fields (rw_opts.leaf_field):
 * RW_LEAF_AS_PYRAMID: as the pyramid's levels (RW_PYR_HOST_ALL: every level's
 * field in host memory; RW_PYR_LEAF_HOST: the leaf field in host memory;
 * otherwise HBM); RW_LEAF_HBM / RW_LEAF_HOST: the leaf field in HBM / in
 * pinned, mapped host memory (coarser fields in HBM); RW_FIELDS_HOST: every
 * level's field in pinned, mapped host memory. */
typedef enum rw_leaf_field {
    RW_LEAF_AS_PYRAMID = 0, RW_LEAF_HBM = 1, RW_LEAF_HOST = 2, RW_FIELDS_HOST = 3
} rw_leaf_field;

/* rw_build_pyramid with placement flags.  RW_PYR_LEAF_HOST: the leaf level
 * (its unorm16 intensities here, and by default the leaf probability fields
 * of the trees created on this pyramid) lives in pinned, mapped host memory instead
 * of HBM; the GPU reads and writes it in place over the host link.  This is
 * the out-of-core mode of Sec. III (volumes whose leaf does not fit in GPU
 * memory): only the coarser levels (about 1/7 of the leaf) and the brick
 * batches of one level occupy HBM.  Results are identical to the HBM
 * placement.  Unknown flag bits: RW_ERR_INVALID_ARG. */
#define RW_PYR_LEAF_HOST 1
/* RW_PYR_HOST_ALL: every level of the pyramid in pinned, mapped host memory,
 * and by default every level's field of the trees built on it: HBM then holds
 * only the working set of one batched level solve (the brick pool and solver
 * vectors of at most rw_opts.max_batch bricks) and the library's workspace.
 * A host input volume is normalised in z-slabs of at most 256 MB, so no
 * device copy of the whole volume is made.  The paper streams bricks from
 * disk (Sec. III-A, IV-A); here the backing store is the host memory the GPU
 * reads and writes in place over the coherent host link. */
#define RW_PYR_HOST_ALL 2
rw_status rw_build_pyramid_ex(const rw_volume* vol, int32_t brick_size, int32_t flags, rw_pyramid** out,
                              void* stream);
/* Number of levels and their dims (levels x 3, x/y/z; level 0 = root). */
rw_status rw_pyramid_info(const rw_pyramid* pyr, int32_t* n_levels, int64_t* dims);
/* Copy level `level` (FP32 intensities; the leaf as q / 65535) to `out`. */
rw_status rw_pyramid_read_level(const rw_pyramid* pyr, int32_t level, float* out, void* stream);
void rw_pyramid_free(rw_pyramid* pyr);

/* Output tree of H_p over `pyr` (kept alive by the caller until rw_tree_free). */
rw_status rw_tree_create(const rw_pyramid* pyr, const rw_opts* opts, rw_tree** out);

/* One level of the top-down procedure (Fig. 3).  level 0: root solve (Eq. 1)
 * with `labels` (stored in the tree; NULL keeps the stored ones).  level k >= 1:
 * all children of solved, non-prunable level-(k-1) nodes are solved in
 * batched launches on their neighbourhood (Eq. 3, s_e = floor(e s)) with user
 * seeds and continuous border seeds upsampled from level k-1 (Eq. 2), started
 * from the upsampled parent (Sec. IV-D2); hom / dt / cfl / prunable are
 * evaluated (Sec. IV-D1); absent nodes take the upsampled parent field.
 * Levels must be refined in order 0, 1, ..., K. */
rw_status rw_refine_level(rw_tree* tree, int32_t level, const rw_labels* labels, rw_stats* stats,
                          void* stream);

/* Incremental labelling, Sec. IV-E: add labels and update every level: the
 * root is re-solved from the old root; children of re-solved nodes that are
 * neither similar (max |new - old| < t_inc without conflicts involving added
 * labels) nor prunable are re-solved from the old field; similar nodes keep
 * their old values and whole old subtree.  Requires a fully refined tree. */
rw_status rw_update_seeds(rw_tree* tree, const rw_labels* added, rw_stats* stats, void* stream);

/* rw_update_seeds on n_trees trees at once (e.g. one per class of a
 * multi-class labelling, Sec. III-B): added[i] (array of n_trees entries,
 * NULL: no new labels) goes to trees[i].  The result of every tree is the one
 * rw_update_seeds gives (up to the rounding of a differently composed batch:
 * reduction orders differ); at each level the nodes of all trees are solved in
 * shared batched launches, so the PCG iterations of the trees run
 * concurrently.  `stats` (nullable) sums over the trees.  RW_ERR_INVALID_ARG
 * unless the trees are distinct, fully refined, on one pyramid and have equal
 * options. */
rw_status rw_update_seeds_trees(rw_tree* const* trees, int32_t n_trees, const rw_labels* added, rw_stats* stats,
                                void* stream);

/* Multi-class labelling (Sec. III-B: one random-walker problem per class,
 * class c's labels as 1 and every other class's as 0; the label of a voxel is
 * the class of highest probability).  `trees` holds one refined tree per
 * class (2 <= n_classes <= RW_MAX_CLASSES), all on one pyramid.  Over box
 * [x0,x1) x [y0,y1) x [z0,z1) of `level` (box NULL: the whole level) writes
 * labels_out[i] = argmax_c P_c[i] (ties: the lowest class index) and, when
 * prob_out is not NULL, the winning probability.  Outputs: host or device
 * memory, x fastest.  RW_ERR_INVALID_ARG for a bad count, level or box, or
 * trees on different pyramids. */
#define RW_MAX_CLASSES 8
rw_status rw_trees_argmax(const rw_tree* const* trees, int32_t n_classes, int32_t level, const int64_t box[6],
                          uint8_t* labels_out, float* prob_out, void* stream);

/* Multi-class labels after an incremental round (Sec. IV-E): rw_trees_argmax
 * over the whole leaf level, recomputed only on the leaf bricks that changed
 * (RW_NODE_CHANGED) in the latest pass of at least one tree; every other
 * voxel of labels_out / prob_out keeps its contents.  Call it after each
 * round in which every tree ran one pass (rw_update_seeds or a full
 * refinement), on outputs holding the previous round's labels.  Outputs:
 * device or page-locked host memory, the leaf level's layout (x fastest);
 * RW_ERR_INVALID_ARG for other memory, a bad count, unrefined trees or trees
 * on different pyramids. */
rw_status rw_trees_argmax_changed(const rw_tree* const* trees, int32_t n_classes, uint8_t* labels_out,
                                  float* prob_out, void* stream);

/* Copy box [x0,x1) x [y0,y1) x [z0,z1) (box = {x0,y0,z0,x1,y1,z1}) of the
 * filled probability field of `level` to `out` (x fastest). */
rw_status rw_tree_read_level(const rw_tree* tree, int32_t level, const int64_t box[6], float* out,
                             void* stream);

/* Per-node results of the last pass over `level` (host arrays of *n_nodes
 * entries, brick order x fastest; pass NULL to query the count): RW_NODE_*
 * flags, brick minimum, maximum and max |new - old| (incremental pass). */
rw_status rw_tree_node_stats(const rw_tree* tree, int32_t level, int64_t* n_nodes, int32_t* flags,
                             float* mn, float* mx, float* maxdiff);
/* Level sharding over several GPUs (Sec. IV-D3: the nodes of a level are
 * independent problems).  Each rank holds the pyramid and its own tree; a
 * level is refined in parts instead of by rw_refine_level:
 *   1. rw_tree_level_nodes lists the nodes the level solves in this pass
 *      (identical on every rank, since every rank finished the same parent
 *      level);
 *   2. rw_refine_level_nodes solves a subset of them (a rank's share, e.g. a
 *      contiguous range in Morton order); it opens the level, and may be
 *      called again for further subsets;
 *   3. rw_tree_export_nodes / rw_tree_import_nodes move solved nodes between
 *      trees (values, flags and min / max / max-diff statistics);
 *   4. rw_refine_level_finish, once every node of the level is present,
 *      evaluates the level as rw_refine_level does after its solve: the fill
 *      of absent nodes and the next level's node list.
 * Full refinements only (not incremental passes).  While a level is open,
 * rw_refine_level and rw_update_seeds on that tree return RW_ERR_INVALID_ARG.
 * Node ids are brick indices of the level, (bz * nby + by) * nbx + bx. */

/* The nodes `level` solves in this pass, ascending (pass nodes = NULL to
 * query *n_nodes).  `level` must be 0 (a new pass), the next level of the
 * pass, or the open level.  HOST arrays. */
rw_status rw_tree_level_nodes(const rw_tree* tree, int32_t level, int64_t* n_nodes, int64_t* nodes);
/* Solve the listed nodes of `level` (HOST array of n_nodes ids, each a node
 * of the level not yet present; n_nodes may be 0).  `labels` as in
 * rw_refine_level, at level 0 only.  stats.bricks_solved counts these
 * nodes. */
rw_status rw_refine_level_nodes(rw_tree* tree, int32_t level, const rw_labels* labels, const int64_t* nodes,
                                int64_t n_nodes, rw_stats* stats, void* stream);
/* Copy present nodes of the open level out: flags (RW_NODE_*, n_nodes
 * int32), node_stats (n_nodes x {min, max, max |new - old|} float32) and
 * values (n_nodes x s^3 float32, each brick x fastest; the voxels of a border
 * brick outside the level are 0).  Each output is nullable; nodes, flags and
 * node_stats are HOST arrays, values host or device memory. */
rw_status rw_tree_export_nodes(const rw_tree* tree, int32_t level, const int64_t* nodes, int64_t n_nodes,
                               int32_t* flags, float* node_stats, float* values, void* stream);
/* Write nodes of the open level that another tree solved (arrays as
 * exported; values host or device memory).  Each node must be a node of the
 * level not yet present here, its flags must carry RW_NODE_SOLVED. */
rw_status rw_tree_import_nodes(rw_tree* tree, int32_t level, const int64_t* nodes, int64_t n_nodes,
                               const int32_t* flags, const float* node_stats, const float* values, void* stream);
/* Close the open level once all its nodes are present (RW_ERR_INVALID_ARG
 * otherwise): node status, the fill of absent nodes from the parent level and
 * the next level's node list; stats count pruned nodes. */
rw_status rw_refine_level_finish(rw_tree* tree, int32_t level, rw_stats* stats, void* stream);

void rw_tree_free(rw_tree* tree);

#ifdef __cplusplus
}
#endif
#endif /* RW_API_H */
