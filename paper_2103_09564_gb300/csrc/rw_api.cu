// C ABI of librw.so (declared in include/rw_api.h), first part: argument
// checks, the device workspace, the PCG driver (refinement rounds, CUDA-graph
// chunks of fused sweeps, per-system convergence), the plain solve and the
// adjoint.  The LOD pyramid and the hierarchical tree are in rw_hier.cu.
#include <cudaTypedefs.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "rw_api.h"
#include "rw_host.h"
#include "rw_internal.h"

using namespace rwk;

namespace rwh {

thread_local std::string g_err;
std::recursive_mutex g_mu;
int64_t g_launches = 0;   // kernels launched since the current call started (guarded by g_mu)


rw_status fail(rw_status st, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}


double now_ms() {
    using namespace std::chrono;
    return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// ---------------------------------------------------------------------------
// Workspace (rw_host.h): one per device, created on first use.
std::map<int, DevWorkspace> g_ws;

rw_status ws_dev(DevWorkspace** out) {
    int dev = 0;
    CK(cudaGetDevice(&dev));
    DevWorkspace& w = g_ws[dev];
    if (!w.stream) {
        CK(cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking));
        CK(cudaMallocHost(&w.pinned, 64));
        CK(cudaDeviceGetAttribute(&w.sms, cudaDevAttrMultiProcessorCount, dev));
    }
    *out = &w;
    return RW_OK;
}

rw_status ws_get(DevWorkspace* w, int slot, size_t bytes, void** out) {
    if (bytes == 0) bytes = 256;
    if (w->cap[slot] < bytes) {
        if (w->p[slot]) {
            CK(cudaStreamSynchronize(w->stream));
            CK(cudaFree(w->p[slot]));
        }
        w->p[slot] = nullptr;
        w->cap[slot] = 0;
        size_t nb = ((bytes + bytes / 8) + 4095) & ~(size_t)4095;
        CK(cudaMalloc(&w->p[slot], nb));
        w->cap[slot] = nb;
    }
    *out = w->p[slot];
    return RW_OK;
}


bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Device address of page-locked (pinned or registered) host memory, which
// kernels can write directly; nullptr for other pointers.
void* pinned_device_alias(void* p) {
    if (!p) return nullptr;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return at.type == cudaMemoryTypeHost ? at.devicePointer : nullptr;
}

// Device view of a caller array: the pointer itself, or a staged copy.
rw_status stage_in(DevWorkspace* w, int slot, const void* p, size_t bytes, const void** out) {
    if (!p) {
        *out = nullptr;
        return RW_OK;
    }
    if (is_device_ptr(p)) {
        *out = p;
        return RW_OK;
    }
    void* d = nullptr;
    RCK(ws_get(w, slot, bytes, &d));
    CK(cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, w->stream));
    *out = d;
    return RW_OK;
}

// Caller stream -> internal stream ordering (inputs produced on `user` are complete).
rw_status enter(DevWorkspace** w, void* user) {
    RCK(ws_dev(w));
    CK(cudaStreamSynchronize(static_cast<cudaStream_t>(user)));
    return RW_OK;
}

rw_status leave(DevWorkspace* w) {
    CK(cudaStreamSynchronize(w->stream));
    CK(cudaGetLastError());
    return RW_OK;
}

rw_status check_opts(const rw_opts& o) {
    if (!(o.beta >= 0.0f) || !(o.w_min >= 0.0f) || !(o.tol >= 0.0) || o.max_iter < 1 || o.refine_rounds < 0 ||
        (o.precision != RW_MIXED && o.precision != RW_FP64) || o.iters_per_graph < 2 || o.tile < 0 || o.tile >= N_TILES ||
        o.brick_size < 2 || !(o.expand >= 1.0f) || o.max_batch < 1 ||
        (o.weight != RW_WEIGHT_GAUSSIAN && o.weight != RW_WEIGHT_POISSON) || o.leaf_field < RW_LEAF_AS_PYRAMID ||
        o.leaf_field > RW_FIELDS_HOST)
        return fail(RW_ERR_INVALID_ARG, "invalid rw_opts");
    if (o.tile != RW_TILE_AUTO && !tile_compiled(o.precision == RW_FP64, o.tile))
        return fail(RW_ERR_INVALID_ARG, "tile %d is not a sweep tile of this precision", o.tile);
    return RW_OK;
}

rw_status check_volume(const rw_volume* v, int64_t* nvox, int64_t* batch) {
    if (!v || !v->data) return fail(RW_ERR_INVALID_ARG, "volume or volume data is NULL");
    if (v->dtype != RW_U16 && v->dtype != RW_F32) return fail(RW_ERR_INVALID_ARG, "unknown dtype %d", v->dtype);
    if (v->storage != RW_STORE_UNORM16 && v->storage != RW_STORE_F32)
        return fail(RW_ERR_INVALID_ARG, "unknown storage %d", v->storage);
    for (int a = 0; a < 3; ++a)
        if (v->dims[a] < 1 || v->dims[a] > (1 << 20)) return fail(RW_ERR_INVALID_ARG, "bad dims");
    *batch = v->batch < 1 ? 1 : v->batch;
    *nvox = v->dims[0] * v->dims[1] * v->dims[2];
    if (*batch > 65535) return fail(RW_ERR_INVALID_ARG, "batch > 65535");
    if (*nvox > ((int64_t)1 << 40)) return fail(RW_ERR_INVALID_ARG, "volume too large");
    return RW_OK;
}

// ---------------------------------------------------------------------------
// Sweep configuration and the autotuner (tile shape, z-chunk, sweeps per graph).
struct SweepCfg {
    int tile = TILE_32x8, tx = 32, ty = 8, nt = 256, zc = 64, ntx = 1, nty = 1, nzc = 1, grid = 1, ipg = 32, waves = 0;
};

struct Tuned {
    int tile, ipg, waves;
};
std::map<std::string, Tuned> g_tuned;  // problem class -> autotuned sweep configuration

std::vector<int> tile_candidates(int fp64, int gtype, int nx) {
    // one list holds tiles of one layout family only (the autotuner times
    // them on the same live vectors): the strip kernel's tiles (its own
    // layout, rows of a multiple of 4 voxels), or the caller-layout k_sweep2
    // tile for boxes narrower than a strip tile
    std::vector<int> c;
    (void)gtype;
    if (fp64) {
        c = {TILE_32x8, TILE_40x8};
    } else if (nx <= 24) {
        c = {TILE_32x8};
    } else if (nx <= 48 || (nx % 40 == 0 && nx <= 160)) {
        c = {TILE_S40x20, TILE_S40x8, TILE_R40x20_D2, TILE_R40x20_D3, TILE_R40x8_D2};
    } else {
        c = {TILE_S64x11,    TILE_S32x22,    TILE_S32x20,    TILE_S64x8,     TILE_S32x20_D3,
             TILE_S64x8_D3,  TILE_S32x22_D1, TILE_S64x8_D1,  TILE_S64x14_D1, TILE_R64x14_D2,
             TILE_R64x14_D1, TILE_R64x11_D2, TILE_R64x11_D3, TILE_R32x22_D2, TILE_R32x20_D3,
             TILE_R64x13_D3, TILE_R64x12_D3};
    }
    std::vector<int> ok;
    for (int t : c)
        if (sweep_occupancy(fp64, gtype, t) > 0) ok.push_back(t);
    return ok;
}

// Even z-chunk depth that minimises the modelled sweep time: a work item
// costs its planes plus a fixed pipeline fill and reduction (~5 plane steps),
// items run in waves of `slots` resident CTAs, at most `max_items` items.
int model_zc(int64_t per_plane, int nz, int64_t slots, int64_t max_items) {
    int best_zc = nz + (nz & 1);
    double best = 1e300;
    for (int zc = 2;; zc += 2) {
        const int64_t items = per_plane * ((nz + zc - 1) / zc);
        if (items <= max_items) {
            const double cost = (double)((items + slots - 1) / slots) * (zc + 5);
            if (cost < best) {
                best = cost;
                best_zc = zc;
            }
        }
        if (zc >= nz) break;
    }
    return best_zc;
}

// waves = 0: the z-chunking of the cost model (model_zc); waves = k >= 1: as
// many z-chunks as fill k whole waves of the persistent grid.
rw_status make_cfg(int fp64, int gtype, int tile, const Boxes& bx, int sms, int ipg, SweepCfg* c, int waves = 0) {
    if (sweep_occupancy(fp64, gtype, tile) <= 0) {
        return fail(RW_ERR_INVALID_ARG, "sweep tile %d not available for this precision/storage", tile);
    }
    CK(sweep_prepare(fp64, gtype, tile));
    c->tile = tile;
    tile_dims(tile, &c->tx, &c->ty);
    c->nt = sweep_threads(tile);
    c->ntx = (bx.nx + c->tx - 1) / c->tx;
    c->nty = (bx.ny + c->ty - 1) / c->ty;
    const int occ = std::max(1, sweep_occupancy(fp64, gtype, tile));
    const int64_t per_plane = (int64_t)bx.nbox * c->ntx * c->nty;
    const int64_t slots = (int64_t)occ * sms;
    int zc;
    if (waves > 0) {
        const int nzc = (int)std::max<int64_t>(1, (waves * slots) / per_plane);
        zc = std::max((bx.nz + nzc - 1) / nzc, std::min(bx.nz, 2));
    } else {
        zc = model_zc(per_plane, bx.nz, slots, INT64_MAX);
    }
    zc = (zc + 1) & ~1;  // chunks start at even planes (the strip kernel's unrolled z loop)
    c->waves = waves;
    c->zc = zc;
    c->nzc = (bx.nz + zc - 1) / zc;
    const int64_t nwork = per_plane * c->nzc;
    c->grid = (int)std::min<int64_t>(nwork, (int64_t)occ * sms);
    c->ipg = ipg;
    return RW_OK;
}

std::string class_key(int fp64, int gtype, const Boxes& bx) {
    char b[160];
    int nb = 1;
    while (nb < bx.nbox) nb *= 4;
    snprintf(b, sizeof(b), "%d/%d/%dx%dx%d/%d", fp64, gtype, bx.nx, bx.ny, bx.nz, nb);
    return b;
}

// ---------------------------------------------------------------------------
// The PCG driver.


// TMA descriptors for a strip-sweep launch: the arrays as 4-D tensors
// [nbox][PZ][PY][PX] of 4-byte words; boxes (TX + 2V) x (TY + 3) x 1 x 1 for u,
// p and the g words, TX x TY x 1 x 1 for delta.  `loop` adds the maps of
// u_out / p_out, read by the odd iterations of a looped sweep.
rw_status strip_maps(int tile, SweepArgs* sa, bool loop = false) {
    if (tile < TILE_STRIP_FIRST) return RW_OK;
    static PFN_cuTensorMapEncodeTiled_v12000 encode = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }();
    if (!encode) return fail(RW_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
    int tx, ty;
    tile_dims(tile, &tx, &ty);
    const int v = tile_margin(tile);
    // 4-D maps (x, y, z, box): a load that reaches beyond a box on any face
    // is filled, with zeros (u, p, delta) or NaN (the g words: absent voxels)
    const cuuint64_t gdim[4] = {(cuuint64_t)sa->px, (cuuint64_t)sa->py, (cuuint64_t)sa->pz, (cuuint64_t)sa->bx.nbox};
    const cuuint64_t gstr[3] = {(cuuint64_t)sa->px * 4, (cuuint64_t)sa->px * (cuuint64_t)sa->py * 4,
                                (cuuint64_t)sa->px * (cuuint64_t)sa->py * (cuuint64_t)sa->pz * 4};
    const cuuint32_t box_t[4] = {(cuuint32_t)(tx + 2 * v), (cuuint32_t)(ty + 3), 1u, 1u};
    // delta: the tile's interior (its first column starts 16-byte aligned)
    const cuuint32_t box_x[4] = {(cuuint32_t)(v == 4 ? tx : tx + 2 * v), (cuuint32_t)ty, 1u, 1u};
    const cuuint32_t es[4] = {1u, 1u, 1u, 1u};
    auto enc = [&](CUtensorMap* m, const void* ptr, const cuuint32_t* box, bool nan_fill = false) {
        return encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(ptr), gdim, gstr, box, es,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      nan_fill ? CU_TENSOR_MAP_FLOAT_OOB_FILL_NAN_REQUEST_ZERO_FMA : CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) ==
               CUDA_SUCCESS;
    };
    if (!enc(&sa->tm.u, sa->u_in, box_t) || !enc(&sa->tm.p, sa->p_in, box_t) || !enc(&sa->tm.g, sa->gc, box_t, true) ||
        !enc(&sa->tm.x, sa->x, box_x) ||
        (loop && (!enc(&sa->tm.ua, sa->u_out, box_t) || !enc(&sa->tm.pa, sa->p_out, box_t))))
        return fail(RW_ERR_CUDA, "TMA descriptor encoding failed (tile %d, box %d x %d x %d)", tile, sa->px, sa->py,
                    sa->pz);
    return RW_OK;
}

// Configuration of a sweep over `nact` compacted systems: the z-splitting is
// deepened so that the systems still iterating fill the GPU again.
void compact_cfg(const SweepCfg& full, int fp64, int gtype, int nz, int nact, int sms, size_t part_elems,
                 SweepCfg* c, int occ_override = 0) {
    *c = full;
    const int occ = occ_override > 0 ? occ_override : std::max(1, sweep_occupancy(fp64, gtype, full.tile));
    const int64_t slots = (int64_t)occ * sms;
    const int64_t per_plane = (int64_t)nact * full.ntx * full.nty;
    // the partials buffer holds (part_elems / 6) items
    const int zc = model_zc(per_plane, nz, slots, std::max<int64_t>((int64_t)(part_elems / 6), per_plane));
    c->zc = zc;
    c->nzc = (nz + zc - 1) / zc;
    c->grid = (int)std::max<int64_t>(1, std::min<int64_t>(per_plane * c->nzc, slots));
    c->ipg = std::min(32, full.ipg * 2);
}

// Replay graph chunks of cfg.ipg sweeps until no system is active.  Whenever
// the number of active systems has halved, the active ones are compacted into
// a list (ascending) and the following sweeps visit only them, with a deeper
// z-splitting: the slow systems of a batch then no longer run at the width
// the whole batch was tiled for.  Once the work of one sweep fits a single
// wave of resident CTAs of a tile with a looped variant, the sweeps run
// looped instead: one cooperative launch iterates until the active count has
// halved (grid barriers in place of kernel boundaries), then the host
// compacts again.  n_active_dev holds {active count, error flag, 5 words of
// grid-barrier state}.
constexpr int kLoopIters = 512;

// Host-side fault injection for tests of the failure path: RW_FAULT=grid_barrier
// makes the looped sweep's grid barrier expect one arrival more than the grid
// has, so every CTA's bounded wait runs out, the kernel flags it and returns,
// and the call reports RW_ERR_TIMEOUT.  Read at every looped launch.
bool fault_grid_barrier() {
    const char* f = getenv("RW_FAULT");
    return f && strcmp(f, "grid_barrier") == 0;
}

// Resident clusters of the cluster-resident solver for boxes of these dims
// (0: not available), cached per dims.  RW_CLUSTER=0 in the environment turns
// the cluster-resident mode off (the batched sweeps then finish every solve).
int cluster_capacity(const Boxes& bx) {
    const char* f = getenv("RW_CLUSTER");
    if (f && strcmp(f, "0") == 0) return 0;
    if (bx.nx > kClusterMaxDim || bx.ny > kClusterMaxDim || bx.nz > kClusterMaxDim || bx.nz < kClusterSize) return 0;
    static std::map<std::array<int, 3>, int> cache;
    const std::array<int, 3> key = {bx.nx, bx.ny, bx.nz};
    auto it = cache.find(key);
    if (it != cache.end()) return it->second;
    const int n = cluster_max_active(bx.nx, bx.ny, bx.nz, kClusterSize);
    cache[key] = n;
    return n;
}

rw_status run_graph_chunks(DevWorkspace* w, const SweepCfg& cfg0, SweepArgs sa, void* const u[2], void* const p[2],
                           int fp64, int gtype, int* n_active_dev, int n_act0, int* list_dev, size_t part_elems,
                           int64_t* sweeps, int64_t cap, double* ms_dev) {
    SweepCfg cfg = cfg0;
    sa.list = nullptr;
    sa.nlist = nullptr;
    int n_cur = sa.bx.nbox;
    cudaGraphExec_t exec = nullptr;
    const int occ_loop = fp64 ? 0 : sweep5_occupancy_loop(cfg0.tile);
    bool loop = false;
    int lpar = 0;  // buffer parity of the next looped launch
    // cluster-resident mode (FP32 sweeps in the strip kernels' layout,
    // small boxes): once the active systems are at most kClusterTurns per
    // resident cluster, the remaining iterations run there; each system keeps
    // its buffer parity
    const int cl_max = (!fp64 && cfg0.tile >= TILE_STRIP_FIRST && tile_margin(cfg0.tile) == 4)
                           ? cluster_capacity(sa.bx) : 0;
    bool clmode = false;
    auto try_cluster = [&](int n) -> bool {
        if (cl_max <= 0 || n > kClusterTurns * cl_max) return false;
        clmode = true;
        return true;
    };
    auto use_cfg = [&](const SweepCfg& c) {
        cfg = c;
        sa.ntx = cfg.ntx;
        sa.nty = cfg.nty;
        sa.nzc = cfg.nzc;
        sa.zc = cfg.zc;
    };
    // switch to (or stay in) looped sweeps when n systems fit one wave
    auto try_loop = [&](int n) -> bool {
        if (occ_loop <= 0) return false;
        SweepCfg c2;
        compact_cfg(cfg0, fp64, gtype, sa.bx.nz, n, w->sms, part_elems, &c2, occ_loop);
        if ((int64_t)n * c2.ntx * c2.nty * c2.nzc > (int64_t)occ_loop * w->sms) return false;
        use_cfg(c2);
        loop = true;
        return true;
    };
    auto capture = [&]() -> rw_status {
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(w->stream, cudaStreamCaptureModeThreadLocal));
        int par = 0;
        cudaError_t le = cudaSuccess;
        for (int j = 0; j < cfg.ipg; ++j) {
            sa.u_in = u[par];
            sa.p_in = p[par];
            sa.u_out = u[par ^ 1];
            sa.p_out = p[par ^ 1];
            sa.parity = par;
            rw_status ms = fp64 ? RW_OK : strip_maps(cfg.tile, &sa);
            cudaError_t e = ms == RW_OK ? launch_sweep(fp64, gtype, cfg.tile, sa, cfg.grid, w->stream)
                                        : cudaErrorInvalidValue;
            if (e != cudaSuccess && le == cudaSuccess) le = e;
            par ^= 1;
        }
        cudaError_t ce = cudaStreamEndCapture(w->stream, &graph);
        if (le != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            CK(le);
        }
        CK(ce);
        cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        CK(ie);
        return RW_OK;
    };
    auto compact = [&](int n_act) -> rw_status {
        if (!list_dev || sa.bx.nbox < 2 || n_act <= 0 || 2 * n_act > n_cur) return RW_OK;
        CK(counted(launch_compact_active(sa.sc, sa.bx.nbox, list_dev, list_dev + sa.bx.nbox, w->stream)));
        sa.list = list_dev;
        sa.nlist = list_dev + sa.bx.nbox;
        n_cur = n_act;
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        if (clmode || try_cluster(n_act)) return RW_OK;
        if (try_loop(n_act)) return RW_OK;
        SweepCfg c2;
        compact_cfg(cfg0, fp64, gtype, sa.bx.nz, n_act, w->sms, part_elems, &c2);
        use_cfg(c2);
        return capture();
    };
    rw_status st = compact(n_act0);
    if (st == RW_OK && !exec && !loop && !clmode && !try_cluster(n_act0) && !try_loop(n_cur)) st = capture();
    if (st != RW_OK) {
        if (exec) cudaGraphExecDestroy(exec);
        return st;
    }
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    CK(cudaEventCreate(&ev0));
    CK(cudaEventCreate(&ev1));
    int n_act = std::max(1, n_act0);
    while (n_act > 0 && *sweeps < cap) {
        int64_t done = cfg.ipg;
        cudaError_t e = cudaSuccess;
        if (clmode) {
            ClusterArgs ca;
            ca.u[0] = static_cast<float*>(u[0]);
            ca.u[1] = static_cast<float*>(u[1]);
            ca.p[0] = static_cast<float*>(p[0]);
            ca.p[1] = static_cast<float*>(p[1]);
            ca.x = static_cast<float*>(sa.x);
            ca.gc = sa.gc;
            ca.px = sa.px;
            ca.py = sa.py;
            ca.pz = sa.pz;
            ca.nx = sa.bx.nx;
            ca.ny = sa.bx.ny;
            ca.nz = sa.bx.nz;
            ca.rs = cluster_row_stride(sa.bx.nx);
            ca.rows = cluster_rows(sa.bx.ny, sa.bx.nz, kClusterSize);
            ca.sc = sa.sc;
            ca.list = sa.list;
            ca.nlist = sa.nlist;
            ca.nbox = sa.bx.nbox;
            ca.n_active = n_active_dev;
            ca.done = n_active_dev + 6;  // the "iterations done" word read back below
            ca.loop_iters = (int)std::min<int64_t>(kLoopIters, cap - *sweeps);
            ca.c2f = sa.c2f;
            ca.wminf = sa.wminf;
            const int ncl = std::max(1, std::min(cl_max, n_act > 0 ? n_act : n_cur));
            e = cudaMemsetAsync(ca.done, 0, sizeof(int), w->stream);
            if (e == cudaSuccess) e = cudaEventRecord(ev0, w->stream);
            if (e == cudaSuccess) e = launch_brick_cluster(ca, ncl, kClusterSize, w->stream);
        } else if (loop) {
            sa.u_in = u[lpar];
            sa.p_in = p[lpar];
            sa.u_out = u[lpar ^ 1];
            sa.p_out = p[lpar ^ 1];
            sa.parity = lpar;
            sa.loop_iters = (int)std::min<int64_t>(kLoopIters, cap - *sweeps);
            sa.loop_stop = list_dev && sa.bx.nbox >= 2 ? n_cur / 2 : 0;  // stop where compaction pays
            sa.gsync = reinterpret_cast<unsigned*>(n_active_dev + 2);
            sa.barrier_extra = fault_grid_barrier() ? 1 : 0;
            st = strip_maps(cfg.tile, &sa, true);
            if (st != RW_OK) break;
            e = cudaMemsetAsync(sa.gsync, 0, 5 * sizeof(unsigned), w->stream);
            if (e == cudaSuccess) e = cudaEventRecord(ev0, w->stream);
            if (e == cudaSuccess) e = sweep5_launch_loop(cfg.tile, sa, cfg.grid, w->stream);
        } else {
            e = cudaEventRecord(ev0, w->stream);
            if (e == cudaSuccess) e = cudaGraphLaunch(exec, w->stream);
        }
        if (e == cudaSuccess) e = cudaEventRecord(ev1, w->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(w->pinned, n_active_dev, 7 * sizeof(int), cudaMemcpyDeviceToHost, w->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
        float ms = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
        if (e != cudaSuccess) {
            cudaGetLastError();
            st = fail(RW_ERR_CUDA, "PCG chunk failed: %s", cudaGetErrorString(e));
            break;
        }
        *ms_dev += ms;
        if (clmode) {
            done = w->pinned[6];  // most iterations any system ran in the launch
            g_launches += 1;
        } else if (loop) {
            done = w->pinned[6];  // iterations the looped launch completed
            lpar = (int)((lpar + done) & 1);
            g_launches += 1;
        } else {
            g_launches += cfg.ipg;
        }
        *sweeps += done;
        n_act = w->pinned[0];
        if (w->pinned[1]) {
            st = fail(RW_ERR_TIMEOUT, "PCG sweep: a load or grid-barrier wait ran out (tile %d)", cfg.tile);
            break;
        }
        if (done <= 0) {
            st = fail(RW_ERR_CUDA, "PCG sweep: a looped launch completed no iteration (tile %d)", cfg.tile);
            break;
        }
        if (n_act > 0 && *sweeps < cap) {
            st = compact(n_act);
            if (st != RW_OK) break;
        }
    }
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (exec) cudaGraphExecDestroy(exec);
    return st;
}

// Time `reps` sweeps of one tile on the live state (they are real PCG
// iterations; an even count keeps the buffer parity).
rw_status time_tile(DevWorkspace* w, const SweepCfg& cfg, SweepArgs sa, void* const u[2], void* const p[2], int fp64,
                    int gtype, int reps, float* ms) {
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventRecord(e0, w->stream));
    int par = 0;
    for (int j = 0; j < reps; ++j) {
        sa.u_in = u[par];
        sa.p_in = p[par];
        sa.u_out = u[par ^ 1];
        sa.p_out = p[par ^ 1];
        sa.parity = par;
        if (!fp64) RCK(strip_maps(cfg.tile, &sa));
        CK(counted(launch_sweep(fp64, gtype, cfg.tile, sa, cfg.grid, w->stream)));
        par ^= 1;
    }
    CK(cudaEventRecord(e1, w->stream));
    CK(cudaEventSynchronize(e1));
    CK(cudaEventElapsedTime(ms, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return RW_OK;
}

// Per-precision sweep set-up: buffers of the vector type, a configuration
// (autotuned once per problem class), partial-sum storage.
struct PrecState {
    int fp64 = 0;
    Pad pad = {};          // layout of u, p, delta, g|code for this precision
    int64_t nvec = 0;      // elements of each streamed vector
    void* u[2] = {nullptr, nullptr};
    void* p[2] = {nullptr, nullptr};
    SweepCfg cfg;
    size_t part_elems = 0;  // doubles in the per-CTA partials buffer
    std::vector<int> cands;
    std::string key;
    bool tune = false;
};

rw_status prec_setup(DevWorkspace* w, const SolveProblem& P, const rw_opts& o, int fp64, PrecState* ps,
                     double** part) {
    const Boxes& bx = P.bx;
    const int64_t ntot = (int64_t)bx.nx * bx.ny * bx.nz * bx.nbox;
    const size_t tsz = fp64 ? 8 : 4;
    ps->fp64 = fp64;
    ps->key = class_key(fp64, P.gtype, bx);
    ps->cands = tile_candidates(fp64, P.gtype, bx.nx);
    if (ps->cands.empty()) return fail(RW_ERR_INVALID_ARG, "no sweep kernel for this precision/storage");
    if (o.tile != RW_TILE_AUTO && sweep_occupancy(fp64, P.gtype, o.tile) > 0)
        ps->cands = {o.tile};  // an explicit tile: its own layout, no tuning
    ps->pad = {};
    ps->nvec = ntot;
    if (!fp64 && ps->cands[0] >= TILE_STRIP_FIRST) {
        // the strip kernel's layout: no margins, rows of a multiple of 4 voxels
        ps->pad.px = (bx.nx + 3) & ~3;
        ps->pad.py = bx.ny;
        ps->pad.pz = bx.nz;
        ps->nvec = (int64_t)ps->pad.px * ps->pad.py * ps->pad.pz * bx.nbox;
    }
    RCK(ws_get(w, S_U0, ps->nvec * tsz, &ps->u[0]));
    RCK(ws_get(w, S_U1, ps->nvec * tsz, &ps->u[1]));
    RCK(ws_get(w, S_P0, ps->nvec * tsz, &ps->p[0]));
    RCK(ws_get(w, S_P1, ps->nvec * tsz, &ps->p[1]));
    if (ps->pad.px) {
        // the columns beyond nx must read as absent voxels with zero vectors
        for (int k = 0; k < 2; ++k) {
            CK(cudaMemsetAsync(ps->u[k], 0, ps->nvec * tsz, w->stream));
            CK(cudaMemsetAsync(ps->p[k], 0, ps->nvec * tsz, w->stream));
        }
    }
    int tile = ps->cands[0];
    int ipg = std::max(2, o.iters_per_graph & ~1);
    int waves = 0;
    ps->tune = false;
    if (o.tile != RW_TILE_AUTO && sweep_occupancy(fp64, P.gtype, o.tile) > 0 &&
        std::find(ps->cands.begin(), ps->cands.end(), o.tile) != ps->cands.end()) {
        tile = o.tile;
    } else if (o.tile == RW_TILE_AUTO) {
        auto it = g_tuned.find(ps->key);
        if (it != g_tuned.end()) {
            tile = it->second.tile;
            ipg = it->second.ipg;
            waves = it->second.waves;
        } else {
            ps->tune = true;
        }
    }
    RCK(make_cfg(fp64, P.gtype, tile, bx, w->sms, ipg, &ps->cfg, waves));
    size_t part_elems = (size_t)bx.nbox * ps->cfg.ntx * ps->cfg.nty * ps->cfg.nzc * 6;
    for (int t : ps->cands)
        for (int wv = 0; wv <= 4; ++wv) {
            SweepCfg c2;
            RCK(make_cfg(fp64, P.gtype, t, bx, w->sms, ipg, &c2, wv));
            part_elems = std::max(part_elems, (size_t)bx.nbox * c2.ntx * c2.nty * c2.nzc * 6);
        }
    RCK(ws_get_t(w, S_PART, part_elems * sizeof(double), part));
    ps->part_elems = part_elems;
    return RW_OK;
}

// Autotuner: on the first round of a new problem class, time 4 sweeps of
// every candidate tile and z-chunking on the live state (real PCG iterations;
// an even count keeps the buffer parity), keep the fastest and size the graph
// chunk to about 4 ms of sweeps.
rw_status autotune(DevWorkspace* w, const SolveProblem& P, PrecState* ps, const SweepArgs& sa, SolveResult* R) {
    float best = 1e30f;
    int best_tile = ps->cfg.tile, best_waves = 0;
    // each distinct (tile, z-chunking) pair runs 4 real sweeps
    for (int t : ps->cands) {
        int seen_nzc[5] = {-1, -1, -1, -1, -1};
        for (int wv = 0; wv <= 4; ++wv) {
            SweepCfg c2;
            RCK(make_cfg(ps->fp64, P.gtype, t, P.bx, w->sms, ps->cfg.ipg, &c2, wv));
            bool dup = false;
            for (int k = 0; k < wv; ++k) dup = dup || seen_nzc[k] == c2.nzc;
            seen_nzc[wv] = c2.nzc;
            if (dup) continue;
            SweepArgs s2 = sa;
            s2.ntx = c2.ntx;
            s2.nty = c2.nty;
            s2.nzc = c2.nzc;
            s2.zc = c2.zc;
            float ms = 0;
            RCK(time_tile(w, c2, s2, ps->u, ps->p, ps->fp64, P.gtype, 4, &ms));
            R->sweeps += 4;
            if (ms < best) {
                best = ms;
                best_tile = t;
                best_waves = wv;
            }
        }
    }
    // graph chunks of ~4 ms: one host round trip per chunk; sweeps past a
    // system's convergence exit at once
    const float per = best / 4.0f;
    int k = (int)std::lround(4.0 / std::max(per, 1e-4f));
    k = std::max(8, std::min(32, k)) & ~1;
    RCK(make_cfg(ps->fp64, P.gtype, best_tile, P.bx, w->sms, k, &ps->cfg, best_waves));
    g_tuned[ps->key] = Tuned{best_tile, k, best_waves};
    ps->tune = false;
    return RW_OK;
}

// Solve every box of P.  Mixed precision: FP32 PCG rounds on the correction,
// each ended by an FP64 residual of x_hi.  A system whose round does not cut
// its true residual by 10x is beyond what FP32 sweeps can resolve (its
// condition number approaches 1/eps_fp32); the remaining work then runs with
// FP64 sweeps on x_hi (one extra round, to tol).
rw_status solve_boxes(DevWorkspace* w, const SolveProblem& P, const rw_opts& o, SolveResult* R) {
    const Boxes& bx = P.bx;
    const int64_t nvox = (int64_t)bx.nx * bx.ny * bx.nz;
    int cur64 = o.precision == RW_FP64 ? 1 : 0;
    float* delta = nullptr;
    BoxScalars* sc = nullptr;
    int* nact = nullptr;
    double *rpart = nullptr, *part = nullptr;
    RCK(ws_get_t(w, S_SC, bx.nbox * sizeof(BoxScalars), &sc));
    RCK(ws_get_t(w, S_NACT, 64, &nact));
    int* list = nullptr;
    RCK(ws_get_t(w, S_LIST, (bx.nbox + 1) * sizeof(int), &list));
    const int bpb = (int)((nvox + 1023) / 1024);  // k_residual: up to 4 voxels per thread
    RCK(ws_get_t(w, S_RPART, (size_t)bx.nbox * bpb * 4 * sizeof(double), &rpart));
    PrecState ps;
    RCK(prec_setup(w, P, o, cur64, &ps, &part));
    if (!cur64) {
        RCK(ws_get_t(w, S_DELTA, ps.nvec * 4, &delta));
        if (ps.pad.px) CK(cudaMemsetAsync(delta, 0, ps.nvec * 4, w->stream));
    }

    ResidArgs ra;
    ra.bx = bx;
    ra.g = P.g;
    ra.gtype = P.gtype;
    ra.code = P.code;
    ra.value = P.value;
    ra.x0 = P.x0;
    ra.rhs = P.rhs;
    ra.x = P.x_hi;
    ra.u = ps.u[0];
    ra.p = ps.p[0];
    ra.p_other = ps.p[1];
    ra.sc = sc;
    ra.keep_p = 0;
    ra.pad = ps.pad;
    ra.part = rpart;
    ra.blocks_per_box = bpb;
    // Poisson weights: the Gaussian form on sqrt(g) with beta / 2
    const bool poisson = o.weight == RW_WEIGHT_POISSON;
    const double beta_w = poisson ? 0.5 * (double)o.beta : (double)o.beta;
    ra.sqrt_g = poisson ? 1 : 0;
    ra.mbeta = -beta_w;
    ra.wmin = (double)o.w_min;

    // FP64 edge weights once per solve (the residual rounds read them) while
    // they fit a fixed budget; beyond it the residual evaluates them in place
    constexpr size_t kW64Budget = (size_t)16 << 30;
    const size_t w64_bytes = (size_t)nvox * bx.nbox * 3 * sizeof(double);
    if (w64_bytes <= kW64Budget) {
        double* w3 = nullptr;
        RCK(ws_get_t(w, S_W64, w64_bytes, &w3));
        CK(counted(launch_weights64(ra, w3, w->stream)));
        ra.w3 = w3;
    }

    uint32_t* gc = nullptr;
    if (!cur64) {
        RCK(ws_get_t(w, S_GC, ps.nvec * 4, &gc));
        // the strip kernel's format marks absent voxels (the columns beyond nx included) NaN
        const int fmt = ps.cands[0] >= TILE_STRIP_FIRST ? 1 : 0;
        if (fmt) CK(counted(launch_fill_u32(gc, ps.nvec, GC_ABSENT, w->stream)));
        else if (ps.pad.px) CK(cudaMemsetAsync(gc, 0, ps.nvec * 4, w->stream));
        CK(counted(launch_pack_gc(bx, ps.pad, P.g, P.gtype, P.code, gc, w->stream, fmt, ra.sqrt_g)));
    }
    CK(cudaMemsetAsync(sc, 0, bx.nbox * sizeof(BoxScalars), w->stream));
    if (P.init_x) CK(counted(launch_init_x(cur64, ra, w->stream)));
    CK(counted(launch_residual(cur64, ra, delta, w->stream)));
    CK(counted(launch_box_reduce(rpart, bpb, bx.nbox, sc, 1, w->stream)));
    CK(counted(launch_zero_homog(cur64, bx, P.code, sc, P.x_hi, w->stream)));

    SweepArgs sa{};
    sa.bx = bx;
    sa.g = P.g;
    sa.code = P.code;
    sa.gc = gc;
    sa.x = cur64 ? (void*)P.x_hi : (void*)delta;
    sa.sc = sc;
    sa.partials = part;
    sa.n_active = nact;
    sa.err = nact + 1;  // the strip sweep's load-wait flag, next to the active count
    CK(cudaMemsetAsync(nact + 1, 0, sizeof(int), w->stream));
    sa.c2f = (float)(-beta_w * 1.4426950408889634);
    sa.sqrt_g = ra.sqrt_g;
    sa.wminf = o.w_min;
    sa.mbeta = -beta_w;
    sa.wmin = (double)o.w_min;
    sa.px = ps.pad.px;
    sa.py = ps.pad.py;
    sa.pz = ps.pad.pz;

    const int mixed_rounds = std::max(1, o.refine_rounds);
    int max_rounds = cur64 ? 1 : mixed_rounds;
    std::vector<BoxScalars> h(bx.nbox);
    std::vector<double> prev(bx.nbox, -1.0);
    const double t0 = now_ms();
    int restart = 1;
    int fp64_restarts = 0;
    for (int r = 0; r < max_rounds; ++r) {
        const double eps_inner = cur64 ? 0.0 : 1e-5;
        CK(cudaMemsetAsync(nact, 0, sizeof(int), w->stream));
        CK(counted(launch_start_round(sc, bx.nbox, r, o.tol, eps_inner, o.max_iter, restart, nact, w->stream)));
        restart = 0;
        CK(cudaMemcpyAsync(h.data(), sc, bx.nbox * sizeof(BoxScalars), cudaMemcpyDeviceToHost, w->stream));
        CK(cudaMemcpyAsync(w->pinned, nact, sizeof(int), cudaMemcpyDeviceToHost, w->stream));
        CK(cudaStreamSynchronize(w->stream));
        if (*w->pinned == 0) break;
        for (int b = 0; b < bx.nbox; ++b) prev[b] = h[b].rr_true;
        R->rounds = r + 1;
        sa.partials = part;
        if (ps.tune) RCK(autotune(w, P, &ps, sa, R));
        sa.ntx = ps.cfg.ntx;
        sa.nty = ps.cfg.nty;
        sa.nzc = ps.cfg.nzc;
        sa.zc = ps.cfg.zc;
        const int64_t cap = R->sweeps + (int64_t)o.max_iter + 4 * ps.cfg.ipg;
        RCK(run_graph_chunks(w, ps.cfg, sa, ps.u, ps.p, cur64, P.gtype, nact, *w->pinned, list, ps.part_elems,
                             &R->sweeps, cap, &R->ms_sweeps));
        // residual replacement: x_hi absorbs the FP32 correction, the FP64
        // residual replaces the recursive one and the search direction is kept
        // (only the systems that iterated in this round: the others' x did not change)
        if (!cur64) CK(counted(launch_accumulate(bx, ps.pad, P.code, delta, P.x_hi, w->stream)));
        ra.keep_p = 1;
        ra.only_moved = 1;
        CK(counted(launch_residual(cur64, ra, delta, w->stream)));
        CK(counted(launch_box_reduce(rpart, bpb, bx.nbox, sc, 0, w->stream, 1)));
        ra.only_moved = 0;
        CK(cudaMemcpyAsync(h.data(), sc, bx.nbox * sizeof(BoxScalars), cudaMemcpyDeviceToHost, w->stream));
        CK(cudaStreamSynchronize(w->stream));
        // FP32 sweeps failed a system when its round ended in a breakdown or
        // cut its true residual by less than 100x: finish with FP64 sweeps.
        // An FP64 round that ended in a breakdown gets one restart.
        bool stagnated = false, broke = false;
        for (int b = 0; b < bx.nbox; ++b) {
            const BoxScalars& S = h[b];
            if (S.nseed == 0 || S.nfree == 0 || !(S.bb > 0.0)) continue;
            if (!(S.rr_true > o.tol * o.tol * S.bb)) continue;
            if (S.status == 5) broke = true;
            if (S.status == 5 || (prev[b] > 0.0 && S.rr_true > 1e-2 * prev[b])) stagnated = true;
        }
        if (!cur64 && stagnated) {
            cur64 = 1;
            RCK(prec_setup(w, P, o, 1, &ps, &part));
            ra.u = ps.u[0];
            ra.p = ps.p[0];
            ra.p_other = ps.p[1];
            ra.keep_p = 0;
            ra.pad = ps.pad;
            sa.px = sa.py = sa.pz = 0;
            sa.x = P.x_hi;
            restart = 1;
            CK(counted(launch_residual(1, ra, nullptr, w->stream)));
            CK(counted(launch_box_reduce(rpart, bpb, bx.nbox, sc, 0, w->stream)));
            max_rounds = r + 3;
            R->fp64_fallback = 1;
        } else if (cur64 && broke && fp64_restarts < 2) {
            ++fp64_restarts;
            restart = 1;
            max_rounds = std::max(max_rounds, r + 2);
        }
    }
    R->sc.resize(bx.nbox);
    CK(cudaMemcpyAsync(R->sc.data(), sc, bx.nbox * sizeof(BoxScalars), cudaMemcpyDeviceToHost, w->stream));
    CK(cudaStreamSynchronize(w->stream));
    R->ms_solve = now_ms() - t0;
    R->tile = ps.cfg.tile;
    R->ipg = ps.cfg.ipg;
    return RW_OK;
}

void stats_from(const SolveResult& R, const rw_opts& o, rw_stats* st, int* n_unconverged, int* n_noseed) {
    int it = 0;
    double rel = 0.0;
    int64_t vi = 0, nf = 0;
    int bad = 0, nos = 0;
    for (const BoxScalars& S : R.sc) {
        it = std::max(it, S.iters);
        vi += (int64_t)S.iters * S.nfree;
        nf += S.nfree;
        if (S.nseed == 0) {
            ++nos;
            continue;
        }
        if (S.bb > 0.0) {
            const double r = std::sqrt(S.rr_true / S.bb);
            rel = std::max(rel, r);
            if (r > o.tol) ++bad;
        }
    }
    if (st) {
        st->iters = std::max(st->iters, it);
        st->refine_rounds = std::max(st->refine_rounds, R.rounds);
        st->rel_resid = std::max(st->rel_resid, rel);
        st->voxel_iters += vi;
        st->free_voxels += nf;
        st->sweeps += R.sweeps;
        st->ms_solve += R.ms_solve;
        st->ms_sweeps += R.ms_sweeps;
        st->tile = R.tile;
        st->iters_per_graph = R.ipg;
        st->not_converged += bad;
        st->fp64_fallbacks += R.fp64_fallback;
    }
    if (n_unconverged) *n_unconverged = bad;
    if (n_noseed) *n_noseed = nos;
}

}  // namespace rwh

using namespace rwh;

// Error text for the other translation units of the library.
void rw_internal_set_error(const char* msg) { g_err = msg; }

// ===========================================================================
extern "C" {

void rw_opts_default(rw_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->beta = 130.0f;
    o->w_min = 1e-30f;
    o->tol = 1e-8;
    o->max_iter = 20000;
    o->precision = RW_MIXED;
    o->refine_rounds = 4;
    o->brick_size = 32;
    o->expand = 1.25f;
    o->t_hom = 0.3f;
    o->t_bin = 0.01f;
    o->t_inc = 0.01f;
    o->prune_hom = 1;
    o->prune_dt = 1;
    o->iters_per_graph = 32;
    o->tile = RW_TILE_AUTO;
    o->batch_bricks = 1;
    o->max_batch = 8192;
    o->leaf_field = RW_LEAF_AS_PYRAMID;
}

const char* rw_last_error(void) { return g_err.c_str(); }

const char* rw_version(void) { return "rw-gb300 0.1 (sm_103a)"; }

rw_status rw_release_workspace(void) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    for (auto& kv : g_ws) {
        DevWorkspace& w = kv.second;
        if (w.stream) cudaStreamSynchronize(w.stream);
        for (int s = 0; s < S_COUNT; ++s)
            if (w.p[s]) cudaFree(w.p[s]);
        if (w.pinned) cudaFreeHost(w.pinned);
        if (w.stream) cudaStreamDestroy(w.stream);
        w = DevWorkspace();
    }
    g_ws.clear();
    return RW_OK;
}

rw_status rw_solve(const rw_volume* vol, const rw_seed_mask* seeds, const rw_opts* opts_in, const float* x0,
                   float* x_out, rw_stats* stats, void* stream) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    g_launches = 0;
    const double t_start = now_ms();
    rw_opts o;
    if (opts_in) o = *opts_in;
    else rw_opts_default(&o);
    RCK(check_opts(o));
    int64_t nvox = 0, batch = 1;
    RCK(check_volume(vol, &nvox, &batch));
    if (!seeds || !seeds->code) return fail(RW_ERR_INVALID_ARG, "seed mask code is NULL");
    if (!x_out) return fail(RW_ERR_INVALID_ARG, "x_out is NULL");
    if (stats) memset(stats, 0, sizeof(*stats));
    DevWorkspace* w = nullptr;
    RCK(enter(&w, stream));
    const int64_t ntot = nvox * batch;
    const size_t vbytes = ntot * (vol->dtype == RW_U16 ? 2 : 4);
    const void *dvol, *dcode, *dval, *dx0;
    RCK(stage_in(w, S_VOL, vol->data, vbytes, &dvol));
    RCK(stage_in(w, S_CODE, seeds->code, ntot, &dcode));
    RCK(stage_in(w, S_VAL, seeds->value, ntot * 4, &dval));
    RCK(stage_in(w, S_X0, x0, ntot * 4, &dx0));
    const int gtype = vol->storage == RW_STORE_F32 ? G_F32 : G_U16;
    void* g = nullptr;
    RCK(ws_get(w, S_G, ntot * (gtype == G_U16 ? 2 : 4), &g));
    CK(counted(launch_quantize(dvol, vol->dtype, ntot, vol->lo, vol->hi, vol->normalize, vol->storage, g, w->stream)));
    double* xhi = nullptr;
    RCK(ws_get_t(w, S_XHI, ntot * 8, &xhi));

    SolveProblem P;
    P.bx.nbox = (int)batch;
    P.bx.nx = (int)vol->dims[0];
    P.bx.ny = (int)vol->dims[1];
    P.bx.nz = (int)vol->dims[2];
    P.bx.ext = nullptr;
    P.g = g;
    P.gtype = gtype;
    P.code = static_cast<const uint8_t*>(dcode);
    P.value = static_cast<const float*>(dval);
    P.x0 = static_cast<const float*>(dx0);
    P.rhs = nullptr;
    P.x_hi = xhi;
    P.init_x = 1;
    SolveResult R;
    RCK(solve_boxes(w, P, o, &R));
    const bool out_dev = is_device_ptr(x_out);
    float* dout = x_out;
    if (!out_dev) RCK(ws_get_t(w, S_OUT, ntot * 4, &dout));
    CK(counted(launch_copy_out(0, P.bx, xhi, dout, w->stream)));
    if (!out_dev) CK(cudaMemcpyAsync(x_out, dout, ntot * 4, cudaMemcpyDeviceToHost, w->stream));
    RCK(leave(w));
    int bad = 0, nos = 0;
    stats_from(R, o, stats, &bad, &nos);
    if (stats) {
        stats->ms = now_ms() - t_start;
        stats->launches = g_launches;
    }
    if (nos > 0) return fail(RW_ERR_NO_SEEDS, "%d volume(s) without any seed", nos);
    if (bad > 0) return fail(RW_ERR_NOT_CONVERGED, "%d system(s) above tol after %d rounds", bad, R.rounds);
    return RW_OK;
}

rw_status rw_solve_adjoint(const rw_volume* vol, const rw_seed_mask* seeds, const rw_opts* opts_in, const float* x,
                           const float* dloss_dx, float* dloss_dg, double* dloss_dbeta, rw_stats* stats,
                           void* stream) {
    std::lock_guard<std::recursive_mutex> lk(g_mu);
    g_launches = 0;
    const double t_start = now_ms();
    rw_opts o;
    if (opts_in) o = *opts_in;
    else rw_opts_default(&o);
    RCK(check_opts(o));
    if (o.weight != RW_WEIGHT_GAUSSIAN) return fail(RW_ERR_UNIMPLEMENTED, "the adjoint supports Gaussian weights only");
    int64_t nvox = 0, batch = 1;
    RCK(check_volume(vol, &nvox, &batch));
    if (!seeds || !seeds->code || !x || !dloss_dx) return fail(RW_ERR_INVALID_ARG, "NULL argument");
    if (stats) memset(stats, 0, sizeof(*stats));
    DevWorkspace* w = nullptr;
    RCK(enter(&w, stream));
    const int64_t ntot = nvox * batch;
    const size_t vbytes = ntot * (vol->dtype == RW_U16 ? 2 : 4);
    const void *dvol, *dcode, *dx, *ddl;
    RCK(stage_in(w, S_VOL, vol->data, vbytes, &dvol));
    RCK(stage_in(w, S_CODE, seeds->code, ntot, &dcode));
    RCK(stage_in(w, S_XF, x, ntot * 4, &dx));
    RCK(stage_in(w, S_RHS, dloss_dx, ntot * 4, &ddl));
    const int gtype = vol->storage == RW_STORE_F32 ? G_F32 : G_U16;
    void* g = nullptr;
    RCK(ws_get(w, S_G, ntot * (gtype == G_U16 ? 2 : 4), &g));
    CK(counted(launch_quantize(dvol, vol->dtype, ntot, vol->lo, vol->hi, vol->normalize, vol->storage, g, w->stream)));
    double* lam = nullptr;
    RCK(ws_get_t(w, S_XHI, ntot * 8, &lam));
    SolveProblem P;
    P.bx.nbox = (int)batch;
    P.bx.nx = (int)vol->dims[0];
    P.bx.ny = (int)vol->dims[1];
    P.bx.nz = (int)vol->dims[2];
    P.bx.ext = nullptr;
    P.g = g;
    P.gtype = gtype;
    P.code = static_cast<const uint8_t*>(dcode);
    P.value = nullptr;  // lambda = 0 on seeds
    P.x0 = nullptr;
    P.rhs = static_cast<const float*>(ddl);
    P.x_hi = lam;
    P.init_x = 1;
    SolveResult R;
    RCK(solve_boxes(w, P, o, &R));

    const int bpb = (int)((nvox + 255) / 256);
    double *apart = nullptr, *dbeta = nullptr;
    RCK(ws_get_t(w, S_ADJ_PART, (size_t)batch * bpb * sizeof(double), &apart));
    RCK(ws_get_t(w, S_DBETA, (size_t)batch * sizeof(double), &dbeta));
    float* ddg = nullptr;
    const bool dg_dev = dloss_dg && is_device_ptr(dloss_dg);
    if (dloss_dg) {
        if (dg_dev) ddg = dloss_dg;
        else RCK(ws_get_t(w, S_DG, ntot * 4, &ddg));
    }
    AdjArgs aa;
    aa.bx = P.bx;
    aa.g = g;
    aa.gtype = gtype;
    aa.code = P.code;
    aa.x = static_cast<const float*>(dx);
    aa.lam = lam;
    aa.dg = ddg;
    aa.part = apart;
    aa.blocks_per_box = bpb;
    aa.beta = (double)o.beta;
    aa.wmin = (double)o.w_min;
    CK(counted(launch_adjoint(aa, w->stream)));
    CK(counted(launch_adjoint_reduce(apart, bpb, (int)batch, dbeta, w->stream)));
    if (dloss_dg && !dg_dev) CK(cudaMemcpyAsync(dloss_dg, ddg, ntot * 4, cudaMemcpyDeviceToHost, w->stream));
    if (dloss_dbeta) {
        CK(cudaMemcpyAsync(dloss_dbeta, dbeta, batch * sizeof(double),
                           is_device_ptr(dloss_dbeta) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, w->stream));
    }
    RCK(leave(w));
    int bad = 0, nos = 0;
    stats_from(R, o, stats, &bad, &nos);
    if (stats) {
        stats->ms = now_ms() - t_start;
        stats->launches = g_launches;
    }
    if (nos > 0) return fail(RW_ERR_NO_SEEDS, "%d volume(s) without any seed", nos);
    if (bad > 0) return fail(RW_ERR_NOT_CONVERGED, "%d adjoint system(s) above tol", bad);
    return RW_OK;
}

}  // extern "C"

