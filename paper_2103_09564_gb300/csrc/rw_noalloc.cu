// rw_solve_noalloc: the plain solve of rw_solve for callers that cannot
// allocate device memory.
//
// Who needs it: code that runs where cudaMalloc / cudaFree are not allowed or
// not wanted — an interactive labelling loop with a latency budget (both
// calls can synchronise the whole device), a plug-in inside a host
// application that owns the GPU memory budget, or a process that must not
// grow its footprint after start-up.  The scratch of the solve lives in one
// file-scope device array of fixed size that every GPU loading this library
// keeps until the process exits.
//
// Differences from rw_solve: device pointers only (no host staging), mixed
// precision only (no FP64 fallback), no internal stream, no CUDA graph and no
// timing events; work runs on the caller's stream, which is synchronised
// before returning.  Limits: RW_NOALLOC_MAX_VOXELS voxels in total over the
// batch, at most RW_NOALLOC_MAX_BATCH volumes.
//
// The first call on a device looks up the array's device address with
// cudaGetSymbolAddress (once per device, with that device current); make that
// first call before any stream capture.  Every call synchronises `stream`
// before it returns (it reads the active-system count on the host between
// sweeps).  Every call uses the same array and leaves its contents behind:
// the call clears what must start at zero, and calls that overlap on the GPU
// (other streams, other threads) race.  Every array must live on the current
// device (or be managed memory): the kernels run there.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "rw_api.h"
#include "rw_internal.h"

using namespace rwk;

void rw_internal_set_error(const char* msg);

namespace {

constexpr int64_t kMaxVoxels = RW_NOALLOC_MAX_VOXELS;
constexpr int64_t kMaxBatch = RW_NOALLOC_MAX_BATCH;
constexpr int64_t kMaxItems = 65536;  // sweep work items (tile x z-chunk) over the batch
constexpr int kTile = TILE_32x8;

// byte offsets of the scratch regions (256-byte aligned)
constexpr size_t al(size_t v) { return (v + 255) & ~(size_t)255; }
constexpr size_t kOffG = 0;                                         // uint16 g
constexpr size_t kOffGC = al(kOffG + kMaxVoxels * 2);               // uint32 g|code
constexpr size_t kOffX = al(kOffGC + kMaxVoxels * 4);               // double x_hi
constexpr size_t kOffD = al(kOffX + kMaxVoxels * 8);                // float delta
constexpr size_t kOffU0 = al(kOffD + kMaxVoxels * 4);               // float u (2 buffers)
constexpr size_t kOffU1 = al(kOffU0 + kMaxVoxels * 4);
constexpr size_t kOffP0 = al(kOffU1 + kMaxVoxels * 4);              // float p (2 buffers)
constexpr size_t kOffP1 = al(kOffP0 + kMaxVoxels * 4);
constexpr size_t kOffRP = al(kOffP1 + kMaxVoxels * 4);              // residual partials
constexpr size_t kRPart = (kMaxVoxels / 256 + kMaxBatch) * 4 * sizeof(double);
constexpr size_t kOffSP = al(kOffRP + kRPart);                      // sweep partials
constexpr size_t kOffSC = al(kOffSP + kMaxItems * 6 * sizeof(double));  // BoxScalars
constexpr size_t kOffNA = al(kOffSC + kMaxBatch * sizeof(BoxScalars));   // active count
constexpr size_t kScratchBytes = al(kOffNA + 256);
// the documented size ("about 12.1 MB") must stay true
static_assert(kScratchBytes > 12000000 && kScratchBytes < 12200000, "update the documented scratch size");

// The scratch array (about 12.1 MB).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_setup_mu;
void* g_scratch_ptr[128] = {};

rw_status fail(rw_status st, const char* msg) {
    rw_internal_set_error(msg);
    return st;
}

rw_status fail_cuda(cudaError_t e, const char* what) {
    char buf[512];
    snprintf(buf, sizeof(buf), "%s failed: %s", what, cudaGetErrorString(e));
    cudaGetLastError();
    rw_internal_set_error(buf);
    return RW_ERR_CUDA;
}

#define NCK(call)                                     \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return fail_cuda(e_, #call); \
    } while (0)

// Device memory of device `dev` (the current one, where the kernels run) or
// managed memory.
bool on_device(const void* p, int dev) {
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type == cudaMemoryTypeDevice) return at.device == dev;
    return at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" rw_status rw_solve_noalloc(const rw_volume* vol, const rw_seed_mask* seeds, const rw_opts* opts_in,
                                      const float* x0, float* x_out, rw_stats* stats, void* stream_v) {
    const auto t_start = std::chrono::steady_clock::now();
    if (stats) memset(stats, 0, sizeof(*stats));
    rw_opts o;
    if (opts_in) o = *opts_in;
    else rw_opts_default(&o);
    if (!vol || !vol->data || !seeds || !seeds->code || !x_out)
        return fail(RW_ERR_INVALID_ARG, "rw_solve_noalloc: NULL volume, seed code or output");
    if (o.precision != RW_MIXED) return fail(RW_ERR_INVALID_ARG, "rw_solve_noalloc: only RW_MIXED precision");
    if (o.weight != RW_WEIGHT_GAUSSIAN)
        return fail(RW_ERR_UNIMPLEMENTED, "rw_solve_noalloc: Gaussian weights only");
    if (!(o.tol >= 0.0) || o.max_iter < 1 || o.iters_per_graph < 2 || o.refine_rounds < 0)
        return fail(RW_ERR_INVALID_ARG, "rw_solve_noalloc: invalid rw_opts");
    if ((vol->dtype != RW_U16 && vol->dtype != RW_F32) || vol->storage != RW_STORE_UNORM16)
        return fail(RW_ERR_INVALID_ARG, "rw_solve_noalloc: needs dtype U16/F32 and unorm16 storage");
    const int64_t batch = vol->batch < 1 ? 1 : vol->batch;
    for (int a = 0; a < 3; ++a)
        if (vol->dims[a] < 1) return fail(RW_ERR_INVALID_ARG, "rw_solve_noalloc: bad dims");
    const int64_t nvox = vol->dims[0] * vol->dims[1] * vol->dims[2];
    const int64_t ntot = nvox * batch;
    if (ntot > kMaxVoxels || batch > kMaxBatch) {
        char buf[256];
        snprintf(buf, sizeof(buf),
                 "rw_solve_noalloc: %lld voxels in %lld volume(s) exceed the fixed scratch (at most %lld voxels, "
                 "%lld volumes); use rw_solve",
                 (long long)ntot, (long long)batch, (long long)kMaxVoxels, (long long)kMaxBatch);
        return fail(RW_ERR_INVALID_ARG, buf);
    }
    int dev = 0;
    NCK(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) return fail(RW_ERR_INVALID_ARG, "rw_solve_noalloc: device index out of range");
    if (!on_device(vol->data, dev) || !on_device(seeds->code, dev) || !on_device(x_out, dev) ||
        (seeds->value && !on_device(seeds->value, dev)) || (x0 && !on_device(x0, dev)))
        return fail(RW_ERR_INVALID_ARG,
                    "rw_solve_noalloc: every array must be device memory of the current device (or managed)");
    cudaStream_t s = static_cast<cudaStream_t>(stream_v);

    // set-up, once per device: the device address of the scratch array
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_setup_mu);
        if (!g_scratch_ptr[dev]) {
            void* ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess) return fail_cuda(e, "cudaGetSymbolAddress(scratch)");
            g_scratch_ptr[dev] = ptr;
        }
        base = static_cast<unsigned char*>(g_scratch_ptr[dev]);
    }
    uint16_t* g = reinterpret_cast<uint16_t*>(base + kOffG);
    uint32_t* gc = reinterpret_cast<uint32_t*>(base + kOffGC);
    double* xhi = reinterpret_cast<double*>(base + kOffX);
    float* delta = reinterpret_cast<float*>(base + kOffD);
    void* u[2] = {base + kOffU0, base + kOffU1};
    void* p[2] = {base + kOffP0, base + kOffP1};
    double* rpart = reinterpret_cast<double*>(base + kOffRP);
    double* part = reinterpret_cast<double*>(base + kOffSP);
    BoxScalars* sc = reinterpret_cast<BoxScalars*>(base + kOffSC);
    int* nact = reinterpret_cast<int*>(base + kOffNA);

    Boxes bx;
    bx.nbox = (int)batch;
    bx.nx = (int)vol->dims[0];
    bx.ny = (int)vol->dims[1];
    bx.nz = (int)vol->dims[2];
    bx.ext = nullptr;

    // sweep configuration: fixed 32x8 tile, z-chunks for parallelism
    int sms = 0;
    NCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int occ = std::max(1, sweep_occupancy(0, G_U16, kTile));
    NCK(sweep_prepare(0, G_U16, kTile));
    int tx = 32, ty = 8;
    tile_dims(kTile, &tx, &ty);
    const int ntx = (bx.nx + tx - 1) / tx, nty = (bx.ny + ty - 1) / ty;
    const int64_t per_plane = (int64_t)bx.nbox * ntx * nty;
    const int64_t want = (int64_t)2 * occ * sms;
    int nzc = (int)std::max<int64_t>(1, (want + per_plane - 1) / per_plane);
    int zc = std::max((bx.nz + nzc - 1) / nzc, std::min(bx.nz, 16));
    nzc = (bx.nz + zc - 1) / zc;
    const int64_t nwork = per_plane * nzc;
    if (nwork > kMaxItems) return fail(RW_ERR_INVALID_ARG, "rw_solve_noalloc: too many sweep tiles for the scratch");
    const int grid = (int)std::min<int64_t>(nwork, (int64_t)occ * sms);
    const int bpb = (int)((nvox + 255) / 256);
    int64_t launches = 0;

    // clear what must start at zero
    NCK(cudaMemsetAsync(sc, 0, batch * sizeof(BoxScalars), s));
    NCK(launch_quantize(vol->data, vol->dtype, ntot, vol->lo, vol->hi, vol->normalize, RW_STORE_UNORM16, g, s));
    NCK(launch_pack_gc(bx, Pad{}, g, G_U16, seeds->code, gc, s));
    ResidArgs ra{};
    ra.bx = bx;
    ra.g = g;
    ra.gtype = G_U16;
    ra.code = seeds->code;
    ra.value = seeds->value;
    ra.x0 = x0;
    ra.rhs = nullptr;
    ra.x = xhi;
    ra.u = u[0];
    ra.p = p[0];
    ra.p_other = p[1];
    ra.sc = sc;
    ra.keep_p = 0;
    ra.part = rpart;
    ra.blocks_per_box = bpb;
    ra.mbeta = -(double)o.beta;
    ra.wmin = (double)o.w_min;
    NCK(launch_init_x(0, ra, s));
    NCK(launch_residual(0, ra, delta, s));
    NCK(launch_box_reduce(rpart, bpb, bx.nbox, sc, 1, s));
    NCK(launch_zero_homog(0, bx, seeds->code, sc, xhi, s));
    launches += 6;

    SweepArgs sa{};
    sa.bx = bx;
    sa.ntx = ntx;
    sa.nty = nty;
    sa.nzc = nzc;
    sa.zc = zc;
    sa.gc = gc;
    sa.x = delta;
    sa.sc = sc;
    sa.partials = part;
    sa.n_active = nact;
    sa.c2f = (float)(-(double)o.beta * 1.4426950408889634);
    sa.wminf = o.w_min;
    sa.mbeta = -(double)o.beta;
    sa.wmin = (double)o.w_min;
    const int ipg = std::max(2, o.iters_per_graph & ~1);
    const int rounds = std::max(1, o.refine_rounds);
    int64_t sweeps = 0;
    int rounds_run = 0;
    for (int r = 0; r < rounds; ++r) {
        NCK(cudaMemsetAsync(nact, 0, sizeof(int), s));
        NCK(launch_start_round(sc, bx.nbox, r, o.tol, 1e-5, o.max_iter, r == 0 ? 1 : 0, nact, s));
        ++launches;
        int n_act = 0;
        NCK(cudaMemcpyAsync(&n_act, nact, sizeof(int), cudaMemcpyDeviceToHost, s));
        NCK(cudaStreamSynchronize(s));
        if (n_act == 0) break;
        rounds_run = r + 1;
        const int64_t cap = sweeps + (int64_t)o.max_iter + 4 * ipg;
        while (n_act > 0 && sweeps < cap) {
            int par = 0;
            for (int j = 0; j < ipg; ++j) {
                sa.u_in = u[par];
                sa.p_in = p[par];
                sa.u_out = u[par ^ 1];
                sa.p_out = p[par ^ 1];
                sa.parity = par;
                NCK(launch_sweep(0, G_U16, kTile, sa, grid, s));
                par ^= 1;
            }
            sweeps += ipg;
            launches += ipg;
            NCK(cudaMemcpyAsync(&n_act, nact, sizeof(int), cudaMemcpyDeviceToHost, s));
            NCK(cudaStreamSynchronize(s));
        }
        NCK(launch_accumulate(bx, Pad{}, seeds->code, delta, xhi, s));
        ra.keep_p = 1;
        NCK(launch_residual(0, ra, delta, s));
        NCK(launch_box_reduce(rpart, bpb, bx.nbox, sc, 0, s));
        launches += 3;
    }
    NCK(launch_copy_out(0, bx, xhi, x_out, s));
    ++launches;
    BoxScalars hs[kMaxBatch];
    NCK(cudaMemcpyAsync(hs, sc, batch * sizeof(BoxScalars), cudaMemcpyDeviceToHost, s));
    NCK(cudaStreamSynchronize(s));
    int bad = 0, nos = 0, it = 0;
    double rel = 0.0;
    int64_t vi = 0, nf = 0;
    for (int64_t b = 0; b < batch; ++b) {
        it = std::max(it, hs[b].iters);
        vi += (int64_t)hs[b].iters * hs[b].nfree;
        nf += hs[b].nfree;
        if (hs[b].nseed == 0) {
            ++nos;
            continue;
        }
        if (hs[b].bb > 0.0) {
            const double rr = std::sqrt(hs[b].rr_true / hs[b].bb);
            rel = std::max(rel, rr);
            if (rr > o.tol) ++bad;
        }
    }
    if (stats) {
        stats->iters = it;
        stats->refine_rounds = rounds_run;
        stats->rel_resid = rel;
        stats->voxel_iters = vi;
        stats->free_voxels = nf;
        stats->sweeps = sweeps;
        stats->launches = launches;
        stats->tile = kTile;
        stats->iters_per_graph = ipg;
        stats->not_converged = bad;
        stats->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    }
    if (nos > 0) return fail(RW_ERR_NO_SEEDS, "rw_solve_noalloc: a volume without any seed");
    if (bad > 0) return fail(RW_ERR_NOT_CONVERGED, "rw_solve_noalloc: a system above tol");
    return RW_OK;
}
