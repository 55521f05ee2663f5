// Host-side facilities shared by the translation units of the C ABI
// (rw_api.cu: workspace, PCG driver, plain solve and adjoint; rw_hier.cu: LOD
// pyramid and hierarchical trees).
#pragma once

#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "rw_api.h"
#include "rw_internal.h"

// Return RW_ERR_OOM / RW_ERR_CUDA (with the call and its error text) when a
// CUDA call fails; RCK returns any status other than RW_OK.
#define CK(call)                                                                                                 \
    do {                                                                                                         \
        cudaError_t e_ = (call);                                                                                 \
        if (e_ != cudaSuccess) {                                                                                 \
            cudaGetLastError();                                                                                  \
            return fail(e_ == cudaErrorMemoryAllocation ? RW_ERR_OOM : RW_ERR_CUDA, "%s failed: %s (%s:%d)", #call, \
                        cudaGetErrorString(e_), __FILE__, __LINE__);                                            \
        }                                                                                                        \
    } while (0)

#define RCK(expr)                       \
    do {                                \
        rw_status r_ = (expr);          \
        if (r_ != RW_OK) return r_;     \
    } while (0)

namespace rwh {

using rwk::Boxes;
using rwk::BoxScalars;

extern thread_local std::string g_err;  // message of the last failure (rw_last_error)
extern std::recursive_mutex g_mu;       // serialises the ABI's calls
extern int64_t g_launches;              // kernels launched since the current call started (guarded by g_mu)

// Record a failure (the message rw_last_error returns) and return its status.
rw_status fail(rw_status st, const char* fmt, ...);
double now_ms();

// Count a kernel launch made through one of the rwk::launch_* helpers.
inline cudaError_t counted(cudaError_t e) {
    ++g_launches;
    return e;
}

// Workspace: named slots of device memory, grown on demand and cached.
enum Slot {
    S_G, S_U0, S_U1, S_P0, S_P1, S_DELTA, S_XHI, S_PART, S_RPART, S_SC, S_NACT, S_VOL, S_CODE, S_VAL, S_X0, S_OUT,
    S_RHS, S_EXT, S_JOBS, S_LAB, S_BFLAGS, S_STATS, S_POOL_G, S_POOL_CODE, S_POOL_X, S_ADJ_PART, S_DBETA, S_DG,
    S_XF, S_STATUS, S_GC, S_LIST, S_W64, S_NODES, S_SHARD_V, S_SHARD_N, S_COUNT
};

struct DevWorkspace {
    void* p[S_COUNT] = {};
    size_t cap[S_COUNT] = {};
    cudaStream_t stream = nullptr;
    int* pinned = nullptr;  // page-locked host words read back after graph chunks
    int sms = 0;
};

rw_status ws_get(DevWorkspace* w, int slot, size_t bytes, void** out);

template <typename P>
rw_status ws_get_t(DevWorkspace* w, int slot, size_t bytes, P** out) {
    void* v = nullptr;
    RCK(ws_get(w, slot, bytes, &v));
    *out = static_cast<P*>(v);
    return RW_OK;
}

bool is_device_ptr(const void* p);
// Device address of page-locked (pinned or registered) host memory, which
// kernels can write directly; nullptr for other pointers.
void* pinned_device_alias(void* p);
// Caller stream -> internal stream ordering (inputs produced on `user` are
// complete); leave() synchronises the internal stream and reports errors.
rw_status enter(DevWorkspace** w, void* user);
rw_status leave(DevWorkspace* w);
// Device view of a caller array: the pointer itself, or a copy staged in
// workspace slot `slot`.
rw_status stage_in(DevWorkspace* w, int slot, const void* p, size_t bytes, const void** out);
rw_status check_opts(const rw_opts& o);
// Checks a volume description; voxels per volume and volumes in the batch.
rw_status check_volume(const rw_volume* v, int64_t* nvox, int64_t* batch);

// The PCG driver over a batch of equally sized boxes.
struct SolveProblem {
    Boxes bx;
    const void* g;
    int gtype;
    const uint8_t* code;
    const float* value;
    const float* x0;
    const float* rhs;
    double* x_hi;
    int init_x;
};

struct SolveResult {
    std::vector<BoxScalars> sc;
    int rounds = 0;
    int64_t sweeps = 0;
    double ms_solve = 0.0;
    double ms_sweeps = 0.0;   // device time of the graph-launched sweeps
    int tile = 0;
    int ipg = 0;
    int fp64_fallback = 0;
};

rw_status solve_boxes(DevWorkspace* w, const SolveProblem& P, const rw_opts& o, SolveResult* R);
void stats_from(const SolveResult& R, const rw_opts& o, rw_stats* st, int* n_unconverged, int* n_noseed);

}  // namespace rwh
