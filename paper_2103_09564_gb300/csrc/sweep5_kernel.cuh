// FP32 fused PCG sweep, register-blocked along x and z.
//
// The iteration of k_sweep (sweep_kernel.cuh: single-reduction Jacobi-PCG
// with explicit A-conjugation, u = D^-1 r stored, weights recomputed from g
// every sweep, six inner products), organised to spend few instructions per
// voxel:
//
// * A thread owns a strip of V = 4 consecutive voxels of one row of the tile
//   (one 16-byte word of every streamed vector) and marches it through z.
//   The strip's own values at z-1, z, z+1 (p_k, the g words, the z-edge
//   weights) stay in registers; only x/y neighbours are exchanged, through
//   double-buffered shared planes read with vector loads (the strip ends
//   through small per-strip arrays).
// * Every edge weight is evaluated once per plane, by the voxel that owns the
//   edge as its forward (+x, +y, +z) edge; the backward weights of a voxel
//   are its neighbours' forward ones.
// * The g words carry the voxel kind in the sign and NaN-ness of the float
//   (free: +g, seed: -g, absent: NaN; g >= 0 always), so a weight is
//   |g_a| - |g_b| -> exp -> floor at w_min with a NaN-propagating max -> NaN
//   to 0: no mask logic per edge.
// * u and p vanish on every non-free voxel, so p_k = u + beta p needs no mask.
// * The operator is applied in difference form, sum_j w_ij (p_i - p_j).
// * delta = (u', A u') is summed over the edges each voxel owns (+x, +y, +z),
//   one plane behind the stencil, from u' of the neighbours.
// * One barrier per plane; the z loop is unrolled by two (z-chunks start at
//   even planes) so the exchange buffers have static parity.  Loads are TMA
//   tile copies (cp.async.bulk.tensor, one per array and plane, issued by one
//   thread) into a ring of NR = D + 2 planes, D planes ahead, completing on
//   one mbarrier per ring slot.  Every wait is bounded: a wait that runs out
//   sets the error flag and the thread stops waiting (it still reaches every
//   barrier, so the CTA finishes).
//
// LOOP = true (small work that fits one wave of resident CTAs, launched
// cooperatively): one launch runs up to A.loop_iters PCG iterations,
// swapping the (u, p) buffers and their TMA descriptors each iteration; a
// grid barrier (arrival counter + generation word, bounded spin) separates
// the iterations, and its last arrival publishes whether any system is
// still active, so every CTA takes the same exit.  Per-system scalars are
// read through L2 (other CTAs update them between iterations).
//
// Tile: TX x TY interior voxels (TX a multiple of V).  The thread grid covers
// strips x = -V .. TX+V-1 (SX = TX/V + 2 strips) and rows y = -1 .. TY+1
// (RY = TY + 3 rows): p_k is needed on x = -1 .. TX+1, y = -1 .. TY+1; u' on
// x = 0 .. TX, y = 0 .. TY (the +x / +y ends of the owned edges).  The
// vectors have no margins: the 4-D tensor maps (x, y, z, box) fill what a
// tile copy reads beyond the box with zeros (u, p, delta) or NaN (g: absent
// voxels), and strips beyond the box do not store.  Rows are padded to a
// multiple of V voxels (16-byte TMA rows and strip starts).
#pragma once

#include <type_traits>

#include "rw_internal.h"
#include "sweep_kernel.cuh"

namespace rwk {

template <int TX, int TY, int V, int D, bool RING = false>
struct Strip {
    static constexpr int SX = TX / V + 2;       // strips per row (one halo strip each side)
    static constexpr int RY = TY + 3;           // rows y = -1 .. TY+1
    static constexpr int WS = TX + 2 * V;       // words per row
    static constexpr int PL = RY * WS;          // words per plane
    static constexpr int PS = RY * SX;          // strips per plane
    static constexpr int NR = D + 2;            // ring planes of p, delta (and g without RING)
    // ring planes of u: with RING, u' replaces u in its slot and is read one
    // step later (the delta of the plane behind), so the slot lives a step longer
    static constexpr int NRU = RING ? D + 3 : D + 2;
    // ring planes of the g words: read only in the step before their plane is
    // processed, so with RING their slot is free one step earlier
    static constexpr int NRG = RING ? D + 1 : D + 2;
    static constexpr int NI = TX * TY;          // interior voxels
    // delta box: the interior (V = 4: its first column is 16-byte aligned),
    // or the full strip width from the halo strip (V = 2)
    static constexpr int XW = V == 4 ? TX : WS, XC = V == 4 ? V : 0;
    static constexpr int PLA = (PL + 31) & ~31; // ring plane stride (128-byte aligned TMA destinations)
    static constexpr int NIA = (XW * TY + 31) & ~31;
    // words: ring (u: NRU planes, p and g: NR), delta ring (interior),
    // exchange planes and strip-end arrays (2 buffers each).  Without RING:
    // planes of p_k, forward x and y weights and u', arrays of the first p_k,
    // last p_k, last forward x weight and first u' of each strip.  With RING,
    // p_k and u' are written into the ring slots of p and u (neighbours read
    // them there): planes of the forward x and y weights and the array of the
    // last forward x weight remain.  Plus alignment slack.
    static constexpr int NEP = RING ? 2 : 4, NES = RING ? 1 : 4;
    static constexpr size_t words = (size_t)(NRU + NR + NRG) * PLA + (size_t)NR * NIA + (size_t)NEP * 2 * PL +
                                    (size_t)NES * 2 * PS + 32;
    static constexpr size_t bytes = words * 4;
};

template <int TX, int TY, int V, int D, bool RING = false>
constexpr size_t sweep5_smem_bytes() {
    return Strip<TX, TY, V, D, RING>::bytes;
}

// V-wide vector loads / stores (V = 4: 128-bit, V = 2: 64-bit).
template <int V>
__device__ __forceinline__ void ldv(const float* p, float* v) {
    if constexpr (V == 4) {
        const float4 a = *reinterpret_cast<const float4*>(p);
        v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
    } else {
        const float2 a = *reinterpret_cast<const float2*>(p);
        v[0] = a.x, v[1] = a.y;
    }
}
template <int V>
__device__ __forceinline__ void ldv(const uint32_t* p, uint32_t* v) {
    if constexpr (V == 4) {
        const uint4 a = *reinterpret_cast<const uint4*>(p);
        v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
    } else {
        const uint2 a = *reinterpret_cast<const uint2*>(p);
        v[0] = a.x, v[1] = a.y;
    }
}
template <int V>
__device__ __forceinline__ void stv(float* p, const float* v) {
    if constexpr (V == 4) *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    else *reinterpret_cast<float2*>(p) = make_float2(v[0], v[1]);
}
// mbarrier and TMA helpers (shared::cta addresses).
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait for the phase `parity` of `bar` to complete.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    for (int it = 0; it < (1 << 22); ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void tma_load4(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                          uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

// Edge weight max(exp(-beta (g_a - g_b)^2), w_min) from two signed g words;
// 0 when either voxel is absent (NaN).
__device__ __forceinline__ float wgt5(uint32_t a, uint32_t b, float c2, float wmin) {
    const float d = fabsf(__uint_as_float(a)) - fabsf(__uint_as_float(b));
    const float e = ex2_approx(c2 * d * d);
    float w;
    asm("max.NaN.f32 %0, %1, %2;" : "=f"(w) : "f"(e), "f"(wmin));
    return fmaxf(w, 0.0f);
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid barrier of iteration `it` of a looped sweep (thread 0 of each CTA
// calls it after the CTA's work): returns whether the next iteration runs,
// i.e. whether more than `stop` systems are still active.
// g = {arrivals, generation, go[2], iterations done}.  A wait that runs out
// sets *err and returns false.  `extra`: arrivals expected beyond the grid
// (0 in normal use; the fault injection of the host sets 1, so that no CTA is
// the last arrival and every wait runs out).
__device__ __forceinline__ bool grid_step(unsigned* g, int it, const int* n_active, int stop, int* err,
                                          int extra) {
    __threadfence();
    const unsigned target = gridDim.x * (unsigned)(it + 1) + (unsigned)extra;
    const unsigned old = atomicAdd(&g[0], 1u);
    if (old == target - 1u) {
        __threadfence();  // the other CTAs' updates of n_active precede their arrivals
        g[2 + (it & 1)] = (*(volatile const int*)n_active > stop) ? 1u : 0u;
        g[4] = (unsigned)(it + 1);
        __threadfence();
        atomicExch(&g[1], (unsigned)(it + 1));
    } else {
        long long spin = 0;
        while (ld_acquire_u32(&g[1]) < (unsigned)(it + 1)) {
            if (++spin > (1LL << 24)) {
                if (err) atomicExch(err, 1);
                return false;
            }
            __nanosleep(64);
        }
    }
    // the next iteration's TMA loads (async proxy) follow the acquired writes
    asm volatile("fence.proxy.async.global;\n" ::: "memory");
    return *(volatile const unsigned*)&g[2 + (it & 1)] != 0u;
}

// A field of the per-system scalars; in a looped sweep other CTAs wrote it
// in the previous iteration, so the load bypasses L1.
template <bool CG, typename T>
__device__ __forceinline__ T scalar_rd(const T* p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

// The whole record of a system's scalars, loaded past L1 (15 independent
// 8-byte loads), and stored back.
__device__ __forceinline__ void scalars_load_cg(const BoxScalars* S, BoxScalars* r) {
    static_assert(sizeof(BoxScalars) % 8 == 0, "8-byte words");
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(S);
    unsigned long long w[sizeof(BoxScalars) / 8];
#pragma unroll
    for (int k = 0; k < (int)(sizeof(BoxScalars) / 8); ++k) w[k] = __ldcg(src + k);
    memcpy(r, w, sizeof(BoxScalars));
}

__device__ __forceinline__ void scalars_store(BoxScalars* S, const BoxScalars& r) {
    unsigned long long w[sizeof(BoxScalars) / 8];
    memcpy(w, &r, sizeof(BoxScalars));
    unsigned long long* dst = reinterpret_cast<unsigned long long*>(S);
#pragma unroll
    for (int k = 0; k < (int)(sizeof(BoxScalars) / 8); ++k) dst[k] = w[k];
}

// Per-strip registers carried from one plane to the next.
template <int V>
struct StripState {
    float pkm[V];   // p_k(z-1)
    float pk0[V];   // p_k(z)
    uint32_t g0[V]; // g word(z)
    float wzm[V];   // w(z-1, z)
};

template <int TX, int TY, int V, int NT, int D, int MINB, bool LOOP = false, bool RING = false>
__global__ void __launch_bounds__(NT, MINB) k_sweep5(const __grid_constant__ SweepArgs A) {
    using L = Strip<TX, TY, V, D, RING>;
    constexpr int SX = L::SX, RY = L::RY, WS = L::WS, PL = L::PL, PS = L::PS, NR = L::NR, NRU = L::NRU,
                  NRG = L::NRG;
    constexpr int PLA = L::PLA, NIA = L::NIA;
    static_assert(V == 2 || V == 4, "strip width");
    static_assert(TX % V == 0, "tile width");
    static_assert(SX * RY <= NT, "threads");
    constexpr int XW = L::XW, XC = L::XC;
    static_assert((WS * 4) % 16 == 0 && (XW * 4) % 16 == 0 && (XC * 4) % 16 == 0 && (TX * 4) % 16 == 0 &&
                      WS <= 256 && RY <= 256,
                  "TMA box");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t mbar[NRU];
    // ring planes start on 128-byte boundaries (TMA destinations)
    const uint32_t raw_base = (uint32_t)__cvta_generic_to_shared(smem_raw);
    unsigned char* smem = smem_raw + ((128u - (raw_base & 127u)) & 127u);
    float* rU = reinterpret_cast<float*>(smem);                  // [NRU][RY][WS] (stride PLA)
    float* rP = rU + NRU * PLA;                                  // [NR][RY][WS]
    uint32_t* rG = reinterpret_cast<uint32_t*>(rP + NR * PLA);  // [NRG][RY][WS]
    float* rX = reinterpret_cast<float*>(rG + NRG * PLA);       // [NR][TY][TX] (stride NIA)
    float* eWY = rX + NR * NIA;                                  // [2][RY][WS]
    float* eWX4 = eWY + 2 * PL;                                  // [2][RY][WS]
    float* eWX = eWX4 + 2 * PL;                                  // [2][RY][SX] last forward x weight
    // without RING only: p_k and u' planes, first / last p_k and first u' per strip
    float* ePK = eWX + 2 * PS;                                   // [2][RY][WS]
    float* eUN = ePK + 2 * PL;                                   // [2][RY][WS]
    float* ePF = eUN + 2 * PL;                                   // [2][RY][SX]
    float* ePL = ePF + 2 * PS;                                   // [2][RY][SX]
    float* eUF = ePL + 2 * PS;                                   // [2][RY][SX]
    __shared__ int s_last;
    static_assert(6 * NT <= NRU * PLA, "the reduction scratch fits the u ring");

    // Threads are ordered by role so that warps are homogeneous: first the
    // strips owning output voxels (rows 0..TY-1, strips 1..TX/V), then the
    // other strips that compute u' (strip SX-1 of those rows, and row TY),
    // then the halo (strip 0 of every row; rows -1 and TY+1), then idle.
    const int tid = threadIdx.x;
    constexpr int NX = TX / V, NIN = TY * NX, NSN = TY + NX + 1, NHA = RY + 2 * (SX - 1);
    // owning strips: the first 8k strips of every row first (a quarter warp of
    // 128-bit shared loads then reads 128 contiguous bytes of one row), then
    // the remaining NX - 8k strips of every row
    constexpr int NX8 = NX / 8 * 8, NXR = NX - NX8 > 0 ? NX - NX8 : 1;  // (NXR unused when NX % 8 == 0)
    int sx, ry;
    if (tid < TY * NX8) {
        ry = 1 + tid / NX8, sx = 1 + tid % NX8;
    } else if (tid < NIN) {
        const int k = tid - TY * NX8;
        ry = 1 + k / NXR, sx = 1 + NX8 + k % NXR;
    } else if (tid < NIN + NSN) {
        const int k = tid - NIN;
        if (k < TY) ry = 1 + k, sx = SX - 1;
        else ry = TY + 1, sx = 1 + (k - TY);
    } else if (tid < NIN + NSN + NHA) {
        const int k = tid - NIN - NSN;
        if (k < RY) ry = k, sx = 0;
        else ry = (k - RY) < SX - 1 ? 0 : RY - 1, sx = 1 + (k - RY) % (SX - 1);
    } else {
        ry = RY, sx = 0;  // idle
    }
    const bool live = ry < RY;
    const int y = ry - 1;
    const bool sten = live && y >= 0 && y <= TY && sx >= 1;                  // computes u' (x = 0..TX+V-1)
    const bool inner = live && y >= 0 && y < TY && sx >= 1 && sx <= TX / V;  // owns output voxels
    const bool has_right = sx + 1 < SX;
    const bool has_down = ry + 1 < RY;
    const int wofs = ry * WS + V * sx;         // this strip in a plane
    const int sofs = ry * SX + sx;             // this strip in a strip array
    const int xofs = y * XW + V * sx - XC;     // this strip in the delta ring (inner only)

    const int tpb = A.ntx * A.nty * A.nzc;
    const int64_t nwork = (int64_t)(A.list ? *A.nlist : A.bx.nbox) * tpb;
    const int PX = A.px, PY = A.py;
    const int64_t plane = (int64_t)PX * PY;
    const int64_t bstride = plane * A.pz;
    const float c2 = A.c2f, wmin = A.wminf;
    const uint32_t sU = (uint32_t)__cvta_generic_to_shared(rU), sP = (uint32_t)__cvta_generic_to_shared(rP);
    const uint32_t sG = (uint32_t)__cvta_generic_to_shared(rG), sX = (uint32_t)__cvta_generic_to_shared(rX);
    const uint32_t sB = (uint32_t)__cvta_generic_to_shared(mbar);
    if (tid == 0) {
#pragma unroll
        for (int k = 0; k < NRU; ++k) mbar_init(sB + 8 * k, 1);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    uint32_t seq = 0;      // planes issued by this CTA so far (the same in every thread)
    bool waited_out = false;
    __shared__ int s_go;

    for (int it = 0; it < (LOOP ? A.loop_iters : 1); ++it) {
    // iteration `it` reads the (u, p) copy of parity A.parity + it
    const bool odd = LOOP && (it & 1);
    const CUtensorMap* mu = odd ? &A.tm.ua : &A.tm.u;
    const CUtensorMap* mp = odd ? &A.tm.pa : &A.tm.p;
    float* const u_out = static_cast<float*>(odd ? const_cast<void*>(A.u_in) : A.u_out);
    float* const p_out = static_cast<float*>(odd ? const_cast<void*>(A.p_in) : A.p_out);
    const int out_par = (A.parity + it + 1) & 1;

    for (int64_t w = blockIdx.x; w < nwork; w += gridDim.x) {
        const int li = (int)(w / tpb);  // position in the list of active systems
        const int box = A.list ? A.list[li] : li;
        const int t = (int)(w - (int64_t)li * tpb);
        BoxScalars* S = A.sc + box;
        if (!scalar_rd<LOOP>(&S->active)) continue;
        const int tx = t % A.ntx, ty = (t / A.ntx) % A.nty, tz = t / (A.ntx * A.nty);
        const float alpha = (float)scalar_rd<LOOP>(&S->alpha);
        // p_k = ku u + bp p: u + beta p, or p itself when the direction is kept
        const bool keep = scalar_rd<LOOP>(&S->phase) == 2;
        const float ku = keep ? 0.0f : 1.0f, bp = keep ? 1.0f : (float)scalar_rd<LOOP>(&S->beta);
        int ez = A.bx.nz;
        if (A.bx.ext) ez = A.bx.ext[3 * box + 2];
        const int z0 = tz * A.zc;  // even: the chunk depth is even
        const int z1 = min(z0 + A.zc, ez);
        float a_gam = 0.f, a_rr = 0.f, a_del = 0.f, a_eps = 0.f, a_pi = 0.f, a_tau = 0.f;
        if (z0 < ez) {
            // this strip's first voxel (inner strips: x = tx TX + V (sx - 1), y = ty TY + ry - 1);
            // strips beyond the box (a tile's ragged edge) do not store
            const int gx = tx * TX + V * (sx - 1), gy = ty * TY + ry - 1;
            const bool in_box = gx < PX && gy < PY;
            const int64_t base = (int64_t)box * bstride + (int64_t)gy * PX + gx;
            float* Xb = static_cast<float*>(A.x) + base;
            float* Uo = u_out + base;
            float* Po = p_out + base;

            // plane z of this work item is the CTA's load number q(z); its p,
            // g and delta sit in ring slot q % NR, its u in slot q % NRU, and it
            // completes phase (q / NRU) & 1 of mbarrier q % NRU
            const uint32_t q0 = seq - (uint32_t)(z0 - 1);
            auto slot = [&](int z) { return (int)((q0 + (uint32_t)z) % NR); };
            auto slotu = [&](int z) { return (int)((q0 + (uint32_t)z) % NRU); };
            auto slotg = [&](int z) { return (int)((q0 + (uint32_t)z) % NRG); };
            auto phase = [&](int z) { return ((q0 + (uint32_t)z) / NRU) & 1u; };
            // TMA box origins: the tile's first strip and row (x = -V, y = -1)
            // for u, p, g; row y = 0 from column x = XC - V for delta; the
            // 4th coordinate is the box
            const int cx = tx * TX - V, cy = ty * TY - 1;
            auto issue = [&](int z) {
                if (tid != 0) return;
                const int sl = slot(z), su = slotu(z);
                const uint32_t bar = sB + 8 * su;
                const bool wx = z >= z0 && z < z1;
                asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
                mbar_expect_tx(bar, (uint32_t)(3 * PL * 4 + (wx ? XW * TY * 4 : 0)));
                tma_load4(sU + su * PLA * 4, mu, cx, cy, z, box, bar);
                tma_load4(sP + sl * PLA * 4, mp, cx, cy, z, box, bar);
                tma_load4(sG + slotg(z) * PLA * 4, &A.tm.g, cx, cy, z, box, bar);
                if (wx) tma_load4(sX + sl * NIA * 4, &A.tm.x, cx + XC, cy + 1, z, box, bar);
            };

            // One plane step.  At entry `in` holds the strip's registers for
            // plane z; `out` receives those for plane z+1.  BC = z & 1.
            auto step = [&](const int z, const StripState<V>& in, StripState<V>& out, auto bcc) {
                constexpr int BC = decltype(bcc)::value, BN = BC ^ 1;
                if (!waited_out && !mbar_wait(sB + 8 * slotu(z + 1), phase(z + 1))) {
                    waited_out = true;
                    if (A.err) atomicExch(A.err, 1);
                }
                __syncthreads();
                if (z + 1 + D <= z1 + 1) issue(z + 1 + D);
                const int sn = slot(z + 1);

                // -- 1: plane z+1 enters: p_k and the z edge (z, z+1)
                float pkn[V], wz0[V];
                uint32_t gn[V];
#pragma unroll
                for (int i = 0; i < V; ++i) pkn[i] = wz0[i] = 0.0f, gn[i] = GC_ABSENT;
                if (live) {
                    float uu[V], pp[V];
                    ldv<V>(rU + slotu(z + 1) * PLA + wofs, uu);
                    ldv<V>(rP + sn * PLA + wofs, pp);
                    ldv<V>(rG + slotg(z + 1) * PLA + wofs, gn);
#pragma unroll
                    for (int i = 0; i < V; ++i) pkn[i] = fmaf(bp, pp[i], ku * uu[i]);
                    if (sten) {
#pragma unroll
                        for (int i = 0; i < V; ++i) wz0[i] = wgt5(in.g0[i], gn[i], c2, wmin);
                    }
                    if constexpr (RING) {
                        stv<V>(rP + sn * PLA + wofs, pkn);  // p_k replaces p in its slot
                    } else {
                        stv<V>(ePK + BN * PL + wofs, pkn);
                        ePF[BN * PS + sofs] = pkn[0];
                        ePL[BN * PS + sofs] = pkn[V - 1];
                    }
                }

                // -- 2: stencil and update at plane z
                float un0[V];
#pragma unroll
                for (int i = 0; i < V; ++i) un0[i] = 0.0f;
                if (sten && z >= z0) {
                    float uu[V], puu[V], pdd[V], wuu[V], wy0[V], wx0[V];
                    ldv<V>(rU + slotu(z) * PLA + wofs, uu);
                    float pl, pr;
                    if constexpr (RING) {
                        const float* pk = rP + slot(z) * PLA;
                        pl = pk[wofs - 1];
                        pr = has_right ? pk[wofs + V] : 0.0f;
                        ldv<V>(pk + wofs - WS, puu);
                        ldv<V>(pk + wofs + WS, pdd);
                    } else {
                        pl = ePL[BC * PS + sofs - 1];
                        pr = has_right ? ePF[BC * PS + sofs + 1] : 0.0f;
                        ldv<V>(ePK + BC * PL + wofs - WS, puu);
                        ldv<V>(ePK + BC * PL + wofs + WS, pdd);
                    }
                    const float wl = eWX[BC * PS + sofs - 1];
                    ldv<V>(eWY + BC * PL + wofs - WS, wuu);
                    ldv<V>(eWY + BC * PL + wofs, wy0);
                    ldv<V>(eWX4 + BC * PL + wofs, wx0);
                    float sv[V], dv[V];
#pragma unroll
                    for (int i = 0; i < V; ++i) {
                        const float p0 = in.pk0[i];
                        const float wL = i == 0 ? wl : wx0[i - 1], wR = wx0[i];
                        const float pL = i == 0 ? pl : in.pk0[i - 1], pR = i == V - 1 ? pr : in.pk0[i + 1];
                        dv[i] = ((wL + wR) + (wuu[i] + wy0[i])) + (in.wzm[i] + wz0[i]);
                        // difference form: the weak edges of a strongly linked
                        // voxel keep their relative precision
                        sv[i] = ((wL * (p0 - pL) + wR * (p0 - pR)) + (wuu[i] * (p0 - puu[i]) + wy0[i] * (p0 - pdd[i]))) +
                                (in.wzm[i] * (p0 - in.pkm[i]) + wz0[i] * (p0 - pkn[i]));
                        // free voxels carry +g (sign bit clear)
                        const bool isfree = (int)in.g0[i] >= 0 && dv[i] > 0.0f;
                        un0[i] = isfree ? uu[i] - alpha * sv[i] * __fdividef(1.0f, dv[i]) : 0.0f;
                    }
                    if constexpr (RING) {
                        stv<V>(rU + slotu(z) * PLA + wofs, un0);  // u' replaces u in its slot
                    } else {
                        stv<V>(eUN + BC * PL + wofs, un0);
                        eUF[BC * PS + sofs] = un0[0];
                    }
                    if (inner && z < z1) {
                        const int64_t pz = (int64_t)z * plane;
                        float xn[V];
                        ldv<V>(rX + slot(z) * NIA + xofs, xn);
#pragma unroll
                        for (int i = 0; i < V; ++i) xn[i] = fmaf(alpha, in.pk0[i], xn[i]);
                        if (in_box) {
                            stv<V>(Uo + pz, un0);
                            stv<V>(Po + pz, in.pk0);
                            stv<V>(Xb + pz, xn);
                        }
#pragma unroll
                        for (int i = 0; i < V; ++i) {
                            // p_k and u' vanish on non-free voxels
                            const float du = dv[i] * un0[i];
                            a_gam = fmaf(du, un0[i], a_gam);
                            a_rr = fmaf(du, du, a_rr);
                            a_eps = fmaf(un0[i], sv[i], a_eps);
                            a_pi = fmaf(in.pk0[i], sv[i], a_pi);
                            a_tau = fmaf(du, in.pk0[i], a_tau);
                        }
                    }
                }

                // -- 3: delta over the edges owned by plane z-1 (+x, +y, +z)
                if (inner && z - 1 >= z0) {
                    float ur, udd[V], unm[V], wxm[V], wym[V];
                    if constexpr (RING) {
                        const float* un = rU + slotu(z - 1) * PLA;
                        ur = un[wofs + V];
                        ldv<V>(un + wofs + WS, udd);
                        ldv<V>(un + wofs, unm);
                    } else {
                        ur = eUF[BN * PS + sofs + 1];
                        ldv<V>(eUN + BN * PL + wofs + WS, udd);
                        ldv<V>(eUN + BN * PL + wofs, unm);
                    }
                    ldv<V>(eWX4 + BN * PL + wofs, wxm);
                    ldv<V>(eWY + BN * PL + wofs, wym);
#pragma unroll
                    for (int i = 0; i < V; ++i) {
                        const float dx = unm[i] - (i < V - 1 ? unm[i + 1] : ur);
                        const float dy = unm[i] - udd[i];
                        const float dz = unm[i] - un0[i];
                        a_del = fmaf(wxm[i] * dx, dx, a_del);
                        a_del = fmaf(wym[i] * dy, dy, a_del);
                        a_del = fmaf(in.wzm[i] * dz, dz, a_del);
                    }
                }

                // -- 4: forward x / y weights of plane z+1 (into the slots plane
                // z-1 used: their last reader was step 3 of this thread).  Of
                // the halo, strip 0 needs its last x weight and row -1 its y
                // weights; row TY+1 none.
                if (live && ry < RY - 1) {
                    const uint32_t* gpl = rG + slotg(z + 1) * PLA;
                    const uint32_t gr = has_right ? gpl[wofs + V] : GC_ABSENT;
                    uint32_t gdd[V];
                    if (has_down) {
                        ldv<V>(gpl + wofs + WS, gdd);
                    } else {
#pragma unroll
                        for (int i = 0; i < V; ++i) gdd[i] = GC_ABSENT;
                    }
                    float wxn[V], wyn[V];
#pragma unroll
                    for (int i = 0; i < V; ++i) {
                        wxn[i] = wgt5(gn[i], i < V - 1 ? gn[i + 1] : gr, c2, wmin);
                        wyn[i] = wgt5(gn[i], gdd[i], c2, wmin);
                    }
                    stv<V>(eWY + BN * PL + wofs, wyn);
                    stv<V>(eWX4 + BN * PL + wofs, wxn);
                    eWX[BN * PS + sofs] = wxn[V - 1];
                }
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    out.pkm[i] = in.pk0[i];
                    out.pk0[i] = pkn[i];
                    out.g0[i] = gn[i];
                    out.wzm[i] = wz0[i];
                }
            };

#pragma unroll
            for (int d = 0; d < D; ++d)
                if (z0 - 1 + d <= z1 + 1) issue(z0 - 1 + d);
            StripState<V> sa, sb;
#pragma unroll
            for (int i = 0; i < V; ++i) {
                sa.pkm[i] = sa.pk0[i] = sa.wzm[i] = 0.0f;
                sa.g0[i] = 0xffc00000u;  // plane z0-2 is never used: absent
            }
            int z = z0 - 2;
            for (; z + 1 <= z1; z += 2) {
                step(z, sa, sb, std::integral_constant<int, 0>());
                step(z + 1, sb, sa, std::integral_constant<int, 1>());
            }
            if (z <= z1) step(z, sa, sb, std::integral_constant<int, 0>());
            seq += (uint32_t)(z1 - z0 + 3);  // planes z0-1 .. z1+1
        }
        // the six sums in double-FP32 (FP32 pipes: on GB300 a chain of
        // dependent FP64 operations here would sit on every sweep's critical
        // path).  The per-thread partials go through shared memory (the u ring,
        // idle between work items: every issued plane has been consumed) and
        // warp j sums partial j: NT / 32 values per lane in two chains, then a
        // shuffle tree.  Per-item results are (hi, lo) float pairs in the
        // 8-byte slots of A.partials.
        const int lane = tid & 31, wid = tid >> 5;
        float* rs = rU;  // [6][NT]
        __syncthreads();  // every thread is done with the ring
        rs[0 * NT + tid] = a_gam;
        rs[1 * NT + tid] = a_rr;
        rs[2 * NT + tid] = a_del;
        rs[3 * NT + tid] = a_eps;
        rs[4 * NT + tid] = a_pi;
        rs[5 * NT + tid] = a_tau;
        __syncthreads();
        // (fewer than six warps: warp w also takes partials w + NT / 32, ...)
        for (int j = wid; j < 6; j += NT / 32) {
            const float* r = rs + j * NT;
            DF c0 = {0.0f, 0.0f}, c1 = {0.0f, 0.0f};
#pragma unroll
            for (int i = 0; i < NT / 32; i += 2) {
                c0 = df_add(c0, DF{r[lane + 32 * i], 0.0f});
                if (i + 1 < NT / 32) c1 = df_add(c1, DF{r[lane + 32 * i + 32], 0.0f});
            }
            DF v = df_add(c0, c1);
#pragma unroll
            for (int m = 16; m > 0; m >>= 1) v = df_add(v, df_shfl_xor(v, m));
            if (lane == 0) {
                float2* pp = reinterpret_cast<float2*>(A.partials + ((int64_t)li * tpb + t) * 6);
                pp[j] = make_float2(v.hi, v.lo);
                __threadfence();
            }
        }
        __syncthreads();
        if (tid == 0) {
            const unsigned prev = atomicAdd(&S->counter, 1u);
            s_last = (prev == (unsigned)tpb - 1u);
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            DF* tot = reinterpret_cast<DF*>(rs);  // [6]
            for (int j = wid; j < 6; j += NT / 32) {
                // warp w: partial j of the tpb work items of the system
                DF v;
                const float2* pb = reinterpret_cast<const float2*>(A.partials + (int64_t)li * tpb * 6) + j;
                DF c0 = {0.0f, 0.0f}, c1 = {0.0f, 0.0f};
                int k = lane;
                for (; k + 32 < tpb; k += 64) {
                    const float2 q0 = __ldcg(pb + 6 * k), q1 = __ldcg(pb + 6 * (k + 32));
                    c0 = df_add(c0, DF{q0.x, q0.y});
                    c1 = df_add(c1, DF{q1.x, q1.y});
                }
                if (k < tpb) {
                    const float2 q0 = __ldcg(pb + 6 * k);
                    c0 = df_add(c0, DF{q0.x, q0.y});
                }
                v = df_add(c0, c1);
#pragma unroll
                for (int m = 16; m > 0; m >>= 1) v = df_add(v, df_shfl_xor(v, m));
                if (lane == 0) tot[j] = v;  // rs is read no more: the items' sums are in A.partials
            }
            __syncthreads();
            if (tid == 0) {
                DF tv[6];
#pragma unroll
                for (int j = 0; j < 6; ++j) tv[j] = tot[j];
                if constexpr (LOOP) {
                    // the record as other CTAs left it, updated in registers
                    BoxScalars loc;
                    scalars_load_cg(S, &loc);
                    loc.counter = 0u;
                    finalize_box_df(&loc, tv, A.n_active, out_par);
                    scalars_store(S, loc);
                } else {
                    S->counter = 0u;
                    finalize_box_df(S, tv, A.n_active, out_par);
                }
            }
        }
        __syncthreads();
    }
    if constexpr (LOOP) {
        // this iteration's global writes become visible to the next one's
        // TMA reads (async proxy) before the grid barrier releases them
        asm volatile("fence.proxy.async.global;\n" ::: "memory");
        __syncthreads();
        if (tid == 0) s_go = grid_step(A.gsync, it, A.n_active, A.loop_stop, A.err, A.barrier_extra) ? 1 : 0;
        __syncthreads();
        if (!s_go) break;
    }
    }
}

}  // namespace rwk
