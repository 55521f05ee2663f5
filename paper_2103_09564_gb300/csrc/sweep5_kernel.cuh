// FP32 fused PCG sweep, register-blocked along x and z.
//
// Same iteration as k_sweep4 (single-reduction Jacobi-PCG with explicit
// A-conjugation, u = D^-1 r stored, weights recomputed from g every sweep,
// six inner products), organised to spend few instructions per voxel:
//
// * A thread owns a strip of four consecutive voxels of one row of the tile
//   (one 16-byte word of every streamed vector) and marches it through z.
//   The strip's own values at z-1, z, z+1 (p_k, the g|code words, the z-edge
//   weights) stay in registers; only x/y neighbours are exchanged, through
//   double-buffered shared planes read with 128-bit loads (the strip ends
//   through small per-strip arrays).
// * Every edge weight is evaluated once per plane, by the voxel that owns the
//   edge as its forward (+x, +y, +z) edge; the backward weights of a voxel
//   are its neighbours' forward ones.
// * The operator is applied in difference form, sum_j w_ij (p_i - p_j).
// * delta = (u', A u') is summed over the edges each voxel owns (+x, +y, +z),
//   one plane behind the stencil, from u' of the neighbours.
// * One barrier per plane.  Loads are 16-byte cp.async copies into a ring of
//   NR = D + 2 planes, issued D planes ahead.
//
// Tile: TX x TY interior voxels (TX a multiple of 4).  The thread grid covers
// strips x = -4 .. TX+3 (SX = TX/4 + 2 strips) and rows y = -1 .. TY+1
// (RY = TY + 3 rows): p_k is needed on x = -1 .. TX+1, y = -1 .. TY+1; u' on
// x = 0 .. TX, y = 0 .. TY (the +x / +y ends of the owned edges).  This needs
// the padded layout with an x margin of 4 voxels (the first strip of a tile
// starts 16-byte aligned) and y / z margins of 2.
#pragma once

#include "rw_internal.h"
#include "sweep4_kernel.cuh"

namespace rwk {

template <int TX, int TY, int D>
struct Strip {
    static constexpr int SX = TX / 4 + 2;       // strips per row (one 4-voxel halo strip each side)
    static constexpr int RY = TY + 3;           // rows y = -1 .. TY+1
    static constexpr int WS = TX + 8;           // words per row
    static constexpr int PL = RY * WS;          // words per plane
    static constexpr int PS = RY * SX;          // strips per plane
    static constexpr int NR = D + 2;            // ring planes
    static constexpr int NI = TX * TY;          // interior voxels
    // words: ring (u, p, g|code; NR planes), delta ring (interior), exchange
    // planes (p_k, forward x and y weights, u'; 2 each), strip-end arrays
    // (first p_k, last p_k, last forward x weight, first u'; 2 each)
    static constexpr size_t words = (size_t)3 * NR * PL + (size_t)NR * NI + (size_t)4 * 2 * PL + (size_t)4 * 2 * PS;
    static constexpr size_t bytes = words * 4;
};

template <int TX, int TY, int D>
constexpr size_t sweep5_smem_bytes() {
    return Strip<TX, TY, D>::bytes;
}

__device__ __forceinline__ float4 lds4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ uint4 lds4u(const uint32_t* p) { return *reinterpret_cast<const uint4*>(p); }
__device__ __forceinline__ void sts4(float* p, float a, float b, float c, float d) {
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void stg4(float* p, float a, float b, float c, float d) {
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}

template <int TX, int TY, int NT, int D, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_sweep5(const SweepArgs A) {
    using L = Strip<TX, TY, D>;
    constexpr int SX = L::SX, RY = L::RY, WS = L::WS, PL = L::PL, PS = L::PS, NR = L::NR;
    static_assert(TX % 4 == 0, "tile width");
    static_assert(SX * RY <= NT, "threads");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* rU = reinterpret_cast<float*>(smem_raw);             // [NR][RY][WS]
    float* rP = rU + NR * PL;                                    // [NR][RY][WS]
    uint32_t* rG = reinterpret_cast<uint32_t*>(rP + NR * PL);   // [NR][RY][WS]
    float* rX = reinterpret_cast<float*>(rG + NR * PL);         // [NR][TY][TX]
    float* ePK = rX + NR * L::NI;                                // [2][RY][WS]
    float* eWY = ePK + 2 * PL;                                   // [2][RY][WS]
    float* eWX4 = eWY + 2 * PL;                                  // [2][RY][WS]
    float* eUN = eWX4 + 2 * PL;                                  // [2][RY][WS]
    float* ePF = eUN + 2 * PL;                                   // [2][RY][SX] first p_k of the strip
    float* ePL = ePF + 2 * PS;                                   // [2][RY][SX] last p_k
    float* eWX = ePL + 2 * PS;                                   // [2][RY][SX] last forward x weight
    float* eUF = eWX + 2 * PS;                                   // [2][RY][SX] first u'
    __shared__ double red[6 * (NT / 32)];
    __shared__ int s_last;

    const int tid = threadIdx.x;
    const int sx = tid % SX, ry = tid / SX;
    const bool live = ry < RY;
    const int y = ry - 1;
    const bool sten = live && y >= 0 && y <= TY && sx >= 1;              // computes u' (x = 0..TX+3)
    const bool inner = live && y >= 0 && y < TY && sx >= 1 && sx <= TX / 4;  // owns output voxels
    const bool has_right = sx + 1 < SX;
    const bool has_down = ry + 1 < RY;
    const int wofs = ry * WS + 4 * sx;      // this strip in a plane
    const int sofs = ry * SX + sx;          // this strip in a strip array
    const int xofs = (y * TX + 4 * (sx - 1));  // this strip in the delta ring (inner only)

    const int tpb = A.ntx * A.nty * A.nzc;
    const int64_t nwork = (int64_t)(A.list ? *A.nlist : A.bx.nbox) * tpb;
    const int PX = A.px, PY = A.py;
    const int64_t plane = (int64_t)PX * PY;
    const int64_t bstride = plane * A.pz;
    const float c2 = A.c2f, wmin = A.wminf;
    const uint32_t s_base = (uint32_t)__cvta_generic_to_shared(smem_raw);

    for (int64_t w = blockIdx.x; w < nwork; w += gridDim.x) {
        const int li = (int)(w / tpb);  // position in the list of active systems
        const int box = A.list ? A.list[li] : li;
        const int t = (int)(w - (int64_t)li * tpb);
        BoxScalars* S = A.sc + box;
        if (!S->active) continue;
        const int tx = t % A.ntx, ty = (t / A.ntx) % A.nty, tz = t / (A.ntx * A.nty);
        const float alpha = (float)S->alpha, bcg = (float)S->beta;
        const bool keep = S->phase == 2;
        int ez = A.bx.nz;
        if (A.bx.ext) ez = A.bx.ext[3 * box + 2];
        const int z0 = tz * A.zc;
        const int z1 = min(z0 + A.zc, ez);
        float a_gam = 0.f, a_rr = 0.f, a_del = 0.f, a_eps = 0.f, a_pi = 0.f, a_tau = 0.f;
        if (z0 < ez) {
            // padded coordinates of this strip: x + 4, y + 2, z + 2
            const int64_t base = (int64_t)box * bstride + (int64_t)(ty * TY + ry + 1) * PX + tx * TX + 4 * sx;
            const float* Ub = static_cast<const float*>(A.u_in) + base;
            const float* Pb = static_cast<const float*>(A.p_in) + base;
            const uint32_t* Gb = A.gc + base;
            float* Xb = static_cast<float*>(A.x) + base;
            float* Uo = static_cast<float*>(A.u_out) + base;
            float* Po = static_cast<float*>(A.p_out) + base;

            auto slot = [](int z) { return (z + 2 * NR) % NR; };
            auto issue = [&](int z) {
                if (!live) return;
                const int64_t pz = (int64_t)(z + 2) * plane;
                const uint32_t so = (uint32_t)((slot(z) * PL + wofs) * 4);
                cp_async16(s_base + so, Ub + pz);
                cp_async16(s_base + (uint32_t)(NR * PL * 4) + so, Pb + pz);
                cp_async16(s_base + (uint32_t)(2 * NR * PL * 4) + so, Gb + pz);
                if (inner && z >= z0 && z < z1)
                    cp_async16(s_base + (uint32_t)((3 * NR * PL + slot(z) * L::NI + xofs) * 4), Xb + pz);
            };

#pragma unroll
            for (int d = 0; d < D; ++d) {
                if (z0 - 1 + d <= z1 + 1) issue(z0 - 1 + d);
                cp_async_commit();
            }
            // registers of this strip (see the step below for their planes)
            float pkm[4] = {0, 0, 0, 0}, pk0[4] = {0, 0, 0, 0};
            uint32_t g0[4] = {0u, 0u, 0u, 0u};
            float wzm[4] = {0, 0, 0, 0};

            // step z: at entry pk0 = p_k(z), pkm = p_k(z-1), g0 = g|code(z),
            // wzm = w(z-1, z).  The strip's forward x / y weights of plane z
            // and u'(z-1) are read back from its own slots of the exchange
            // planes (only this thread writes them).
            for (int z = z0 - 2; z <= z1; ++z) {
                cp_async_wait<D - 1>();
                __syncthreads();
                if (z + 1 + D <= z1 + 1) issue(z + 1 + D);
                cp_async_commit();
                const int bn = (z + 1) & 1, bc = z & 1;
                const int sn = slot(z + 1);

                // -- 1: plane z+1 enters: p_k and the z edge (z, z+1)
                float pkn[4] = {0, 0, 0, 0}, wz0[4] = {0, 0, 0, 0};
                uint32_t gn[4] = {0u, 0u, 0u, 0u};
                if (live) {
                    const float4 u4 = lds4(rU + sn * PL + wofs);
                    const float4 p4 = lds4(rP + sn * PL + wofs);
                    const uint4 g4 = lds4u(rG + sn * PL + wofs);
                    const float uu[4] = {u4.x, u4.y, u4.z, u4.w}, pp[4] = {p4.x, p4.y, p4.z, p4.w};
                    gn[0] = g4.x;
                    gn[1] = g4.y;
                    gn[2] = g4.z;
                    gn[3] = g4.w;
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const bool fr = (gn[i] & 3u) == 1u;
                        pkn[i] = keep ? pp[i] : (fr ? fmaf(bcg, pp[i], uu[i]) : 0.0f);
                        wz0[i] = wgt(g0[i], gn[i], c2, wmin);
                    }
                    sts4(ePK + bn * PL + wofs, pkn[0], pkn[1], pkn[2], pkn[3]);
                    ePF[bn * PS + sofs] = pkn[0];
                    ePL[bn * PS + sofs] = pkn[3];
                }

                // -- 2: stencil and update at plane z
                float un0[4] = {0, 0, 0, 0};
                if (sten && z >= z0) {
                    const float4 uk = lds4(rU + slot(z) * PL + wofs);
                    const float uu[4] = {uk.x, uk.y, uk.z, uk.w};
                    const float pl = ePL[bc * PS + sofs - 1];
                    const float pr = has_right ? ePF[bc * PS + sofs + 1] : 0.0f;
                    const float wl = eWX[bc * PS + sofs - 1];
                    const float4 pu = lds4(ePK + bc * PL + wofs - WS);
                    const float4 pd = lds4(ePK + bc * PL + wofs + WS);
                    const float4 wu = lds4(eWY + bc * PL + wofs - WS);
                    const float4 wyo = lds4(eWY + bc * PL + wofs);
                    const float4 wxo = lds4(eWX4 + bc * PL + wofs);
                    const float puu[4] = {pu.x, pu.y, pu.z, pu.w}, pdd[4] = {pd.x, pd.y, pd.z, pd.w};
                    const float wuu[4] = {wu.x, wu.y, wu.z, wu.w};
                    const float wy0[4] = {wyo.x, wyo.y, wyo.z, wyo.w}, wx0[4] = {wxo.x, wxo.y, wxo.z, wxo.w};
                    float sv[4], dv[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float p0 = pk0[i];
                        const float wL = i == 0 ? wl : wx0[i - 1], wR = wx0[i];
                        const float pL = i == 0 ? pl : pk0[i - 1], pR = i == 3 ? pr : pk0[i + 1];
                        dv[i] = ((wL + wR) + (wuu[i] + wy0[i])) + (wzm[i] + wz0[i]);
                        // difference form: the weak edges of a strongly linked
                        // voxel keep their relative precision
                        sv[i] = ((wL * (p0 - pL) + wR * (p0 - pR)) + (wuu[i] * (p0 - puu[i]) + wy0[i] * (p0 - pdd[i]))) +
                                (wzm[i] * (p0 - pkm[i]) + wz0[i] * (p0 - pkn[i]));
                        const bool isfree = (g0[i] & 3u) == 1u && dv[i] > 0.0f;
                        un0[i] = isfree ? uu[i] - alpha * sv[i] * __fdividef(1.0f, dv[i]) : 0.0f;
                    }
                    sts4(eUN + bc * PL + wofs, un0[0], un0[1], un0[2], un0[3]);
                    eUF[bc * PS + sofs] = un0[0];
                    if (inner && z < z1) {
                        const int64_t pz = (int64_t)(z + 2) * plane;
                        const float4 xs = lds4(rX + slot(z) * L::NI + xofs);
                        stg4(Uo + pz, un0[0], un0[1], un0[2], un0[3]);
                        stg4(Po + pz, pk0[0], pk0[1], pk0[2], pk0[3]);
                        stg4(Xb + pz, fmaf(alpha, pk0[0], xs.x), fmaf(alpha, pk0[1], xs.y), fmaf(alpha, pk0[2], xs.z),
                             fmaf(alpha, pk0[3], xs.w));
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            // p_k and u' vanish on non-free voxels
                            const float du = dv[i] * un0[i];
                            a_gam = fmaf(du, un0[i], a_gam);
                            a_rr = fmaf(du, du, a_rr);
                            a_eps = fmaf(un0[i], sv[i], a_eps);
                            a_pi = fmaf(pk0[i], sv[i], a_pi);
                            a_tau = fmaf(du, pk0[i], a_tau);
                        }
                    }
                }

                // -- 3: delta over the edges owned by plane z-1 (+x, +y, +z)
                if (inner && z - 1 >= z0) {
                    const int bp = bn;  // (z - 1) & 1
                    const float ur = eUF[bp * PS + sofs + 1];
                    const float4 ud = lds4(eUN + bp * PL + wofs + WS);
                    const float4 um = lds4(eUN + bp * PL + wofs);
                    const float4 wxv = lds4(eWX4 + bp * PL + wofs);
                    const float4 wyv = lds4(eWY + bp * PL + wofs);
                    const float udd[4] = {ud.x, ud.y, ud.z, ud.w}, unm[4] = {um.x, um.y, um.z, um.w};
                    const float wxm[4] = {wxv.x, wxv.y, wxv.z, wxv.w}, wym[4] = {wyv.x, wyv.y, wyv.z, wyv.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float dx = unm[i] - (i < 3 ? unm[i + 1] : ur);
                        const float dy = unm[i] - udd[i];
                        const float dz = unm[i] - un0[i];
                        a_del = fmaf(wxm[i] * dx, dx, a_del);
                        a_del = fmaf(wym[i] * dy, dy, a_del);
                        a_del = fmaf(wzm[i] * dz, dz, a_del);
                    }
                }

                // -- 4: forward x / y weights of plane z+1 (into the slots plane
                // z-1 used: its last reader was step 3 of this thread)
                if (live) {
                    const uint32_t gr = has_right ? rG[sn * PL + wofs + 4] : 0u;
                    const uint4 gd = has_down ? lds4u(rG + sn * PL + wofs + WS) : make_uint4(0u, 0u, 0u, 0u);
                    const uint32_t gdd[4] = {gd.x, gd.y, gd.z, gd.w};
                    float wxn[4], wyn[4];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        wxn[i] = wgt(gn[i], i < 3 ? gn[i + 1] : gr, c2, wmin);
                        wyn[i] = wgt(gn[i], gdd[i], c2, wmin);
                    }
                    sts4(eWY + bn * PL + wofs, wyn[0], wyn[1], wyn[2], wyn[3]);
                    sts4(eWX4 + bn * PL + wofs, wxn[0], wxn[1], wxn[2], wxn[3]);
                    eWX[bn * PS + sofs] = wxn[3];
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    pkm[i] = pk0[i];
                    pk0[i] = pkn[i];
                    g0[i] = gn[i];
                    wzm[i] = wz0[i];
                }
            }
            cp_async_wait<0>();
        }
        const float fv[6] = {a_gam, a_rr, a_del, a_eps, a_pi, a_tau};
        double v[6];
        block_reduce_f32<NT, 6>(fv, v, red);
        if (tid == 0) {
            double* pp = A.partials + ((int64_t)li * tpb + t) * 6;
#pragma unroll
            for (int k = 0; k < 6; ++k) pp[k] = v[k];
            __threadfence();
            const unsigned prev = atomicAdd(&S->counter, 1u);
            s_last = (prev == (unsigned)tpb - 1u);
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            double tv[6] = {0, 0, 0, 0, 0, 0};
            const double* pb = A.partials + (int64_t)li * tpb * 6;
            for (int k = tid; k < tpb; k += NT)
#pragma unroll
                for (int j = 0; j < 6; ++j) tv[j] += __ldcg(pb + 6 * k + j);
            block_reduce<NT, 6>(tv, red);
            if (tid == 0) {
                S->counter = 0u;
                finalize_box(S, tv, A.n_active, A.parity ^ 1);
            }
        }
        __syncthreads();
    }
}

}  // namespace rwk
