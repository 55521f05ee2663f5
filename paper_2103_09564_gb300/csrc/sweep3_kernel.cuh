// FP32 fused PCG sweep, warp-row variant.
//
// Same iteration, operands and pipeline as k_sweep2 (sweep2_kernel.cuh), laid
// out so that one warp owns one 32-voxel row of the halo'd tile: the tile is
// 28 voxels wide plus a 2-voxel halo on each side, so lane = x position in the
// row.  In-row neighbours come from warp shuffles instead of shared memory,
// every per-row address is computed once per work item, the global offset of
// a plane is one pointer increment, and the preconditioner division uses the
// fast reciprocal.  Rows are dealt round-robin to the warps of the CTA.
#pragma once

#include "rw_internal.h"
#include "sweep2_kernel.cuh"

namespace rwk {

template <int TY, int D>
constexpr size_t sweep3_smem_bytes() {
    return (size_t)32 * (TY + 4) * 4 * (3 * (D + 2) + 14) + (size_t)28 * TY * 4 * (D + 2);
}

template <int TY, int NW, int D>
__global__ void __launch_bounds__(NW * 32, (65536 / (NW * 32 * 64)) > 1 ? (65536 / (NW * 32 * 64)) : 1)
    k_sweep3(const SweepArgs A) {
    constexpr int TX = 28, W2 = 32, H2 = TY + 4, R2 = W2 * H2, NI = TX * TY, NR = D + 2, NT = NW * 32;
    constexpr int RA = (H2 + NW - 1) / NW;        // rows of stage A per warp
    constexpr unsigned FULL = 0xffffffffu;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* rU = reinterpret_cast<float*>(smem_raw);
    float* rP = rU + NR * R2;
    uint32_t* rG = reinterpret_cast<uint32_t*>(rP + NR * R2);
    float* sP = reinterpret_cast<float*>(rG + NR * R2);
    float* sWx = sP + 3 * R2;
    float* sWy = sWx + 3 * R2;
    float* sWz = sWy + 3 * R2;
    float* sUn = sWz + 3 * R2;
    float* rX = sUn + 2 * R2;
    __shared__ double red[6 * NW];
    __shared__ int s_last;

    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, tid = threadIdx.x;
    const int tpb = A.ntx * A.nty * A.nzc;
    const int64_t nwork = (int64_t)(A.list ? *A.nlist : A.bx.nbox) * tpb;
    const int nx = A.bx.nx, ny = A.bx.ny, nz = A.bx.nz;
    const int64_t plane = (int64_t)nx * ny;
    const int64_t bstride = plane * nz;
    const float c2 = A.c2f, wmin = A.wminf;

    for (int64_t w = blockIdx.x; w < nwork; w += gridDim.x) {
        const int li = (int)(w / tpb);  // position in the list of active systems
        const int box = A.list ? A.list[li] : li;
        const int t = (int)(w - (int64_t)li * tpb);
        BoxScalars* S = A.sc + box;
        if (!S->active) continue;
        const int tx = t % A.ntx, ty = (t / A.ntx) % A.nty, tz = t / (A.ntx * A.nty);
        const float alpha = (float)S->alpha, bcg = (float)S->beta;
        const bool keep_p = S->phase == 2;
        int ex = nx, ey = ny, ez = nz;
        if (A.bx.ext) {
            ex = A.bx.ext[3 * box];
            ey = A.bx.ext[3 * box + 1];
            ez = A.bx.ext[3 * box + 2];
        }
        const int ox = tx * TX, oy = ty * TY, z0 = tz * A.zc;
        const int z1 = min(z0 + A.zc, ez);
        float a_gam = 0.f, a_rr = 0.f, a_del = 0.f, a_eps = 0.f, a_pi = 0.f, a_tau = 0.f;
        if (ox < ex && oy < ey && z0 < ez) {
            const int64_t base = (int64_t)box * bstride;
            const int gx = ox + lane - 2;
            const bool xin = gx >= 0 && gx < ex;
            const bool lane_int = lane >= 2 && lane < TX + 2 && gx < ex;  // interior column
            // per-row in-plane offsets and validity of this warp's stage-A rows
            int roff[RA];
            bool rok[RA];
#pragma unroll
            for (int k = 0; k < RA; ++k) {
                const int r = wid + k * NW;
                const int gy = oy + r - 2;
                roff[k] = gy * nx + gx;
                rok[k] = r < H2 && xin && gy >= 0 && gy < ey;
            }
            const float* Ub = static_cast<const float*>(A.u_in) + base;
            const float* Pb = static_cast<const float*>(A.p_in) + base;
            const uint32_t* Gb = A.gc + base;
            float* Xb = static_cast<float*>(A.x) + base;
            float* Uo = static_cast<float*>(A.u_out) + base;
            float* Po = static_cast<float*>(A.p_out) + base;

            auto issue = [&](int z) {
                const int slot = (z + 4 * NR) % NR;
                const bool zok = z >= 0 && z < ez;
                const int64_t pz = (int64_t)z * plane;
#pragma unroll
                for (int k = 0; k < RA; ++k) {
                    const int r = wid + k * NW;
                    if (r >= H2) break;
                    const int e = r * W2 + lane;
                    const bool ok = zok && rok[k];
                    const int64_t gi = ok ? pz + roff[k] : 0;
                    const int nb = ok ? 4 : 0;
                    cp_async4(rU + slot * R2 + e, Ub + gi, nb);
                    cp_async4(rP + slot * R2 + e, Pb + gi, nb);
                    cp_async4(rG + slot * R2 + e, Gb + gi, nb);
                    if (z >= z0 && z < z1 && r >= 2 && r < TY + 2 && lane_int && oy + r - 2 < ey)
                        cp_async4(rX + slot * NI + (r - 2) * TX + (lane - 2), Xb + pz + roff[k], 4);
                }
            };

#pragma unroll
            for (int d = 0; d < D; ++d) {
                if (z0 - 2 + d <= z1) issue(z0 - 2 + d);
                cp_async_commit();
            }
            for (int zf = z0 - 2; zf <= z1 + 1; ++zf) {
                cp_async_wait<D - 1>();
                __syncthreads();
                if (zf + D <= z1) issue(zf + D);
                cp_async_commit();
                // -- C: delta over the owned edges of plane zc = zf-2
                const int zc = zf - 2;
                if (zc >= z0 && zc < z1) {
                    const float* U0 = sUn + (zc & 1) * R2;
                    const float* Ul = sUn + ((zc + 1) & 1) * R2;
                    const int c3 = (zc + 6) % 3;
                    const float* Wx = sWx + c3 * R2;
                    const float* Wy = sWy + c3 * R2;
                    const float* Wz = sWz + c3 * R2;
                    for (int r = 2 + wid; r < TY + 2; r += NW) {
                        const int e = r * W2 + lane;
                        const float u0 = U0[e];
                        const float ur = __shfl_down_sync(FULL, u0, 1);
                        if (lane_int && oy + r - 2 < ey) {
                            const float dx = u0 - ur, dy = u0 - U0[e + W2], dz = u0 - Ul[e];
                            a_del += Wx[e] * dx * dx + Wy[e] * dy * dy + Wz[e] * dz * dz;
                        }
                    }
                }
                // -- A: p_k and forward edge weights on plane zf
                if (zf <= z1) {
                    const int s = (zf + 4 * NR) % NR, sp = (zf - 1 + 4 * NR) % NR;
                    const int f3 = (zf + 6) % 3;
                    const float* U = rU + s * R2;
                    const float* Pm = rP + s * R2;
                    const uint32_t* G = rG + s * R2;
                    const uint32_t* Gp = rG + sp * R2;
                    const bool zedge = zf > z0 - 2;
#pragma unroll
                    for (int k = 0; k < RA; ++k) {
                        const int r = wid + k * NW;
                        if (r >= H2) break;
                        const int e = r * W2 + lane;
                        const uint32_t g0 = G[e];
                        const uint32_t gr = __shfl_down_sync(FULL, g0, 1);
                        const uint32_t gd = (r + 1 < H2) ? G[e + W2] : 0u;
                        sP[f3 * R2 + e] = keep_p ? Pm[e] : (((g0 & 3u) == 1u) ? U[e] + bcg * Pm[e] : 0.0f);
                        sWx[f3 * R2 + e] = lane < 31 ? w_of(g0, gr, c2, wmin) : 0.0f;
                        sWy[f3 * R2 + e] = w_of(g0, gd, c2, wmin);
                        sWz[f3 * R2 + e] = zedge ? w_of(Gp[e], g0, c2, wmin) : 0.0f;
                    }
                }
                __syncthreads();
                // -- B: plane zm = zf-1 on the halo-1 region (rows 1..H2-2)
                const int zm = zf - 1;
                if (zm >= z0 - 1 && zm < z1) {
                    const int s = (zm + 4 * NR) % NR;
                    const int m3 = (zm + 6) % 3, l3 = (zm + 5) % 3, h3 = (zm + 7) % 3;
                    const float* P = sP + m3 * R2;
                    const float* Pl = sP + l3 * R2;
                    const float* Ph = sP + h3 * R2;
                    const float* Wx = sWx + m3 * R2;
                    const float* Wy = sWy + m3 * R2;
                    const float* Wzl = sWz + m3 * R2;
                    const float* Wzh = sWz + h3 * R2;
                    const uint32_t* G = rG + s * R2;
                    const float* U = rU + s * R2;
                    float* Un = sUn + (zm & 1) * R2;
                    const bool out = zm >= z0;
                    const int64_t pz = (int64_t)zm * plane;
                    for (int r = 1 + wid; r < H2 - 1; r += NW) {
                        const int e = r * W2 + lane;
                        const float p0 = P[e];
                        const float pxl = __shfl_up_sync(FULL, p0, 1);
                        const float pxr = __shfl_down_sync(FULL, p0, 1);
                        const float wxp = Wx[e];
                        const float wxm = __shfl_up_sync(FULL, wxp, 1);
                        const uint32_t g = G[e];
                        float un = 0.0f, d = 0.0f, sv = 0.0f;
                        const bool fr = (g & 3u) == 1u && lane >= 1 && lane < 31;
                        if (fr) {
                            const float wym = Wy[e - W2], wyp = Wy[e], wzm = Wzl[e], wzp = Wzh[e];
                            d = ((wxm + wxp) + (wym + wyp)) + (wzm + wzp);
                            // difference form (see k_sweep)
                            sv = ((wxm * (p0 - pxl) + wxp * (p0 - pxr)) + (wym * (p0 - P[e - W2]) + wyp * (p0 - P[e + W2]))) +
                                 (wzm * (p0 - Pl[e]) + wzp * (p0 - Ph[e]));
                            if (d > 0.0f) un = U[e] - alpha * __fdividef(sv, d);
                        }
                        Un[e] = un;
                        if (out && r >= 2 && r < TY + 2 && lane_int && oy + r - 2 < ey) {
                            const int64_t gi = pz + (int64_t)(oy + r - 2) * nx + gx;
                            Uo[gi] = un;
                            Po[gi] = p0;
                            if (fr) {
                                Xb[gi] = rX[s * NI + (r - 2) * TX + (lane - 2)] + alpha * p0;
                                const float du = d * un;
                                a_gam += du * un;
                                a_rr += du * du;
                                a_eps += un * sv;
                                a_pi += p0 * sv;
                                a_tau += du * p0;
                            }
                        }
                    }
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
