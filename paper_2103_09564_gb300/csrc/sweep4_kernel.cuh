// FP32 fused PCG sweep on a padded layout.
//
// Same iteration as k_sweep2 (single-reduction Jacobi-PCG with explicit
// A-conjugation, u = D^-1 r stored, weights recomputed from g, six inner
// products per sweep), with the integer work taken out of the hot loop:
//
// * The vectors the sweep streams (u, p, delta and the packed g|code words)
//   live in a padded layout: every box is stored as [PZ][PY][PX] with a margin
//   of absent voxels (code 0, all values 0) of two voxels in front of x, y and
//   z and at least two behind, and PX, PY cover whole tiles.  Tile loads and
//   stores therefore never leave the array and need no bounds checks: the
//   margins read as absent voxels, which have no edges.
// * A tile row of TX + 4 words starts 16-byte aligned, so each row is copied
//   with 16-byte cp.async (4 voxels per instruction), D planes ahead.
// * The code of a voxel (0 absent, 1 free, 2 seed) enters the arithmetic as
//   0/1 factors instead of branches; ring slots are powers of two; the
//   per-thread shared-memory offsets do not depend on the tile and are set up
//   once per CTA.
#pragma once

#include "rw_internal.h"
#include "sweep2_kernel.cuh"

namespace rwk {

__device__ __forceinline__ void cp_async16(uint32_t saddr, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(uint32_t saddr, const void* gmem) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(saddr), "l"(gmem) : "memory");
}

template <int TX, int TY, int NR>
constexpr size_t sweep4_smem_bytes() {
    // raw u, p, g|code: NR slots; p_k and three weight planes: 4 slots;
    // u_k+1: 2 slots (all R2 words); delta of the interior: NR slots
    return (size_t)(TX + 4) * (TY + 4) * 4 * (3 * NR + 4 * 4 + 2) + (size_t)TX * TY * 4 * NR;
}

__device__ __forceinline__ float wgt(uint32_t a, uint32_t b, float c2, float wmin) {
    const float d = __uint_as_float(a & ~3u) - __uint_as_float(b & ~3u);
    const float w = fmaxf(ex2_approx(c2 * d * d), wmin);
    return ((a & 3u) && (b & 3u)) ? w : 0.0f;
}

template <int TX, int TY, int NT, int D, int NR>
__global__ void __launch_bounds__(NT, (65536 / (NT * 64)) > 1 ? (65536 / (NT * 64)) : 1)
    k_sweep4(const SweepArgs A) {
    static_assert((NR & (NR - 1)) == 0 && NR >= D + 2, "ring size");
    static_assert(TX % 4 == 0, "tile width");
    constexpr int W2 = TX + 4, H2 = TY + 4, R2 = W2 * H2, Q2 = R2 / 4, QW = W2 / 4;
    constexpr int W1 = TX + 2, H1 = TY + 2, R1 = W1 * H1, NI = TX * TY, NIH = NI / 2;
    constexpr int JA = (R2 + NT - 1) / NT, JB = (R1 + NT - 1) / NT, JC = (NI + NT - 1) / NT;
    constexpr int JQ = (Q2 + NT - 1) / NT, JX = (NIH + NT - 1) / NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* rU = reinterpret_cast<float*>(smem_raw);            // [NR][R2]
    float* rP = rU + NR * R2;                                   // [NR][R2]
    uint32_t* rG = reinterpret_cast<uint32_t*>(rP + NR * R2);  // [NR][R2]
    float* sP = reinterpret_cast<float*>(rG + NR * R2);        // [4][R2]
    float* sWx = sP + 4 * R2;                                   // [4][R2]
    float* sWy = sWx + 4 * R2;
    float* sWz = sWy + 4 * R2;
    float* sUn = sWz + 4 * R2;                                  // [2][R2]
    float* rX = sUn + 2 * R2;                                   // [NR][NI]
    __shared__ double red[6 * (NT / 32)];
    __shared__ int s_last;

    const int tid = threadIdx.x;
    const int tpb = A.ntx * A.nty * A.nzc;
    const int64_t nwork = (int64_t)(A.list ? *A.nlist : A.bx.nbox) * tpb;
    const int PX = A.px, PY = A.py;
    const int64_t plane = (int64_t)PX * PY;
    const int64_t bstride = plane * A.pz;
    const float c2 = A.c2f, wmin = A.wminf;
    const uint32_t s_base = (uint32_t)__cvta_generic_to_shared(smem_raw);

    // tile-independent element tables
    int qrow[JQ], qcol[JQ];  // load quads: row in the tile, word column
#pragma unroll
    for (int j = 0; j < JQ; ++j) {
        const int q = tid + j * NT;
        qrow[j] = q < Q2 ? q / QW : -1;
        qcol[j] = (q % QW) * 4;
    }
    int xrow[JX], xcol[JX];  // delta pairs of the interior
#pragma unroll
    for (int j = 0; j < JX; ++j) {
        const int h = tid + j * NT;
        xrow[j] = h < NIH ? h / (TX / 2) : -1;
        xcol[j] = (h % (TX / 2)) * 2;
    }
    int bE[JB], bI[JB];  // stage B element (R2 index) and interior index (or -1)
#pragma unroll
    for (int j = 0; j < JB; ++j) {
        const int e1 = tid + j * NT;
        const int jx = e1 % W1 + 1, jy = e1 / W1 + 1;
        bE[j] = e1 < R1 ? jy * W2 + jx : -1;
        bI[j] = (e1 < R1 && jx >= 2 && jx < TX + 2 && jy >= 2 && jy < TY + 2) ? (jy - 2) * TX + (jx - 2) : -1;
    }
    int cE[JC];
#pragma unroll
    for (int j = 0; j < JC; ++j) {
        const int e0 = tid + j * NT;
        cE[j] = e0 < NI ? (e0 / TX + 2) * W2 + (e0 % TX + 2) : -1;
    }
    int aF[JA];  // stage A element flags: 1 has a +x neighbour, 2 has a +y neighbour
#pragma unroll
    for (int j = 0; j < JA; ++j) {
        const int e = tid + j * NT;
        aF[j] = ((e % W2) != W2 - 1 ? 1 : 0) | (e < R2 - W2 ? 2 : 0);
    }

    for (int64_t w = blockIdx.x; w < nwork; w += gridDim.x) {
        const int li = (int)(w / tpb);  // position in the list of active systems
        const int box = A.list ? A.list[li] : li;
        const int t = (int)(w - (int64_t)li * tpb);
        BoxScalars* S = A.sc + box;
        if (!S->active) continue;
        const int tx = t % A.ntx, ty = (t / A.ntx) % A.nty, tz = t / (A.ntx * A.nty);
        const float alpha = (float)S->alpha, bcg = (float)S->beta;
        const float keep = S->phase == 2 ? 1.0f : 0.0f;
        int ez = A.bx.nz;
        if (A.bx.ext) ez = A.bx.ext[3 * box + 2];
        const int z0 = tz * A.zc;
        const int z1 = min(z0 + A.zc, ez);
        float a_gam = 0.f, a_rr = 0.f, a_del = 0.f, a_eps = 0.f, a_pi = 0.f, a_tau = 0.f;
        if (z0 < ez) {
            // padded coordinates: the tile's halo row starts at x = tx * TX,
            // y = ty * TY (user x - 2, y - 2); plane z sits at z + 2
            const int64_t base = (int64_t)box * bstride;
            const int ox = tx * TX, oy = ty * TY;
            const float* Ub = static_cast<const float*>(A.u_in) + base;
            const float* Pb = static_cast<const float*>(A.p_in) + base;
            const uint32_t* Gb = A.gc + base;
            float* Xb = static_cast<float*>(A.x) + base;
            float* Uo = static_cast<float*>(A.u_out) + base;
            float* Po = static_cast<float*>(A.p_out) + base;
            int qoff[JQ], xoff[JX], boff[JB];
#pragma unroll
            for (int j = 0; j < JQ; ++j) qoff[j] = (oy + qrow[j]) * PX + ox + qcol[j];
#pragma unroll
            for (int j = 0; j < JB; ++j) boff[j] = bI[j] >= 0 ? (oy + 2 + bI[j] / TX) * PX + ox + 2 + bI[j] % TX : 0;
#pragma unroll
            for (int j = 0; j < JX; ++j) xoff[j] = (oy + 2 + xrow[j]) * PX + ox + 2 + xcol[j];

            auto issue = [&](int z) {
                const int slot = z & (NR - 1);
                const int64_t pz = (int64_t)(z + 2) * plane;
#pragma unroll
                for (int j = 0; j < JQ; ++j) {
                    if (qrow[j] < 0) continue;
                    const int64_t gi = pz + qoff[j];
                    const uint32_t so = (uint32_t)((slot * R2 + qrow[j] * W2 + qcol[j]) * 4);
                    cp_async16(s_base + so, Ub + gi);
                    cp_async16(s_base + (uint32_t)(NR * R2 * 4) + so, Pb + gi);
                    cp_async16(s_base + (uint32_t)(2 * NR * R2 * 4) + so, Gb + gi);
                }
                if (z >= z0 && z < z1) {
                    const uint32_t xb = (uint32_t)((3 * NR * R2 + 4 * 4 * R2 + 2 * R2 + slot * NI) * 4);
#pragma unroll
                    for (int j = 0; j < JX; ++j) {
                        if (xrow[j] < 0) continue;
                        cp_async8(s_base + xb + (uint32_t)((xrow[j] * TX + xcol[j]) * 4), Xb + pz + xoff[j]);
                    }
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
                // -- C: delta over the owned edges (+x, +y, -z) of plane zf-2
                const int zc = zf - 2;
                if (zc >= z0 && zc < z1) {
                    const float* U0 = sUn + (zc & 1) * R2;
                    const float* Ul = sUn + ((zc + 1) & 1) * R2;
                    const int c4 = (zc & 3) * R2;
#pragma unroll
                    for (int j = 0; j < JC; ++j) {
                        const int e = cE[j];
                        if (e < 0) continue;
                        const float u0 = U0[e];
                        const float dx = u0 - U0[e + 1], dy = u0 - U0[e + W2], dz = u0 - Ul[e];
                        a_del += sWx[c4 + e] * dx * dx + sWy[c4 + e] * dy * dy + sWz[c4 + e] * dz * dz;
                    }
                }
                // -- A: p_k and the forward edge weights of plane zf
                if (zf <= z1) {
                    const int s = (zf & (NR - 1)) * R2, sp = ((zf - 1) & (NR - 1)) * R2;
                    const int f4 = (zf & 3) * R2;
                    const bool zedge = zf > z0 - 2;
#pragma unroll
                    for (int j = 0; j < JA; ++j) {
                        const int e = tid + j * NT;
                        if (e >= R2) continue;
                        const uint32_t g0 = rG[s + e];
                        const float fr = (g0 & 3u) == 1u ? 1.0f : 0.0f;
                        const float pm = rP[s + e];
                        sP[f4 + e] = keep * pm + (1.0f - keep) * fr * (rU[s + e] + bcg * pm);
                        // the last column / row has no forward edge inside the tile
                        const uint32_t gr = (aF[j] & 1) ? rG[s + e + 1] : 0u;
                        const uint32_t gd = (aF[j] & 2) ? rG[s + e + W2] : 0u;
                        sWx[f4 + e] = wgt(g0, gr, c2, wmin);
                        sWy[f4 + e] = wgt(g0, gd, c2, wmin);
                        sWz[f4 + e] = zedge ? wgt(rG[sp + e], g0, c2, wmin) : 0.0f;
                    }
                }
                __syncthreads();
                // -- B: plane zm = zf-1 on the halo-1 region
                const int zm = zf - 1;
                if (zm >= z0 - 1 && zm < z1) {
                    const int s = (zm & (NR - 1)) * R2;
                    const int m4 = (zm & 3) * R2, l4 = ((zm - 1) & 3) * R2, h4 = ((zm + 1) & 3) * R2;
                    float* Un = sUn + (zm & 1) * R2;
                    const bool out = zm >= z0;
                    const int64_t pz = (int64_t)(zm + 2) * plane;
                    const float* xs = rX + (zm & (NR - 1)) * NI;
#pragma unroll
                    for (int j = 0; j < JB; ++j) {
                        const int e = bE[j];
                        if (e < 0) continue;
                        const float p0 = sP[m4 + e];
                        const float wxm = sWx[m4 + e - 1], wxp = sWx[m4 + e], wym = sWy[m4 + e - W2],
                                    wyp = sWy[m4 + e], wzm = sWz[m4 + e], wzp = sWz[h4 + e];
                        const float d = ((wxm + wxp) + (wym + wyp)) + (wzm + wzp);
                        // difference form (see k_sweep): the weak edges of a
                        // strongly linked voxel keep their relative precision
                        const float sv = ((wxm * (p0 - sP[m4 + e - 1]) + wxp * (p0 - sP[m4 + e + 1])) +
                                          (wym * (p0 - sP[m4 + e - W2]) + wyp * (p0 - sP[m4 + e + W2]))) +
                                         (wzm * (p0 - sP[l4 + e]) + wzp * (p0 - sP[h4 + e]));
                        const bool isfree = (rG[s + e] & 3u) == 1u && d > 0.0f;
                        const float fr = isfree ? 1.0f : 0.0f;
                        const float inv = isfree ? __fdividef(1.0f, d) : 0.0f;
                        const float un = fr * (rU[s + e] - alpha * sv * inv);
                        Un[e] = un;
                        const int ii = bI[j];
                        if (out && ii >= 0) {
                            const int64_t gi = pz + boff[j];
                            Uo[gi] = un;
                            Po[gi] = p0;
                            Xb[gi] = xs[ii] + alpha * fr * p0;
                            const float du = d * un;
                            a_gam += du * un;
                            a_rr += du * du;
                            a_eps += un * sv * fr;
                            a_pi += p0 * sv * fr;
                            a_tau += du * p0;
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
