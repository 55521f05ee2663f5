// FP32 fused PCG sweep with an asynchronous plane pipeline.
//
// Same iteration as k_sweep (sweep_kernel.cuh: single-reduction Jacobi-PCG,
// u = D^-1 r stored, weights recomputed from g), organised for latency
// hiding and a low instruction count:
//
// * g and the seed code travel together in one 32-bit word: the FP32
//   intensity with its two low mantissa bits replaced by the code
//   (0 absent, 1 free, 2 seed; the g perturbation is below 3 ulp and the
//   FP64 residual rounds use the exact g).  Every operand is then a 4-byte
//   cp.async into shared memory, issued D planes ahead; halo voxels outside
//   the box are zero-filled by the copy (src-size 0), which reads as
//   "absent": no bounds branches in the arithmetic.
// * The three inner products of an iteration: gamma = sum d u^2 and
//   rr = sum (d u)^2 per voxel, and delta = u^T A u summed edge-wise,
//   delta = sum over edges of w (u_p - u_q)^2 with u = 0 on seeds and absent
//   voxels (the Dirichlet-energy identity of Sec. III-B), each edge owned by
//   one interior voxel (its +x, +y and -z edges).
// * Per z-plane step of the front zf: wait for plane zf, one barrier,
//   then [delta on plane zf-2] + [p_k and forward weights on plane zf],
//   a second barrier, then [s = A p_k, u_k+1, x, outputs on plane zf-1].
#pragma once

#include "rw_internal.h"
#include "sweep_kernel.cuh"

namespace rwk {

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem, int src_bytes) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

__device__ __forceinline__ float w_of(uint32_t a, uint32_t b, float c2, float wmin) {
    // both endpoints present (code != 0): max(exp(-beta d^2), w_min); else 0
    if (!((a & 3u) && (b & 3u))) return 0.0f;
    const float d = __uint_as_float(a & ~3u) - __uint_as_float(b & ~3u);
    return fmaxf(ex2_approx(c2 * d * d), wmin);
}

template <int TX, int TY, int D>
constexpr size_t sweep2_smem_bytes() {
    return (size_t)(TX + 4) * (TY + 4) * 4 * (3 * (D + 2) + 14) + (size_t)TX * TY * 4 * (D + 2);
}

// at most 64 registers per thread where that lets two or more CTAs share an SM
template <int NT>
constexpr int sweep2_min_blocks() {
    return (65536 / (NT * 64)) > 1 ? (65536 / (NT * 64)) : 1;
}

template <int TX, int TY, int NT, int D>
__global__ void __launch_bounds__(NT, sweep2_min_blocks<NT>()) k_sweep2(const SweepArgs A) {
    constexpr int W2 = TX + 4, H2 = TY + 4, R2 = W2 * H2;
    constexpr int W1 = TX + 2, H1 = TY + 2, R1 = W1 * H1;
    constexpr int NI = TX * TY, NR = D + 2;
    constexpr int JA = (R2 + NT - 1) / NT, JB = (R1 + NT - 1) / NT, JC = (NI + NT - 1) / NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* rU = reinterpret_cast<float*>(smem_raw);           // [NR][R2] u_k
    float* rP = rU + NR * R2;                                  // [NR][R2] p_k-1
    uint32_t* rG = reinterpret_cast<uint32_t*>(rP + NR * R2);  // [NR][R2] packed g|code
    float* sP = reinterpret_cast<float*>(rG + NR * R2);       // [3][R2] p_k
    float* sWx = sP + 3 * R2;                                   // [3][R2] w(i, i+x)
    float* sWy = sWx + 3 * R2;                                  // [3][R2] w(i, i+y)
    float* sWz = sWy + 3 * R2;                                  // [3][R2] w(i-z, i)
    float* sUn = sWz + 3 * R2;                                  // [2][R2] u_k+1
    float* rX = sUn + 2 * R2;                                   // [NR][NI] x (delta)
    __shared__ double red[6 * (NT / 32)];
    __shared__ int s_last;

    const int tid = threadIdx.x;
    const int tpb = A.ntx * A.nty * A.nzc;
    const int64_t nwork = (int64_t)(A.list ? *A.nlist : A.bx.nbox) * tpb;
    const int nx = A.bx.nx, ny = A.bx.ny, nz = A.bx.nz;
    const int64_t plane = (int64_t)nx * ny;
    const int64_t bstride = plane * nz;
    const uint32_t* __restrict__ GC = A.gc;
    float* __restrict__ X = static_cast<float*>(A.x);
    const float* __restrict__ Uin = static_cast<const float*>(A.u_in);
    const float* __restrict__ Pin = static_cast<const float*>(A.p_in);
    float* __restrict__ Uout = static_cast<float*>(A.u_out);
    float* __restrict__ Pout = static_cast<float*>(A.p_out);
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
            // per-item element tables: A over R2, B over R1, C over the interior
            int aoff[JA], aflag[JA];
#pragma unroll
            for (int j = 0; j < JA; ++j) {
                const int e = tid + j * NT;
                const int ix = e % W2, iy = e / W2;
                const int gx = ox + ix - 2, gy = oy + iy - 2;
                aoff[j] = gy * nx + gx;
                int f = 0;
                if (e < R2) {
                    f |= 16;
                    if (gx >= 0 && gx < ex && gy >= 0 && gy < ey) f |= 1;
                    if (ix + 1 < W2) f |= 2;
                    if (iy + 1 < H2) f |= 4;
                    if (ix >= 1 && ix < W2 - 1 && iy >= 1 && iy < H2 - 1) f |= 8;
                }
                aflag[j] = f;
            }
            int be[JB], bi[JB], boff[JB];
#pragma unroll
            for (int j = 0; j < JB; ++j) {
                const int e1 = tid + j * NT;
                const int jx = e1 % W1 + 1, jy = e1 / W1 + 1;
                be[j] = (e1 < R1) ? jy * W2 + jx : -1;
                const int gx = ox + jx - 2, gy = oy + jy - 2;
                const bool inter = e1 < R1 && jx >= 2 && jx < TX + 2 && jy >= 2 && jy < TY + 2 && gx < ex && gy < ey;
                bi[j] = inter ? (jy - 2) * TX + (jx - 2) : -1;
                boff[j] = gy * nx + gx;
            }
            int ce[JC], coff[JC];
#pragma unroll
            for (int j = 0; j < JC; ++j) {
                const int e0 = tid + j * NT;
                const int jx = e0 % TX, jy = e0 / TX;
                const bool ok = e0 < NI && ox + jx < ex && oy + jy < ey;
                ce[j] = ok ? (jy + 2) * W2 + (jx + 2) : -1;
                coff[j] = (oy + jy) * nx + (ox + jx);
            }

            auto issue = [&](int z) {
                const int slot = (z + 4 * NR) % NR;
                const bool zok = z >= 0 && z < ez;
                const int64_t pb = base + (int64_t)z * plane;
#pragma unroll
                for (int j = 0; j < JA; ++j) {
                    if (!(aflag[j] & 16)) continue;
                    const int e = tid + j * NT;
                    const bool ok = zok && (aflag[j] & 1);
                    const int64_t gi = ok ? pb + aoff[j] : 0;
                    const int nb = ok ? 4 : 0;
                    cp_async4(rU + slot * R2 + e, Uin + gi, nb);
                    cp_async4(rP + slot * R2 + e, Pin + gi, nb);
                    cp_async4(rG + slot * R2 + e, GC + gi, nb);
                }
                if (z >= z0 && z < z1) {
#pragma unroll
                    for (int j = 0; j < JC; ++j) {
                        if (ce[j] < 0) continue;
                        cp_async4(rX + slot * NI + tid + j * NT, X + pb + coff[j], 4);
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
                // -- C: delta over the owned edges of plane zc = zf-2
                const int zc = zf - 2;
                if (zc >= z0 && zc < z1) {
                    const float* U0 = sUn + (zc & 1) * R2;
                    const float* Ul = sUn + ((zc + 1) & 1) * R2;
                    const int c3 = (zc + 6) % 3;
                    const float* Wx = sWx + c3 * R2;
                    const float* Wy = sWy + c3 * R2;
                    const float* Wz = sWz + c3 * R2;
#pragma unroll
                    for (int j = 0; j < JC; ++j) {
                        const int e = ce[j];
                        if (e < 0) continue;
                        const float u0 = U0[e];
                        const float dx = u0 - U0[e + 1], dy = u0 - U0[e + W2], dz = u0 - Ul[e];
                        a_del += Wx[e] * dx * dx + Wy[e] * dy * dy + Wz[e] * dz * dz;
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
                    for (int j = 0; j < JA; ++j) {
                        const int f = aflag[j];
                        if (!(f & 16)) continue;
                        const int e = tid + j * NT;
                        const uint32_t g0 = G[e];
                        sP[f3 * R2 + e] = keep_p ? Pm[e] : (((g0 & 3u) == 1u) ? U[e] + bcg * Pm[e] : 0.0f);
                        sWx[f3 * R2 + e] = (f & 2) ? w_of(g0, G[e + 1], c2, wmin) : 0.0f;
                        sWy[f3 * R2 + e] = (f & 4) ? w_of(g0, G[e + W2], c2, wmin) : 0.0f;
                        sWz[f3 * R2 + e] = (zedge && (f & 8)) ? w_of(Gp[e], g0, c2, wmin) : 0.0f;
                    }
                }
                __syncthreads();
                // -- B: plane zm = zf-1 on the halo-1 region
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
                    const int64_t pb = base + (int64_t)zm * plane;
#pragma unroll
                    for (int j = 0; j < JB; ++j) {
                        const int e = be[j];
                        if (e < 0) continue;
                        const float p0 = P[e];
                        float un = 0.0f, d = 0.0f, sv = 0.0f;
                        if ((G[e] & 3u) == 1u) {
                            const float wxm = Wx[e - 1], wxp = Wx[e], wym = Wy[e - W2], wyp = Wy[e], wzm = Wzl[e],
                                        wzp = Wzh[e];
                            d = ((wxm + wxp) + (wym + wyp)) + (wzm + wzp);
                            // difference form (see k_sweep)
                            sv = ((wxm * (p0 - P[e - 1]) + wxp * (p0 - P[e + 1])) +
                                  (wym * (p0 - P[e - W2]) + wyp * (p0 - P[e + W2]))) +
                                 (wzm * (p0 - Pl[e]) + wzp * (p0 - Ph[e]));
                            if (d > 0.0f) un = U[e] - alpha * sv / d;
                        }
                        Un[e] = un;
                        if (out && bi[j] >= 0) {
                            const int64_t gi = pb + boff[j];
                            Uout[gi] = un;
                            Pout[gi] = p0;
                            if ((G[e] & 3u) == 1u) {
                                X[gi] = rX[s * NI + bi[j]] + alpha * p0;
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
