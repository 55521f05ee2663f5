// Cluster-resident PCG for small systems (brick neighbourhoods of up to 40
// voxels per axis, the root of a brick-32 pyramid): one thread-block cluster
// per system keeps the whole FP32 state on chip across iterations.
//
// The batched sweeps stream every system through HBM / L2 once per iteration;
// when only a few systems are left (the slow bricks of a level, the small
// coarse levels), an iteration costs the latency of its loads, of the
// two-stage reduction and of a grid-wide synchronisation, about ten
// microseconds, whatever the size.  Here the z planes of a system are split
// over the CL CTAs of a cluster (CL = 16, non-portable cluster size, one CTA
// per SM): every CTA holds u, p_k, the correction delta, the diagonal and the
// three forward edge weights of its planes in shared memory (the weights and
// the diagonal are computed once per launch, g does not change), the boundary
// planes of p_k and u' move to the neighbouring CTAs through distributed
// shared memory, the six inner products of a sweep are summed per CTA and
// broadcast to every CTA of the cluster, and hardware cluster barriers
// separate the phases.  Every CTA then runs the same scalar recurrences on
// the same sums in the same order, so all of them take the same exit.
//
// One iteration is the sweep of the strip kernels (same recurrences,
// single-reduction PCG with u = D^-1 r stored, difference-form stencil, FP32
// per-thread partial sums, double-FP32 block and cluster sums and scalar
// recurrences): p_k = ku u + bp p,
// s = A p_k, u' = u - alpha D^-1 s (free voxels), delta += alpha p_k, and
// gamma, ||D u'||^2, u'^T A u', (u', s), (p_k, s), (D u', p_k).  A launch runs
// up to `loop_iters` iterations of each system; the state is read from and
// written back to the padded global arrays of the system's current buffer
// parity (BoxScalars::par, unchanged), so the batched driver continues from
// it (refinement rounds, FP64 residual).  Clusters never wait on each other:
// each one takes systems of the list in turn.
#include "sweep5_kernel.cuh"

namespace rwk {

namespace {

constexpr int kClNT = 512;

__device__ __forceinline__ uint32_t cl_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cl_size() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cl_id() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cl_count() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}
// Cluster-wide barrier: shared-memory writes (local and remote) before it are
// visible to every CTA of the cluster after it.
__device__ __forceinline__ void cl_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n"
                 "barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}
// Address of the same shared-memory location in CTA `rank` of the cluster.
__device__ __forceinline__ uint32_t cl_map(uint32_t saddr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(saddr), "r"(rank));
    return r;
}
__device__ __forceinline__ void cl_st4(uint32_t addr, float4 v) {
    asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w)
                 : "memory");
}
__device__ __forceinline__ void cl_st2(uint32_t addr, float a, float b) {
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(addr), "f"(a), "f"(b) : "memory");
}

// Copy one plane (pls floats, a multiple of 4) to the same place in CTA `rank`.
__device__ __forceinline__ void plane_to(const float* src, const float* dst_local, uint32_t rank, int pls) {
    const uint32_t dst = cl_map((uint32_t)__cvta_generic_to_shared(dst_local), rank);
    const float4* s4 = reinterpret_cast<const float4*>(src);
    for (int q = threadIdx.x; q < pls / 4; q += kClNT) cl_st4(dst + 16u * (uint32_t)q, s4[q]);
}

// The scalar state of a system during a launch (the FP64 fields of its
// BoxScalars record as double-FP32 numbers).
struct ClState {
    DF gam, alpha, beta, rr, tol2;
    int iters, max_iter, phase, active, status;
};

}  // namespace

__global__ void __launch_bounds__(kClNT, 1) k_brick_cluster(const __grid_constant__ ClusterArgs A) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ BoxScalars S;
    __shared__ ClState T;
    __shared__ DF wsum[6][kClNT / 32];

    const int tid = threadIdx.x;
    const int NX = A.nx, NY = A.ny, NZ = A.nz;
    const int PLS = A.pls, NZL = A.nzl;
    const uint32_t rank = cl_rank(), CL = cl_size();
    const int z0 = (int)((rank * (uint32_t)NZ) / CL), z1 = (int)(((rank + 1) * (uint32_t)NZ) / CL);
    const int nzl = z1 - z0;
    float* U = reinterpret_cast<float*>(smem_raw);  // [NZL][PLS]: u, then u'
    float* Pk = U + NZL * PLS;                       // p, then p_k
    float* X = Pk + NZL * PLS;                       // correction delta
    float* Dg = X + NZL * PLS;                       // diagonal (0 on voxels that are not free)
    float* WX = Dg + NZL * PLS;                      // forward weights (i, i+x), (i, i+y), (i, i+z)
    float* WY = WX + NZL * PLS;
    float* WZ = WY + NZL * PLS;
    float* WZB = WZ + NZL * PLS;                     // [PLS] weight (z0-1, z0)
    float* PKB = WZB + PLS;                          // p_k of plane z0-1
    float* PKA = PKB + PLS;                          // p_k of plane z1
    float* UA = PKA + PLS;                           // u' of plane z1
    DF* part = reinterpret_cast<DF*>(UA + PLS);      // [CL][6] every CTA's sums
    const uint32_t part_s = (uint32_t)__cvta_generic_to_shared(part);

    const int64_t plane_g = (int64_t)A.px * A.py;
    const int64_t bstride = plane_g * A.pz;
    const int nlist = A.list ? *A.nlist : A.nbox;
    // voxel loops run over rows (plane, y) of the own planes: thread tid owns
    // column x = tid % NX of rows tid / NX, tid / NX + RPI, ... (no division
    // per voxel; threads beyond RPI * NX idle in the loops)
    const int RPI = kClNT / NX;
    const int tx = tid % NX, trow = tid / NX;
    const bool tlive = trow < RPI;
    const int nrows = nzl * NY;

    for (int li = (int)cl_id(); li < nlist; li += (int)cl_count()) {
        const int box = A.list ? A.list[li] : li;
        BoxScalars* Sg = A.sc + box;
        __syncthreads();  // every thread is done with the previous record
        if (tid == 0) scalars_load_cg(Sg, &S);
        __syncthreads();
        if (!S.active) continue;  // the same record in every CTA: a uniform skip
        if (tid == 0) {
            T.gam = df_of(S.gam);
            T.alpha = df_of(S.alpha);
            T.beta = df_of(S.beta);
            T.rr = df_of(S.rr);
            T.tol2 = df_of(S.tol2);
            T.iters = S.iters;
            T.max_iter = S.max_iter;
            T.phase = S.phase;
            T.active = S.active;
            T.status = S.status;
        }
        const int par = S.par;
        float* ug = A.u[par];
        float* pg = A.p[par];
        float* xg = A.x;
        const uint32_t* gg = A.gc;
        const int64_t gbase = (int64_t)box * bstride;

        // state of the own planes; weights and diagonal from the g words
        for (int row = tlive ? trow : nrows, lz = row / NY, y = row - lz * NY; row < nrows;
             row += RPI, y += RPI) {
            while (y >= NY) y -= NY, ++lz;
            const int x = tx, r = y * NX + x;
            const int o = lz * PLS + r;
            // padded layout: x margin 4, y and z margins 2, margins absent
            const int64_t gi = gbase + (int64_t)(z0 + lz + 2) * plane_g + (int64_t)(y + 2) * A.px + (x + 4);
            U[o] = __ldcg(ug + gi);
            Pk[o] = __ldcg(pg + gi);
            X[o] = __ldcg(xg + gi);
            const uint32_t g0 = gg[gi];
            const float wR = wgt5(g0, gg[gi + 1], A.c2f, A.wminf);
            const float wD = wgt5(g0, gg[gi + A.px], A.c2f, A.wminf);
            const float wF = wgt5(g0, gg[gi + plane_g], A.c2f, A.wminf);
            const float wL = wgt5(gg[gi - 1], g0, A.c2f, A.wminf);
            const float wU = wgt5(gg[gi - A.px], g0, A.c2f, A.wminf);
            const float wB = wgt5(gg[gi - plane_g], g0, A.c2f, A.wminf);
            WX[o] = wR;
            WY[o] = wD;
            WZ[o] = wF;
            if (lz == 0) WZB[r] = wB;
            const float d = ((wL + wR) + (wU + wD)) + (wB + wF);
            Dg[o] = ((int)g0 >= 0 && d > 0.0f) ? d : 0.0f;  // free voxels carry +g
        }
        for (int r = tid; r < PLS; r += kClNT) PKB[r] = PKA[r] = UA[r] = 0.0f;
        cl_sync();  // set up everywhere before any remote write

        int it = 0;
        for (;;) {
            const float alpha = T.alpha.hi + T.alpha.lo;
            const bool keep = T.phase == 2;
            const float ku = keep ? 0.0f : 1.0f, bp = keep ? 1.0f : T.beta.hi + T.beta.lo;
            // -- A: p_k = ku u + bp p, boundary planes to the neighbours
            // (the few padding words of each plane are updated too, and never read)
            for (int i = tid; i < nzl * PLS; i += kClNT) Pk[i] = fmaf(bp, Pk[i], ku * U[i]);
            __syncthreads();
            if (nzl > 0) {
                if (rank > 0) plane_to(Pk, PKA, rank - 1, PLS);
                if (rank + 1 < CL) plane_to(Pk + (nzl - 1) * PLS, PKB, rank + 1, PLS);
            }
            cl_sync();
            // -- B: stencil, update, five of the six inner products
            float a_gam = 0.f, a_rr = 0.f, a_del = 0.f, a_eps = 0.f, a_pi = 0.f, a_tau = 0.f;
            for (int row = tlive ? trow : nrows, lz = row / NY, y = row - lz * NY; row < nrows;
                 row += RPI, y += RPI) {
                while (y >= NY) y -= NY, ++lz;
                const int x = tx, r = y * NX + x;
                const int o = lz * PLS + r;
                const float p0 = Pk[o];
                const float pL = x > 0 ? Pk[o - 1] : 0.0f, wL = x > 0 ? WX[o - 1] : 0.0f;
                const float pR = x + 1 < NX ? Pk[o + 1] : 0.0f, wR = WX[o];
                const float pU = y > 0 ? Pk[o - NX] : 0.0f, wU = y > 0 ? WY[o - NX] : 0.0f;
                const float pD = y + 1 < NY ? Pk[o + NX] : 0.0f, wD = WY[o];
                const float pB = lz > 0 ? Pk[o - PLS] : PKB[r], wB = lz > 0 ? WZ[o - PLS] : WZB[r];
                const float pF = lz + 1 < nzl ? Pk[o + PLS] : PKA[r], wF = WZ[o];
                // difference form: the weak edges of a strongly linked voxel keep their precision
                const float sv = ((wL * (p0 - pL) + wR * (p0 - pR)) + (wU * (p0 - pU) + wD * (p0 - pD))) +
                                 (wB * (p0 - pB) + wF * (p0 - pF));
                const float d = Dg[o];
                const float un = d > 0.0f ? U[o] - alpha * sv * __fdividef(1.0f, d) : 0.0f;
                X[o] = fmaf(alpha, p0, X[o]);
                U[o] = un;
                const float du = d * un;
                a_gam = fmaf(du, un, a_gam);
                a_rr = fmaf(du, du, a_rr);
                a_eps = fmaf(un, sv, a_eps);
                a_pi = fmaf(p0, sv, a_pi);
                a_tau = fmaf(du, p0, a_tau);
            }
            __syncthreads();
            if (nzl > 0 && rank > 0) plane_to(U, UA, rank - 1, PLS);
            cl_sync();
            // -- C: delta = u'^T A u' over the forward edges of the own voxels
            for (int row = tlive ? trow : nrows, lz = row / NY, y = row - lz * NY; row < nrows;
                 row += RPI, y += RPI) {
                while (y >= NY) y -= NY, ++lz;
                const int x = tx, r = y * NX + x;
                const int o = lz * PLS + r;
                const float un = U[o];
                if (x + 1 < NX) {
                    const float dx = un - U[o + 1];
                    a_del = fmaf(WX[o] * dx, dx, a_del);
                }
                if (y + 1 < NY) {
                    const float dy = un - U[o + NX];
                    a_del = fmaf(WY[o] * dy, dy, a_del);
                }
                const float dz = un - (lz + 1 < nzl ? U[o + PLS] : UA[r]);
                a_del = fmaf(WZ[o] * dz, dz, a_del);
            }
            // six sums: warp trees, then a tree over the warps, in double-FP32
            {
                DF v[6] = {{a_gam, 0.f}, {a_rr, 0.f}, {a_del, 0.f}, {a_eps, 0.f}, {a_pi, 0.f}, {a_tau, 0.f}};
#pragma unroll
                for (int m = 16; m > 0; m >>= 1)
#pragma unroll
                    for (int k = 0; k < 6; ++k) v[k] = df_add(v[k], df_shfl_xor(v[k], m));
                const int lane = tid & 31, wid = tid >> 5;
                if (lane == 0)
#pragma unroll
                    for (int k = 0; k < 6; ++k) wsum[k][wid] = v[k];
                __syncthreads();
                if (wid == 0) {
#pragma unroll
                    for (int k = 0; k < 6; ++k) v[k] = lane < kClNT / 32 ? wsum[k][lane] : DF{0.f, 0.f};
#pragma unroll
                    for (int m = 16; m > 0; m >>= 1)
#pragma unroll
                        for (int k = 0; k < 6; ++k) v[k] = df_add(v[k], df_shfl_xor(v[k], m));
                    // this CTA's sums into slot `rank` of every CTA's table (lane t: CTA t)
                    if (lane < (int)CL) {
                        const uint32_t dst = cl_map(part_s, (uint32_t)lane) + 8u * 6u * rank;
#pragma unroll
                        for (int k = 0; k < 6; ++k) cl_st2(dst + 8u * k, v[k].hi, v[k].lo);
                    }
                }
            }
            cl_sync();
            // every CTA: the cluster's sums (a tree over the CTAs, the same order
            // everywhere) and the scalar recurrences, in warp 0
            if (tid < 32) {
                DF v[6];
#pragma unroll
                for (int k = 0; k < 6; ++k) v[k] = tid < (int)CL ? part[tid * 6 + k] : DF{0.f, 0.f};
#pragma unroll
                for (int m = 16; m > 0; m >>= 1)
#pragma unroll
                    for (int k = 0; k < 6; ++k) v[k] = df_add(v[k], df_shfl_xor(v[k], m));
                if (tid == 0) {
                    // the recurrences of the strip kernels' last CTA (finalize_box)
                    const DF g = v[0], rr = v[1], dl = v[2], ep = v[3], pi = v[4], tau = v[5];
                    bool stop;
                    T.rr = rr;
                    if (T.phase == 0) {
                        T.phase = 1;
                        T.gam = g;
                        stop = !df_gt(rr, T.tol2) || !df_pos(g) || !df_pos(dl);
                        T.alpha = stop ? DF{0.f, 0.f} : df_div(g, dl);
                        T.beta = DF{0.f, 0.f};
                    } else {
                        if (T.phase == 1) T.iters += 1;
                        T.phase = 1;
                        const DF bcg = df_pos(pi) ? df_neg(df_div(ep, pi)) : DF{0.f, 0.f};
                        const DF den = df_add(df_add(dl, df_mul(DF{2.f, 0.f}, df_mul(bcg, ep))),
                                              df_mul(df_mul(bcg, bcg), pi));
                        const DF num = df_add(g, df_mul(bcg, tau));
                        const bool ok = df_pos(pi) && df_pos(den) && df_pos(num);
                        const bool above = df_gt(rr, T.tol2);
                        stop = !above || T.iters >= T.max_iter || !ok;
                        if (!ok && above) T.status = 5;
                        if (!stop) {
                            T.beta = bcg;
                            T.alpha = df_div(num, den);
                            T.gam = g;
                        }
                    }
                    if (stop) T.active = 0;
                }
            }
            __syncthreads();
            ++it;
            if (!T.active || it >= A.loop_iters) break;  // identical in every CTA
        }
        if (tid == 0) {  // the record as FP64, buffer parity unchanged
            S.gam = df_dbl(T.gam);
            S.alpha = df_dbl(T.alpha);
            S.beta = df_dbl(T.beta);
            S.rr = df_dbl(T.rr);
            S.iters = T.iters;
            S.phase = T.phase;
            S.active = T.active;
            S.status = T.status;
        }
        __syncthreads();

        // write the state back into the system's buffer
        for (int row = tlive ? trow : nrows, lz = row / NY, y = row - lz * NY; row < nrows;
             row += RPI, y += RPI) {
            while (y >= NY) y -= NY, ++lz;
            const int x = tx, r = y * NX + x;
            const int o = lz * PLS + r;
            const int64_t gi = gbase + (int64_t)(z0 + lz + 2) * plane_g + (int64_t)(y + 2) * A.px + (x + 4);
            ug[gi] = U[o];
            pg[gi] = Pk[o];
            xg[gi] = X[o];
        }
        if (rank == 0 && tid == 0) {
            scalars_store(Sg, S);
            if (!S.active) atomicSub(A.n_active, 1);
            atomicMax(A.done, it);
        }
        __syncthreads();
    }
}

size_t cluster_smem_bytes(int nx, int ny, int nz, int cl) {
    const int pls = ((nx * ny) + 3) & ~3;
    const int nzl = (nz + cl - 1) / cl;
    return ((size_t)7 * nzl * pls + (size_t)4 * pls) * sizeof(float) + (size_t)cl * 6 * 2 * sizeof(float);
}

// Clusters of `cl` CTAs that can be resident at once (0: the launch is not possible).
int cluster_max_active(int nx, int ny, int nz, int cl) {
    const size_t smem = cluster_smem_bytes(nx, ny, nz, cl);
    if (cudaFuncSetAttribute(k_brick_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
        cudaFuncSetAttribute(k_brick_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)cl);
    cfg.blockDim = dim3(kClNT);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, k_brick_cluster, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

cudaError_t launch_brick_cluster(const ClusterArgs& a, int nclusters, int cl, cudaStream_t s) {
    const size_t smem = cluster_smem_bytes(a.nx, a.ny, a.nz, cl);
    cudaError_t e = cudaFuncSetAttribute(k_brick_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_brick_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nclusters * cl));
    cfg.blockDim = dim3(kClNT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)cl;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_brick_cluster, a);
}

}  // namespace rwk
