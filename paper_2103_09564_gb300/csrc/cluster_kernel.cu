// Cluster-resident PCG for small systems (brick neighbourhoods of up to 40
// voxels per axis, the root of a brick-32 pyramid): one thread-block cluster
// per system keeps the whole FP32 state on chip across iterations.
//
// The batched sweeps stream every system through HBM / L2 once per iteration;
// when only a few systems are left (the slow bricks of a level, the small
// coarse levels), an iteration costs the latency of its loads, of the
// two-stage reduction and of a grid-wide synchronisation, about ten
// microseconds, whatever the size.  Here the rows (z, y) of a system, in
// z-major order, are split into CL contiguous ranges of equal size (+-1), one
// per CTA of a cluster (CL = 16, non-portable cluster size, one CTA per SM).
// Every CTA holds in shared memory u, p_k, the correction delta, the diagonal
// and the three forward edge weights of its rows, and ghost copies of the NY
// rows (one plane) on either side of its range: p_k of the ghost rows is
// formed locally from ghost u and ghost p by the same expression the owner
// uses, so the only exchange of an iteration is u' of the first and the last
// NY own rows, written into the neighbours' ghost slots (double-buffered by
// iteration parity) through distributed shared memory.  The weights and the
// diagonal are computed once per launch (g does not change).
//
// One iteration is the sweep of the strip kernels (same recurrences,
// single-reduction PCG with u = D^-1 r stored, difference-form stencil, FP32
// per-thread partial sums, double-FP32 block and cluster sums and scalar
// recurrences): p_k = ku u + bp p, s = A p_k, u' = u - alpha D^-1 s (free
// voxels), delta += alpha p_k, and gamma, ||D u'||^2, u'^T A u', (u', s),
// (p_k, s), (D u', p_k).  Two cluster barriers per iteration: the first
// after the u' exchange (the edges into the upper ghost rows need the
// neighbour's u'; the CTA sums the other edges of u'^T A u' while the rows
// travel), the second after every CTA has written its six sums into every
// CTA's table.  Every CTA then runs the same scalar recurrences on the same
// sums in the same order, so all of them take the same exit.  A launch runs
// up to `loop_iters` iterations of each system; the state is read from and
// written back to the global arrays (the strip kernel's layout) of the system's current buffer
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

// Copy n floats (a multiple of 4, 16-byte aligned) to the place of dst_local in CTA `rank`.
__device__ __forceinline__ void block_to(const float* src, const float* dst_local, uint32_t rank, int n) {
    const uint32_t dst = cl_map((uint32_t)__cvta_generic_to_shared(dst_local), rank);
    const float4* s4 = reinterpret_cast<const float4*>(src);
    for (int q = threadIdx.x; q < n / 4; q += kClNT) cl_st4(dst + 16u * (uint32_t)q, s4[q]);
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
    __shared__ float red6[6][kClNT];

    const int tid = threadIdx.x;
    const int NX = A.nx, NY = A.ny, NZ = A.nz;
    const int RS = A.rs, ROWS = A.rows;  // row stride (floats, a multiple of 4) and most own rows of a CTA
    const uint32_t rank = cl_rank(), CL = cl_size();
    const int NR = NZ * NY;  // rows of the system
    const int r0 = (int)(((uint32_t)NR * rank) / CL), r1 = (int)(((uint32_t)NR * (rank + 1)) / CL);
    const int nown = r1 - r0;  // >= NY: the host requires NZ >= CL
    const int G = NY * RS;     // floats of one block of NY rows
    // shared memory, rows of RS floats.  Local row L of P, WY, WZ is system row
    // r0 - NY + L: the lower ghost rows, the own rows, then (P only) the upper ghost rows.
    float* P = reinterpret_cast<float*>(smem_raw);  // [ROWS + 2 NY] p, then p_k
    float* U = P + (ROWS + 2 * NY) * RS;             // [ROWS] own u, then u'
    float* UG = U + ROWS * RS;                       // [2 parities][lower, upper][NY] ghost u
    float* X = UG + 4 * G;                           // [ROWS] correction delta
    float* Dg = X + ROWS * RS;                       // [ROWS] diagonal (0 on voxels that are not free)
    float* WX = Dg + ROWS * RS;                      // [ROWS] forward weight (i, i+x)
    float* WY = WX + ROWS * RS;                      // [ROWS + NY] forward weight (i, i+y)
    float* WZ = WY + (ROWS + NY) * RS;               // [ROWS + NY] forward weight (i, i+z)
    DF* part = reinterpret_cast<DF*>(WZ + (ROWS + NY) * RS);  // [CL][6] every CTA's sums
    const uint32_t part_s = (uint32_t)__cvta_generic_to_shared(part);
    const int n_smem = (7 * ROWS + 8 * NY) * RS;

    const int64_t plane_g = (int64_t)A.px * A.py;
    const int64_t bstride = plane_g * A.pz;
    const int nlist = A.list ? *A.nlist : A.nbox;
    // voxel loops run over rows: thread tid owns column x = tid % NX of rows
    // tid / NX, tid / NX + RPI, ... (threads beyond RPI * NX idle in the loops)
    const int RPI = kClNT / NX;
    const int tx = tid % NX, trow = tid / NX;
    const bool tlive = trow < RPI;
    // the strip kernel's layout (no margins, rows of A.px >= NX voxels): system row R = z NY + y
    auto gidx = [&](int64_t gbase, int R) -> int64_t { return gbase + (int64_t)R * A.px + tx; };

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

        // zero everything (padding columns and unwritten ghost slots stay 0)
        for (int i = tid; i < n_smem; i += kClNT) P[i] = 0.0f;
        __syncthreads();
        // own rows: state, forward weights, diagonal (neighbours beyond the box are absent)
        {
            int y = (r0 + trow) % NY, z = (r0 + trow) / NY;
            for (int j = tlive ? trow : nown; j < nown; j += RPI, y += RPI) {
                while (y >= NY) y -= NY, ++z;
                const int64_t gi = gidx(gbase, r0 + j);
                const int o = j * RS + tx, l = (j + NY) * RS + tx;
                U[o] = __ldcg(ug + gi);
                P[l] = __ldcg(pg + gi);
                X[o] = __ldcg(xg + gi);
                const uint32_t g0 = gg[gi];
                const uint32_t gR = tx + 1 < A.px ? gg[gi + 1] : GC_ABSENT, gL = tx > 0 ? gg[gi - 1] : GC_ABSENT;
                const uint32_t gD = y + 1 < NY ? gg[gi + A.px] : GC_ABSENT, gU = y > 0 ? gg[gi - A.px] : GC_ABSENT;
                const uint32_t gF = z + 1 < NZ ? gg[gi + plane_g] : GC_ABSENT, gB = z > 0 ? gg[gi - plane_g] : GC_ABSENT;
                const float wR = wgt5(g0, gR, A.c2f, A.wminf);
                const float wD = wgt5(g0, gD, A.c2f, A.wminf);
                const float wF = wgt5(g0, gF, A.c2f, A.wminf);
                const float wL = wgt5(gL, g0, A.c2f, A.wminf);
                const float wU = wgt5(gU, g0, A.c2f, A.wminf);
                const float wB = wgt5(gB, g0, A.c2f, A.wminf);
                WX[o] = wR;
                WY[l] = wD;
                WZ[l] = wF;
                const float d = ((wL + wR) + (wU + wD)) + (wB + wF);
                Dg[o] = ((int)g0 >= 0 && d > 0.0f) ? d : 0.0f;  // free voxels carry +g
            }
        }
        // ghost rows inside the system: u (both parity slots), p, and the
        // forward y / z weights of the lower ones (rows beyond the system stay 0)
        for (int j = tlive ? trow : NY; j < NY; j += RPI) {
            const int o = j * RS + tx;
            const int rlo = r0 - NY + j, rhi = r1 + j;
            if (rlo >= 0) {
                const int64_t glo = gidx(gbase, rlo);
                const int y = rlo % NY;
                UG[o] = UG[2 * G + o] = __ldcg(ug + glo);
                P[o] = __ldcg(pg + glo);
                const uint32_t g0 = gg[glo];
                WY[o] = wgt5(g0, y + 1 < NY ? gg[glo + A.px] : GC_ABSENT, A.c2f, A.wminf);
                WZ[o] = wgt5(g0, gg[glo + plane_g], A.c2f, A.wminf);  // rlo + NY < NR: own row
            }
            if (rhi < NR) {
                const int64_t ghi = gidx(gbase, rhi);
                UG[G + o] = UG[3 * G + o] = __ldcg(ug + ghi);
                P[(NY + nown) * RS + o] = __ldcg(pg + ghi);
            }
        }
        cl_sync();  // set up everywhere before any remote write

        int it = 0;
        // iteration loops run over strips of 4 voxels of a row (one float4 of
        // every array; padding columns x >= NX hold zero state and weights and
        // act as absent voxels): thread tid owns strip tq = tid % Q of rows
        // tid / Q, tid / Q + RPP, ...
        const int Q = RS / 4, RPP = kClNT / Q;
        const int tq = tid % Q, trw = tid / Q;
        const bool slive = trw < RPP;
        const float4* P4 = reinterpret_cast<const float4*>(P);
        const float4* W4X = reinterpret_cast<const float4*>(WX);
        const float4* W4Y = reinterpret_cast<const float4*>(WY);
        const float4* W4Z = reinterpret_cast<const float4*>(WZ);
        const float4* D4 = reinterpret_cast<const float4*>(Dg);
        float4* U4 = reinterpret_cast<float4*>(U);
        float4* X4 = reinterpret_cast<float4*>(X);
        const int Q4 = G / 4;  // float4 of a block of NY rows
        for (;;) {
            const int sl = it & 1;  // ghost u of this iteration: slot sl; the neighbours write u' into sl ^ 1
            const float* UGlo = UG + (2 * sl) * G;
            const float* UGhi = UGlo + G;
            float* const UNlo = UG + (2 * (sl ^ 1)) * G;
            float* const UNhi = UNlo + G;
            const float alpha = T.alpha.hi + T.alpha.lo;
            const bool keep = T.phase == 2;
            const float ku = keep ? 0.0f : 1.0f, bp = keep ? 1.0f : T.beta.hi + T.beta.lo;
            // -- 1: p_k = ku u + bp p on the own and the ghost rows
            {
                float4* Pw = reinterpret_cast<float4*>(P);
                const float4* ul = reinterpret_cast<const float4*>(UGlo);
                const float4* uh = reinterpret_cast<const float4*>(UGhi);
                const int hi0 = (NY + nown) * Q;
                auto pk = [&](float4 p, float4 u) {
                    return make_float4(fmaf(bp, p.x, ku * u.x), fmaf(bp, p.y, ku * u.y), fmaf(bp, p.z, ku * u.z),
                                       fmaf(bp, p.w, ku * u.w));
                };
                for (int i = tid; i < Q4; i += kClNT) {
                    Pw[i] = pk(Pw[i], ul[i]);
                    Pw[hi0 + i] = pk(Pw[hi0 + i], uh[i]);
                }
                for (int i = tid; i < nown * Q; i += kClNT) Pw[Q4 + i] = pk(Pw[Q4 + i], U4[i]);
            }
            __syncthreads();
            // -- 2: stencil, update, five of the six inner products (own rows)
            float a_gam = 0.f, a_rr = 0.f, a_del = 0.f, a_eps = 0.f, a_pi = 0.f, a_tau = 0.f;
            {
                int y = (r0 + trw) % NY;
                for (int j = slive ? trw : nown; j < nown; j += RPP, y += RPP) {
                    while (y >= NY) y -= NY;
                    const int o = j * Q + tq, l = (j + NY) * Q + tq;  // float4 indices
                    const float4 pc = P4[l];
                    const float pl = tq > 0 ? P[4 * l - 1] : 0.0f, pr = tq + 1 < Q ? P[4 * l + 4] : 0.0f;
                    const float wxl = tq > 0 ? WX[4 * o - 1] : 0.0f;
                    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
                    const float4 pu = y > 0 ? P4[l - Q] : z4, pd = y + 1 < NY ? P4[l + Q] : z4;
                    const float4 wu = y > 0 ? W4Y[l - Q] : z4, wd = W4Y[l];
                    const float4 pb = P4[l - Q4], pf = P4[l + Q4];
                    const float4 wb = W4Z[l - Q4], wf = W4Z[l];
                    const float4 wx = W4X[o], dg = D4[o];
                    float4 uu = U4[o], xx = X4[o];
                    const float p[4] = {pc.x, pc.y, pc.z, pc.w}, w[4] = {wx.x, wx.y, wx.z, wx.w};
                    const float PU[4] = {pu.x, pu.y, pu.z, pu.w}, PD[4] = {pd.x, pd.y, pd.z, pd.w};
                    const float WU[4] = {wu.x, wu.y, wu.z, wu.w}, WD[4] = {wd.x, wd.y, wd.z, wd.w};
                    const float PB[4] = {pb.x, pb.y, pb.z, pb.w}, PF[4] = {pf.x, pf.y, pf.z, pf.w};
                    const float WB[4] = {wb.x, wb.y, wb.z, wb.w}, WF[4] = {wf.x, wf.y, wf.z, wf.w};
                    const float D[4] = {dg.x, dg.y, dg.z, dg.w};
                    float un[4] = {uu.x, uu.y, uu.z, uu.w}, xv[4] = {xx.x, xx.y, xx.z, xx.w};
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const float p0 = p[i];
                        const float pL = i == 0 ? pl : p[i - 1], wL = i == 0 ? wxl : w[i - 1];
                        const float pR = i == 3 ? pr : p[i + 1], wR = w[i];
                        // difference form: the weak edges of a strongly linked voxel keep their precision
                        const float sv = ((wL * (p0 - pL) + wR * (p0 - pR)) + (WU[i] * (p0 - PU[i]) + WD[i] * (p0 - PD[i]))) +
                                         (WB[i] * (p0 - PB[i]) + WF[i] * (p0 - PF[i]));
                        const float d = D[i];
                        un[i] = d > 0.0f ? un[i] - alpha * sv * __fdividef(1.0f, d) : 0.0f;
                        xv[i] = fmaf(alpha, p0, xv[i]);
                        const float du = d * un[i];
                        a_gam = fmaf(du, un[i], a_gam);
                        a_rr = fmaf(du, du, a_rr);
                        a_eps = fmaf(un[i], sv, a_eps);
                        a_pi = fmaf(p0, sv, a_pi);
                        a_tau = fmaf(du, p0, a_tau);
                    }
                    U4[o] = make_float4(un[0], un[1], un[2], un[3]);
                    X4[o] = make_float4(xv[0], xv[1], xv[2], xv[3]);
                }
            }
            __syncthreads();
            // -- 3: u' of the first / last NY own rows to the neighbours' ghost slots; meanwhile
            // delta = u'^T A u' over the forward edges of the own voxels that stay inside the range
            if (rank > 0) block_to(U, UNhi, rank - 1, G);
            if (rank + 1 < CL) block_to(U + (nown - NY) * RS, UNlo, rank + 1, G);
            {
                int y = (r0 + trw) % NY;
                for (int j = slive ? trw : nown; j < nown; j += RPP, y += RPP) {
                    while (y >= NY) y -= NY;
                    const int o = j * Q + tq, l = (j + NY) * Q + tq;
                    const float4 u4 = U4[o], wx = W4X[o];
                    const float ur = tq + 1 < Q ? U[4 * o + 4] : 0.0f;
                    float dx = u4.x - u4.y;
                    a_del = fmaf(wx.x * dx, dx, a_del);
                    dx = u4.y - u4.z;
                    a_del = fmaf(wx.y * dx, dx, a_del);
                    dx = u4.z - u4.w;
                    a_del = fmaf(wx.z * dx, dx, a_del);
                    dx = u4.w - ur;
                    a_del = fmaf(wx.w * dx, dx, a_del);
                    if (y + 1 < NY && j + 1 < nown) {
                        const float4 v = U4[o + Q], wy = W4Y[l];
                        a_del = fmaf(wy.x * (u4.x - v.x), u4.x - v.x, a_del);
                        a_del = fmaf(wy.y * (u4.y - v.y), u4.y - v.y, a_del);
                        a_del = fmaf(wy.z * (u4.z - v.z), u4.z - v.z, a_del);
                        a_del = fmaf(wy.w * (u4.w - v.w), u4.w - v.w, a_del);
                    }
                    if (j + NY < nown) {
                        const float4 v = U4[o + Q4], wz = W4Z[l];
                        a_del = fmaf(wz.x * (u4.x - v.x), u4.x - v.x, a_del);
                        a_del = fmaf(wz.y * (u4.y - v.y), u4.y - v.y, a_del);
                        a_del = fmaf(wz.z * (u4.z - v.z), u4.z - v.z, a_del);
                        a_del = fmaf(wz.w * (u4.w - v.w), u4.w - v.w, a_del);
                    }
                }
            }
            cl_sync();
            // the edges into the upper ghost rows (u' of rank + 1; zero beyond the system)
            {
                const int jb = nown - NY;
                const float4* uh = reinterpret_cast<const float4*>(UNhi);
                int y = (r0 + jb + trw) % NY;
                for (int j = slive ? jb + trw : nown; j < nown; j += RPP, y += RPP) {
                    while (y >= NY) y -= NY;
                    const int o = j * Q + tq, l = (j + NY) * Q + tq;
                    const float4 u4 = U4[o];
                    const float4 v = uh[(j - jb) * Q + tq], wz = W4Z[l];
                    a_del = fmaf(wz.x * (u4.x - v.x), u4.x - v.x, a_del);
                    a_del = fmaf(wz.y * (u4.y - v.y), u4.y - v.y, a_del);
                    a_del = fmaf(wz.z * (u4.z - v.z), u4.z - v.z, a_del);
                    a_del = fmaf(wz.w * (u4.w - v.w), u4.w - v.w, a_del);
                    if (j == nown - 1 && y + 1 < NY) {
                        const float4 v0 = uh[tq], wy = W4Y[l];
                        a_del = fmaf(wy.x * (u4.x - v0.x), u4.x - v0.x, a_del);
                        a_del = fmaf(wy.y * (u4.y - v0.y), u4.y - v0.y, a_del);
                        a_del = fmaf(wy.z * (u4.z - v0.z), u4.z - v0.z, a_del);
                        a_del = fmaf(wy.w * (u4.w - v0.w), u4.w - v0.w, a_del);
                    }
                }
            }
            // six sums of the CTA in double-FP32: the per-thread partials through
            // shared memory, warp k sums partial k (16 per lane, two chains, then a
            // shuffle tree) and writes it into slot `rank` of every CTA's table
            red6[0][tid] = a_gam;
            red6[1][tid] = a_rr;
            red6[2][tid] = a_del;
            red6[3][tid] = a_eps;
            red6[4][tid] = a_pi;
            red6[5][tid] = a_tau;
            __syncthreads();
            {
                const int lane = tid & 31, wid = tid >> 5;
                if (wid < 6) {
                    const float* r = red6[wid];
                    DF c0 = {r[lane], 0.f}, c1 = {r[lane + 32], 0.f};
#pragma unroll
                    for (int i = 2; i < kClNT / 32; i += 2) {
                        c0 = df_add(c0, DF{r[lane + 32 * i], 0.f});
                        c1 = df_add(c1, DF{r[lane + 32 * i + 32], 0.f});
                    }
                    DF v = df_add(c0, c1);
#pragma unroll
                    for (int m = 16; m > 0; m >>= 1) v = df_add(v, df_shfl_xor(v, m));
                    if (lane < (int)CL) cl_st2(cl_map(part_s, (uint32_t)lane) + 8u * (6u * rank + (uint32_t)wid), v.hi, v.lo);
                }
            }
            cl_sync();
            // every CTA: the cluster's sums (a tree over the CTAs, the same order
            // everywhere) and the scalar recurrences, in warp 0
            if (tid < 32) {
                DF v[6];
#pragma unroll
                for (int k = 0; k < 6; ++k) v[k] = tid < (int)CL ? part[tid * 6 + k] : DF{0.f, 0.f};
                int m0 = 1;
                while (2 * m0 < (int)CL) m0 <<= 1;
                for (int m = m0; m > 0; m >>= 1)
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

        // write the state of the own rows back into the system's buffer
        for (int j = tlive ? trow : nown; j < nown; j += RPI) {
            const int64_t gi = gidx(gbase, r0 + j);
            const int o = j * RS + tx;
            ug[gi] = U[o];
            pg[gi] = P[(j + NY) * RS + tx];
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

int cluster_row_stride(int nx) { return (nx + 3) & ~3; }
int cluster_rows(int ny, int nz, int cl) { return (ny * nz + cl - 1) / cl; }

size_t cluster_smem_bytes(int nx, int ny, int nz, int cl) {
    const size_t rows = (size_t)7 * cluster_rows(ny, nz, cl) + (size_t)8 * ny;
    return rows * cluster_row_stride(nx) * sizeof(float) + (size_t)cl * 6 * 2 * sizeof(float);
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
