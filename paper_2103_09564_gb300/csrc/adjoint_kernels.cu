// Adjoint of the random walker solve (gradient of a loss l(x); not in the
// paper).  With A(w) x_U = b(w) and lambda solving A lambda = (dl/dx)_U
// (lambda = 0 on seeds), every edge contributes
//   dl/dw_pq = -(lambda_p - lambda_q)(x_p - x_q),
// and w = exp(-beta (g_p - g_q)^2) (zero derivative where the w_min clamp is
// active) gives dw/dbeta = -d^2 w, dw/dg_p = -2 beta d w, d = g_p - g_q.
// One thread per voxel gathers dl/dg over its six edges; dl/dbeta sums the
// forward edge of each voxel (FP64 block partials, reduced per box).
#include "rw_internal.h"

namespace rwk {

__device__ __forceinline__ float gflt(const void* g, int gtype, int64_t i) {
    return gtype == G_U16 ? (float)static_cast<const uint16_t*>(g)[i] * (1.0f / 65535.0f)
                          : static_cast<const float*>(g)[i];
}

__global__ void __launch_bounds__(256) k_adjoint(const AdjArgs a) {
    const int box = blockIdx.y;
    const int nx = a.bx.nx, ny = a.bx.ny, nz = a.bx.nz;
    const int64_t nvox = (int64_t)nx * ny * nz;
    const int64_t li = (int64_t)blockIdx.x * 256 + threadIdx.x;
    double db = 0.0;
    if (li < nvox) {
        int x, y, z;
        vox_xyz(li, nx, ny, nvox, &x, &y, &z);
        int ex = nx, ey = ny, ez = nz;
        if (a.bx.ext) {
            ex = a.bx.ext[3 * box];
            ey = a.bx.ext[3 * box + 1];
            ez = a.bx.ext[3 * box + 2];
        }
        const int64_t base = (int64_t)box * nvox;
        const int64_t i = base + li;
        float dg = 0.0f;
        const uint8_t ci = (x < ex && y < ey && z < ez) ? a.code[i] : ABSENT;
        if (ci != ABSENT) {
            const float gi = gflt(a.g, a.gtype, i);
            const double li_ = (ci == FREE) ? a.lam[i] : 0.0;
            const double xi = (double)a.x[i];
            const int nbx[6] = {x + 1, x, x, x - 1, x, x};
            const int nby[6] = {y, y + 1, y, y, y - 1, y};
            const int nbz[6] = {z, z, z + 1, z, z, z - 1};
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                if (nbx[k] < 0 || nbx[k] >= ex || nby[k] < 0 || nby[k] >= ey || nbz[k] < 0 || nbz[k] >= ez) continue;
                const int64_t j = base + ((int64_t)nbz[k] * ny + nby[k]) * nx + nbx[k];
                const uint8_t cj = a.code[j];
                if (cj == ABSENT || (ci != FREE && cj != FREE)) continue;
                const float d = gi - gflt(a.g, a.gtype, j);
                const float e = expf((float)(-a.beta) * d * d);
                if (!((double)e > a.wmin)) continue;
                const double lj = (cj == FREE) ? a.lam[j] : 0.0;
                const double dl_dw = -(li_ - lj) * (xi - (double)a.x[j]);
                dg += (float)(dl_dw * (-2.0 * a.beta * (double)d * (double)e));
                if (k < 3) db += dl_dw * (-(double)d * (double)d * (double)e);
            }
        }
        if (a.dg) a.dg[i] = dg;
    }
    __shared__ double red[8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) db += __shfl_down_sync(0xffffffffu, db, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = db;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int k = 0; k < 8; ++k) s += red[k];
        a.part[(int64_t)box * a.blocks_per_box + blockIdx.x] = s;
    }
}

cudaError_t launch_adjoint(const AdjArgs& a, cudaStream_t s) {
    dim3 grid((unsigned)a.blocks_per_box, (unsigned)a.bx.nbox);
    k_adjoint<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

__global__ void k_adjoint_reduce(const double* part, int bpb, double* dbeta) {
    __shared__ double red[256];
    double v = 0.0;
    for (int k = threadIdx.x; k < bpb; k += 256) v += part[(int64_t)blockIdx.x * bpb + k];
    red[threadIdx.x] = v;
    __syncthreads();
    for (int st = 128; st > 0; st >>= 1) {
        if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) dbeta[blockIdx.x] = red[0];
}

cudaError_t launch_adjoint_reduce(const double* part, int blocks_per_box, int nbox, double* dbeta, cudaStream_t s) {
    k_adjoint_reduce<<<nbox, 256, 0, s>>>(part, blocks_per_box, dbeta);
    return cudaGetLastError();
}

}  // namespace rwk
