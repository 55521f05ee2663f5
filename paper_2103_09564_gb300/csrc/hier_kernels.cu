// Kernels of the hierarchical procedure: normalisation/quantisation, LOD
// pyramid (Sec. III-A), brick neighbourhood gather with border seeds (Eqs. 2
// and 3), label rasterisation, contraction with pruning statistics (Sec.
// IV-D1 / IV-E) and the level fill through pruned holes (Sec. IV-D1).
#include <float.h>

#include "rw_internal.h"

namespace rwk {

// ---------------------------------------------------------------------------
// Normalisation window and unorm16 storage.  Each step is one correctly
// rounded FP32 operation so the stored codes are reproducible bit for bit:
//   g = clamp((v - lo) / (hi - lo), 0, 1);  q = round_half_even(g * 65535).
__global__ void k_quantize(const void* v, int dtype, int64_t n, float lo, float hi, int normalize, int storage,
                           void* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float g;
    if (dtype == 1) {  // RW_F32
        const float vv = static_cast<const float*>(v)[i];
        if (normalize) {
            const float span = __fsub_rn(hi, lo);
            g = span > 0.0f ? __fdiv_rn(__fsub_rn(vv, lo), span) : 0.0f;
        } else {
            g = vv;
        }
    } else {
        const uint16_t q = static_cast<const uint16_t*>(v)[i];
        if (!normalize) {
            if (storage == 0) {
                static_cast<uint16_t*>(out)[i] = q;
                return;
            }
            g = __fdiv_rn((float)q, 65535.0f);
        } else {
            const float span = __fsub_rn(hi, lo);
            g = span > 0.0f ? __fdiv_rn(__fsub_rn((float)q, lo), span) : 0.0f;
        }
    }
    if (!(g > 0.0f)) g = 0.0f;
    if (g > 1.0f) g = 1.0f;
    if (storage == 0) static_cast<uint16_t*>(out)[i] = (uint16_t)__float2uint_rn(__fmul_rn(g, 65535.0f));
    else static_cast<float*>(out)[i] = g;
}

cudaError_t launch_quantize(const void* v, int dtype, int64_t n, float lo, float hi, int normalize, int storage,
                            void* out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_quantize<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(v, dtype, n, lo, hi, normalize, storage, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// One pyramid step: parent = mean of the existing 2x2x2 children, summed in
// the fixed order ((c0+c1)+(c2+c3))+((c4+c5)+(c6+c7)) (child k = dx+2dy+4dz,
// missing children as +0) and scaled by 1/count (count is a power of two).
template <bool U16>
__global__ void k_downsample(const void* fine, int nx, int ny, int nz, float* coarse) {
    const int cx = (nx + 1) / 2, cy = (ny + 1) / 2, cz = (nz + 1) / 2;
    const int64_t n = (int64_t)cx * cy * cz;
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    const int X = (int)(o % cx), Y = (int)((o / cx) % cy), Z = (int)(o / ((int64_t)cx * cy));
    float c[8];
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int x = 2 * X + (k & 1), y = 2 * Y + ((k >> 1) & 1), z = 2 * Z + ((k >> 2) & 1);
        if (x < nx && y < ny && z < nz) {
            const int64_t i = ((int64_t)z * ny + y) * nx + x;
            c[k] = U16 ? __fdiv_rn((float)static_cast<const uint16_t*>(fine)[i], 65535.0f)
                       : static_cast<const float*>(fine)[i];
            ++cnt;
        } else {
            c[k] = 0.0f;
        }
    }
    const float s01 = __fadd_rn(c[0], c[1]), s23 = __fadd_rn(c[2], c[3]);
    const float s45 = __fadd_rn(c[4], c[5]), s67 = __fadd_rn(c[6], c[7]);
    const float sum = __fadd_rn(__fadd_rn(s01, s23), __fadd_rn(s45, s67));
    coarse[o] = __fmul_rn(sum, __fdiv_rn(1.0f, (float)cnt));
}

cudaError_t launch_downsample_u16(const uint16_t* fine, int nx, int ny, int nz, float* coarse, cudaStream_t s) {
    const int64_t n = (int64_t)((nx + 1) / 2) * ((ny + 1) / 2) * ((nz + 1) / 2);
    k_downsample<true><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(fine, nx, ny, nz, coarse);
    return cudaGetLastError();
}

cudaError_t launch_downsample_f32(const float* fine, int nx, int ny, int nz, float* coarse, cudaStream_t s) {
    const int64_t n = (int64_t)((nx + 1) / 2) * ((ny + 1) / 2) * ((nz + 1) / 2);
    k_downsample<false><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(fine, nx, ny, nz, coarse);
    return cudaGetLastError();
}

__global__ void k_leaf_to_f32(const uint16_t* q, int64_t n, float* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __fdiv_rn((float)q[i], 65535.0f);
}

cudaError_t launch_leaf_to_f32(const uint16_t* q, int64_t n, float* out, cudaStream_t s) {
    k_leaf_to_f32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(q, n, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Trilinear sample of the filled level k-1 field at the centre of level-k
// voxel (X, Y, Z): u = (i + 0.5)/2 - 0.5 per axis, clamp-to-edge.  For even
// i the two parent taps are i/2-1, i/2 with weights 1/4, 3/4; for odd i they
// are i/2, i/2+1 with weights 3/4, 1/4.
__device__ __forceinline__ void taps(int i, int n, int* a, int* b, float* wa, float* wb) {
    const int h = i >> 1;
    if (i & 1) {
        *a = h;
        *b = h + 1;
        *wa = 0.75f;
        *wb = 0.25f;
    } else {
        *a = h - 1;
        *b = h;
        *wa = 0.25f;
        *wb = 0.75f;
    }
    *a = min(max(*a, 0), n - 1);
    *b = min(max(*b, 0), n - 1);
}

__device__ __forceinline__ float upsample_at(const float* P, int px, int py, int pz, int X, int Y, int Z) {
    int xa, xb, ya, yb, za, zb;
    float wxa, wxb, wya, wyb, wza, wzb;
    taps(X, px, &xa, &xb, &wxa, &wxb);
    taps(Y, py, &ya, &yb, &wya, &wyb);
    taps(Z, pz, &za, &zb, &wza, &wzb);
    const int64_t sy = px, sz = (int64_t)px * py;
    const float c00 = wxa * P[za * sz + ya * sy + xa] + wxb * P[za * sz + ya * sy + xb];
    const float c01 = wxa * P[za * sz + yb * sy + xa] + wxb * P[za * sz + yb * sy + xb];
    const float c10 = wxa * P[zb * sz + ya * sy + xa] + wxb * P[zb * sz + ya * sy + xb];
    const float c11 = wxa * P[zb * sz + yb * sy + xa] + wxb * P[zb * sz + yb * sy + xb];
    return wza * (wya * c00 + wyb * c01) + wzb * (wya * c10 + wyb * c11);
}

// Neighbourhood N(n) of every active node (Eq. 3) into the brick pool:
// intensities, seed codes and the FP64 initial iterate.  The one-voxel outer
// layer of the clipped neighbourhood on faces inside the level volume holds
// continuous seeds sampled from the parent level (Eq. 2); other voxels start
// from the upsampled parent (Sec. IV-D2) or the given initial field.
__global__ void k_gather(const GatherArgs a) {
    double* x_hi = a.x_out;
    const int box = blockIdx.y;
    const int nx = a.bx.nx, ny = a.bx.ny, nz = a.bx.nz;
    const int64_t nvox = (int64_t)nx * ny * nz;
    const int64_t li = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (li >= nvox) return;
    int x, y, z;
    vox_xyz(li, nx, ny, nvox, &x, &y, &z);
    const BrickJob J = a.jobs[box];
    const int64_t i = (int64_t)box * nvox + li;
    if (x >= J.ex || y >= J.ey || z >= J.ez) {
        a.code_out[i] = ABSENT;
        a.g_out[i] = 0.0f;
        x_hi[i] = 0.0;
        return;
    }
    const int X = J.rx0 + x, Y = J.ry0 + y, Z = J.rz0 + z;
    const int64_t li_lvl = ((int64_t)Z * a.ly + Y) * a.lx + X;
    a.g_out[i] = a.gq ? __fdiv_rn((float)a.gq[li_lvl], 65535.0f) : a.gf[li_lvl];
    const float up = a.parent ? upsample_at(a.parent, a.px, a.py, a.pz, X, Y, Z) : 0.0f;
    const bool border = ((J.faces & 1) && x == 0) || ((J.faces & 2) && x == J.ex - 1) ||
                        ((J.faces & 4) && y == 0) || ((J.faces & 8) && y == J.ey - 1) ||
                        ((J.faces & 16) && z == 0) || ((J.faces & 32) && z == J.ez - 1);
    if (border) {
        a.code_out[i] = SEED;
        x_hi[i] = (double)up;
    } else {
        a.code_out[i] = FREE;
        x_hi[i] = (double)(a.init ? a.init[li_lvl] : up);
    }
}

cudaError_t launch_gather(const GatherArgs& a, cudaStream_t s) {
    const int64_t nvox = (int64_t)a.bx.nx * a.bx.ny * a.bx.nz;
    dim3 grid((unsigned)((nvox + 255) / 256), (unsigned)a.bx.nbox);
    k_gather<<<grid, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// User labels rasterised at level k (T_n, Sec. IV-A): a non-conflicting label
// voxel inside the neighbourhood becomes a seed (overriding a border seed); a
// conflicting one stays as it is and marks the node (cfl, Sec. IV-D1).
__global__ void k_apply_labels(const Boxes bx, const BrickJob* jobs, const LabelVox* lab, int nlab, uint8_t* code,
                               double* x, int* box_flags) {
    const int box = blockIdx.y;
    const int l = blockIdx.x * blockDim.x + threadIdx.x;
    if (l >= nlab) return;
    const BrickJob J = jobs[box];
    const LabelVox L = lab[l];
    const int x0 = L.x - J.rx0, y0 = L.y - J.ry0, z0 = L.z - J.rz0;
    if (x0 < 0 || x0 >= J.ex || y0 < 0 || y0 >= J.ey || z0 < 0 || z0 >= J.ez) return;
    if (L.flags & 1) {
        atomicOr(&box_flags[box], (L.flags & 2) ? (16 | 128) : 16);
        return;
    }
    const int64_t i = (int64_t)box * bx.nx * bx.ny * bx.nz + ((int64_t)z0 * bx.ny + y0) * bx.nx + x0;
    code[i] = SEED;
    x[i] = (double)L.value;
}

cudaError_t launch_apply_labels(const Boxes& bx, const BrickJob* jobs, const LabelVox* lab, int nlab, uint8_t* code,
                                double* x, int* box_flags, cudaStream_t s) {
    if (nlab == 0 || bx.nbox == 0) return cudaSuccess;
    dim3 grid((unsigned)((nlab + 127) / 128), (unsigned)bx.nbox);
    k_apply_labels<<<grid, 128, 0, s>>>(bx, jobs, lab, nlab, code, x, box_flags);
    return cudaGetLastError();
}

// Contract N^-1 (Eq. 3): write the brick part of each solved neighbourhood
// into the level field and reduce min, max (hom / dt) and max |new - old|
// (similarity, Sec. IV-E).  One CTA per brick.
__global__ void __launch_bounds__(256) k_contract(const ContractArgs a) {
    const double* xs = a.x;
    const int box = blockIdx.x;
    if (a.skip && a.skip[box]) return;  // uniform over the block
    const BrickJob J = a.jobs[box];
    const int s = a.s;
    const int bx0 = J.bx * s, by0 = J.by * s, bz0 = J.bz * s;
    const int sx = min(s, a.lx - bx0), sy = min(s, a.ly - by0), sz = min(s, a.lz - bz0);
    const int64_t nb = (int64_t)sx * sy * sz;
    const int64_t pstride = (int64_t)a.bx.nx * a.bx.ny * a.bx.nz;
    float mn = FLT_MAX, mx = -FLT_MAX, md = 0.0f;
    for (int64_t k = threadIdx.x; k < nb; k += blockDim.x) {
        const int x = (int)(k % sx), y = (int)((k / sx) % sy), z = (int)(k / ((int64_t)sx * sy));
        const int X = bx0 + x, Y = by0 + y, Z = bz0 + z;
        const int px = X - J.rx0, py = Y - J.ry0, pz = Z - J.rz0;
        const float v = (float)xs[(int64_t)box * pstride + ((int64_t)pz * a.bx.ny + py) * a.bx.nx + px];
        const int64_t li = ((int64_t)Z * a.ly + Y) * a.lx + X;
        if (a.old) md = fmaxf(md, fabsf(v - a.old[li]));  // read before the write below (in place)
        if (!a.stats_only) a.field[li] = v;
        mn = fminf(mn, v);
        mx = fmaxf(mx, v);
    }
    __shared__ float r[3][8];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_down_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_down_sync(0xffffffffu, mx, o));
        md = fmaxf(md, __shfl_down_sync(0xffffffffu, md, o));
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        r[0][wid] = mn;
        r[1][wid] = mx;
        r[2][wid] = md;
    }
    __syncthreads();
    if (threadIdx.x == 0 && a.stats) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) {
            mn = fminf(mn, r[0][k]);
            mx = fmaxf(mx, r[1][k]);
            md = fmaxf(md, r[2][k]);
        }
        a.stats[3 * box] = mn;
        a.stats[3 * box + 1] = mx;
        a.stats[3 * box + 2] = md;
    }
}

cudaError_t launch_contract(const ContractArgs& a, cudaStream_t s) {
    if (a.bx.nbox == 0) return cudaSuccess;
    k_contract<<<a.bx.nbox, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// Level fill: voxels of absent nodes take the upsampled parent field (the
// nearest transitive parent's values, Sec. IV-D1).  The field is updated in
// place: solved nodes were written by k_contract, reused nodes keep the
// values of the previous pass.
// One thread per 8 consecutive voxels of a row (grid: x octets and rows in
// x / y, planes in z).  Children 8q .. 8q+7 of a row read parent columns
// 4q-1 .. 4q+4 (clamped); each column is interpolated in y, then z, and the
// children combine two columns with weights 1/4, 3/4 (the taps of
// upsample_at, applied axis by axis).  Brick indices by shifts when s is a
// power of two.
__global__ void k_fill(const FillArgs a) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int X0 = 8 * q;
    const int Y = blockIdx.y * blockDim.y + threadIdx.y;
    const int Z = blockIdx.z;
    if (X0 >= a.lx || Y >= a.ly) return;
    const bool pow2 = (a.s & (a.s - 1)) == 0;
    const int sh = __ffs(a.s) - 1;
    const int bz = pow2 ? Z >> sh : Z / a.s, by = pow2 ? Y >> sh : Y / a.s;
    const uint8_t* strow = a.status + (int64_t)(bz * a.nby + by) * a.nbx;
    bool wr[8];
    if ((a.s & 7) == 0) {  // the octet lies in one brick
        const bool w = strow[pow2 ? X0 >> sh : X0 / a.s] == 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) wr[k] = w && X0 + k < a.lx;
    } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) wr[k] = X0 + k < a.lx && strow[(X0 + k) / a.s] == 0;
    }
    bool any = false;
#pragma unroll
    for (int k = 0; k < 8; ++k) any = any || wr[k];
    if (!any) return;
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = 0.0f;
    if (a.parent) {
        int ya, yb, za, zb;
        float wya, wyb, wza, wzb;
        taps(Y, a.py, &ya, &yb, &wya, &wyb);
        taps(Z, a.pz, &za, &zb, &wza, &wzb);
        const int64_t sy = a.px, sz = (int64_t)a.px * a.py;
        const float* Paa = a.parent + za * sz + ya * sy;
        const float* Pab = a.parent + za * sz + yb * sy;
        const float* Pba = a.parent + zb * sz + ya * sy;
        const float* Pbb = a.parent + zb * sz + yb * sy;
        float c[6];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const int j = min(max(4 * q - 1 + k, 0), a.px - 1);
            const float ca = fmaf(wya, Paa[j], wyb * Pab[j]);  // z = za
            const float cb = fmaf(wya, Pba[j], wyb * Pbb[j]);  // z = zb
            c[k] = fmaf(wza, ca, wzb * cb);
        }
#pragma unroll
        for (int m = 0; m < 8; m += 2) {
            const int h = m >> 1;
            v[m] = fmaf(0.25f, c[h], 0.75f * c[h + 1]);
            v[m + 1] = fmaf(0.75f, c[h + 1], 0.25f * c[h + 2]);
        }
    }
    float* out = a.field + ((int64_t)Z * a.ly + Y) * a.lx + X0;
#pragma unroll
    for (int h = 0; h < 8; h += 4) {
        if (wr[h] && wr[h + 1] && wr[h + 2] && wr[h + 3] && ((reinterpret_cast<uintptr_t>(out + h) & 15u) == 0)) {
            *reinterpret_cast<float4*>(out + h) = make_float4(v[h], v[h + 1], v[h + 2], v[h + 3]);
        } else {
#pragma unroll
            for (int k = h; k < h + 4; ++k)
                if (wr[k]) out[k] = v[k];
        }
    }
}

cudaError_t launch_fill(const FillArgs& a, cudaStream_t s) {
    if ((int64_t)a.lx * a.ly * a.lz == 0) return cudaSuccess;
    const dim3 blk(32, 8, 1);
    const dim3 grid((unsigned)((a.lx + 255) / 256), (unsigned)((a.ly + 7) / 8), (unsigned)a.lz);
    k_fill<<<grid, blk, 0, s>>>(a);
    return cudaGetLastError();
}

__global__ void k_read_box(const float* field, int lx, int ly, int x0, int y0, int z0, int bx, int by, int bz,
                           float* out) {
    const int64_t n = (int64_t)bx * by * bz;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int x = (int)(k % bx), y = (int)((k / bx) % by), z = (int)(k / ((int64_t)bx * by));
    out[k] = field[((int64_t)(z0 + z) * ly + (y0 + y)) * lx + (x0 + x)];
}

// Argmax over the class fields (ties: the lowest class index) of m <= 4
// consecutive voxels starting at level index i0; one 128-bit load per class
// when the four voxels are aligned.
__device__ __forceinline__ void argmax4(const ClassFields& f, int64_t i0, int m, uint32_t* lw, float* pv) {
    *lw = 0;
    if (m == 4 && (i0 & 3) == 0) {
        float4 b = *reinterpret_cast<const float4*>(f.P[0] + i0);
        int c0 = 0, c1 = 0, c2 = 0, c3 = 0;
        for (int c = 1; c < f.n; ++c) {
            const float4 v = *reinterpret_cast<const float4*>(f.P[c] + i0);
            if (v.x > b.x) b.x = v.x, c0 = c;
            if (v.y > b.y) b.y = v.y, c1 = c;
            if (v.z > b.z) b.z = v.z, c2 = c;
            if (v.w > b.w) b.w = v.w, c3 = c;
        }
        *lw = (uint32_t)c0 | ((uint32_t)c1 << 8) | ((uint32_t)c2 << 16) | ((uint32_t)c3 << 24);
        pv[0] = b.x, pv[1] = b.y, pv[2] = b.z, pv[3] = b.w;
        return;
    }
    for (int j = 0; j < m; ++j) {
        int best = 0;
        float pb = f.P[0][i0 + j];
        for (int c = 1; c < f.n; ++c) {
            const float v = f.P[c][i0 + j];
            if (v > pb) {
                pb = v;
                best = c;
            }
        }
        *lw |= (uint32_t)best << (8 * j);
        pv[j] = pb;
    }
}

// Multi-class labels: argmax over the class fields of one level (ties: the
// lowest class index) on a box of the level.  One thread per 4 consecutive
// outputs (x fastest), stored as one 32-bit word (labels) and one 128-bit
// word (probabilities) where aligned: the outputs may be page-locked host
// memory, written across the host link.
__global__ void k_argmax(const __grid_constant__ ClassFields f, int lx, int ly, int x0, int y0, int z0, int bx,
                         int by, int bz, uint8_t* labels, float* prob) {
    const int64_t n = (int64_t)bx * by * bz;
    const int64_t k0 = 4 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    if (k0 >= n) return;
    const int m = n - k0 < 4 ? (int)(n - k0) : 4;
    uint32_t lw = 0;
    float pv[4] = {0.f, 0.f, 0.f, 0.f};
    if (bx == lx && by == ly) {
        // whole planes: the box is one contiguous range of the level
        argmax4(f, (int64_t)z0 * ly * lx + k0, m, &lw, pv);
    } else {
        int x, y, z;
        vox_xyz(k0, bx, by, n, &x, &y, &z);
        for (int j = 0; j < m; ++j) {
            uint32_t l1;
            float p1;
            argmax4(f, ((int64_t)(z0 + z) * ly + (y0 + y)) * lx + (x0 + x), 1, &l1, &p1);
            lw |= l1 << (8 * j);
            pv[j] = p1;
            if (++x == bx) {
                x = 0;
                if (++y == by) y = 0, ++z;
            }
        }
    }
    uint8_t* lo = labels + k0;
    if (m == 4 && (reinterpret_cast<uintptr_t>(lo) & 3u) == 0) {
        *reinterpret_cast<uint32_t*>(lo) = lw;
    } else {
        for (int j = 0; j < m; ++j) lo[j] = (uint8_t)(lw >> (8 * j));
    }
    if (prob) {
        float* po = prob + k0;
        if (m == 4 && (reinterpret_cast<uintptr_t>(po) & 15u) == 0) {
            *reinterpret_cast<float4*>(po) = make_float4(pv[0], pv[1], pv[2], pv[3]);
        } else {
            for (int j = 0; j < m; ++j) po[j] = pv[j];
        }
    }
}

cudaError_t launch_argmax(const ClassFields& f, int lx, int ly, const int64_t box[6], uint8_t* labels, float* prob,
                          cudaStream_t s) {
    const int bx = (int)(box[3] - box[0]), by = (int)(box[4] - box[1]), bz = (int)(box[5] - box[2]);
    const int64_t n = (int64_t)bx * by * bz;
    if (n == 0) return cudaSuccess;
    const int64_t nt = (n + 3) / 4;
    k_argmax<<<(unsigned)((nt + 255) / 256), 256, 0, s>>>(f, lx, ly, (int)box[0], (int)box[1], (int)box[2], bx, by,
                                                           bz, labels, prob);
    return cudaGetLastError();
}

// Argmax on a list of bricks: block (brick, plane of the brick), each thread
// 4 consecutive voxels of a row (as k_argmax), outputs in the level's layout.
__global__ void k_argmax_nodes(const __grid_constant__ ClassFields f, int lx, int ly, int lz, int s, int nbx, int nby,
                               const int64_t* nodes, uint8_t* labels, float* prob) {
    const int64_t nd = nodes[blockIdx.x];
    const int bx = (int)(nd % nbx), by = (int)((nd / nbx) % nby), bz = (int)(nd / ((int64_t)nbx * nby));
    const int Z = bz * s + (int)blockIdx.y;
    if (Z >= lz) return;
    const int qr = (s + 3) / 4;  // quads per brick row
    for (int t = threadIdx.x; t < qr * s; t += blockDim.x) {
        const int y = t / qr, xq = 4 * (t - y * qr);
        const int Y = by * s + y, X0 = bx * s + xq;
        if (Y >= ly || X0 >= lx) continue;
        const int m = min(4, min(s - xq, lx - X0));
        const int64_t i0 = ((int64_t)Z * ly + Y) * lx + X0;
        uint32_t lw = 0;
        float pv[4] = {0.f, 0.f, 0.f, 0.f};
        argmax4(f, i0, m, &lw, pv);
        uint8_t* lo = labels + i0;
        if (m == 4 && (reinterpret_cast<uintptr_t>(lo) & 3u) == 0) {
            *reinterpret_cast<uint32_t*>(lo) = lw;
        } else {
            for (int j = 0; j < m; ++j) lo[j] = (uint8_t)(lw >> (8 * j));
        }
        if (prob) {
            float* po = prob + i0;
            if (m == 4 && (reinterpret_cast<uintptr_t>(po) & 15u) == 0) {
                *reinterpret_cast<float4*>(po) = make_float4(pv[0], pv[1], pv[2], pv[3]);
            } else {
                for (int j = 0; j < m; ++j) po[j] = pv[j];
            }
        }
    }
}

cudaError_t launch_argmax_nodes(const ClassFields& f, int lx, int ly, int lz, int s, int nbx, int nby,
                                const int64_t* nodes, int64_t n_nodes, uint8_t* labels, float* prob, cudaStream_t st) {
    if (n_nodes == 0) return cudaSuccess;
    if (n_nodes > 0x7fffffff || s > 65535) return cudaErrorInvalidValue;
    k_argmax_nodes<<<dim3((unsigned)n_nodes, (unsigned)s), 256, 0, st>>>(f, lx, ly, lz, s, nbx, nby, nodes, labels,
                                                                         prob);
    return cudaGetLastError();
}

cudaError_t launch_read_box(const float* field, int lx, int ly, int lz, const int64_t box[6], float* out,
                            cudaStream_t s) {
    (void)lz;
    const int bx = (int)(box[3] - box[0]), by = (int)(box[4] - box[1]), bz = (int)(box[5] - box[2]);
    const int64_t n = (int64_t)bx * by * bz;
    if (n == 0) return cudaSuccess;
    k_read_box<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(field, lx, ly, (int)box[0], (int)box[1], (int)box[2], bx,
                                                            by, bz, out);
    return cudaGetLastError();
}

// Copy the bricks listed in `nodes` (brick indices, x fastest) between a
// level field and a packed array [n][s][s][s] (x fastest within a brick):
// to_packed = 1 exports (voxels of a truncated border brick outside the level
// are written as 0), 0 imports (only voxels inside the level are written).
__global__ void k_brick_io(float* field, int lx, int ly, int lz, int s, int nbx, int nby, const int64_t* nodes,
                           int64_t n, float* packed, int to_packed) {
    const int64_t per = (int64_t)s * s * s;
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n * per) return;
    const int64_t i = k / per, r = k - i * per;
    const int64_t b = nodes[i];
    const int bx = (int)(b % nbx), by = (int)((b / nbx) % nby), bz = (int)(b / ((int64_t)nbx * nby));
    const int x = bx * s + (int)(r % s), y = by * s + (int)((r / s) % s), z = bz * s + (int)(r / ((int64_t)s * s));
    const bool in = x < lx && y < ly && z < lz;
    const int64_t f = ((int64_t)z * ly + y) * lx + x;
    if (to_packed) packed[k] = in ? field[f] : 0.0f;
    else if (in) field[f] = packed[k];
}

cudaError_t launch_brick_io(float* field, int lx, int ly, int lz, int s, int nbx, int nby, const int64_t* nodes,
                            int64_t n, float* packed, int to_packed, cudaStream_t st) {
    const int64_t tot = n * (int64_t)s * s * s;
    if (tot <= 0) return cudaSuccess;
    k_brick_io<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(field, lx, ly, lz, s, nbx, nby, nodes, n, packed,
                                                               to_packed);
    return cudaGetLastError();
}

}  // namespace rwk
