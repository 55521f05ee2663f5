// Fused PCG sweep: one kernel per iteration of the random walker solve
// L_U x_U = -B^T x_M (Sec. III-B) with the Jacobi preconditioner (Sec. V,
// CG with Jacobi preconditioner).
//
// The CG recurrences are arranged so that the two inner products of an
// iteration are taken in the same sweep (the single-reduction arrangement of
// Chronopoulos and Gear).  Storing u = D^-1 r instead of r, one sweep reads
// x, u_k, p_k-1, g and the seed code and writes x, u_k+1 and p_k:
//
//   p_k    = u_k + beta_k p_k-1                    (pointwise, tile + halo 2)
//   s_k    = A p_k                                  (7-point stencil, halo 1)
//   x_k+1  = x_k + alpha_k p_k
//   u_k+1  = u_k - alpha_k D^-1 s_k                 (halo 1)
//   w_k+1  = A u_k+1                                (interior)
//   gamma  = (r, u) = sum d u^2,  delta = (u, w),  rr = sum (d u)^2
//
// and alpha_k+1 = gamma_k+1 / (delta_k+1 - beta_k+1 gamma_k+1 / alpha_k),
// beta_k+1 = gamma_k+1 / gamma_k are formed by the last CTA of the system.
// A = D - W is never stored: the six edge weights
// w = max(exp(-beta (g_p - g_q)^2), w_min) are recomputed from g in shared
// memory (FP32: ex2.approx; FP64: exp).  Seeds keep u = p = 0, absent voxels
// and voxels outside the box have no edges.
//
// Tiling: a CTA owns a TX x TY column block of one box and marches through a
// z-chunk with ring buffers of planes (p and u_k with a 2-voxel halo, u_k+1
// with a 1-voxel halo, forward edge weights), so every voxel of x, u, p is
// read and written once per sweep from HBM; halo planes and columns come from
// L2.  Per-thread partial sums run in T (at most one element per plane),
// block and grid reductions in FP64 (warp shuffles, then the last CTA of the
// system sums the per-CTA partials in a fixed order: results are
// deterministic).  No CTA waits on another: the last-block pattern uses one
// atomic counter per system and never spins.
#pragma once

#include "rw_internal.h"

namespace rwk {

__device__ __forceinline__ float ex2_approx(float a) {
    float r;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}

__device__ __forceinline__ double weight64(double dg, double mbeta, double wmin);  // below

template <typename T>
struct Num;
template <>
struct Num<float> {
    typedef float acc;
    __device__ __forceinline__ static float w(float a, float b, const SweepArgs& A) {
        const float d = a - b;
        return fmaxf(ex2_approx(A.c2f * d * d), A.wminf);
    }
};
template <>
struct Num<double> {
    typedef double acc;
    __device__ __forceinline__ static double w(double a, double b, const SweepArgs& A) {
        return weight64(a - b, A.mbeta, A.wmin);
    }
};

template <typename T, typename G>
__device__ __forceinline__ T gval(const G* g, int64_t i) {
    if constexpr (sizeof(G) == 2) {
        if constexpr (sizeof(T) == 4) return (float)g[i] * (1.0f / 65535.0f);
        else return (double)g[i] / 65535.0;
    } else {
        return (T)g[i];
    }
}

// Block-wide FP64 sum of NV per-thread values (warp shuffles, then one warp);
// the result is valid in thread 0.  red: NV * (NT / 32) doubles.
template <int NT, int NV>
__device__ __forceinline__ void block_reduce(double* v, double* red) {
    constexpr int NW = NT / 32;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) red[k * NW + wid] = v[k];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] = lane < NW ? red[k * NW + lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int k = 0; k < NV; ++k) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    }
    __syncthreads();
}

// Same for FP32 per-thread partials: the 32 lanes of a warp are summed in
// FP32 (a few roundings on top of each thread's FP32 sum), the warp partials
// in FP64 and in a fixed order.  Result in v of warp 0.
template <int NT, int NV>
__device__ __forceinline__ void block_reduce_f32(const float* f, double* v, double* red) {
    constexpr int NW = NT / 32;
    float t[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) t[k] = f[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < NV; ++k) t[k] += __shfl_down_sync(0xffffffffu, t[k], o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) red[k * NW + wid] = (double)t[k];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] = lane < NW ? red[k * NW + lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int k = 0; k < NV; ++k) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    }
    __syncthreads();
}

// Double-FP32 numbers (hi + lo, about 48 significant bits) for the per-iteration
// sums and scalar recurrences: on GB300 a dependent chain of FP64 operations
// costs far more than the sweep of a small system, FP32 operations do not.
// Addition is Knuth's TwoSum, products use the exact FMA remainder (Dekker's
// product with a fused multiply-add), division one correction step.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF df_fast(float a, float b) {  // |a| >= |b|
    const float s = a + b;
    return DF{s, b - (s - a)};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb);
    return df_fast(s, e + (a.lo + b.lo));
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
    const float p = a.hi * b.hi;
    const float e = fmaf(a.hi, b.hi, -p);
    return df_fast(p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e)));
}
// a / b: a first quotient, the exact remainder a - q1 b in double-FP32, and a
// correction quotient of the remainder.  The correction absorbs the few ulps
// of error of the fast FP32 quotients (|b| < 2^126).
__device__ __forceinline__ DF df_div(DF a, DF b) {
    const float q1 = __fdividef(a.hi, b.hi);
    const DF r = df_add(a, df_mul(DF{-q1, 0.0f}, b));
    return df_fast(q1, __fdividef(r.hi, b.hi));
}
__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }
__device__ __forceinline__ bool df_pos(DF a) { return a.hi > 0.0f || (a.hi == 0.0f && a.lo > 0.0f); }
__device__ __forceinline__ bool df_gt(DF a, DF b) { return df_pos(df_add(a, df_neg(b))); }
__device__ __forceinline__ DF df_of(double x) {
    const float h = (float)x;
    return DF{h, (float)(x - (double)h)};
}
__device__ __forceinline__ double df_dbl(DF a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ DF df_shfl_xor(DF a, int m) {
    return DF{__shfl_xor_sync(0xffffffffu, a.hi, m), __shfl_xor_sync(0xffffffffu, a.lo, m)};
}

// exp(x) for x <= 0 in double-FP32: the argument reduced by k ln 2 (ln 2 as
// a two-float constant, k = round(x log2 e)), a Taylor series of degree 12 on
// |r| <= ln 2 / 2 in Horner form, scaled by 2^k.  Relative error below 5e-13
// for x >= -69 (e^-69 ~ 1e-30, the default w_min; the two-float argument
// carries |x| 2^-48 of absolute error); below that the low part underflows
// (1e-8 relative at e^-87), and x < -87 gives 0 (the caller's floor applies).
__host__ __device__ constexpr double df_inv_fact(int n) { return n <= 1 ? 1.0 : df_inv_fact(n - 1) / n; }
#define RW_DF_CONST(v) DF{(float)(v), (float)((v) - (double)(float)(v))}
__device__ __forceinline__ DF df_exp_neg(DF x) {
    if (!(x.hi >= -87.0f)) return DF{0.0f, 0.0f};
    constexpr double kLn2 = 0.69314718055994530942;
    const float k = rintf(x.hi * 1.44269504088896341f);
    const DF r = df_add(x, df_neg(df_mul(DF{k, 0.0f}, RW_DF_CONST(kLn2))));
    DF p = RW_DF_CONST(df_inv_fact(12));
#define RW_HORNER(n) p = df_add(df_mul(p, r), RW_DF_CONST(df_inv_fact(n)))
    RW_HORNER(11); RW_HORNER(10); RW_HORNER(9); RW_HORNER(8); RW_HORNER(7); RW_HORNER(6);
    RW_HORNER(5); RW_HORNER(4); RW_HORNER(3); RW_HORNER(2); RW_HORNER(1); RW_HORNER(0);
#undef RW_HORNER
    const float sc = __int_as_float((127 + (int)k) << 23);  // 2^k, k in [-126, 0]
    return DF{p.hi * sc, p.lo * sc};
}
#undef RW_DF_CONST

// The FP64 edge weight max(exp(mbeta dg^2), w_min) (mbeta = -beta) of the
// residual and of the FP64 sweeps: the argument in FP64, the exponential in
// double-FP32 on the FP32 pipes (GB300's FP64 rate makes an FP64 exp the
// cost of a residual pass).
__device__ __forceinline__ double weight64(double dg, double mbeta, double wmin) {
    const double t = mbeta * dg * dg;
    const float th = (float)t;
    const DF e = df_exp_neg(DF{th, (float)(t - (double)th)});
    return fmax((double)e.hi + (double)e.lo, wmin);
}

// finalize_box (below) in double-FP32: the same recurrences and decisions on
// the six sums of a sweep, without a chain of dependent FP64 operations (the
// record keeps FP64 fields; they are converted on the way in and out).
template <typename SP>
__device__ __forceinline__ void finalize_box_df(SP S, const DF* v, int* n_active, int out_par) {
    const DF g = v[0], rr = v[1], dl = v[2], ep = v[3], pi = v[4], tau = v[5];
    const DF tol2 = df_of(S->tol2);
    bool stop;
    S->par = out_par;
    S->rr = df_dbl(rr);
    if (S->phase == 0) {
        // restart sweep (alpha = beta = 0, p = u): alpha_0 = gamma_0 / delta_0
        S->phase = 1;
        S->gam = df_dbl(g);
        stop = !df_gt(rr, tol2) || !df_pos(g) || !df_pos(dl);
        S->alpha = stop ? 0.0 : df_dbl(df_div(g, dl));
        S->beta = 0.0;
    } else {
        if (S->phase == 1) S->iters += 1;
        S->phase = 1;
        const DF bcg = df_pos(pi) ? df_neg(df_div(ep, pi)) : DF{0.0f, 0.0f};
        const DF den = df_add(df_add(dl, df_mul(DF{2.0f, 0.0f}, df_mul(bcg, ep))), df_mul(df_mul(bcg, bcg), pi));
        const DF num = df_add(g, df_mul(bcg, tau));
        const bool ok = df_pos(pi) && df_pos(den) && df_pos(num);
        const bool above = df_gt(rr, tol2);
        stop = !above || S->iters >= S->max_iter || !ok;
        if (!ok && above) S->status = 5;
        if (!stop) {
            S->beta = df_dbl(bcg);
            S->alpha = df_dbl(df_div(num, den));
            S->gam = df_dbl(g);
        }
    }
    if (stop) {
        S->active = 0;
        atomicSub(n_active, 1);
    }
}

// Scalar recurrences of the system after its sweep (run by one thread of the
// last CTA).  v = {gamma, ||r||^2, delta, eps, pi, tau} of the sweep that
// produced u = u_k+1 from the direction p = p_k:
//   gamma = (r, u), delta = (u, A u), eps = (u, A p), pi = (p, A p),
//   tau = (r, p), with r = D u.
// The next direction p' = u + beta p is made A-conjugate to p explicitly,
// beta = -eps / pi, and the step is the exact line minimum along it,
//   alpha = (r, p') / (p', A p') = (gamma + beta tau) / (delta + 2 beta eps + beta^2 pi).
// In exact arithmetic these equal the classic PCG scalars; computing them from
// the sweep's own inner products keeps them valid after the residual is
// replaced by the FP64 one (the search direction survives the replacement).
// out_par is the buffer index the sweep wrote.
template <typename SP>  // BoxScalars* or volatile BoxScalars* (read through L2)
__device__ __forceinline__ void finalize_box(SP S, const double* v, int* n_active, int out_par) {
    const double g = v[0], rr = v[1], dl = v[2], ep = v[3], pi = v[4], tau = v[5];
    bool stop;
    S->par = out_par;
    S->rr = rr;
    if (S->phase == 0) {
        // restart sweep (alpha = beta = 0, p = u): alpha_0 = gamma_0 / delta_0
        S->phase = 1;
        S->gam = g;
        stop = !(rr > S->tol2) || !(g > 0.0) || !(dl > 0.0);
        S->alpha = stop ? 0.0 : g / dl;
        S->beta = 0.0;
    } else {
        if (S->phase == 1) S->iters += 1;
        S->phase = 1;
        const double bcg = pi > 0.0 ? -ep / pi : 0.0;
        const double den = dl + 2.0 * bcg * ep + bcg * bcg * pi;
        const double num = g + bcg * tau;
        const bool ok = pi > 0.0 && den > 0.0 && num > 0.0;
        stop = !(rr > S->tol2) || S->iters >= S->max_iter || !ok;
        if (!ok && rr > S->tol2) S->status = 5;
        if (!stop) {
            S->beta = bcg;
            S->alpha = num / den;
            S->gam = g;
        }
    }
    if (stop) {
        S->active = 0;
        atomicSub(n_active, 1);
    }
}

template <typename T>
constexpr int sweep_planes_bytes(int R2) {
    return (int)sizeof(T) * R2 * 22 + 2 * R2;
}

template <typename T, typename G, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT) k_sweep(const SweepArgs A) {
    constexpr int W2 = TX + 4, H2 = TY + 4, R2 = W2 * H2;
    constexpr int W1 = TX + 2, H1 = TY + 2, R1 = W1 * H1;
    typedef typename Num<T>::acc acc;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* sP = reinterpret_cast<T*>(smem_raw);  // [3][R2] p_k
    T* sUk = sP + 3 * R2;                     // [2][R2] u_k
    T* sUn = sUk + 2 * R2;                    // [3][R2] u_k+1
    T* sG = sUn + 3 * R2;                     // [2][R2] g
    T* sWx = sG + 2 * R2;                     // [4][R2] weight (i, i+x)
    T* sWy = sWx + 4 * R2;                    // [4][R2] weight (i, i+y)
    T* sWz = sWy + 4 * R2;                    // [4][R2] weight (i-z, i)
    uint8_t* sC = reinterpret_cast<uint8_t*>(sWz + 4 * R2);  // [2][R2] code
    __shared__ double red[6 * (NT / 32)];
    __shared__ int s_last;

    const int tid = threadIdx.x;
    const int tpb = A.ntx * A.nty * A.nzc;
    const int64_t nwork = (int64_t)(A.list ? *A.nlist : A.bx.nbox) * tpb;
    const int nx = A.bx.nx, ny = A.bx.ny, nz = A.bx.nz;
    const int64_t bstride = (int64_t)nx * ny * nz;
    const G* __restrict__ gin = static_cast<const G*>(A.g);
    const uint8_t* __restrict__ cin = A.code;
    T* __restrict__ X = static_cast<T*>(A.x);
    const T* __restrict__ Uin = static_cast<const T*>(A.u_in);
    const T* __restrict__ Pin = static_cast<const T*>(A.p_in);
    T* __restrict__ Uout = static_cast<T*>(A.u_out);
    T* __restrict__ Pout = static_cast<T*>(A.p_out);

    for (int64_t w = blockIdx.x; w < nwork; w += gridDim.x) {
        const int li = (int)(w / tpb);  // position in the list of active systems
        const int box = A.list ? A.list[li] : li;
        const int t = (int)(w - (int64_t)li * tpb);
        BoxScalars* S = A.sc + box;
        if (!S->active) continue;  // same value for every thread of the CTA
        const int tx = t % A.ntx, ty = (t / A.ntx) % A.nty, tz = t / (A.ntx * A.nty);
        const T alpha = (T)S->alpha, bcg = (T)S->beta;
        const bool keep_p = S->phase == 2;
        int ex = nx, ey = ny, ez = nz;
        if (A.bx.ext) {
            ex = A.bx.ext[3 * box];
            ey = A.bx.ext[3 * box + 1];
            ez = A.bx.ext[3 * box + 2];
        }
        const int ox = tx * TX, oy = ty * TY, z0 = tz * A.zc;
        const int z1 = min(z0 + A.zc, ez);
        const int64_t base = (int64_t)box * bstride;
        acc a_gam = 0, a_rr = 0, a_del = 0, a_eps = 0, a_pi = 0, a_tau = 0;

        if (ox < ex && oy < ey && z0 < ez) {
            for (int zf = z0 - 2; zf <= z1 + 1; ++zf) {
                const int f3 = (zf + 6) % 3, f2 = (zf + 6) & 1, f4 = (zf + 8) & 3, p2 = (zf + 5) & 1;
                // -- A1: load plane zf (halo 2), p_k = u_k + beta p_k-1
                for (int e = tid; e < R2; e += NT) {
                    const int ix = e % W2, iy = e / W2;
                    const int gx = ox + ix - 2, gy = oy + iy - 2;
                    uint8_t c = ABSENT;
                    T gv = 0, uk = 0, pm = 0;
                    if (gx >= 0 && gx < ex && gy >= 0 && gy < ey && zf >= 0 && zf < ez) {
                        const int64_t i = base + ((int64_t)zf * ny + gy) * nx + gx;
                        c = cin[i];
                        gv = gval<T, G>(gin, i);
                        if (A.sqrt_g) gv = sqrt(gv);
                        uk = Uin[i];
                        pm = Pin[i];
                    }
                    sC[f2 * R2 + e] = c;
                    sG[f2 * R2 + e] = gv;
                    sUk[f2 * R2 + e] = uk;
                    sP[f3 * R2 + e] = keep_p ? pm : ((c == FREE) ? uk + bcg * pm : (T)0);
                }
                __syncthreads();
                // -- A2: forward edge weights of plane zf (and z-edges to zf-1)
                for (int e = tid; e < R2; e += NT) {
                    const int ix = e % W2, iy = e / W2;
                    const uint8_t c0 = sC[f2 * R2 + e];
                    const T g0 = sG[f2 * R2 + e];
                    T wx = 0, wy = 0, wz = 0;
                    if (c0 != ABSENT) {
                        if (ix + 1 < W2 && sC[f2 * R2 + e + 1] != ABSENT) wx = Num<T>::w(g0, sG[f2 * R2 + e + 1], A);
                        if (iy + 1 < H2 && sC[f2 * R2 + e + W2] != ABSENT) wy = Num<T>::w(g0, sG[f2 * R2 + e + W2], A);
                        if (zf > z0 - 2 && sC[p2 * R2 + e] != ABSENT) wz = Num<T>::w(sG[p2 * R2 + e], g0, A);
                    }
                    sWx[f4 * R2 + e] = wx;
                    sWy[f4 * R2 + e] = wy;
                    sWz[f4 * R2 + e] = wz;
                }
                __syncthreads();
                // -- B: plane zm = zf-1 on the halo-1 region
                const int zm = zf - 1;
                if (zm >= z0 - 1) {
                    const int m3 = (zm + 6) % 3, m2 = (zm + 6) & 1, m4 = (zm + 8) & 3;
                    const int l3 = (zm + 5) % 3;  // plane zm-1
                    const T* P = sP + m3 * R2;
                    const T* Pl = sP + l3 * R2;
                    const T* Ph = sP + f3 * R2;
                    const T* Wx = sWx + m4 * R2;
                    const T* Wy = sWy + m4 * R2;
                    const T* Wzl = sWz + m4 * R2;
                    const T* Wzh = sWz + f4 * R2;
                    const bool zint = (zm >= z0 && zm < z1);
                    for (int e1 = tid; e1 < R1; e1 += NT) {
                        const int jx = e1 % W1 + 1, jy = e1 / W1 + 1;
                        const int e = jy * W2 + jx;
                        const uint8_t c = sC[m2 * R2 + e];
                        const T p0 = P[e];
                        T un = 0, d = 0, sv = 0;
                        if (c == FREE) {
                            const T wxm = Wx[e - 1], wxp = Wx[e], wym = Wy[e - W2], wyp = Wy[e], wzm = Wzl[e],
                                    wzp = Wzh[e];
                            d = ((wxm + wxp) + (wym + wyp)) + (wzm + wzp);
                            // difference form: every edge keeps its own
                            // relative precision (d * p0 - sum w p_j would
                            // cancel the weak edges of a strongly linked voxel)
                            sv = ((wxm * (p0 - P[e - 1]) + wxp * (p0 - P[e + 1])) +
                                  (wym * (p0 - P[e - W2]) + wyp * (p0 - P[e + W2]))) +
                                 (wzm * (p0 - Pl[e]) + wzp * (p0 - Ph[e]));
                            if (d > (T)0) un = sUk[m2 * R2 + e] - alpha * sv / d;
                        }
                        sUn[m3 * R2 + e] = un;
                        if (zint && jx >= 2 && jx < TX + 2 && jy >= 2 && jy < TY + 2) {
                            const int gx = ox + jx - 2, gy = oy + jy - 2;
                            if (gx < ex && gy < ey) {
                                const int64_t i = base + ((int64_t)zm * ny + gy) * nx + gx;
                                Uout[i] = un;
                                Pout[i] = p0;
                                if (c == FREE) {
                                    X[i] = X[i] + alpha * p0;
                                    const acc du = (acc)d * (acc)un;
                                    a_gam += du * (acc)un;
                                    a_rr += du * du;
                                    a_eps += (acc)un * (acc)sv;
                                    a_pi += (acc)p0 * (acc)sv;
                                    a_tau += du * (acc)p0;
                                }
                            }
                        }
                    }
                }
                __syncthreads();
                // -- C: plane zw = zf-2 interior, delta = (u, A u)
                const int zw = zf - 2;
                if (zw >= z0 && zw < z1) {
                    const int w3 = (zw + 6) % 3, w4 = (zw + 8) & 3, wn4 = (zw + 9) & 3;
                    const T* U = sUn + w3 * R2;
                    const T* Ul = sUn + ((zw + 5) % 3) * R2;
                    const T* Uh = sUn + ((zw + 7) % 3) * R2;
                    const T* Wx = sWx + w4 * R2;
                    const T* Wy = sWy + w4 * R2;
                    const T* Wzl = sWz + w4 * R2;
                    const T* Wzh = sWz + wn4 * R2;
                    for (int e0 = tid; e0 < TX * TY; e0 += NT) {
                        const int jx = e0 % TX + 2, jy = e0 / TX + 2;
                        const int e = jy * W2 + jx;
                        const T u0 = U[e];
                        if (u0 != (T)0 && ox + jx - 2 < ex && oy + jy - 2 < ey) {
                            const T wxm = Wx[e - 1], wxp = Wx[e], wym = Wy[e - W2], wyp = Wy[e], wzm = Wzl[e],
                                    wzp = Wzh[e];
                            const T au = ((wxm * (u0 - U[e - 1]) + wxp * (u0 - U[e + 1])) +
                                          (wym * (u0 - U[e - W2]) + wyp * (u0 - U[e + W2]))) +
                                         (wzm * (u0 - Ul[e]) + wzp * (u0 - Uh[e]));
                            a_del += (acc)u0 * (acc)au;
                        }
                    }
                }
            }
        }
        // -- reductions: block (FP64), then the last CTA of the system
        double v[6] = {(double)a_gam, (double)a_rr, (double)a_del, (double)a_eps, (double)a_pi, (double)a_tau};
        block_reduce<NT, 6>(v, red);
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
