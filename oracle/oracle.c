/* FP64 CPU oracle of the random walker — TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow and direct.  Each function names the passage of the paper it
 * follows.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
 * leg may load this code; it shares nothing with the CUDA library.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fno-fast-math -shared -fPIC.
 * -ffp-contract=off keeps every FP32 operation of the quantisation and the
 * pyramid a separately rounded IEEE operation.
 *
 * Reductions are summed per z-plane and then over planes in order, so results
 * do not depend on the thread count.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define FREE 0
#define SEED 1
#define ABSENT 2

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ---------------------------------------------------------------------------
 * Normalisation and storage.  The paper defines weights on intensities
 * n[p] (Sec. III-B) without fixing their scale; the reading used here is a
 * min-max window [lo, hi] clamped to [0, 1], stored as unorm16:
 *   g = clamp((v - lo) / (hi - lo), 0, 1);  q = round_half_even(g * 65535).
 * Every step is one IEEE FP32 operation. */
static uint16_t quant_one(float v, float lo, float hi, int normalize) {
    float g;
    if (normalize) {
        float span = hi - lo;
        g = (span > 0.0f) ? (v - lo) / span : 0.0f;
    } else {
        g = v;
    }
    if (!(g > 0.0f)) g = 0.0f;  /* also maps NaN to 0 */
    if (g > 1.0f) g = 1.0f;
    float s = g * 65535.0f;
    return (uint16_t)rintf(s);
}

void oracle_quantize_f32(const float* v, int64_t n, float lo, float hi, int normalize, uint16_t* q) {
    for (int64_t i = 0; i < n; ++i) q[i] = quant_one(v[i], lo, hi, normalize);
}

void oracle_quantize_u16(const uint16_t* v, int64_t n, float lo, float hi, int normalize, uint16_t* q) {
    for (int64_t i = 0; i < n; ++i) {
        if (normalize) {
            q[i] = quant_one((float)v[i], lo, hi, 1);
        } else {
            q[i] = v[i]; /* already unorm16 */
        }
    }
}

/* ---------------------------------------------------------------------------
 * LOD pyramid, Sec. III-A: a parent voxel is the mean of its 2x2x2 children;
 * at odd borders only the existing children (1, 2 or 4) are averaged (Sec.
 * IV-A, uneven volumes).  Fixed order: children indexed k = a + 2b + 4c,
 * sum ((c0+c1)+(c2+c3))+((c4+c5)+(c6+c7)) with missing children as +0, then
 * multiply by 1/count (count is a power of two, so the scaling is exact). */
void oracle_downsample(const float* fine, int nx, int ny, int nz, float* coarse) {
    int cx = (nx + 1) / 2, cy = (ny + 1) / 2, cz = (nz + 1) / 2;
    for (int Z = 0; Z < cz; ++Z)
        for (int Y = 0; Y < cy; ++Y)
            for (int X = 0; X < cx; ++X) {
                float c[8];
                int count = 0;
                for (int k = 0; k < 8; ++k) {
                    int x = 2 * X + (k & 1), y = 2 * Y + ((k >> 1) & 1), z = 2 * Z + ((k >> 2) & 1);
                    if (x < nx && y < ny && z < nz) {
                        c[k] = fine[((int64_t)z * ny + y) * nx + x];
                        ++count;
                    } else {
                        c[k] = 0.0f;
                    }
                }
                float s01 = c[0] + c[1];
                float s23 = c[2] + c[3];
                float s45 = c[4] + c[5];
                float s67 = c[6] + c[7];
                float lo4 = s01 + s23;
                float hi4 = s45 + s67;
                float sum = lo4 + hi4;
                float inv = 1.0f / (float)count;
                coarse[((int64_t)Z * cy + Y) * cx + X] = sum * inv;
            }
}

/* ---------------------------------------------------------------------------
 * Random walker system, Sec. III-B.  Vertices are voxels, edges join
 * 6-neighbours, w_pq = exp(-beta (n[p] - n[q])^2).  The weight is clamped
 * below by w_min so that the FP system stays non-singular when the exponential
 * underflows (a reading; w_min = 0 reproduces the paper's formula). */
double oracle_weight(double a, double b, double beta, double w_min) {
    double d = a - b;
    double w = exp(-beta * d * d);
    return w > w_min ? w : w_min;
}

typedef struct {
    int nx, ny, nz;
    int64_t n;
    double *wx, *wy, *wz; /* forward edges (i, i+1), (i, i+nx), (i, i+nx*ny); 0 if absent */
    double* d;            /* weighted degree: sum of the weights of all edges at i */
} graph_t;

static void graph_build(graph_t* G, int nx, int ny, int nz, const double* g, const uint8_t* code,
                        double beta, double w_min) {
    G->nx = nx; G->ny = ny; G->nz = nz;
    G->n = (int64_t)nx * ny * nz;
    G->wx = (double*)calloc((size_t)G->n, sizeof(double));
    G->wy = (double*)calloc((size_t)G->n, sizeof(double));
    G->wz = (double*)calloc((size_t)G->n, sizeof(double));
    G->d = (double*)calloc((size_t)G->n, sizeof(double));
    const int64_t sy = nx, sz = (int64_t)nx * ny;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int64_t i = z * sz + y * sy + x;
                if (code[i] == ABSENT) continue;
                if (x + 1 < nx && code[i + 1] != ABSENT) G->wx[i] = oracle_weight(g[i], g[i + 1], beta, w_min);
                if (y + 1 < ny && code[i + sy] != ABSENT) G->wy[i] = oracle_weight(g[i], g[i + sy], beta, w_min);
                if (z + 1 < nz && code[i + sz] != ABSENT) G->wz[i] = oracle_weight(g[i], g[i + sz], beta, w_min);
            }
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int64_t i = z * sz + y * sy + x;
                double s = G->wx[i] + G->wy[i] + G->wz[i];
                if (x > 0) s += G->wx[i - 1];
                if (y > 0) s += G->wy[i - sy];
                if (z > 0) s += G->wz[i - sz];
                G->d[i] = s;
            }
}

static void graph_free(graph_t* G) {
    free(G->wx); free(G->wy); free(G->wz); free(G->d);
}

/* Sum over the 6 neighbours j of w_ij * v_j (v given on all voxels). */
static inline double nb_sum(const graph_t* G, const double* v, int x, int y, int z, int64_t i) {
    const int64_t sy = G->nx, sz = (int64_t)G->nx * G->ny;
    double s = 0.0;
    if (x + 1 < G->nx) s += G->wx[i] * v[i + 1];
    if (x > 0) s += G->wx[i - 1] * v[i - 1];
    if (y + 1 < G->ny) s += G->wy[i] * v[i + sy];
    if (y > 0) s += G->wy[i - sy] * v[i - sy];
    if (z + 1 < G->nz) s += G->wz[i] * v[i + sz];
    if (z > 0) s += G->wz[i - sz] * v[i - sz];
    return s;
}

/* q = L_U p on free voxels (p must be zero on non-free voxels), 0 elsewhere. */
static void apply_LU(const graph_t* G, const uint8_t* code, const double* p, double* q) {
    const int64_t sy = G->nx, sz = (int64_t)G->nx * G->ny;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < G->nz; ++z)
        for (int y = 0; y < G->ny; ++y)
            for (int x = 0; x < G->nx; ++x) {
                int64_t i = z * sz + y * sy + x;
                q[i] = (code[i] == FREE) ? G->d[i] * p[i] - nb_sum(G, p, x, y, z, i) : 0.0;
            }
}

/* Plane-ordered dot product over free voxels. */
static double dot_free(const graph_t* G, const uint8_t* code, const double* a, const double* b,
                       double* plane_acc) {
    const int64_t sz = (int64_t)G->nx * G->ny;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < G->nz; ++z) {
        double s = 0.0;
        for (int64_t k = 0; k < sz; ++k) {
            int64_t i = z * sz + k;
            if (code[i] == FREE) s += a[i] * b[i];
        }
        plane_acc[z] = s;
    }
    double s = 0.0;
    for (int z = 0; z < G->nz; ++z) s += plane_acc[z];
    return s;
}

/* Right-hand side b = -B^T x_M (+ rhs): b_i = sum over seeded neighbours j of
 * w_ij m_j, for free i.  xs holds the seed values on seeds, 0 elsewhere. */
static void build_rhs(const graph_t* G, const uint8_t* code, const double* xs, const double* rhs, double* b) {
    const int64_t sy = G->nx, sz = (int64_t)G->nx * G->ny;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < G->nz; ++z)
        for (int y = 0; y < G->ny; ++y)
            for (int x = 0; x < G->nx; ++x) {
                int64_t i = z * sz + y * sy + x;
                b[i] = (code[i] == FREE) ? nb_sum(G, xs, x, y, z, i) + (rhs ? rhs[i] : 0.0) : 0.0;
            }
}

double oracle_residual(int nx, int ny, int nz, const double* g, const uint8_t* code,
                       const double* x, const double* rhs, double beta, double w_min, double* r) {
    graph_t G;
    graph_build(&G, nx, ny, nz, g, code, beta, w_min);
    int64_t n = G.n;
    double* xs = (double*)calloc((size_t)n, sizeof(double));
    double* xu = (double*)calloc((size_t)n, sizeof(double));
    double* b = (double*)calloc((size_t)n, sizeof(double));
    double* q = (double*)calloc((size_t)n, sizeof(double));
    double* acc = (double*)calloc((size_t)nz, sizeof(double));
    for (int64_t i = 0; i < n; ++i) {
        xs[i] = (code[i] == SEED) ? x[i] : 0.0;
        xu[i] = (code[i] == FREE) ? x[i] : 0.0;
    }
    build_rhs(&G, code, xs, rhs, b);
    apply_LU(&G, code, xu, q);
    for (int64_t i = 0; i < n; ++i) r[i] = (code[i] == FREE) ? b[i] - q[i] : 0.0;
    double bb = dot_free(&G, code, b, b, acc);
    free(xs); free(xu); free(b); free(q); free(acc);
    graph_free(&G);
    return sqrt(bb);
}

/* Jacobi-preconditioned conjugate gradients (Sec. IV-D2 and Sec. V: CG with
 * Jacobi preconditioner; the initial guess is taken from xin).  Stops when
 * ||r||_2 <= tol ||b||_2 (relative to the right-hand side, a reading of the
 * paper's absolute 1e-2 criterion) or after max_iter iterations. */
int oracle_rw_solve(int nx, int ny, int nz, const double* g, const uint8_t* code,
                    const double* xin, const double* rhs, double beta, double w_min,
                    double tol, int max_iter, double* x, int* iters, double* relres) {
    int64_t n = (int64_t)nx * ny * nz;
    int64_t nseed = 0;
    for (int64_t i = 0; i < n; ++i) nseed += (code[i] == SEED);
    if (nseed == 0) return 2;

    graph_t G;
    graph_build(&G, nx, ny, nz, g, code, beta, w_min);
    double* xs = (double*)calloc((size_t)n, sizeof(double));
    double* b = (double*)calloc((size_t)n, sizeof(double));
    double* r = (double*)calloc((size_t)n, sizeof(double));
    double* zv = (double*)calloc((size_t)n, sizeof(double));
    double* p = (double*)calloc((size_t)n, sizeof(double));
    double* q = (double*)calloc((size_t)n, sizeof(double));
    double* acc = (double*)calloc((size_t)nz, sizeof(double));

    for (int64_t i = 0; i < n; ++i) {
        xs[i] = (code[i] == SEED) ? xin[i] : 0.0;
        /* unknowns start from the initial guess; a free vertex without any
         * edge (all neighbours absent) keeps it */
        x[i] = (code[i] == SEED) ? xin[i] : (code[i] == FREE ? xin[i] : 0.0);
    }
    build_rhs(&G, code, xs, rhs, b);
    double bnorm = sqrt(dot_free(&G, code, b, b, acc));
    int it = 0;
    int status = 0;
    if (bnorm == 0.0) {
        /* homogeneous system: x_U = 0 exactly */
        for (int64_t i = 0; i < n; ++i)
            if (code[i] == FREE) x[i] = 0.0;
    } else {
        /* r = b - A x,  z = D^-1 r,  p = z */
        for (int64_t i = 0; i < n; ++i) p[i] = (code[i] == FREE) ? x[i] : 0.0;
        apply_LU(&G, code, p, q);
        for (int64_t i = 0; i < n; ++i) {
            r[i] = (code[i] == FREE) ? b[i] - q[i] : 0.0;
            zv[i] = (code[i] == FREE && G.d[i] > 0.0) ? r[i] / G.d[i] : 0.0;
            p[i] = zv[i];
        }
        double rho = dot_free(&G, code, r, zv, acc);
        double rn = sqrt(dot_free(&G, code, r, r, acc));
        status = 3;
        if (rn <= tol * bnorm) status = 0;
        while (status != 0 && it < max_iter) {
            apply_LU(&G, code, p, q);
            double pq = dot_free(&G, code, p, q, acc);
            if (!(pq > 0.0)) break;
            double alpha = rho / pq;
            for (int64_t i = 0; i < n; ++i) {
                if (code[i] != FREE) continue;
                x[i] += alpha * p[i];
                r[i] -= alpha * q[i];
            }
            ++it;
            rn = sqrt(dot_free(&G, code, r, r, acc));
            if (rn <= tol * bnorm) { status = 0; break; }
            for (int64_t i = 0; i < n; ++i)
                zv[i] = (code[i] == FREE && G.d[i] > 0.0) ? r[i] / G.d[i] : 0.0;
            double rho_new = dot_free(&G, code, r, zv, acc);
            double bcg = rho_new / rho;
            rho = rho_new;
            for (int64_t i = 0; i < n; ++i) p[i] = (code[i] == FREE) ? zv[i] + bcg * p[i] : 0.0;
        }
    }
    if (relres) {
        /* true residual of the returned iterate */
        for (int64_t i = 0; i < n; ++i) p[i] = (code[i] == FREE) ? x[i] : 0.0;
        apply_LU(&G, code, p, q);
        for (int64_t i = 0; i < n; ++i) r[i] = (code[i] == FREE) ? b[i] - q[i] : 0.0;
        double tr = sqrt(dot_free(&G, code, r, r, acc));
        *relres = (bnorm > 0.0) ? tr / bnorm : tr;
    }
    if (iters) *iters = it;
    free(xs); free(b); free(r); free(zv); free(p); free(q); free(acc);
    graph_free(&G);
    return status;
}

/* Adjoint of the solve.  With A(w) x_U = b(w) and a loss l(x):
 *   dl/dw_ij = -(lambda_i - lambda_j)(x_i - x_j),  lambda = 0 on seeds,
 * which covers free-free edges (through A) and free-seed edges (through A
 * and b).  Chain rule through w = exp(-beta d^2), d = g_i - g_j (zero where
 * the w_min clamp is active):
 *   dw/dbeta = -d^2 w,  dw/dg_i = -2 beta d w,  dw/dg_j = +2 beta d w. */
double oracle_adjoint_grad(int nx, int ny, int nz, const double* g, const uint8_t* code,
                           const double* x, const double* lam, double beta, double w_min,
                           double* dg) {
    const int64_t sy = nx, sz = (int64_t)nx * ny;
    int64_t n = (int64_t)nx * ny * nz;
    double dbeta = 0.0;
    for (int64_t i = 0; i < n; ++i) dg[i] = 0.0;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x0 = 0; x0 < nx; ++x0) {
                int64_t i = z * sz + y * sy + x0;
                if (code[i] == ABSENT) continue;
                int64_t nbr[3] = {x0 + 1 < nx ? i + 1 : -1, y + 1 < ny ? i + sy : -1, z + 1 < nz ? i + sz : -1};
                for (int a = 0; a < 3; ++a) {
                    int64_t j = nbr[a];
                    if (j < 0 || code[j] == ABSENT) continue;
                    if (code[i] != FREE && code[j] != FREE) continue;
                    double li = (code[i] == FREE) ? lam[i] : 0.0;
                    double lj = (code[j] == FREE) ? lam[j] : 0.0;
                    double dl_dw = -(li - lj) * (x[i] - x[j]);
                    double d = g[i] - g[j];
                    double e = exp(-beta * d * d);
                    if (!(e > w_min)) continue; /* clamped: no dependence on g or beta */
                    dbeta += dl_dw * (-d * d * e);
                    dg[i] += dl_dw * (-2.0 * beta * d * e);
                    dg[j] += dl_dw * (2.0 * beta * d * e);
                }
            }
    return dbeta;
}
