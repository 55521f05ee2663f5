/* FP64 CPU oracle of the random walker — TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may load
 * this library.  It shares no code, header, table or constant with the CUDA
 * library; the product path never calls it.
 *
 * Layout: dense [z][y][x] arrays (x fastest), dims (nx, ny, nz).
 * Voxel codes: 0 = free (unknown), 1 = seed (Dirichlet value), 2 = absent
 * (not a vertex of the graph: no edges).
 */
#ifndef RW_ORACLE_H
#define RW_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Intensity normalisation window and unorm16 storage (FP32 arithmetic). */
void oracle_quantize_f32(const float* v, int64_t n, float lo, float hi, int normalize, uint16_t* q);
void oracle_quantize_u16(const uint16_t* v, int64_t n, float lo, float hi, int normalize, uint16_t* q);

/* One 2x2x2 mean-filter + downsample step of the LOD pyramid (Sec. III-A), FP32. */
void oracle_downsample(const float* fine, int nx, int ny, int nz, float* coarse);

/* Edge weight of Sec. III-B: max(exp(-beta (a-b)^2), w_min). */
double oracle_weight(double a, double b, double beta, double w_min);

/* Plain random walker (Sec. III-B): solve L_U x_U = -B^T x_M (plus optional
 * extra right-hand side on free voxels) by FP64 Jacobi-PCG.
 * xin: seed values at seeds, initial guess at free voxels.  x: full output.
 * Returns 0 ok, 2 no seeds, 3 not converged.  iters/relres may be NULL. */
int oracle_rw_solve(int nx, int ny, int nz, const double* g, const uint8_t* code,
                    const double* xin, const double* rhs, double beta, double w_min,
                    double tol, int max_iter, double* x, int* iters, double* relres);

/* r = b - A x over free voxels (0 elsewhere), FP64.  Returns ||b||_2. */
double oracle_residual(int nx, int ny, int nz, const double* g, const uint8_t* code,
                       const double* x, const double* rhs, double beta, double w_min, double* r);

/* Gradient of a loss through the solve (adjoint, Sec. III-B system):
 * given x (the solution) and lambda (solution of A lambda = dl/dx_U, zero on
 * seeds), accumulate dl/dg per voxel and return dl/dbeta. */
double oracle_adjoint_grad(int nx, int ny, int nz, const double* g, const uint8_t* code,
                           const double* x, const double* lam, double beta, double w_min,
                           double* dg);

int oracle_num_threads(void);

#ifdef __cplusplus
}
#endif
#endif
