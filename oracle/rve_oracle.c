/*
 * rve_oracle.c -- plain FP64 CPU oracle for the RVE corrector method of
 * Khoromskaia, Khoromskij & Otto, "Numerical study in stochastic
 * homogenization for elliptic PDEs: convergence rate in the size of
 * representative volume elements" (arXiv:1903.12227).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product path
 * (the CUDA library and its Python binding) never calls it, and shares no
 * code, header or table with it.
 *
 * What it computes, step by step, in the order of the paper:
 *   1. the random covered set G = union of square inclusions (Sec. 2, Eq.
 *      "Stoch-decomp", coefficient Eq. "coef_diag");
 *   2. the sparse Galerkin stiffness matrix, assembled as a sum over cells of
 *      local Kronecker products a_c (K1 (x) M1 + M1 (x) K1) inserted at the
 *      cell's (periodically wrapped) nodes (Sec. 3.2-3.3, Eq. "As_Kron");
 *   3. the Galerkin right-hand sides f_i = -int a d_i psi (Eq.
 *      "FEM_discr_RHS"), with the stiffness's own quadrature (Sec. 4.3);
 *   4. preconditioned CG (Sec. 3.4) with B = c0 A_Delta + delta I, A_Delta the
 *      periodic 5-point finite-difference Laplacian (Eq. "Lap_Kron",
 *      "BC_Neu_peri"), inverted by a plain radix-2 complex FFT written here;
 *   5. the homogenized matrix, in the energy form (Eq. "wg01" rewritten as in
 *      the symmetry argument of Sec. 4.3) and the flux form (Eq.
 *      "Ahom_m_entry"), each integrated cell by cell from its definition;
 *   6. the derivative of the energy form with respect to each cell value;
 *   7. ensemble statistics: empirical mean (Eq. "A_hom_Empir"), the paper's
 *      standard-deviation estimators (Eqs. "Var1", "Var2") and the rescaled
 *      covariance / quartic tensor (Eq. "quartic");
 *   8. for a general load (the FEM convergence test of Sec. 3.5): the mass
 *      matrix M1 (x) M1 applied cell by cell, and the solve A u = b;
 *   9. the 3D extension (Sec. 2: the setting carries over to d > 2; Sec.
 *      3.1-3.2 and Eq. "As_Kron_d": multilinear elements on cubes and the
 *      rank-3 Kronecker Laplacian): cubes, the trilinear element
 *      K1(x)M1(x)M1 + M1(x)K1(x)M1 + M1(x)M1(x)K1, the 7-point Laplacian
 *      preconditioner, three correctors, 3x3 A_hom.
 *
 * Readings of the paper that this oracle fixes (where it is silent or
 * garbled) are listed beside each function.  Everything is FP64.
 *
 * Grid: n = L*m0 unique nodes per axis on the torus [0,L)^2, h = 1/m0.
 * Node (i1,i2) sits at (i1 h, i2 h); cell (c1,c2) is the square with lower
 * left node (c1,c2).  Linear index i1*n + i2 (big-endian order, Sec. 3.2).
 */
#include "rve_oracle.h"

#define ORC_PI 3.14159265358979323846264338327950288

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* 1. Random field                                                           */
/* ------------------------------------------------------------------------ */

/* SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): the k-th output (k = 1, 2, ...) of the stream
 * seeded with s is mix(s + k * GAMMA). */
#define ORC_GAMMA 0x9E3779B97F4A7C15ULL

uint64_t orc_splitmix64_mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t orc_splitmix64_output(uint64_t seed, uint64_t k)
{
    return orc_splitmix64_mix(seed + k * ORC_GAMMA);
}

/* Per-realization key: output number (index+1) of the stream seeded by the
 * run seed, so realization k of a run is a pure function of (seed, k). */
uint64_t orc_realization_key(uint64_t seed, uint64_t index)
{
    return orc_splitmix64_output(seed, index + 1);
}

/* Draw number `ctr` under tag `tag` from a realization's key. */
uint64_t orc_draw(uint64_t key, uint32_t tag, uint64_t ctr)
{
    return orc_splitmix64_output(key, ((uint64_t)tag << 40) + ctr + 1);
}

/* Uniform integer in [0, n): the high 64 bits of the 128-bit product
 * (Lemire, ACM TOMS 2019, without the rejection step).  For n = 2^p this is
 * the top p bits of the draw. */
static uint32_t orc_uniform_below(uint64_t v, uint32_t n)
{
    unsigned __int128 prod = (unsigned __int128)v * (unsigned __int128)n;
    return (uint32_t)(prod >> 64);
}

void orc_corners(const orc_realization* r, int32_t* corners)
{
    const uint32_t n = (uint32_t)(r->L * r->m0);
    const uint64_t key = orc_realization_key(r->seed, r->index);
    for (int64_t k = 0; k < r->n_incl; ++k) {
        corners[2 * k + 0] = (int32_t)orc_uniform_below(
            orc_draw(key, ORC_TAG_CORNER, (uint64_t)(2 * k + 0)), n);
        corners[2 * k + 1] = (int32_t)orc_uniform_below(
            orc_draw(key, ORC_TAG_CORNER, (uint64_t)(2 * k + 1)), n);
    }
}

/* Covered set as the union of the inclusions (Eq. "Stoch-decomp"): every
 * inclusion marks its s x s cells, wrapping periodically.  mask[c1*n+c2]. */
void orc_gen_field(const orc_realization* r, uint8_t* mask)
{
    const int64_t n = (int64_t)r->L * r->m0;
    const int64_t s = r->incl_cells;
    memset(mask, 0, (size_t)(n * n));
    int32_t* c = (int32_t*)malloc(sizeof(int32_t) * 2 * (size_t)(r->n_incl > 0 ? r->n_incl : 1));
    orc_corners(r, c);
    for (int64_t k = 0; k < r->n_incl; ++k)
        for (int64_t d1 = 0; d1 < s; ++d1)
            for (int64_t d2 = 0; d2 < s; ++d2) {
                int64_t i1 = (c[2 * k] + d1) % n;
                int64_t i2 = (c[2 * k + 1] + d2) % n;
                mask[i1 * n + i2] = 1;
            }
    free(c);
}

/* Coefficient a = a_matrix outside and a_incl inside the covered set
 * (Eq. "coef_diag" with the two values given explicitly). */
void orc_coef_from_mask(int64_t n, const uint8_t* mask, double a_matrix,
                        double a_incl, double* coef)
{
    for (int64_t c = 0; c < n * n; ++c) coef[c] = mask[c] ? a_incl : a_matrix;
}

/* ------------------------------------------------------------------------ */
/* 2. Local Kronecker element matrix and sparse assembly                     */
/* ------------------------------------------------------------------------ */

/* 1D P1 element matrices on an interval of length h (midpoint/exact rule,
 * Eq. "stiff_matrix_1point"): stiffness K1 = (1/h)[1 -1; -1 1]; mass
 * M1 = (h/6)[2 1; 1 2] (consistent) or (h/2) I (trapezoid, the paper's
 * lumped I-hat of Eq. "As_Kron").  The 2D element matrix of the Q1 square is
 * E = K1 (x) M1 + M1 (x) K1 (rank-2 Kronecker form of Sec. 3.2); local node
 * order (a1,a2) = 00, 01, 10, 11 (a1 slow, as the big-endian index). */
void orc_element_matrix(int scheme, double h, double E[16])
{
    double K1[2][2] = {{1.0 / h, -1.0 / h}, {-1.0 / h, 1.0 / h}};
    double M1[2][2];
    if (scheme == ORC_SCHEME_LUMPED) {
        M1[0][0] = h / 2; M1[0][1] = 0; M1[1][0] = 0; M1[1][1] = h / 2;
    } else {
        M1[0][0] = 2 * h / 6; M1[0][1] = h / 6; M1[1][0] = h / 6; M1[1][1] = 2 * h / 6;
    }
    for (int a1 = 0; a1 < 2; ++a1)
        for (int a2 = 0; a2 < 2; ++a2)
            for (int b1 = 0; b1 < 2; ++b1)
                for (int b2 = 0; b2 < 2; ++b2) {
                    int row = a1 * 2 + a2, col = b1 * 2 + b2;
                    /* Kronecker product (A (x) B)[(a1,a2),(b1,b2)] = A[a1][b1] B[a2][b2] */
                    E[row * 4 + col] = K1[a1][b1] * M1[a2][b2] + M1[a1][b1] * K1[a2][b2];
                }
}

/* Global node numbers of cell (c1,c2)'s four corners in local order. */
static void orc_cell_nodes(int64_t n, int64_t c1, int64_t c2, int64_t g[4])
{
    int64_t p1 = (c1 + 1) % n, p2 = (c2 + 1) % n;
    g[0] = c1 * n + c2;
    g[1] = c1 * n + p2;
    g[2] = p1 * n + c2;
    g[3] = p1 * n + p2;
}

typedef struct { int64_t row, col; double val; } orc_triplet;

static int orc_triplet_cmp(const void* a, const void* b)
{
    const orc_triplet* x = (const orc_triplet*)a;
    const orc_triplet* y = (const orc_triplet*)b;
    if (x->row != y->row) return x->row < y->row ? -1 : 1;
    if (x->col != y->col) return x->col < y->col ? -1 : 1;
    return 0;
}

/* A = sum_c a_c * P_c^T E P_c, i.e. the per-cell Kronecker blocks of Eq.
 * "As_Kron" inserted at the cell's nodes; the periodic wrap is the torus
 * itself (wrap cells carry their own coefficient).  COO -> CSR with the
 * duplicates summed.  Returns nnz; rowptr has n*n+1 entries and colidx/vals
 * room for 9*n*n entries. */
int64_t orc_assemble(int64_t n, double h, const double* coef, int scheme,
                     int64_t* rowptr, int64_t* colidx, double* vals)
{
    double E[16];
    orc_element_matrix(scheme, h, E);
    const int64_t N = n * n;
    orc_triplet* t = (orc_triplet*)malloc(sizeof(orc_triplet) * (size_t)(16 * N));
    int64_t nt = 0;
    for (int64_t c1 = 0; c1 < n; ++c1)
        for (int64_t c2 = 0; c2 < n; ++c2) {
            int64_t g[4];
            orc_cell_nodes(n, c1, c2, g);
            double a = coef[c1 * n + c2];
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) {
                    t[nt].row = g[i];
                    t[nt].col = g[j];
                    t[nt].val = a * E[i * 4 + j];
                    ++nt;
                }
        }
    qsort(t, (size_t)nt, sizeof(orc_triplet), orc_triplet_cmp);
    int64_t nnz = 0;
    for (int64_t r = 0; r <= N; ++r) rowptr[r] = 0;
    for (int64_t k = 0; k < nt; ++k) {
        if (k > 0 && t[k].row == t[k - 1].row && t[k].col == t[k - 1].col) {
            vals[nnz - 1] += t[k].val;            /* duplicate (row,col): sum */
        } else {
            colidx[nnz] = t[k].col;
            vals[nnz] = t[k].val;
            rowptr[t[k].row + 1] += 1;            /* count entries per row */
            ++nnz;
        }
    }
    for (int64_t r = 0; r < N; ++r) rowptr[r + 1] += rowptr[r];
    free(t);
    return nnz;
}

void orc_spmv(int64_t N, const int64_t* rowptr, const int64_t* colidx,
              const double* vals, const double* x, double* y)
{
    for (int64_t r = 0; r < N; ++r) {
        double s = 0.0;
        for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) s += vals[k] * x[colidx[k]];
        y[r] = s;
    }
}

/* ------------------------------------------------------------------------ */
/* 3. Right-hand sides                                                        */
/* ------------------------------------------------------------------------ */

/* Nodal values xi_i of the affine function x_i on one cell (local order
 * 00,01,10,11): x_1 = a1 h, x_2 = a2 h. */
static void orc_xi(int i, double h, double xi[4])
{
    const int a1[4] = {0, 0, 1, 1}, a2[4] = {0, 1, 0, 1};
    for (int k = 0; k < 4; ++k) xi[k] = (i == 0 ? a1[k] : a2[k]) * h;
}

/* f_i = -int a grad(psi) . e_i = -sum_c a_c P_c^T E xi_i, since on each cell
 * e_i = grad x_i and x_i lies in the local Q1 space (Galerkin RHS of Eq.
 * "FEM_discr_RHS" with the stiffness's quadrature).  f[i*N + node]. */
void orc_rhs(int64_t n, double h, const double* coef, int scheme, double* f)
{
    double E[16];
    orc_element_matrix(scheme, h, E);
    const int64_t N = n * n;
    memset(f, 0, sizeof(double) * 2 * (size_t)N);
    for (int i = 0; i < 2; ++i) {
        double xi[4], Exi[4];
        orc_xi(i, h, xi);
        for (int r = 0; r < 4; ++r) {
            Exi[r] = 0;
            for (int c = 0; c < 4; ++c) Exi[r] += E[r * 4 + c] * xi[c];
        }
        for (int64_t c1 = 0; c1 < n; ++c1)
            for (int64_t c2 = 0; c2 < n; ++c2) {
                int64_t g[4];
                orc_cell_nodes(n, c1, c2, g);
                double a = coef[c1 * n + c2];
                for (int r = 0; r < 4; ++r) f[i * N + g[r]] -= a * Exi[r];
            }
    }
}

/* ------------------------------------------------------------------------ */
/* 4. Preconditioner and PCG                                                  */
/* ------------------------------------------------------------------------ */

/* In-place iterative radix-2 complex FFT of length n (power of two):
 * sign = -1 forward (exp(-2 pi i jk/n)), +1 backward (unnormalised). */
static void orc_fft1d(int64_t n, double* re, double* im, int sign)
{
    for (int64_t i = 1, j = 0; i < n; ++i) {
        int64_t bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            double tr = re[i]; re[i] = re[j]; re[j] = tr;
            double ti = im[i]; im[i] = im[j]; im[j] = ti;
        }
    }
    for (int64_t len = 2; len <= n; len <<= 1) {
        for (int64_t i = 0; i < n; i += len)
            for (int64_t k = 0; k < len / 2; ++k) {
                double ang = sign * 2.0 * ORC_PI * (double)k / (double)len;
                double wr = cos(ang), wi = sin(ang);
                int64_t a = i + k, b = i + k + len / 2;
                double xr = re[b] * wr - im[b] * wi;
                double xi = re[b] * wi + im[b] * wr;
                re[b] = re[a] - xr; im[b] = im[a] - xi;
                re[a] += xr; im[a] += xi;
            }
    }
}

/* 2D FFT: every row, then every column. */
static void orc_fft2d(int64_t n, double* re, double* im, int sign)
{
    double* cr = (double*)malloc(sizeof(double) * (size_t)n);
    double* ci = (double*)malloc(sizeof(double) * (size_t)n);
    for (int64_t i1 = 0; i1 < n; ++i1) orc_fft1d(n, re + i1 * n, im + i1 * n, sign);
    for (int64_t i2 = 0; i2 < n; ++i2) {
        for (int64_t i1 = 0; i1 < n; ++i1) { cr[i1] = re[i1 * n + i2]; ci[i1] = im[i1 * n + i2]; }
        orc_fft1d(n, cr, ci, sign);
        for (int64_t i1 = 0; i1 < n; ++i1) { re[i1 * n + i2] = cr[i1]; im[i1 * n + i2] = ci[i1]; }
    }
    free(cr);
    free(ci);
}

/* Eigenvalue of the periodic 5-point Laplacian A_Delta (Eq. "Lap_Kron"
 * with the periodic 1D matrix Delta_P of Eq. "BC_Neu_peri", sign flipped so
 * that A_Delta is positive semidefinite) at frequency (k1,k2). */
double orc_laplacian_eig(int64_t n, int64_t k1, int64_t k2)
{
    double s1 = sin(ORC_PI * (double)k1 / (double)n);
    double s2 = sin(ORC_PI * (double)k2 / (double)n);
    return 4.0 * s1 * s1 + 4.0 * s2 * s2;
}

/* z = B^{-1} r with B = c0 A_Delta + delta I (Sec. 3.4).  delta = 0 reads
 * as the delta -> 0 limit on the mean-zero subspace: the constant mode of
 * z is set to zero. */
void orc_precond(int64_t n, double c0, double delta, const double* r, double* z)
{
    const int64_t N = n * n;
    if (n < 1 || (n & (n - 1)) != 0) {           /* radix-2 FFT: n = 2^p */
        for (int64_t k = 0; k < N; ++k) z[k] = NAN;
        return;
    }
    double* re = (double*)malloc(sizeof(double) * (size_t)N);
    double* im = (double*)calloc((size_t)N, sizeof(double));
    memcpy(re, r, sizeof(double) * (size_t)N);
    orc_fft2d(n, re, im, -1);
    for (int64_t k1 = 0; k1 < n; ++k1)
        for (int64_t k2 = 0; k2 < n; ++k2) {
            double sigma = c0 * orc_laplacian_eig(n, k1, k2) + delta;
            double inv = (k1 == 0 && k2 == 0 && delta == 0.0) ? 0.0 : 1.0 / sigma;
            re[k1 * n + k2] *= inv;
            im[k1 * n + k2] *= inv;
        }
    orc_fft2d(n, re, im, +1);
    for (int64_t k = 0; k < N; ++k) z[k] = re[k] / (double)N;
    free(re);
    free(im);
}

static double orc_dot(int64_t N, const double* a, const double* b)
{
    double s = 0.0;
    for (int64_t k = 0; k < N; ++k) s += a[k] * b[k];
    return s;
}

/* Preconditioned CG (Saad, Iterative Methods for Sparse Linear Systems,
 * 2nd ed., Algorithm 9.1) from u = 0, stopped when the recursive residual
 * satisfies ||r|| <= tol ||f|| (MATLAB pcg's relative-residual rule, Sec.
 * 3.4).  The solution is returned with zero mean.  Returns the number of
 * operator applications (iterations); *relres_true gets ||f-Au||/||f||.
 * f = 0 gives u = 0 after 0 iterations. */
int orc_pcg(int64_t n, const int64_t* rowptr, const int64_t* colidx,
            const double* vals, double c0, double delta, const double* f,
            double tol, int max_iter, double* u, double* relres_true)
{
    const int64_t N = n * n;
    double* r = (double*)malloc(sizeof(double) * (size_t)N);
    double* z = (double*)malloc(sizeof(double) * (size_t)N);
    double* p = (double*)malloc(sizeof(double) * (size_t)N);
    double* q = (double*)malloc(sizeof(double) * (size_t)N);
    memset(u, 0, sizeof(double) * (size_t)N);
    memcpy(r, f, sizeof(double) * (size_t)N);
    double fnorm = sqrt(orc_dot(N, f, f));
    int it = 0;
    if (fnorm > 0.0) {
        orc_precond(n, c0, delta, r, z);
        memcpy(p, z, sizeof(double) * (size_t)N);
        double rz = orc_dot(N, r, z);
        while (it < max_iter) {
            orc_spmv(N, rowptr, colidx, vals, p, q);
            ++it;
            double alpha = rz / orc_dot(N, p, q);
            for (int64_t k = 0; k < N; ++k) { u[k] += alpha * p[k]; r[k] -= alpha * q[k]; }
            if (sqrt(orc_dot(N, r, r)) <= tol * fnorm) break;
            orc_precond(n, c0, delta, r, z);
            double rz_new = orc_dot(N, r, z);
            double beta = rz_new / rz;
            rz = rz_new;
            for (int64_t k = 0; k < N; ++k) p[k] = z[k] + beta * p[k];
        }
    }
    double mean = 0.0;
    for (int64_t k = 0; k < N; ++k) mean += u[k];
    mean /= (double)N;
    for (int64_t k = 0; k < N; ++k) u[k] -= mean;
    if (relres_true) {
        orc_spmv(N, rowptr, colidx, vals, u, q);
        double s = 0.0;
        for (int64_t k = 0; k < N; ++k) s += (f[k] - q[k]) * (f[k] - q[k]);
        *relres_true = fnorm > 0.0 ? sqrt(s) / fnorm : 0.0;
    }
    free(r); free(z); free(p); free(q);
    return it;
}

/* ------------------------------------------------------------------------ */
/* 5-6. Homogenized matrix and its gradient                                   */
/* ------------------------------------------------------------------------ */

/* Local nodal values of x_i + phi_i on cell (c1,c2). */
static void orc_local_v(int64_t n, double h, const double* u_i, int i,
                        int64_t c1, int64_t c2, double v[4])
{
    int64_t g[4];
    double xi[4];
    orc_cell_nodes(n, c1, c2, g);
    orc_xi(i, h, xi);
    for (int k = 0; k < 4; ++k) v[k] = xi[k] + u_i[g[k]];
}

/* Energy form a_ij = (1/L^2) int (e_j + grad phi_j) . a (e_i + grad phi_i),
 * integrated exactly cell by cell with the element matrix (the quadrature of
 * the stiffness, Sec. 4.3), and the flux form of Eq. "Ahom_m_entry",
 * a_ij = (1/L^2) int a (delta_ij + d_j phi_i), whose cell integral of the
 * bilinear d_j(x_i+phi_i) is h/2 times the difference of the two edge sums
 * across direction j.  A[2*i + j]. */
void orc_a_hom(int64_t n, double h, double Lsize, const double* coef, int scheme,
               const double* u /* [2][N] */, double* A_energy, double* A_flux)
{
    double E[16];
    orc_element_matrix(scheme, h, E);
    const int64_t N = n * n;
    double en[4] = {0, 0, 0, 0}, fl[4] = {0, 0, 0, 0};
    for (int64_t c1 = 0; c1 < n; ++c1)
        for (int64_t c2 = 0; c2 < n; ++c2) {
            double a = coef[c1 * n + c2];
            double v[2][4];
            orc_local_v(n, h, u, 0, c1, c2, v[0]);
            orc_local_v(n, h, u + N, 1, c1, c2, v[1]);
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) {
                    double s = 0.0;
                    for (int r = 0; r < 4; ++r)
                        for (int c = 0; c < 4; ++c) s += v[j][r] * E[r * 4 + c] * v[i][c];
                    en[2 * i + j] += a * s;
                    /* int_cell d_1 w = h/2 (w10 + w11 - w00 - w01),
                       int_cell d_2 w = h/2 (w01 + w11 - w00 - w10) */
                    double d = (j == 0) ? 0.5 * h * (v[i][2] + v[i][3] - v[i][0] - v[i][1])
                                        : 0.5 * h * (v[i][1] + v[i][3] - v[i][0] - v[i][2]);
                    fl[2 * i + j] += a * d;
                }
        }
    const double vol = Lsize * Lsize;
    for (int k = 0; k < 4; ++k) {
        if (A_energy) A_energy[k] = en[k] / vol;
        if (A_flux) A_flux[k] = fl[k] / vol;
    }
}

/* d(sum_ij G_ij a^E_ij)/d a_c = (1/L^2) sum_ij G_ij int_cell (e_i + grad
 * phi_i).(e_j + grad phi_j): each a^E_ij is (a polarisation of) a minimum
 * of a quadratic energy in phi, so only the explicit dependence on a_c
 * survives.  grad[c1*n + c2]. */
void orc_a_hom_grad(int64_t n, double h, double Lsize, int scheme,
                    const double* u, const double G[4], double* grad)
{
    double E[16];
    orc_element_matrix(scheme, h, E);
    const int64_t N = n * n;
    const double vol = Lsize * Lsize;
    for (int64_t c1 = 0; c1 < n; ++c1)
        for (int64_t c2 = 0; c2 < n; ++c2) {
            double v[2][4];
            orc_local_v(n, h, u, 0, c1, c2, v[0]);
            orc_local_v(n, h, u + N, 1, c1, c2, v[1]);
            double g = 0.0;
            for (int i = 0; i < 2; ++i)
                for (int j = 0; j < 2; ++j) {
                    double s = 0.0;
                    for (int r = 0; r < 4; ++r)
                        for (int c = 0; c < 4; ++c) s += v[i][r] * E[r * 4 + c] * v[j][c];
                    g += G[2 * i + j] * s;
                }
            grad[c1 * n + c2] = g / vol;
        }
}

/* ------------------------------------------------------------------------ */
/* Whole realization                                                          */
/* ------------------------------------------------------------------------ */

int orc_solve_coef(int64_t L, int64_t m0, const double* coef, double c0,
                   int scheme, double tol, int max_iter, double delta,
                   double* u /* [2][N] or NULL */, orc_result* res)
{
    const int64_t n = L * m0;
    const int64_t N = n * n;
    const double h = 1.0 / (double)m0;
    if (n < 2 || (n & (n - 1)) != 0) return -2;   /* radix-2 FFT: n = 2^p */
    int64_t* rowptr = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N + 1));
    int64_t* colidx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(9 * N));
    double* vals = (double*)malloc(sizeof(double) * (size_t)(9 * N));
    double* f = (double*)malloc(sizeof(double) * (size_t)(2 * N));
    double* uu = u ? u : (double*)malloc(sizeof(double) * (size_t)(2 * N));
    if (!rowptr || !colidx || !vals || !f || !uu) return -1;
    orc_assemble(n, h, coef, scheme, rowptr, colidx, vals);
    orc_rhs(n, h, coef, scheme, f);
    for (int i = 0; i < 2; ++i) {
        double rr = 0.0;
        res->iters[i] = orc_pcg(n, rowptr, colidx, vals, c0, delta, f + i * N, tol,
                                max_iter, uu + i * N, &rr);
        res->relres_true[i] = rr;
    }
    orc_a_hom(n, h, (double)L, coef, scheme, uu, res->A_energy, res->A_flux);
    double s = 0.0;
    for (int64_t k = 0; k < N; ++k) s += coef[k];
    res->mean_a = s / (double)N;
    free(rowptr); free(colidx); free(vals); free(f);
    if (!u) free(uu);
    return 0;
}

/* Element mass matrix M1 (x) M1 in local order 00, 01, 10, 11, with the 1D
 * mass of the scheme: consistent (h/6)[[2,1],[1,2]], lumped (h/2) I. */
void orc_mass_element(int scheme, double h, double M[16])
{
    double M1[2][2];
    if (scheme == ORC_SCHEME_LUMPED) {
        M1[0][0] = h / 2; M1[0][1] = 0; M1[1][0] = 0; M1[1][1] = h / 2;
    } else {
        M1[0][0] = 2 * h / 6; M1[0][1] = h / 6; M1[1][0] = h / 6; M1[1][1] = 2 * h / 6;
    }
    for (int a1 = 0; a1 < 2; ++a1)
        for (int a2 = 0; a2 < 2; ++a2)
            for (int b1 = 0; b1 < 2; ++b1)
                for (int b2 = 0; b2 < 2; ++b2)
                    M[(a1 * 2 + a2) * 4 + b1 * 2 + b2] = M1[a1][b1] * M1[a2][b2];
}

/* y = M x: the global mass matrix applied cell by cell (sum over cells of
 * P_c^T M_elem P_c x), periodic. */
void orc_apply_mass(int64_t n, double h, int scheme, const double* x, double* y)
{
    double M[16];
    orc_mass_element(scheme, h, M);
    memset(y, 0, sizeof(double) * (size_t)(n * n));
    for (int64_t c1 = 0; c1 < n; ++c1)
        for (int64_t c2 = 0; c2 < n; ++c2) {
            int64_t g[4];
            orc_cell_nodes(n, c1, c2, g);
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) y[g[i]] += M[i * 4 + j] * x[g[j]];
        }
}

/* A u = b for a mean-zero load vector b (assembled stiffness, PCG with the
 * FFT preconditioner); u is returned mean-zero.  Returns the iterations,
 * or -2 when n is not a power of two. */
int orc_solve_load(int64_t L, int64_t m0, const double* coef, double c0, int scheme,
                   const double* b, double tol, int max_iter, double delta, double* u,
                   double* relres_true)
{
    const int64_t n = L * m0;
    const int64_t N = n * n;
    const double h = 1.0 / (double)m0;
    if (n < 2 || (n & (n - 1)) != 0) return -2;
    int64_t* rowptr = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N + 1));
    int64_t* colidx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(9 * N));
    double* vals = (double*)malloc(sizeof(double) * (size_t)(9 * N));
    if (!rowptr || !colidx || !vals) return -1;
    orc_assemble(n, h, coef, scheme, rowptr, colidx, vals);
    const int it = orc_pcg(n, rowptr, colidx, vals, c0, delta, b, tol, max_iter, u, relres_true);
    free(rowptr); free(colidx); free(vals);
    return it;
}

int orc_solve_realization(const orc_realization* r, int scheme, double tol,
                          int max_iter, double delta, uint8_t* mask_out,
                          double* u, orc_result* res)
{
    const int64_t n = (int64_t)r->L * r->m0;
    const int64_t N = n * n;
    uint8_t* mask = mask_out ? mask_out : (uint8_t*)malloc((size_t)N);
    double* coef = (double*)malloc(sizeof(double) * (size_t)N);
    orc_gen_field(r, mask);
    orc_coef_from_mask(n, mask, r->a_matrix, r->a_incl, coef);
    double c0 = 0.5 * (r->a_matrix + r->a_incl);
    int rc = orc_solve_coef(r->L, r->m0, coef, c0, scheme, tol, max_iter, delta, u, res);
    free(coef);
    if (!mask_out) free(mask);
    return rc;
}

/* Many realizations, one per OpenMP thread (used to time the CPU baseline).
 * Returns the number of threads used. */
int orc_solve_batch(const orc_realization* r, int batch, int scheme, double tol,
                    int max_iter, double delta, orc_result* res, int threads)
{
    int used = 1;
#ifdef _OPENMP
    /* the thread count applies to this call only (omp_set_num_threads would
     * carry it over to every later call in the process); 0 = the default
     * team size (OMP_NUM_THREADS, else every core) */
    const int nt = threads > 0 ? threads : omp_get_max_threads();
#pragma omp parallel num_threads(nt)
    {
#pragma omp single
        used = omp_get_num_threads();
#pragma omp for schedule(dynamic, 1)
        for (int b = 0; b < batch; ++b)
            orc_solve_realization(&r[b], scheme, tol, max_iter, delta, NULL, NULL, &res[b]);
    }
#else
    (void)threads;
    for (int b = 0; b < batch; ++b)
        orc_solve_realization(&r[b], scheme, tol, max_iter, delta, NULL, NULL, &res[b]);
#endif
    return used;
}

/* ------------------------------------------------------------------------ */
/* 7. Ensemble statistics                                                     */
/* ------------------------------------------------------------------------ */

/* A: [N][4] row-major (a11,a12,a21,a22).  Outputs: mean[4]; var[4] unbiased
 * (N-1); std12_paper = sqrt(mean a12^2) (Eq. "Var1"); stddiff_paper =
 * sqrt(mean (a11-a22)^2) (Eq. "Var2"); Q[16] = L^d/(N-1) sum (A-mean)(x)2
 * as the 4x4 Kronecker unfolding of Eq. "quartic": Q[4*p+q] with p,q over
 * the entries in (a11,a12,a21,a22) order. */
void orc_statistics(int64_t N, const double* A, double L, int d, double* mean,
                    double* var, double* std12_paper, double* stddiff_paper, double* Q)
{
    for (int k = 0; k < 4; ++k) {
        double s = 0.0;
        for (int64_t m = 0; m < N; ++m) s += A[4 * m + k];
        mean[k] = s / (double)N;
    }
    double s12 = 0.0, sd = 0.0;
    for (int64_t m = 0; m < N; ++m) {
        s12 += A[4 * m + 1] * A[4 * m + 1];
        double d = A[4 * m + 0] - A[4 * m + 3];
        sd += d * d;
    }
    *std12_paper = sqrt(s12 / (double)N);
    *stddiff_paper = sqrt(sd / (double)N);
    double scale = pow(L, (double)d) / (double)(N - 1);
    for (int p = 0; p < 4; ++p)
        for (int q = 0; q < 4; ++q) {
            double s = 0.0;
            for (int64_t m = 0; m < N; ++m)
                s += (A[4 * m + p] - mean[p]) * (A[4 * m + q] - mean[q]);
            Q[4 * p + q] = scale * s;
        }
    for (int k = 0; k < 4; ++k) var[k] = Q[4 * k + k] / pow(L, (double)d);
}

/* The same for 3D: A [N][9] row-major; Q[81] = L^3/(N-1) sum (A-mean)(x)2,
 * Q[9*p+q] with p, q over the entries a11 .. a33. */
void orc3_statistics(int64_t N, const double* A, double L, double* mean, double* var, double* Q)
{
    for (int k = 0; k < 9; ++k) {
        double s = 0.0;
        for (int64_t m = 0; m < N; ++m) s += A[9 * m + k];
        mean[k] = s / (double)N;
    }
    const double L3 = L * L * L;
    for (int p = 0; p < 9; ++p)
        for (int q = 0; q < 9; ++q) {
            double s = 0.0;
            for (int64_t m = 0; m < N; ++m)
                s += (A[9 * m + p] - mean[p]) * (A[9 * m + q] - mean[q]);
            Q[9 * p + q] = L3 * s / (double)(N - 1);
        }
    for (int k = 0; k < 9; ++k) var[k] = Q[9 * k + k] / L3;
}

/* ------------------------------------------------------------------------ */
/* 9. The 3D extension (the paper's remark on 3D): cubes, trilinear Q1       */
/* ------------------------------------------------------------------------ */
/* Grid: n = L*m0 nodes per axis on the torus [0,L)^3, node (i1,i2,i3) at
 * index (i1*n + i2)*n + i3; cell (c1,c2,c3) has lower corner node (c1,c2,c3);
 * local corner a = 4 a1 + 2 a2 + a3 (a_k in {0,1}).  Correctors u_1..u_3
 * stored [3][N]. */

/* Covered set: N_inc cubes of side s (cells) with lower corners drawn from
 * the counter RNG (tag 1, draws 3k, 3k+1, 3k+2 per cube), periodic wrap. */
void orc3_gen_field(const orc_realization* r, uint8_t* mask)
{
    const int64_t n = (int64_t)r->L * r->m0, s = r->incl_cells;
    memset(mask, 0, (size_t)(n * n * n));
    const uint64_t key = orc_realization_key(r->seed, r->index);
    for (int64_t k = 0; k < r->n_incl; ++k) {
        int64_t c[3];
        for (int a = 0; a < 3; ++a) {
            const uint64_t v = orc_draw(key, 1, 3 * (uint64_t)k + (uint64_t)a);
            c[a] = (int64_t)(((unsigned __int128)v * (uint64_t)n) >> 64);
        }
        for (int64_t d1 = 0; d1 < s; ++d1)
            for (int64_t d2 = 0; d2 < s; ++d2)
                for (int64_t d3 = 0; d3 < s; ++d3)
                    mask[(((c[0] + d1) % n) * n + (c[1] + d2) % n) * n + (c[2] + d3) % n] = 1;
    }
}

/* Element matrix K1 (x) M1 (x) M1 + M1 (x) K1 (x) M1 + M1 (x) M1 (x) K1. */
void orc3_element_matrix(int scheme, double h, double E[64])
{
    double K1[2][2] = {{1.0 / h, -1.0 / h}, {-1.0 / h, 1.0 / h}};
    double M1[2][2];
    if (scheme == ORC_SCHEME_LUMPED) {
        M1[0][0] = h / 2; M1[0][1] = 0; M1[1][0] = 0; M1[1][1] = h / 2;
    } else {
        M1[0][0] = 2 * h / 6; M1[0][1] = h / 6; M1[1][0] = h / 6; M1[1][1] = 2 * h / 6;
    }
    for (int a = 0; a < 8; ++a)
        for (int b = 0; b < 8; ++b) {
            const int a1 = a >> 2, a2 = (a >> 1) & 1, a3 = a & 1;
            const int b1 = b >> 2, b2 = (b >> 1) & 1, b3 = b & 1;
            E[a * 8 + b] = K1[a1][b1] * M1[a2][b2] * M1[a3][b3] +
                           M1[a1][b1] * K1[a2][b2] * M1[a3][b3] +
                           M1[a1][b1] * M1[a2][b2] * K1[a3][b3];
        }
}

static void orc3_cell_nodes(int64_t n, int64_t c1, int64_t c2, int64_t c3, int64_t g[8])
{
    for (int a = 0; a < 8; ++a) {
        const int64_t i1 = (c1 + (a >> 2)) % n, i2 = (c2 + ((a >> 1) & 1)) % n, i3 = (c3 + (a & 1)) % n;
        g[a] = (i1 * n + i2) * n + i3;
    }
}

/* CSR stiffness (27 entries per row), summed over cells as in 2D. */
int64_t orc3_assemble(int64_t n, double h, const double* coef, int scheme, int64_t* rowptr,
                      int64_t* colidx, double* vals)
{
    double E[64];
    orc3_element_matrix(scheme, h, E);
    const int64_t N = n * n * n;
    orc_triplet* t = (orc_triplet*)malloc(sizeof(orc_triplet) * (size_t)(64 * N));
    int64_t nt = 0;
    for (int64_t c1 = 0; c1 < n; ++c1)
        for (int64_t c2 = 0; c2 < n; ++c2)
            for (int64_t c3 = 0; c3 < n; ++c3) {
                int64_t g[8];
                orc3_cell_nodes(n, c1, c2, c3, g);
                const double a = coef[(c1 * n + c2) * n + c3];
                for (int i = 0; i < 8; ++i)
                    for (int j = 0; j < 8; ++j) {
                        t[nt].row = g[i];
                        t[nt].col = g[j];
                        t[nt].val = a * E[i * 8 + j];
                        ++nt;
                    }
            }
    qsort(t, (size_t)nt, sizeof(orc_triplet), orc_triplet_cmp);
    int64_t nnz = 0;
    for (int64_t r = 0; r <= N; ++r) rowptr[r] = 0;
    for (int64_t k = 0; k < nt; ++k) {
        if (k > 0 && t[k].row == t[k - 1].row && t[k].col == t[k - 1].col) {
            vals[nnz - 1] += t[k].val;
        } else {
            colidx[nnz] = t[k].col;
            vals[nnz] = t[k].val;
            rowptr[t[k].row + 1] += 1;
            ++nnz;
        }
    }
    for (int64_t r = 0; r < N; ++r) rowptr[r + 1] += rowptr[r];
    free(t);
    return nnz;
}

/* f_i = -sum_c a_c P_c^T E xi_i, xi_i = h (corner bit of axis i). */
void orc3_rhs(int64_t n, double h, const double* coef, int scheme, double* f)
{
    double E[64];
    orc3_element_matrix(scheme, h, E);
    const int64_t N = n * n * n;
    memset(f, 0, sizeof(double) * 3 * (size_t)N);
    for (int i = 0; i < 3; ++i) {
        double Exi[8];
        for (int r = 0; r < 8; ++r) {
            Exi[r] = 0.0;
            for (int c = 0; c < 8; ++c) Exi[r] += E[r * 8 + c] * h * (double)((c >> (2 - i)) & 1);
        }
        for (int64_t c1 = 0; c1 < n; ++c1)
            for (int64_t c2 = 0; c2 < n; ++c2)
                for (int64_t c3 = 0; c3 < n; ++c3) {
                    int64_t g[8];
                    orc3_cell_nodes(n, c1, c2, c3, g);
                    const double a = coef[(c1 * n + c2) * n + c3];
                    for (int r = 0; r < 8; ++r) f[i * N + g[r]] -= a * Exi[r];
                }
    }
}

/* z = B^{-1} r, B = c0 A_Delta + delta I with A_Delta the periodic 7-point
 * Laplacian (eigenvalues 4 sin^2(pi k1/n) + 4 sin^2(pi k2/n) + 4
 * sin^2(pi k3/n)); the constant mode is dropped when delta = 0. */
void orc3_precond(int64_t n, double c0, double delta, const double* r, double* z)
{
    const int64_t N = n * n * n;
    if (n < 1 || (n & (n - 1)) != 0) {
        for (int64_t k = 0; k < N; ++k) z[k] = NAN;
        return;
    }
    double* re = (double*)malloc(sizeof(double) * (size_t)N);
    double* im = (double*)calloc((size_t)N, sizeof(double));
    double* lr = (double*)malloc(sizeof(double) * (size_t)n);
    double* li = (double*)malloc(sizeof(double) * (size_t)n);
    memcpy(re, r, sizeof(double) * (size_t)N);
    for (int pass = 0; pass < 2; ++pass) {
        const int sign = pass == 0 ? -1 : +1;
        for (int axis = 0; axis < 3; ++axis) {
            const int64_t stride = axis == 0 ? n * n : (axis == 1 ? n : 1);
            for (int64_t a = 0; a < n; ++a)
                for (int64_t b = 0; b < n; ++b) {
                    int64_t base;
                    if (axis == 0) base = a * n + b;
                    else if (axis == 1) base = a * n * n + b;
                    else base = (a * n + b) * n;
                    for (int64_t k = 0; k < n; ++k) { lr[k] = re[base + k * stride]; li[k] = im[base + k * stride]; }
                    orc_fft1d(n, lr, li, sign);
                    for (int64_t k = 0; k < n; ++k) { re[base + k * stride] = lr[k]; im[base + k * stride] = li[k]; }
                }
        }
        if (pass == 0) {
            for (int64_t k1 = 0; k1 < n; ++k1)
                for (int64_t k2 = 0; k2 < n; ++k2)
                    for (int64_t k3 = 0; k3 < n; ++k3) {
                        const double s1 = sin(ORC_PI * (double)k1 / (double)n);
                        const double s2 = sin(ORC_PI * (double)k2 / (double)n);
                        const double s3 = sin(ORC_PI * (double)k3 / (double)n);
                        const double sigma = c0 * 4.0 * (s1 * s1 + s2 * s2 + s3 * s3) + delta;
                        const int64_t idx = (k1 * n + k2) * n + k3;
                        const double inv = (k1 == 0 && k2 == 0 && k3 == 0 && delta == 0.0) ? 0.0 : 1.0 / sigma;
                        re[idx] *= inv;
                        im[idx] *= inv;
                    }
        }
    }
    for (int64_t k = 0; k < N; ++k) z[k] = re[k] / (double)N;
    free(re); free(im); free(lr); free(li);
}

/* PCG as orc_pcg, on n^3 unknowns with the 3D preconditioner. */
int orc3_pcg(int64_t n, const int64_t* rowptr, const int64_t* colidx, const double* vals,
             double c0, double delta, const double* f, double tol, int max_iter, double* u,
             double* relres_true)
{
    const int64_t N = n * n * n;
    double* r = (double*)malloc(sizeof(double) * (size_t)N);
    double* z = (double*)malloc(sizeof(double) * (size_t)N);
    double* p = (double*)malloc(sizeof(double) * (size_t)N);
    double* q = (double*)malloc(sizeof(double) * (size_t)N);
    memset(u, 0, sizeof(double) * (size_t)N);
    memcpy(r, f, sizeof(double) * (size_t)N);
    const double fnorm = sqrt(orc_dot(N, f, f));
    int it = 0;
    if (fnorm > 0.0) {
        orc3_precond(n, c0, delta, r, z);
        memcpy(p, z, sizeof(double) * (size_t)N);
        double rz = orc_dot(N, r, z);
        while (it < max_iter) {
            orc_spmv(N, rowptr, colidx, vals, p, q);
            ++it;
            const double alpha = rz / orc_dot(N, p, q);
            for (int64_t k = 0; k < N; ++k) { u[k] += alpha * p[k]; r[k] -= alpha * q[k]; }
            if (sqrt(orc_dot(N, r, r)) <= tol * fnorm) break;
            orc3_precond(n, c0, delta, r, z);
            const double rz_new = orc_dot(N, r, z);
            const double beta = rz_new / rz;
            rz = rz_new;
            for (int64_t k = 0; k < N; ++k) p[k] = z[k] + beta * p[k];
        }
    }
    double mean = 0.0;
    for (int64_t k = 0; k < N; ++k) mean += u[k];
    mean /= (double)N;
    for (int64_t k = 0; k < N; ++k) u[k] -= mean;
    if (relres_true) {
        orc_spmv(N, rowptr, colidx, vals, u, q);
        double s = 0.0;
        for (int64_t k = 0; k < N; ++k) s += (f[k] - q[k]) * (f[k] - q[k]);
        *relres_true = fnorm > 0.0 ? sqrt(s) / fnorm : 0.0;
    }
    free(r); free(z); free(p); free(q);
    return it;
}

/* 3x3 homogenized matrices, cell by cell: energy (1/L^3) sum_c a_c v_i^T E
 * v_j with v_i = xi_i + P_c u_i, flux (1/L^3) sum_c a_c int_c d_j (x_i +
 * phi_i) (the exact integral of the trilinear derivative: h^2/4 times the
 * sum over the four cell edges along axis j of the end differences). */
void orc3_a_hom(int64_t n, double h, double Lsize, const double* coef, int scheme,
                const double* u, double* A_energy, double* A_flux)
{
    double E[64];
    orc3_element_matrix(scheme, h, E);
    const int64_t N = n * n * n;
    double en[9] = {0}, fl[9] = {0};
    for (int64_t c1 = 0; c1 < n; ++c1)
        for (int64_t c2 = 0; c2 < n; ++c2)
            for (int64_t c3 = 0; c3 < n; ++c3) {
                int64_t g[8];
                orc3_cell_nodes(n, c1, c2, c3, g);
                const double a = coef[(c1 * n + c2) * n + c3];
                double v[3][8];
                for (int i = 0; i < 3; ++i)
                    for (int k = 0; k < 8; ++k)
                        v[i][k] = u[i * N + g[k]] + h * (double)((k >> (2 - i)) & 1);
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) {
                        double s = 0.0;
                        for (int r = 0; r < 8; ++r)
                            for (int c = 0; c < 8; ++c) s += v[j][r] * E[r * 8 + c] * v[i][c];
                        en[3 * i + j] += a * s;
                        double d = 0.0;
                        for (int k = 0; k < 8; ++k)
                            d += ((k >> (2 - j)) & 1) ? v[i][k] : -v[i][k];
                        fl[3 * i + j] += a * 0.25 * h * h * d;
                    }
            }
    const double vol = Lsize * Lsize * Lsize;
    for (int k = 0; k < 9; ++k) {
        if (A_energy) A_energy[k] = en[k] / vol;
        if (A_flux) A_flux[k] = fl[k] / vol;
    }
}

/* Field, assembly, the three corrector solves and A_hom of one 3D
 * realization.  u (or NULL): [3][n^3]. */
int orc3_solve_realization(const orc_realization* r, int scheme, double tol, int max_iter,
                           double delta, uint8_t* mask_out, double* u, orc3_result* res)
{
    const int64_t n = (int64_t)r->L * r->m0;
    const int64_t N = n * n * n;
    const double h = 1.0 / (double)r->m0;
    if (n < 2 || (n & (n - 1)) != 0) return -2;
    uint8_t* mask = mask_out ? mask_out : (uint8_t*)malloc((size_t)N);
    double* coef = (double*)malloc(sizeof(double) * (size_t)N);
    int64_t* rowptr = (int64_t*)malloc(sizeof(int64_t) * (size_t)(N + 1));
    int64_t* colidx = (int64_t*)malloc(sizeof(int64_t) * (size_t)(27 * N));
    double* vals = (double*)malloc(sizeof(double) * (size_t)(27 * N));
    double* f = (double*)malloc(sizeof(double) * 3 * (size_t)N);
    double* uu = u ? u : (double*)malloc(sizeof(double) * 3 * (size_t)N);
    if (!mask || !coef || !rowptr || !colidx || !vals || !f || !uu) return -1;
    orc3_gen_field(r, mask);
    double s = 0.0;
    for (int64_t k = 0; k < N; ++k) {
        coef[k] = mask[k] ? r->a_incl : r->a_matrix;
        s += coef[k];
    }
    res->mean_a = s / (double)N;
    const double c0 = 0.5 * (r->a_matrix + r->a_incl);
    orc3_assemble(n, h, coef, scheme, rowptr, colidx, vals);
    orc3_rhs(n, h, coef, scheme, f);
    for (int i = 0; i < 3; ++i) {
        double rr = 0.0;
        res->iters[i] = orc3_pcg(n, rowptr, colidx, vals, c0, delta, f + i * N, tol, max_iter,
                                 uu + i * N, &rr);
        res->relres_true[i] = rr;
    }
    orc3_a_hom(n, h, (double)r->L, coef, scheme, uu, res->A_energy, res->A_flux);
    free(coef); free(rowptr); free(colidx); free(vals); free(f);
    if (!u) free(uu);
    if (!mask_out) free(mask);
    return 0;
}
