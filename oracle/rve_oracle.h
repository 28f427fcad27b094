/*
 * rve_oracle.h -- declarations of the FP64 CPU oracle (test infrastructure
 * only; see rve_oracle.c).  This header belongs to the oracle alone: the
 * CUDA library neither includes it nor shares any type with it.
 */
#ifndef RVE_ORACLE_H
#define RVE_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_SCHEME_CONSISTENT 0
#define ORC_SCHEME_LUMPED 1
#define ORC_TAG_CORNER 1u

/* One realization: L cells of unit side per axis, m0 grid cells per unit,
 * inclusions of incl_cells x incl_cells grid cells, n_incl of them. */
typedef struct {
    int32_t L, m0, incl_cells, n_incl;
    double a_matrix, a_incl;
    uint64_t seed, index;
} orc_realization;

typedef struct {
    double A_energy[4], A_flux[4];
    double relres_true[2];
    double mean_a;
    int32_t iters[2];
} orc_result;

uint64_t orc_splitmix64_mix(uint64_t z);
uint64_t orc_splitmix64_output(uint64_t seed, uint64_t k);
uint64_t orc_realization_key(uint64_t seed, uint64_t index);
uint64_t orc_draw(uint64_t key, uint32_t tag, uint64_t ctr);
void orc_corners(const orc_realization* r, int32_t* corners);
void orc_gen_field(const orc_realization* r, uint8_t* mask);
void orc_coef_from_mask(int64_t n, const uint8_t* mask, double a_matrix,
                        double a_incl, double* coef);

void orc_element_matrix(int scheme, double h, double E[16]);
int64_t orc_assemble(int64_t n, double h, const double* coef, int scheme,
                     int64_t* rowptr, int64_t* colidx, double* vals);
void orc_spmv(int64_t N, const int64_t* rowptr, const int64_t* colidx,
              const double* vals, const double* x, double* y);
void orc_rhs(int64_t n, double h, const double* coef, int scheme, double* f);

double orc_laplacian_eig(int64_t n, int64_t k1, int64_t k2);
void orc_precond(int64_t n, double c0, double delta, const double* r, double* z);
int orc_pcg(int64_t n, const int64_t* rowptr, const int64_t* colidx,
            const double* vals, double c0, double delta, const double* f,
            double tol, int max_iter, double* u, double* relres_true);

void orc_a_hom(int64_t n, double h, double Lsize, const double* coef, int scheme,
               const double* u, double* A_energy, double* A_flux);
void orc_a_hom_grad(int64_t n, double h, double Lsize, int scheme,
                    const double* u, const double G[4], double* grad);

int orc_solve_coef(int64_t L, int64_t m0, const double* coef, double c0,
                   int scheme, double tol, int max_iter, double delta,
                   double* u, orc_result* res);
int orc_solve_realization(const orc_realization* r, int scheme, double tol,
                          int max_iter, double delta, uint8_t* mask_out,
                          double* u, orc_result* res);
int orc_solve_batch(const orc_realization* r, int batch, int scheme, double tol,
                    int max_iter, double delta, orc_result* res, int threads);

/* General right-hand side (Sec. 3.5, the FEM convergence test): the load
 * vector of a nodal load through the Q1 mass matrix, and the periodic
 * solve A u = b for a given mean-zero load vector b. */
void orc_mass_element(int scheme, double h, double M[16]);
void orc_apply_mass(int64_t n, double h, int scheme, const double* x, double* y);
int orc_solve_load(int64_t L, int64_t m0, const double* coef, double c0, int scheme,
                   const double* b, double tol, int max_iter, double delta, double* u,
                   double* relres_true);

void orc3_statistics(int64_t N, const double* A, double L, double* mean, double* var, double* Q);
/* The 3D extension (cubes, trilinear Q1, 3x3 A_hom). */
typedef struct {
    int iters[3];
    double relres_true[3];
    double A_energy[9], A_flux[9];
    double mean_a;
} orc3_result;
void orc3_gen_field(const orc_realization* r, uint8_t* mask);
void orc3_element_matrix(int scheme, double h, double E[64]);
int64_t orc3_assemble(int64_t n, double h, const double* coef, int scheme, int64_t* rowptr,
                      int64_t* colidx, double* vals);
void orc3_rhs(int64_t n, double h, const double* coef, int scheme, double* f);
void orc3_precond(int64_t n, double c0, double delta, const double* r, double* z);
int orc3_pcg(int64_t n, const int64_t* rowptr, const int64_t* colidx, const double* vals,
             double c0, double delta, const double* f, double tol, int max_iter, double* u,
             double* relres_true);
void orc3_a_hom(int64_t n, double h, double Lsize, const double* coef, int scheme,
                const double* u, double* A_energy, double* A_flux);
int orc3_solve_realization(const orc_realization* r, int scheme, double tol, int max_iter,
                           double delta, uint8_t* mask_out, double* u, orc3_result* res);

void orc_statistics(int64_t N, const double* A, double L, int d, double* mean,
                    double* var, double* std12_paper, double* stddiff_paper,
                    double* Q);

#ifdef __cplusplus
}
#endif
#endif
