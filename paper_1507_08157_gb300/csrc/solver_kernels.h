// Declarations of the solver primitives defined in solver_kernels.cu and spectrum.cu.
#pragma once

#include "tddft_internal.h"

namespace tddft {

// d_i = sum_e X_i[e] Y_i[e] for i < n (float64, fixed order); scratch as for gram
template <typename T>
void dots(cudaStream_t st, const T *X, long long sx, const T *Y, long long sy, int n, long long len,
          double *d, double *scratch);

// out = -z + beta * prev, beta a device scalar
template <typename T>
void direction(cudaStream_t st, T *out, const T *z, const T *prev, const double *beta, long long n);

// p_b <- r_b + beta[b] p_b
template <typename T>
void cg_dir(cudaStream_t st, T *p, const T *r, const double *beta, long long len, int nb);

void make_q(cudaStream_t st, int k, const double *A, double *Q, double *coef);
void eval_finish(cudaStream_t st, int k, const double *Q, const double *d, double *out, int *status);
void conj_coeff(cudaStream_t st, int k2, const double *gz, const double *gzp, const double *gd,
                int restart, const double *flip, double *sc);
void line_gs(cudaStream_t st, int k, const double *A, const double *BDf, const double *CDfD,
             const double *PP, const double *PD, const double *DP, const double *DD, const double *Q,
             double *lam, double *Cp, double *Cq, double *flip, int *status);
void init_gs(cudaStream_t st, int k, const double *PP, double *Cp, double *Cq, int *status);
void cg_init(cudaStream_t st, int n, double tol, const double *rr0, double *rr, double *r0,
             int *active, int *n_active);
void cg_scalars(cudaStream_t st, int n, int phase, double tol, const double *pLp,
                const double *rr_new, double *rr, const double *r0, double *alpha, double *beta,
                int *active, int *n_active);
// Ritz values omega [k] ascending of the symmetrised Q, the pairing errors [2k] and, if vecs is
// not NULL, the eigenvectors [k][k] (column m belongs to omega[m])
void subspace(cudaStream_t st, int k, const double *A, double *omega, double *pairing, double *vecs = nullptr);

// transition dipoles (oscillator strengths, spectra): per-block partial sums of x_a rho_s over the
// n^3 grid, x_a(i) = i h - L/2; partials [k][nblk][3]
template <typename T>
void dipole_partials(cudaStream_t st, const T *rho, int n, double h, double L, int k, int nblk, double *partials);
// Ritz strengths: mu_m = dV sum_j vecs[j][m] mu_j, f_m = (2/3) omega_m |mu_m|^2; out = [f k][mu k x 3]
void ritz_strengths(cudaStream_t st, int k, const double *omega, const double *vecs, const double *partials,
                    int nblk, double dV, double *out);
// S(E_e) = sum_i f_i (gamma / pi) / ((E_e - omega_i)^2 + gamma^2) for n energies
void lorentz_spectrum(cudaStream_t st, int k, const double *omega, const double *f, double gamma, int n,
                      const double *E, double *S);

}  // namespace tddft
