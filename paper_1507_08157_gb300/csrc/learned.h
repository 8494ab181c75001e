// Declarations of the learned atom-block preconditioner (learned.cu).
#pragma once

#include "tddft.h"
#include "tddft_internal.h"

namespace tddft {

int mlp_n_block(const tddft_mlp *m);
int mlp_n_feat(const tddft_mlp *m);
long long mlp_version(const tddft_mlp *m);    // changes whenever the parameters change

// vec(A) rows [n][n_b^2] of the model for feature rows F [n][n_f], bfloat16-rounded parameters
void mlp_block_maps(cudaStream_t st, tddft_mlp *m, long long n, const float *F, float *A);

// feature rows F [na na][n_f] = [fc_I, fv_J, dist_IJ]
void learned_feature_rows(cudaStream_t st, const float *fc, const float *fv, const float *dist, int na, int nca,
                          int nva, float *F);

// out[I] = [A_II, S_II] (nb x nb blocks, row-major) for the na atoms of the n x n matrices A, S
template <typename T>
void learned_fixed_features(cudaStream_t st, const T *A, const T *S, int n, int nb, int na, float *out);

// input rows X [k na na][n_in] and block scales s of the 2k gradient matrices h (p then q)
template <typename T>
void learned_features(cudaStream_t st, const T *h, int k, int na, int nca, int nva, int nc, int nv,
                      const float *fc, const float *fv, const float *dist, float *X, float *s);

// z_IJ = h_IJ + A_IJ h_IJ for the 2k matrices (p then q), A [na na][n_b^2]
template <typename T>
void learned_apply(cudaStream_t st, const float *A, const T *h, int k, int na, int nca, int nva, int nc, int nv, T *z);

// target rows Y = (z - h) blocks / s and row weights w = s^2 / (sum of s^2 over the state's rows)
template <typename T>
void learned_targets(cudaStream_t st, const T *z, const T *h, const float *s, int k, int na, int nca, int nva, int nc,
                     int nv, float *Y, float *w);

}  // namespace tddft
