// Cluster-blocked sparse layout of the truncated (linear-scaling) form: internal declarations.
//
// Atoms are grouped into spatially compact clusters (Morton order, at most CB_R chi and CB_C phi
// functions per cluster). Every matrix is stored as a list of dense cluster blocks (block sparse
// row): chi x phi matrices (the response kernels and everything of their shape) in blocks of
// CB_R x CB_C on the kernel pattern, chi x chi constants in CB_R x CB_R blocks and phi x phi
// constants in CB_C x CB_C blocks on their own patterns. Padding rows and columns of a block are
// zero, and so are the entries of a block whose atom pair lies outside the pattern (a 0/1 mask in
// the block layout applies the atom-level truncation inside the blocks).
#pragma once

#include "tddft.h"
#include "tddft_internal.h"

#include <memory>
#include <vector>

namespace tddft {

constexpr int CB_R = 128;   // chi rows of a cluster block (padded)
constexpr int CB_C = 64;    // phi columns of a cluster block (padded)
constexpr long long CB_SIZE = (long long)CB_R * CB_C;

// pattern of a cluster-blocked matrix, blocks in row-major order of (block row, block column)
struct BlockPattern {
    int nr = 0, nc = 0;
    std::vector<int> row_ptr;   // [nr + 1]
    std::vector<int> col;       // [nnzb], ascending within a row
    int nnzb() const { return row_ptr.empty() ? 0 : row_ptr.back(); }
    int find(int a, int b) const;   // block index of (a, b), or -1
};

// The block pairs of C = A B on fixed patterns: for every output block with at least one
// contributing pair, the list of (A block, B block); output blocks with none are listed apart.
struct PairList {
    int nout = 0, npairs = 0, nempty = 0;
    int *out = nullptr;     // [nout] output block
    int *ptr = nullptr;     // [nout + 1] into pa / pb
    int *pa = nullptr;      // [npairs]
    int *pb = nullptr;      // [npairs]
    int *empty = nullptr;   // [nempty] output blocks without pairs
    long long nnz_flops = 0;   // 2 * sum over pairs of the padded block product (per batch entry)
    double alg_flops = 0.0;    // 2 * sum over contributing atom-block triples (I, K, J) of n_I n_K n_J
};

// the constants of the operator and the solver, by role
enum { SP_M = 0, SP_P = 1, SP_R = 2, SP_A = 3, SP_S = 4, SP_T = 5, SP_NCONST = 6 };
// chi side: M_c = P^c_t H^chi, P^c_t, R_c = P^c_t S^chi, A_c = S^chi P^c_t S^chi, S^chi,
//           R_c^T = S^chi P^c_t
// phi side: M_v = H^phi P^v_t, P^v_t, R_v = S^phi P^v_t, A_v = S^phi P^v_t S^phi, S^phi,
//           R_v^T = P^v_t S^phi

struct SparseLayout {
    Mem mem;
    int natoms = 0, ncl = 0, nc = 0, nv = 0;
    double cell = 0.0, r_cut = 0.0, r_k = 0.0;
    BlockPattern pk;                                 // chi x phi kernel pattern (clusters)
    BlockPattern pcc[SP_NCONST], pvv[SP_NCONST];     // constants' patterns
    PairList left[SP_NCONST], right[SP_NCONST];      // C_x Y and Y D_x into the kernel pattern
    double *cc64[SP_NCONST] = {}, *vv64[SP_NCONST] = {};   // constant blocks, float64
    // device index arrays
    int *blk_row = nullptr, *blk_col = nullptr;      // [pk.nnzb]
    int *blk_of = nullptr;                           // [ncl * ncl] kernel block of (A, B), or -1
    int *rowfun = nullptr, *colfun = nullptr;        // [ncl * CB_R], [ncl * CB_C]: function or -1
    int *chi_cl = nullptr, *chi_row = nullptr;       // [nc]
    int *phi_cl = nullptr, *phi_col = nullptr;       // [nv]
    int *chi_atom = nullptr, *phi_atom = nullptr;    // [nc], [nv]
    int *chi_first = nullptr, *phi_first = nullptr, *phi_cnt = nullptr;   // [natoms]
    long long *abi_off = nullptr;                    // [natoms * natoms] offset of atom block (I, J) or -1
    double *pos = nullptr;                           // [natoms * 3]
    // the boundary's atom-blocked pattern of the kernels (host)
    std::vector<long long> abi_row_ptr, abi_blk_off;
    std::vector<int> abi_col;
    long long nnz_abi = 0;
    std::vector<unsigned char> amask;                // [natoms * natoms] kernel pattern of atom pairs
    long long len() const { return (long long)pk.nnzb() * CB_SIZE; }
    long long cc_len(int x) const { return (long long)pcc[x].nnzb() * CB_R * CB_R; }
    long long vv_len(int x) const { return (long long)pvv[x].nnzb() * CB_C * CB_C; }
};

// Build the layout of a system: clusters, patterns, index arrays, the truncated ground-state
// kernels and the constant products in float64 on the device (CUDA-core block products), and
// the pair lists. Throws CudaError / std::bad_alloc; argument errors as std::invalid_argument.
std::unique_ptr<SparseLayout> sparse_build(cudaStream_t st, const tddft_sparse_system *s);

// C_b[o] = mask (alpha sum_pairs A_b[pa] B_b[pb] + beta C_b[o]) over the listed outputs, blocks
// row-major of BR x BK (A), BK x BC (B), BR x BC (C); batch strides in elements (0: shared);
// mask [outputs][BR x BC] or null; on the CUDA cores
template <typename T>
void bsr_simt(cudaStream_t st, int BR, int BK, int BC, const PairList &pl, int nblk_out, const T *A, long long sA,
              const T *B, long long sB, T *C, long long sC, int nb, T alpha, T beta, const T *mask);

// the same product on the tensor cores (float32, tcgen05 kind::tf32; three-term split unless
// approx), B given transposed: Bt blocks BC x BK row-major. BR = 128, BC = 64, BK in {64, 128}.
void bsr_tc(cudaStream_t st, int BK, const PairList &pl, int nblk_A, const float *A, long long sA, int nblk_B,
            const float *Bt, long long sB, float *C, long long sC, int nb, float alpha, float beta,
            const float *mask, bool approx);
bool bsr_tc_available();

// out[b][blk] = in[b][blk]^T for nblk blocks of R x Cc per batch entry (row-major in and out)
template <typename T>
void bsr_transpose(cudaStream_t st, const T *in, T *out, int R, int Cc, long long nblk, int nb);

// conversions between the boundary's atom-blocked order [k][nnz_abi] (float64), the cluster
// blocks [k][len] (T) and dense [k][nc][nv] (T) for the grid kernels
template <typename T>
void cb_from_abi(cudaStream_t st, const SparseLayout &L, const double *src, T *dst, int k);
template <typename T>
void cb_to_abi(cudaStream_t st, const SparseLayout &L, const T *src, double *dst, int k);
template <typename T>
void cb_to_dense(cudaStream_t st, const SparseLayout &L, const T *src, T *dst, int k);
template <typename T>
void cb_from_dense(cudaStream_t st, const SparseLayout &L, const T *src, T *dst, const T *mask, int k);
// the 0/1 kernel-pattern mask in the cluster-block layout
template <typename T>
void cb_mask(cudaStream_t st, const SparseLayout &L, T *mask);

}  // namespace tddft
