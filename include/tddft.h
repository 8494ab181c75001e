/*
 * tddft.h -- C ABI of the GB300 full-TDDFT (Tsiper p/q) operator and PCG eigensolver.
 *
 * Method: linear-response TDDFT beyond the Tamm-Dancoff approximation in a mixed representation
 * of localised conduction functions {chi} and valence functions {phi} (Zuehlsdorff, Hine, Payne,
 * Haynes, "Linear-scaling time-dependent density-functional theory beyond the Tamm-Dancoff
 * approximation", 2015). Equation names below are the paper's labels.
 *
 * Conventions (all entry points):
 *  - Hartree atomic units (bohr, Ha). All arrays are row-major (C order). Grid arrays are
 *    [ix][iy][iz] with z fastest; n^3 points on a cubic periodic cell.
 *  - Matrices are dense float64: N_chi x N_chi, N_phi x N_phi, and response kernels N_chi x N_phi
 *    (rows = chi functions, columns = phi functions). A batch of k kernels is [k][N_chi][N_phi].
 *  - Ownership: the caller owns every pointer it passes. tddft_create deep-copies the system into
 *    device memory owned by the context; nothing keeps a caller pointer after a call returns.
 *  - Host or device: array arguments of tddft_apply, tddft_state_create/get and the component
 *    entry points may be host memory or device memory of the context's GPU; the library tells
 *    them apart with cudaPointerGetAttributes. Device pointers must be 8-byte aligned.
 *  - Ordering: all GPU work is issued on the stream given to tddft_create; calls return after
 *    their results are in the caller's buffers (they synchronise that stream).
 *  - Errors: a non-zero tddft_status; the message is kept on the context (tddft_last_error).
 *    Nothing throws across the ABI. Outputs are undefined after an error, except where noted.
 *  - Threads: a context (and its states) must not be used by two threads at once.
 */
#ifndef TDDFT_H
#define TDDFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TDDFT_OK = 0,
    TDDFT_E_INVALID = 1,        /* bad argument, size or layout */
    TDDFT_E_NOMEM = 2,          /* device allocation failed */
    TDDFT_E_CUDA = 3,           /* CUDA runtime error (message names the call) */
    TDDFT_E_NOT_CONVERGED = 4,  /* tddft_solve hit max_iter; outputs hold the last iterate */
    TDDFT_E_BREAKDOWN = 5,      /* NaN/Inf, or a non-positive norm in Gram-Schmidt */
    TDDFT_E_TIMEOUT = 6,        /* a bounded wait inside a tensor-core kernel expired (limit:
                                   tddft_options.spin_limit_cycles). Any call that runs the
                                   tensor-core products or grid kernels of a TDDFT_MIXED context
                                   (apply, the component entry points, state_create, pcg_step,
                                   solve, oscillator_strengths, the allocation-free density) and
                                   tddft_wait_check can return it; the kernel gives up, lets its
                                   copies in flight land, frees its tensor memory and returns, and
                                   the context stays usable */
    TDDFT_E_PAIRING = 7         /* converged pairs fail the +-omega pairing check */
} tddft_status;

enum { TDDFT_FP64 = 0, TDDFT_MIXED = 1 };                       /* tddft_options.precision */
enum { TDDFT_MODE_FULL = 0, TDDFT_MODE_TDA = 1, TDDFT_MODE_D_ONLY = 2 };
enum { TDDFT_PRECOND_NONE = 0, TDDFT_PRECOND_ITER = 1, TDDFT_PRECOND_LEARNED = 2, TDDFT_PRECOND_EXACT = 3 };
enum { TDDFT_FXC_NONE = 0, TDDFT_FXC_LDA_PW92 = 1 };

/* Localised functions tabulated in periodic boxes (paper Sec. II C: NGWFs phi_alpha, chi_alpha).
 * Function f covers the grid points ((ox+i) mod n, (oy+j) mod n, (oz+l) mod n) for
 * 0 <= i < ex, 0 <= j < ey, 0 <= l < ez, with box[6f..6f+5] = (ox, oy, oz, ex, ey, ez),
 * 0 <= o < n, 1 <= e <= n. Its values are val[off[f] .. off[f+1]), C order (l fastest), and
 * off[f+1] - off[f] = ex*ey*ez; with val NULL they are val32 (float32) instead, which halves the
 * host memory of large systems. atom[f] is the owning atom (used for the kernel cutoff). */
typedef struct {
    int32_t nfun;
    const int32_t *atom;
    const int32_t *box;
    const int64_t *off;
    const double *val;
    const float *val32;
} tddft_funcs;

/* One system: the ground-state inputs the linear-response calculation takes as given
 * (Sec. II C). All host pointers. */
typedef struct {
    double cell;              /* cubic cell side (bohr) */
    int32_t n;                /* grid points per side: 2^a 3^b 5^c, 8 <= n <= 256 */
    int32_t natoms;
    const double *pos;        /* [natoms][3] (bohr) */
    tddft_funcs phi;          /* valence functions, N_phi = phi.nfun */
    tddft_funcs chi;          /* conduction functions, N_chi = chi.nfun */
    const double *S_chi;      /* [N_chi][N_chi] overlap <chi_a|chi_b> */
    const double *S_phi;      /* [N_phi][N_phi] */
    const double *H_chi;      /* [N_chi][N_chi] Kohn-Sham Hamiltonian in chi */
    const double *H_phi;      /* [N_phi][N_phi] */
    const double *P_v;        /* [N_phi][N_phi] valence density kernel (contravariant) */
    const double *P_c;        /* [N_chi][N_chi] conduction density kernel (contravariant) */
    const double *n0;         /* [n^3] ground-state density (bohr^-3), for f_xc */
    int32_t fxc_kind;         /* TDDFT_FXC_LDA_PW92 or TDDFT_FXC_NONE (Hartree only) */
    double kernel_cutoff;     /* bohr; <= 0: response kernels not truncated. Otherwise the
                                 auxiliary matrices L (Eq. auxiliary) keep entry (a,b) only when
                                 the minimum-image distance of the atoms of chi_a and phi_b is
                                 <= kernel_cutoff */
} tddft_system;

/* An atom-blocked sparse matrix (block sparse row). Block rows and block columns are atoms; block
 * (I, J) is dim(I) x dim(J) with dim(I) the number of functions of atom I in the row set (chi or
 * phi, as the field's name says) and dim(J) likewise in the column set; a function set lists its
 * functions grouped by atom (atom[] nondecreasing), and the rows of a block follow that order.
 *   row_ptr [natoms + 1]: blocks of row I are row_ptr[I] .. row_ptr[I+1]-1
 *   col_idx [nnzb]: column atom of each block, strictly ascending within a row
 *   blk_off [nnzb + 1]: values of block b are val[blk_off[b] .. blk_off[b+1]), row-major,
 *                       blk_off[b+1] - blk_off[b] = dim(I) dim(J)
 * Absent blocks are zero. All host pointers, owned by the caller. */
typedef struct {
    const int64_t *row_ptr;
    const int32_t *col_idx;
    const int64_t *blk_off;
    const double *val;
} tddft_bsr;

/* One system in the truncated (linear-scaling) form of Sec. IV: every density matrix truncated by
 * atom-pair distance so that every matrix product scales linearly with the number of atoms.
 * Ground-state matrices come atom-blocked; see tddft_create_sparse for the semantics. */
typedef struct {
    double cell;              /* cubic cell side (bohr) */
    int32_t n;                /* grid points per side: 2^a 3^b 5^c, 8 <= n <= 256 */
    int32_t natoms;
    const double *pos;        /* [natoms][3] (bohr) */
    tddft_funcs phi;          /* valence functions, grouped by atom, <= 64 per atom */
    tddft_funcs chi;          /* conduction functions, grouped by atom, <= 128 per atom */
    tddft_bsr S_chi, H_chi, P_c;   /* chi x chi */
    tddft_bsr S_phi, H_phi, P_v;   /* phi x phi */
    const double *n0;         /* [n^3] ground-state density (bohr^-3), for f_xc */
    int32_t fxc_kind;         /* TDDFT_FXC_LDA_PW92 or TDDFT_FXC_NONE */
    double kernel_cutoff;     /* bohr, > 0: the pattern of every chi x phi matrix (atom pairs
                                 within this minimum-image distance) */
    double density_kernel_cutoff;  /* bohr; > 0: P^c and P^v are truncated to atom pairs within
                                 it; <= 0: they are used as given */
} tddft_sparse_system;

typedef struct {
    int32_t precision;        /* TDDFT_FP64: all arithmetic in float64.
                                 TDDFT_MIXED: matrices, grids and FFTs in float32; traces,
                                 line search, Gram-Schmidt, eigenvalues in float64 */
    int32_t mode;             /* TDDFT_MODE_FULL (Eq. operator_RPA); TDDFT_MODE_TDA (B = 0:
                                 f_p = A p, f_q = A q); TDDFT_MODE_D_ONLY (coupling K = 0) */
    int32_t precond;          /* TDDFT_PRECOND_ITER: CG solve of Eq. precond; NONE: identity;
                                 LEARNED: the atom-block network bound by tddft_set_mlp, with the
                                 CG solve as fallback; EXACT: Eq. precond solved exactly in the
                                 eigenbases of its two operators on the conduction x valence
                                 subspace (diagonalised once at tddft_create; INVALID when P^c or
                                 P^v is not idempotent) */
    int32_t precond_maxit;    /* inner CG iterations cap (default 50) */
    double precond_tol;       /* inner CG relative residual (default 1e-4) */
    double tol;               /* convergence: max residual (Ha) <= tol and max |d omega| <= tol/10 */
    int32_t max_iter;         /* outer iteration cap of tddft_solve */
    int32_t reapply_every;    /* recompute f = f(P) from scratch every this many steps (10) */
    int32_t restart_every;    /* Polak-Ribiere restart period (10) */
    int32_t precond_adaptive; /* 0: inner CG to precond_tol every step. 1: loose first, tight at the
                                 end (Sec. IV A suggests it): the step's inner tolerance is
                                 min(0.1, max(precond_tol, largest residual of the iterate in Ha)) */
    int64_t spin_limit_cycles; /* limit of every bounded wait in the context's tensor-core kernels,
                                 in SM clock cycles (clock64); <= 0: the default 4e9 (about 2 s).
                                 An expired wait makes the call return TDDFT_E_TIMEOUT */
} tddft_options;

typedef struct tddft_ctx tddft_ctx;
typedef struct tddft_state tddft_state;

/* Fill *opt with the defaults: FP64, FULL, ITER, 50, 1e-4, tol 1e-6, 500, 10, 10, not adaptive,
 * spin limit 0 (the default 4e9 cycles). */
void tddft_default_options(tddft_options *opt);

/* Build a context on the current CUDA device: copies the system to the device, builds the
 * grid-tile tables of the functions, f_xc[n0] (Sec. II A, LDA) and the products
 * M_c = P^c H^chi, M_v = H^phi P^v, R_c = P^c S^chi, R_v = S^phi P^v used by Eqs.
 * operator_RPA and auxiliary. cuda_stream: a cudaStream_t, or NULL for the default stream.
 * Errors: INVALID (sizes, grid not 2/3/5-smooth, a box wider than the cell), NOMEM, CUDA. */
tddft_status tddft_create(const tddft_system *sys, const tddft_options *opt, void *cuda_stream,
                          tddft_ctx **out);
void tddft_destroy(tddft_ctx *ctx);

/* A context in the truncated (linear-scaling) form (Sec. IV, "Linear-scaling capabilities"; the
 * auxiliary matrices of Sec. III A, Eq. auxiliary). Semantics:
 *  - P^c_t, P^v_t: P^c and P^v with the atom blocks beyond density_kernel_cutoff removed;
 *  - products of ground-state matrices are exact: M_c = P^c_t H^chi, M_v = H^phi P^v_t,
 *    R_c = P^c_t S^chi, R_v = S^phi P^v_t, A_c = S^chi R_c, A_v = R_v S^phi;
 *  - every product whose result is a chi x phi matrix is truncated to the kernel pattern (atom
 *    pairs within kernel_cutoff), a chain of two products after each one; so Eq. operator_RPA
 *    reads f_p = T(M_c P^p) - T(P^p M_v), f_q = T(M_c P^q) - T(P^q M_v) + 2 T(T(P^c_t V) P^v_t)
 *    with V = T(V_SCF[P^q]), the trace metric is <X, Y> = sum cov(X) * Y with
 *    cov(X) = T(T(S^chi X) S^phi), Eq. auxiliary is P = T(T(R_c L) R_v), the L-gradient is
 *    that map's adjoint applied to cov(g), T(R_c^T T(cov(g) R_v^T)) (the exact gradient of the
 *    sum functional in L), Eq. precond's operator T(M_c G) - T(G M_v); a step whose inner-CG
 *    result does not descend takes the search gradient instead (counted in tddft_state_stats).
 * Every chi x phi array at the boundary of a sparse context (tddft_apply, tddft_state_create,
 * tddft_state_get, tddft_response_density's P, tddft_potential_integrals' out) is [k][nnz]: the
 * values of the kernel pattern in the atom-blocked order tddft_kernel_pattern describes. Inside,
 * atoms are grouped into spatial clusters and every matrix is a list of dense cluster blocks
 * (128 chi x 64 phi for the kernels) multiplied block by block, only over pairs of nonzero blocks
 * (tensor cores for TDDFT_MIXED). Preconditioners: TDDFT_PRECOND_ITER (CG on Eq. precond in the
 * trace metric) or NONE; others give INVALID. Errors: INVALID (sizes, patterns, functions not
 * grouped by atom, more than 128 chi or 64 phi functions on an atom, kernel_cutoff <= 0), NOMEM,
 * CUDA. */
tddft_status tddft_create_sparse(const tddft_sparse_system *sys, const tddft_options *opt, void *cuda_stream,
                                 tddft_ctx **out);

/* The atom-blocked pattern of the response kernels of a sparse context (the order of its
 * boundary arrays): nnzb blocks and nnz values; row_ptr [natoms + 1], col_idx [nnzb] and
 * blk_off [nnzb + 1] as in tddft_bsr (rows chi atoms, columns phi atoms). Any pointer may be
 * NULL (call once for the sizes). INVALID for a dense context. */
tddft_status tddft_kernel_pattern(const tddft_ctx *ctx, int64_t *nnzb, int64_t *nnz, int64_t *row_ptr,
                                  int32_t *col_idx, int64_t *blk_off);

/* Set-up of nsys independent systems of any sizes (a batch): out[i] receives the context of
 * sys[i] as tddft_create makes it, except that each context owns a non-blocking CUDA stream of
 * its own (ordered after the work queued on cuda_stream at the call) and waits on it through a
 * blocking-sync event, so that the systems overlap on the device and many host threads can
 * drive them. The set-ups run on up to 16 host threads. Each context is destroyed with
 * tddft_destroy as usual. On an error every context made so far is destroyed, out[] is all
 * NULL and the first failing system's status is returned. */
tddft_status tddft_create_batch(const tddft_system *sys, int32_t nsys, const tddft_options *opt,
                                void *cuda_stream, tddft_ctx **out);

/* tddft_solve (Sec. III C) for nsys systems at once: st[i] is a state of ctx[i] (contexts
 * pairwise distinct, best from tddft_create_batch). Host threads (nthreads, <= 0 for up to 16)
 * take the systems largest first (k x grid work) and iterate each to convergence; the device
 * interleaves the systems' kernels. omega and resid (either may be NULL) receive system i's k_i
 * values at offset k_0 + ... + k_{i-1}; iters[i] and status[i] (either may be NULL) its
 * iteration count and its tddft_solve status. Returns OK if every system returned OK, else the
 * first non-OK status in system order (INVALID for bad arguments, before any work). The
 * tensor-core kernels share one error word for expired bounded waits, so such an error is
 * reported by whichever system reads it first. */
tddft_status tddft_solve_batch(tddft_ctx *const *ctx, tddft_state *const *st, int32_t nsys,
                               int32_t nthreads, double *omega, double *resid, int32_t *iters,
                               int32_t *status);

const char *tddft_last_error(const tddft_ctx *ctx);
tddft_status tddft_dims(const tddft_ctx *ctx, int32_t *n_chi, int32_t *n_phi, int32_t *n);

/* The operator of Eq. operator_RPA on k state pairs:
 *   f_p = P^c H^chi P^p - P^p H^phi P^v
 *   f_q = P^c H^chi P^q - P^q H^phi P^v + 2 P^c V_SCF[P^q] P^v
 * with V_SCF[P]_ab = <chi_a| v_H[rho] + f_xc rho |phi_b> and rho(r) = sum chi_a P_ab phi_b
 * (Secs. II A, II C, III A). Pp, Pq: [k][N_chi][N_phi]; fp, fq: same shape, written.
 * The mode option selects TDA (B = 0) or D_ONLY instead. */
tddft_status tddft_apply(tddft_ctx *ctx, int32_t k, const double *Pp, const double *Pq,
                         double *fp, double *fq);

/* Components of V_SCF, for element-by-element checks:
 *   tddft_response_density: rho_s(r) = sum_ab chi_a(r) P_s,ab phi_b(r); P [k][N_chi][N_phi],
 *     rho [k][n^3].
 *   tddft_response_potential: V_s = v_H[rho_s] + f_xc rho_s (periodic, G = 0 dropped);
 *     rho, V [k][n^3].
 *   tddft_potential_integrals: out_s,ab = dV sum_r chi_a(r) V_s(r) phi_b(r); V [k][n^3],
 *     out [k][N_chi][N_phi].
 *   tddft_fxc: the f_xc[n0] grid [n^3] the context uses. */
tddft_status tddft_response_density(tddft_ctx *ctx, int32_t k, const double *P, double *rho);
tddft_status tddft_response_potential(tddft_ctx *ctx, int32_t k, const double *rho, double *V);
tddft_status tddft_potential_integrals(tddft_ctx *ctx, int32_t k, const double *V, double *out);
tddft_status tddft_fxc(tddft_ctx *ctx, double *fxc);

/* Autotuner of the tensor-core grid kernels' tile shapes (no counterpart in the paper). For a
 * TDDFT_MIXED context it times, on k trial states of the context's own system (deterministic
 * pseudo-random P and V), every candidate cut of the grid work into tensor-core units:
 *   response_density: the per-tile kernels (kind 0, when every tile fits them) and units of at
 *     most chi_chunk x phi_chunk functions of a tile (kind 1; chi 128..320 in steps of 64, phi 64
 *     or 128);
 *   potential_integrals: units of at most chi_chunk (128, 256, 384) x phi_chunk (32, 64, 128).
 * Each candidate runs once to warm up and three times timed with CUDA events on the context's
 * stream (ms = the mean). The fastest of each stage is installed and kept by the context for all
 * later calls (chosen = 1). out receives up to cap entries, count the number of candidates.
 * INVALID for k outside 1..32 or a context without the tensor-core grid kernels. */
typedef struct {
    char stage[32];
    int32_t kind;        /* 0: per-tile kernels, 1: units */
    int32_t chi_chunk;   /* largest chi count of a unit (0 for kind 0) */
    int32_t phi_chunk;   /* largest phi count of a unit */
    int32_t chosen;      /* 1 for the candidate installed */
    double ms;           /* mean time of one call for k states */
} tddft_tuning_entry;

tddft_status tddft_autotune(tddft_ctx *ctx, int32_t k, tddft_tuning_entry *out, int32_t cap, int32_t *count);

/* Check of the bounded-wait path (no counterpart in the paper; it tests the library's failure
 * detection without faulting or hanging the GPU): launches one small kernel on the context's
 * stream that waits, with the context's spin_limit_cycles, on a shared-memory barrier that
 * nothing completes, so the wait must expire. Returns TDDFT_E_TIMEOUT when it did and the
 * context is usable afterwards (the expected result); TDDFT_E_CUDA if the launch failed. */
tddft_status tddft_wait_check(tddft_ctx *ctx);

/* Allocation-free response density. The paper has no counterpart: this is a library-level
 * variant of tddft_response_density for callers that cannot allocate device memory when they
 * need a density (a process whose own pool allocator already holds the device memory, or a
 * latency-bound loop in which cudaMalloc / cudaFree, which synchronise the device, are not
 * allowed). It computes the same rho_s(r) = sum_ab chi_a(r) P_s,ab phi_b(r) (Sec. II C) with the
 * same tensor-core kernel, but takes float32 device buffers and uses no context workspace.
 *   ctx: a TDDFT_MIXED context whose grid products run on the tensor cores; anything else
 *        returns TDDFT_E_INVALID. Call with the context's device current.
 *   k:   number of states, 1 <= k <= TDDFT_NOALLOC_MAX_STATES (TDDFT_E_INVALID otherwise).
 *   P:   device pointer, float32 [k][N_chi][N_phi], read only, owned by the caller.
 *   rho: device pointer, float32 [k][n^3] (x slowest), every element written, owned by the
 *        caller.
 * Scratch: one fixed array of about 520 bytes per device in the library's static device memory
 * (64 max-reduction words, 64 scales, a wait-expiry flag). The first call on a device looks up
 * its address (cudaGetSymbolAddress) and loads the kernels; make that first call before the
 * phase that must not allocate. Each call clears the array on the stream before use, so the
 * caller zeroes nothing. All calls on one device share the array: overlapping calls (two host
 * threads, or two contexts on different streams) race and must be serialised by the caller.
 * The call makes no cudaMalloc / cudaFree and no allocating library call; it waits for the
 * context's stream at the end to read the flag, and returns TDDFT_E_TIMEOUT if a bounded wait
 * in the kernel expired. */
#define TDDFT_NOALLOC_MAX_STATES 64
tddft_status tddft_response_density_noalloc(tddft_ctx *ctx, int32_t k, const float *P, float *rho);

/* Solver state for k trial pairs (Sec. III C). Y0 [k][N_chi][N_phi] is the random start X
 * (Y = 0, so p = q = X); it is masked to the kernel pattern, mapped through Eq. auxiliary,
 * sign-flipped and Gram-Schmidt orthonormalised in the metric of Eq. ortho, then f is applied.
 * Errors: INVALID, BREAKDOWN (dependent start vectors), NOMEM, CUDA. */
tddft_status tddft_state_create(tddft_ctx *ctx, int32_t k, const double *Y0, tddft_state **out);
void tddft_state_destroy(tddft_state *st);

/* One preconditioned CG iteration (Sec. III C): Q_ij, multi-state gradient, preconditioner
 * (Eq. precond), Polak-Ribiere conjugation, one line step minimising the sum functional of
 * Eq. Tsiper_multiple, sign flip + Gram-Schmidt (Eq. ortho). omega [k] (ascending eigenvalues
 * of Q) and resid [k] (per-pair gradient norms) describe the iterate the step started from.
 * Either may be NULL. */
tddft_status tddft_pcg_step(tddft_ctx *ctx, tddft_state *st, double *omega, double *resid);

/* Iterate until max resid <= tol and max |d omega| <= tol/10, or max_iter. omega [k] = final
 * eigenvalues of Q ascending (Sec. III C subspace diagonalisation), resid [k], iters (may be
 * NULL). NOT_CONVERGED leaves the last iterate's values in the outputs. Then checks the pairing
 * of the converged Ritz pairs: each half of the Tsiper numerator must equal omega within
 * 10 * max(resid) * (1 + |omega|) (PAIRING otherwise). */
tddft_status tddft_solve(tddft_ctx *ctx, tddft_state *st, double *omega, double *resid,
                         int32_t *iters);

/* Copy out the current trial pairs and operator images ([k][N_chi][N_phi] each; any may be
 * NULL) and L (the masked search variables) if Lp/Lq are given. */
tddft_status tddft_state_get(tddft_ctx *ctx, const tddft_state *st, double *Pp, double *Pq,
                             double *fp, double *fq, double *Lp, double *Lq);

/* Oscillator strengths of the current Ritz pairs (the paper reports its results as energies
 * with oscillator strengths, Sec. IV). The pairs are rotated by the eigenvectors of the
 * symmetrised Q of the subspace diagonalisation (Sec. III C); the transition dipole of pair m is
 * the dipole of its response density rho^q (Sec. II C) with the position of grid point i along
 * an axis taken as i h - L/2 (from the cell centre), and f_m = (2/3) omega_m |mu_m|^2 with
 * <p_m, q_m> = 1. Outputs (host, any may be NULL): omega [k] ascending (Ha), f [k]
 * (dimensionless), mu [k][3] (e bohr; the sign of each row is arbitrary). Meaningful at
 * convergence; any iterate gives the values of its subspace. */
tddft_status tddft_oscillator_strengths(tddft_ctx *ctx, tddft_state *st, double *omega, double *f,
                                        double *mu);

/* Broadened absorption spectrum S(E_e) = sum_i f_i (gamma / pi) / ((E_e - omega_i)^2 + gamma^2)
 * for n energies E (Ha), gamma the half width at half maximum (Ha; the paper's figures use
 * 0.025 eV). omega, f [k], E and S [n] are host or device buffers; runs on the context's stream.
 * INVALID for k <= 0, n <= 0, gamma <= 0 or NULL buffers. */
tddft_status tddft_spectrum(tddft_ctx *ctx, int32_t k, const double *omega, const double *f,
                            double gamma, int32_t n, const double *E, double *S);

/* Conduction projector of the joint unoccupied representation {varphi} = {phi} (+) {chi}
 * (Sec. II C, Eq. proj): P^c = S^-1 - S^-1 S^{varphi phi} P^v S^{phi varphi} S^-1, with S the
 * overlap of the joint functions [n_joint][n_joint], S_joint_phi = S^{varphi phi}
 * [n_joint][n_phi] and P_v [n_phi][n_phi]; P_c [n_joint][n_joint] out. The result projects onto
 * the whole unoccupied space the joint functions represent; a context made with chi := the
 * joint functions, S_chi := S, H_chi := the joint Hamiltonian and this P_c solves in that
 * representation (the paper's production setting). Float64 on the device (S^-1 from the
 * coupled Newton-Schulz square roots); buffers host or device, work on cuda_stream, synchronous.
 * INVALID for non-positive sizes or NULL buffers, or when S is not positive definite. */
tddft_status tddft_joint_projector(void *cuda_stream, int32_t n_joint, int32_t n_phi,
                                   const double *S_joint, const double *S_joint_phi,
                                   const double *P_v, double *P_c);

/* Checkpoint and resume of a PCG state (Sec. III C carries, from one iteration to the next, the
 * trial pairs with their operator images and the previous search direction with its
 * preconditioned gradient; the checkpoint holds exactly these). tddft_state_export writes into
 * the caller's host buffer buf of *len bytes: with buf NULL it only stores the size needed in
 * *len; a buffer smaller than that gives INVALID (with *len set to the size). Layout: a 48-byte
 * header (magic "TDDFTST1", version 1, precision, k, N_chi, N_phi, iteration count, learned
 * fallbacks, previous-omega flag as int32, inner CG iterations as int64), the previous omega [k]
 * and five conjugation scalars as float64, then Y, P, f, cov(P), the previous direction, its
 * image, the previous preconditioned gradient and its image, each [2k][N_chi][N_phi] in the
 * context's working type (float64 for FP64, float32 for MIXED), native byte order.
 * tddft_state_import makes a new state from such a buffer (len exactly the exported size) on a
 * context of the same precision and sizes (INVALID otherwise); its further steps are those the
 * exported state would have taken, up to the rounding order of the grid integrals' atomic
 * accumulation, which varies from run to run. The caller owns buf; the state belongs to the
 * context it was imported on and is freed with tddft_state_destroy. */
tddft_status tddft_state_export(tddft_ctx *ctx, const tddft_state *st, void *buf, size_t *len);
tddft_status tddft_state_import(tddft_ctx *ctx, const void *buf, size_t len, tddft_state **out);

/* Per Ritz pair of the current subspace: omega [k] ascending and pairing [2k] =
 * |<p, f_p> - omega|, |<q, f_q> - omega| (an eigenpair has both zero; (-p, q) is then the
 * -omega partner of Eq. (1)). */
tddft_status tddft_subspace(tddft_ctx *ctx, tddft_state *st, double *omega, double *pairing);

/* Atom-pair pattern of the response kernels: mask [natoms][natoms], 1 where a chi on atom I and
 * a phi on atom J are coupled (distance <= kernel_cutoff, or everywhere with no cutoff). */
tddft_status tddft_pattern(const tddft_ctx *ctx, uint8_t *mask);

/* ---- Learned atom-block preconditioner ---------------------------------------------------------
 * A stand-in for the inner-CG solve of Eq. precond (Sec. III B) inside the PCG of Sec. III C: each
 * atom block (chi-atom I, phi-atom J) of the search gradient h goes to z_IJ = h_IJ + A_IJ h_IJ,
 * blocks read as vectors (p block then q block, row-major), with the n_b x n_b matrix A_IJ
 * predicted by a 3-layer perceptron from the block's fixed features. The map is linear in h, as
 * the CG solve is. Needs equal function counts n_c (chi) and n_v (phi) on every atom, functions
 * grouped by atom. Training rows (state i, I, J; J fastest):
 *   input  x = [b, f], b = [h^p_IJ / s, h^q_IJ / s]                 (n_b = 2 n_c n_v)
 *                      f = [M^c_II, S^chi_II, M^v_JJ, S^phi_JJ, d_IJ / 10]
 *                                                                   (n_f = 2 n_c^2 + 2 n_v^2 + 1)
 *   target y = [(z^p_IJ - h^p_IJ) / s, (z^q_IJ - h^q_IJ) / s]       (n_b)
 *   weight w = s^2 / (sum of s^2 over the rows of the same state)
 * with s the Frobenius norm of the pair (h^p_IJ, h^q_IJ), M^c = P^c H^chi, M^v = H^phi P^v, d_IJ
 * the minimum-image atom distance in bohr. The model's output for a row is A(f) b. With
 * truncation the kernel mask follows the map. When the learned direction is not a descent
 * direction of the sum functional, the step takes the CG solve instead (counted in
 * tddft_state_stats). The paper has no network: this is the learned stand-in its
 * preconditioner admits. */
typedef struct tddft_mlp tddft_mlp;

/* Model for n_b-entry blocks and n_f features with hidden width `width`, on the current device,
 * parameters zero. The perceptron is n_f -> width -> width -> n_b^2 with ReLU after the two hidden
 * layers: H1 = relu(F W1 + b1), H2 = relu(H1 W2 + b2), vec(A) = H2 W3 + b3 (A row-major).
 * Parameter vector (float32, tddft_mlp_size entries): W1 [n_f][width], b1 [width],
 * W2 [width][width], b2, W3 [width][n_b^2], b3 [n_b^2], each row-major, concatenated.
 * 1 <= n_b <= 128, 1 <= n_f, width <= 4096 (INVALID otherwise). One model serves one stream at a
 * time. */
tddft_status tddft_mlp_create(int32_t n_block, int32_t n_feat, int32_t width, tddft_mlp **out);
void tddft_mlp_destroy(tddft_mlp *m);
const char *tddft_mlp_last_error(const tddft_mlp *m);
int64_t tddft_mlp_size(const tddft_mlp *m);
/* Copy the parameter vector in (resets the Adam moments and step count) or out; host or device
 * pointers. The inference copy is the parameters rounded to bfloat16 (nearest, ties to even). */
tddft_status tddft_mlp_set(tddft_mlp *m, const float *theta);
tddft_status tddft_mlp_get(const tddft_mlp *m, float *theta);
/* Y [n][n_b] = A(f_r) b_r for rows X [n][n_b + n_f] = [b, f], with the bfloat16-rounded
 * parameters; device pointers, float32, row-major. Products on the tensor cores, float32
 * accumulation. */
tddft_status tddft_mlp_forward(tddft_mlp *m, int64_t n, const float *X, float *Y);
/* Weighted mean-squared loss L = sum_r w_r sum_j (y_rj - T_rj)^2 / (n n_b) of the model over n
 * rows with the float32 parameters, and its gradient (backpropagation; relu'(0) = 0). X, T and
 * the row weights w [n] are device pointers (w NULL: all 1); loss, grad host (either may be NULL;
 * grad has tddft_mlp_size entries). */
tddft_status tddft_mlp_loss_grad(tddft_mlp *m, int64_t n, const float *X, const float *T, const float *w,
                                 double *loss, float *grad);
/* steps Adam updates (Kingma & Ba: beta1 0.9, beta2 0.999, eps 1e-8, learning rate lr) of the
 * weighted loss on minibatches of `batch` rows: step s uses rows order[s*batch .. (s+1)*batch)
 * (host int64 indices into the n rows of X, T, w, which are device pointers; w may be NULL).
 * loss_first / loss_last (may be NULL): the loss of the first and last minibatch before their
 * updates. */
tddft_status tddft_mlp_train(tddft_mlp *m, int64_t n, const float *X, const float *T, const float *w,
                             int32_t steps, int32_t batch, float lr, const int64_t *order,
                             double *loss_first, double *loss_last);
/* n_b and n_f of the rows for this context's system (INVALID without equal per-atom counts). */
tddft_status tddft_learned_dims(const tddft_ctx *ctx, int32_t *n_block, int32_t *n_feat);
/* Bind the model used by TDDFT_PRECOND_LEARNED (NULL unbinds); the context does not own it and
 * recomputes its block maps A_IJ whenever the model's parameters change. */
tddft_status tddft_set_mlp(tddft_ctx *ctx, tddft_mlp *m);
/* Training rows at the state's current iterate: inputs from its search gradient h, targets from
 * the CG solve z = mask * Pinv(h) of Eq. precond, and row weights. X [count][n_b + n_f],
 * T [count][n_b], w [count], device pointers, count = k natoms^2 (returned); cap smaller than
 * count returns INVALID. */
tddft_status tddft_samples(tddft_ctx *ctx, tddft_state *st, int64_t cap, float *X, float *T, float *w,
                           int64_t *count);
/* Counters of a state: PCG steps taken, steps whose preconditioned direction was not a descent
 * direction and fell back (the learned map to the CG solve; in the truncated form, the inner CG
 * to the search gradient itself), and inner CG iterations summed over steps (any pointer may be
 * NULL). */
tddft_status tddft_state_stats(const tddft_state *st, int32_t *iters, int32_t *fallbacks,
                               int64_t *inner_iters);

/* Per-stage launch timing. tddft_profile(ctx, 1) clears the counters and starts recording a CUDA
 * event pair on the context's stream around every launch; tddft_profile(ctx, 0) stops. Stages:
 * gemm, response_density, potential_integrals, fft_poisson_fxc, trace, vector, small_fp64.
 * tddft_profile_read synchronises and fills up to cap entries (count = entries written). flops
 * and bytes are algorithmic counts (for response_density and potential_integrals:
 * 2 * pair_points per state and the nonzero table values plus the grids; for gemm 2MNK, and in
 * the truncated form 2 n_I n_K n_J summed over the atom-block triples that contribute). */
typedef struct {
    char name[32];
    int64_t launches;
    double ms;        /* summed event-to-event time of the stage's launches */
    double flops;
    double bytes;
} tddft_stage_stats;

tddft_status tddft_profile(tddft_ctx *ctx, int32_t enable);
tddft_status tddft_profile_read(tddft_ctx *ctx, tddft_stage_stats *out, int32_t cap, int32_t *count);

/* Algorithmic work of the grid contractions: pair_points = sum over grid points of
 * (number of chi nonzero there) * (number of phi nonzero there) = sum over (a, b) of
 * |supp chi_a  intersect  supp phi_b|; table_values = nonzero tabulated values of both sets. */
tddft_status tddft_work(const tddft_ctx *ctx, double *pair_points, double *table_values);

/* Environment variables. Each selects an alternative code path of the same operation, for
 * comparisons and tests; none skips work. TDDFT_NO_TC is read once per process, the others at
 * every tddft_create (or, for TDDFT_NO_PERSISTENT_DENSITY, at the first density launch).
 *   TDDFT_NO_TC=1                  matrix products on CUDA cores instead of tcgen05 (and with
 *                                  them the tensor-core grid kernels)
 *   TDDFT_NO_GRID_TC=1             response density and potential integrals on CUDA cores
 *   TDDFT_NO_PERSISTENT_DENSITY=1  the per-tile tensor-core density kernel instead of the
 *                                  persistent one
 *   TDDFT_NO_QUAD_GATHER=1         gather the density's P block element by element instead of
 *                                  by aligned groups of four phi
 *   TDDFT_NO_REDUCED_PRECOND=1     the inner CG of the iterative preconditioner on the full
 *                                  N_chi x N_phi space instead of the conduction x valence
 *                                  subspace
 *   TDDFT_NO_DENSITY_UNITS=1       the CUDA-core density on systems whose tiles exceed the
 *                                  per-tile tensor-core kernels, instead of the density units
 *   TDDFT_DENSITY_UNITS=1          the density units even where the per-tile kernels fit
 *   TDDFT_INTEGRALS_CHUNK=nc,np    largest chi / phi slot counts of one tensor-core integrals
 *                                  unit (multiples of 128 up to 384, and of 16 up to 128;
 *                                  default 384,128); smaller values cut tiles that would fit,
 *                                  which tests the cut on small systems */

#ifdef __cplusplus
}
#endif

#endif /* TDDFT_H */
