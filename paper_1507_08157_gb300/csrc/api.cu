// C ABI of libtddft: context construction, the batched full-TDDFT operator (Eq. operator_RPA)
// and the preconditioned CG eigensolver of Sec. III C, orchestrated on one CUDA stream.
#include "tddft.h"
#include "learned.h"
#include "solver_kernels.h"
#include "sparse.h"
#include "tddft_internal.h"

#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <initializer_list>
#include <memory>
#include <new>
#include <stdexcept>
#include <string>
#include <thread>
#include <vector>

namespace tddft {

void check(cudaError_t e, const char *where) {
    if (e != cudaSuccess) throw CudaError{e, where};
}
void check_launch(const char *where) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw CudaError{e, where};
}

namespace roots {
// kernels of the coupled Newton-Schulz iteration for the overlap square roots (float64)
__global__ void ns_init_kernel(const double *S, double inv_c, double *Y, double *Z, int n) {
    const long long tot = (long long)n * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        Y[i] = S[i] * inv_c;
        Z[i] = (i / n == i % n) ? 1.0 : 0.0;
    }
}
// T = (3 I - T) / 2 and dev = max |T_old - I| (bit pattern of a non-negative double)
__global__ void ns_step_kernel(double *T, int n, unsigned long long *dev) {
    const long long tot = (long long)n * n;
    double m = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        const double d = (i / n == i % n) ? 1.0 : 0.0;
        m = fmax(m, fabs(T[i] - d));
        T[i] = 0.5 * (3.0 * d - T[i]);
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(dev, (unsigned long long)__double_as_longlong(m));
}
// max |A - B| over n entries into *dev (bit pattern of a non-negative double)
__global__ void maxdiff_kernel(const double *A, const double *B, long long n, unsigned long long *dev) {
    double m = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m = fmax(m, fabs(A[i] - B[i]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(dev, (unsigned long long)__double_as_longlong(m));
}
__global__ void scale_kernel64(const double *X, double a, double *Y, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        Y[i] = a * X[i];
}


// two-sided Jacobi on a symmetric n x n matrix in round-robin order (set-up of the exact
// preconditioner): in round r the n (padded to even m) indices form m / 2 disjoint pairs, whose
// rotations commute; angles first, then the columns of A and V, then the rows of A
__device__ __forceinline__ void rr_pair(int m, int r, int t, int &p, int &q) {
    p = t == 0 ? m - 1 : (r + t) % (m - 1);
    q = t == 0 ? r : (r - t + m - 1) % (m - 1);
    if (p > q) {
        const int x = p;
        p = q;
        q = x;
    }
}
__global__ void jac_angles_kernel(const double *A, int n, int m, int r, double *cs) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m / 2) return;
    int p, q;
    rr_pair(m, r, t, p, q);
    double c = 1.0, sn = 0.0;
    if (q < n) {
        const double apq = A[(long long)p * n + q];
        if (apq != 0.0) {
            const double theta = (A[(long long)q * n + q] - A[(long long)p * n + p]) / (2.0 * apq);
            const double tt = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            c = rsqrt(tt * tt + 1.0);
            sn = tt * c;
        }
    }
    cs[2 * t] = c;
    cs[2 * t + 1] = sn;
}
__global__ void jac_cols_kernel(double *A, double *V, int n, int m, int r, const double *cs) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)(m / 2) * n) return;
    const int pr = (int)(i / n), row = (int)(i - (long long)pr * n);
    int p, q;
    rr_pair(m, r, pr, p, q);
    const double c = cs[2 * pr], sn = cs[2 * pr + 1];
    if (q >= n || sn == 0.0) return;
    double *a = A + (long long)row * n, *v = V + (long long)row * n;
    const double ap = a[p], aq = a[q], vp = v[p], vq = v[q];
    a[p] = c * ap - sn * aq;
    a[q] = sn * ap + c * aq;
    v[p] = c * vp - sn * vq;
    v[q] = sn * vp + c * vq;
}
__global__ void jac_rows_kernel(double *A, int n, int m, int r, const double *cs) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)(m / 2) * n) return;
    const int pr = (int)(i / n), col = (int)(i - (long long)pr * n);
    int p, q;
    rr_pair(m, r, pr, p, q);
    const double c = cs[2 * pr], sn = cs[2 * pr + 1];
    if (q >= n || sn == 0.0) return;
    const double ap = A[(long long)p * n + col], aq = A[(long long)q * n + col];
    A[(long long)p * n + col] = c * ap - sn * aq;
    A[(long long)q * n + col] = sn * ap + c * aq;
}
// sums of squares: [0] off-diagonal, [1] all (float64 atomics: only a stopping test)
__global__ void offnorm_kernel(const double *A, int n, double *out) {
    const long long tot = (long long)n * n;
    double off = 0.0, all = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        const double x = A[i] * A[i];
        all += x;
        if (i / n != i % n) off += x;
    }
    for (int o = 16; o > 0; o >>= 1) {
        off += __shfl_xor_sync(0xffffffffu, off, o);
        all += __shfl_xor_sync(0xffffffffu, all, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(out, off);
        atomicAdd(out + 1, all);
    }
}
__global__ void sym_identity_kernel(double *A, double *V, int n) {
    const long long tot = (long long)n * n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / n, c = i - r * n;
        if (r < c) {
            const double x = 0.5 * (A[i] + A[c * n + r]);
            A[i] = x;
            A[c * n + r] = x;
        }
        V[i] = r == c ? 1.0 : 0.0;
    }
}
// the exact preconditioner's denominators 1 / (lambda_c,i - lambda_v,j) from the two diagonals
__global__ void denominators_kernel(const double *Ac, int rc, const double *Av, int rv, double *D) {
    const long long tot = (long long)rc * rv;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const long long i = e / rv, j = e - i * rv;
        D[e] = 1.0 / (Ac[i * rc + i] - Av[j * rv + j]);
    }
}

// float32 -> float16 (round to nearest even), bit patterns out
__global__ void f16_kernel(const float *__restrict__ in, unsigned short *__restrict__ out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = __half_as_ushort(__float2half_rn(in[i]));
}

// deterministic pseudo-random values in [-1, 1) (splitmix64 of the index and a seed), for the
// autotuner's trial inputs
__global__ void fill_random_kernel(float *__restrict__ x, long long n, unsigned long long seed) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        x[i] = (float)((double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0);
    }
}

}  // namespace roots

namespace {
void to_f16(cudaStream_t st, const float *in, unsigned short *out, long long n) {
    if (n <= 0) return;
    roots::f16_kernel<<<(int)std::min<long long>((n + 255) / 256, 8 * 1216), 256, 0, st>>>(in, out, n);
    check_launch("f16_kernel");
}
}  // namespace

namespace {

struct InvalidArg {
    std::string msg;
};
struct Breakdown {
    std::string msg;
};
struct TimeoutErr {
    std::string msg;
};

// device ordinal of a device (or managed) pointer, -1 for anything else
int device_of(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) ? a.device : -1;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename T>
struct Impl {
    Mem mem;
    TileSet<T> chi, phi;
    T *Sc = nullptr, *Sv = nullptr, *Pc = nullptr, *Pv = nullptr, *Mc = nullptr, *Mv = nullptr;
    T *Rc = nullptr, *Rv = nullptr, *Ac = nullptr, *Av = nullptr, *mask = nullptr, *fxc = nullptr;
    // preconditioner in Loewdin variables: S^{1/2}, S^{-1/2} of both overlaps and the transformed
    // M~c = Sc^{1/2} Mc Sc^{-1/2}, M~v = Sv^{-1/2} Mv Sv^{1/2}
    T *Sch = nullptr, *Scmh = nullptr, *Svh = nullptr, *Svmh = nullptr, *Mct = nullptr, *Mvt = nullptr;
    // the same CG on orthonormal bases U_c, U_v of the ranges of the Loewdin projectors (rc, rv > 0
    // when P^c and P^v are idempotent): in Wc = U_c^T Sc^{1/2} [rc][nc], Wv = Sv^{1/2} U_v [nv][rv],
    // out Vc = Sc^{-1/2} U_c [nc][rc], Vv = U_v^T Sv^{-1/2} [rv][nv], operators Mch = U_c^T M~c U_c,
    // Mvh = U_v^T M~v U_v
    int rc = 0, rv = 0;
    T *Wc = nullptr, *Wv = nullptr, *Vc = nullptr, *Vv = nullptr, *Mch = nullptr, *Mvh = nullptr;
    // exact preconditioner: Wc, Wv, Vc, Vv taken into the eigenbases of Mch and Mvh, and the
    // denominators Dn [rc][rv] = 1 / (lambda_c,i - lambda_v,j)
    bool exact = false;
    T *Dn = nullptr;
    double *fxc64 = nullptr;
    // tensor-core grid path (float32 contexts): point-major f16 chi tables [tile][512][CK]
    unsigned short *chi_pm = nullptr;
    unsigned short *chi_fm16 = nullptr;   // function-major f16 chi tables [slot][512]
    unsigned short *phi_fm16 = nullptr;   // function-major f16 phi tables [slot][512]
    unsigned short *phi_pm = nullptr;     // point-major f16 phi tables [tile][512][NPmax], zero padded
    // dense tiles: density units with chunked point-major f16 tables ([chunk][512][64] chi,
    // [chunk][512][32] phi)
    bool dens_units = false;              // the density runs on units (selected)
    bool units_ok = false;                // chunked tables built (every tile's phi in whole quads)
    unsigned short *chi_pmc = nullptr, *phi_pmc = nullptr;
    long long nchunks_chi = 0;
    DUnit *dunits = nullptr;
    int ndunits = 0;
    int dens_cut[2] = {320, 128}, int_cut[2] = {384, 128};   // unit cuts in use (chi, phi)
    std::vector<int> coff_h, poff_h, cfirst_h, pfirst_h;    // host tile offsets, first chunks
    Mem umem_dens, umem_int;              // unit lists (replaced when the autotuner recuts)
    int *live_tiles = nullptr;            // tiles with both chi and phi (the persistent density's items)
    int nlive = 0;
    int CK = 0, NPmax = 0, nslots_chi = 0, nslots_phi = 0, maxc = 0;
    int NPint = 0;            // phi rows of the integrals' B stage (the largest unit's phi, to 16)
    bool grid_tc = false, integrals_tc = false;
    bool phi_quads = false;   // every tile's phi list is whole aligned groups of 4 (vector gather)
    // integrals launches: units (tiles, or chunks of dense tiles) grouped by 128-row chi blocks
    VTile *int_units = nullptr;
    int int_count[3] = {0, 0, 0};
    unsigned *tc_bits = nullptr;
    float *tc_scale = nullptr;
    // operator workspace, sized for up to `cap` grid states
    Mem wmem;
    int cap = 0;
    T *rho = nullptr, *V = nullptr, *Vmat = nullptr, *tmp = nullptr, *bufP = nullptr, *bufF = nullptr;
    void *fft = nullptr;
    double *stage = nullptr;
    // learned preconditioner: per-atom features, feature rows of the na^2 blocks and their maps A
    // (lmemf); block scales for `lrows` sample rows (lmemr)
    Mem lmemf, lmemr;
    long long lrows = 0;
    float *lfc = nullptr, *lfv = nullptr, *ldist = nullptr, *lF = nullptr, *lA = nullptr, *ls = nullptr;
    const tddft_mlp *lA_model = nullptr;
    long long lA_version = -1;
    // truncated (sparse) form: constants as cluster blocks in T (chi x chi, phi x phi, and the phi
    // ones transposed for the tensor-core products), a dense scratch for the grid kernels and the
    // transposed right operands of the tensor-core left products (workspace)
    T *cc[SP_NCONST] = {}, *vv[SP_NCONST] = {}, *vvT[SP_NCONST] = {};
    T *dense = nullptr, *opT = nullptr;
};

}  // namespace
}  // namespace tddft

using namespace tddft;

struct tddft_ctx {
    cudaStream_t st = nullptr;
    tddft_options opt{};
    int prec = TDDFT_FP64;
    int n = 0, nt = 0, natoms = 0, nc = 0, nv = 0;
    double cell = 0.0, dV = 0.0;
    bool trunc = false;
    double pair_points = 0.0, table_values = 0.0;
    Profiler *prof = nullptr;
    bool prof_on = false;
    std::vector<uint8_t> amask;
    // equal per-atom function counts (atom-major order) for the learned preconditioner
    bool uniform = false;
    int nca = 0, nva = 0;
    std::vector<float> adist;     // [natoms][natoms] minimum-image distance / 10 bohr
    tddft_mlp *mlp = nullptr;
    std::string err;
    std::unique_ptr<Impl<double>> d64;
    std::unique_ptr<Impl<float>> d32;
    // contexts of a batch own their stream and wait on it through a blocking-sync event, so that
    // many host threads can drive systems at once without spinning
    bool own_stream = false;
    cudaEvent_t sync_ev = nullptr;
    int *hword = nullptr;   // pinned: the tensor-core kernels' error word, read with each status
    int device = 0;         // the CUDA device the context was made on
    bool sparse = false;    // truncated (linear-scaling) form: cluster-blocked matrices
    std::unique_ptr<SparseLayout> sp;
    GridShape grid() const { return GridShape{n, nt, cell, dV, pair_points, table_values}; }
    ~tddft_ctx();
    long long len() const { return sparse ? sp->len() : (long long)nc * nv; }
    long long nnz_abi() const { return sparse ? sp->nnz_abi : (long long)nc * nv; }   // values per state at the ABI
    long long n3() const { return (long long)n * n * n; }
};

namespace tddft {
bool tc_enabled();
int *tc_error_word();
void tc_error_fetch(cudaStream_t st, int *host);
void tc_release_stream(cudaStream_t st);
void tc_error_clear(cudaStream_t st);
void tc_wait_probe(cudaStream_t st);
void build_point_major_f16(const int *off_h, const float *val_h_or_null, const double *vald_h_or_null,
                           int ntiles, int CK, unsigned short *out_h);
int density_tc_group(int KBmax, int NP, int k);
int integrals_tc_group(int NP, int k, int maxc);
void potential_integrals_tc(cudaStream_t st, const GridShape &g, const TileSet<float> &chi,
                            const TileSet<float> &phi, const unsigned short *chi_fm16, int nslots,
                            const unsigned short *phi_fm16, int nslots_phi, int NPmax,
                            int maxc, int nchi, int nphi, const float *V, int k, float *out, unsigned *scratch_bits,
                            float *scale, const VTile *unit_list, const int *units_by_blocks, int *err);
void response_density_tc(cudaStream_t st, const GridShape &g, const TileSet<float> &chi,
                         const TileSet<float> &phi, const unsigned short *chi_pm, int CK, int NPmax, int nphi,
                         const float *P, long long sP, int k, float *rho, unsigned *scratch_bits,
                         float *scale, int *err, bool phi_quads, const unsigned short *phi_pm,
                         const int *live_tiles, int nlive);
long long build_chunked_pm(cudaStream_t st, Mem &mem, const TileSet<float> &ts, const std::vector<int> &off_h, int W,
                           unsigned short **out, std::vector<int> &first);
void response_density_units(cudaStream_t st, const GridShape &g, const TileSet<float> &chi, const TileSet<float> &phi,
                            const unsigned short *chi_pmc, long long nchunks_chi, const unsigned short *phi_pmc,
                            const DUnit *units, int nunits, int nphi, const float *P, long long sP, int k, float *rho,
                            unsigned *scratch_bits, float *scale, int *err);
int noalloc_max_states();
void response_density_tc_noalloc(cudaStream_t st, const GridShape &g, const TileSet<float> &chi,
                                 const TileSet<float> &phi, const unsigned short *chi_pm, int CK, int NPmax,
                                 int nphi, const float *P, long long sP, int k, float *rho,
                                 const unsigned short *phi_pm);
int response_density_tc_noalloc_error(cudaStream_t st);
Profiler *profiler_new();
void profiler_delete(Profiler *p);
void profiler_read(Profiler *p, long long *launches, double *ms, double *flops, double *bytes);
void profiler_reset(Profiler *p);
}  // namespace tddft

namespace {
// float32 constants of a context: the tensor-core GEMM caches their split copies
void register_constants(Impl<float> &I) {
    const float *ps[] = {I.Sc, I.Sv, I.Pc, I.Pv, I.Mc, I.Mv, I.Rc, I.Rv, I.Ac, I.Av, I.Sch, I.Scmh, I.Svh, I.Svmh,
                         I.Mct, I.Mvt, I.Wc, I.Wv, I.Vc, I.Vv, I.Mch, I.Mvh};
    for (const float *p : ps)
        if (p) tc_register_constant(p);
}
void register_constants(Impl<double> &) {}
}  // namespace

tddft_ctx::~tddft_ctx() {
    if (own_stream && st) cudaStreamSynchronize(st);
    if (prof) profiler_delete(prof);
    if (d32) {
        Impl<float> &I = *d32;
        const float *ps[] = {I.Sc, I.Sv, I.Pc, I.Pv, I.Mc, I.Mv, I.Rc, I.Rv, I.Ac, I.Av, I.Sch, I.Scmh, I.Svh, I.Svmh,
                             I.Mct, I.Mvt, I.Wc, I.Wv, I.Vc, I.Vv, I.Mch, I.Mvh};
        for (const float *p : ps)
            if (p) tc_unregister_constant(p);
    }
    d64.reset();
    d32.reset();
    if (sync_ev) cudaEventDestroy(sync_ev);
    if (hword) cudaFreeHost(hword);
    if (own_stream && st) {
        tc_release_stream(st);
        cudaStreamDestroy(st);
    }
}

namespace {

template <typename T> Impl<T> &impl(tddft_ctx *c);
template <> Impl<double> &impl<double>(tddft_ctx *c) { return *c->d64; }
template <> Impl<float> &impl<float>(tddft_ctx *c) { return *c->d32; }

// wait for the context's stream: a blocking-sync event for batch contexts, else a stream sync
cudaError_t ctx_sync(tddft_ctx *c) {
    if (c->sync_ev) {
        cudaError_t e = cudaEventRecord(c->sync_ev, c->st);
        return e != cudaSuccess ? e : cudaEventSynchronize(c->sync_ev);
    }
    return cudaStreamSynchronize(c->st);
}

struct ProfilerBinding {
    ProfilerBinding(tddft_ctx *c) { active_profiler() = (c->prof_on ? c->prof : nullptr); }
    ~ProfilerBinding() { active_profiler() = nullptr; }
};

// the context's bounded-wait limit for the kernels launched during one call
struct WaitLimitBinding {
    WaitLimitBinding(tddft_ctx *c) {
        active_wait_limit() = c->opt.spin_limit_cycles > 0 ? (long long)c->opt.spin_limit_cycles : DEFAULT_WAIT_LIMIT;
    }
    ~WaitLimitBinding() { active_wait_limit() = DEFAULT_WAIT_LIMIT; }
};

template <typename F>
tddft_status guarded(tddft_ctx *c, F &&f) {
    try {
        ProfilerBinding pb(c);
        WaitLimitBinding wb(c);
        return f();
    } catch (const CudaError &e) {
        c->err = std::string(e.where) + ": " + cudaGetErrorString(e.code);
        cudaGetLastError();
        return e.code == cudaErrorMemoryAllocation ? TDDFT_E_NOMEM : TDDFT_E_CUDA;
    } catch (const InvalidArg &e) {
        c->err = e.msg;
        return TDDFT_E_INVALID;
    } catch (const Breakdown &e) {
        c->err = e.msg;
        return TDDFT_E_BREAKDOWN;
    } catch (const TimeoutErr &e) {
        c->err = e.msg;
        return TDDFT_E_TIMEOUT;
    } catch (const std::bad_alloc &) {
        c->err = "out of memory";
        return TDDFT_E_NOMEM;
    }
}

// ---- grid tables -------------------------------------------------------------------------------
// value i of a function set's tables (float64, or float32 when val is null)
struct FuncVals {
    const double *v64;
    const float *v32;
    double operator[](long long i) const { return v64 ? v64[i] : (double)v32[i]; }
};

template <typename T>
void build_tiles(const tddft_funcs &fs, int n, int nt, Mem &mem, TileSet<T> &out,
                 std::vector<int> &cnt) {
    const int ntiles = nt * nt * nt;
    const int nf = fs.nfun;
    const FuncVals fv{fs.val, fs.val32};
    std::vector<std::vector<int>> ftiles(nf);
#pragma omp parallel
    {
        std::vector<int> mark(ntiles, 0);
        int stamp = 0;
#pragma omp for schedule(dynamic, 4)
        for (int f = 0; f < nf; ++f) {
            ++stamp;
            const int *b = fs.box + 6 * f;
            const long long v = fs.off[f];
            for (int i = 0; i < b[3]; ++i) {
                const int gx = (b[0] + i) % n;
                for (int j = 0; j < b[4]; ++j) {
                    const int gy = (b[1] + j) % n;
                    const long long row = v + ((long long)i * b[4] + j) * b[5];
                    for (int l = 0; l < b[5]; ++l) {
                        if (fv[row + l] == 0.0) continue;
                        const int gz = (b[2] + l) % n;
                        const int t = ((gx / TILE) * nt + gy / TILE) * nt + gz / TILE;
                        if (mark[t] != stamp) {
                            mark[t] = stamp;
                            ftiles[f].push_back(t);
                        }
                    }
                }
            }
        }
    }
    // functions of one atom that share a box are listed together on every tile any of them
    // touches (a narrow function's table may hold exact zeros where its neighbours do not), so
    // that an atom's functions stay consecutive in every tile's list
    for (int f0 = 0; f0 < nf;) {
        int f1 = f0 + 1;
        while (f1 < nf && fs.atom[f1] == fs.atom[f0] && std::equal(fs.box + 6 * f1, fs.box + 6 * f1 + 6, fs.box + 6 * f0))
            ++f1;
        if (f1 - f0 > 1) {
            std::vector<int> u;
            for (int f = f0; f < f1; ++f) u.insert(u.end(), ftiles[f].begin(), ftiles[f].end());
            std::sort(u.begin(), u.end());
            u.erase(std::unique(u.begin(), u.end()), u.end());
            for (int f = f0; f < f1; ++f) ftiles[f] = u;
        }
        f0 = f1;
    }
    std::vector<int> off(ntiles + 1, 0);
    for (int f = 0; f < nf; ++f)
        for (int t : ftiles[f]) off[t + 1]++;
    int maxper = 0;
    for (int t = 0; t < ntiles; ++t) {
        maxper = std::max(maxper, off[t + 1]);
        off[t + 1] += off[t];
    }
    const long long slots = off[ntiles];
    std::vector<int> ids(slots);
    std::vector<std::vector<int>> fslot(nf);
    {
        std::vector<int> pos(off.begin(), off.end() - 1);
        for (int f = 0; f < nf; ++f) {
            fslot[f].reserve(ftiles[f].size());
            for (int t : ftiles[f]) {
                fslot[f].push_back(pos[t]);
                ids[pos[t]++] = f;
            }
        }
    }
    std::vector<T> val((size_t)slots * TILE_PTS, T(0));
#pragma omp parallel
    {
        std::vector<int> slot_of(ntiles, -1);
#pragma omp for schedule(dynamic, 4)
        for (int f = 0; f < nf; ++f) {
            for (size_t a = 0; a < ftiles[f].size(); ++a) slot_of[ftiles[f][a]] = fslot[f][a];
            const int *b = fs.box + 6 * f;
            const long long v = fs.off[f];
            for (int i = 0; i < b[3]; ++i) {
                const int gx = (b[0] + i) % n;
                for (int j = 0; j < b[4]; ++j) {
                    const int gy = (b[1] + j) % n;
                    const long long row = v + ((long long)i * b[4] + j) * b[5];
                    for (int l = 0; l < b[5]; ++l) {
                        const double x = fv[row + l];
                        if (x == 0.0) continue;
                        const int gz = (b[2] + l) % n;
                        const int t = ((gx / TILE) * nt + gy / TILE) * nt + gz / TILE;
                        const int lp = ((gx % TILE) * TILE + gy % TILE) * TILE + gz % TILE;
                        val[(size_t)slot_of[t] * TILE_PTS + lp] = T(x);
                    }
                }
            }
            for (int t : ftiles[f]) slot_of[t] = -1;
        }
    }
    // nonzero values per (tile, point), for the algorithmic work counts
    cnt.assign((size_t)ntiles * TILE_PTS, 0);
#pragma omp parallel for schedule(dynamic, 16)
    for (int t = 0; t < ntiles; ++t)
        for (int sl = off[t]; sl < off[t + 1]; ++sl)
            for (int lp = 0; lp < TILE_PTS; ++lp)
                if (val[(size_t)sl * TILE_PTS + lp] != T(0)) cnt[(size_t)t * TILE_PTS + lp]++;
    int *d_off = mem.template alloc<int>(off.size());
    int *d_ids = mem.template alloc<int>(ids.size());
    T *d_val = mem.template alloc<T>(val.size());
    check(cudaMemcpy(d_off, off.data(), off.size() * sizeof(int), cudaMemcpyHostToDevice), "upload tile off");
    check(cudaMemcpy(d_ids, ids.data(), ids.size() * sizeof(int), cudaMemcpyHostToDevice), "upload tile ids");
    check(cudaMemcpy(d_val, val.data(), val.size() * sizeof(T), cudaMemcpyHostToDevice), "upload tile values");
    out.ntiles = ntiles;
    out.max_per_tile = maxper;
    out.off = d_off;
    out.ids = d_ids;
    out.val = d_val;
}

void validate_funcs(const tddft_funcs &fs, int n, int natoms, const char *name) {
    if (fs.nfun <= 0 || !fs.atom || !fs.box || !fs.off || (!fs.val && !fs.val32))
        throw InvalidArg{std::string(name) + ": empty or null function set"};
    if (fs.off[0] != 0) throw InvalidArg{std::string(name) + ": off[0] must be 0"};
    for (int f = 0; f < fs.nfun; ++f) {
        const int *b = fs.box + 6 * f;
        for (int a = 0; a < 3; ++a)
            if (b[a] < 0 || b[a] >= n || b[3 + a] < 1 || b[3 + a] > n)
                throw InvalidArg{std::string(name) + ": box out of range (origin in [0,n), extent in [1,n])"};
        if (fs.off[f + 1] - fs.off[f] != (long long)b[3] * b[4] * b[5])
            throw InvalidArg{std::string(name) + ": off does not match the box extents"};
        if (fs.atom[f] < 0 || fs.atom[f] >= natoms) throw InvalidArg{std::string(name) + ": atom index out of range"};
    }
}

// ---- transfers at the ABI ----------------------------------------------------------------------
template <typename T>
void upload(tddft_ctx *c, Impl<T> &I, const double *src, T *dst, long long count) {
    if (is_device_ptr(src)) {
        convert<double, T>(c->st, src, dst, count);
    } else {
        check(cudaMemcpyAsync(I.stage, src, count * sizeof(double), cudaMemcpyHostToDevice, c->st), "H2D");
        convert<double, T>(c->st, I.stage, dst, count);
    }
}

template <typename T>
void download(tddft_ctx *c, Impl<T> &I, const T *src, double *dst, long long count) {
    if (!dst) return;
    if (is_device_ptr(dst)) {
        convert<T, double>(c->st, src, dst, count);
    } else {
        convert<T, double>(c->st, src, I.stage, count);
        check(cudaMemcpyAsync(dst, I.stage, count * sizeof(double), cudaMemcpyDeviceToHost, c->st), "D2H");
        check(ctx_sync(c), "sync D2H");
    }
}

template <> void download<double>(tddft_ctx *c, Impl<double> &I, const double *src, double *dst, long long count) {
    if (!dst) return;
    check(cudaMemcpyAsync(dst, src, count * sizeof(double), cudaMemcpyDefault, c->st), "copy out");
    check(ctx_sync(c), "sync copy out");
}

// k chi x phi matrices across the ABI: dense [k][N_chi][N_phi], or in a sparse context [k][nnz]
// in the atom-blocked order of the kernel pattern (converted to and from the cluster blocks)
template <typename T>
void abi_in(tddft_ctx *c, Impl<T> &I, const double *src, T *dst, int k) {
    if (!c->sparse) {
        upload<T>(c, I, src, dst, (long long)k * c->len());
        return;
    }
    const long long n = (long long)k * c->nnz_abi();
    const double *d = src;
    if (!is_device_ptr(src)) {
        check(cudaMemcpyAsync(I.stage, src, n * sizeof(double), cudaMemcpyHostToDevice, c->st), "H2D");
        d = I.stage;
    }
    cb_from_abi<T>(c->st, *c->sp, d, dst, k);
}

template <typename T>
void abi_out(tddft_ctx *c, Impl<T> &I, const T *src, double *dst, int k) {
    if (!dst) return;
    if (!c->sparse) {
        download<T>(c, I, src, dst, (long long)k * c->len());
        return;
    }
    const long long n = (long long)k * c->nnz_abi();
    if (is_device_ptr(dst)) {
        cb_to_abi<T>(c->st, *c->sp, src, dst, k);
    } else {
        cb_to_abi<T>(c->st, *c->sp, src, I.stage, k);
        check(cudaMemcpyAsync(dst, I.stage, n * sizeof(double), cudaMemcpyDeviceToHost, c->st), "D2H");
        check(ctx_sync(c), "sync D2H");
    }
}

// workspace for the operator on up to `states` grid states (2k for a batch of k pairs)
template <typename T>
void ensure_workspace(tddft_ctx *c, Impl<T> &I, int states) {
    if (states <= I.cap) return;
    check(ctx_sync(c), "sync before workspace");
    I.wmem.release();
    const long long len = c->len(), n3 = c->n3();
    I.rho = I.wmem.template alloc<T>((size_t)states * n3);
    I.V = I.wmem.template alloc<T>((size_t)states * n3);
    I.fft = I.wmem.template alloc<T>((size_t)((states + 1) / 2) * n3 * 2);
    I.Vmat = I.wmem.template alloc<T>((size_t)states * len);
    I.tmp = I.wmem.template alloc<T>((size_t)states * len);
    I.bufP = I.wmem.template alloc<T>((size_t)states * len);
    I.bufF = I.wmem.template alloc<T>((size_t)states * len);
    I.stage = I.wmem.template alloc<double>(
        (size_t)std::max({states * len, states * n3, states * c->nnz_abi()}));
    I.tc_bits = I.wmem.template alloc<unsigned>((size_t)states);
    I.tc_scale = I.wmem.template alloc<float>((size_t)states);
    if (c->sparse) {
        // the grid kernels address P and V densely; the tensor-core left products take their
        // right operand block-transposed
        I.dense = I.wmem.template alloc<T>((size_t)states * c->nc * c->nv);
        I.opT = I.wmem.template alloc<T>((size_t)states * len);
    }
    I.cap = states;
}

// response density of ns states into I.rho: tensor cores (f16 operands) for float32 contexts
// whose tiles fit, CUDA cores otherwise
template <typename T>
void density(tddft_ctx *c, Impl<T> &I, const T *P, int ns) {
    if (c->sparse) {
        cb_to_dense<T>(c->st, *c->sp, P, I.dense, ns);
        P = I.dense;
    }
    if constexpr (sizeof(T) == 4) {
        if (I.dens_units) {
            response_density_units(c->st, c->grid(), I.chi, I.phi, I.chi_pmc, I.nchunks_chi, I.phi_pmc, I.dunits,
                                   I.ndunits, c->nv, P, (long long)c->nc * c->nv, ns, I.rho, I.tc_bits, I.tc_scale,
                                   tc_error_word());
            return;
        }
        if (I.grid_tc) {
            response_density_tc(c->st, c->grid(), I.chi, I.phi, I.chi_pm, I.CK, I.NPmax, c->nv, P,
                                (long long)c->nc * c->nv, ns,
                                I.rho, I.tc_bits, I.tc_scale, tc_error_word(), I.phi_quads, I.phi_pm,
                                I.live_tiles, I.nlive);
            return;
        }
    }
    response_density<T>(c->st, c->grid(), I.chi, I.phi, c->nv, P, (long long)c->nc * c->nv, ns, I.rho);
}

template <typename T>
void integrals(tddft_ctx *c, Impl<T> &I, int ns) {
    // sparse form: the dense integrals into the scratch, then T(V) into the cluster blocks
    T *out = c->sparse ? I.dense : I.Vmat;
    bool done = false;
    if constexpr (sizeof(T) == 4) {
        if (I.integrals_tc) {
            potential_integrals_tc(c->st, c->grid(), I.chi, I.phi, I.chi_fm16, I.nslots_chi, I.phi_fm16, I.nslots_phi,
                                   I.NPint, I.maxc, c->nc,
                                   c->nv, I.V, ns, out, I.tc_bits, I.tc_scale, I.int_units, I.int_count,
                                   tc_error_word());
            done = true;
        }
    }
    if (!done) potential_integrals<T>(c->st, c->grid(), I.chi, I.phi, c->nc, c->nv, I.V, ns, out);
    if (c->sparse) cb_from_dense<T>(c->st, *c->sp, I.dense, I.Vmat, I.mask, ns);
}

// ---- products with the constants -------------------------------------------------------------------
// chi x chi constant by role (SP_M: P^c H^chi, SP_P: P^c, SP_R: P^c S^chi, SP_A: S^chi P^c S^chi,
// SP_S: S^chi) and the phi x phi ones (H^phi P^v, P^v, S^phi P^v, S^phi P^v S^phi, S^phi)
template <typename T>
const T *cconst(Impl<T> &I, int x) {
    const T *m[SP_NCONST] = {I.Mc, I.Pc, I.Rc, I.Ac, I.Sc};
    return m[x];
}
template <typename T>
const T *vconst(Impl<T> &I, int x) {
    const T *m[SP_NCONST] = {I.Mv, I.Pv, I.Rv, I.Av, I.Sv};
    return m[x];
}

bool sparse_tc(tddft_ctx *c) { return c->prec == TDDFT_MIXED && tc_enabled() && bsr_tc_available(); }

// out_b = alpha C_x X_b + beta out_b for nb chi x phi matrices; in the sparse form a block-sparse
// product cut to the kernel pattern (Sec. IV truncation)
template <typename T>
void lprod(tddft_ctx *c, Impl<T> &I, int x, const T *X, T *out, int nb, T alpha, T beta, bool approx = false) {
    const long long len = c->len();
    if (!c->sparse) {
        const int nc = c->nc, nv = c->nv;
        gemm<T>(c->st, false, false, nc, nv, nc, alpha, cconst(I, x), nc, 0, X, nv, len, beta, out, nv, len, nb, approx);
        return;
    }
    const SparseLayout &L = *c->sp;
    const PairList &pl = L.left[x];
    ProfScope ps(c->st, ST_GEMM, pl.alg_flops * nb,
                 sizeof(T) * ((double)L.cc_len(x) + (double)len * nb * (beta == T(0) ? 2 : 3)));
    if constexpr (sizeof(T) == 4) {
        if (sparse_tc(c)) {
            bsr_transpose<T>(c->st, X, I.opT, CB_R, CB_C, L.pk.nnzb(), nb);
            bsr_tc(c->st, CB_R, pl, L.pcc[x].nnzb(), (const float *)I.cc[x], 0, L.pk.nnzb(), (const float *)I.opT, len,
                   (float *)out, len, nb, (float)alpha, (float)beta, (const float *)I.mask, approx);
            return;
        }
    }
    bsr_simt<T>(c->st, CB_R, CB_R, CB_C, pl, L.pk.nnzb(), I.cc[x], 0, X, len, out, len, nb, alpha, beta, I.mask);
}

// out_b = alpha X_b D_x + beta out_b
template <typename T>
void rprod(tddft_ctx *c, Impl<T> &I, const T *X, int x, T *out, int nb, T alpha, T beta, bool approx = false) {
    const long long len = c->len();
    if (!c->sparse) {
        const int nc = c->nc, nv = c->nv;
        gemm<T>(c->st, false, false, nb * nc, nv, nv, alpha, X, nv, 0, vconst(I, x), nv, 0, beta, out, nv, 0, 1, approx);
        return;
    }
    const SparseLayout &L = *c->sp;
    const PairList &pl = L.right[x];
    ProfScope ps(c->st, ST_GEMM, pl.alg_flops * nb,
                 sizeof(T) * ((double)L.vv_len(x) + (double)len * nb * (beta == T(0) ? 2 : 3)));
    if constexpr (sizeof(T) == 4) {
        if (sparse_tc(c)) {
            bsr_tc(c->st, CB_C, pl, L.pk.nnzb(), (const float *)X, len, L.pvv[x].nnzb(), (const float *)I.vvT[x], 0,
                   (float *)out, len, nb, (float)alpha, (float)beta, (const float *)I.mask, approx);
            return;
        }
    }
    bsr_simt<T>(c->st, CB_R, CB_C, CB_C, pl, L.pk.nnzb(), X, len, I.vv[x], 0, out, len, nb, alpha, beta, I.mask);
}

// the error word of the tensor-core kernels (bounded waits that expired), read with one stream wait
void check_tc_error(tddft_ctx *c) {
    tc_error_fetch(c->st, c->hword);
    check(ctx_sync(c), "sync tc error");
    if (*c->hword) {
        tc_error_clear(c->st);
        throw TimeoutErr{"a bounded wait in a tensor-core kernel expired"};
    }
}

// ---- the operator (Eq. operator_RPA) -------------------------------------------------------------
// P, f: [2][k][N_chi][N_phi] (the k p-matrices, then the k q-matrices). With `mirror` in TDA mode
// the caller guarantees p = q (the solver's iterates in the Tamm-Dancoff approximation, where
// X is the only unknown): A is applied to the p half alone and f_q is a copy of f_p.
template <typename T>
void apply_impl(tddft_ctx *c, Impl<T> &I, int k, const T *P, T *f, bool mirror = false) {
    if (mirror && c->opt.mode == TDDFT_MODE_TDA) {
        const long long len = c->len();
        ensure_workspace(c, I, 2 * k);
        cudaStream_t st = c->st;
        lprod<T>(c, I, SP_M, P, f, k, T(1), T(0));
        rprod<T>(c, I, P, SP_M, f, k, T(-1), T(1));
        density(c, I, P, k);
        hartree_fxc<T>(st, c->grid(), I.rho, I.fxc, k, I.V, I.fft);
        integrals(c, I, k);
        lprod<T>(c, I, SP_P, I.Vmat, I.tmp, k, T(1), T(0));
        rprod<T>(c, I, I.tmp, SP_P, f, k, T(1), T(1));
        check(cudaMemcpyAsync(f + k * len, f, k * len * sizeof(T), cudaMemcpyDeviceToDevice, st), "mirror f_q");
        return;
    }
    ensure_workspace(c, I, 2 * k);
    const long long len = c->len();
    cudaStream_t st = c->st;
    // Kohn-Sham difference part: f = (P^c H^chi) P - P (H^phi P^v) on all 2k matrices
    lprod<T>(c, I, SP_M, P, f, 2 * k, T(1), T(0));
    rprod<T>(c, I, P, SP_M, f, 2 * k, T(-1), T(1));
    if (c->opt.mode == TDDFT_MODE_D_ONLY) return;
    const bool tda = c->opt.mode == TDDFT_MODE_TDA;
    const int ns = tda ? 2 * k : k;
    const T *Ps = tda ? P : P + k * len;
    T *fs = tda ? f : f + k * len;
    const T alpha = tda ? T(1) : T(2);
    const GridShape g = c->grid();
    density(c, I, Ps, ns);
    hartree_fxc<T>(st, g, I.rho, I.fxc, ns, I.V, I.fft);
    integrals(c, I, ns);
    // coupling: f_q += 2 P^c V_SCF P^v
    lprod<T>(c, I, SP_P, I.Vmat, I.tmp, ns, T(1), T(0));
    rprod<T>(c, I, I.tmp, SP_P, fs, ns, alpha, T(1));
}

// ---- context construction ----------------------------------------------------------------------
// S^{1/2} and S^{-1/2} of a symmetric positive definite n x n matrix (device, float64): Y -> A^{1/2},
// Z -> A^{-1/2} for A = S / c, c >= the largest eigenvalue (max absolute row sum of the host copy)
void overlap_roots(cudaStream_t st, Mem &tmp, const double *S_dev, const double *S_host, int n, double *Sh,
                   double *Smh) {
    double c = 0.0;
    for (int i = 0; i < n; ++i) {
        double r = 0.0;
        for (int j = 0; j < n; ++j) r += std::fabs(S_host[(size_t)i * n + j]);
        c = std::max(c, r);
    }
    if (!(c > 0.0)) throw InvalidArg{"overlap matrix is zero"};
    const long long nn = (long long)n * n;
    double *Y = tmp.alloc<double>(nn), *Z = tmp.alloc<double>(nn), *T = tmp.alloc<double>(nn);
    double *Y2 = tmp.alloc<double>(nn), *Z2 = tmp.alloc<double>(nn);
    unsigned long long *dev = tmp.alloc<unsigned long long>(1);
    const int gb = (int)std::min<long long>((nn + 255) / 256, 1216);
    roots::ns_init_kernel<<<gb, 256, 0, st>>>(S_dev, 1.0 / c, Y, Z, n);
    check_launch("ns_init");
    int settled = 0;
    for (int it = 0; it < 100 && settled < 2; ++it) {
        gemm<double>(st, false, false, n, n, n, 1.0, Z, n, 0, Y, n, 0, 0.0, T, n, 0, 1);   // T = Z Y
        check(cudaMemsetAsync(dev, 0, sizeof(unsigned long long), st), "memset ns dev");
        roots::ns_step_kernel<<<gb, 256, 0, st>>>(T, n, dev);
        check_launch("ns_step");
        gemm<double>(st, false, false, n, n, n, 1.0, Y, n, 0, T, n, 0, 0.0, Y2, n, 0, 1);  // Y T
        gemm<double>(st, false, false, n, n, n, 1.0, T, n, 0, Z, n, 0, 0.0, Z2, n, 0, 1);  // T Z
        std::swap(Y, Y2);
        std::swap(Z, Z2);
        unsigned long long hb = 0;
        check(cudaMemcpyAsync(&hb, dev, sizeof(hb), cudaMemcpyDeviceToHost, st), "D2H ns dev");
        check(cudaStreamSynchronize(st), "sync ns");
        double d;
        std::memcpy(&d, &hb, sizeof(d));
        if (!std::isfinite(d)) throw InvalidArg{"overlap square root did not converge (matrix not positive definite?)"};
        // quadratic convergence: once |ZY - I| is below 1e-10 one more step reaches the rounding floor
        if (d < 1e-10) ++settled;
    }
    if (settled < 2) throw InvalidArg{"overlap square root did not converge (matrix not positive definite?)"};
    roots::scale_kernel64<<<gb, 256, 0, st>>>(Y, std::sqrt(c), Sh, nn);
    check_launch("scale root");
    roots::scale_kernel64<<<gb, 256, 0, st>>>(Z, 1.0 / std::sqrt(c), Smh, nn);
    check_launch("scale inverse root");
}

// Orthonormal basis U [n][r] of the range of the Loewdin projector Pi = Sh P Sh (Sh = S^{1/2}),
// r = round(trace Pi): U = Y (Y^T Y)^{-1/2} with Y = Pi Omega, Omega a seeded Gaussian n x r
// matrix. Returns r, or 0 when Pi is not idempotent to 1e-8 (then no reduced space is used).
// A = V diag(A') V^T for a symmetric n x n float64 matrix on the device: A is symmetrised and
// overwritten by its (numerically) diagonal form A', V receives the eigenvectors as columns
void sym_eig(cudaStream_t st, Mem &tmp, double *A, int n, double *V) {
    const int m = n + (n & 1), half = m / 2;
    double *cs = tmp.alloc<double>((size_t)m + 2), *nrm = tmp.alloc<double>(2);
    const long long nn = (long long)n * n, work = (long long)half * n;
    const int g1 = (int)std::min<long long>((nn + 255) / 256, 1216);
    roots::sym_identity_kernel<<<g1, 256, 0, st>>>(A, V, n);
    check_launch("sym_identity");
    double h[2];
    for (int sweep = 0; sweep < 30; ++sweep) {
        check(cudaMemsetAsync(nrm, 0, 2 * sizeof(double), st), "memset offnorm");
        roots::offnorm_kernel<<<g1, 256, 0, st>>>(A, n, nrm);
        check_launch("offnorm");
        check(cudaMemcpyAsync(h, nrm, 2 * sizeof(double), cudaMemcpyDeviceToHost, st), "D2H offnorm");
        check(cudaStreamSynchronize(st), "sync offnorm");
        if (!(h[0] > 1e-28 * h[1])) break;
        for (int r = 0; r < m - 1; ++r) {
            roots::jac_angles_kernel<<<(half + 127) / 128, 128, 0, st>>>(A, n, m, r, cs);
            roots::jac_cols_kernel<<<(int)((work + 255) / 256), 256, 0, st>>>(A, V, n, m, r, cs);
            roots::jac_rows_kernel<<<(int)((work + 255) / 256), 256, 0, st>>>(A, n, m, r, cs);
        }
        check_launch("jacobi round");
    }
    if (h[0] > 1e-20 * h[1]) throw Breakdown{"Jacobi eigensolver of the preconditioner did not converge"};
}

int projector_basis(cudaStream_t st, Mem &tmp, const double *Sh, const double *P, int n, unsigned long long seed,
                    double **U_out) {
    const long long nn = (long long)n * n;
    double *W = tmp.alloc<double>(nn), *Pi = tmp.alloc<double>(nn), *Pi2 = tmp.alloc<double>(nn);
    gemm<double>(st, false, false, n, n, n, 1.0, Sh, n, 0, P, n, 0, 0.0, W, n, 0, 1);
    gemm<double>(st, false, false, n, n, n, 1.0, W, n, 0, Sh, n, 0, 0.0, Pi, n, 0, 1);
    gemm<double>(st, false, false, n, n, n, 1.0, Pi, n, 0, Pi, n, 0, 0.0, Pi2, n, 0, 1);
    unsigned long long *dev = tmp.alloc<unsigned long long>(1);
    check(cudaMemsetAsync(dev, 0, sizeof(unsigned long long), st), "memset");
    roots::maxdiff_kernel<<<(int)std::min<long long>((nn + 255) / 256, 1216), 256, 0, st>>>(Pi2, Pi, nn, dev);
    check_launch("maxdiff");
    std::vector<double> diag((size_t)n);
    check(cudaMemcpy2DAsync(diag.data(), sizeof(double), Pi, (size_t)(n + 1) * sizeof(double), sizeof(double), n,
                            cudaMemcpyDeviceToHost, st),
          "D2H projector diagonal");
    unsigned long long hb = 0;
    check(cudaMemcpyAsync(&hb, dev, sizeof(hb), cudaMemcpyDeviceToHost, st), "D2H idempotency");
    check(cudaStreamSynchronize(st), "sync projector");
    double dev_max;
    std::memcpy(&dev_max, &hb, sizeof(dev_max));
    double tr = 0.0;
    for (double d : diag) tr += d;
    const int r = (int)std::lround(tr);
    if (!(dev_max < 1e-8) || r < 1 || r >= n || std::fabs(tr - r) > 1e-6) return 0;
    // seeded Gaussian Omega (splitmix64 + Box-Muller)
    std::vector<double> om((size_t)n * r);
    unsigned long long x = seed;
    auto next = [&]() {
        unsigned long long z = (x += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return (double)((z ^ (z >> 31)) >> 11) * (1.0 / 9007199254740992.0);
    };
    for (size_t i = 0; i < om.size(); i += 2) {
        const double u1 = std::max(next(), 1e-300), u2 = next();
        const double rad = std::sqrt(-2.0 * std::log(u1));
        om[i] = rad * std::cos(6.283185307179586 * u2);
        if (i + 1 < om.size()) om[i + 1] = rad * std::sin(6.283185307179586 * u2);
    }
    double *Om = tmp.alloc<double>((long long)n * r), *Y = tmp.alloc<double>((long long)n * r);
    double *G = tmp.alloc<double>((long long)r * r), *Gh = tmp.alloc<double>((long long)r * r);
    double *Gmh = tmp.alloc<double>((long long)r * r), *U = tmp.alloc<double>((long long)n * r);
    check(cudaMemcpyAsync(Om, om.data(), om.size() * sizeof(double), cudaMemcpyHostToDevice, st), "upload Omega");
    gemm<double>(st, false, false, n, r, n, 1.0, Pi, n, 0, Om, r, 0, 0.0, Y, r, 0, 1);          // Y = Pi Omega
    gemm<double>(st, true, false, r, r, n, 1.0, Y, r, 0, Y, r, 0, 0.0, G, r, 0, 1);             // G = Y^T Y
    std::vector<double> gh((size_t)r * r);
    check(cudaMemcpyAsync(gh.data(), G, gh.size() * sizeof(double), cudaMemcpyDeviceToHost, st), "D2H gram");
    check(cudaStreamSynchronize(st), "sync gram");
    overlap_roots(st, tmp, G, gh.data(), r, Gh, Gmh);
    gemm<double>(st, false, false, n, r, r, 1.0, Y, r, 0, Gmh, r, 0, 0.0, U, r, 0, 1);          // U = Y G^{-1/2}
    *U_out = U;
    return r;
}

// ---- tensor-core units of the grid kernels (the cuts are what the autotuner varies) -------------
// chunked point-major f16 tables of both sets for the density units; false unless every tile's
// phi list is whole aligned atom quads
bool build_density_chunks(tddft_ctx *c, Impl<float> &I) {
    if (I.units_ok) return true;
    const int ntl = I.chi.ntiles;
    const std::vector<int> &coff = I.coff_h, &poff = I.poff_h;
    std::vector<int> pids(poff[ntl]);
    if (!pids.empty())
        check(cudaMemcpy(pids.data(), I.phi.ids, pids.size() * sizeof(int), cudaMemcpyDeviceToHost), "D2H phi ids");
    for (int t = 0; t < ntl; ++t) {
        const int p0 = poff[t], np = poff[t + 1] - p0;
        if (np % 4) return false;
        for (int q = 0; q + 3 < np; q += 4)
            if (!(pids[p0 + q] % 4 == 0 && pids[p0 + q + 1] == pids[p0 + q] + 1 && pids[p0 + q + 2] == pids[p0 + q] + 2 &&
                  pids[p0 + q + 3] == pids[p0 + q] + 3))
                return false;
    }
    I.nchunks_chi = build_chunked_pm(c->st, I.mem, I.chi, coff, 64, &I.chi_pmc, I.cfirst_h);
    build_chunked_pm(c->st, I.mem, I.phi, poff, 32, &I.phi_pmc, I.pfirst_h);
    I.units_ok = true;
    return true;
}

// the density's units: chunks of at most cch chi (a multiple of 64, <= 320) and pch phi (a
// multiple of 32, <= 128) of each tile
void set_density_units(Impl<float> &I, int cch, int pch) {
    const int ntl = I.chi.ntiles;
    const std::vector<int> &coff = I.coff_h, &poff = I.poff_h;
    std::vector<DUnit> us;
    for (int t = 0; t < ntl; ++t) {
        const int nct = coff[t + 1] - coff[t], npt = poff[t + 1] - poff[t];
        if (nct == 0 || npt == 0) continue;
        for (int cc = 0; cc < nct; cc += cch)
            for (int pc = 0; pc < npt; pc += pch)
                us.push_back(DUnit{t, coff[t] + cc, std::min(cch, nct - cc), poff[t] + pc, std::min(pch, npt - pc),
                                   I.cfirst_h[t] + cc / 64, I.pfirst_h[t] + pc / 32, 0});
    }
    I.umem_dens.release();
    I.ndunits = (int)us.size();
    I.dunits = I.umem_dens.alloc<DUnit>(std::max<size_t>(1, us.size()));
    if (!us.empty())
        check(cudaMemcpy(I.dunits, us.data(), us.size() * sizeof(DUnit), cudaMemcpyHostToDevice), "upload density units");
    I.dens_cut[0] = cch;
    I.dens_cut[1] = pch;
}

// the integrals' units: chunks of at most cch chi (a multiple of 128, <= 384) and pch phi (a
// multiple of 16, <= 128), listed by class of 128-row chi blocks; false if they do not fit
bool set_integrals_units(Impl<float> &I, int cch, int pch) {
    const int ntl = I.chi.ntiles;
    const std::vector<int> &coff = I.coff_h, &poff = I.poff_h;
    std::vector<VTile> by[3];
    int maxnc = 0, maxnp = 0;
    for (int t = 0; t < ntl; ++t) {
        const int nct = coff[t + 1] - coff[t], npt = poff[t + 1] - poff[t];
        if (nct == 0 || npt == 0) continue;
        for (int cc = 0; cc < nct; cc += cch)
            for (int pc = 0; pc < npt; pc += pch) {
                const VTile u{t, coff[t] + cc, std::min(cch, nct - cc), poff[t] + pc, std::min(pch, npt - pc), 0};
                maxnc = std::max(maxnc, u.nc);
                maxnp = std::max(maxnp, u.np);
                by[(u.nc - 1) / 128].push_back(u);
            }
    }
    const int NPi = std::max(16, (maxnp + 15) / 16 * 16);
    if (integrals_tc_group(NPi, 1, maxnc) < 1) return false;
    std::vector<VTile> all;
    for (int q = 0; q < 3; ++q) {
        I.int_count[q] = (int)by[q].size();
        all.insert(all.end(), by[q].begin(), by[q].end());
    }
    I.umem_int.release();
    I.int_units = I.umem_int.alloc<VTile>(std::max<size_t>(1, all.size()));
    if (!all.empty())
        check(cudaMemcpy(I.int_units, all.data(), all.size() * sizeof(VTile), cudaMemcpyHostToDevice),
              "upload integrals units");
    I.maxc = maxnc;
    I.NPint = NPi;
    I.int_cut[0] = cch;
    I.int_cut[1] = pch;
    return true;
}

template <typename T>
void build_dense_matrices(tddft_ctx *c, Impl<T> *I, const tddft_system *s, Mem &tmpm);
template <typename T>
void build_sparse_matrices(tddft_ctx *c, Impl<T> *I);

// s: a dense system, or null with ss: a system of the truncated form
template <typename T>
void build_impl(tddft_ctx *c, const tddft_system *s, const tddft_sparse_system *ss = nullptr) {
    auto I = std::make_unique<Impl<T>>();
    const int n = c->n;
    cudaStream_t st = c->st;
    const tddft_funcs &chi_f = s ? s->chi : ss->chi, &phi_f = s ? s->phi : ss->phi;
    const double *n0_in = s ? s->n0 : ss->n0;
    const int fxc_kind = s ? s->fxc_kind : ss->fxc_kind;
    std::vector<int> cc_cnt, cv_cnt;
    build_tiles<T>(chi_f, n, c->nt, I->mem, I->chi, cc_cnt);
    build_tiles<T>(phi_f, n, c->nt, I->mem, I->phi, cv_cnt);
    if constexpr (sizeof(T) == 4) {
        // tensor-core grid path: point-major f16 chi copy, state-group shape
        const char *ng = std::getenv("TDDFT_NO_GRID_TC");
        if (tc_enabled() && !(ng && ng[0] == '1')) {
            const int ntl = I->chi.ntiles;
            std::vector<int> coff(ntl + 1), poff(ntl + 1);
            check(cudaMemcpy(coff.data(), I->chi.off, coff.size() * sizeof(int), cudaMemcpyDeviceToHost), "D2H off");
            check(cudaMemcpy(poff.data(), I->phi.off, poff.size() * sizeof(int), cudaMemcpyDeviceToHost), "D2H off");
            int maxc = 0, maxp = 0;
            for (int t = 0; t < ntl; ++t) {
                maxc = std::max(maxc, coff[t + 1] - coff[t]);
                maxp = std::max(maxp, poff[t + 1] - poff[t]);
            }
            const int CK = std::max(64, (maxc + 63) / 64 * 64);
            const int NP = std::max(16, (maxp + 15) / 16 * 16);
            // float32 tables on the host, fetched once for whichever tensor-core path needs them
            std::vector<float> cval, pv;
            auto fetch_tables = [&]() {
                if (cval.empty()) {
                    cval.resize((size_t)coff[ntl] * TILE_PTS);
                    check(cudaMemcpy(cval.data(), I->chi.val, cval.size() * sizeof(float), cudaMemcpyDeviceToHost),
                          "D2H chi tables");
                }
                if (pv.empty()) {
                    pv.resize((size_t)poff[ntl] * TILE_PTS);
                    check(cudaMemcpy(pv.data(), I->phi.val, pv.size() * sizeof(float), cudaMemcpyDeviceToHost),
                          "D2H phi tables");
                }
            };
            if (NP <= 256 && density_tc_group(CK / 64, NP, 1) >= 1) {
                fetch_tables();
                std::vector<unsigned short> pm((size_t)ntl * TILE_PTS * CK, 0);
                build_point_major_f16(coff.data(), cval.data(), nullptr, ntl, CK, pm.data());
                I->chi_pm = I->mem.template alloc<unsigned short>(pm.size());
                check(cudaMemcpy(I->chi_pm, pm.data(), pm.size() * sizeof(unsigned short), cudaMemcpyHostToDevice),
                      "upload point-major chi");
                I->CK = CK;
                {
                    std::vector<int> live;
                    for (int t = 0; t < ntl; ++t)
                        if (coff[t + 1] > coff[t] && poff[t + 1] > poff[t]) live.push_back(t);
                    I->nlive = (int)live.size();
                    I->live_tiles = I->mem.template alloc<int>(std::max<size_t>(1, live.size()));
                    if (!live.empty())
                        check(cudaMemcpy(I->live_tiles, live.data(), live.size() * sizeof(int), cudaMemcpyHostToDevice),
                              "upload live tiles");
                }
                // point-major f16 phi tables for the density epilogue
                if (NP % 32 == 0) {
                    std::vector<unsigned short> ppm((size_t)ntl * TILE_PTS * NP, 0);
                    build_point_major_f16(poff.data(), pv.data(), nullptr, ntl, NP, ppm.data());
                    I->phi_pm = I->mem.template alloc<unsigned short>(ppm.size());
                    check(cudaMemcpy(I->phi_pm, ppm.data(), ppm.size() * sizeof(unsigned short),
                                     cudaMemcpyHostToDevice),
                          "upload point-major phi");
                }
                I->NPmax = NP;
                I->grid_tc = true;
                {
                    // whole aligned phi quads in every tile (4 functions per atom, grouped by atom)
                    std::vector<int> pids(poff[ntl]);
                    check(cudaMemcpy(pids.data(), I->phi.ids, pids.size() * sizeof(int), cudaMemcpyDeviceToHost),
                          "D2H phi ids");
                    bool ok = c->nv % 4 == 0 && NP % 4 == 0;
                    for (int t = 0; t < ntl && ok; ++t) {
                        const int p0 = poff[t], np = poff[t + 1] - p0;
                        if (np % 4) ok = false;
                        for (int q = 0; q + 3 < np && ok; q += 4)
                            ok = pids[p0 + q] % 4 == 0 && pids[p0 + q + 1] == pids[p0 + q] + 1 &&
                                 pids[p0 + q + 2] == pids[p0 + q] + 2 && pids[p0 + q + 3] == pids[p0 + q] + 3;
                    }
                    const char *nq = std::getenv("TDDFT_NO_QUAD_GATHER");
                    I->phi_quads = ok && !(nq && nq[0] == '1');
                }
            }
            I->coff_h = coff;
            I->poff_h = poff;
            // dense tiles: the density in units of <= 320 chi and <= 128 phi of a tile, when every
            // tile's phi list is whole aligned atom quads (the P gather loads four phi at once);
            // TDDFT_DENSITY_UNITS=1 takes them even where the per-tile kernels fit
            {
                const char *nu = std::getenv("TDDFT_NO_DENSITY_UNITS");
                const char *fu = std::getenv("TDDFT_DENSITY_UNITS");
                const bool want = !I->grid_tc || (fu && fu[0] == '1');
                if (want && !(nu && nu[0] == '1') && c->nv % 4 == 0 && build_density_chunks(c, *I)) {
                    set_density_units(*I, 320, 128);
                    I->dens_units = true;
                }
            }
            // integrals: units of at most 384 chi and 128 phi slots of one tile (a denser tile is
            // cut into several). TDDFT_INTEGRALS_CHUNK="nc,np" cuts smaller units (multiples of
            // 128 and 16), for tests of the cut on small systems.
            {
                int cch = 384, pch = 128;
                if (const char *e = std::getenv("TDDFT_INTEGRALS_CHUNK")) {
                    int a = 0, b = 0;
                    if (std::sscanf(e, "%d,%d", &a, &b) == 2 && a >= 128 && a <= 384 && a % 128 == 0 && b >= 16 &&
                        b <= 128 && b % 16 == 0) {
                        cch = a;
                        pch = b;
                    }
                }
                if (set_integrals_units(*I, cch, pch)) {
                    // function-major f16 copies of both tables, rounded on the device (the f16 phi
                    // rows are the integrals' B operand, TMA-loaded and scaled by V in place)
                    const long long nch = (long long)coff[ntl] * TILE_PTS, nph = (long long)poff[ntl] * TILE_PTS;
                    I->chi_fm16 = I->mem.template alloc<unsigned short>(std::max<long long>(1, nch));
                    to_f16(st, reinterpret_cast<const float *>(I->chi.val), I->chi_fm16, nch);
                    I->nslots_chi = coff[ntl];
                    I->phi_fm16 = I->mem.template alloc<unsigned short>(std::max<long long>(1, nph));
                    to_f16(st, reinterpret_cast<const float *>(I->phi.val), I->phi_fm16, nph);
                    I->nslots_phi = poff[ntl];
                    I->integrals_tc = true;
                }
            }
        }
    }
    double pp = 0.0, tv = 0.0;
    for (size_t i = 0; i < cc_cnt.size(); ++i) {
        pp += (double)cc_cnt[i] * cv_cnt[i];
        tv += cc_cnt[i] + cv_cnt[i];
    }
    c->pair_points = pp;
    c->table_values = tv;
    Mem tmpm;
    auto up64 = [&](const double *h, long long cnt) {
        double *d = tmpm.alloc<double>(cnt);
        check(cudaMemcpyAsync(d, h, cnt * sizeof(double), cudaMemcpyHostToDevice, st), "upload matrix");
        return d;
    };
    auto keep = [&](const double *d, long long cnt) {
        T *o = I->mem.template alloc<T>(cnt);
        convert<double, T>(st, d, o, cnt);
        return o;
    };
    if (s) build_dense_matrices<T>(c, I.get(), s, tmpm);
    else build_sparse_matrices<T>(c, I.get());
    // f_xc[n0], float64, once per system
    const long long n3 = c->n3();
    I->fxc64 = I->mem.template alloc<double>(n3);
    if (fxc_kind == TDDFT_FXC_LDA_PW92) {
        double *n0 = up64(n0_in, n3);
        fxc_lda(st, n0, I->fxc64, n3);
        I->fxc = keep(I->fxc64, n3);
    } else {
        check(cudaMemsetAsync(I->fxc64, 0, n3 * sizeof(double), st), "memset fxc");
        I->fxc = nullptr;
    }
    check(ctx_sync(c), "build sync");
    if constexpr (sizeof(T) == 8) c->d64 = std::move(I);
    else c->d32 = std::move(I);
}

// the cluster-block constants of the truncated form in T (and the phi ones transposed for the
// tensor-core right products), and the kernel-pattern mask
template <typename T>
void build_sparse_matrices(tddft_ctx *c, Impl<T> *I) {
    const SparseLayout &L = *c->sp;
    cudaStream_t st = c->st;
    const bool tc = sparse_tc(c);
    for (int x = 0; x < SP_NCONST; ++x) {
        const long long nc_ = L.cc_len(x), nv_ = L.vv_len(x);
        I->cc[x] = I->mem.template alloc<T>(std::max<long long>(1, nc_));
        convert<double, T>(st, L.cc64[x], I->cc[x], nc_);
        I->vv[x] = I->mem.template alloc<T>(std::max<long long>(1, nv_));
        convert<double, T>(st, L.vv64[x], I->vv[x], nv_);
        if (tc) {
            I->vvT[x] = I->mem.template alloc<T>(std::max<long long>(1, nv_));
            bsr_transpose<T>(st, I->vv[x], I->vvT[x], CB_C, CB_C, L.pvv[x].nnzb(), 1);
        }
    }
    I->mask = I->mem.template alloc<T>(std::max<long long>(1, L.len()));
    cb_mask<T>(st, L, I->mask);
}

// the dense constants: products, overlap roots and the preconditioner's bases (float64 on the
// device, kept in T), and the kernel-pattern mask
template <typename T>
void build_dense_matrices(tddft_ctx *c, Impl<T> *I, const tddft_system *s, Mem &tmpm) {
    const int nc = c->nc, nv = c->nv;
    cudaStream_t st = c->st;
    auto up64 = [&](const double *h, long long cnt) {
        double *d = tmpm.alloc<double>(cnt);
        check(cudaMemcpyAsync(d, h, cnt * sizeof(double), cudaMemcpyHostToDevice, st), "upload matrix");
        return d;
    };
    const long long cc = (long long)nc * nc, vv = (long long)nv * nv;
    double *Sc = up64(s->S_chi, cc), *Sv = up64(s->S_phi, vv), *Hc = up64(s->H_chi, cc);
    double *Hv = up64(s->H_phi, vv), *Pc = up64(s->P_c, cc), *Pv = up64(s->P_v, vv);
    double *Mc = tmpm.alloc<double>(cc), *Rc = tmpm.alloc<double>(cc), *Ac = tmpm.alloc<double>(cc);
    double *Mv = tmpm.alloc<double>(vv), *Rv = tmpm.alloc<double>(vv), *Av = tmpm.alloc<double>(vv);
    gemm<double>(st, false, false, nc, nc, nc, 1.0, Pc, nc, 0, Hc, nc, 0, 0.0, Mc, nc, 0, 1);   // P^c H^chi
    gemm<double>(st, false, false, nv, nv, nv, 1.0, Hv, nv, 0, Pv, nv, 0, 0.0, Mv, nv, 0, 1);   // H^phi P^v
    gemm<double>(st, false, false, nc, nc, nc, 1.0, Pc, nc, 0, Sc, nc, 0, 0.0, Rc, nc, 0, 1);   // P^c S^chi
    gemm<double>(st, false, false, nv, nv, nv, 1.0, Sv, nv, 0, Pv, nv, 0, 0.0, Rv, nv, 0, 1);   // S^phi P^v
    gemm<double>(st, false, false, nc, nc, nc, 1.0, Sc, nc, 0, Rc, nc, 0, 0.0, Ac, nc, 0, 1);   // S P^c S
    gemm<double>(st, false, false, nv, nv, nv, 1.0, Rv, nv, 0, Sv, nv, 0, 0.0, Av, nv, 0, 1);   // S P^v S
    // Loewdin variables of the preconditioner's CG: G~ = Sc^{1/2} G Sv^{1/2} turns the trace metric
    // into the Frobenius product and the operator into M~c G~ - G~ M~v
    double *Sch = tmpm.alloc<double>(cc), *Scmh = tmpm.alloc<double>(cc), *Svh = tmpm.alloc<double>(vv),
           *Svmh = tmpm.alloc<double>(vv), *Mct = tmpm.alloc<double>(cc), *Mvt = tmpm.alloc<double>(vv),
           *W = tmpm.alloc<double>(std::max(cc, vv));
    overlap_roots(st, tmpm, Sc, s->S_chi, nc, Sch, Scmh);
    overlap_roots(st, tmpm, Sv, s->S_phi, nv, Svh, Svmh);
    gemm<double>(st, false, false, nc, nc, nc, 1.0, Sch, nc, 0, Mc, nc, 0, 0.0, W, nc, 0, 1);
    gemm<double>(st, false, false, nc, nc, nc, 1.0, W, nc, 0, Scmh, nc, 0, 0.0, Mct, nc, 0, 1);  // Sc^1/2 Mc Sc^-1/2
    gemm<double>(st, false, false, nv, nv, nv, 1.0, Svmh, nv, 0, Mv, nv, 0, 0.0, W, nv, 0, 1);
    gemm<double>(st, false, false, nv, nv, nv, 1.0, W, nv, 0, Svh, nv, 0, 0.0, Mvt, nv, 0, 1);   // Sv^-1/2 Mv Sv^1/2
    // conduction x valence subspace of the preconditioner's solutions (exact when P^c, P^v are
    // projectors): the CG iterates stay in it, so it runs there on rc x rv matrices
    double *Uc = nullptr, *Uv = nullptr;
    int rc = projector_basis(st, tmpm, Sch, Pc, nc, 0x5eed0001ull, &Uc);
    int rv = rc ? projector_basis(st, tmpm, Svh, Pv, nv, 0x5eed0002ull, &Uv) : 0;
    if (!rv) rc = 0;
    double *Wc = nullptr, *Wv = nullptr, *Vc = nullptr, *Vv = nullptr, *Mch = nullptr, *Mvh = nullptr;
    if (rc) {
        const long long crc = (long long)nc * rc, vrv = (long long)nv * rv;
        Wc = tmpm.alloc<double>(crc); Wv = tmpm.alloc<double>(vrv); Vc = tmpm.alloc<double>(crc);
        Vv = tmpm.alloc<double>(vrv); Mch = tmpm.alloc<double>((long long)rc * rc); Mvh = tmpm.alloc<double>((long long)rv * rv);
        double *T1 = tmpm.alloc<double>(std::max(crc, vrv));
        gemm<double>(st, true, false, rc, nc, nc, 1.0, Uc, rc, 0, Sch, nc, 0, 0.0, Wc, nc, 0, 1);   // U_c^T Sc^1/2
        gemm<double>(st, false, false, nv, rv, nv, 1.0, Svh, nv, 0, Uv, rv, 0, 0.0, Wv, rv, 0, 1);  // Sv^1/2 U_v
        gemm<double>(st, false, false, nc, rc, nc, 1.0, Scmh, nc, 0, Uc, rc, 0, 0.0, Vc, rc, 0, 1); // Sc^-1/2 U_c
        gemm<double>(st, true, false, rv, nv, nv, 1.0, Uv, rv, 0, Svmh, nv, 0, 0.0, Vv, nv, 0, 1);  // U_v^T Sv^-1/2
        gemm<double>(st, false, false, nc, rc, nc, 1.0, Mct, nc, 0, Uc, rc, 0, 0.0, T1, rc, 0, 1);
        gemm<double>(st, true, false, rc, rc, nc, 1.0, Uc, rc, 0, T1, rc, 0, 0.0, Mch, rc, 0, 1);  // U_c^T M~c U_c
        gemm<double>(st, false, false, nv, rv, nv, 1.0, Mvt, nv, 0, Uv, rv, 0, 0.0, T1, rv, 0, 1);
        gemm<double>(st, true, false, rv, rv, nv, 1.0, Uv, rv, 0, T1, rv, 0, 0.0, Mvh, rv, 0, 1);  // U_v^T M~v U_v
    }
    double *Dn = nullptr;
    if (c->opt.precond == TDDFT_PRECOND_EXACT) {
        // Mch and Mvh are symmetric on the subspace (U^T H~ U of the Loewdin Hamiltonians), so
        // Eq. precond becomes diagonal in their eigenbases: Mch = Ec Lc Ec^T, Mvh = Ev Lv Ev^T
        if (!rc) throw InvalidArg{"the exact preconditioner needs idempotent P^c and P^v"};
        const long long cc2 = (long long)rc * rc, vv2 = (long long)rv * rv;
        double *Ac = tmpm.alloc<double>(cc2), *Av = tmpm.alloc<double>(vv2);
        double *Ec = tmpm.alloc<double>(cc2), *Ev = tmpm.alloc<double>(vv2);
        check(cudaMemcpyAsync(Ac, Mch, cc2 * sizeof(double), cudaMemcpyDeviceToDevice, st), "copy Mch");
        check(cudaMemcpyAsync(Av, Mvh, vv2 * sizeof(double), cudaMemcpyDeviceToDevice, st), "copy Mvh");
        sym_eig(st, tmpm, Ac, rc, Ec);
        sym_eig(st, tmpm, Av, rv, Ev);
        Dn = tmpm.alloc<double>((long long)rc * rv);
        roots::denominators_kernel<<<(int)std::min<long long>(((long long)rc * rv + 255) / 256, 1216), 256, 0, st>>>(
            Ac, rc, Av, rv, Dn);
        check_launch("denominators");
        const long long crc = (long long)nc * rc, vrv = (long long)nv * rv;
        double *W2 = tmpm.alloc<double>(crc), *V2 = tmpm.alloc<double>(crc);
        double *W3 = tmpm.alloc<double>(vrv), *V3 = tmpm.alloc<double>(vrv);
        gemm<double>(st, true, false, rc, nc, rc, 1.0, Ec, rc, 0, Wc, nc, 0, 0.0, W2, nc, 0, 1);   // Ec^T Wc
        gemm<double>(st, false, false, nv, rv, rv, 1.0, Wv, rv, 0, Ev, rv, 0, 0.0, W3, rv, 0, 1);  // Wv Ev
        gemm<double>(st, false, false, nc, rc, rc, 1.0, Vc, rc, 0, Ec, rc, 0, 0.0, V2, rc, 0, 1);  // Vc Ec
        gemm<double>(st, true, false, rv, nv, rv, 1.0, Ev, rv, 0, Vv, nv, 0, 0.0, V3, nv, 0, 1);   // Ev^T Vv
        Wc = W2;
        Wv = W3;
        Vc = V2;
        Vv = V3;
    }
    auto keep = [&](const double *d, long long cnt) {
        T *o = I->mem.template alloc<T>(cnt);
        convert<double, T>(st, d, o, cnt);
        return o;
    };
    I->Sc = keep(Sc, cc); I->Sv = keep(Sv, vv); I->Pc = keep(Pc, cc); I->Pv = keep(Pv, vv);
    I->Mc = keep(Mc, cc); I->Mv = keep(Mv, vv); I->Rc = keep(Rc, cc); I->Rv = keep(Rv, vv);
    I->Ac = keep(Ac, cc); I->Av = keep(Av, vv);
    I->Sch = keep(Sch, cc); I->Scmh = keep(Scmh, cc); I->Svh = keep(Svh, vv); I->Svmh = keep(Svmh, vv);
    I->Mct = keep(Mct, cc); I->Mvt = keep(Mvt, vv);
    const char *nr = std::getenv("TDDFT_NO_REDUCED_PRECOND");
    if (Dn) {
        I->exact = true;
        I->Dn = keep(Dn, (long long)rc * rv);
    }
    if (rc && (Dn || !(nr && nr[0] == '1'))) {
        I->rc = rc;
        I->rv = rv;
        I->Wc = keep(Wc, (long long)rc * nc); I->Wv = keep(Wv, (long long)nv * rv);
        I->Vc = keep(Vc, (long long)nc * rc); I->Vv = keep(Vv, (long long)rv * nv);
        I->Mch = keep(Mch, (long long)rc * rc); I->Mvh = keep(Mvh, (long long)rv * rv);
    }
    register_constants(*I);
    // kernel pattern mask over (chi, phi) function pairs
    std::vector<double> m((size_t)nc * nv);
    for (int a = 0; a < nc; ++a)
        for (int b = 0; b < nv; ++b)
            m[(size_t)a * nv + b] = c->amask[(size_t)s->chi.atom[a] * c->natoms + s->phi.atom[b]] ? 1.0 : 0.0;
    double *dm = up64(m.data(), (long long)nc * nv);
    I->mask = keep(dm, (long long)nc * nv);
    check(ctx_sync(c), "build sync");
}

}  // namespace

// ================================================================================================
// state of the PCG solver

namespace {

template <typename T>
struct StateBufs {
    Mem mem;
    T *Y, *P, *f, *g, *G1, *h, *z, *Z, *dir, *D, *fD, *covP, *covD;
    T *pdir, *pD, *pz, *pZ, *tmp;
    T *cr, *cp, *cLp, *cLpp, *cpv, *cLv;   // inner CG
    T *qr = nullptr, *qp = nullptr, *qL = nullptr, *qz = nullptr;   // inner CG on the reduced space
    double *A, *BDf, *CDfD, *PP, *PD, *DP, *DD, *Q, *coef, *Cp, *Cq, *lam, *sc, *flip;
    double *dvec, *dvec2, *dvec3, *evout;
    double *cg_pLp, *cg_rr, *cg_rrn, *cg_r0, *cg_alpha, *cg_beta, *gscr;
    int *status, *cg_active, *cg_nactive;
};

}  // namespace

struct tddft_state {
    tddft_ctx *ctx = nullptr;
    int k = 0;
    int it = 0;
    int fallbacks = 0;             // learned steps that took the CG solve instead
    long long inner_iters = 0;     // inner CG iterations over all steps
    bool evaluated = false;
    bool have_prev_omega = false;
    std::vector<double> omega, resid, omega_prev;
    std::unique_ptr<StateBufs<double>> s64;
    std::unique_ptr<StateBufs<float>> s32;
    double *host = nullptr;   // pinned, 4k + 16 doubles: [omega k][resid k][status, n_active][lam]
                              // (tddft_subspace uses [omega k][pairing 2k])
    ~tddft_state() {
        if (host) cudaFreeHost(host);
    }
};

namespace {

template <typename T> StateBufs<T> &bufs(tddft_state *s);
template <> StateBufs<double> &bufs<double>(tddft_state *s) { return *s->s64; }
template <> StateBufs<float> &bufs<float>(tddft_state *s) { return *s->s32; }

template <typename T>
void alloc_state(tddft_ctx *c, tddft_state *S) {
    auto B = std::make_unique<StateBufs<T>>();
    const size_t n2 = (size_t)2 * S->k * c->len();
    T **mats[] = {&B->Y, &B->P, &B->f, &B->g, &B->G1, &B->h, &B->z, &B->Z, &B->dir, &B->D,
                  &B->fD, &B->covP, &B->covD, &B->pdir, &B->pD, &B->pz, &B->pZ, &B->tmp,
                  &B->cr, &B->cp, &B->cLp, &B->cLpp, &B->cpv, &B->cLv};
    for (T **m : mats) *m = B->mem.template alloc<T>(n2);
    const size_t k2 = 2 * S->k, kk4 = k2 * k2, kk = (size_t)S->k * S->k;
    double **sm[] = {&B->A, &B->BDf, &B->CDfD, &B->PP, &B->PD, &B->DP, &B->DD, &B->coef};
    for (double **m : sm) *m = B->mem.template alloc<double>(kk4);
    B->Q = B->mem.template alloc<double>(kk);
    B->Cp = B->mem.template alloc<double>(kk);
    B->Cq = B->mem.template alloc<double>(kk);
    B->lam = B->mem.template alloc<double>(1);
    B->sc = B->mem.template alloc<double>(4);
    B->flip = B->mem.template alloc<double>(1);
    double **vv[] = {&B->dvec, &B->dvec2, &B->dvec3, &B->evout, &B->cg_pLp, &B->cg_rr, &B->cg_rrn,
                     &B->cg_r0, &B->cg_alpha, &B->cg_beta};
    for (double **m : vv) *m = B->mem.template alloc<double>(k2);
    B->gscr = B->mem.template alloc<double>((size_t)gram_scratch_doubles(64, 32));
    {
        Impl<T> &I = impl<T>(c);
        if (I.rc) {
            const size_t nq = (size_t)2 * S->k * I.rc * I.rv;
            B->qr = B->mem.template alloc<T>(nq);
            B->qp = B->mem.template alloc<T>(nq);
            B->qL = B->mem.template alloc<T>(nq);
            B->qz = B->mem.template alloc<T>(nq);
        }
    }
    B->status = B->mem.template alloc<int>(1);
    B->cg_active = B->mem.template alloc<int>(k2);
    B->cg_nactive = B->mem.template alloc<int>(1);
    check(cudaMemsetAsync(B->sc, 0, 4 * sizeof(double), c->st), "memset sc");
    check(cudaMemsetAsync(B->flip, 0, sizeof(double), c->st), "memset flip");
    check(cudaMemsetAsync(B->status, 0, sizeof(int), c->st), "memset status");
    check(cudaMemsetAsync(B->pdir, 0, n2 * sizeof(T), c->st), "memset pdir");
    check(cudaMemsetAsync(B->pD, 0, n2 * sizeof(T), c->st), "memset pD");
    check(cudaMemsetAsync(B->pz, 0, n2 * sizeof(T), c->st), "memset pz");
    check(cudaMemsetAsync(B->pZ, 0, n2 * sizeof(T), c->st), "memset pZ");
    if constexpr (sizeof(T) == 8) S->s64 = std::move(B);
    else S->s32 = std::move(B);
}

// cov(X) = S^chi X S^phi for 2k matrices
template <typename T>
void covariant(tddft_ctx *c, Impl<T> &I, int nb, const T *X, T *out, T *tmp) {
    lprod<T>(c, I, SP_S, X, tmp, nb, T(1), T(0));
    rprod<T>(c, I, tmp, SP_S, out, nb, T(1), T(0));
}

// out = C_x X D_x for nb matrices (x = SP_R: Eq. auxiliary; SP_A: the L-gradient; SP_P: P^c G P^v)
template <typename T>
void sandwich_x(tddft_ctx *c, Impl<T> &I, int nb, int x, const T *X, T *out, T *tmp, bool approx = false) {
    lprod<T>(c, I, x, X, tmp, nb, T(1), T(0), approx);
    rprod<T>(c, I, tmp, x, out, nb, T(1), T(0), approx);
}

// out = L X R (left nc x nc, right nv x nv dense matrices) for nb matrices
template <typename T>
void sandwich(tddft_ctx *c, int nb, const T *Lm, const T *X, const T *Rm, T *out, T *tmp, bool approx = false) {
    const int nc = c->nc, nv = c->nv;
    const long long len = c->len();
    gemm<T>(c->st, false, false, nc, nv, nc, T(1), Lm, nc, 0, X, nv, len, T(0), tmp, nv, len, nb, approx);
    gemm<T>(c->st, false, false, nb * nc, nv, nv, T(1), tmp, nv, 0, Rm, nv, 0, T(0), out, nv, 0, 1, approx);
}

void sync_status(tddft_ctx *c, tddft_state *S, const int *dstatus) {
    check(cudaMemcpyAsync(reinterpret_cast<int *>(S->host + 2 * S->k), dstatus, sizeof(int),
                          cudaMemcpyDeviceToHost, c->st),
          "D2H status");
    check_tc_error(c);   // waits for the status copy too
    const int stv = *reinterpret_cast<int *>(S->host + 2 * S->k);
    if (stv == DEV_BREAKDOWN) throw Breakdown{"non-positive norm in Gram-Schmidt (dependent trial pairs)"};
    if (stv == DEV_NAN) throw Breakdown{"NaN or Inf in the trial pairs"};
    if (stv == DEV_NAN_EVAL) throw Breakdown{"NaN or Inf in Q or the residuals of the trial pairs"};
    if (stv == DEV_NAN_LINE) throw Breakdown{"NaN or Inf in the line-search traces (directions or f of them)"};
    if (stv == DEV_NAN_INIT) throw Breakdown{"NaN or Inf in the starting trial pairs"};
}

// recombine Y, P, f and cov(P) with the Gram-Schmidt coefficients (sign flips folded into Cq);
// cov is linear, so cov(P) follows the same combinations as P
template <typename T>
void recombine(tddft_ctx *c, StateBufs<T> &B, int k) {
    const long long len = c->len();
    T *arrs[] = {B.Y, B.P, B.f, B.covP};
    for (T *X : arrs) {
        check(cudaMemcpyAsync(B.tmp, X, 2 * k * len * sizeof(T), cudaMemcpyDeviceToDevice, c->st), "copy recombine");
        combine<T>(c->st, B.Cp, k, k, k, B.tmp, len, X, len, len, false);
        combine<T>(c->st, B.Cq, k, k, k, B.tmp + k * len, len, X + k * len, len, len, false);
    }
}

template <typename T>
void state_init(tddft_ctx *c, tddft_state *S, const double *Y0) {
    Impl<T> &I = impl<T>(c);
    StateBufs<T> &B = bufs<T>(S);
    const int k = S->k;
    const long long len = c->len();
    ensure_workspace(c, I, 2 * k);
    // Y = mask * Y0 for both p and q (X random, Y = 0 => p = q)
    abi_in<T>(c, I, Y0, B.Y, k);
    if (c->trunc) mask_mul<T>(c->st, B.Y, I.mask, len, k);
    check(cudaMemcpyAsync(B.Y + k * len, B.Y, k * len * sizeof(T), cudaMemcpyDeviceToDevice, c->st), "copy Y");
    // P = P^c S^chi L S^phi P^v (Eq. auxiliary)
    sandwich_x<T>(c, I, 2 * k, SP_R, B.Y, B.P, B.tmp);
    covariant<T>(c, I, 2 * k, B.P, B.covP, B.tmp);
    gram<T>(c->st, B.covP, len, 2 * k, B.P, len, 2 * k, len, B.PP, B.gscr);
    init_gs(c->st, k, B.PP, B.Cp, B.Cq, B.status);
    sync_status(c, S, B.status);
    check(cudaMemsetAsync(B.f, 0, 2 * k * len * sizeof(T), c->st), "memset f");
    recombine<T>(c, B, k);
    apply_impl<T>(c, I, k, B.P, B.f, true);
    check(ctx_sync(c), "sync init");
}

// Q, omega, gradient and residuals of the current iterate
template <typename T>
void evaluate(tddft_ctx *c, tddft_state *S) {
    Impl<T> &I = impl<T>(c);
    StateBufs<T> &B = bufs<T>(S);
    const int k = S->k;
    const long long len = c->len();
    cudaStream_t st = c->st;
    // cov(P) is carried along with P (state creation, line step, recombination, re-application)
    gram<T>(st, B.covP, len, 2 * k, B.f, len, 2 * k, len, B.A, B.gscr);   // A[x][y] = <P_x, f_y>
    make_q(st, k, B.A, B.Q, B.coef);
    // g = f - swap(P) Q^T
    check(cudaMemcpyAsync(B.g, B.f, 2 * k * len * sizeof(T), cudaMemcpyDeviceToDevice, st), "copy g");
    combine<T>(st, B.coef, 2 * k, 2 * k, 2 * k, B.P, len, B.g, len, len, true);
    if (c->sparse) {
        // truncated form: G_L is the exact gradient of the sum functional with respect to L
        // through the truncated map P = T(T(R_c L) R_v): its adjoint applied to the Frobenius
        // gradient cov(g), G_L = T(R_c^T T(cov(g) R_v^T)); residual = Frobenius norm
        covariant<T>(c, I, 2 * k, B.g, B.G1, B.tmp);
        rprod<T>(c, I, B.G1, SP_T, B.tmp, 2 * k, T(1), T(0));
        lprod<T>(c, I, SP_T, B.tmp, B.G1, 2 * k, T(1), T(0));
        dots<T>(st, B.G1, len, B.G1, len, 2 * k, len, B.dvec, B.gscr);
    } else if (c->trunc) {
        // G_L = mask * (S P^c S) g (S P^v S) (the exact L-gradient when only L is truncated);
        // residual = Frobenius norm. With the exact preconditioner G_L only steers the search
        // (its error changes the direction and the residual's last digits, not the fixed point,
        // where g = 0): one TF32 MMA per product
        sandwich_x<T>(c, I, 2 * k, SP_A, B.g, B.G1, B.tmp, I.exact);
        mask_mul<T>(st, B.G1, I.mask, len, 2 * k);
        dots<T>(st, B.G1, len, B.G1, len, 2 * k, len, B.dvec, B.gscr);
    } else {
        covariant<T>(c, I, 2 * k, B.g, B.G1, B.tmp);   // cov(g)
        dots<T>(st, B.g, len, B.G1, len, 2 * k, len, B.dvec, B.gscr);
    }
    eval_finish(st, k, B.Q, B.dvec, B.evout, B.status);
    check(cudaMemcpyAsync(S->host, B.evout, 2 * k * sizeof(double), cudaMemcpyDeviceToHost, st), "D2H eval");
    sync_status(c, S, B.status);
    S->omega.assign(S->host, S->host + k);
    S->resid.assign(S->host + k, S->host + 2 * k);
    S->evaluated = true;
}

// z = Pinv(h): CG on P^c H^chi G - G H^phi P^v = h (Eq. precond) in the trace metric, for the 2k
// systems at once. Systems stop individually (relative residual precond_tol, non-positive
// curvature); the loop ends when none is active or after precond_maxit iterations.
template <typename T>
void precondition(tddft_ctx *c, tddft_state *S, const T *h, T *z) {
    Impl<T> &I = impl<T>(c);
    StateBufs<T> &B = bufs<T>(S);
    const int k2 = 2 * S->k, nc = c->nc, nv = c->nv;
    const long long len = c->len(), tot = k2 * len;
    cudaStream_t st = c->st;
    if (c->opt.precond == TDDFT_PRECOND_NONE) {
        check(cudaMemcpyAsync(z, h, tot * sizeof(T), cudaMemcpyDeviceToDevice, st), "copy z");
        return;
    }
    // CG in Loewdin variables X~ = Sc^{1/2} X Sv^{1/2}: the trace metric of Eq. precond's CG becomes
    // the Frobenius product and L becomes M~c X~ - X~ M~v, so an iteration takes two products
    // instead of four; the iterates are those of the CG in the original variables
    // inner tolerance: fixed, or loose early and tight at the end (adaptive)
    double ptol = c->opt.precond_tol;
    if (c->opt.precond_adaptive && !S->resid.empty()) {
        const double rmax = *std::max_element(S->resid.begin(), S->resid.end());
        ptol = std::min(0.1, std::max(c->opt.precond_tol, rmax));
    }
    if (c->sparse) {
        // truncated form: CG in the original variables on T(M_c G) - T(G M_v) = h with the metric
        // <X, Y> = sum cov(X) * Y, from G = 0 (every product block-sparse, cut to the pattern)
        T *r = B.cr, *p = B.cp, *Lp = B.cLp, *cv = B.cLpp;
        check(cudaMemsetAsync(z, 0, tot * sizeof(T), st), "memset z");
        check(cudaMemcpyAsync(r, h, tot * sizeof(T), cudaMemcpyDeviceToDevice, st), "copy r");
        check(cudaMemcpyAsync(p, h, tot * sizeof(T), cudaMemcpyDeviceToDevice, st), "copy p");
        covariant<T>(c, I, k2, r, cv, B.tmp);
        dots<T>(st, cv, len, r, len, k2, len, B.dvec2, B.gscr);
        cg_init(st, k2, ptol, B.dvec2, B.cg_rr, B.cg_r0, B.cg_active, B.cg_nactive);
        int *hn = reinterpret_cast<int *>(S->host + 2 * S->k) + 1;
        for (int it = 0; it < c->opt.precond_maxit; ++it) {
            check(cudaMemcpyAsync(hn, B.cg_nactive, sizeof(int), cudaMemcpyDeviceToHost, st), "D2H n_active");
            check(ctx_sync(c), "sync cg");
            if (*hn == 0) break;
            S->inner_iters += 1;
            lprod<T>(c, I, SP_M, p, Lp, k2, T(1), T(0));
            rprod<T>(c, I, p, SP_M, Lp, k2, T(-1), T(1));
            covariant<T>(c, I, k2, p, cv, B.tmp);
            dots<T>(st, cv, len, Lp, len, k2, len, B.cg_pLp, B.gscr);
            cg_scalars(st, k2, 0, ptol, B.cg_pLp, B.cg_rrn, B.cg_rr, B.cg_r0, B.cg_alpha, B.cg_beta, B.cg_active,
                       B.cg_nactive);
            axpy_dev<T>(st, B.cg_alpha, 1, 1.0, z, p, len, k2);
            axpy_dev<T>(st, B.cg_alpha, 1, -1.0, r, Lp, len, k2);
            covariant<T>(c, I, k2, r, cv, B.tmp);
            dots<T>(st, cv, len, r, len, k2, len, B.cg_rrn, B.gscr);
            cg_scalars(st, k2, 1, ptol, B.cg_pLp, B.cg_rrn, B.cg_rr, B.cg_r0, B.cg_alpha, B.cg_beta, B.cg_active,
                       B.cg_nactive);
            cg_dir<T>(st, p, r, B.cg_beta, len, k2);
        }
        return;
    }
    if (I.exact) {
        // Eq. precond solved exactly: coordinates in the eigenbases of Mch and Mvh, divided by
        // lambda_c,i - lambda_v,j, and back: z = (Vc Ec) [(Ec^T Wc h Wv Ev) / (Lc - Lv)] (Ev^T Vv)
        const int rc = I.rc, rv = I.rv;
        const long long lr = (long long)rc * rv;
        // (a preconditioner's errors change the search direction, not the fixed point: one TF32
        // MMA per product)
        gemm<T>(st, false, false, rc, nv, nc, T(1), I.Wc, nc, 0, h, nv, len, T(0), B.tmp, nv, (long long)rc * nv, k2,
                true);
        gemm<T>(st, false, false, k2 * rc, rv, nv, T(1), B.tmp, nv, 0, I.Wv, rv, 0, T(0), B.qr, rv, 0, 1, true);
        mask_mul<T>(st, B.qr, I.Dn, lr, k2);
        gemm<T>(st, false, false, nc, rv, rc, T(1), I.Vc, rc, 0, B.qr, rv, lr, T(0), B.tmp, rv, (long long)nc * rv, k2,
                true);
        gemm<T>(st, false, false, k2 * nc, nv, rv, T(1), B.tmp, rv, 0, I.Vv, nv, 0, T(0), z, nv, 0, 1, true);
        return;
    }
    if (I.rc) {
        // the same CG on the rc x rv coordinates of the conduction x valence subspace:
        // r^ = U_c^T h~ U_v, z = Sc^{-1/2} U_c z^ U_v^T Sv^{-1/2}
        const int rc = I.rc, rv = I.rv;
        const long long lr = (long long)rc * rv;
        T *r = B.qr, *p = B.qp, *Lp = B.qL, *zh = B.qz;
        gemm<T>(st, false, false, rc, nv, nc, T(1), I.Wc, nc, 0, h, nv, len, T(0), B.tmp, nv, (long long)rc * nv, k2);
        gemm<T>(st, false, false, k2 * rc, rv, nv, T(1), B.tmp, nv, 0, I.Wv, rv, 0, T(0), r, rv, 0, 1);
        check(cudaMemsetAsync(zh, 0, k2 * lr * sizeof(T), st), "memset z");
        check(cudaMemcpyAsync(p, r, k2 * lr * sizeof(T), cudaMemcpyDeviceToDevice, st), "copy p");
        dots<T>(st, r, lr, r, lr, k2, lr, B.dvec2, B.gscr);
        cg_init(st, k2, ptol, B.dvec2, B.cg_rr, B.cg_r0, B.cg_active, B.cg_nactive);
        int *hn = reinterpret_cast<int *>(S->host + 2 * S->k) + 1;
        for (int it = 0; it < c->opt.precond_maxit; ++it) {
            check(cudaMemcpyAsync(hn, B.cg_nactive, sizeof(int), cudaMemcpyDeviceToHost, st), "D2H n_active");
            check(ctx_sync(c), "sync cg");
            if (*hn == 0) break;
            S->inner_iters += 1;
            gemm<T>(st, false, false, rc, rv, rc, T(1), I.Mch, rc, 0, p, rv, lr, T(0), Lp, rv, lr, k2);
            gemm<T>(st, false, false, k2 * rc, rv, rv, T(-1), p, rv, 0, I.Mvh, rv, 0, T(1), Lp, rv, 0, 1);
            dots<T>(st, p, lr, Lp, lr, k2, lr, B.cg_pLp, B.gscr);
            cg_scalars(st, k2, 0, ptol, B.cg_pLp, B.cg_rrn, B.cg_rr, B.cg_r0, B.cg_alpha, B.cg_beta, B.cg_active,
                       B.cg_nactive);
            axpy_dev<T>(st, B.cg_alpha, 1, 1.0, zh, p, lr, k2);
            axpy_dev<T>(st, B.cg_alpha, 1, -1.0, r, Lp, lr, k2);
            dots<T>(st, r, lr, r, lr, k2, lr, B.cg_rrn, B.gscr);
            cg_scalars(st, k2, 1, ptol, B.cg_pLp, B.cg_rrn, B.cg_rr, B.cg_r0, B.cg_alpha, B.cg_beta, B.cg_active,
                       B.cg_nactive);
            cg_dir<T>(st, p, r, B.cg_beta, lr, k2);
        }
        gemm<T>(st, false, false, nc, rv, rc, T(1), I.Vc, rc, 0, zh, rv, lr, T(0), B.tmp, rv, (long long)nc * rv, k2);
        gemm<T>(st, false, false, k2 * nc, nv, rv, T(1), B.tmp, rv, 0, I.Vv, nv, 0, T(0), z, nv, 0, 1);
        return;
    }
    T *r = B.cLpp, *zt = B.cr, *p = B.cp, *Lp = B.cLp;
    check(cudaMemsetAsync(zt, 0, tot * sizeof(T), st), "memset z");
    sandwich<T>(c, k2, I.Sch, h, I.Svh, r, B.tmp);           // r~ = h~
    check(cudaMemcpyAsync(p, r, tot * sizeof(T), cudaMemcpyDeviceToDevice, st), "copy p");
    dots<T>(st, r, len, r, len, k2, len, B.dvec2, B.gscr);
    cg_init(st, k2, ptol, B.dvec2, B.cg_rr, B.cg_r0, B.cg_active, B.cg_nactive);
    int *hn = reinterpret_cast<int *>(S->host + 2 * S->k) + 1;
    for (int it = 0; it < c->opt.precond_maxit; ++it) {
        check(cudaMemcpyAsync(hn, B.cg_nactive, sizeof(int), cudaMemcpyDeviceToHost, st), "D2H n_active");
        check(ctx_sync(c), "sync cg");
        if (*hn == 0) break;
        S->inner_iters += 1;
        gemm<T>(st, false, false, nc, nv, nc, T(1), I.Mct, nc, 0, p, nv, len, T(0), Lp, nv, len, k2);
        gemm<T>(st, false, false, k2 * nc, nv, nv, T(-1), p, nv, 0, I.Mvt, nv, 0, T(1), Lp, nv, 0, 1);
        dots<T>(st, p, len, Lp, len, k2, len, B.cg_pLp, B.gscr);
        cg_scalars(st, k2, 0, ptol, B.cg_pLp, B.cg_rrn, B.cg_rr, B.cg_r0, B.cg_alpha,
                   B.cg_beta, B.cg_active, B.cg_nactive);
        axpy_dev<T>(st, B.cg_alpha, 1, 1.0, zt, p, len, k2);
        axpy_dev<T>(st, B.cg_alpha, 1, -1.0, r, Lp, len, k2);
        dots<T>(st, r, len, r, len, k2, len, B.cg_rrn, B.gscr);
        cg_scalars(st, k2, 1, ptol, B.cg_pLp, B.cg_rrn, B.cg_rr, B.cg_r0, B.cg_alpha,
                   B.cg_beta, B.cg_active, B.cg_nactive);
        cg_dir<T>(st, p, r, B.cg_beta, len, k2);
    }
    sandwich<T>(c, k2, I.Scmh, zt, I.Svmh, z, B.tmp);        // z = Sc^{-1/2} z~ Sv^{-1/2}
}

// learned preconditioner: fixed features and feature rows on first use; scales for k states
template <typename T>
void ensure_learned(tddft_ctx *c, Impl<T> &I, int k) {
    if (!c->uniform) throw InvalidArg{"the learned preconditioner needs equal function counts on every atom"};
    const int na = c->natoms;
    if (!I.lfc) {
        const int nb = 2 * c->nca * c->nva, nf = 2 * c->nca * c->nca + 2 * c->nva * c->nva + 1;
        I.lfc = I.lmemf.template alloc<float>((size_t)na * 2 * c->nca * c->nca);
        I.lfv = I.lmemf.template alloc<float>((size_t)na * 2 * c->nva * c->nva);
        I.ldist = I.lmemf.template alloc<float>((size_t)na * na);
        I.lF = I.lmemf.template alloc<float>((size_t)na * na * nf);
        I.lA = I.lmemf.template alloc<float>((size_t)na * na * nb * nb);
        check(cudaMemcpyAsync(I.ldist, c->adist.data(), (size_t)na * na * sizeof(float), cudaMemcpyHostToDevice,
                              c->st),
              "upload atom distances");
        learned_fixed_features<T>(c->st, I.Mc, I.Sc, c->nc, c->nca, na, I.lfc);
        learned_fixed_features<T>(c->st, I.Mv, I.Sv, c->nv, c->nva, na, I.lfv);
        learned_feature_rows(c->st, I.lfc, I.lfv, I.ldist, na, c->nca, c->nva, I.lF);
        check(ctx_sync(c), "sync learned features");
    }
    const long long rows = (long long)k * na * na;
    if (rows <= I.lrows) return;
    check(ctx_sync(c), "sync before learned buffers");
    I.lmemr.release();
    I.ls = I.lmemr.template alloc<float>((size_t)rows);
    I.lrows = rows;
}

// z_IJ = h_IJ + A_IJ h_IJ with the block maps of the bound model (recomputed when it changes)
template <typename T>
void learned_precondition(tddft_ctx *c, tddft_state *S, const T *h, T *z) {
    Impl<T> &I = impl<T>(c);
    const int k = S->k, na = c->natoms;
    if (!c->mlp) throw InvalidArg{"TDDFT_PRECOND_LEARNED without a model (tddft_set_mlp)"};
    if (mlp_n_block(c->mlp) != 2 * c->nca * c->nva ||
        mlp_n_feat(c->mlp) != 2 * c->nca * c->nca + 2 * c->nva * c->nva + 1)
        throw InvalidArg{"model sizes do not match the system's rows (tddft_learned_dims)"};
    ensure_learned<T>(c, I, k);
    if (I.lA_model != c->mlp || I.lA_version != mlp_version(c->mlp)) {
        mlp_block_maps(c->st, c->mlp, (long long)na * na, I.lF, I.lA);
        I.lA_model = c->mlp;
        I.lA_version = mlp_version(c->mlp);
    }
    learned_apply<T>(c->st, I.lA, h, k, na, c->nca, c->nva, c->nc, c->nv, z);
}

// the gradient the preconditioner acts on: g, or P^c G_L P^v with truncation
template <typename T>
const T *search_gradient(tddft_ctx *c, tddft_state *S) {
    Impl<T> &I = impl<T>(c);
    StateBufs<T> &B = bufs<T>(S);
    if (c->trunc) {
        // P^c G_L P^v; with the exact preconditioner it only feeds that preconditioner, whose
        // errors change the search direction and not the fixed point: one TF32 MMA per product
        sandwich_x<T>(c, I, 2 * S->k, SP_P, B.G1, B.h, B.tmp, I.exact);
        return B.h;
    }
    return B.g;
}

// one PCG update from an evaluated iterate (Sec. III C)
template <typename T>
void update(tddft_ctx *c, tddft_state *S) {
    Impl<T> &I = impl<T>(c);
    StateBufs<T> &B = bufs<T>(S);
    const int k = S->k, k2 = 2 * k;
    const long long len = c->len(), tot = k2 * len;
    cudaStream_t st = c->st;
    // preconditioned gradient in the search variables
    const T *h = search_gradient<T>(c, S);
    // z from the learned map (mode 1), the preconditioner of the options (0), or the search
    // gradient itself (2)
    auto precondition_and_dots = [&](int mode) {
        if (mode == 1) learned_precondition<T>(c, S, h, B.z);
        else if (mode == 0) precondition<T>(c, S, h, B.z);
        else check(cudaMemcpyAsync(B.z, h, tot * sizeof(T), cudaMemcpyDeviceToDevice, st), "copy z");
        if (c->trunc) mask_mul<T>(st, B.z, I.mask, len, k2);
        sandwich_x<T>(c, I, k2, SP_R, B.z, B.Z, B.tmp);     // Z = P^c S z S P^v (Eq. auxiliary)
        // Polak-Ribiere over the set
        if (c->trunc) {
            dots<T>(st, B.G1, len, B.z, len, k2, len, B.dvec, B.gscr);
            dots<T>(st, B.G1, len, B.pz, len, k2, len, B.dvec2, B.gscr);
            dots<T>(st, B.G1, len, B.pdir, len, k2, len, B.dvec3, B.gscr);
        } else {
            dots<T>(st, B.G1, len, B.Z, len, k2, len, B.dvec, B.gscr);
            dots<T>(st, B.G1, len, B.pZ, len, k2, len, B.dvec2, B.gscr);
            dots<T>(st, B.G1, len, B.pD, len, k2, len, B.dvec3, B.gscr);
        }
    };
    const bool learned = c->opt.precond == TDDFT_PRECOND_LEARNED;
    auto slope_sum = [&]() {
        check(cudaMemcpyAsync(S->host, B.dvec, k2 * sizeof(double), cudaMemcpyDeviceToHost, st), "D2H gz");
        check(ctx_sync(c), "sync gz");
        double gz = 0.0;
        for (int i = 0; i < k2; ++i) gz += S->host[i];
        return gz;
    };
    precondition_and_dots(learned ? 1 : 0);
    if (learned) {
        // the CG solve stands in when -z is not a descent direction (<g, Z> summed <= 0)
        if (!(slope_sum() > 0.0)) {
            S->fallbacks += 1;
            precondition_and_dots(0);
        }
    } else if (c->sparse && c->opt.precond == TDDFT_PRECOND_ITER) {
        // truncated form: with every product cut to the pattern, and P^c, P^v truncated, the
        // inner CG's operator need not be positive definite, and its result need not be a
        // descent direction (<G_L, z> summed <= 0, the CG stopped on non-positive curvature);
        // that step then takes the search gradient itself
        if (!(slope_sum() > 0.0)) {
            S->fallbacks += 1;
            precondition_and_dots(2);
        }
    }
    const int restart = (S->it == 0 || S->it % std::max(1, c->opt.restart_every) == 0) ? 1 : 0;
    conj_coeff(st, k2, B.dvec, B.dvec2, B.dvec3, restart, B.flip, B.sc);
    direction<T>(st, B.dir, B.z, B.pdir, B.sc + 2, tot);
    direction<T>(st, B.D, B.Z, B.pD, B.sc + 2, tot);
    // one operator application on the directions
    apply_impl<T>(c, I, k, B.D, B.fD, true);
    covariant<T>(c, I, k2, B.D, B.covD, B.tmp);
    {
        // the six traces of the line step in two passes (cov(D) and cov(P) read once each)
        const T *yd[4] = {B.f, B.fD, B.P, B.D};
        double *gd[4] = {B.BDf, B.CDfD, B.DP, B.DD};
        gram_multi<T>(st, B.covD, len, k2, 4, yd, len, k2, len, gd, B.gscr);
        const T *yp[2] = {B.P, B.D};
        double *gp[2] = {B.PP, B.PD};
        gram_multi<T>(st, B.covP, len, k2, 2, yp, len, k2, len, gp, B.gscr);
    }
    line_gs(st, k, B.A, B.BDf, B.CDfD, B.PP, B.PD, B.DP, B.DD, B.Q, B.lam, B.Cp, B.Cq, B.flip,
            B.status);
    axpy_dev<T>(st, B.lam, 0, 1.0, B.Y, B.dir, tot, 1);
    axpy_dev<T>(st, B.lam, 0, 1.0, B.P, B.D, tot, 1);
    axpy_dev<T>(st, B.lam, 0, 1.0, B.f, B.fD, tot, 1);
    axpy_dev<T>(st, B.lam, 0, 1.0, B.covP, B.covD, tot, 1);
    recombine<T>(c, B, k);
    check(cudaMemcpyAsync(S->host + 2 * k + 1, B.lam, sizeof(double), cudaMemcpyDeviceToHost, st), "D2H lam");
    sync_status(c, S, B.status);
    S->it += 1;
    if (c->opt.reapply_every > 0 && S->it % c->opt.reapply_every == 0) {
        // P = P^c S L S P^v afresh from the search variables (Eq. auxiliary), then f = f(P)
        check(cudaMemcpyAsync(B.tmp, B.Y, tot * sizeof(T), cudaMemcpyDeviceToDevice, st), "copy Y");
        if (c->trunc) mask_mul<T>(st, B.tmp, I.mask, len, k2);
        sandwich_x<T>(c, I, k2, SP_R, B.tmp, B.P, B.cLpp);
        covariant<T>(c, I, k2, B.P, B.covP, B.tmp);
        apply_impl<T>(c, I, k, B.P, B.f, true);
    }
    std::swap(B.pdir, B.dir);
    std::swap(B.pD, B.D);
    std::swap(B.pz, B.z);
    std::swap(B.pZ, B.Z);
    S->omega_prev = S->omega;
    S->have_prev_omega = true;
    S->evaluated = false;
}

template <typename T>
bool converged(tddft_ctx *c, tddft_state *S) {
    if (!S->have_prev_omega) return false;
    double rmax = 0.0, dmax = 0.0;
    for (int i = 0; i < S->k; ++i) {
        rmax = std::max(rmax, S->resid[i]);
        dmax = std::max(dmax, std::fabs(S->omega[i] - S->omega_prev[i]));
    }
    return rmax <= c->opt.tol && dmax <= 0.1 * c->opt.tol;
}

template <typename T>
void subspace_pairs(tddft_ctx *c, tddft_state *S, double *omega, double *pairing) {
    StateBufs<T> &B = bufs<T>(S);
    const int k = S->k;
    if (!S->evaluated) evaluate<T>(c, S);
    subspace(c->st, k, B.A, B.evout, B.dvec3);
    check(cudaMemcpyAsync(S->host, B.evout, k * sizeof(double), cudaMemcpyDeviceToHost, c->st), "D2H omega");
    check(cudaMemcpyAsync(S->host + k, B.dvec3, 2 * k * sizeof(double), cudaMemcpyDeviceToHost, c->st), "D2H pairing");
    check(ctx_sync(c), "sync subspace");
    if (omega) std::memcpy(omega, S->host, k * sizeof(double));
    if (pairing) std::memcpy(pairing, S->host + k, 2 * k * sizeof(double));
}

template <typename T>
tddft_status solve_impl(tddft_ctx *c, tddft_state *S, double *omega, double *resid, int32_t *iters) {
    bool conv = false;
    for (int it = 0; it < c->opt.max_iter; ++it) {
        evaluate<T>(c, S);
        if (converged<T>(c, S)) {
            conv = true;
            break;
        }
        update<T>(c, S);
    }
    if (!conv) {
        evaluate<T>(c, S);
        conv = converged<T>(c, S);
    }
    if (omega) std::memcpy(omega, S->omega.data(), S->k * sizeof(double));
    if (resid) std::memcpy(resid, S->resid.data(), S->k * sizeof(double));
    if (iters) *iters = S->it;
    if (!conv) {
        c->err = "not converged within max_iter";
        return TDDFT_E_NOT_CONVERGED;
    }
    if (!c->trunc) {
        std::vector<double> om(S->k), pr(2 * S->k);
        subspace_pairs<T>(c, S, om.data(), pr.data());
        double rmax = 0.0, omax = 0.0, pmax = 0.0;
        for (int i = 0; i < S->k; ++i) {
            rmax = std::max(rmax, S->resid[i]);
            omax = std::max(omax, std::fabs(om[i]));
        }
        for (double v : pr) pmax = std::max(pmax, v);
        if (pmax > 10.0 * rmax * (1.0 + omax) + 1e-10) {
            c->err = "converged pairs fail the +-omega pairing check";
            return TDDFT_E_PAIRING;
        }
    }
    return TDDFT_OK;
}

}  // namespace

namespace {

// checkpoint layout: header, host scalars, omega_prev [k], the conjugation scalars, then the eight
// device arrays that carry from one PCG step to the next, each [2k][N_chi][N_phi] of T
constexpr char CKPT_MAGIC[8] = {'T', 'D', 'D', 'F', 'T', 'S', 'T', '1'};
constexpr int32_t CKPT_VERSION = 1;
struct CkptHeader {
    char magic[8];
    int32_t version, precision, k, n_chi, n_phi, it, fallbacks, have_prev_omega;
    int64_t inner_iters;
};
static_assert(sizeof(CkptHeader) == 48, "checkpoint header layout");
constexpr int CKPT_SCALARS = 5;   // conjugation scalars (4) and the Gram-Schmidt reorder flag

template <typename T>
std::array<T *, 8> carried(StateBufs<T> &B) {
    return {B.Y, B.P, B.f, B.covP, B.pdir, B.pD, B.pz, B.pZ};
}

size_t ckpt_bytes(const tddft_ctx *c, int k, int prec) {
    const size_t el = prec == TDDFT_FP64 ? sizeof(double) : sizeof(float);
    return sizeof(CkptHeader) + (size_t)(k + CKPT_SCALARS) * sizeof(double) + 8 * (size_t)2 * k * c->len() * el;
}

}  // namespace

// ================================================================================================
// ABI

#define DISPATCH(ctx, EXPR)                                   \
    ((ctx)->prec == TDDFT_FP64 ? ([&]() { using T = double; return EXPR; })() \
                               : ([&]() { using T = float; return EXPR; })())

extern "C" {

void tddft_default_options(tddft_options *o) {
    if (!o) return;
    o->precision = TDDFT_FP64;
    o->mode = TDDFT_MODE_FULL;
    o->precond = TDDFT_PRECOND_ITER;
    o->precond_maxit = 50;
    o->precond_tol = 1e-4;
    o->tol = 1e-6;
    o->max_iter = 500;
    o->reapply_every = 10;
    o->restart_every = 10;
    o->precond_adaptive = 0;
    o->spin_limit_cycles = 0;
}

tddft_status tddft_create(const tddft_system *s, const tddft_options *opt, void *stream,
                          tddft_ctx **out) {
    if (!out) return TDDFT_E_INVALID;
    *out = nullptr;
    auto c = std::make_unique<tddft_ctx>();
    if (opt) c->opt = *opt;
    else tddft_default_options(&c->opt);
    c->st = static_cast<cudaStream_t>(stream);
    c->prec = c->opt.precision;
    tddft_status rc = guarded(c.get(), [&]() -> tddft_status {
        if (!s) throw InvalidArg{"null system"};
        if (c->prec != TDDFT_FP64 && c->prec != TDDFT_MIXED) throw InvalidArg{"unknown precision"};
        if (c->opt.mode < 0 || c->opt.mode > 2) throw InvalidArg{"unknown mode"};
        if (c->opt.precond < 0 || c->opt.precond > 3) throw InvalidArg{"unknown preconditioner"};
        if (!(s->cell > 0.0)) throw InvalidArg{"cell must be positive"};
        if (!fft_size_ok(s->n)) throw InvalidArg{"grid size must be 2^a 3^b 5^c with 8 <= n <= 256"};
        if (s->natoms <= 0 || !s->pos) throw InvalidArg{"no atoms"};
        if (!s->S_chi || !s->S_phi || !s->H_chi || !s->H_phi || !s->P_v || !s->P_c) throw InvalidArg{"null matrix"};
        if (s->fxc_kind == TDDFT_FXC_LDA_PW92 && !s->n0) throw InvalidArg{"LDA kernel needs n0"};
        validate_funcs(s->phi, s->n, s->natoms, "phi");
        validate_funcs(s->chi, s->n, s->natoms, "chi");
        c->n = s->n;
        c->nt = (s->n + TILE - 1) / TILE;
        c->natoms = s->natoms;
        c->nc = s->chi.nfun;
        c->nv = s->phi.nfun;
        c->cell = s->cell;
        const double h = s->cell / s->n;
        c->dV = h * h * h;
        c->trunc = s->kernel_cutoff > 0.0;
        // per-atom function counts and atom distances (learned preconditioner)
        c->uniform = s->chi.nfun % s->natoms == 0 && s->phi.nfun % s->natoms == 0;
        if (c->uniform) {
            c->nca = s->chi.nfun / s->natoms;
            c->nva = s->phi.nfun / s->natoms;
            for (int f = 0; f < s->chi.nfun && c->uniform; ++f) c->uniform = s->chi.atom[f] == f / c->nca;
            for (int f = 0; f < s->phi.nfun && c->uniform; ++f) c->uniform = s->phi.atom[f] == f / c->nva;
        }
        c->adist.assign((size_t)s->natoms * s->natoms, 0.0f);
        for (int a = 0; a < s->natoms; ++a)
            for (int b = 0; b < s->natoms; ++b) {
                double d2 = 0.0;
                for (int x = 0; x < 3; ++x) {
                    double d = s->pos[3 * a + x] - s->pos[3 * b + x];
                    d -= s->cell * std::nearbyint(d / s->cell);
                    d2 += d * d;
                }
                c->adist[(size_t)a * s->natoms + b] = (float)(std::sqrt(d2) / 10.0);
            }
        c->amask.assign((size_t)s->natoms * s->natoms, 1);
        if (c->trunc) {
            for (int a = 0; a < s->natoms; ++a)
                for (int b = 0; b < s->natoms; ++b) {
                    double d2 = 0.0;
                    for (int x = 0; x < 3; ++x) {
                        double d = s->pos[3 * a + x] - s->pos[3 * b + x];
                        d -= s->cell * std::nearbyint(d / s->cell);
                        d2 += d * d;
                    }
                    c->amask[(size_t)a * s->natoms + b] = std::sqrt(d2) <= s->kernel_cutoff ? 1 : 0;
                }
        }
        check(cudaGetDevice(&c->device), "cudaGetDevice");
        check(cudaMallocHost(reinterpret_cast<void **>(&c->hword), sizeof(int)), "cudaMallocHost");
        *c->hword = 0;
        if (c->prec == TDDFT_FP64) build_impl<double>(c.get(), s);
        else build_impl<float>(c.get(), s);
        return TDDFT_OK;
    });
    if (rc != TDDFT_OK) {
        static thread_local std::string last;
        last = c->err;
        std::fprintf(stderr, "tddft_create: %s\n", last.c_str());
        return rc;
    }
    *out = c.release();
    return TDDFT_OK;
}

tddft_status tddft_create_sparse(const tddft_sparse_system *s, const tddft_options *opt, void *stream,
                                 tddft_ctx **out) {
    if (!out) return TDDFT_E_INVALID;
    *out = nullptr;
    auto c = std::make_unique<tddft_ctx>();
    if (opt) c->opt = *opt;
    else tddft_default_options(&c->opt);
    c->st = static_cast<cudaStream_t>(stream);
    c->prec = c->opt.precision;
    tddft_status rc = guarded(c.get(), [&]() -> tddft_status {
        if (!s) throw InvalidArg{"null system"};
        if (c->prec != TDDFT_FP64 && c->prec != TDDFT_MIXED) throw InvalidArg{"unknown precision"};
        if (c->opt.mode < 0 || c->opt.mode > 2) throw InvalidArg{"unknown mode"};
        if (c->opt.precond != TDDFT_PRECOND_ITER && c->opt.precond != TDDFT_PRECOND_NONE)
            throw InvalidArg{"the truncated form takes the iterative preconditioner or none"};
        if (!(s->cell > 0.0)) throw InvalidArg{"cell must be positive"};
        if (!fft_size_ok(s->n)) throw InvalidArg{"grid size must be 2^a 3^b 5^c with 8 <= n <= 256"};
        if (s->natoms <= 0 || !s->pos) throw InvalidArg{"no atoms"};
        if (!(s->kernel_cutoff > 0.0)) throw InvalidArg{"the truncated form needs kernel_cutoff > 0"};
        if (s->fxc_kind == TDDFT_FXC_LDA_PW92 && !s->n0) throw InvalidArg{"LDA kernel needs n0"};
        validate_funcs(s->phi, s->n, s->natoms, "phi");
        validate_funcs(s->chi, s->n, s->natoms, "chi");
        c->n = s->n;
        c->nt = (s->n + TILE - 1) / TILE;
        c->natoms = s->natoms;
        c->nc = s->chi.nfun;
        c->nv = s->phi.nfun;
        c->cell = s->cell;
        const double h = s->cell / s->n;
        c->dV = h * h * h;
        c->trunc = true;
        c->sparse = true;
        c->uniform = false;   // the learned preconditioner is not offered in this form
        check(cudaGetDevice(&c->device), "cudaGetDevice");
        check(cudaMallocHost(reinterpret_cast<void **>(&c->hword), sizeof(int)), "cudaMallocHost");
        *c->hword = 0;
        try {
            c->sp = sparse_build(c->st, s);
        } catch (const std::invalid_argument &e) {
            throw InvalidArg{e.what()};
        }
        c->amask = c->sp->amask;
        c->adist.assign((size_t)s->natoms * s->natoms, 0.0f);
        if (c->prec == TDDFT_FP64) build_impl<double>(c.get(), nullptr, s);
        else build_impl<float>(c.get(), nullptr, s);
        return TDDFT_OK;
    });
    if (rc != TDDFT_OK) {
        std::fprintf(stderr, "tddft_create_sparse: %s\n", c->err.c_str());
        return rc;
    }
    *out = c.release();
    return TDDFT_OK;
}

tddft_status tddft_kernel_pattern(const tddft_ctx *c, int64_t *nnzb, int64_t *nnz, int64_t *row_ptr, int32_t *col_idx,
                                  int64_t *blk_off) {
    if (!c || !c->sparse) return TDDFT_E_INVALID;
    const SparseLayout &L = *c->sp;
    if (nnzb) *nnzb = (int64_t)L.abi_col.size();
    if (nnz) *nnz = L.nnz_abi;
    if (row_ptr) std::copy(L.abi_row_ptr.begin(), L.abi_row_ptr.end(), row_ptr);
    if (col_idx) std::copy(L.abi_col.begin(), L.abi_col.end(), col_idx);
    if (blk_off) std::copy(L.abi_blk_off.begin(), L.abi_blk_off.end(), blk_off);
    return TDDFT_OK;
}

tddft_status tddft_create_batch(const tddft_system *sys, int32_t nsys, const tddft_options *opt, void *stream,
                                tddft_ctx **out) {
    if (!sys || !out || nsys <= 0) return TDDFT_E_INVALID;
    for (int i = 0; i < nsys; ++i) out[i] = nullptr;
    cudaStream_t caller = static_cast<cudaStream_t>(stream);
    cudaEvent_t ready = nullptr;
    if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(ready, caller) != cudaSuccess) {
        if (ready) cudaEventDestroy(ready);
        return TDDFT_E_CUDA;
    }
    std::vector<tddft_status> rc(nsys, TDDFT_OK);
    std::atomic<int> next{0};
    int dev = 0;
    cudaGetDevice(&dev);
    auto worker = [&]() {
        cudaSetDevice(dev);   // the caller's device in every host thread
        for (int i = next++; i < nsys; i = next++) {
            cudaStream_t st = nullptr;
            cudaEvent_t ev = nullptr;
            if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
                cudaStreamWaitEvent(st, ready, 0) != cudaSuccess ||
                cudaEventCreateWithFlags(&ev, cudaEventBlockingSync | cudaEventDisableTiming) != cudaSuccess) {
                if (st) cudaStreamDestroy(st);
                if (ev) cudaEventDestroy(ev);
                rc[i] = TDDFT_E_CUDA;
                continue;
            }
            tddft_ctx *c = nullptr;
            rc[i] = tddft_create(&sys[i], opt, st, &c);
            if (rc[i] != TDDFT_OK) {
                cudaStreamSynchronize(st);
                cudaStreamDestroy(st);
                cudaEventDestroy(ev);
                continue;
            }
            c->own_stream = true;
            c->sync_ev = ev;
            out[i] = c;
        }
    };
    const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
    const int nt = std::max(1, std::min({(int)nsys, 16, hw}));
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
    worker();
    for (std::thread &t : pool) t.join();
    cudaEventDestroy(ready);
    for (int i = 0; i < nsys; ++i)
        if (rc[i] != TDDFT_OK) {
            for (int j = 0; j < nsys; ++j) {
                tddft_destroy(out[j]);
                out[j] = nullptr;
            }
            return rc[i];
        }
    return TDDFT_OK;
}

tddft_status tddft_solve_batch(tddft_ctx *const *ctx, tddft_state *const *st, int32_t nsys, int32_t nthreads,
                               double *omega, double *resid, int32_t *iters, int32_t *status) {
    if (!ctx || !st || nsys <= 0) return TDDFT_E_INVALID;
    std::vector<long long> off(nsys + 1, 0);
    for (int i = 0; i < nsys; ++i) {
        if (!ctx[i] || !st[i] || st[i]->ctx != ctx[i]) return TDDFT_E_INVALID;
        for (int j = 0; j < i; ++j)
            if (ctx[j] == ctx[i]) return TDDFT_E_INVALID;   // a context is driven by one thread at a time
        off[i + 1] = off[i] + st[i]->k;
    }
    // largest systems first, so that the long solves start early
    std::vector<int> order(nsys);
    for (int i = 0; i < nsys; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return ctx[a]->pair_points * st[a]->k > ctx[b]->pair_points * st[b]->k;
    });
    std::vector<tddft_status> rc(nsys, TDDFT_OK);
    std::vector<int32_t> it(nsys, 0);
    std::atomic<int> next{0};
    int dev = 0;
    cudaGetDevice(&dev);
    auto worker = [&]() {
        cudaSetDevice(dev);
        for (int q = next++; q < nsys; q = next++) {
            const int i = order[q];
            rc[i] = tddft_solve(ctx[i], st[i], omega ? omega + off[i] : nullptr, resid ? resid + off[i] : nullptr,
                                &it[i]);
        }
    };
    int nt = nthreads > 0 ? nthreads : 16;
    nt = std::max(1, std::min(nt, (int)nsys));
    std::vector<std::thread> pool;
    for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
    worker();
    for (std::thread &t : pool) t.join();
    tddft_status first = TDDFT_OK;
    for (int i = 0; i < nsys; ++i) {
        if (iters) iters[i] = it[i];
        if (status) status[i] = rc[i];
        if (first == TDDFT_OK && rc[i] != TDDFT_OK) first = rc[i];
    }
    return first;
}

tddft_status tddft_joint_projector(void *cuda_stream, int32_t n_joint, int32_t n_phi, const double *S_joint,
                                   const double *S_joint_phi, const double *P_v, double *P_c) {
    if (n_joint <= 0 || n_phi <= 0 || !S_joint || !S_joint_phi || !P_v || !P_c) return TDDFT_E_INVALID;
    tddft_ctx tmp;   // carries the error text only
    tmp.st = static_cast<cudaStream_t>(cuda_stream);
    const tddft_status rc = guarded(&tmp, [&]() -> tddft_status {
        cudaStream_t st = tmp.st;
        const int nj = n_joint, nv = n_phi;
        const long long jj = (long long)nj * nj, jv = (long long)nj * nv, vv = (long long)nv * nv;
        Mem m;
        double *S = m.alloc<double>(jj), *Sjp = m.alloc<double>(jv), *Pv = m.alloc<double>(vv);
        check(cudaMemcpyAsync(S, S_joint, jj * sizeof(double), cudaMemcpyDefault, st), "copy S_joint");
        check(cudaMemcpyAsync(Sjp, S_joint_phi, jv * sizeof(double), cudaMemcpyDefault, st), "copy S_joint_phi");
        check(cudaMemcpyAsync(Pv, P_v, vv * sizeof(double), cudaMemcpyDefault, st), "copy P_v");
        std::vector<double> Sh_host((size_t)jj);
        check(cudaMemcpyAsync(Sh_host.data(), S, jj * sizeof(double), cudaMemcpyDeviceToHost, st), "D2H S_joint");
        check(cudaStreamSynchronize(st), "sync joint projector");
        double *Sh = m.alloc<double>(jj), *Smh = m.alloc<double>(jj), *X = m.alloc<double>(jj);
        overlap_roots(st, m, S, Sh_host.data(), nj, Sh, Smh);
        gemm<double>(st, false, false, nj, nj, nj, 1.0, Smh, nj, 0, Smh, nj, 0, 0.0, X, nj, 0, 1);        // S^-1
        double *T1 = m.alloc<double>(jv), *T = m.alloc<double>(jj), *Y = m.alloc<double>(jj);
        gemm<double>(st, false, false, nj, nv, nv, 1.0, Sjp, nv, 0, Pv, nv, 0, 0.0, T1, nv, 0, 1);         // S^{vp} P^v
        gemm<double>(st, false, true, nj, nj, nv, 1.0, T1, nv, 0, Sjp, nv, 0, 0.0, T, nj, 0, 1);          // .. S^{pv}
        gemm<double>(st, false, false, nj, nj, nj, 1.0, X, nj, 0, T, nj, 0, 0.0, Y, nj, 0, 1);            // S^-1 T
        double *Pc = m.alloc<double>(jj);
        check(cudaMemcpyAsync(Pc, X, jj * sizeof(double), cudaMemcpyDeviceToDevice, st), "copy S^-1");
        gemm<double>(st, false, false, nj, nj, nj, -1.0, Y, nj, 0, X, nj, 0, 1.0, Pc, nj, 0, 1);          // X - Y X
        check(cudaMemcpyAsync(P_c, Pc, jj * sizeof(double), cudaMemcpyDefault, st), "copy P_c");
        check(cudaStreamSynchronize(st), "sync joint projector");
        return TDDFT_OK;
    });
    if (rc != TDDFT_OK) std::fprintf(stderr, "tddft_joint_projector: %s\n", tmp.err.c_str());
    return rc;
}

void tddft_destroy(tddft_ctx *c) {
    if (!c) return;
    cudaStreamSynchronize(c->st);
    delete c;
}

const char *tddft_last_error(const tddft_ctx *c) { return c ? c->err.c_str() : "null context"; }

tddft_status tddft_dims(const tddft_ctx *c, int32_t *nc, int32_t *nv, int32_t *n) {
    if (!c) return TDDFT_E_INVALID;
    if (nc) *nc = c->nc;
    if (nv) *nv = c->nv;
    if (n) *n = c->n;
    return TDDFT_OK;
}

tddft_status tddft_apply(tddft_ctx *c, int32_t k, const double *Pp, const double *Pq, double *fp,
                         double *fq) {
    if (!c) return TDDFT_E_INVALID;
    return guarded(c, [&]() -> tddft_status {
        if (k <= 0 || !Pp || !Pq || !fp || !fq) throw InvalidArg{"tddft_apply: bad arguments"};
        const long long kl = (long long)k * c->len();
        return DISPATCH(c, ([&]() {
            Impl<T> &I = impl<T>(c);
            ensure_workspace(c, I, 2 * k);
            abi_in<T>(c, I, Pp, I.bufP, k);
            abi_in<T>(c, I, Pq, I.bufP + kl, k);
            apply_impl<T>(c, I, k, I.bufP, I.bufF);
            abi_out<T>(c, I, I.bufF, fp, k);
            abi_out<T>(c, I, I.bufF + kl, fq, k);
            check_tc_error(c);
            return TDDFT_OK;
        })());
    });
}

tddft_status tddft_response_density(tddft_ctx *c, int32_t k, const double *P, double *rho) {
    if (!c) return TDDFT_E_INVALID;
    return guarded(c, [&]() -> tddft_status {
        if (k <= 0 || !P || !rho) throw InvalidArg{"tddft_response_density: bad arguments"};
        return DISPATCH(c, ([&]() {
            Impl<T> &I = impl<T>(c);
            ensure_workspace(c, I, k);
            abi_in<T>(c, I, P, I.bufP, k);
            density(c, I, I.bufP, k);
            download<T>(c, I, I.rho, rho, (long long)k * c->n3());
            check_tc_error(c);
            return TDDFT_OK;
        })());
    });
}

tddft_status tddft_response_potential(tddft_ctx *c, int32_t k, const double *rho, double *V) {
    if (!c) return TDDFT_E_INVALID;
    return guarded(c, [&]() -> tddft_status {
        if (k <= 0 || !rho || !V) throw InvalidArg{"tddft_response_potential: bad arguments"};
        return DISPATCH(c, ([&]() {
            Impl<T> &I = impl<T>(c);
            ensure_workspace(c, I, k);
            upload<T>(c, I, rho, I.rho, (long long)k * c->n3());
            hartree_fxc<T>(c->st, c->grid(), I.rho, I.fxc, k, I.V, I.fft);
            download<T>(c, I, I.V, V, (long long)k * c->n3());
            check(ctx_sync(c), "sync potential");
            return TDDFT_OK;
        })());
    });
}

tddft_status tddft_potential_integrals(tddft_ctx *c, int32_t k, const double *V, double *out) {
    if (!c) return TDDFT_E_INVALID;
    return guarded(c, [&]() -> tddft_status {
        if (k <= 0 || !V || !out) throw InvalidArg{"tddft_potential_integrals: bad arguments"};
        return DISPATCH(c, ([&]() {
            Impl<T> &I = impl<T>(c);
            ensure_workspace(c, I, k);
            upload<T>(c, I, V, I.V, (long long)k * c->n3());
            integrals(c, I, k);
            abi_out<T>(c, I, I.Vmat, out, k);
            check_tc_error(c);
            return TDDFT_OK;
        })());
    });
}

tddft_status tddft_fxc(tddft_ctx *c, double *fxc) {
    if (!c || !fxc) return TDDFT_E_INVALID;
    return guarded(c, [&]() -> tddft_status {
        const double *src = c->prec == TDDFT_FP64 ? c->d64->fxc64 : c->d32->fxc64;
        check(cudaMemcpyAsync(fxc, src, c->n3() * sizeof(double), cudaMemcpyDefault, c->st), "copy fxc");
        check(ctx_sync(c), "sync fxc");
        return TDDFT_OK;
    });
}

tddft_status tddft_state_create(tddft_ctx *c, int32_t k, const double *Y0, tddft_state **out) {
    if (!c || !out) return TDDFT_E_INVALID;
    *out = nullptr;
    auto S = std::make_unique<tddft_state>();
    tddft_status rc = guarded(c, [&]() -> tddft_status {
        if (k <= 0 || k > KMAX || !Y0) throw InvalidArg{"tddft_state_create: need 1 <= k <= 16 and Y0"};
        S->ctx = c;
        S->k = k;
        check(cudaMallocHost(reinterpret_cast<void **>(&S->host), (4 * k + 16) * sizeof(double)), "cudaMallocHost");
        return DISPATCH(c, ([&]() {
            alloc_state<T>(c, S.get());
            state_init<T>(c, S.get(), Y0);
            return TDDFT_OK;
        })());
    });
    if (rc == TDDFT_OK) *out = S.release();
    return rc;
}

void tddft_state_destroy(tddft_state *s) {
    if (!s) return;
    cudaDeviceSynchronize();   // the state's buffers may still be in use by queued work
    delete s;
}

tddft_status tddft_pcg_step(tddft_ctx *c, tddft_state *S, double *omega, double *resid) {
    if (!c || !S || S->ctx != c) return TDDFT_E_INVALID;
    return guarded(c, [&]() -> tddft_status {
        return DISPATCH(c, ([&]() {
            if (!S->evaluated) evaluate<T>(c, S);
            if (omega) std::memcpy(omega, S->omega.data(), S->k * sizeof(double));
            if (resid) std::memcpy(resid, S->resid.data(), S->k * sizeof(double));
            update<T>(c, S);
            return TDDFT_OK;
        })());
    });
}

tddft_status tddft_solve(tddft_ctx *c, tddft_state *S, double *omega, double *resid, int32_t *iters) {
    if (!c || !S || S->ctx != c) return TDDFT_E_INVALID;
    return guarded(c, [&]() -> tddft_status {
        return DISPATCH(c, (solve_impl<T>(c, S, omega, resid, iters)));
    });
}

tddft_status tddft_state_get(tddft_ctx *c, const tddft_state *S, double *Pp, double *Pq, double *fp,
                             double *fq, double *Lp, double *Lq) {
    if (!c || !S || S->ctx != c) return TDDFT_E_INVALID;
    return guarded(c, [&]() -> tddft_status {
        return DISPATCH(c, ([&]() {
            Impl<T> &I = impl<T>(c);
            StateBufs<T> &B = bufs<T>(const_cast<tddft_state *>(S));
            const long long kl = (long long)S->k * c->len();
            ensure_workspace(c, I, 2 * S->k);
            abi_out<T>(c, I, B.P, Pp, S->k);
            abi_out<T>(c, I, B.P + kl, Pq, S->k);
            abi_out<T>(c, I, B.f, fp, S->k);
            abi_out<T>(c, I, B.f + kl, fq, S->k);
            abi_out<T>(c, I, B.Y, Lp, S->k);
            abi_out<T>(c, I, B.Y + kl, Lq, S->k);
            check(ctx_sync(c), "sync state_get");
            return TDDFT_OK;
        })());
    });
}

tddft_status tddft_state_export(tddft_ctx *c, const tddft_state *S, void *buf, size_t *len) {
    if (!c || !S || S->ctx != c || !len) return TDDFT_E_INVALID;
    return guarded(c, [&]() -> tddft_status {
        const size_t need = ckpt_bytes(c, S->k, c->prec);
        if (!buf) {
            *len = need;
            return TDDFT_OK;
        }
        if (*len < need) {
            *len = need;
            throw InvalidArg{"tddft_state_export: buffer too small"};
        }
        *len = need;
        return DISPATCH(c, ([&]() {
            tddft_state *Sm = const_cast<tddft_state *>(S);
            StateBufs<T> &B = bufs<T>(Sm);
            unsigned char *o = static_cast<unsigned char *>(buf);
            CkptHeader h{};
            std::memcpy(h.magic, CKPT_MAGIC, 8);
            h.version = CKPT_VERSION;
            h.precision = c->prec;
            h.k = S->k;
            h.n_chi = c->nc;
            h.n_phi = c->nv;
            h.it = S->it;
            h.fallbacks = S->fallbacks;
            h.have_prev_omega = S->have_prev_omega ? 1 : 0;
            h.inner_iters = S->inner_iters;
            std::memcpy(o, &h, sizeof h);
            o += sizeof h;
            std::vector<double> om(S->k, 0.0);
            if (S->have_prev_omega) std::copy(S->omega_prev.begin(), S->omega_prev.end(), om.begin());
            std::memcpy(o, om.data(), S->k * sizeof(double));
            o += S->k * sizeof(double);
            check(cudaMemcpyAsync(o, B.sc, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->st), "D2H sc");
            check(cudaMemcpyAsync(o + 4 * sizeof(double), B.flip, sizeof(double), cudaMemcpyDeviceToHost, c->st),
                  "D2H flip");
            o += CKPT_SCALARS * sizeof(double);
            const size_t bytes = (size_t)2 * S->k * c->len() * sizeof(T);
            for (T *X : carried<T>(B)) {
                check(cudaMemcpyAsync(o, X, bytes, cudaMemcpyDeviceToHost, c->st), "D2H checkpoint");
                o += bytes;
            }
            check(ctx_sync(c), "sync export");
            return TDDFT_OK;
        })());
    });
}

tddft_status tddft_state_import(tddft_ctx *c, const void *buf, size_t len, tddft_state **out) {
    if (!c || !buf || !out) return TDDFT_E_INVALID;
    *out = nullptr;
    auto S = std::make_unique<tddft_state>();
    tddft_status rc = guarded(c, [&]() -> tddft_status {
        CkptHeader h{};
        if (len < sizeof h) throw InvalidArg{"tddft_state_import: truncated checkpoint"};
        std::memcpy(&h, buf, sizeof h);
        if (std::memcmp(h.magic, CKPT_MAGIC, 8) != 0 || h.version != CKPT_VERSION)
            throw InvalidArg{"tddft_state_import: not a checkpoint of this format"};
        if (h.precision != c->prec || h.n_chi != c->nc || h.n_phi != c->nv)
            throw InvalidArg{"tddft_state_import: checkpoint precision or sizes differ from the context"};
        if (h.k <= 0 || h.k > KMAX || h.it < 0) throw InvalidArg{"tddft_state_import: bad header"};
        if (len != ckpt_bytes(c, h.k, c->prec)) throw InvalidArg{"tddft_state_import: length does not match"};
        S->ctx = c;
        S->k = h.k;
        S->it = h.it;
        S->fallbacks = h.fallbacks;
        S->inner_iters = h.inner_iters;
        S->have_prev_omega = h.have_prev_omega != 0;
        check(cudaMallocHost(reinterpret_cast<void **>(&S->host), (4 * S->k + 16) * sizeof(double)),
              "cudaMallocHost");
        return DISPATCH(c, ([&]() {
            Impl<T> &I = impl<T>(c);
            alloc_state<T>(c, S.get());
            ensure_workspace(c, I, 2 * S->k);
            StateBufs<T> &B = bufs<T>(S.get());
            const unsigned char *p = static_cast<const unsigned char *>(buf) + sizeof h;
            const double *om = reinterpret_cast<const double *>(p);
            if (S->have_prev_omega) S->omega_prev.assign(om, om + S->k);
            p += S->k * sizeof(double);
            check(cudaMemcpyAsync(B.sc, p, 4 * sizeof(double), cudaMemcpyHostToDevice, c->st), "H2D sc");
            check(cudaMemcpyAsync(B.flip, p + 4 * sizeof(double), sizeof(double), cudaMemcpyHostToDevice, c->st),
                  "H2D flip");
            p += CKPT_SCALARS * sizeof(double);
            const size_t bytes = (size_t)2 * S->k * c->len() * sizeof(T);
            for (T *X : carried<T>(B)) {
                check(cudaMemcpyAsync(X, p, bytes, cudaMemcpyHostToDevice, c->st), "H2D checkpoint");
                p += bytes;
            }
            check(ctx_sync(c), "sync import");
            return TDDFT_OK;
        })());
    });
    if (rc == TDDFT_OK) *out = S.release();
    return rc;
}

tddft_status tddft_oscillator_strengths(tddft_ctx *c, tddft_state *S, double *omega, double *f, double *mu) {
    if (!c || !S || S->ctx != c) return TDDFT_E_INVALID;
    return guarded(c, [&]() -> tddft_status {
        return DISPATCH(c, ([&]() {
            Impl<T> &I = impl<T>(c);
            StateBufs<T> &B = bufs<T>(S);
            const int k = S->k;
            const long long len = c->len();
            if (!S->evaluated) evaluate<T>(c, S);
            ensure_workspace(c, I, 2 * k);
            // Ritz values and vectors of the symmetrised Q; eigenvectors in coef (k x k)
            subspace(c->st, k, B.A, B.evout, B.dvec3, B.coef);
            density(c, I, B.P + k * len, k);                  // rho^q of the current q_j
            const int nblk = 152;
            double *part = B.gscr, *out = B.gscr + (size_t)KMAX * nblk * 3;
            const double h = c->cell / c->n;
            dipole_partials<T>(c->st, I.rho, c->n, h, c->cell, k, nblk, part);
            ritz_strengths(c->st, k, B.evout, B.coef, part, nblk, c->dV, out);
            std::vector<double> hv(4 * (size_t)k), om(k);
            check(cudaMemcpyAsync(om.data(), B.evout, k * sizeof(double), cudaMemcpyDeviceToHost, c->st), "D2H omega");
            check(cudaMemcpyAsync(hv.data(), out, 4 * k * sizeof(double), cudaMemcpyDeviceToHost, c->st), "D2H f");
            check_tc_error(c);
            if (omega) std::memcpy(omega, om.data(), k * sizeof(double));
            if (f) std::memcpy(f, hv.data(), k * sizeof(double));
            if (mu) std::memcpy(mu, hv.data() + k, 3 * k * sizeof(double));
            return TDDFT_OK;
        })());
    });
}

tddft_status tddft_spectrum(tddft_ctx *c, int32_t k, const double *omega, const double *f, double gamma, int32_t n,
                            const double *E, double *S) {
    if (!c) return TDDFT_E_INVALID;
    return guarded(c, [&]() -> tddft_status {
        if (k <= 0 || n <= 0 || !omega || !f || !E || !S || !(gamma > 0.0))
            throw InvalidArg{"tddft_spectrum: bad arguments"};
        Mem tmp;
        double *d = tmp.alloc<double>(2 * (size_t)k + 2 * (size_t)n);
        check(cudaMemcpyAsync(d, omega, k * sizeof(double), cudaMemcpyDefault, c->st), "copy omega");
        check(cudaMemcpyAsync(d + k, f, k * sizeof(double), cudaMemcpyDefault, c->st), "copy f");
        check(cudaMemcpyAsync(d + 2 * k, E, n * sizeof(double), cudaMemcpyDefault, c->st), "copy E");
        lorentz_spectrum(c->st, k, d, d + k, gamma, n, d + 2 * k, d + 2 * k + n);
        check(cudaMemcpyAsync(S, d + 2 * k + n, n * sizeof(double), cudaMemcpyDefault, c->st), "copy S");
        check(ctx_sync(c), "sync spectrum");
        return TDDFT_OK;
    });
}

tddft_status tddft_subspace(tddft_ctx *c, tddft_state *S, double *omega, double *pairing) {
    if (!c || !S || S->ctx != c) return TDDFT_E_INVALID;
    return guarded(c, [&]() -> tddft_status {
        return DISPATCH(c, ([&]() {
            subspace_pairs<T>(c, S, omega, pairing);
            return TDDFT_OK;
        })());
    });
}

tddft_status tddft_profile(tddft_ctx *c, int32_t enable) {
    if (!c) return TDDFT_E_INVALID;
    return guarded(c, [&]() -> tddft_status {
        check(ctx_sync(c), "sync profile");
        if (!c->prof) c->prof = profiler_new();
        profiler_reset(c->prof);
        c->prof_on = enable != 0;
        return TDDFT_OK;
    });
}

tddft_status tddft_profile_read(tddft_ctx *c, tddft_stage_stats *out, int32_t cap, int32_t *count) {
    if (!c || !out || cap < 0) return TDDFT_E_INVALID;
    return guarded(c, [&]() -> tddft_status {
        long long l[ST_COUNT] = {};
        double ms[ST_COUNT] = {}, fl[ST_COUNT] = {}, by[ST_COUNT] = {};
        if (c->prof) profiler_read(c->prof, l, ms, fl, by);
        const int nst = std::min<int>(cap, ST_COUNT);
        for (int i = 0; i < nst; ++i) {
            std::memset(&out[i], 0, sizeof(out[i]));
            std::strncpy(out[i].name, stage_name(i), sizeof(out[i].name) - 1);
            out[i].launches = l[i];
            out[i].ms = ms[i];
            out[i].flops = fl[i];
            out[i].bytes = by[i];
        }
        if (count) *count = nst;
        return TDDFT_OK;
    });
}

tddft_status tddft_work(const tddft_ctx *c, double *pair_points, double *table_values) {
    if (!c) return TDDFT_E_INVALID;
    if (pair_points) *pair_points = c->pair_points;
    if (table_values) *table_values = c->table_values;
    return TDDFT_OK;
}

tddft_status tddft_response_density_noalloc(tddft_ctx *c, int32_t k, const float *P, float *rho) {
    if (!c) return TDDFT_E_INVALID;
    return guarded(c, [&]() -> tddft_status {
        if (c->prec != TDDFT_MIXED || !c->d32 || !c->d32->grid_tc)
            throw InvalidArg{"tddft_response_density_noalloc: needs a mixed-precision context on the tensor-core path"};
        if (k < 1 || k > noalloc_max_states())
            throw InvalidArg{"tddft_response_density_noalloc: k must be between 1 and " +
                             std::to_string(noalloc_max_states())};
        if (!P || !rho || !is_device_ptr(P) || !is_device_ptr(rho))
            throw InvalidArg{"tddft_response_density_noalloc: P and rho must be device pointers"};
        // the scratch array's address and the kernel are those of the current device: it must be
        // the context's, and so must the buffers
        int cur = -1;
        check(cudaGetDevice(&cur), "cudaGetDevice");
        if (cur != c->device || device_of(P) != c->device || device_of(rho) != c->device)
            throw InvalidArg{"tddft_response_density_noalloc: the current device and the devices of P and rho must "
                             "be the context's device"};
        Impl<float> &I = *c->d32;
        response_density_tc_noalloc(c->st, c->grid(), I.chi, I.phi, I.chi_pm, I.CK, I.NPmax, c->nv, P,
                                    (long long)c->nc * c->nv, k,
                                    rho, I.phi_pm);
        if (response_density_tc_noalloc_error(c->st))
            throw TimeoutErr{"a bounded wait in the density kernel expired"};
        return TDDFT_OK;
    });
}

tddft_status tddft_autotune(tddft_ctx *c, int32_t k, tddft_tuning_entry *out, int32_t cap, int32_t *count) {
    if (!c) return TDDFT_E_INVALID;
    return guarded(c, [&]() -> tddft_status {
        if (k < 1 || k > 2 * KMAX) throw InvalidArg{"tddft_autotune: need 1 <= k <= 32"};
        if (c->prec != TDDFT_MIXED || !c->d32 || !tc_enabled())
            throw InvalidArg{"tddft_autotune: the tensor-core grid kernels belong to mixed-precision contexts"};
        Impl<float> &I = *c->d32;
        ensure_workspace(c, I, k);
        cudaStream_t st = c->st;
        const long long nP = (long long)k * c->len(), nV = (long long)k * c->n3();
        roots::fill_random_kernel<<<1216, 256, 0, st>>>(I.bufP, nP, 0x7a11ull);
        roots::fill_random_kernel<<<1216, 256, 0, st>>>(I.V, nV, 0x7a12ull);
        check_launch("fill_random_kernel");
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        check(cudaEventCreate(&e0), "cudaEventCreate");
        check(cudaEventCreate(&e1), "cudaEventCreate");
        struct Ev {
            cudaEvent_t a, b;
            ~Ev() { cudaEventDestroy(a); cudaEventDestroy(b); }
        } evs{e0, e1};
        auto time_it = [&](auto &&fn) {
            fn();   // warm-up
            check(cudaEventRecord(e0, st), "cudaEventRecord");
            for (int r = 0; r < 3; ++r) fn();
            check(cudaEventRecord(e1, st), "cudaEventRecord");
            check(cudaEventSynchronize(e1), "cudaEventSynchronize");
            float ms = 0.0f;
            check(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
            return ms / 3.0;
        };
        std::vector<tddft_tuning_entry> rows;
        auto add = [&](const char *stage, int kind, int a, int b, double ms) {
            tddft_tuning_entry e{};
            std::strncpy(e.stage, stage, sizeof(e.stage) - 1);
            e.kind = kind;
            e.chi_chunk = a;
            e.phi_chunk = b;
            e.ms = ms;
            rows.push_back(e);
        };
        // response density: the per-tile kernels (when every tile fits them) and units of each cut
        {
            const bool units_possible = c->nv % 4 == 0 && build_density_chunks(c, I);
            int best = -1;
            double best_ms = 1e300;
            if (I.grid_tc) {
                I.dens_units = false;
                add("response_density", 0, 0, 0, time_it([&]() { density(c, I, I.bufP, k); }));
                best = (int)rows.size() - 1;
                best_ms = rows.back().ms;
            }
            if (units_possible) {
                const int cuts[][2] = {{320, 128}, {256, 128}, {192, 128}, {128, 128}, {320, 64}, {192, 64}, {128, 64}};
                for (const auto &cut : cuts) {
                    set_density_units(I, cut[0], cut[1]);
                    I.dens_units = true;
                    add("response_density", 1, cut[0], cut[1], time_it([&]() { density(c, I, I.bufP, k); }));
                    if (rows.back().ms < best_ms) {
                        best_ms = rows.back().ms;
                        best = (int)rows.size() - 1;
                    }
                }
            }
            if (best >= 0) {
                rows[best].chosen = 1;
                if (rows[best].kind == 1) {
                    set_density_units(I, rows[best].chi_chunk, rows[best].phi_chunk);
                    I.dens_units = true;
                } else {
                    I.dens_units = false;
                }
            }
        }
        // potential integrals: unit cuts (chi a multiple of 128, phi of 16)
        if (I.integrals_tc) {
            const int cuts[][2] = {{384, 128}, {256, 128}, {128, 128}, {384, 64}, {256, 64}, {128, 64}, {384, 32}};
            int best = -1;
            double best_ms = 1e300;
            for (const auto &cut : cuts) {
                if (!set_integrals_units(I, cut[0], cut[1])) continue;
                add("potential_integrals", 1, cut[0], cut[1], time_it([&]() { integrals(c, I, k); }));
                if (rows.back().ms < best_ms) {
                    best_ms = rows.back().ms;
                    best = (int)rows.size() - 1;
                }
            }
            if (best >= 0) {
                rows[best].chosen = 1;
                set_integrals_units(I, rows[best].chi_chunk, rows[best].phi_chunk);
            }
        }
        check_tc_error(c);
        const int n = std::min<int>(cap, (int)rows.size());
        for (int i = 0; i < n && out; ++i) out[i] = rows[i];
        if (count) *count = (int)rows.size();
        return TDDFT_OK;
    });
}

tddft_status tddft_wait_check(tddft_ctx *c) {
    if (!c) return TDDFT_E_INVALID;
    return guarded(c, [&]() -> tddft_status {
        tc_wait_probe(c->st);
        check_tc_error(c);   // throws TimeoutErr when the probe's wait expired, as it must
        c->err = "the bounded wait of the probe did not expire";
        return TDDFT_E_CUDA;
    });
}

tddft_status tddft_learned_dims(const tddft_ctx *c, int32_t *n_block, int32_t *n_feat) {
    if (!c) return TDDFT_E_INVALID;
    if (!c->uniform) {
        const_cast<tddft_ctx *>(c)->err = "the learned preconditioner needs equal function counts on every atom";
        return TDDFT_E_INVALID;
    }
    if (n_block) *n_block = 2 * c->nca * c->nva;
    if (n_feat) *n_feat = 2 * c->nca * c->nca + 2 * c->nva * c->nva + 1;
    return TDDFT_OK;
}

tddft_status tddft_set_mlp(tddft_ctx *c, tddft_mlp *m) {
    if (!c) return TDDFT_E_INVALID;
    c->mlp = m;
    return TDDFT_OK;
}

tddft_status tddft_samples(tddft_ctx *c, tddft_state *S, int64_t cap, float *X, float *Tg, float *Wt,
                           int64_t *count) {
    if (!c || !S || S->ctx != c || !X || !Tg || !Wt) return TDDFT_E_INVALID;
    return guarded(c, [&]() -> tddft_status {
        if (!c->uniform) throw InvalidArg{"the learned preconditioner needs equal function counts on every atom"};
        const long long rows = (long long)S->k * c->natoms * c->natoms;
        if (count) *count = rows;
        if (cap < rows) throw InvalidArg{"tddft_samples: cap smaller than k * natoms^2"};
        if (!is_device_ptr(X) || !is_device_ptr(Tg) || !is_device_ptr(Wt))
            throw InvalidArg{"tddft_samples: X, T and w must be device pointers"};
        return DISPATCH(c, ([&]() {
            Impl<T> &I = impl<T>(c);
            StateBufs<T> &B = bufs<T>(S);
            const int k = S->k, k2 = 2 * k, na = c->natoms;
            if (!S->evaluated) evaluate<T>(c, S);
            ensure_learned<T>(c, I, k);
            const T *h = search_gradient<T>(c, S);
            precondition<T>(c, S, h, B.z);
            if (c->trunc) mask_mul<T>(c->st, B.z, I.mask, c->len(), k2);
            learned_features<T>(c->st, h, k, na, c->nca, c->nva, c->nc, c->nv, I.lfc, I.lfv, I.ldist, X, I.ls);
            learned_targets<T>(c->st, B.z, h, I.ls, k, na, c->nca, c->nva, c->nc, c->nv, Tg, Wt);
            check(ctx_sync(c), "sync samples");
            return TDDFT_OK;
        })());
    });
}

tddft_status tddft_state_stats(const tddft_state *S, int32_t *iters, int32_t *fallbacks, int64_t *inner_iters) {
    if (!S) return TDDFT_E_INVALID;
    if (iters) *iters = S->it;
    if (fallbacks) *fallbacks = S->fallbacks;
    if (inner_iters) *inner_iters = S->inner_iters;
    return TDDFT_OK;
}

tddft_status tddft_pattern(const tddft_ctx *c, uint8_t *mask) {
    if (!c || !mask) return TDDFT_E_INVALID;
    std::memcpy(mask, c->amask.data(), c->amask.size());
    return TDDFT_OK;
}

}  // extern "C"
