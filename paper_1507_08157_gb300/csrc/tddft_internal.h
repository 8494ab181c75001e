// Internal declarations shared by the translation units of libtddft.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <new>
#include <string>
#include <vector>

namespace tddft {

constexpr int TILE = 8;                  // grid tile edge (points); a tile holds 512 points
constexpr int TILE_PTS = TILE * TILE * TILE;

struct CudaError {
    cudaError_t code;
    std::string where;
};

// owning list of device allocations (freed on release or destruction)
struct Mem {
    std::vector<void *> ptrs;
    template <typename T>
    T *alloc(size_t n) {
        void *p = nullptr;
        if (n == 0) n = 1;
        cudaError_t e = cudaMalloc(&p, n * sizeof(T));
        if (e != cudaSuccess) {
            cudaGetLastError();
            throw std::bad_alloc();
        }
        ptrs.push_back(p);
        return static_cast<T *>(p);
    }
    void release() {
        for (void *p : ptrs) cudaFree(p);
        ptrs.clear();
    }
    ~Mem() { release(); }
};

void check(cudaError_t e, const char *where);   // throws CudaError on failure
void check_launch(const char *where);           // cudaGetLastError after a launch

// ---- per-stage launch timing (CUDA events on the launching stream) -------------------------------
enum Stage {
    ST_GEMM = 0, ST_DENSITY, ST_INTEGRALS, ST_FFT, ST_TRACE, ST_VECTOR, ST_SMALL, ST_COUNT
};
const char *stage_name(int s);

struct Profiler;                        // defined in profile.cu
Profiler *&active_profiler();           // thread-local; null when profiling is off

// Limit of every bounded wait inside the tensor-core kernels, in clock64 ticks: thread-local, set
// for the duration of a call from the context's options (tddft_options.spin_limit_cycles) and read
// by the launchers, which pass it to the kernels.
constexpr long long DEFAULT_WAIT_LIMIT = 4000000000LL;   // about 2 s at 2 GHz
long long &active_wait_limit();

// Records an event pair around one launch when a profiler is active; `flops` and `bytes` are the
// algorithmic counts of the launch.
struct ProfScope {
    Profiler *p;
    cudaStream_t st;
    int stage;
    double flops, bytes;
    void *ev0;
    ProfScope(cudaStream_t st, int stage, double flops, double bytes);
    ~ProfScope();
};

// Per-tile lists of the functions whose support touches the tile, and their values on the
// tile's 512 points (local index (lx*8 + ly)*8 + lz; zero outside the support and the grid).
template <typename T>
struct TileSet {
    int ntiles = 0;
    int max_per_tile = 0;
    const int *off = nullptr;     // [ntiles+1] slot offsets
    const int *ids = nullptr;     // [slots] function index
    const T *val = nullptr;       // [slots][512]
};

// One unit of the tensor-core integrals launches: a grid tile with a chunk of its chi slots (at
// most three 128-row blocks) and a chunk of its phi slots (at most 128). A tile whose lists fit is
// one unit; a denser tile is cut into several units, each adding its part into the output.
struct VTile {
    int t;        // grid tile (whose 512 points the unit sums over)
    int c0, nc;   // first chi slot, count
    int p0, np;   // first phi slot, count
    int pad;
};

// One unit of the tensor-core density on dense tiles: a chunk of a tile's chi slots (at most five
// blocks of 64) and of its phi slots (at most 128, in chunks of 32), with the indices of their first
// 64-wide chi chunk and 32-wide phi chunk in the chunked point-major tables.
struct DUnit {
    int t;        // grid tile
    int c0, nc;   // first chi slot, count
    int p0, np;   // first phi slot, count
    int cch;      // first chi chunk
    int pch;      // first phi chunk
    int pad;
};

struct GridShape {
    int n;          // points per side
    int nt;         // tiles per side = ceil(n / 8)
    double cell;
    double dV;
    double pair_points = 0.0;   // sum over grid points of (#chi nonzero) * (#phi nonzero)
    double table_values = 0.0;  // nonzero tabulated values of chi and phi
};

// ---------------------------------------------------------------------------------------------
// float32 matrices that stay fixed while registered: the tensor-core GEMM keeps their split
// (hi/lo, K-major) copies; unregister before freeing them
void tc_register_constant(const float *p);
void tc_unregister_constant(const float *p);

// dense GEMM, row-major: C[b] = alpha * op(A[b]) op(B[b]) + beta * C[b]. approx: a float32
// product on the tensor cores may take one TF32 MMA instead of the three-term split (about 1e-3
// relative error; for operands whose errors the method tolerates, such as a preconditioner's)
template <typename T>
void gemm(cudaStream_t st, bool ta, bool tb, int M, int N, int K, T alpha, const T *A, int lda,
          long long sA, const T *B, int ldb, long long sB, T beta, T *C, int ldc, long long sC,
          int batch, bool approx = false);

// ---------------------------------------------------------------------------------------------
// grid work
template <typename T>
void response_density(cudaStream_t st, const GridShape &g, const TileSet<T> &chi,
                      const TileSet<T> &phi, int nphi, const T *P, long long sP, int k, T *rho);

template <typename T>
void potential_integrals(cudaStream_t st, const GridShape &g, const TileSet<T> &chi,
                         const TileSet<T> &phi, int nchi, int nphi, const T *V, int k, T *out);

// V_s = v_H[rho_s] + fxc * rho_s for k states; work: complex buffer of ceil(k/2) * n^3
template <typename T>
void hartree_fxc(cudaStream_t st, const GridShape &g, const T *rho, const T *fxc, int k, T *V,
                 void *work);

void fxc_lda(cudaStream_t st, const double *n0, double *fxc, long long npts);

bool fft_size_ok(int n);

// ---------------------------------------------------------------------------------------------
// solver primitives
// G[i][j] = sum_e X_i[e] * Y_j[e], i < nx, j < ny (float64 result; fixed reduction order).
// X_i = X + i*sx, Y_j = Y + j*sy. scratch: >= gram_scratch_doubles(nx, ny) doubles.
long long gram_scratch_doubles(int nx, int ny);
template <typename T>
void gram(cudaStream_t st, const T *X, long long sx, int nx, const T *Y, long long sy, int ny,
          long long len, double *G, double *scratch);
// several Gram matrices of one X at once: Y[q] (q < nset <= 4) holds `per` rows of stride sy and
// G[q] receives [nx][per]; X is read once for all of them
template <typename T>
void gram_multi(cudaStream_t st, const T *X, long long sx, int nx, int nset, const T *const *Y, long long sy,
                int per, long long len, double *const *G, double *scratch);

// out_i = beta * out_i + sum_j C[i*ldc + j] * in_j (C float64 on the device), out != in.
template <typename T>
void combine(cudaStream_t st, const double *C, int ldc, int nout, int nin, const T *in,
             long long sin, T *out, long long sout, long long len, bool accumulate);

// X_b[e] *= mask[e % len] for b < nb
template <typename T>
void mask_mul(cudaStream_t st, T *X, const T *mask, long long len, int nb);

template <typename Tin, typename Tout>
void convert(cudaStream_t st, const Tin *in, Tout *out, long long n);

// y_b += sgn * a[b * a_stride] * x_b over nb blocks of len; a on the device (float64)
template <typename T>
void axpy_dev(cudaStream_t st, const double *a, int a_stride, double sgn, T *y, const T *x,
              long long len, int nb);

// ---------------------------------------------------------------------------------------------
// small float64 linear algebra on the device (one thread; k <= KMAX)
constexpr int KMAX = 16;

// Status word bits written by the small kernels
enum { DEV_OK = 0, DEV_BREAKDOWN = 1, DEV_NAN = 2, DEV_NAN_EVAL = 3, DEV_NAN_LINE = 4, DEV_NAN_INIT = 5 };

}  // namespace tddft
