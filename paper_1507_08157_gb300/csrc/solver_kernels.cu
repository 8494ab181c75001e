// Solver primitives: trace products with float64 accumulation in a fixed order, linear
// combinations of state matrices, masks, and the small float64 algebra of the PCG step
// (paper Sec. III C): Q matrix, sum-functional line step, sign flip + Gram-Schmidt in the metric
// of Eq. ortho, subspace eigenvalues.
#include "solver_kernels.h"

#include <algorithm>
#include <cmath>
#include <cstdlib>

namespace tddft {

namespace {

constexpr int GCH = 64;        // elements per staged chunk in the trace kernels
constexpr int GMAXQ = 8;       // pair slots per thread (pairs <= 2048)
constexpr int GBLOCKS = 304;   // 2 blocks per SM on 152 SMs

// ------------------------------------------------------------------------------------------------
// G[i][j] = sum_e X_i[e] Y_j[e] (or only i == j when diag). float32 inputs: 64-term float32
// partial sums per chunk (products of float32 values are exact in the float64 accumulator's
// range but not in float32; the chunk sums carry ~64 ulp), accumulated in float64 across chunks.
template <typename T>
__global__ void __launch_bounds__(256) gram_partial(const T *__restrict__ X, long long sx, int nx,
                                                    const T *__restrict__ Y, long long sy, int ny,
                                                    long long len, bool diag,
                                                    double *__restrict__ partial) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *xs = reinterpret_cast<T *>(smem_raw);   // [nx][GCH+1]
    T *ys = xs + nx * (GCH + 1);               // [ny][GCH+1]
    const int pairs = diag ? nx : nx * ny;
    double acc[GMAXQ];
#pragma unroll
    for (int q = 0; q < GMAXQ; ++q) acc[q] = 0.0;
    const long long nchunks = (len + GCH - 1) / GCH;
    for (long long c = blockIdx.x; c < nchunks; c += gridDim.x) {
        const long long e0 = c * GCH;
        for (int i = threadIdx.x; i < nx * GCH; i += blockDim.x) {
            const int r = i / GCH, e = i - r * GCH;
            xs[r * (GCH + 1) + e] = (e0 + e < len) ? X[r * sx + e0 + e] : T(0);
        }
        for (int i = threadIdx.x; i < ny * GCH; i += blockDim.x) {
            const int r = i / GCH, e = i - r * GCH;
            ys[r * (GCH + 1) + e] = (e0 + e < len) ? Y[r * sy + e0 + e] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < GMAXQ; ++q) {
            const int p = threadIdx.x + 256 * q;
            if (p >= pairs) break;
            const int i = diag ? p : p / ny, j = diag ? p : p - (p / ny) * ny;
            const T *xr = xs + i * (GCH + 1);
            const T *yr = ys + j * (GCH + 1);
            T part = T(0);
#pragma unroll 16
            for (int e = 0; e < GCH; ++e) part = fma(xr[e], yr[e], part);
            acc[q] += (double)part;
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < GMAXQ; ++q) {
        const int p = threadIdx.x + 256 * q;
        if (p < pairs) partial[(long long)blockIdx.x * pairs + p] = acc[q];
    }
}

__global__ void gram_final(const double *__restrict__ partial, int nblocks, int pairs,
                           double *__restrict__ G) {
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < pairs; p += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += partial[(long long)b * pairs + p];
        G[p] = s;
    }
}

template <typename T>
void gram_impl(cudaStream_t st, const T *X, long long sx, int nx, const T *Y, long long sy, int ny,
               long long len, bool diag, double *G, double *scratch) {
    const int pairs = diag ? nx : nx * ny;
    if (pairs <= 0) return;
    if (pairs > 256 * GMAXQ || nx > 64 || ny > 64)
        throw CudaError{cudaErrorInvalidValue, "gram: too many pairs"};
    const long long nchunks = (len + GCH - 1) / GCH;
    const int nb = (int)(nchunks < GBLOCKS ? (nchunks > 0 ? nchunks : 1) : GBLOCKS);
    const size_t sm = sizeof(T) * (size_t)(nx + ny) * (GCH + 1);
    ProfScope ps(st, ST_TRACE, 2.0 * pairs * (double)len, sizeof(T) * (double)(nx + ny) * len);
    static bool attr = false;
    if (!attr) {
        check(cudaFuncSetAttribute(gram_partial<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)(sizeof(T) * 128 * (GCH + 1))),
              "attr gram");
        attr = true;
    }
    gram_partial<T><<<nb, 256, sm, st>>>(X, sx, nx, Y, sy, ny, len, diag, scratch);
    check_launch("gram_partial");
    gram_final<<<(pairs + 255) / 256, 256, 0, st>>>(scratch, nb, pairs, G);
    check_launch("gram_final");
}

// ------------------------------------------------------------------------------------------------
// Register-tiled trace products. Block (x, y): element slice x, pair tile y of 8 x 8 (i, j);
// each thread accumulates its 64 products over a strided run of elements (float32 products
// summed in T per run of at most RUN elements, then in float64), the block reduces in float64
// in a fixed order and writes one partial per pair; gram_final sums the partials over slices.
constexpr int RUN = 32;

template <typename T>
__global__ void __launch_bounds__(256) gram_tiled(const T *__restrict__ X, long long sx, int nx,
                                                  const T *__restrict__ Y, long long sy, int ny,
                                                  long long len, int tiles_j, double *__restrict__ partial,
                                                  int pairs) {
    __shared__ double red[8][8][33];
    const int ti = blockIdx.y / tiles_j, tj = blockIdx.y - ti * tiles_j;
    const int i0 = ti * 8, j0 = tj * 8;
    double acc[8][8];
    T run[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] = 0.0, run[a][b] = T(0);
    const long long stride = (long long)gridDim.x * blockDim.x;
    int cnt = 0;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len; e += stride) {
        T xv[8], yv[8];
#pragma unroll
        for (int a = 0; a < 8; ++a) xv[a] = (i0 + a < nx) ? X[(i0 + a) * sx + e] : T(0);
#pragma unroll
        for (int b = 0; b < 8; ++b) yv[b] = (j0 + b < ny) ? Y[(j0 + b) * sy + e] : T(0);
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int b = 0; b < 8; ++b) run[a][b] = fma(xv[a], yv[b], run[a][b]);
        if (++cnt == RUN) {
#pragma unroll
            for (int a = 0; a < 8; ++a)
#pragma unroll
                for (int b = 0; b < 8; ++b) acc[a][b] += (double)run[a][b], run[a][b] = T(0);
            cnt = 0;
        }
    }
    // warp reduction (fixed butterfly order), then across the 8 warps through shared memory
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) {
            double v = acc[a][b] + (double)run[a][b];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[a][b][warp] = v;
        }
    __syncthreads();
    if (threadIdx.x < 64) {
        const int a = threadIdx.x >> 3, b = threadIdx.x & 7;
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += red[a][b][w];
        const int i = i0 + a, j = j0 + b;
        if (i < nx && j < ny) partial[(long long)blockIdx.x * pairs + i * ny + j] = v;
    }
}

// d_i = sum_e X_i[e] Y_i[e]: one row per blockIdx.y, float32 runs of RUN then float64
template <typename T>
__global__ void __launch_bounds__(256) dots_kernel(const T *__restrict__ X, long long sx, const T *__restrict__ Y,
                                                   long long sy, long long len, int n, double *__restrict__ partial) {
    __shared__ double red[8];
    const int i = blockIdx.y;
    const T *x = X + i * sx;
    const T *y = Y + i * sy;
    double acc = 0.0;
    T run = T(0);
    int cnt = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len; e += stride) {
        run = fma(x[e], y[e], run);
        if (++cnt == RUN) {
            acc += (double)run;
            run = T(0);
            cnt = 0;
        }
    }
    acc += (double)run;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += red[w];
        partial[(long long)blockIdx.x * n + i] = v;
    }
}

// ------------------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) combine_kernel(const double *__restrict__ C, int ldc, int nout,
                                                      int nin, const T *__restrict__ in,
                                                      long long sin, T *__restrict__ out,
                                                      long long sout, long long len, bool accumulate) {
    __shared__ T Cs[32 * 32];
    // every slot the product loop reads is written (zero past nin): stale shared memory from an
    // earlier kernel may hold NaN patterns, and NaN * 0 is NaN
    for (int i = threadIdx.x; i < nout * 32; i += blockDim.x) {
        const int r = i >> 5, c = i & 31;
        Cs[i] = c < nin ? T(C[r * ldc + c]) : T(0);
    }
    __syncthreads();
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len;
         e += (long long)gridDim.x * blockDim.x) {
        T x[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) x[j] = j < nin ? in[j * sin + e] : T(0);
        for (int i = 0; i < nout; ++i) {
            T s = accumulate ? out[i * sout + e] : T(0);
#pragma unroll
            for (int j = 0; j < 32; ++j) s = fma(Cs[i * 32 + j], x[j], s);
            out[i * sout + e] = s;
        }
    }
}

template <typename T>
__global__ void mask_kernel(T *__restrict__ X, const T *__restrict__ mask, long long len, int nb) {
    const long long tot = len * nb;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x)
        X[i] *= mask[i % len];
}

template <typename Tin, typename Tout>
__global__ void convert_kernel(const Tin *__restrict__ in, Tout *__restrict__ out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = Tout(in[i]);
}

template <typename T>
__global__ void axpy_dev_kernel(const double *__restrict__ a, int a_stride, double sgn,
                                T *__restrict__ y, const T *__restrict__ x, long long len, int nb) {
    const long long tot = len * nb;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(i / len);
        y[i] = fma(T(sgn * a[b * a_stride]), x[i], y[i]);
    }
}

// out = -z + beta * prev (beta on the device)
template <typename T>
__global__ void direction_kernel(T *__restrict__ out, const T *__restrict__ z,
                                 const T *__restrict__ prev, const double *__restrict__ beta,
                                 long long n) {
    const T b = T(*beta);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = b != T(0) ? fma(b, prev[i], -z[i]) : -z[i];
}

int grid_for(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < 4 * 152 ? (b > 0 ? b : 1) : 4 * 152);
}

// ------------------------------------------------------------------------------------------------
// small float64 algebra (single thread)
__device__ bool chol_solve(int k, const double *M, const double *B, double *X, double *L) {
    // L L^T = M; X = M^-1 B (B, X: k x k)
    for (int i = 0; i < k; ++i) {
        for (int j = 0; j <= i; ++j) {
            double s = M[i * k + j];
            for (int p = 0; p < j; ++p) s -= L[i * k + p] * L[j * k + p];
            if (i == j) {
                if (!(s > 0.0)) return false;
                L[i * k + i] = sqrt(s);
            } else {
                L[i * k + j] = s / L[j * k + j];
            }
        }
    }
    for (int c = 0; c < k; ++c) {
        for (int i = 0; i < k; ++i) {   // forward
            double s = B[i * k + c];
            for (int p = 0; p < i; ++p) s -= L[i * k + p] * X[p * k + c];
            X[i * k + c] = s / L[i * k + i];
        }
        for (int i = k - 1; i >= 0; --i) {   // backward with L^T
            double s = X[i * k + c];
            for (int p = i + 1; p < k; ++p) s -= L[p * k + i] * X[p * k + c];
            X[i * k + c] = s / L[i * k + i];
        }
    }
    return true;
}

struct LineBlocks {
    double N0[KMAX * KMAX], N1[KMAX * KMAX], N2[KMAX * KMAX];
    double M0[KMAX * KMAX], M1[KMAX * KMAX], M2[KMAX * KMAX];
};

struct Scratch {
    double M[KMAX * KMAX], N[KMAX * KMAX], dM[KMAX * KMAX], dN[KMAX * KMAX];
    double W[KMAX * KMAX], X[KMAX * KMAX], Z[KMAX * KMAX], T[KMAX * KMAX], L[KMAX * KMAX];
};

// Omega(lam) = Tr[M^-1 N]/2 and its derivative; returns false when M is not positive definite
__device__ bool sum_functional(int k, const LineBlocks &lb, double lam, double *f, double *d,
                               Scratch &s) {
    const int kk = k * k;
    for (int i = 0; i < kk; ++i) {
        s.M[i] = lb.M0[i] + lam * lb.M1[i] + lam * lam * lb.M2[i];
        s.N[i] = lb.N0[i] + lam * lb.N1[i] + lam * lam * lb.N2[i];
        s.dM[i] = lb.M1[i] + 2.0 * lam * lb.M2[i];
        s.dN[i] = lb.N1[i] + 2.0 * lam * lb.N2[i];
    }
    if (!chol_solve(k, s.M, s.N, s.W, s.L)) return false;
    chol_solve(k, s.M, s.dN, s.X, s.L);
    for (int i = 0; i < k; ++i)          // T = dM W
        for (int j = 0; j < k; ++j) {
            double acc = 0.0;
            for (int p = 0; p < k; ++p) acc += s.dM[i * k + p] * s.W[p * k + j];
            s.T[i * k + j] = acc;
        }
    chol_solve(k, s.M, s.T, s.Z, s.L);
    double tw = 0.0, tx = 0.0, tz = 0.0;
    for (int i = 0; i < k; ++i) {
        tw += s.W[i * k + i];
        tx += s.X[i * k + i];
        tz += s.Z[i * k + i];
    }
    *f = 0.5 * tw;
    *d = 0.5 * (tx - tz);
    return true;
}

__device__ double line_step(int k, const LineBlocks &lb, Scratch &s) {
    double f0, d0;
    if (!sum_functional(k, lb, 0.0, &f0, &d0, s) || !isfinite(d0) || d0 >= 0.0) return 0.0;
    // Newton estimate with M0 = I: h0 = Tr[2 N2 - 2 M1 N1 + 2 M1 M1 N0 - 2 M2 N0] / 2
    double h0 = 0.0;
    for (int i = 0; i < k; ++i) {
        double t = 2.0 * lb.N2[i * k + i];
        for (int p = 0; p < k; ++p) {
            t -= 2.0 * lb.M1[i * k + p] * lb.N1[p * k + i];
            t -= 2.0 * lb.M2[i * k + p] * lb.N0[p * k + i];
            double m1m1 = 0.0;
            for (int q = 0; q < k; ++q) m1m1 += lb.M1[i * k + q] * lb.M1[q * k + p];
            t += 2.0 * m1m1 * lb.N0[p * k + i];
        }
        h0 += 0.5 * t;
    }
    double hi = (h0 > 0.0 && isfinite(h0)) ? -d0 / h0 : 1.0;
    double lo = 0.0, dlo = d0, dhi = 0.0, f, d;
    // bracket: dOmega < 0 at lo, >= 0 (or M not positive definite) at hi
    int it = 0;
    for (; it < 60; ++it) {
        if (!sum_functional(k, lb, hi, &f, &d, s)) d = INFINITY;
        if (d >= 0.0) break;
        lo = hi;
        dlo = d;
        hi = 2.0 * hi;
    }
    dhi = d;
    // past the positive-definite region: bisect until dOmega is finite at hi
    for (int b = 0; b < 200 && !isfinite(dhi); ++b) {
        const double mid = 0.5 * (lo + hi);
        if (!sum_functional(k, lb, mid, &f, &d, s)) d = INFINITY;
        if (d < 0.0) { lo = mid; dlo = d; }
        else { hi = mid; dhi = d; }
    }
    // Illinois regula falsi on dOmega(lambda) inside [lo, hi], to machine precision
    int side = 0;
    for (int r = 0; r < 100; ++r) {
        if (!(hi - lo > 4e-16 * hi)) break;
        double x = (isfinite(dhi) && dhi != dlo) ? hi - dhi * (hi - lo) / (dhi - dlo) : 0.5 * (lo + hi);
        if (!(x > lo && x < hi)) x = 0.5 * (lo + hi);
        if (!sum_functional(k, lb, x, &f, &d, s)) d = INFINITY;
        if (d == 0.0) return x;
        if (d < 0.0) {
            lo = x;
            dlo = d;
            if (side == -1) dhi *= 0.5;
            side = -1;
        } else {
            hi = x;
            dhi = d;
            if (side == +1) dlo *= 0.5;
            side = +1;
        }
    }
    return 0.5 * (lo + hi);
}

// classical Gram-Schmidt twice on coefficient vectors; rows of C are the new vectors
__device__ bool gram_schmidt(int k, const double *Mg, const int *order, double *C) {
    for (int i = 0; i < k * k; ++i) C[i] = 0.0;
    for (int a = 0; a < k; ++a) {
        const int i = order[a];
        double v[KMAX];
        for (int j = 0; j < k; ++j) v[j] = (j == i) ? 1.0 : 0.0;
        for (int pass = 0; pass < 2; ++pass) {
            double coef[KMAX];
            for (int b = 0; b < a; ++b) {
                const int j = order[b];
                double s = 0.0;
                for (int p = 0; p < k; ++p)
                    for (int q = 0; q < k; ++q) s += v[p] * Mg[p * k + q] * C[j * k + q];
                coef[b] = s;
            }
            for (int b = 0; b < a; ++b) {
                const int j = order[b];
                for (int p = 0; p < k; ++p) v[p] -= coef[b] * C[j * k + p];
            }
        }
        double nrm = 0.0;
        for (int p = 0; p < k; ++p)
            for (int q = 0; q < k; ++q) nrm += v[p] * Mg[p * k + q] * v[q];
        const double ref = fabs(Mg[i * k + i]) > 1.0 ? fabs(Mg[i * k + i]) : 1.0;
        if (!isfinite(nrm) || nrm <= 1e-12 * ref) return false;
        const double inv = 1.0 / sqrt(nrm);
        for (int p = 0; p < k; ++p) C[i * k + p] = v[p] * inv;
    }
    return true;
}

// cyclic Jacobi eigenvalues of a symmetric k x k matrix, ascending
__device__ void jacobi_eigenvalues(int k, const double *A, double *w) {
    double a[KMAX * KMAX];
    for (int i = 0; i < k * k; ++i) a[i] = A[i];
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) {
                tot += a[i * k + j] * a[i * k + j];
                if (i != j) off += a[i * k + j] * a[i * k + j];
            }
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < k; ++p)
            for (int q = p + 1; q < k; ++q) {
                const double apq = a[p * k + q];
                if (apq == 0.0) continue;
                const double theta = (a[q * k + q] - a[p * k + p]) / (2.0 * apq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int r = 0; r < k; ++r) {   // columns p, q
                    const double arp = a[r * k + p], arq = a[r * k + q];
                    a[r * k + p] = c * arp - s * arq;
                    a[r * k + q] = s * arp + c * arq;
                }
                for (int r = 0; r < k; ++r) {   // rows p, q
                    const double apr = a[p * k + r], aqr = a[q * k + r];
                    a[p * k + r] = c * apr - s * aqr;
                    a[q * k + r] = s * apr + c * aqr;
                }
            }
    }
    for (int i = 0; i < k; ++i) w[i] = a[i * k + i];
    for (int i = 1; i < k; ++i) {   // insertion sort
        const double x = w[i];
        int j = i - 1;
        while (j >= 0 && w[j] > x) {
            w[j + 1] = w[j];
            --j;
        }
        w[j + 1] = x;
    }
}

// ---- kernels ----------------------------------------------------------------------------------

// From A[x][y] = <cov(P_x), f_y> (x, y over p_0..p_k-1, q_0..q_k-1): Q_ij = (A[j][i] +
// A[k+j][k+i]) / 2 (Sec. III C) and the gradient coefficients on P:
// g_p,i = f_p,i - sum_j Q_ij P_q,j ; g_q,i = f_q,i - sum_j Q_ij P_p,j  (coef[2k][2k]).
__global__ void make_q_kernel(int k, const double *A, double *Q, double *coef) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int k2 = 2 * k;
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) Q[i * k + j] = 0.5 * (A[j * k2 + i] + A[(k + j) * k2 + k + i]);
    for (int i = 0; i < k2 * k2; ++i) coef[i] = 0.0;
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) {
            coef[i * k2 + k + j] = -Q[i * k + j];          // g_p,i  <-  P_q,j
            coef[(k + i) * k2 + j] = -Q[i * k + j];        // g_q,i  <-  P_p,j
        }
}

// residuals and Ritz values: r_i = sqrt(d_p,i + d_q,i); omega = eig(sym Q); out = [omega, r]
__global__ void eval_finish_kernel(int k, const double *Q, const double *d, double *out,
                                   int *status) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double S[KMAX * KMAX];
    bool bad = false;
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) {
            S[i * k + j] = 0.5 * (Q[i * k + j] + Q[j * k + i]);
            if (!isfinite(S[i * k + j])) bad = true;
        }
    for (int i = 0; i < k; ++i) {
        const double r2 = d[i] + d[k + i];
        out[k + i] = sqrt(r2 > 0.0 ? r2 : 0.0);
        if (!isfinite(r2)) bad = true;
    }
    if (bad) {
        *status = DEV_NAN_EVAL;
        for (int i = 0; i < k; ++i) out[i] = NAN;
        return;
    }
    jacobi_eigenvalues(k, S, out);
}

// Polak-Ribiere coefficient over the whole set (sums of the 2k dot products)
//   sc[0] = gz (this step), sc[1] = gz_prev, sc[2] = beta, sc[3] = slope
__global__ void conj_kernel(int k2, const double *gz_d, const double *gzp_d, const double *gd_d,
                            int restart, const double *flip, double *sc) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    if (*flip != 0.0) restart = 1;
    double gz = 0.0, gzp = 0.0, gd = 0.0;
    for (int i = 0; i < k2; ++i) {
        gz += gz_d[i];
        gzp += gzp_d[i];
        gd += gd_d[i];
    }
    double beta = 0.0;
    if (!restart && sc[1] != 0.0) {
        beta = (gz - gzp) / sc[1];
        if (!(beta > 0.0)) beta = 0.0;
    }
    // slope along d = -z + beta d_prev: -gz + beta <g, d_prev>
    if (beta > 0.0 && -gz + beta * gd >= 0.0) beta = 0.0;
    sc[0] = gz;
    sc[1] = gz;
    sc[2] = beta;
    sc[3] = -gz + beta * gd;
}

// Line step and re-orthonormalisation.
//  A  = gram(cov P, f), BDf = gram(cov D, f), CDfD = gram(cov D, fD)    [2k x 2k]
//  PP = gram(cov P, P), PD = gram(cov P, D), DP = gram(cov D, P), DD = gram(cov D, D)
// Outputs: lam[0]; Cp, Cq [k][k] combination coefficients (sign flips folded into Cq);
// flip_any -> sc_flip[0]; status.

// single-thread version of the line step and re-orthonormalisation
__global__ void line_gs_kernel(int k, const double *A, const double *BDf, const double *CDfD,
                               const double *PP, const double *PD, const double *DP,
                               const double *DD, const double *Q, double *lam, double *Cp,
                               double *Cq, double *sc_flip, int *status) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int k2 = 2 * k;
    LineBlocks lb;
    Scratch s;
    double T0[KMAX * KMAX], T1[KMAX * KMAX], T2[KMAX * KMAX];
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) {
            const int e = i * k + j;
            const double n0ij = A[i * k2 + j] + A[(k + i) * k2 + k + j];
            const double n0ji = A[j * k2 + i] + A[(k + j) * k2 + k + i];
            lb.N0[e] = 0.5 * (n0ij + n0ji);
            const double efij = BDf[i * k2 + j] + BDf[(k + i) * k2 + k + j];
            const double efji = BDf[j * k2 + i] + BDf[(k + j) * k2 + k + i];
            lb.N1[e] = efij + efji;
            const double n2ij = CDfD[i * k2 + j] + CDfD[(k + i) * k2 + k + j];
            const double n2ji = CDfD[j * k2 + i] + CDfD[(k + j) * k2 + k + i];
            lb.N2[e] = 0.5 * (n2ij + n2ji);
            T0[e] = PP[i * k2 + k + j];
            T1[e] = PD[i * k2 + k + j] + DP[i * k2 + k + j];
            T2[e] = DD[i * k2 + k + j];
        }
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) {
            const int e = i * k + j;
            lb.M0[e] = 0.5 * (T0[e] + T0[j * k + i]);
            lb.M1[e] = 0.5 * (T1[e] + T1[j * k + i]);
            lb.M2[e] = 0.5 * (T2[e] + T2[j * k + i]);
        }
    for (int e = 0; e < k * k; ++e)
        if (!isfinite(lb.N0[e]) || !isfinite(lb.N1[e]) || !isfinite(lb.N2[e]) || !isfinite(lb.M1[e]) ||
            !isfinite(lb.M2[e])) {
            *status = DEV_NAN_LINE;
            return;
        }
    const double l = line_step(k, lb, s);
    *lam = l;
    double Tm[KMAX * KMAX], Mg[KMAX * KMAX], sg[KMAX];
    for (int i = 0; i < k * k; ++i) Tm[i] = T0[i] + l * T1[i] + l * l * T2[i];
    int any = 0;
    for (int i = 0; i < k; ++i) {
        sg[i] = Tm[i * k + i] < 0.0 ? -1.0 : 1.0;
        if (sg[i] < 0.0) any = 1;
    }
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) Mg[i * k + j] = 0.5 * (Tm[i * k + j] * sg[j] + Tm[j * k + i] * sg[i]);
    int order[KMAX];
    for (int i = 0; i < k; ++i) order[i] = i;
    for (int i = 1; i < k; ++i) {
        const int x = order[i];
        int j = i - 1;
        while (j >= 0 && Q[order[j] * k + order[j]] > Q[x * k + x]) {
            order[j + 1] = order[j];
            --j;
        }
        order[j + 1] = x;
    }
    if (!gram_schmidt(k, Mg, order, Cp)) {
        *status = DEV_BREAKDOWN;
        return;
    }
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) Cq[i * k + j] = Cp[i * k + j] * sg[j];
    *sc_flip = any ? 1.0 : 0.0;
}

// initial orthonormalisation: T0 from PP only, identity order
__global__ void init_gs_kernel(int k, const double *PP, double *Cp, double *Cq, int *status) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int k2 = 2 * k;
    double sg[KMAX], Mg[KMAX * KMAX];
    for (int i = 0; i < k; ++i) sg[i] = PP[i * k2 + k + i] < 0.0 ? -1.0 : 1.0;
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) {
            const double tij = PP[i * k2 + k + j] * sg[j], tji = PP[j * k2 + k + i] * sg[i];
            Mg[i * k + j] = 0.5 * (tij + tji);
            if (!isfinite(Mg[i * k + j])) {
                *status = DEV_NAN_INIT;
                return;
            }
        }
    int order[KMAX];
    for (int i = 0; i < k; ++i) order[i] = i;
    if (!gram_schmidt(k, Mg, order, Cp)) {
        *status = DEV_BREAKDOWN;
        return;
    }
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) Cq[i * k + j] = Cp[i * k + j] * sg[j];
}

// inner CG scalars for 2k systems. phase 0: alpha = rr / pLp for active systems (0 otherwise);
// phase 1: beta = rr_new / rr, rr <- rr_new, active <- still above tolerance; counts active.
__global__ void cg_scalars_kernel(int n, int phase, double tol, const double *pLp,
                                  const double *rr_new, double *rr, const double *r0, double *alpha,
                                  double *beta, int *active, int *n_active) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int cnt = 0;
    for (int i = 0; i < n; ++i) {
        if (phase == 0) {
            const bool go = active[i] && pLp[i] > 0.0 && isfinite(pLp[i]);
            if (!go) active[i] = 0;
            alpha[i] = go ? rr[i] / pLp[i] : 0.0;
        } else {
            const double b = (active[i] && rr[i] != 0.0) ? rr_new[i] / rr[i] : 0.0;
            beta[i] = b;
            if (active[i]) {
                rr[i] = rr_new[i];
                if (!(sqrt(rr_new[i] > 0.0 ? rr_new[i] : 0.0) > tol * r0[i])) active[i] = 0;
            }
            cnt += active[i];
        }
    }
    if (phase == 1) *n_active = cnt;
}

__global__ void cg_init_kernel(int n, double tol, const double *rr0, double *rr, double *r0,
                               int *active, int *n_active) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int cnt = 0;
    for (int i = 0; i < n; ++i) {
        rr[i] = rr0[i];
        r0[i] = sqrt(rr0[i] > 0.0 ? rr0[i] : 0.0);
        active[i] = (r0[i] > 0.0 && isfinite(r0[i])) ? 1 : 0;
        cnt += active[i];
    }
    *n_active = cnt;
}

// p <- r + beta p for each system (beta on the device)
template <typename T>
__global__ void cg_dir_kernel(T *__restrict__ p, const T *__restrict__ r,
                              const double *__restrict__ beta, long long len, int nb) {
    const long long tot = len * nb;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(i / len);
        p[i] = fma(T(beta[b]), p[i], r[i]);
    }
}

// Ritz pairs of Q and the pairing errors: rotated halves |<p, f_p>_a - omega_a|,
// |<q, f_q>_a - omega_a| from the p-part and q-part matrices of A.
__global__ void subspace_kernel(int k, const double *A, double *omega, double *pairing) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int k2 = 2 * k;
    double Q[KMAX * KMAX], Ap[KMAX * KMAX], Aq[KMAX * KMAX], V[KMAX * KMAX];
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) {
            Ap[i * k + j] = 0.5 * (A[i * k2 + j] + A[j * k2 + i]);                    // <p_i, f_p,j> sym
            Aq[i * k + j] = 0.5 * (A[(k + i) * k2 + k + j] + A[(k + j) * k2 + k + i]);
            Q[i * k + j] = 0.5 * (Ap[i * k + j] + Aq[i * k + j]);
        }
    // Jacobi with eigenvectors
    double a[KMAX * KMAX];
    for (int i = 0; i < k * k; ++i) a[i] = Q[i];
    for (int i = 0; i < k; ++i)
        for (int j = 0; j < k; ++j) V[i * k + j] = i == j ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0, tot = 0.0;
        for (int i = 0; i < k * k; ++i) tot += a[i] * a[i];
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j)
                if (i != j) off += a[i * k + j] * a[i * k + j];
        if (off <= 1e-30 * tot || off == 0.0) break;
        for (int p = 0; p < k; ++p)
            for (int q = p + 1; q < k; ++q) {
                const double apq = a[p * k + q];
                if (apq == 0.0) continue;
                const double theta = (a[q * k + q] - a[p * k + p]) / (2.0 * apq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                for (int r = 0; r < k; ++r) {
                    const double arp = a[r * k + p], arq = a[r * k + q];
                    a[r * k + p] = c * arp - s * arq;
                    a[r * k + q] = s * arp + c * arq;
                    const double vrp = V[r * k + p], vrq = V[r * k + q];
                    V[r * k + p] = c * vrp - s * vrq;
                    V[r * k + q] = s * vrp + c * vrq;
                }
                for (int r = 0; r < k; ++r) {
                    const double apr = a[p * k + r], aqr = a[q * k + r];
                    a[p * k + r] = c * apr - s * aqr;
                    a[q * k + r] = s * apr + c * aqr;
                }
            }
    }
    int idx[KMAX];
    for (int i = 0; i < k; ++i) idx[i] = i;
    for (int i = 1; i < k; ++i) {
        const int x = idx[i];
        int j = i - 1;
        while (j >= 0 && a[idx[j] * k + idx[j]] > a[x * k + x]) {
            idx[j + 1] = idx[j];
            --j;
        }
        idx[j + 1] = x;
    }
    for (int m = 0; m < k; ++m) {
        const int c = idx[m];
        const double om = a[c * k + c];
        double hp = 0.0, hq = 0.0;
        for (int i = 0; i < k; ++i)
            for (int j = 0; j < k; ++j) {
                hp += V[i * k + c] * Ap[i * k + j] * V[j * k + c];
                hq += V[i * k + c] * Aq[i * k + j] * V[j * k + c];
            }
        omega[m] = om;
        pairing[2 * m] = fabs(hp - om);
        pairing[2 * m + 1] = fabs(hq - om);
    }
}

}  // namespace

// ---- host wrappers ------------------------------------------------------------------------------

constexpr int TRACE_SLICES = 152;

long long gram_scratch_doubles(int nx, int ny) { return (long long)2 * TRACE_SLICES * nx * ny + 64; }

template <typename T>
void gram(cudaStream_t st, const T *X, long long sx, int nx, const T *Y, long long sy, int ny,
          long long len, double *G, double *scratch) {
    const int pairs = nx * ny;
    if (pairs <= 0) return;
    if (nx > 64 || ny > 64) throw CudaError{cudaErrorInvalidValue, "gram: too many matrices"};
    ProfScope ps(st, ST_TRACE, 2.0 * pairs * (double)len, sizeof(T) * (double)(nx + ny) * len);
    const int ti = (nx + 7) / 8, tj = (ny + 7) / 8;
    const long long per = (len + 255) / 256;
    const int slices = (int)std::min<long long>(TRACE_SLICES, std::max<long long>(1, per));
    gram_tiled<T><<<dim3(slices, ti * tj), 256, 0, st>>>(X, sx, nx, Y, sy, ny, len, tj, scratch, pairs);
    check_launch("gram_tiled");
    gram_final<<<(pairs + 255) / 256, 256, 0, st>>>(scratch, slices, pairs, G);
    check_launch("gram_final");
}

template <typename T>
void dots(cudaStream_t st, const T *X, long long sx, const T *Y, long long sy, int n, long long len,
          double *d, double *scratch) {
    if (n <= 0) return;
    ProfScope ps(st, ST_TRACE, 2.0 * n * (double)len, sizeof(T) * 2.0 * n * len);
    const long long per = (len + 255) / 256;
    const int slices = (int)std::min<long long>(2 * TRACE_SLICES, std::max<long long>(1, per));
    dots_kernel<T><<<dim3(slices, n), 256, 0, st>>>(X, sx, Y, sy, len, n, scratch);
    check_launch("dots_kernel");
    gram_final<<<(n + 255) / 256, 256, 0, st>>>(scratch, slices, n, d);
    check_launch("gram_final");
}

template <typename T>
void combine(cudaStream_t st, const double *C, int ldc, int nout, int nin, const T *in, long long sin,
             T *out, long long sout, long long len, bool accumulate) {
    if (nout > 32 || nin > 32) throw CudaError{cudaErrorInvalidValue, "combine: too many states"};
    ProfScope ps(st, ST_VECTOR, 2.0 * nout * nin * (double)len,
                 sizeof(T) * (double)(nin + nout * (accumulate ? 2 : 1)) * len);
    combine_kernel<T><<<grid_for(len), 256, 0, st>>>(C, ldc, nout, nin, in, sin, out, sout, len,
                                                      accumulate);
    check_launch("combine_kernel");
}

template <typename T>
void mask_mul(cudaStream_t st, T *X, const T *mask, long long len, int nb) {
    ProfScope ps(st, ST_VECTOR, (double)len * nb, sizeof(T) * (2.0 * nb + 1.0) * len);
    mask_kernel<T><<<grid_for(len * nb), 256, 0, st>>>(X, mask, len, nb);
    check_launch("mask_kernel");
}

template <typename Tin, typename Tout>
void convert(cudaStream_t st, const Tin *in, Tout *out, long long n) {
    ProfScope ps(st, ST_VECTOR, 0.0, (double)(sizeof(Tin) + sizeof(Tout)) * n);
    convert_kernel<Tin, Tout><<<grid_for(n), 256, 0, st>>>(in, out, n);
    check_launch("convert_kernel");
}

template <typename T>
void axpy_dev(cudaStream_t st, const double *a, int a_stride, double sgn, T *y, const T *x,
              long long len, int nb) {
    ProfScope ps(st, ST_VECTOR, 2.0 * len * nb, 3.0 * sizeof(T) * len * nb);
    axpy_dev_kernel<T><<<grid_for(len * nb), 256, 0, st>>>(a, a_stride, sgn, y, x, len, nb);
    check_launch("axpy_dev_kernel");
}

template <typename T>
void direction(cudaStream_t st, T *out, const T *z, const T *prev, const double *beta, long long n) {
    ProfScope ps(st, ST_VECTOR, 2.0 * n, 3.0 * sizeof(T) * n);
    direction_kernel<T><<<grid_for(n), 256, 0, st>>>(out, z, prev, beta, n);
    check_launch("direction_kernel");
}

template <typename T>
void cg_dir(cudaStream_t st, T *p, const T *r, const double *beta, long long len, int nb) {
    ProfScope ps(st, ST_VECTOR, 2.0 * len * nb, 3.0 * sizeof(T) * len * nb);
    cg_dir_kernel<T><<<grid_for(len * nb), 256, 0, st>>>(p, r, beta, len, nb);
    check_launch("cg_dir_kernel");
}

void make_q(cudaStream_t st, int k, const double *A, double *Q, double *coef) {
    ProfScope ps(st, ST_SMALL, 0.0, 0.0);
    make_q_kernel<<<1, 1, 0, st>>>(k, A, Q, coef);
    check_launch("make_q_kernel");
}
void eval_finish(cudaStream_t st, int k, const double *Q, const double *d, double *out, int *status) {
    ProfScope ps(st, ST_SMALL, 0.0, 0.0);
    eval_finish_kernel<<<1, 1, 0, st>>>(k, Q, d, out, status);
    check_launch("eval_finish_kernel");
}
void conj_coeff(cudaStream_t st, int k2, const double *gz, const double *gzp, const double *gd,
                int restart, const double *flip, double *sc) {
    ProfScope ps(st, ST_SMALL, 0.0, 0.0);
    conj_kernel<<<1, 1, 0, st>>>(k2, gz, gzp, gd, restart, flip, sc);
    check_launch("conj_kernel");
}
void line_gs(cudaStream_t st, int k, const double *A, const double *BDf, const double *CDfD,
             const double *PP, const double *PD, const double *DP, const double *DD, const double *Q,
             double *lam, double *Cp, double *Cq, double *flip, int *status) {
    ProfScope ps(st, ST_SMALL, 0.0, 0.0);
    line_gs_kernel<<<1, 1, 0, st>>>(k, A, BDf, CDfD, PP, PD, DP, DD, Q, lam, Cp, Cq, flip, status);
    check_launch("line_gs_kernel");
}
void init_gs(cudaStream_t st, int k, const double *PP, double *Cp, double *Cq, int *status) {
    ProfScope ps(st, ST_SMALL, 0.0, 0.0);
    init_gs_kernel<<<1, 1, 0, st>>>(k, PP, Cp, Cq, status);
    check_launch("init_gs_kernel");
}
void cg_init(cudaStream_t st, int n, double tol, const double *rr0, double *rr, double *r0,
             int *active, int *n_active) {
    ProfScope ps(st, ST_SMALL, 0.0, 0.0);
    cg_init_kernel<<<1, 1, 0, st>>>(n, tol, rr0, rr, r0, active, n_active);
    check_launch("cg_init_kernel");
}
void cg_scalars(cudaStream_t st, int n, int phase, double tol, const double *pLp, const double *rr_new,
                double *rr, const double *r0, double *alpha, double *beta, int *active, int *n_active) {
    ProfScope ps(st, ST_SMALL, 0.0, 0.0);
    cg_scalars_kernel<<<1, 1, 0, st>>>(n, phase, tol, pLp, rr_new, rr, r0, alpha, beta, active, n_active);
    check_launch("cg_scalars_kernel");
}
void subspace(cudaStream_t st, int k, const double *A, double *omega, double *pairing) {
    ProfScope ps(st, ST_SMALL, 0.0, 0.0);
    subspace_kernel<<<1, 1, 0, st>>>(k, A, omega, pairing);
    check_launch("subspace_kernel");
}

#define INST(T)                                                                                   \
    template void gram<T>(cudaStream_t, const T *, long long, int, const T *, long long, int,      \
                          long long, double *, double *);                                         \
    template void dots<T>(cudaStream_t, const T *, long long, const T *, long long, int, long long, \
                          double *, double *);                                                    \
    template void combine<T>(cudaStream_t, const double *, int, int, int, const T *, long long,    \
                             T *, long long, long long, bool);                                    \
    template void mask_mul<T>(cudaStream_t, T *, const T *, long long, int);                      \
    template void axpy_dev<T>(cudaStream_t, const double *, int, double, T *, const T *, long long, \
                              int);                                                               \
    template void direction<T>(cudaStream_t, T *, const T *, const T *, const double *, long long); \
    template void cg_dir<T>(cudaStream_t, T *, const T *, const double *, long long, int);
INST(float)
INST(double)
#undef INST
template void convert<double, float>(cudaStream_t, const double *, float *, long long);
template void convert<float, double>(cudaStream_t, const float *, double *, long long);
template void convert<double, double>(cudaStream_t, const double *, double *, long long);

}  // namespace tddft
