// Solver primitives: trace products with float64 accumulation in a fixed order, linear
// combinations of state matrices, masks, and the small float64 algebra of the PCG step
// (paper Sec. III C): Q matrix, sum-functional line step, sign flip + Gram-Schmidt in the metric
// of Eq. ortho, subspace eigenvalues.
#include "solver_kernels.h"

#include <algorithm>
#include <initializer_list>
#include <cmath>
#include <cstdlib>

namespace tddft {

namespace {


// ------------------------------------------------------------------------------------------------
// G[p] = sum over the slices of partial[slice][p]: one warp per output, lanes stride the slices,
// then a fixed butterfly (deterministic)
__global__ void gram_final(const double *__restrict__ partial, int nblocks, int pairs,
                           double *__restrict__ G) {
    const int lane = threadIdx.x & 31;
    const int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (p >= pairs) return;
    double s = 0.0;
    for (int b = lane; b < nblocks; b += 32) s += partial[(long long)b * pairs + p];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) G[p] = s;
}

// up to four Gram matrices of one X against several Y sets, [nx][per] each
struct GOut {
    double *g[4];
};
__global__ void gram_final_multi(const double *__restrict__ partial, int nblocks, int pairs, int ny, int per,
                                 GOut out) {
    const int lane = threadIdx.x & 31;
    const int p = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (p >= pairs) return;
    double s = 0.0;
    for (int b = lane; b < nblocks; b += 32) s += partial[(long long)b * pairs + p];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) {
        const int i = p / ny, j = p - i * ny, q = j / per;
        out.g[q][i * per + (j - q * per)] = s;
    }
}

// the Y rows of a trace product: row j is row (j % per) of set j / per
template <typename T>
struct YSet {
    const T *p[4];
    int per;
};

// ------------------------------------------------------------------------------------------------
// Register-tiled trace products. Block (x, y): pair tile x of TI x TJ (i, j), element slice y
// (consecutive blocks share a slice, so the rows a tile re-reads come from L2). Each thread sums
// its products in T over runs of RUN elements and the runs in T again (at most RUN * RUN
// elements per thread by the choice of the slice count), the warp reduces in T by a fixed
// butterfly, the block sums its 8 warps in float64 and writes one partial per pair; gram_final
// sums the partials over slices in float64. float64 arithmetic is scarce on this part, so it is
// kept off the per-element path.
constexpr int RUN = 32;
constexpr int TI = 4;   // pair tile: TI x TJ (TJ = 8 for scalar loads, 4 for pairs of elements)

// VEC consecutive elements per load (float4 / double2 when every row start is aligned and len
// a multiple of VEC), so that more bytes are in flight per load instruction
template <typename T, int VEC> struct VecLd;
template <typename T> struct VecLd<T, 1> {
    static __device__ __forceinline__ void ld(const T *p, long long e, T *o) { o[0] = p[e]; }
};
template <> struct VecLd<float, 2> {
    static __device__ __forceinline__ void ld(const float *p, long long e, float *o) {
        const float2 v = reinterpret_cast<const float2 *>(p)[e];
        o[0] = v.x, o[1] = v.y;
    }
};
template <> struct VecLd<float, 4> {
    static __device__ __forceinline__ void ld(const float *p, long long e, float *o) {
        const float4 v = reinterpret_cast<const float4 *>(p)[e];
        o[0] = v.x, o[1] = v.y, o[2] = v.z, o[3] = v.w;
    }
};
template <> struct VecLd<double, 2> {
    static __device__ __forceinline__ void ld(const double *p, long long e, double *o) {
        const double2 v = reinterpret_cast<const double2 *>(p)[e];
        o[0] = v.x, o[1] = v.y;
    }
};

template <typename T, int VEC, int TJ>
__global__ void __launch_bounds__(256, 2) gram_tiled(const T *__restrict__ X, long long sx, int nx,
                                                     const YSet<T> ys, long long sy, int ny,
                                                     long long len, int tiles_j, double *__restrict__ partial,
                                                     int pairs) {
    __shared__ double red[TI][TJ][8];
    const int ti = blockIdx.x / tiles_j, tj = blockIdx.x - ti * tiles_j;
    const int i0 = ti * TI, j0 = tj * TJ;
    const T *yr[TJ];
#pragma unroll
    for (int b = 0; b < TJ; ++b) {
        const int j = j0 + b < ny ? j0 + b : 0, q = j / ys.per;
        yr[b] = ys.p[q] + (long long)(j - q * ys.per) * sy;
    }
    T tot[TI][TJ], run[TI][TJ];
#pragma unroll
    for (int a = 0; a < TI; ++a)
#pragma unroll
        for (int b = 0; b < TJ; ++b) tot[a][b] = T(0), run[a][b] = T(0);
    const long long stride = (long long)gridDim.y * blockDim.x;
    const long long nvec = len / VEC;
    int cnt = 0;
    for (long long e = blockIdx.y * (long long)blockDim.x + threadIdx.x; e < nvec; e += stride) {
        T xv[TI][VEC], yv[TJ][VEC];
#pragma unroll
        for (int a = 0; a < TI; ++a) {
            if (i0 + a < nx) VecLd<T, VEC>::ld(X + (i0 + a) * sx, e, xv[a]);
            else
#pragma unroll
                for (int u = 0; u < VEC; ++u) xv[a][u] = T(0);
        }
#pragma unroll
        for (int b = 0; b < TJ; ++b) {
            if (j0 + b < ny) VecLd<T, VEC>::ld(yr[b], e, yv[b]);
            else
#pragma unroll
                for (int u = 0; u < VEC; ++u) yv[b][u] = T(0);
        }
#pragma unroll
        for (int u = 0; u < VEC; ++u)
#pragma unroll
            for (int a = 0; a < TI; ++a)
#pragma unroll
                for (int b = 0; b < TJ; ++b) run[a][b] = fma(xv[a][u], yv[b][u], run[a][b]);
        if (++cnt == RUN / VEC) {
#pragma unroll
            for (int a = 0; a < TI; ++a)
#pragma unroll
                for (int b = 0; b < TJ; ++b) tot[a][b] += run[a][b], run[a][b] = T(0);
            cnt = 0;
        }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < TI; ++a)
#pragma unroll
        for (int b = 0; b < TJ; ++b) {
            T v = tot[a][b] + run[a][b];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0) red[a][b][warp] = (double)v;
        }
    __syncthreads();
    if (threadIdx.x < TI * TJ) {
        const int a = threadIdx.x / TJ, b = threadIdx.x - a * TJ;
        double v = 0.0;
        for (int w = 0; w < 8; ++w) v += red[a][b][w];
        const int i = i0 + a, j = j0 + b;
        if (i < nx && j < ny) partial[(long long)blockIdx.y * pairs + i * ny + j] = v;
    }
}

// d_i = sum_e X_i[e] Y_i[e]: one row per blockIdx.y, the same two-level runs and reductions
template <typename T>
__global__ void __launch_bounds__(256) dots_kernel(const T *__restrict__ X, long long sx, const T *__restrict__ Y,
                                                   long long sy, long long len, int n, double *__restrict__ partial) {
    __shared__ double red[8];
    const int i = blockIdx.y;
    const T *x = X + i * sx;
    const T *y = Y + i * sy;
    T tot = T(0), run = T(0);
    int cnt = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < len; e += stride) {
        run = fma(x[e], y[e], run);
        if (++cnt == RUN) {
            tot += run;
            run = T(0);
            cnt = 0;
        }
    }
    T v = tot + run;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += red[w];
        partial[(long long)blockIdx.x * n + i] = s;
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

template <typename Tin, typename Tout>
__global__ void convert_kernel(const Tin *__restrict__ in, Tout *__restrict__ out, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = Tout(in[i]);
}

// 16-byte vectors of T (4 float or 2 double) for the batched element-wise kernels
template <typename T> struct Vec16;
template <> struct Vec16<float> {
    using type = float4;
    static constexpr int n = 4;
    __device__ static float4 fma1(float a, float4 x, float4 y) {
        return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
    }
    __device__ static float4 mul(float4 x, float4 m) { return make_float4(x.x * m.x, x.y * m.y, x.z * m.z, x.w * m.w); }
};
template <> struct Vec16<double> {
    using type = double2;
    static constexpr int n = 2;
    __device__ static double2 fma1(double a, double2 x, double2 y) { return make_double2(fma(a, x.x, y.x), fma(a, x.y, y.y)); }
    __device__ static double2 mul(double2 x, double2 m) { return make_double2(x.x * m.x, x.y * m.y); }
};

// ------------------------------------------------------------------------------------------------
// Trace products with every row read once: block s takes one contiguous range of elements and
// all nx x ny pairs. Chunks of 256 bytes of each of the nx + ny rows stream through a ring of
// GST shared-memory stages by cp.async (16-byte copies, zero fill past the range), so that
// several chunks per block are in flight. A staged row takes 272 bytes (17 16-byte units, an
// odd number), and thread (a, b) of the pair grid owns the rows a, a + gx, a + 2 gx, a + 3 gx of
// X and b, b + gy, ... of Y, so the 16-byte reads of the lanes of a warp (consecutive b) fall on
// distinct bank groups. The pair grid (at most 128 threads) is held twice: the two halves of
// the block take the two halves of every chunk. Products are summed in T over a half chunk,
// those sums in a compensated (Kahan) sum in T; the halves meet in shared memory at the end and
// partial[s][pair] is written in float64, summed over the slices by gram_final_multi.
template <typename T> __host__ __device__ constexpr int gram_chunk() { return 256 / (int)sizeof(T); }
template <typename T> __host__ __device__ constexpr int gram_row() { return 272 / (int)sizeof(T); }
constexpr int GQ = 4;           // pair tile edge
constexpr int GST = 4;          // ring stages
constexpr int GMAXT = 10;       // 16-byte copies per thread and chunk: nx + ny <= 160

__device__ __forceinline__ void cp_async16(void *dst, const void *src, bool full) {
    const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(full ? 16 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <typename T>
__global__ void __launch_bounds__(256) gram_rows_kernel(const T *__restrict__ X, long long sx, int nx,
                                                        const YSet<T> ys, long long sy, int ny, long long len,
                                                        long long per_slice, int RX, int RY,
                                                        double *__restrict__ partial, int pairs) {
    extern __shared__ __align__(16) unsigned char gram_smem[];
    constexpr int VW = Vec16<T>::n;
    constexpr int GC = gram_chunk<T>();      // elements per staged chunk of a row
    constexpr int RS = gram_row<T>();        // staged row stride (elements)
    constexpr int TPR = GC / VW;             // 16-byte copies per row and chunk (16)
    T *ring = reinterpret_cast<T *>(gram_smem);
    const int stage_elems = (RX + RY) * RS;
    const int gy = (ny + GQ - 1) / GQ, gx = (nx + GQ - 1) / GQ;
    const int t = threadIdx.x, half = t >> 7, tl = t & 127;
    const bool owner = tl < gx * gy;
    const int ta = owner ? tl / gy : 0, tb = owner ? tl - (tl / gy) * gy : 0;
    const long long e0 = (long long)blockIdx.x * per_slice;
    const long long e1 = e0 + per_slice < len ? e0 + per_slice : len;
    const int nch = e1 > e0 ? (int)((e1 - e0 + GC - 1) / GC) : 0;
    const int tasks = (nx + ny) * TPR;

    auto issue = [&](int ch) {
        if (ch < nch) {
            T *stg = ring + (ch % GST) * stage_elems;
#pragma unroll
            for (int m = 0; m < GMAXT; ++m) {
                const int q = t + 256 * m;
                if (q < tasks) {
                    const int row = q / TPR, g = q - row * TPR;
                    const long long e = e0 + (long long)ch * GC + (long long)g * VW;
                    const T *src;
                    int srow;
                    if (row < nx) {
                        src = X + row * sx;
                        srow = row;
                    } else {
                        const int j = row - nx, s = j / ys.per;
                        const T *set = s == 0 ? ys.p[0] : s == 1 ? ys.p[1] : s == 2 ? ys.p[2] : ys.p[3];
                        src = set + (long long)(j - s * ys.per) * sy;
                        srow = RX + j;
                    }
                    const bool in = e < e1;
                    cp_async16(stg + srow * RS + g * VW, in ? src + e : src, in);
                }
            }
        }
        cp_async_commit();
    };

    T tot[GQ][GQ], cmp[GQ][GQ];
#pragma unroll
    for (int a = 0; a < GQ; ++a)
#pragma unroll
        for (int b = 0; b < GQ; ++b) tot[a][b] = T(0), cmp[a][b] = T(0);
#pragma unroll
    for (int c = 0; c < GST - 1; ++c) issue(c);
    for (int ch = 0; ch < nch; ++ch) {
        cp_async_wait<GST - 2>();
        __syncthreads();             // chunk ch has landed for every thread; stage (ch - 1) is free
        issue(ch + GST - 1);
        if (owner) {
            const T *stg = ring + (ch % GST) * stage_elems;
            T run[GQ][GQ];
#pragma unroll
            for (int a = 0; a < GQ; ++a)
#pragma unroll
                for (int b = 0; b < GQ; ++b) run[a][b] = T(0);
#pragma unroll 2
            for (int c = half * (GC / 2); c < (half + 1) * (GC / 2); c += VW) {
                T xa[GQ][VW], yb[GQ][VW];
#pragma unroll
                for (int a = 0; a < GQ; ++a) {
                    const auto v = *reinterpret_cast<const typename Vec16<T>::type *>(stg + (ta + a * gx) * RS + c);
                    const T *pv = reinterpret_cast<const T *>(&v);
#pragma unroll
                    for (int u = 0; u < VW; ++u) xa[a][u] = pv[u];
                }
#pragma unroll
                for (int b = 0; b < GQ; ++b) {
                    const auto v = *reinterpret_cast<const typename Vec16<T>::type *>(stg + (RX + tb + b * gy) * RS + c);
                    const T *pv = reinterpret_cast<const T *>(&v);
#pragma unroll
                    for (int u = 0; u < VW; ++u) yb[b][u] = pv[u];
                }
#pragma unroll
                for (int u = 0; u < VW; ++u)
#pragma unroll
                    for (int a = 0; a < GQ; ++a)
#pragma unroll
                        for (int b = 0; b < GQ; ++b) run[a][b] = fma(xa[a][u], yb[b][u], run[a][b]);
            }
#pragma unroll
            for (int a = 0; a < GQ; ++a)
#pragma unroll
                for (int b = 0; b < GQ; ++b) {
                    const T y = run[a][b] - cmp[a][b];
                    const T s = tot[a][b] + y;
                    cmp[a][b] = (s - tot[a][b]) - y;
                    tot[a][b] = s;
                }
        }
    }
    cp_async_wait<0>();
    __syncthreads();                 // the ring is free: the second half hands over its sums
    double *hand = reinterpret_cast<double *>(gram_smem);   // [GQ * GQ][128]
    if (owner && half == 1)
#pragma unroll
        for (int a = 0; a < GQ; ++a)
#pragma unroll
            for (int b = 0; b < GQ; ++b) hand[(a * GQ + b) * 128 + tl] = (double)tot[a][b] - (double)cmp[a][b];
    __syncthreads();
    if (!owner || half == 1) return;
#pragma unroll
    for (int a = 0; a < GQ; ++a)
#pragma unroll
        for (int b = 0; b < GQ; ++b) {
            const int i = ta + a * gx, j = tb + b * gy;
            if (i < nx && j < ny)
                partial[(long long)blockIdx.x * pairs + i * ny + j] =
                    ((double)tot[a][b] - (double)cmp[a][b]) + hand[(a * GQ + b) * 128 + tl];
        }
}

// Batched element-wise kernels: blockIdx.y = matrix b of nb, blockIdx.x strides over the len
// entries of one matrix (in 16-byte vectors when len allows), so the per-matrix coefficient is
// read once per thread and no index division runs per element.
// y_b += sgn * a[b * a_stride] * x_b
template <typename T, bool VEC>
__global__ void axpy_dev_kernel(const double *__restrict__ a, int a_stride, double sgn, T *__restrict__ y,
                                const T *__restrict__ x, long long len) {
    const int b = blockIdx.y;
    const T c = T(sgn * a[(long long)b * a_stride]);
    const long long base = (long long)b * len;
    if (VEC) {
        using V = typename Vec16<T>::type;
        V *yv = reinterpret_cast<V *>(y + base);
        const V *xv = reinterpret_cast<const V *>(x + base);
        const long long nv = len / Vec16<T>::n;
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nv; i += (long long)gridDim.x * blockDim.x)
            yv[i] = Vec16<T>::fma1(c, xv[i], yv[i]);
    } else {
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
            y[base + i] = fma(c, x[base + i], y[base + i]);
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

// grid of a batched element-wise launch: x blocks over one matrix of len entries (vectors of
// 16 bytes when len and the pointers allow), y = the nb matrices; about 8 blocks per SM in all
dim3 batched_grid(long long len, int nb, bool vec, int per) {
    const long long units = vec ? len / per : len;
    long long bx = (units + 255) / 256;
    const long long cap = std::max<long long>(1, 8 * 152 / std::max(1, nb));
    bx = std::max<long long>(1, std::min(bx, cap));
    return dim3((unsigned)bx, (unsigned)nb);
}

template <typename T>
bool vec_ok(long long len, std::initializer_list<const void *> ptrs) {
    if (len % (16 / (long long)sizeof(T))) return false;
    for (const void *p : ptrs)
        if (reinterpret_cast<unsigned long long>(p) % 16) return false;
    return true;
}

int grid_for(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < 4 * 152 ? (b > 0 ? b : 1) : 4 * 152);
}

// ------------------------------------------------------------------------------------------------
// Small float64 algebra for one thread block (k <= KMAX, so k * k <= 256 threads hold one matrix
// element each). Matrices live in shared memory; every routine is entered and left by all
// threads of the block, and the steps that must follow one another (pivots, Gram-Schmidt
// vectors) are the only sequential parts: float64 latency and block barriers are what this
// code costs on this part, not arithmetic.
constexpr int SB_THREADS = 256;

struct SbLine {
    double N0[KMAX * KMAX], N1[KMAX * KMAX], N2[KMAX * KMAX];
    double M0[KMAX * KMAX], M1[KMAX * KMAX], M2[KMAX * KMAX];
    double A[2][KMAX * KMAX];              // M, reduced in place to M^-1 (two buffers)
    double dM[KMAX * KMAX], N[KMAX * KMAX], dN[KMAX * KMAX];
    double T[KMAX * KMAX], Z[KMAX * KMAX];
    double red[SB_THREADS / 32][3];
    double out[4];
    int bad;
};

// Omega(lam) = Tr[M^-1 N]/2 and dOmega/dlam = Tr[M^-1 dN - M^-1 dM M^-1 N]/2 with
// M = M0 + lam M1 + lam^2 M2, N likewise; false (in every thread) if M is not positive definite.
// M^-1 by Gauss-Jordan elimination without pivoting, one pivot per step with every element
// updated at once: for a symmetric M the pivots are those of its L D L^T factorisation, so all
// are positive exactly when M is positive definite. The traces are element-wise sums
// (Tr[A B] = sum_ij A_ij B_ji), so only W = M^-1 N and U = M^-1 dM are formed:
// Omega = Tr[W]/2, dOmega = (sum_ij Minv_ij dN_ji - sum_ij U_ij W_ji)/2.
__device__ bool sb_sum_functional(int k, SbLine &s, double lam, double *f, double *d) {
    const int t = threadIdx.x, kk = k * k;
    const int i = t < kk ? t / k : 0, j = t < kk ? t - i * k : 0;
    if (t < kk) {
        s.A[0][t] = s.M0[t] + lam * s.M1[t] + lam * lam * s.M2[t];
        s.dM[t] = s.M1[t] + 2.0 * lam * s.M2[t];
        s.N[t] = s.N0[t] + lam * s.N1[t] + lam * lam * s.N2[t];
        s.dN[t] = s.N1[t] + 2.0 * lam * s.N2[t];
    }
    __syncthreads();
    int cur = 0;
    for (int p = 0; p < k; ++p) {
        const double *a = s.A[cur];
        const double piv = a[p * k + p];
        if (!(piv > 0.0)) {                 // the same value in every thread
            __syncthreads();
            return false;
        }
        if (t < kk) {
            const double r = 1.0 / piv;
            double v;
            if (i == p) v = (j == p) ? r : a[t] * r;
            else if (j == p) v = -a[t] * r;
            else v = a[t] - a[i * k + p] * a[p * k + j] * r;
            s.A[cur ^ 1][t] = v;
        }
        cur ^= 1;
        __syncthreads();
    }
    const double *mi = s.A[cur];
    if (t < kk) {
        double w = 0.0, u = 0.0;
        for (int q = 0; q < k; ++q) {
            w += mi[i * k + q] * s.N[q * k + j];
            u += mi[i * k + q] * s.dM[q * k + j];
        }
        s.T[t] = w;
        s.Z[t] = u;
    }
    __syncthreads();
    double v0 = 0.0, v1 = 0.0, v2 = 0.0;
    if (t < kk) {
        v0 = i == j ? s.T[t] : 0.0;
        v1 = mi[t] * s.dN[j * k + i];
        v2 = s.Z[t] * s.T[j * k + i];
    }
    for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_xor_sync(0xffffffffu, v0, o);
        v1 += __shfl_xor_sync(0xffffffffu, v1, o);
        v2 += __shfl_xor_sync(0xffffffffu, v2, o);
    }
    if ((t & 31) == 0) {
        s.red[t >> 5][0] = v0;
        s.red[t >> 5][1] = v1;
        s.red[t >> 5][2] = v2;
    }
    __syncthreads();
    if (t == 0) {
        double tw = 0.0, tx = 0.0, tz = 0.0;
        for (int w = 0; w < (kk + 31) / 32; ++w) {
            tw += s.red[w][0];
            tx += s.red[w][1];
            tz += s.red[w][2];
        }
        s.out[0] = 0.5 * tw;
        s.out[1] = 0.5 * (tx - tz);
    }
    __syncthreads();
    *f = s.out[0];
    *d = s.out[1];
    __syncthreads();
    return true;
}

// Minimiser of Omega along the common step (every thread returns the same value): a Newton
// estimate from the second derivative at 0 (with M0 = I), doubled until dOmega >= 0 brackets the
// root, bisection while M is indefinite at the upper end, then Illinois regula falsi on dOmega
// to machine precision
__device__ double sb_line_step(int k, SbLine &s) {
    double f0, d0;
    if (!sb_sum_functional(k, s, 0.0, &f0, &d0) || !isfinite(d0) || d0 >= 0.0) return 0.0;
    const int t = threadIdx.x;
    // h0 = Tr[2 N2 - 2 M1 N1 + 2 M1 M1 N0 - 2 M2 N0] / 2, one row per thread, summed in order
    if (t < k) {
        const int i = t;
        double h = 2.0 * s.N2[i * k + i];
        for (int p = 0; p < k; ++p) {
            h -= 2.0 * s.M1[i * k + p] * s.N1[p * k + i];
            h -= 2.0 * s.M2[i * k + p] * s.N0[p * k + i];
            double m1m1 = 0.0;
            for (int q = 0; q < k; ++q) m1m1 += s.M1[i * k + q] * s.M1[q * k + p];
            h += 2.0 * m1m1 * s.N0[p * k + i];
        }
        s.T[i] = 0.5 * h;
    }
    __syncthreads();
    if (t == 0) {
        double h0 = 0.0;
        for (int i = 0; i < k; ++i) h0 += s.T[i];
        s.out[2] = h0;
    }
    __syncthreads();
    const double h0 = s.out[2];
    __syncthreads();
    double hi = (h0 > 0.0 && isfinite(h0)) ? -d0 / h0 : 1.0;
    double lo = 0.0, dlo = d0, dhi = 0.0, f, d = d0;
    for (int it = 0; it < 60; ++it) {
        if (!sb_sum_functional(k, s, hi, &f, &d)) d = INFINITY;
        if (d >= 0.0) break;
        lo = hi;
        dlo = d;
        hi = 2.0 * hi;
    }
    dhi = d;
    for (int b = 0; b < 200 && !isfinite(dhi); ++b) {
        const double mid = 0.5 * (lo + hi);
        if (!sb_sum_functional(k, s, mid, &f, &d)) d = INFINITY;
        if (d < 0.0) { lo = mid; dlo = d; }
        else { hi = mid; dhi = d; }
    }
    int side = 0;
    for (int r = 0; r < 100; ++r) {
        if (!(hi - lo > 4e-16 * hi)) break;
        double x = (isfinite(dhi) && dhi != dlo) ? hi - dhi * (hi - lo) / (dhi - dlo) : 0.5 * (lo + hi);
        if (!(x > lo && x < hi)) x = 0.5 * (lo + hi);
        if (!sb_sum_functional(k, s, x, &f, &d)) d = INFINITY;
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

// Classical Gram-Schmidt run twice on coefficient vectors in the metric Mg, vectors taken in
// the given order; rows of C are the new vectors. u and coef are k-vectors of work space.
// False (in every thread) if a norm is not positive.
__device__ bool sb_gram_schmidt(int k, const double *Mg, const int *order, double *C, double *v,
                                double *u, double *coef, int *bad) {
    const int t = threadIdx.x;
    if (t < k * k) C[t] = 0.0;
    if (t == 0) *bad = 0;
    __syncthreads();
    for (int a = 0; a < k; ++a) {
        const int i = order[a];
        if (t < k) v[t] = (t == i) ? 1.0 : 0.0;
        __syncthreads();
        for (int pass = 0; pass < 2; ++pass) {
            if (t < k) {                    // u = Mg v
                double acc = 0.0;
                for (int q = 0; q < k; ++q) acc += Mg[t * k + q] * v[q];
                u[t] = acc;
            }
            __syncthreads();
            if (t < a) {                    // coef_b = <v, C_order[b]>_Mg
                const int j = order[t];
                double acc = 0.0;
                for (int p = 0; p < k; ++p) acc += C[j * k + p] * u[p];
                coef[t] = acc;
            }
            __syncthreads();
            if (t < k) {
                double x = v[t];
                for (int b = 0; b < a; ++b) x -= coef[b] * C[order[b] * k + t];
                v[t] = x;
            }
            __syncthreads();
        }
        if (t < k) {
            double acc = 0.0;
            for (int q = 0; q < k; ++q) acc += Mg[t * k + q] * v[q];
            u[t] = acc;
        }
        __syncthreads();
        if (t == 0) {
            double nrm = 0.0;
            for (int p = 0; p < k; ++p) nrm += v[p] * u[p];
            const double ref = fabs(Mg[i * k + i]) > 1.0 ? fabs(Mg[i * k + i]) : 1.0;
            if (!isfinite(nrm) || nrm <= 1e-12 * ref) *bad = 1;
            coef[KMAX] = *bad ? 0.0 : rsqrt(nrm);
        }
        __syncthreads();
        if (*bad) return false;
        if (t < k) C[i * k + t] = v[t] * coef[KMAX];
        __syncthreads();
    }
    return true;
}

// Eigenvalues of a symmetric k x k matrix, ascending, into w (written by thread 0); a is
// overwritten. Jacobi sweeps in round-robin (tournament) order: the k (padded to even m) indices
// meet in m - 1 rounds of m / 2 disjoint pairs, and a round's rotations commute, so their angles
// are computed in parallel and applied together (columns, then rows). cs holds 2 KMAX + 1 values.
__device__ void sb_jacobi_eigenvalues(int k, double *a, double *w, double *cs) {
    const int t = threadIdx.x;
    const int m = k + (k & 1), half = m / 2;
    for (int sweep = 0; sweep < 60; ++sweep) {
        if (t == 0) {
            double off = 0.0, tot = 0.0;
            for (int i = 0; i < k; ++i)
                for (int j = 0; j < k; ++j) {
                    tot += a[i * k + j] * a[i * k + j];
                    if (i != j) off += a[i * k + j] * a[i * k + j];
                }
            cs[2 * KMAX] = (off <= 1e-30 * tot || off == 0.0) ? 1.0 : 0.0;
        }
        __syncthreads();
        const bool done = cs[2 * KMAX] != 0.0;
        __syncthreads();
        if (done) break;
        for (int r = 0; r < m - 1; ++r) {
            if (t < half) {
                // pair t of round r: index m - 1 meets r, the others pair up around the circle
                int p = t == 0 ? m - 1 : (r + t) % (m - 1);
                int q = t == 0 ? r : (r - t + m - 1) % (m - 1);
                if (p > q) { const int x = p; p = q; q = x; }
                double c = 1.0, sn = 0.0;
                if (q < k) {
                    const double apq = a[p * k + q];
                    if (apq != 0.0) {
                        const double theta = (a[q * k + q] - a[p * k + p]) / (2.0 * apq);
                        const double tt = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                        c = rsqrt(tt * tt + 1.0);
                        sn = tt * c;
                    }
                }
                cs[2 * t] = c;
                cs[2 * t + 1] = sn;
            }
            __syncthreads();
            if (t < half * k) {             // columns p, q of row t % k for pair t / k
                const int pr = t / k, row = t - pr * k;
                int p = pr == 0 ? m - 1 : (r + pr) % (m - 1);
                int q = pr == 0 ? r : (r - pr + m - 1) % (m - 1);
                if (p > q) { const int x = p; p = q; q = x; }
                const double c = cs[2 * pr], sn = cs[2 * pr + 1];
                if (q < k && sn != 0.0) {
                    const double arp = a[row * k + p], arq = a[row * k + q];
                    a[row * k + p] = c * arp - sn * arq;
                    a[row * k + q] = sn * arp + c * arq;
                }
            }
            __syncthreads();
            if (t < half * k) {             // rows p, q of column t % k for pair t / k
                const int pr = t / k, col = t - pr * k;
                int p = pr == 0 ? m - 1 : (r + pr) % (m - 1);
                int q = pr == 0 ? r : (r - pr + m - 1) % (m - 1);
                if (p > q) { const int x = p; p = q; q = x; }
                const double c = cs[2 * pr], sn = cs[2 * pr + 1];
                if (q < k && sn != 0.0) {
                    const double apr = a[p * k + col], aqr = a[q * k + col];
                    a[p * k + col] = c * apr - sn * aqr;
                    a[q * k + col] = sn * apr + c * aqr;
                }
            }
            __syncthreads();
        }
    }
    if (t == 0) {
        for (int i = 0; i < k; ++i) w[i] = a[i * k + i];
        for (int i = 1; i < k; ++i) {
            const double x = w[i];
            int j = i - 1;
            while (j >= 0 && w[j] > x) {
                w[j + 1] = w[j];
                --j;
            }
            w[j + 1] = x;
        }
    }
    __syncthreads();
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
__global__ void __launch_bounds__(SB_THREADS) eval_finish_kernel(int k, const double *Q, const double *d,
                                                                 double *out, int *status) {
    __shared__ double S[KMAX * KMAX], cs[2 * KMAX + 2];
    __shared__ int bad;
    const int t = threadIdx.x, kk = k * k;
    if (t == 0) bad = 0;
    __syncthreads();
    if (t < kk) {
        const int i = t / k, j = t - i * k;
        S[t] = 0.5 * (Q[i * k + j] + Q[j * k + i]);
        if (!isfinite(S[t])) bad = 1;
    }
    if (t < k) {
        const double r2 = d[t] + d[k + t];
        out[k + t] = sqrt(r2 > 0.0 ? r2 : 0.0);
        if (!isfinite(r2)) bad = 1;
    }
    __syncthreads();
    if (bad) {
        if (t == 0) *status = DEV_NAN_EVAL;
        if (t < k) out[t] = NAN;
        return;
    }
    sb_jacobi_eigenvalues(k, S, out, cs);
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

// Line step and re-orthonormalisation for one thread block of SB_THREADS threads
__global__ void __launch_bounds__(SB_THREADS) line_gs_kernel(int k, const double *A, const double *BDf,
                                                             const double *CDfD, const double *PP,
                                                             const double *PD, const double *DP,
                                                             const double *DD, const double *Q, double *lam,
                                                             double *Cp, double *Cq, double *sc_flip,
                                                             int *status) {
    __shared__ SbLine s;
    __shared__ double T0[KMAX * KMAX], T1[KMAX * KMAX], T2[KMAX * KMAX], Mg[KMAX * KMAX], C[KMAX * KMAX];
    __shared__ double sg[KMAX], v[KMAX], u[KMAX], coef[KMAX + 1];
    __shared__ int order[KMAX], flags[2];
    const int t = threadIdx.x, k2 = 2 * k, kk = k * k;
    if (t == 0) flags[0] = 0;
    __syncthreads();
    if (t < kk) {
        const int i = t / k, j = t - i * k;
        const double n0ij = A[i * k2 + j] + A[(k + i) * k2 + k + j];
        const double n0ji = A[j * k2 + i] + A[(k + j) * k2 + k + i];
        s.N0[t] = 0.5 * (n0ij + n0ji);
        const double efij = BDf[i * k2 + j] + BDf[(k + i) * k2 + k + j];
        const double efji = BDf[j * k2 + i] + BDf[(k + j) * k2 + k + i];
        s.N1[t] = efij + efji;
        const double n2ij = CDfD[i * k2 + j] + CDfD[(k + i) * k2 + k + j];
        const double n2ji = CDfD[j * k2 + i] + CDfD[(k + j) * k2 + k + i];
        s.N2[t] = 0.5 * (n2ij + n2ji);
        T0[t] = PP[i * k2 + k + j];                          // <p_i, q_j>
        T1[t] = PD[i * k2 + k + j] + DP[i * k2 + k + j];     // <p_i, Dq_j> + <Dp_i, q_j>
        T2[t] = DD[i * k2 + k + j];                          // <Dp_i, Dq_j>
    }
    __syncthreads();
    if (t < kk) {
        const int i = t / k, j = t - i * k;
        s.M0[t] = 0.5 * (T0[t] + T0[j * k + i]);
        s.M1[t] = 0.5 * (T1[t] + T1[j * k + i]);
        s.M2[t] = 0.5 * (T2[t] + T2[j * k + i]);
        if (!isfinite(s.N0[t]) || !isfinite(s.N1[t]) || !isfinite(s.N2[t]) || !isfinite(s.M1[t]) ||
            !isfinite(s.M2[t]))
            flags[0] = 1;
    }
    __syncthreads();
    if (flags[0]) {
        if (t == 0) *status = DEV_NAN_LINE;
        return;
    }
    const double l = sb_line_step(k, s);
    if (t < kk) T0[t] = T0[t] + l * T1[t] + l * l * T2[t];   // <p_i, q_j> at the new point
    __syncthreads();
    if (t < k) sg[t] = T0[t * k + t] < 0.0 ? -1.0 : 1.0;
    __syncthreads();
    if (t < kk) {
        const int i = t / k, j = t - i * k;
        Mg[t] = 0.5 * (T0[t] * sg[j] + T0[j * k + i] * sg[i]);
    }
    if (t == 0) {
        *lam = l;
        int any = 0;
        for (int i = 0; i < k; ++i) any |= sg[i] < 0.0;
        flags[1] = any;
        // Gram-Schmidt order: ascending Ritz diagonal Q_ii (insertion sort, stable)
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
    }
    __syncthreads();
    if (!sb_gram_schmidt(k, Mg, order, C, v, u, coef, &s.bad)) {
        if (t == 0) *status = DEV_BREAKDOWN;
        return;
    }
    if (t < kk) {
        const int j = t % k;
        Cp[t] = C[t];
        Cq[t] = C[t] * sg[j];
    }
    if (t == 0) *sc_flip = flags[1] ? 1.0 : 0.0;
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
    // one thread per system (n <= blockDim.x)
    const int i = threadIdx.x;
    int act = 0;
    if (i < n) {
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
            act = active[i];
        }
    }
    const int cnt = __syncthreads_count(act);
    if (phase == 1 && i == 0) *n_active = cnt;
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

// X_b *= mask (blockIdx.y = b)
template <typename T, bool VEC>
__global__ void mask_kernel(T *__restrict__ X, const T *__restrict__ mask, long long len) {
    const long long base = (long long)blockIdx.y * len;
    if (VEC) {
        using V = typename Vec16<T>::type;
        V *xv = reinterpret_cast<V *>(X + base);
        const V *mv = reinterpret_cast<const V *>(mask);
        const long long nv = len / Vec16<T>::n;
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nv; i += (long long)gridDim.x * blockDim.x)
            xv[i] = Vec16<T>::mul(xv[i], mv[i]);
    } else {
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
            X[base + i] *= mask[i];
    }
}

// p_b <- r_b + beta_b p_b (beta on the device; blockIdx.y = b)
template <typename T, bool VEC>
__global__ void cg_dir_kernel(T *__restrict__ p, const T *__restrict__ r, const double *__restrict__ beta,
                              long long len) {
    const int b = blockIdx.y;
    const T c = T(beta[b]);
    const long long base = (long long)b * len;
    if (VEC) {
        using V = typename Vec16<T>::type;
        V *pv = reinterpret_cast<V *>(p + base);
        const V *rv = reinterpret_cast<const V *>(r + base);
        const long long nv = len / Vec16<T>::n;
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nv; i += (long long)gridDim.x * blockDim.x)
            pv[i] = Vec16<T>::fma1(c, pv[i], rv[i]);
    } else {
        for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
            p[base + i] = fma(c, p[base + i], r[base + i]);
    }
}

// Ritz pairs of Q and the pairing errors: rotated halves |<p, f_p>_a - omega_a|,
// |<q, f_q>_a - omega_a| from the p-part and q-part matrices of A.
__global__ void subspace_kernel(int k, const double *A, double *omega, double *pairing, double *vecs) {
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
        if (vecs)
            for (int i = 0; i < k; ++i) vecs[i * k + m] = V[i * k + c];   // column m: Ritz pair m
    }
}

}  // namespace

// ---- host wrappers ------------------------------------------------------------------------------

constexpr int TRACE_SLICES = 152;

long long gram_scratch_doubles(int nx, int ny) { return (long long)2 * TRACE_SLICES * nx * ny + 64; }

// slices of a trace launch: `want`, fewer for short vectors (one 256-thread block per slice
// holds at least one element per thread), more (up to `cap`) when a thread would otherwise
// sum more than RUN * RUN elements
int trace_slices(long long len, int want, int cap) {
    const long long per = (len + 255) / 256;
    long long s = std::min<long long>(want, std::max<long long>(1, per));
    const long long need = (len + 256LL * RUN * RUN - 1) / (256LL * RUN * RUN);
    s = std::max(s, std::min<long long>(need, cap));
    return (int)s;
}

template <typename T>
void gram(cudaStream_t st, const T *X, long long sx, int nx, const T *Y, long long sy, int ny,
          long long len, double *G, double *scratch) {
    gram_multi<T>(st, X, sx, nx, 1, &Y, sy, ny, len, &G, scratch);
}

template <typename T>
void gram_multi(cudaStream_t st, const T *X, long long sx, int nx, int nset, const T *const *Y, long long sy,
                int per, long long len, double *const *G, double *scratch) {
    if (nx <= 0 || per <= 0 || nset < 1) return;
    if (nset > 4 || nx * per > 64 * 32) throw CudaError{cudaErrorInvalidValue, "gram: too many matrices"};
    if (nx * per * nset > 64 * 32) {
        // the partial sums of all pairs must fit the scratch: split the sets
        const int h = nset / 2;
        gram_multi<T>(st, X, sx, nx, h, Y, sy, per, len, G, scratch);
        gram_multi<T>(st, X, sx, nx, nset - h, Y + h, sy, per, len, G + h, scratch);
        return;
    }
    const int ny = nset * per, pairs = nx * ny;
    ProfScope ps(st, ST_TRACE, 2.0 * pairs * (double)len, sizeof(T) * (double)(nx + ny) * len);
    YSet<T> ys{};
    GOut go{};
    for (int q = 0; q < 4; ++q) {
        ys.p[q] = q < nset ? Y[q] : Y[0];
        go.g[q] = q < nset ? G[q] : G[0];
    }
    ys.per = per;
    constexpr int VW = sizeof(T) == 4 ? 4 : 2;   // 16-byte loads
    bool vec = len % VW == 0 && sx % VW == 0 && sy % VW == 0 && reinterpret_cast<uintptr_t>(X) % 16 == 0;
    for (int q = 0; q < nset; ++q) vec = vec && reinterpret_cast<uintptr_t>(Y[q]) % 16 == 0;
    const int gx = (nx + GQ - 1) / GQ, gy = (ny + GQ - 1) / GQ;
    if (vec && len > 0 && nx + ny <= 256 * GMAXT / 16 && gx * gy <= 128) {
        // every row read once (all pairs of a slice in one block)
        constexpr int GC = gram_chunk<T>();
        const long long chunks = (len + GC - 1) / GC;
        const long long want = std::max<long long>(1, std::min<long long>(2 * TRACE_SLICES, (chunks + 15) / 16));
        const long long per_slice = (chunks + want - 1) / want * GC;
        const int slices = (int)((len + per_slice - 1) / per_slice);
        const int RX = GQ * gx, RY = GQ * gy;
        const size_t smem = std::max((size_t)GST * (RX + RY) * gram_row<T>() * sizeof(T),
                                     (size_t)GQ * GQ * 128 * sizeof(double));
        // the attribute is set once, to the most any launch asks for: contexts on other host
        // threads launch this kernel concurrently, and a per-launch value would race with them
        static const bool attr = []() {
            check(cudaFuncSetAttribute(gram_rows_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024),
                  "gram_rows smem");
            return true;
        }();
        (void)attr;
        gram_rows_kernel<T><<<slices, 256, smem, st>>>(X, sx, nx, ys, sy, ny, len, per_slice, RX, RY, scratch, pairs);
        check_launch("gram_rows_kernel");
        gram_final_multi<<<(pairs + 7) / 8, 256, 0, st>>>(scratch, slices, pairs, ny, per, go);
        check_launch("gram_final");
        return;
    }
    const int slices = trace_slices(len, TRACE_SLICES, 2 * TRACE_SLICES);
    const int ti = (nx + TI - 1) / TI;
    if (vec) {
        const int tj = (ny + 3) / 4;
        gram_tiled<T, VW, 4><<<dim3(ti * tj, slices), 256, 0, st>>>(X, sx, nx, ys, sy, ny, len, tj, scratch, pairs);
    } else {
        const int tj = (ny + 7) / 8;
        gram_tiled<T, 1, 8><<<dim3(ti * tj, slices), 256, 0, st>>>(X, sx, nx, ys, sy, ny, len, tj, scratch, pairs);
    }
    check_launch("gram_tiled");
    gram_final_multi<<<(pairs + 7) / 8, 256, 0, st>>>(scratch, slices, pairs, ny, per, go);
    check_launch("gram_final");
}

template <typename T>
void dots(cudaStream_t st, const T *X, long long sx, const T *Y, long long sy, int n, long long len,
          double *d, double *scratch) {
    if (n <= 0) return;
    ProfScope ps(st, ST_TRACE, 2.0 * n * (double)len, sizeof(T) * 2.0 * n * len);
    const int slices = trace_slices(len, 2 * TRACE_SLICES, 2 * TRACE_SLICES);
    dots_kernel<T><<<dim3(slices, n), 256, 0, st>>>(X, sx, Y, sy, len, n, scratch);
    check_launch("dots_kernel");
    gram_final<<<(n + 7) / 8, 256, 0, st>>>(scratch, slices, n, d);
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
    if (nb <= 0) return;
    const bool v = vec_ok<T>(len, {X, mask});
    const dim3 g = batched_grid(len, nb, v, Vec16<T>::n);
    if (v) mask_kernel<T, true><<<g, 256, 0, st>>>(X, mask, len);
    else mask_kernel<T, false><<<g, 256, 0, st>>>(X, mask, len);
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
    if (nb <= 0) return;
    const bool v = vec_ok<T>(len, {y, x});
    const dim3 g = batched_grid(len, nb, v, Vec16<T>::n);
    if (v) axpy_dev_kernel<T, true><<<g, 256, 0, st>>>(a, a_stride, sgn, y, x, len);
    else axpy_dev_kernel<T, false><<<g, 256, 0, st>>>(a, a_stride, sgn, y, x, len);
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
    if (nb <= 0) return;
    const bool v = vec_ok<T>(len, {p, r});
    const dim3 g = batched_grid(len, nb, v, Vec16<T>::n);
    if (v) cg_dir_kernel<T, true><<<g, 256, 0, st>>>(p, r, beta, len);
    else cg_dir_kernel<T, false><<<g, 256, 0, st>>>(p, r, beta, len);
    check_launch("cg_dir_kernel");
}

void make_q(cudaStream_t st, int k, const double *A, double *Q, double *coef) {
    ProfScope ps(st, ST_SMALL, 0.0, 0.0);
    make_q_kernel<<<1, 1, 0, st>>>(k, A, Q, coef);
    check_launch("make_q_kernel");
}
void eval_finish(cudaStream_t st, int k, const double *Q, const double *d, double *out, int *status) {
    ProfScope ps(st, ST_SMALL, 0.0, 0.0);
    eval_finish_kernel<<<1, SB_THREADS, 0, st>>>(k, Q, d, out, status);
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
    line_gs_kernel<<<1, SB_THREADS, 0, st>>>(k, A, BDf, CDfD, PP, PD, DP, DD, Q, lam, Cp, Cq, flip, status);
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
    cg_scalars_kernel<<<1, 32 * ((n + 31) / 32), 0, st>>>(n, phase, tol, pLp, rr_new, rr, r0, alpha, beta, active,
                                                          n_active);
    check_launch("cg_scalars_kernel");
}
void subspace(cudaStream_t st, int k, const double *A, double *omega, double *pairing, double *vecs) {
    ProfScope ps(st, ST_SMALL, 0.0, 0.0);
    subspace_kernel<<<1, 1, 0, st>>>(k, A, omega, pairing, vecs);
    check_launch("subspace_kernel");
}

#define INST(T)                                                                                   \
    template void gram<T>(cudaStream_t, const T *, long long, int, const T *, long long, int,      \
                          long long, double *, double *);                                         \
    template void gram_multi<T>(cudaStream_t, const T *, long long, int, int, const T *const *,     \
                                long long, int, long long, double *const *, double *);            \
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
