// Dense row-major GEMM on CUDA cores (float32 / float64), batched with strides.
//
// C[b] = alpha * op(A[b]) * op(B[b]) + beta * C[b], op = identity or transpose.
// 64x64 output tile per 256-thread block, 16-deep K slices staged in shared memory; thread
// (tx, ty) owns rows ty + 16u and columns tx + 16v (u, v < 4), so shared-memory reads are
// broadcasts (A) or conflict-free (B) and the C stores are coalesced along tx.
#include "tddft_internal.h"

#include <cstdlib>

namespace tddft {

void tc_gemm(cudaStream_t st, bool ta, bool tb, int M, int N, int K, float alpha, const float *A, int lda,
             long long sA, const float *B, int ldb, long long sB, float beta, float *C, int ldc, long long sC,
             int batch, bool split);
bool tc_gemm_available();

bool tc_enabled() {
    static const bool on = []() {
        const char *e = std::getenv("TDDFT_NO_TC");
        return !(e && e[0] == '1') && tc_gemm_available();
    }();
    return on;
}

namespace {

constexpr int BM = 64, BN = 64, BK = 16;

template <typename T, bool TA, bool TB>
__global__ void __launch_bounds__(256) gemm_kernel(int M, int N, int K, T alpha,
                                                   const T *__restrict__ A, int lda, long long sA,
                                                   const T *__restrict__ B, int ldb, long long sB,
                                                   T beta, T *__restrict__ C, int ldc,
                                                   long long sC) {
    __shared__ T As[BK][BM + 1];
    __shared__ T Bs[BK][BN + 1];
    const int b = blockIdx.z;
    A += (long long)b * sA;
    B += (long long)b * sB;
    C += (long long)b * sC;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int t = threadIdx.x;
    const int tx = t & 15, ty = t >> 4;
    T acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = T(0);

    for (int k0 = 0; k0 < K; k0 += BK) {
        // A tile: op(A)(m, k) for m < 64, k < 16
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int m, kk;
            if (!TA) { kk = t & 15; m = (t >> 4) + 16 * i; }
            else { m = t & 63; kk = (t >> 6) + 4 * i; }
            const int gm = m0 + m, gk = k0 + kk;
            T v = T(0);
            if (gm < M && gk < K) v = TA ? A[(long long)gk * lda + gm] : A[(long long)gm * lda + gk];
            As[kk][m] = v;
        }
        // B tile: op(B)(k, n) for k < 16, n < 64
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            int n, kk;
            if (!TB) { n = t & 63; kk = (t >> 6) + 4 * i; }
            else { kk = t & 15; n = (t >> 4) + 16 * i; }
            const int gn = n0 + n, gk = k0 + kk;
            T v = T(0);
            if (gn < N && gk < K) v = TB ? B[(long long)gn * ldb + gk] : B[(long long)gk * ldb + gn];
            Bs[kk][n] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            T a[4], bb[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = As[kk][ty + 16 * u];
#pragma unroll
            for (int v = 0; v < 4; ++v) bb[v] = Bs[kk][tx + 16 * v];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], bb[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int gm = m0 + ty + 16 * u;
        if (gm >= M) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int gn = n0 + tx + 16 * v;
            if (gn >= N) continue;
            T *c = &C[(long long)gm * ldc + gn];
            *c = (beta == T(0)) ? alpha * acc[u][v] : fma(alpha, acc[u][v], beta * *c);
        }
    }
}

template <typename T, bool TA, bool TB>
void launch(cudaStream_t st, int M, int N, int K, T alpha, const T *A, int lda, long long sA,
            const T *B, int ldb, long long sB, T beta, T *C, int ldc, long long sC, int batch) {
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, batch);
    gemm_kernel<T, TA, TB><<<grid, 256, 0, st>>>(M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C,
                                                  ldc, sC);
    check_launch("gemm_kernel");
}

}  // namespace

template <typename T>
void gemm(cudaStream_t st, bool ta, bool tb, int M, int N, int K, T alpha, const T *A, int lda,
          long long sA, const T *B, int ldb, long long sB, T beta, T *C, int ldc, long long sC,
          int batch, bool approx) {
    if (M <= 0 || N <= 0 || batch <= 0) return;
    const double bytes = sizeof(T) * ((double)M * K * (sA ? batch : 1) + (double)K * N * (sB ? batch : 1) +
                                      (double)M * N * batch * (beta == T(0) ? 1 : 2));
    ProfScope ps(st, ST_GEMM, 2.0 * M * N * K * batch, bytes);
    // float32 products of useful size go to the tensor cores (three-term TF32 split: float32
    // accuracy); float64 and tiny products stay on the CUDA cores
    if (sizeof(T) == 4 && tc_enabled() && (double)M * N * K * batch >= 2.0e6) {
        tc_gemm(st, ta, tb, M, N, K, (float)alpha, (const float *)A, lda, sA, (const float *)B, ldb, sB,
                (float)beta, (float *)C, ldc, sC, batch, !approx);
        return;
    }
    if (!ta && !tb) launch<T, false, false>(st, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch);
    else if (!ta && tb) launch<T, false, true>(st, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch);
    else if (ta && !tb) launch<T, true, false>(st, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch);
    else launch<T, true, true>(st, M, N, K, alpha, A, lda, sA, B, ldb, sB, beta, C, ldc, sC, batch);
}

template void gemm<float>(cudaStream_t, bool, bool, int, int, int, float, const float *, int,
                          long long, const float *, int, long long, float, float *, int,
                          long long, int, bool);
template void gemm<double>(cudaStream_t, bool, bool, int, int, int, double, const double *, int,
                           long long, const double *, int, long long, double, double *, int,
                           long long, int, bool);

}  // namespace tddft
