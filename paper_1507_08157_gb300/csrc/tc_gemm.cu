// Tensor-core GEMM for sm_103a: tcgen05.mma (kind::tf32) with TMA-staged operands and a TMEM
// accumulator, float32 in and out, float32 accuracy by the three-term TF32 split.
//
//   C[b] = alpha * A[b] * B[b]^T + beta * C[b]      A: M x K, B: N x K, both K contiguous.
//
// The split: x = x_hi + x_lo with x_hi = x rounded to tf32 (cvt.rna.tf32.f32, low 13 mantissa
// bits zero) and x_lo = x - x_hi (exact in float32, |x_lo| <= 2^-11 |x|). Then
// x*y ~= x_hi y_hi + x_hi y_lo + x_lo y_hi; the dropped x_lo y_lo term and the tf32 reading of the
// lo parts leave a relative error of about 2^-21 per product (plain TF32: 2^-11).
//
// The split is made inside the kernel: TMA brings the raw float32 tiles of A and B, warps 0-3
// round each element to tf32 in place (hi) and write x - hi into a second tile of the same
// swizzled layout (lo), so the operands cross L2 once, as float32.
//
// Persistent kernel, one CTA of 320 threads per SM looping over 128 x 128 output tiles (n
// fastest, then m, then the batch): warps 0-3 read the accumulator out of TMEM (warp w owns
// lanes 32w..32w+31, i.e. tile rows) and write C through a shared-memory block so that each
// store covers 128 contiguous bytes of a row; warps 4-7 split the staged tiles; warp 8 lane 0
// issues the TMA loads; warp 9 allocates TMEM and its lane 0 issues the MMAs. Two TMEM
// accumulators let the epilogue of one tile overlap the MMAs of the next. K in slices of 32
// floats (one 128-byte swizzle row), mbarrier ring of 3 stages (split) or 4 (plain TF32). Every
// wait is bounded: on expiry the block records an error and skips to the teardown, which always
// frees TMEM.
#include "tc_common.cuh"
#include "tddft_internal.h"

#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

namespace tddft {

namespace {

constexpr int TBM = 128, TBN = 128, TBK = 32;
template <int NSPLIT> __host__ __device__ constexpr int stages() { return NSPLIT == 1 ? 4 : 3; }
constexpr int TSTAGES = 4;   // control-block capacity (>= stages<NSPLIT>())
constexpr int TILE_BYTES = TBM * TBK * 4;                  // 16 KB per operand tile

struct __align__(8) TcShared {
    unsigned long long full[TSTAGES];
    unsigned long long split[TSTAGES];
    unsigned long long empty[TSTAGES];
    unsigned long long acc_full[2];
    unsigned long long acc_empty[2];
    unsigned long long drain;      // MMA completion after an abort (teardown only)
    unsigned int tmem_base;
    int abort;
};

constexpr int GEMM_THREADS = 320;
constexpr int STAGE_FLOATS = 4 * 32 * 33;      // epilogue staging: one 32 x 33 block per warp

using namespace tc;

__device__ __forceinline__ float tf32_rna_dev(float x) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// NSPLIT = 1: plain TF32 on the raw tiles; 3: three-term split, hi/lo made in shared memory
// With the split, an operand is either raw (split here) or arrives split (hi and lo maps):
// a_split / b_split select the latter.
// TN: output tile width (128, or 112 when N is a multiple of 112, so that N = 560 needs no padding)
template <int NSPLIT, int TN>
__global__ void __launch_bounds__(GEMM_THREADS, 1) tc_gemm_kernel(
    const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB,
    const __grid_constant__ CUtensorMap mAlo, const __grid_constant__ CUtensorMap mBlo, int a_split, int b_split,
    int M, int N, int K, int batchA, int batchB, int batch, float alpha, float beta, float *__restrict__ C, int ldc,
    long long sC, int *err, long long wlim) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<unsigned long long>(smem_raw) + 1023ull) & ~1023ull);
    constexpr int NT = NSPLIT == 1 ? 2 : 4;   // operand tiles per stage: A, B (hi in place), A lo, B lo
    constexpr int S = stages<NSPLIT>();
    unsigned char *tiles = base;
    float *staging = reinterpret_cast<float *>(base + (size_t)S * NT * TILE_BYTES);
    TcShared *ctl = reinterpret_cast<TcShared *>(staging + STAGE_FLOATS);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tn = (N + TN - 1) / TN, tm = (M + TBM - 1) / TBM;
    const int ntiles = tn * tm * batch;
    const int nk = (K + TBK - 1) / TBK;
    volatile int *abort = &ctl->abort;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&ctl->full[s], 1);
            mbar_init(&ctl->split[s], 128);
            mbar_init(&ctl->empty[s], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&ctl->acc_full[i], 1);
            mbar_init(&ctl->acc_empty[i], 128);
        }
        mbar_init(&ctl->drain, 1);
        ctl->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 9) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ctl->tmem_base)),
                     "r"(2 * TBN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = ctl->tmem_base;

    if (warp == 8) {
        if (lane == 0) {
            // TMA producer: raw float32 tiles of A and B, for every K slice of every tile
            long long it = 0;
            bool go = true;
            for (int t = blockIdx.x; t < ntiles && go; t += gridDim.x) {
                const int n0 = (t % tn) * TN, m0 = ((t / tn) % tm) * TBM, b = t / (tn * tm);
                const int ba = batchA > 1 ? b : 0, bb = batchB > 1 ? b : 0;
                for (int kb = 0; kb < nk; ++kb, ++it) {
                    const int s = (int)(it % S);
                    const unsigned par = (unsigned)(((it / S) & 1) ^ 1);
                    if (!mbar_wait(&ctl->empty[s], par, abort, wlim)) {
                        go = false;
                        break;
                    }
                    unsigned char *st = tiles + (size_t)s * NT * TILE_BYTES;
                    const int bytes = TILE_BYTES * (1 + (NSPLIT == 3 ? a_split : 0)) +
                                      TN * TBK * 4 * (1 + (NSPLIT == 3 ? b_split : 0));
                    mbar_expect_tx(&ctl->full[s], bytes);
                    tma_load_3d(st, &mA, &ctl->full[s], kb * TBK, m0, ba);
                    tma_load_3d(st + TILE_BYTES, &mB, &ctl->full[s], kb * TBK, n0, bb);
                    if (NSPLIT == 3 && a_split) tma_load_3d(st + 2 * TILE_BYTES, &mAlo, &ctl->full[s], kb * TBK, m0, ba);
                    if (NSPLIT == 3 && b_split) tma_load_3d(st + 3 * TILE_BYTES, &mBlo, &ctl->full[s], kb * TBK, n0, bb);
                }
            }
            // after an abort, the loads already issued land before the block exits
            if (*abort)
                for (long long j = it > S ? it - S : 0; j < it; ++j)
                    mbar_drain(&ctl->full[j % S], (unsigned)((j / S) & 1), wlim);
        }
    } else if (warp == 9) {
        if (lane == 0) {
            // MMA issuer: accumulator tcount % 2 per tile
            constexpr unsigned idesc = idesc_tf32(TBM, TN);
            long long it = 0;
            int tcount = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++tcount) {
                const int buf = tcount & 1, use = tcount >> 1;
                if (!mbar_wait(&ctl->acc_empty[buf], (unsigned)((use & 1) ^ 1), abort, wlim)) break;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const unsigned acc_t = tmem + (unsigned)(buf * TBN);
                for (int kb = 0; kb < nk; ++kb, ++it) {
                    const int s = (int)(it % S);
                    const unsigned par = (unsigned)((it / S) & 1);
                    if (!mbar_wait(NSPLIT == 3 ? &ctl->split[s] : &ctl->full[s], par, abort, wlim)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    unsigned char *st = tiles + (size_t)s * NT * TILE_BYTES;
                    const unsigned a = smem_u32(st), bt = smem_u32(st + TILE_BYTES);
#pragma unroll
                    for (int kk = 0; kk < TBK / 8; ++kk) {
                        const unsigned off = kk * 32;   // 8 tf32 = 32 bytes along K inside the swizzle row
                        const unsigned acc = (kb > 0 || kk > 0) ? 1u : 0u;
                        mma_tf32(acc_t, smem_desc(a + off), smem_desc(bt + off), idesc, acc);
                        if (NSPLIT == 3) {
                            const unsigned alo = smem_u32(st + 2 * TILE_BYTES), blo = smem_u32(st + 3 * TILE_BYTES);
                            mma_tf32(acc_t, smem_desc(a + off), smem_desc(blo + off), idesc, 1u);
                            mma_tf32(acc_t, smem_desc(alo + off), smem_desc(bt + off), idesc, 1u);
                        }
                    }
                    mma_commit(&ctl->empty[s]);
                }
                if (!ok) break;
                mma_commit(&ctl->acc_full[buf]);
            }
            // after an abort, the MMAs already issued finish before TMEM is freed
            if (*abort) {
                mma_commit(&ctl->drain);
                mbar_drain(&ctl->drain, 0, wlim);
            }
        }
    } else if (warp >= 4) {
        if (NSPLIT == 3) {
            // split each staged pair of tiles: hi = rna_tf32(x) in place, lo = x - hi alongside
            // (an element-wise map, so the swizzled layout carries over unchanged)
            const int ts = threadIdx.x - 128;
            long long it = 0;
            bool go = true;
            for (int t = blockIdx.x; t < ntiles && go; t += gridDim.x) {
                for (int kb = 0; kb < nk; ++kb, ++it) {
                    const int s = (int)(it % S);
                    const unsigned par = (unsigned)((it / S) & 1);
                    if (!mbar_wait(&ctl->full[s], par, abort, wlim)) {
                        go = false;
                        break;
                    }
                    unsigned char *st = tiles + (size_t)s * NT * TILE_BYTES;
#pragma unroll
                    for (int op = 0; op < 2; ++op) {
                        if (op == 0 ? a_split : b_split) continue;   // arrived split
                        float4 *hi = reinterpret_cast<float4 *>(st + op * TILE_BYTES);
                        float4 *lo = reinterpret_cast<float4 *>(st + (2 + op) * TILE_BYTES);
                        const int nvec = (op == 0 ? TBM : TN) * TBK / 4;
#pragma unroll 4
                        for (int i = ts; i < nvec; i += 128) {
                            const float4 x = hi[i];
                            float4 h, l;
                            h.x = tf32_rna_dev(x.x);
                            h.y = tf32_rna_dev(x.y);
                            h.z = tf32_rna_dev(x.z);
                            h.w = tf32_rna_dev(x.w);
                            l.x = x.x - h.x;
                            l.y = x.y - h.y;
                            l.z = x.z - h.z;
                            l.w = x.w - h.w;
                            hi[i] = h;
                            lo[i] = l;
                        }
                    }
                    fence_async_smem();
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&ctl->split[s])) : "memory");
                }
            }
        }
    } else {
        // epilogue (warps 0-3): TMEM -> registers -> 32 x 32 staging block -> C rows
        float *stg = staging + warp * 32 * 33;
        int tcount = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++tcount) {
            const int buf = tcount & 1, use = tcount >> 1;
            if (!mbar_wait(&ctl->acc_full[buf], (unsigned)(use & 1), abort, wlim)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int n0 = (t % tn) * TN, m0 = ((t / tn) % tm) * TBM, b = t / (tn * tm);
            float *Cb = C + (long long)b * sC;
            for (int c0 = 0; c0 < TN; c0 += 32) {
                const int col = n0 + c0 + lane;
                const bool colok = c0 + lane < TN && col < N;
                const int nrow = min(32, M - (m0 + warp * 32));   // rows of this warp inside C
                float *cw = Cb + (long long)(m0 + warp * 32) * ldc + col;
                // with beta, read the 32 old values of this column strip first: independent loads
                // in flight together, instead of one round trip per row behind each store
                float old[32];
                if (beta != 0.0f) {
#pragma unroll
                    for (int rr = 0; rr < 32; ++rr)
                        old[rr] = (rr < nrow && colok) ? cw[(long long)rr * ldc] : 0.0f;
                }
                float v[32];
                tmem_ld32(tmem + (unsigned)(buf * TBN) + ((unsigned)(warp * 32) << 16) + (unsigned)c0, v);
#pragma unroll
                for (int j = 0; j < 32; ++j) stg[lane * 33 + j] = v[j];
                __syncwarp();
                if (beta == 0.0f) {
#pragma unroll 8
                    for (int rr = 0; rr < 32; ++rr)
                        if (rr < nrow && colok) cw[(long long)rr * ldc] = alpha * stg[rr * 33 + lane];
                } else {
#pragma unroll
                    for (int rr = 0; rr < 32; ++rr)
                        if (rr < nrow && colok) cw[(long long)rr * ldc] = fmaf(alpha, stg[rr * 33 + lane], beta * old[rr]);
                }
                __syncwarp();
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&ctl->acc_empty[buf])) : "memory");
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 9) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TBN));
    }
    if (threadIdx.x == 0 && ctl->abort) atomicExch(err, 1);
}

// ---- host side ---------------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, []() {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 3-D map over [batch][rows][K] float32 with row stride ld and batch stride sb (elements);
// box 32 (K) x 128 rows x 1, 128-byte swizzle, zero fill outside.
bool make_map(CUtensorMap *map, const float *ptr, int K, int rows, int ld, long long sb, int batch, int box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)(batch > 0 ? batch : 1)};
    const long long bs = (batch > 1) ? sb * 4 : (long long)ld * rows * 4;
    cuuint64_t strides[2] = {(cuuint64_t)ld * 4, (cuuint64_t)(bs > 0 ? ((bs + 15) / 16) * 16 : 16)};
    cuuint32_t box[3] = {TBK, (cuuint32_t)box_rows, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(ptr), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

size_t tc_smem(int nsplit) {
    return (nsplit == 1 ? (size_t)stages<1>() * 2 : (size_t)stages<3>() * 4) * TILE_BYTES +
           STAGE_FLOATS * sizeof(float) + sizeof(TcShared) + 1024;
}

int sm_count() {
    static const int n = []() {
        int dev = 0, v = 0;
        check(cudaGetDevice(&dev), "cudaGetDevice");
        check(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev), "SM count");
        return v;
    }();
    return n;
}

int *error_word() {
    static int *const w = []() {
        int *p = nullptr;
        check(cudaMalloc(&p, sizeof(int)), "cudaMalloc tc error word");
        check(cudaMemset(p, 0, sizeof(int)), "memset tc error word");
        return p;
    }();
    return w;
}

}  // namespace

bool tc_gemm_available() { return encode_fn() != nullptr; }

// 3-D tiled float32 map, 128-byte swizzle, zero fill outside: dims d0 (contiguous) x d1 x d2,
// strides of dims 1 and 2 in bytes, box b0 x b1 x 1
bool encode_map_3d_f32(CUtensorMap *map, const float *ptr, unsigned long long d0, unsigned long long d1,
                       unsigned long long d2, unsigned long long s1_bytes, unsigned long long s2_bytes, unsigned b0,
                       unsigned b1) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[3] = {d0, d1, d2};
    cuuint64_t strides[2] = {s1_bytes, s2_bytes};
    cuuint32_t box[3] = {b0, b1, 1};
    cuuint32_t estr[3] = {1, 1, 1};
    return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float *>(ptr), dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 2-D tiled map, 128-byte swizzle, zero fill outside: `inner` elements per row (contiguous),
// `rows` rows `row_bytes` apart; box box_inner x box_rows
bool encode_map_2d(CUtensorMap *map, CUtensorMapDataType dt, const void *ptr, unsigned long long inner,
                   unsigned long long rows, unsigned long long row_bytes, unsigned box_inner, unsigned box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {inner, rows};
    cuuint64_t strides[1] = {row_bytes};
    cuuint32_t box[2] = {box_inner, box_rows};
    cuuint32_t estr[2] = {1, 1};
    return fn(map, dt, 2, const_cast<void *>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
              CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// C[b] = alpha * A[b] B[b]^T + beta C[b] with A (M x K, ld lda, batch stride sA; 0 = shared) and
// B (N x K, ldb, sB), both K-contiguous. split: three-term TF32 split; an operand with a lo part
// (Alo / Blo non-null, same layout) arrives split, one without is split inside the kernel.
// Rows must start on 16-byte boundaries: lda, ldb, sA, sB multiples of 4 and the pointers
// 16-byte aligned.
void tc_gemm_nt(cudaStream_t st, int M, int N, int K, float alpha, const float *A, const float *Alo, int lda,
                long long sA, const float *B, const float *Blo, int ldb, long long sB, float beta, float *C, int ldc,
                long long sC, int batch, bool split) {
    const int nsplit = split ? 3 : 1;
    const int TN = (N % 112 == 0) ? 112 : 128;
    CUtensorMap ma, mb, malo, mblo;
    const int bA = sA ? batch : 1, bB = sB ? batch : 1;
    if (!make_map(&ma, A, K, M, lda, sA, bA, TBM) || !make_map(&mb, B, K, N, ldb, sB, bB, TN))
        throw CudaError{cudaErrorInvalidValue, "cuTensorMapEncodeTiled"};
    const bool asp = split && Alo, bsp = split && Blo;
    if ((asp && !make_map(&malo, Alo, K, M, lda, sA, bA, TBM)) || (bsp && !make_map(&mblo, Blo, K, N, ldb, sB, bB, TN)))
        throw CudaError{cudaErrorInvalidValue, "cuTensorMapEncodeTiled (lo)"};
    if (!asp) malo = ma;
    if (!bsp) mblo = mb;
    const size_t sm = tc_smem(nsplit);
    static const bool attrs = [&]() {   // once per process, thread-safe
        check(cudaFuncSetAttribute(tc_gemm_kernel<1, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem(1)),
              "attr tc1");
        check(cudaFuncSetAttribute(tc_gemm_kernel<1, 112>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem(1)),
              "attr tc1");
        check(cudaFuncSetAttribute(tc_gemm_kernel<3, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem(3)),
              "attr tc3");
        check(cudaFuncSetAttribute(tc_gemm_kernel<3, 112>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem(3)),
              "attr tc3");
        return true;
    }();
    (void)attrs;
    const long long ntiles = (long long)((N + TN - 1) / TN) * ((M + TBM - 1) / TBM) * batch;
    const int grid = (int)std::min<long long>(ntiles, sm_count());
    int *err = error_word();
    const long long wlim = active_wait_limit();
    const int as = asp ? 1 : 0, bs = bsp ? 1 : 0;
    if (nsplit == 3 && TN == 112)
        tc_gemm_kernel<3, 112><<<grid, GEMM_THREADS, sm, st>>>(ma, mb, malo, mblo, as, bs, M, N, K, bA, bB, batch,
                                                               alpha, beta, C, ldc, sC, err, wlim);
    else if (nsplit == 3)
        tc_gemm_kernel<3, 128><<<grid, GEMM_THREADS, sm, st>>>(ma, mb, malo, mblo, as, bs, M, N, K, bA, bB, batch,
                                                               alpha, beta, C, ldc, sC, err, wlim);
    else if (TN == 112)
        tc_gemm_kernel<1, 112><<<grid, GEMM_THREADS, sm, st>>>(ma, mb, malo, mblo, 0, 0, M, N, K, bA, bB, batch, alpha,
                                                               beta, C, ldc, sC, err, wlim);
    else
        tc_gemm_kernel<1, 128><<<grid, GEMM_THREADS, sm, st>>>(ma, mb, malo, mblo, 0, 0, M, N, K, bA, bB, batch, alpha,
                                                               beta, C, ldc, sC, err, wlim);
    check_launch("tc_gemm_kernel");
}

namespace {

__device__ __forceinline__ float tf32_rna(float x) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// hi/lo split of nb matrices (rows x cols, ld / s_in) into row-major outputs of row length ldo
// (>= cols, the pad written as zeros)
__global__ void split_kernel(const float *__restrict__ in, int rows, int cols, int ld, long long s_in,
                             float *__restrict__ hi, float *__restrict__ lo, int ldo, long long s_out, int nb) {
    const long long per = (long long)rows * ldo, tot = per * nb;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot;
         i += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(i / per);
        const long long r = (i - b * per) / ldo, c = (i - b * per) - r * ldo;
        const float x = c < cols ? in[b * s_in + r * ld + c] : 0.0f;
        if (lo) {
            const float h = tf32_rna(x);
            hi[b * s_out + r * ldo + c] = h;
            lo[b * s_out + r * ldo + c] = x - h;
        } else {
            hi[b * s_out + r * ldo + c] = x;
        }
    }
}

// out[b][c][r] = in[b][r][c] (32 x 32 tiles through shared memory), rows of the output padded to
// ldo (>= rows) with zeros, with the hi/lo split when lo is given
__global__ void transpose_split_kernel(const float *__restrict__ in, int rows, int cols, int ld,
                                       long long s_in, float *__restrict__ hi, float *__restrict__ lo,
                                       int ldo, long long s_out) {
    __shared__ float t[32][33];
    const int b = blockIdx.z;
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    const float *src = in + (long long)b * s_in;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        t[i][threadIdx.x] = (r < rows && c < cols) ? src[(long long)r * ld + c] : 0.0f;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (c < cols && r < ldo) {
            const float x = t[threadIdx.x][i];
            const long long o = (long long)b * s_out + (long long)c * ldo + r;
            if (lo) {
                const float h = tf32_rna(x);
                hi[o] = h;
                lo[o] = x - h;
            } else {
                hi[o] = x;
            }
        }
    }
}

// scratch for the split operands, one buffer per stream (grown on demand, never shrunk): work on
// one stream runs in order, so its products may share a buffer, while products on different
// streams (the contexts of a batch) run concurrently and must not
struct Scratch {
    float *p = nullptr;
    size_t cap = 0;
    float *get(size_t n) {
        if (n > cap) {
            if (p) cudaFree(p);   // synchronises the device: earlier users of the buffer are done
            p = nullptr;
            check(cudaMalloc(&p, n * sizeof(float)), "cudaMalloc tc scratch");
            cap = n;
        }
        return p;
    }
};
std::mutex g_scratch_mu;
std::vector<std::pair<cudaStream_t, Scratch *>> g_scratch;
Scratch &scratch(cudaStream_t st) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    for (auto &e : g_scratch)
        if (e.first == st) return *e.second;
    g_scratch.push_back({st, new Scratch});
    return *g_scratch.back().second;
}

int grid1(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < 8 * 152 ? (b > 0 ? b : 1) : 8 * 152);
}

}  // namespace

// Operands registered as constant (matrices fixed for the life of a context) keep a K-major
// hi/lo copy, made on first use and freed when they are unregistered.
namespace {
struct SplitCopy {
    bool trans;
    int rows, cols, ld;
    float *hi, *lo;
    int kp;
};
std::mutex g_const_mu;
std::vector<std::pair<const float *, std::vector<SplitCopy>>> g_const;   // registered pointer -> copies

std::vector<SplitCopy> *const_entry(const float *p) {
    for (auto &e : g_const)
        if (e.first == p) return &e.second;
    return nullptr;
}

// hi/lo K-major copy of a constant operand: rows x K out of a (rows x K, !trans) or (K x rows,
// trans) matrix with leading dimension ld
bool const_split(cudaStream_t st, const float *p, bool trans, int rows, int K, int ld, SplitCopy *out) {
    std::lock_guard<std::mutex> lock(g_const_mu);
    std::vector<SplitCopy> *v = const_entry(p);
    if (!v) return false;
    for (const SplitCopy &c : *v)
        if (c.trans == trans && c.rows == rows && c.cols == K && c.ld == ld) {
            *out = c;
            return true;
        }
    SplitCopy c{trans, rows, K, ld, nullptr, nullptr, (K + 3) / 4 * 4};
    const size_t n = (size_t)rows * c.kp;
    check(cudaMalloc(&c.hi, n * sizeof(float)), "cudaMalloc constant split");
    check(cudaMalloc(&c.lo, n * sizeof(float)), "cudaMalloc constant split");
    if (!trans) {
        split_kernel<<<grid1((long long)n), 256, 0, st>>>(p, rows, K, ld, 0, c.hi, c.lo, c.kp, 0, 1);
    } else {
        dim3 g((rows + 31) / 32, (c.kp + 31) / 32, 1);
        transpose_split_kernel<<<g, dim3(32, 8), 0, st>>>(p, K, rows, ld, 0, c.hi, c.lo, c.kp, 0);
    }
    check_launch("constant split");
    v->push_back(c);
    *out = c;
    return true;
}
}  // namespace

void tc_register_constant(const float *p) {
    std::lock_guard<std::mutex> lock(g_const_mu);
    if (!const_entry(p)) g_const.push_back({p, {}});
}

void tc_unregister_constant(const float *p) {
    std::lock_guard<std::mutex> lock(g_const_mu);
    for (size_t i = 0; i < g_const.size(); ++i)
        if (g_const[i].first == p) {
            for (SplitCopy &c : g_const[i].second) {
                cudaFree(c.hi);
                cudaFree(c.lo);
            }
            g_const.erase(g_const.begin() + (long)i);
            return;
        }
}

// Dispatch of a row-major C[b] = alpha op(A[b]) op(B[b]) + beta C[b] onto the tensor cores. The
// kernel wants both operands K-contiguous with 16-byte row starts. A registered constant operand
// comes from its cached hi/lo copy; a K-contiguous variable operand goes in as it lies and is
// split inside the kernel; any other operand gets a hi/lo K-major copy in scratch.
void tc_gemm(cudaStream_t st, bool ta, bool tb, int M, int N, int K, float alpha, const float *A, int lda,
             long long sA, const float *B, int ldb, long long sB, float beta, float *C, int ldc, long long sC,
             int batch, bool split) {
    const int bA = sA ? batch : 1, bB = sB ? batch : 1;
    auto direct = [](const float *p, int ld, long long s) {
        return reinterpret_cast<unsigned long long>(p) % 16 == 0 && ld % 4 == 0 && s % 4 == 0;
    };
    SplitCopy cav{}, cbv{};
    const SplitCopy *ca = (split && bA == 1 && const_split(st, A, ta, M, K, lda, &cav)) ? &cav : nullptr;
    const SplitCopy *cb = (split && bB == 1 && const_split(st, B, !tb, N, K, ldb, &cbv)) ? &cbv : nullptr;
    const bool a_direct = !ca && !ta && direct(A, lda, sA), b_direct = !cb && tb && direct(B, ldb, sB);
    const bool a_copy = !ca && !a_direct, b_copy = !cb && !b_direct;
    const int Kp = (K + 3) / 4 * 4;                     // 16-byte rows for the tensor maps
    const int nsp = split ? 2 : 1;                      // copies carry hi and lo when splitting
    auto up64 = [](size_t n) { return (n + 63) / 64 * 64; };
    const size_t na = a_copy ? up64((size_t)M * Kp * bA) : 0, nbt = b_copy ? up64((size_t)N * Kp * bB) : 0;
    float *base = (na + nbt) ? scratch(st).get(nsp * (na + nbt)) : nullptr;
    const float *Ak = A, *Alo = nullptr, *Bk = B, *Blo = nullptr;
    int lak = lda, lbk = ldb;
    long long sak = sA, sbk = sB;
    if (ca) {
        Ak = ca->hi;
        Alo = ca->lo;
        lak = ca->kp;
        sak = 0;
    } else if (a_copy) {
        float *Ah = base, *Al = split ? base + na : nullptr;
        const long long sa = (long long)M * Kp;
        if (!ta) {
            split_kernel<<<grid1((long long)M * Kp * bA), 256, 0, st>>>(A, M, K, lda, sA, Ah, Al, Kp, sa, bA);
        } else {
            dim3 g((M + 31) / 32, (Kp + 31) / 32, bA);
            transpose_split_kernel<<<g, dim3(32, 8), 0, st>>>(A, K, M, lda, sA, Ah, Al, Kp, sa);
        }
        check_launch("tc copy A");
        Ak = Ah;
        Alo = Al;
        lak = Kp;
        sak = bA > 1 ? sa : 0;
    }
    if (cb) {
        Bk = cb->hi;
        Blo = cb->lo;
        lbk = cb->kp;
        sbk = 0;
    } else if (b_copy) {
        float *Bh = base + nsp * na, *Bl = split ? base + nsp * na + nbt : nullptr;
        const long long sb = (long long)N * Kp;
        if (tb) {
            split_kernel<<<grid1((long long)N * Kp * bB), 256, 0, st>>>(B, N, K, ldb, sB, Bh, Bl, Kp, sb, bB);
        } else {
            dim3 g((N + 31) / 32, (Kp + 31) / 32, bB);
            transpose_split_kernel<<<g, dim3(32, 8), 0, st>>>(B, K, N, ldb, sB, Bh, Bl, Kp, sb);
        }
        check_launch("tc copy B");
        Bk = Bh;
        Blo = Bl;
        lbk = Kp;
        sbk = bB > 1 ? sb : 0;
    }
    // both maps span the K real columns (copies are zero-padded to Kp; reads past K fill zeros)
    tc_gemm_nt(st, M, N, K, alpha, Ak, Alo, lak, sak, Bk, Blo, lbk, sbk, beta, C, ldc, sC, batch, split);
}

int *tc_error_word() { return error_word(); }

namespace {
// waits, with the caller's limit, on a barrier that nothing completes: the wait must expire and
// set the error word (a check of the bounded-wait path that faults nothing)
__global__ void wait_probe_kernel(int *err, long long wlim) {
    __shared__ unsigned long long bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile int *ab = &abort_flag;
        if (!mbar_wait(&bar, 0, ab, wlim)) atomicExch(err, 1);
    }
}
}  // namespace

void tc_wait_probe(cudaStream_t st) {
    wait_probe_kernel<<<1, 32, 0, st>>>(error_word(), active_wait_limit());
    check_launch("wait_probe_kernel");
}

void tc_error_fetch(cudaStream_t st, int *host) {
    check(cudaMemcpyAsync(host, error_word(), sizeof(int), cudaMemcpyDeviceToHost, st), "D2H tc error");
}

void tc_error_clear(cudaStream_t st) { check(cudaMemsetAsync(error_word(), 0, sizeof(int), st), "clear tc error"); }


// free the split scratch of a stream that is about to be destroyed (its work has completed)
void tc_release_stream(cudaStream_t st) {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    for (size_t i = 0; i < g_scratch.size(); ++i)
        if (g_scratch[i].first == st) {
            if (g_scratch[i].second->p) cudaFree(g_scratch[i].second->p);
            delete g_scratch[i].second;
            g_scratch.erase(g_scratch.begin() + (long)i);
            return;
        }
}

}  // namespace tddft
