// Block-sparse products of the truncated form on the tensor cores (sm_103a, tcgen05 kind::tf32):
//
//   C[b][o] = mask[o] * (alpha * sum over the pairs (i, j) of o of A[b][i] Bt[b][j]^T + beta * C[b][o])
//
// over the listed output blocks o of a cluster-blocked matrix (Sec. IV's truncated products: only
// pairs of present blocks are multiplied, and the result is cut to the pattern of C by the mask).
// A blocks are 128 x BK and Bt blocks 64 x BK, both K contiguous; C blocks 128 x 64, row-major.
// Float32 accuracy by the three-term TF32 split made in shared memory (as in the dense kernel:
// x = hi + lo, hi = x rounded to tf32, three MMAs per product); `approx` takes one MMA.
//
// Persistent, one CTA of 320 threads per SM over (output block, batch entry) tiles: warp 8 lane 0
// issues the TMA loads (one 32-wide K slice of an A block and of a Bt block per stage), warps 4-7
// split them, warp 9 allocates TMEM and its lane 0 issues the MMAs into one of two 64-column
// accumulators, warps 0-3 read the accumulator out (lane = row), apply alpha, beta and the mask
// and store the block through shared memory so that each store is one 256-byte row. Every wait is
// bounded; after an expired wait the loads and MMAs in flight are drained, TMEM is freed and the
// error word is set.
#include "sparse.h"
#include "tc_common.cuh"

#include <cuda.h>

#include <algorithm>

namespace tddft {

bool encode_map_3d_f32(CUtensorMap *map, const float *ptr, unsigned long long d0, unsigned long long d1,
                       unsigned long long d2, unsigned long long s1_bytes, unsigned long long s2_bytes, unsigned b0,
                       unsigned b1);
int *tc_error_word();
bool tc_gemm_available();

namespace {

using namespace tc;

constexpr int BT_THREADS = 320;
constexpr int BT_STAGES = 4;
constexpr int A_BYTES = 128 * 32 * 4;   // 16 KB: one K slice of an A block
constexpr int B_BYTES = 64 * 32 * 4;    // 8 KB: one K slice of a Bt block

struct __align__(8) BtShared {
    unsigned long long full[BT_STAGES];
    unsigned long long split[BT_STAGES];
    unsigned long long empty[BT_STAGES];
    unsigned long long acc_full[2];
    unsigned long long acc_empty[2];
    unsigned long long drain;
    unsigned int tmem_base;
    int abort;
};

__device__ __forceinline__ float tf32_hi(float x) {
    unsigned r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

template <int NSPLIT>
__host__ __device__ constexpr int stage_bytes() {
    return NSPLIT == 3 ? 2 * (A_BYTES + B_BYTES) : A_BYTES + B_BYTES;
}

template <int NSPLIT>
__global__ void __launch_bounds__(BT_THREADS, 1) bsr_tc_kernel(
    const __grid_constant__ CUtensorMap mA, const __grid_constant__ CUtensorMap mB, int nks,
    const int *__restrict__ out, const int *__restrict__ ptr, const int *__restrict__ pa,
    const int *__restrict__ pb, int nout, int nb, int offA, int offB, float alpha, float beta,
    float *__restrict__ C, long long sC, const float *__restrict__ mask, int *err, long long wlim) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<unsigned long long>(smem_raw) + 1023ull) & ~1023ull);
    constexpr int SB = stage_bytes<NSPLIT>();
    unsigned char *tiles = base;
    float *staging = reinterpret_cast<float *>(base + (size_t)BT_STAGES * SB);   // 4 warps x 32 x 33
    BtShared *ctl = reinterpret_cast<BtShared *>(staging + 4 * 32 * 33);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntiles = nout * nb;
    volatile int *abort = &ctl->abort;

    if (threadIdx.x == 0) {
        for (int s = 0; s < BT_STAGES; ++s) {
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
                     "r"(128));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = ctl->tmem_base;

    if (warp == 8) {
        if (lane == 0) {
            long long it = 0;
            bool go = true;
            for (int t = blockIdx.x; t < ntiles && go; t += gridDim.x) {
                const int oi = t % nout, b = t / nout;
                for (int j = ptr[oi]; j < ptr[oi + 1] && go; ++j) {
                    const int ia = pa[j] + b * offA, ib = pb[j] + b * offB;
                    for (int ks = 0; ks < nks; ++ks, ++it) {
                        const int s = (int)(it % BT_STAGES);
                        const unsigned par = (unsigned)(((it / BT_STAGES) & 1) ^ 1);
                        if (!mbar_wait(&ctl->empty[s], par, abort, wlim)) {
                            go = false;
                            break;
                        }
                        unsigned char *st = tiles + (size_t)s * SB;
                        mbar_expect_tx(&ctl->full[s], A_BYTES + B_BYTES);
                        tma_load_3d(st, &mA, &ctl->full[s], ks * 32, 0, ia);
                        tma_load_3d(st + A_BYTES, &mB, &ctl->full[s], ks * 32, 0, ib);
                    }
                }
            }
            if (*abort)
                for (long long j = it > BT_STAGES ? it - BT_STAGES : 0; j < it; ++j)
                    mbar_drain(&ctl->full[j % BT_STAGES], (unsigned)((j / BT_STAGES) & 1), wlim);
        }
    } else if (warp == 9) {
        if (lane == 0) {
            constexpr unsigned idesc = idesc_tf32(128, 64);
            long long it = 0;
            int tcount = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++tcount) {
                const int oi = t % nout;
                const int buf = tcount & 1, use = tcount >> 1;
                if (!mbar_wait(&ctl->acc_empty[buf], (unsigned)((use & 1) ^ 1), abort, wlim)) break;
                tc_fence_after();
                const unsigned acc_t = tmem + (unsigned)(buf * 64);
                const int nsl = (ptr[oi + 1] - ptr[oi]) * nks;
                for (int q = 0; q < nsl; ++q, ++it) {
                    const int s = (int)(it % BT_STAGES);
                    const unsigned par = (unsigned)((it / BT_STAGES) & 1);
                    if (!mbar_wait(NSPLIT == 3 ? &ctl->split[s] : &ctl->full[s], par, abort, wlim)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    unsigned char *st = tiles + (size_t)s * SB;
                    const unsigned a = smem_u32(st), bt = smem_u32(st + A_BYTES);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const unsigned off = kk * 32;   // 8 tf32 along K inside the 128-byte swizzle row
                        mma_tf32(acc_t, smem_desc(a + off), smem_desc(bt + off), idesc, (q > 0 || kk > 0) ? 1u : 0u);
                        if (NSPLIT == 3) {
                            const unsigned alo = smem_u32(st + A_BYTES + B_BYTES),
                                           blo = smem_u32(st + 2 * A_BYTES + B_BYTES);
                            mma_tf32(acc_t, smem_desc(a + off), smem_desc(blo + off), idesc, 1u);
                            mma_tf32(acc_t, smem_desc(alo + off), smem_desc(bt + off), idesc, 1u);
                        }
                    }
                    mma_commit(&ctl->empty[s]);
                }
                if (!ok) break;
                mma_commit(&ctl->acc_full[buf]);
            }
            if (*abort) {
                mma_commit(&ctl->drain);
                mbar_drain(&ctl->drain, 0, wlim);
            }
        }
    } else if (warp >= 4) {
        if (NSPLIT == 3) {
            // hi = rna_tf32(x) in place, lo = x - hi into the stage's lo tiles (same swizzle)
            const int ts = threadIdx.x - 128;
            long long it = 0;
            bool go = true;
            for (int t = blockIdx.x; t < ntiles && go; t += gridDim.x) {
                const int oi = t % nout;
                const int nsl = (ptr[oi + 1] - ptr[oi]) * nks;
                for (int q = 0; q < nsl; ++q, ++it) {
                    const int s = (int)(it % BT_STAGES);
                    const unsigned par = (unsigned)((it / BT_STAGES) & 1);
                    if (!mbar_wait(&ctl->full[s], par, abort, wlim)) {
                        go = false;
                        break;
                    }
                    unsigned char *st = tiles + (size_t)s * SB;
                    float4 *hi = reinterpret_cast<float4 *>(st);
                    float4 *lo = reinterpret_cast<float4 *>(st + A_BYTES + B_BYTES);
                    constexpr int nvec = (A_BYTES + B_BYTES) / 16;   // A and B slices are contiguous
#pragma unroll 4
                    for (int i = ts; i < nvec; i += 128) {
                        const float4 x = hi[i];
                        float4 h, l;
                        h.x = tf32_hi(x.x);
                        h.y = tf32_hi(x.y);
                        h.z = tf32_hi(x.z);
                        h.w = tf32_hi(x.w);
                        l.x = x.x - h.x;
                        l.y = x.y - h.y;
                        l.z = x.z - h.z;
                        l.w = x.w - h.w;
                        hi[i] = h;
                        lo[i] = l;
                    }
                    fence_async_smem();
                    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&ctl->split[s])) : "memory");
                }
            }
        }
    } else {
        // epilogue: TMEM -> registers -> 32 x 33 staging block per warp -> coalesced rows of C
        float *stg = staging + warp * 32 * 33;
        int tcount = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++tcount) {
            const int oi = t % nout, b = t / nout, o = out[oi];
            const int buf = tcount & 1, use = tcount >> 1;
            if (!mbar_wait(&ctl->acc_full[buf], (unsigned)(use & 1), abort, wlim)) break;
            tc_fence_after();
            float *Cb = C + (long long)b * sC + (long long)o * CB_SIZE + (long long)(warp * 32) * CB_C;
            const float *mb = mask ? mask + (long long)o * CB_SIZE + (long long)(warp * 32) * CB_C : nullptr;
            for (int c0 = 0; c0 < 64; c0 += 32) {
                float old[32];
                if (beta != 0.0f) {
#pragma unroll
                    for (int rr = 0; rr < 32; ++rr) old[rr] = Cb[rr * CB_C + c0 + lane];
                }
                float v[32];
                tmem_ld32(tmem + (unsigned)(buf * 64) + ((unsigned)(warp * 32) << 16) + (unsigned)c0, v);
#pragma unroll
                for (int j = 0; j < 32; ++j) stg[lane * 33 + j] = v[j];
                __syncwarp();
                if (beta != 0.0f) {
#pragma unroll
                    for (int rr = 0; rr < 32; ++rr) {
                        float x = fmaf(beta, old[rr], alpha * stg[rr * 33 + lane]);
                        if (mb) x *= mb[rr * CB_C + c0 + lane];
                        Cb[rr * CB_C + c0 + lane] = x;
                    }
                } else {
#pragma unroll 8
                    for (int rr = 0; rr < 32; ++rr) {
                        float x = alpha * stg[rr * 33 + lane];
                        if (mb) x *= mb[rr * CB_C + c0 + lane];
                        Cb[rr * CB_C + c0 + lane] = x;
                    }
                }
                __syncwarp();
            }
            tc_fence_before();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&ctl->acc_empty[buf])) : "memory");
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 9) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(128));
    }
    if (threadIdx.x == 0 && ctl->abort) atomicExch(err, 1);
}

// output blocks without pairs: C = mask (beta C)
__global__ void bsr_tc_empty_kernel(const int *__restrict__ empty, float *__restrict__ C, long long sC, float beta,
                                    const float *__restrict__ mask) {
    const int o = empty[blockIdx.x];
    float *Cb = C + (long long)blockIdx.y * sC + (long long)o * CB_SIZE;
    const float *mb = mask ? mask + (long long)o * CB_SIZE : nullptr;
    for (int i = threadIdx.x; i < CB_SIZE; i += blockDim.x) {
        float v = beta == 0.0f ? 0.0f : beta * Cb[i];
        if (mb) v *= mb[i];
        Cb[i] = v;
    }
}

template <int NSPLIT>
size_t bt_smem() {
    return 1024 + (size_t)BT_STAGES * stage_bytes<NSPLIT>() + 4 * 32 * 33 * sizeof(float) + sizeof(BtShared);
}

int sm_count_bt() {
    static const int n = []() {
        int dev = 0, v = 0;
        check(cudaGetDevice(&dev), "cudaGetDevice");
        check(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev), "SM count");
        return v;
    }();
    return n;
}

}  // namespace

bool bsr_tc_available() { return tc_gemm_available(); }

void bsr_tc(cudaStream_t st, int BK, const PairList &pl, int nblk_A, const float *A, long long sA, int nblk_B,
            const float *Bt, long long sB, float *C, long long sC, int nb, float alpha, float beta, const float *mask,
            bool approx) {
    if (nb <= 0) return;
    if (BK != 64 && BK != 128) throw CudaError{cudaErrorInvalidValue, "bsr_tc: K block must be 64 or 128"};
    if ((sA && sA != (long long)nblk_A * 128 * BK) || (sB && sB != (long long)nblk_B * 64 * BK))
        throw CudaError{cudaErrorInvalidValue, "bsr_tc: batch strides must be whole block lists"};
    if (pl.nempty > 0) {
        for (int o0 = 0; o0 < pl.nempty; o0 += 65535)
            for (int b0 = 0; b0 < nb; b0 += 65535) {
                dim3 grid(std::min(65535, pl.nempty - o0), std::min(65535, nb - b0));
                bsr_tc_empty_kernel<<<grid, 256, 0, st>>>(pl.empty + o0, C + b0 * sC, sC, beta, mask);
                check_launch("bsr_tc_empty_kernel");
            }
    }
    if (pl.nout == 0) return;
    const unsigned long long nA = (unsigned long long)nblk_A * (sA ? nb : 1), nB = (unsigned long long)nblk_B * (sB ? nb : 1);
    CUtensorMap ma, mb;
    if (!encode_map_3d_f32(&ma, A, BK, 128, nA, (unsigned long long)BK * 4, (unsigned long long)BK * 4 * 128, 32, 128) ||
        !encode_map_3d_f32(&mb, Bt, BK, 64, nB, (unsigned long long)BK * 4, (unsigned long long)BK * 4 * 64, 32, 64))
        throw CudaError{cudaErrorInvalidValue, "cuTensorMapEncodeTiled (bsr)"};
    static const bool attrs = []() {
        check(cudaFuncSetAttribute(bsr_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bt_smem<1>()),
              "attr bsr_tc 1");
        check(cudaFuncSetAttribute(bsr_tc_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bt_smem<3>()),
              "attr bsr_tc 3");
        return true;
    }();
    (void)attrs;
    const long long ntiles = (long long)pl.nout * nb;
    if (ntiles > (1LL << 31) - 1) throw CudaError{cudaErrorInvalidValue, "bsr_tc: too many output tiles"};
    const int grid = (int)std::min<long long>(ntiles, sm_count_bt());
    const int offA = sA ? nblk_A : 0, offB = sB ? nblk_B : 0;
    if (approx)
        bsr_tc_kernel<1><<<grid, BT_THREADS, bt_smem<1>(), st>>>(ma, mb, BK / 32, pl.out, pl.ptr, pl.pa, pl.pb, pl.nout,
                                                                 nb, offA, offB, alpha, beta, C, sC, mask,
                                                                 tc_error_word(), active_wait_limit());
    else
        bsr_tc_kernel<3><<<grid, BT_THREADS, bt_smem<3>(), st>>>(ma, mb, BK / 32, pl.out, pl.ptr, pl.pa, pl.pb, pl.nout,
                                                                 nb, offA, offB, alpha, beta, C, sC, mask,
                                                                 tc_error_word(), active_wait_limit());
    check_launch("bsr_tc_kernel");
}

}  // namespace tddft
