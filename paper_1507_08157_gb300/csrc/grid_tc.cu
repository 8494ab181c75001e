// Response density on the tensor cores (mixed precision): rho_s(r) = sum_ab chi_a(r) P_s,ab phi_b(r)
// (paper Secs. II C, III A) as one tcgen05 kind::f16 product per 8^3 grid tile,
//
//   T[r][(s,b)] = sum_a X[r][a] P_s[a][b]        (M = tile points, K = chi functions of the tile,
//                                                  N = states x phi functions of the tile)
//   rho_s(r)    = sum_b T[r][(s,b)] Phi[b][r]     (epilogue, read out of TMEM lane by lane)
//
// Operands are float16 with float32 accumulation: the point-major chi block of the tile comes in
// by TMA (128-byte swizzle), the P block is gathered by the threads from the state matrices
// (scaled per state by a power of two so its largest entry is <= 1) and written in the same
// swizzled K-major layout. CTA = (state group, tile); consecutive CTAs share a tile so its chi
// block is read from HBM once and from L2 by the other groups. Every point is written by exactly
// one CTA per state (owner computes, no atomics). Waits are bounded; TMEM is always freed.
#include "tc_common.cuh"
#include "tddft_internal.h"

#include <cuda_fp16.h>

#include <algorithm>
#include <cstdlib>
#include <mutex>

namespace tddft {

using namespace tc;

namespace {

struct __align__(8) DensShared {
    unsigned long long a_full[4];
    unsigned long long a_empty[4];
    unsigned long long acc_full[2];
    unsigned long long acc_empty[2];
    unsigned long long b_ready[16];   // per 64-wide K block of the gathered P block
    unsigned long long drain;         // MMA completion after an abort (teardown only)
    unsigned int tmem_base;
    int abort;
};

constexpr int DENS_THREADS = 384;      // warps 0-3 and 8-11 gather + epilogue, 4 TMA, 5 MMA, 6-7 gather
constexpr int DENS_GATHER = 320;       // gathering threads: warps 0-3 and 6-11
constexpr int DENS_STAGES = 4;         // chi-block ring (16 KB each)
constexpr int DENS_KBMAX = 16;         // K blocks of the gathered P block (CK <= 1024)

__device__ __forceinline__ int gather_rank(int warp, int lane) { return (warp < 4 ? warp : warp - 2) * 32 + lane; }

__global__ void __launch_bounds__(DENS_THREADS, 1) density_tc_kernel(
    const __grid_constant__ CUtensorMap mX,   // point-major chi: [tile*512 + point][CK] f16
    int n, int nt, int KBmax, int NP, int G, int k, const int *__restrict__ coff, const int *__restrict__ cids,
    const int *__restrict__ poff, const int *__restrict__ pids, const float *__restrict__ pval, int nphi,
    const float *__restrict__ P, long long sP, const float *__restrict__ pscale, float *__restrict__ rho,
    int *err, int quad, const unsigned short *__restrict__ phi_pm, long long wlim) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<unsigned long long>(smem_raw) + 1023ull) & ~1023ull);
    const int t = blockIdx.y, grp = blockIdx.x;
    const int s0 = grp * G;
    const int gs = min(G, k - s0);                      // states in this group
    const int c0 = coff[t], nc = coff[t + 1] - c0;
    const int p0 = poff[t], np = poff[t + 1] - p0;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long n3 = (long long)n * n * n;
    const int tx = t / (nt * nt), ty = (t / nt) % nt, tz = t % nt;
    if (nc == 0 || np == 0) {
        for (int lp = threadIdx.x; lp < TILE_PTS; lp += blockDim.x) {
            const int gx = tx * TILE + (lp >> 6), gy = ty * TILE + ((lp >> 3) & 7), gz = tz * TILE + (lp & 7);
            if (gx < n && gy < n && gz < n)
                for (int s = 0; s < gs; ++s) rho[(long long)(s0 + s) * n3 + ((long long)gx * n + gy) * n + gz] = 0.0f;
        }
        return;
    }
    const int KB = (nc + 63) / 64;                       // 64-wide K blocks (128 bytes of f16)
    const int NB = G * NP;                               // B rows (multiple of 16, <= 256)
    unsigned char *A = base;                             // ring of DENS_STAGES x [128 rows x 128 B]
    unsigned char *B = base + DENS_STAGES * 16384;       // KBmax x [NB rows x 128 B]
    DensShared *ctl = reinterpret_cast<DensShared *>(B + (size_t)KBmax * NB * 128);
    volatile int *abort = &ctl->abort;

    if (threadIdx.x == 0) {
        for (int i = 0; i < DENS_STAGES; ++i) {
            mbar_init(&ctl->a_full[i], 1);
            mbar_init(&ctl->a_empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&ctl->acc_full[i], 1);
            mbar_init(&ctl->acc_empty[i], 256);
        }
        for (int i = 0; i < DENS_KBMAX; ++i) mbar_init(&ctl->b_ready[i], DENS_GATHER);
        mbar_init(&ctl->drain, 1);
        ctl->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ctl->tmem_base)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = ctl->tmem_base;

    if (warp == 4) {
        // TMA producer: chi blocks (pb, kb) through the ring
        if (lane == 0) {
            int i = 0;
            for (int pb = 0; pb < TILE_PTS / 128 && !*abort; ++pb)
                for (int kb = 0; kb < KB; ++kb, ++i) {
                    const int st = i % DENS_STAGES, use = i / DENS_STAGES;
                    if (use > 0 && !mbar_wait(&ctl->a_empty[st], (use - 1) & 1, abort, wlim)) break;
                    mbar_expect_tx(&ctl->a_full[st], 16384);
                    tma_load_2d(A + st * 16384, &mX, &ctl->a_full[st], kb * 64, t * TILE_PTS + pb * 128);
                }
            // after an abort, the loads already issued land before the block exits
            if (*abort)
                for (int j = i > DENS_STAGES ? i - DENS_STAGES : 0; j < i; ++j)
                    mbar_drain(&ctl->a_full[j % DENS_STAGES], (unsigned)((j / DENS_STAGES) & 1), wlim);
        }
    } else if (warp == 5) {
        // MMA issuer: accumulator pb % 2, one commit per chi block (frees the ring slot)
        if (lane == 0) {
            const unsigned idesc = idesc_f16(128, NB);
            bool ok = true;
            int i = 0;
            for (int pb = 0; pb < TILE_PTS / 128 && ok; ++pb) {
                const int acc = pb & 1, use = pb >> 1;
                if (use > 0 && !mbar_wait(&ctl->acc_empty[acc], (use - 1) & 1, abort, wlim)) break;
                tc_fence_after();
                for (int kb = 0; kb < KB; ++kb, ++i) {
                    const int st = i % DENS_STAGES, u = i / DENS_STAGES;
                    // the P block's K block kb is gathered (the first M block waits, the rest pass)
                    if (!mbar_wait(&ctl->b_ready[kb], 0, abort, wlim) || !mbar_wait(&ctl->a_full[st], u & 1, abort, wlim)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const unsigned a = smem_u32(A + st * 16384), bb = smem_u32(B + (size_t)kb * NB * 128);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma_f16(tmem + acc * 256, smem_desc(a + kk * 32), smem_desc(bb + kk * 32), idesc,
                                (kb > 0 || kk > 0) ? 1u : 0u);
                    mma_commit(&ctl->a_empty[st]);
                }
                mma_commit(&ctl->acc_full[acc]);
            }
            // after an abort, the MMAs already issued finish before TMEM is freed
            if (*abort) {
                mma_commit(&ctl->drain);
                mbar_drain(&ctl->drain, 0, wlim);
            }
        }
    }
    if ((warp < 4 || warp >= 6) && quad) {
        // gather the P block by phi quads: the tile's phi list holds whole atoms of 4 consecutive
        // functions, so P[a][b0 .. b0+3] is one aligned 16-byte load; item = (row quad, 8-wide K
        // chunk), quads fastest so a warp reads 512 contiguous bytes of one P row per load
        const int rank = gather_rank(warp, lane);
        const int nq = NB / 4, chunks = KB * 8, total = nq * chunks;
        // a thread's items come in increasing K order: once its next item lies in K block q, its
        // share of every block before q is stored and it arrives on those blocks' barriers
        int sig = 0;
        auto signal_upto = [&](int q) {
            if (sig >= q) return;
            fence_async_smem();
            for (; sig < q; ++sig)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&ctl->b_ready[sig])) : "memory");
        };
        for (int i0 = rank; i0 < total; i0 += 2 * DENS_GATHER) {
            float4 v[2][8];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int idx = i0 + u * DENS_GATHER;
                const int qd = idx % nq, ch = idx / nq;
                const int sl = (qd * 4) / NP, b0 = qd * 4 - sl * NP;
                const bool live = idx < total && sl < gs && b0 < np;
                const float *Ps = P + (long long)(s0 + (live ? sl : 0)) * sP + (live ? pids[p0 + b0] : 0);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int a = (ch >> 3) * 64 + (ch & 7) * 8 + j;
                    v[u][j] = (live && a < nc) ? __ldg(reinterpret_cast<const float4 *>(Ps + (long long)cids[c0 + a] * nphi))
                                               : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                }
            }
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int idx = i0 + u * DENS_GATHER;
                if (idx >= total) continue;
                const int qd = idx % nq, ch = idx / nq;
                const int sl = (qd * 4) / NP;
                const float sc = sl < gs ? pscale[s0 + sl] : 0.0f;
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    unsigned short h[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float x = r == 0 ? v[u][j].x : r == 1 ? v[u][j].y : r == 2 ? v[u][j].z : v[u][j].w;
                        h[j] = __half_as_ushort(__float2half_rn(x * sc));
                    }
                    uint4 q;
                    q.x = h[0] | ((unsigned)h[1] << 16);
                    q.y = h[2] | ((unsigned)h[3] << 16);
                    q.z = h[4] | ((unsigned)h[5] << 16);
                    q.w = h[6] | ((unsigned)h[7] << 16);
                    *reinterpret_cast<uint4 *>(B + (size_t)(ch >> 3) * NB * 128 + sw128_offset(qd * 4 + r, ch & 7)) = q;
                }
            }
            signal_upto(min(KB, ((i0 + 2 * DENS_GATHER) / nq) >> 3));
        }
        signal_upto(KB);
    } else if (warp < 4 || warp >= 6) {
        // gather the P block: row (s, b), K = a, 8 consecutive a per 16-byte chunk; four items in
        // flight per thread (32 independent loads)
        const int rank = gather_rank(warp, lane);
        const int chunks = KB * 8;
        const int total = NB * chunks;
        int sig = 0;   // as above: arrive on each K block once this thread's share of it is stored
        auto signal_upto = [&](int q) {
            if (sig >= q) return;
            fence_async_smem();
            for (; sig < q; ++sig)
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&ctl->b_ready[sig])) : "memory");
        };
        for (int i0 = rank; i0 < total; i0 += 4 * DENS_GATHER) {
            float v[4][8];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int idx = i0 + u * DENS_GATHER;
                const int row = idx % NB, ch = idx / NB;
                const int sl = row / NP, b = row - sl * NP;
                const bool live = idx < total && sl < gs && b < np;
                const float *Ps = P + (long long)(s0 + (live ? sl : 0)) * sP + (live ? pids[p0 + b] : 0);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const int a = (ch >> 3) * 64 + (ch & 7) * 8 + j;
                    v[u][j] = (live && a < nc) ? Ps[(long long)cids[c0 + a] * nphi] : 0.0f;
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int idx = i0 + u * DENS_GATHER;
                if (idx >= total) continue;
                const int row = idx % NB, ch = idx / NB;
                const int sl = row / NP;
                const float sc = sl < gs ? pscale[s0 + sl] : 0.0f;
                unsigned short h[8];
#pragma unroll
                for (int j = 0; j < 8; ++j) h[j] = __half_as_ushort(__float2half_rn(v[u][j] * sc));
                uint4 q;
                q.x = h[0] | ((unsigned)h[1] << 16);
                q.y = h[2] | ((unsigned)h[3] << 16);
                q.z = h[4] | ((unsigned)h[5] << 16);
                q.w = h[6] | ((unsigned)h[7] << 16);
                *reinterpret_cast<uint4 *>(B + (size_t)(ch >> 3) * NB * 128 + sw128_offset(row, ch & 7)) = q;
            }
            signal_upto(min(KB, ((i0 + 4 * DENS_GATHER) / NB) >> 3));
        }
        signal_upto(KB);
    }
    if (warp < 4 || warp >= 8) {
        // epilogue: rho_s(r) = sum_b T[r][(s,b)] phi_b(r) for the 128 points of block pb. Two
        // groups of four warps (0-3 and 8-11) read the same TMEM lanes (warp % 4 selects the
        // quarter) and split the states: the first half of the group's states to one, the rest
        // to the other
        const int eg = warp < 4 ? 0 : 1, quarter = warp & 3;
        const int gsplit = (gs + 1) / 2;
        const bool aligned = NP % 32 == 0 && phi_pm != nullptr;
        const int sbeg = aligned ? (eg ? gsplit : 0) : 0;
        const int send = aligned ? (eg ? gs : gsplit) : (eg ? 0 : gs);
        for (int pb = 0; pb < TILE_PTS / 128; ++pb) {
            const int acc = pb & 1;
            const bool ok = mbar_wait(&ctl->acc_full[acc], (pb >> 1) & 1, abort, wlim) && !*abort;
            tc_fence_after();
            const int lp = pb * 128 + quarter * 32 + lane;
            float r[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) r[q] = 0.0f;
            if (aligned) {
                // every 32-column chunk belongs to one state: skip the chunks that are all padding
                // (warp-uniform), prefetch the next chunk's phi while this chunk's columns come
                // out of TMEM, and add one dot product per chunk
                auto live = [&](int cc) {
                    const int sl = cc / NP;
                    return sl < gs && cc - sl * NP < np;
                };
                const int cend = send * NP;
                int c = sbeg * NP;
                while (c < cend && !live(c)) c += 32;
                // phi kept as float16 pairs in registers (16 per chunk) and widened at the dot
                auto load_q = [&](int cc, uint4 *dst) {
                    const uint4 *q = reinterpret_cast<const uint4 *>(
                        phi_pm + ((long long)t * TILE_PTS + lp) * NP + (cc - (cc / NP) * NP));
#pragma unroll
                    for (int w = 0; w < 4; ++w) dst[w] = __ldg(q + w);
                };
                uint4 ph[4];
                if (c < cend) load_q(c, ph);
                while (c < cend) {
                    int cn = c + 32;
                    while (cn < cend && !live(cn)) cn += 32;
                    uint4 phn[4];
                    if (cn < cend) load_q(cn, phn);
                    float v[32];
                    tmem_ld32(tmem + acc * 256 + ((unsigned)(quarter * 32) << 16) + (unsigned)c, v);
                    float d = 0.0f;
#pragma unroll
                    for (int w = 0; w < 4; ++w) {
                        const __half2 *h = reinterpret_cast<const __half2 *>(&ph[w]);
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const float2 f2 = __half22float2(h[e]);
                            d = fmaf(v[8 * w + 2 * e], f2.x, d);
                            d = fmaf(v[8 * w + 2 * e + 1], f2.y, d);
                        }
                    }
                    const int sl = c / NP;
#pragma unroll
                    for (int q = 0; q < 16; ++q)
                        if (q == sl) r[q] += d;
                    if (cn < cend) {
#pragma unroll
                        for (int w = 0; w < 4; ++w) ph[w] = phn[w];
                    }
                    c = cn;
                }
            } else if (eg == 0) {
                for (int c = 0; c < NB; c += 32) {
                    float v[32];
                    tmem_ld32(tmem + acc * 256 + ((unsigned)(quarter * 32) << 16) + (unsigned)c, v);
                    float ph[32];
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int col = c + j, sl = col / NP, b = col - sl * NP;
                        ph[j] = (sl < gs && b < np) ? pval[(long long)(p0 + b) * TILE_PTS + lp] : 0.0f;
                    }
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const int sl = (c + j) / NP;
                        const float w = v[j] * ph[j];
#pragma unroll
                        for (int q = 0; q < 16; ++q)
                            if (q == sl) r[q] += w;
                    }
                }
            }
            tc_fence_before();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&ctl->acc_empty[acc])) : "memory");
            const int gx = tx * TILE + (lp >> 6), gy = ty * TILE + ((lp >> 3) & 7), gz = tz * TILE + (lp & 7);
            if (ok && gx < n && gy < n && gz < n) {
                const long long gi = ((long long)gx * n + gy) * n + gz;
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    if (q >= sbeg && q < send) rho[(long long)(s0 + q) * n3 + gi] = r[q] / pscale[s0 + q];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 5) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
    }
    if (threadIdx.x == 0 && ctl->abort) atomicExch(err, 1);
}

// ------------------------------------------------------------------------------------------------
// Persistent variant: one CTA per SM walks a list of work items (tile, state) and overlaps the
// P-block gather of its next item with the MMAs and epilogue of the current one (two B buffers).
// 512 threads: warps 0-3 and 8-11 are the epilogue groups (accumulator 0 / 1, i.e. even / odd
// 128-point blocks, on the TMEM lanes warp % 4), warp 4 the TMA producer, warp 5 the MMA issuer,
// warps 6-7 and 12-15 gather. For systems whose tile phi lists are whole aligned atom quads, one
// state per item (NB = NP <= 128) and at most PDENS_KB K blocks of 64 chi per tile.
constexpr int PDENS_THREADS = 512;
constexpr int PDENS_GATHER = 192;      // warps 6-7 and 12-15
constexpr int PDENS_STAGES = 4;        // chi-block ring (16 KB each)
constexpr int PDENS_KB = 5;            // K blocks per B buffer (2 x 5 x 16 KB + ring = 224 KB)

struct __align__(8) PDensShared {
    unsigned long long a_full[PDENS_STAGES];
    unsigned long long a_empty[PDENS_STAGES];
    unsigned long long acc_full[2];
    unsigned long long acc_empty[2];
    unsigned long long b_full[2];
    unsigned long long b_free[2];
    unsigned long long drain;
    unsigned int tmem_base;
    int abort;
};

__device__ __forceinline__ int pgather_rank(int warp, int lane) {
    return (warp < 8 ? warp - 6 : warp - 10) * 32 + lane;   // warps 6, 7, 12-15 -> 0 .. 191
}

__global__ void __launch_bounds__(PDENS_THREADS, 1) density_tc_persistent_kernel(
    const __grid_constant__ CUtensorMap mX,   // point-major chi: [tile*512 + point][CK] f16
    int n, int nt, int NP, int k, const int *__restrict__ items_tiles, int nitems,
    const int *__restrict__ coff, const int *__restrict__ cids, const int *__restrict__ poff,
    const int *__restrict__ pids, int nphi, const unsigned short *__restrict__ phi_pm,
    const float *__restrict__ P, long long sP, const float *__restrict__ pscale, float *__restrict__ rho,
    int *err, long long wlim) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<unsigned long long>(smem_raw) + 1023ull) & ~1023ull);
    const int NB = NP;
    unsigned char *A = base;                                      // ring [STAGES][128 x 128 B]
    unsigned char *Bb = base + PDENS_STAGES * 16384;              // [2][PDENS_KB][NB x 128 B]
    const size_t bsize = (size_t)PDENS_KB * NB * 128;
    PDensShared *ctl = reinterpret_cast<PDensShared *>(Bb + 2 * bsize);
    volatile int *abort = &ctl->abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long n3 = (long long)n * n * n;
    if (threadIdx.x == 0) {
        for (int i = 0; i < PDENS_STAGES; ++i) {
            mbar_init(&ctl->a_full[i], 1);
            mbar_init(&ctl->a_empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&ctl->acc_full[i], 1);
            mbar_init(&ctl->acc_empty[i], 128);
            mbar_init(&ctl->b_full[i], PDENS_GATHER);
            mbar_init(&ctl->b_free[i], 1);
        }
        mbar_init(&ctl->drain, 1);
        ctl->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ctl->tmem_base)),
                     "r"(256));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = ctl->tmem_base;
    // items of this CTA: it = blockIdx.x + j * gridDim.x; item -> (tile list entry it / k, state it % k)

    if (warp == 4) {
        // TMA producer: for every item, the chi blocks (pb, kb) through the ring
        if (lane == 0) {
            long long q = 0;
            for (int it = blockIdx.x; it < nitems && !*abort; it += gridDim.x) {
                const int t = items_tiles[it / k];
                const int KB = (coff[t + 1] - coff[t] + 63) / 64;
                for (int pb = 0; pb < TILE_PTS / 128; ++pb)
                    for (int kb = 0; kb < KB; ++kb, ++q) {
                        const int st = (int)(q % PDENS_STAGES);
                        const long long use = q / PDENS_STAGES;
                        if (use > 0 && !mbar_wait(&ctl->a_empty[st], (unsigned)((use - 1) & 1), abort, wlim)) break;
                        mbar_expect_tx(&ctl->a_full[st], 16384);
                        tma_load_2d(A + st * 16384, &mX, &ctl->a_full[st], kb * 64, t * TILE_PTS + pb * 128);
                    }
            }
            // after an abort, the loads already issued land before the block exits
            if (*abort)
                for (long long j = q > PDENS_STAGES ? q - PDENS_STAGES : 0; j < q; ++j)
                    mbar_drain(&ctl->a_full[j % PDENS_STAGES], (unsigned)((j / PDENS_STAGES) & 1), wlim);
        }
    } else if (warp == 5) {
        // MMA issuer
        if (lane == 0) {
            const unsigned idesc = idesc_f16(128, NB);
            long long q = 0, pbg = 0;
            int j = 0;
            bool ok = true;
            for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x, ++j) {
                const int t = items_tiles[it / k];
                const int KB = (coff[t + 1] - coff[t] + 63) / 64;
                const int buf = j & 1;
                if (!mbar_wait(&ctl->b_full[buf], (unsigned)((j >> 1) & 1), abort, wlim)) break;
                tc_fence_after();
                const unsigned char *B = Bb + buf * bsize;
                for (int pb = 0; pb < TILE_PTS / 128 && ok; ++pb, ++pbg) {
                    const int acc = (int)(pbg & 1);
                    const long long ause = pbg >> 1;
                    if (ause > 0 && !mbar_wait(&ctl->acc_empty[acc], (unsigned)((ause - 1) & 1), abort, wlim)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    for (int kb = 0; kb < KB; ++kb, ++q) {
                        const int st = (int)(q % PDENS_STAGES);
                        if (!mbar_wait(&ctl->a_full[st], (unsigned)((q / PDENS_STAGES) & 1), abort, wlim)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const unsigned a = smem_u32(A + st * 16384), bb = smem_u32(B + (size_t)kb * NB * 128);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            mma_f16(tmem + acc * 128, smem_desc(a + kk * 32), smem_desc(bb + kk * 32), idesc,
                                    (kb > 0 || kk > 0) ? 1u : 0u);
                        mma_commit(&ctl->a_empty[st]);
                    }
                    if (!ok) break;
                    mma_commit(&ctl->acc_full[acc]);
                }
                if (!ok) break;
                mma_commit(&ctl->b_free[buf]);   // this item's B buffer is free once its MMAs finish
            }
            if (*abort) {
                mma_commit(&ctl->drain);
                mbar_drain(&ctl->drain, 0, wlim);
            }
        }
    } else if ((warp >= 6 && warp < 8) || warp >= 12) {
        // gather the P block of each item into B[j % 2] by phi quads (aligned groups of four)
        const int rank = pgather_rank(warp, lane);
        int j = 0;
        for (int it = blockIdx.x; it < nitems; it += gridDim.x, ++j) {
            const int t = items_tiles[it / k], s = it % k;
            const int c0 = coff[t], nc = coff[t + 1] - c0;
            const int p0 = poff[t], np = poff[t + 1] - p0;
            const int KB = (nc + 63) / 64;
            const int buf = j & 1;
            if (j >= 2 && !mbar_wait(&ctl->b_free[buf], (unsigned)(((j >> 1) - 1) & 1), abort, wlim)) break;
            unsigned char *B = Bb + buf * bsize;
            const float sc = pscale[s];
            const float *Ps = P + (long long)s * sP;
            const int nq = NB / 4, total = nq * KB * 8;
            for (int i0 = rank; i0 < total; i0 += 2 * PDENS_GATHER) {
                float4 v[2][8];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int idx = i0 + u * PDENS_GATHER;
                    const int qd = idx % nq, ch = idx / nq;
                    const bool live = idx < total && qd * 4 < np;
                    const float *Pq = Ps + (live ? pids[p0 + qd * 4] : 0);
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int a = (ch >> 3) * 64 + (ch & 7) * 8 + e;
                        v[u][e] = (live && a < nc) ? __ldg(reinterpret_cast<const float4 *>(Pq + (long long)cids[c0 + a] * nphi))
                                                   : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    }
                }
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int idx = i0 + u * PDENS_GATHER;
                    if (idx >= total) continue;
                    const int qd = idx % nq, ch = idx / nq;
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        unsigned short h[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const float x = r == 0 ? v[u][e].x : r == 1 ? v[u][e].y : r == 2 ? v[u][e].z : v[u][e].w;
                            h[e] = __half_as_ushort(__float2half_rn(x * sc));
                        }
                        uint4 qv;
                        qv.x = h[0] | ((unsigned)h[1] << 16);
                        qv.y = h[2] | ((unsigned)h[3] << 16);
                        qv.z = h[4] | ((unsigned)h[5] << 16);
                        qv.w = h[6] | ((unsigned)h[7] << 16);
                        *reinterpret_cast<uint4 *>(B + (size_t)(ch >> 3) * NB * 128 + sw128_offset(qd * 4 + r, ch & 7)) = qv;
                    }
                }
            }
            fence_async_smem();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&ctl->b_full[buf])) : "memory");
        }
    } else {
        // epilogue groups: warps 0-3 take accumulator 0 (even point blocks), warps 8-11 accumulator 1
        const int eg = warp < 4 ? 0 : 1, quarter = warp & 3;
        long long ause = 0;
        for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
            const int t = items_tiles[it / k], s = it % k;
            const int p0 = poff[t], np = poff[t + 1] - p0;
            const int tx = t / (nt * nt), ty = (t / nt) % nt, tz = t % nt;
            const float inv = 1.0f / pscale[s];
            bool stop = false;
            for (int pb = eg; pb < TILE_PTS / 128; pb += 2, ++ause) {
                const bool ok = mbar_wait(&ctl->acc_full[eg], (unsigned)(ause & 1), abort, wlim) && !*abort;
                tc_fence_after();
                const int lp = pb * 128 + quarter * 32 + lane;
                float r = 0.0f;
                if (ok) {
                    const uint4 *q = reinterpret_cast<const uint4 *>(phi_pm + ((long long)t * TILE_PTS + lp) * NP);
                    for (int c = 0; c < np; c += 32) {
                        uint4 ph[4];
#pragma unroll
                        for (int w = 0; w < 4; ++w) ph[w] = __ldg(q + c / 8 + w);
                        float v[32];
                        tmem_ld32(tmem + eg * 128 + ((unsigned)(quarter * 32) << 16) + (unsigned)c, v);
#pragma unroll
                        for (int w = 0; w < 4; ++w) {
                            const __half2 *h = reinterpret_cast<const __half2 *>(&ph[w]);
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const float2 f2 = __half22float2(h[e]);
                                r = fmaf(v[8 * w + 2 * e], f2.x, r);
                                r = fmaf(v[8 * w + 2 * e + 1], f2.y, r);
                            }
                        }
                    }
                }
                tc_fence_before();
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&ctl->acc_empty[eg])) : "memory");
                if (!ok) {
                    stop = true;
                    break;
                }
                const int gx = tx * TILE + (lp >> 6), gy = ty * TILE + ((lp >> 3) & 7), gz = tz * TILE + (lp & 7);
                if (gx < n && gy < n && gz < n) rho[(long long)s * n3 + ((long long)gx * n + gy) * n + gz] = r * inv;
            }
            if (stop) break;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 5) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
    }
    if (threadIdx.x == 0 && ctl->abort) atomicExch(err, 1);
}

// ------------------------------------------------------------------------------------------------
// Dense tiles (more chi or phi on a tile than the per-tile kernels hold, as in the solvated
// systems of Sec. IV): each tile's lists are cut into units of at most 5 x 64 chi and 4 x 32 phi,
// and each unit adds
//   rho_s(r) += sum_{b in unit} [ sum_{a in unit} chi_a(r) P_s,ab ] phi_b(r)
// for the tile's 512 points into rho with float32 reductions. Persistent, one CTA per SM over
// (unit, state) items, with the roles of the persistent per-tile kernel: warp 4 brings the chi
// chunks of the unit by TMA from a chunked point-major table [chunk][512][64] (chunk = 64
// consecutive chi slots of one tile, zero padded), warp 5 issues the MMAs (M = 128 points,
// N = 128 phi rows, K = the unit's chi), warps 6-7 and 12-15 gather the next item's P block
// (float16, scaled per state) into the other B buffer, and the two epilogue groups (warps 0-3,
// 8-11) read their accumulator and multiply by phi from a chunked point-major table
// [chunk][512][32]. Every wait is bounded.
constexpr int UD_KB = 5;              // chi blocks of 64 per unit
constexpr int UD_NB = 128;            // phi rows of the B operand

__global__ void __launch_bounds__(PDENS_THREADS, 1) density_units_kernel(
    const __grid_constant__ CUtensorMap mX,   // [chi chunk * 512 + point][64] f16, box 64 x 128
    int n, int nt, int k, const DUnit *__restrict__ units, int nitems, const int *__restrict__ cids,
    const int *__restrict__ pids, int nphi, const unsigned short *__restrict__ phi_pmc,
    const float *__restrict__ P, long long sP, const float *__restrict__ pscale, float *__restrict__ rho,
    int *err, long long wlim) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<unsigned long long>(smem_raw) + 1023ull) & ~1023ull);
    constexpr int NB = UD_NB;
    unsigned char *A = base;                                      // ring [STAGES][128 x 128 B]
    unsigned char *Bb = base + PDENS_STAGES * 16384;              // [2][UD_KB][NB x 128 B]
    constexpr size_t bsize = (size_t)UD_KB * NB * 128;
    PDensShared *ctl = reinterpret_cast<PDensShared *>(Bb + 2 * bsize);
    volatile int *abort = &ctl->abort;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long n3 = (long long)n * n * n;
    if (threadIdx.x == 0) {
        for (int i = 0; i < PDENS_STAGES; ++i) {
            mbar_init(&ctl->a_full[i], 1);
            mbar_init(&ctl->a_empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&ctl->acc_full[i], 1);
            mbar_init(&ctl->acc_empty[i], 128);
            mbar_init(&ctl->b_full[i], PDENS_GATHER);
            mbar_init(&ctl->b_free[i], 1);
        }
        mbar_init(&ctl->drain, 1);
        ctl->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ctl->tmem_base)),
                     "r"(256));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = ctl->tmem_base;

    if (warp == 4) {
        if (lane == 0) {
            long long q = 0;
            for (int it = blockIdx.x; it < nitems && !*abort; it += gridDim.x) {
                const DUnit u = units[it / k];
                const int KB = (u.nc + 63) / 64;
                for (int pb = 0; pb < TILE_PTS / 128; ++pb)
                    for (int kb = 0; kb < KB; ++kb, ++q) {
                        const int st = (int)(q % PDENS_STAGES);
                        const long long use = q / PDENS_STAGES;
                        if (use > 0 && !mbar_wait(&ctl->a_empty[st], (unsigned)((use - 1) & 1), abort, wlim)) break;
                        mbar_expect_tx(&ctl->a_full[st], 16384);
                        tma_load_2d(A + st * 16384, &mX, &ctl->a_full[st], 0, (u.cch + kb) * TILE_PTS + pb * 128);
                    }
            }
            if (*abort)
                for (long long j = q > PDENS_STAGES ? q - PDENS_STAGES : 0; j < q; ++j)
                    mbar_drain(&ctl->a_full[j % PDENS_STAGES], (unsigned)((j / PDENS_STAGES) & 1), wlim);
        }
    } else if (warp == 5) {
        if (lane == 0) {
            const unsigned idesc = idesc_f16(128, NB);
            long long q = 0, pbg = 0;
            int j = 0;
            bool ok = true;
            for (int it = blockIdx.x; it < nitems && ok; it += gridDim.x, ++j) {
                const DUnit u = units[it / k];
                const int KB = (u.nc + 63) / 64;
                const int buf = j & 1;
                if (!mbar_wait(&ctl->b_full[buf], (unsigned)((j >> 1) & 1), abort, wlim)) break;
                tc_fence_after();
                const unsigned char *B = Bb + buf * bsize;
                for (int pb = 0; pb < TILE_PTS / 128 && ok; ++pb, ++pbg) {
                    const int acc = (int)(pbg & 1);
                    const long long ause = pbg >> 1;
                    if (ause > 0 && !mbar_wait(&ctl->acc_empty[acc], (unsigned)((ause - 1) & 1), abort, wlim)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    for (int kb = 0; kb < KB; ++kb, ++q) {
                        const int st = (int)(q % PDENS_STAGES);
                        if (!mbar_wait(&ctl->a_full[st], (unsigned)((q / PDENS_STAGES) & 1), abort, wlim)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                        const unsigned a = smem_u32(A + st * 16384), bb = smem_u32(B + (size_t)kb * NB * 128);
#pragma unroll
                        for (int kk = 0; kk < 4; ++kk)
                            mma_f16(tmem + acc * 128, smem_desc(a + kk * 32), smem_desc(bb + kk * 32), idesc,
                                    (kb > 0 || kk > 0) ? 1u : 0u);
                        mma_commit(&ctl->a_empty[st]);
                    }
                    if (!ok) break;
                    mma_commit(&ctl->acc_full[acc]);
                }
                if (!ok) break;
                mma_commit(&ctl->b_free[buf]);
            }
            if (*abort) {
                mma_commit(&ctl->drain);
                mbar_drain(&ctl->drain, 0, wlim);
            }
        }
    } else if ((warp >= 6 && warp < 8) || warp >= 12) {
        // the P block of each item (rows = the unit's phi, K = its chi) by phi quads, zeros past
        // the unit's counts (every row and K column of the buffer is written)
        const int rank = pgather_rank(warp, lane);
        int j = 0;
        for (int it = blockIdx.x; it < nitems; it += gridDim.x, ++j) {
            const DUnit u = units[it / k];
            const int s = it % k;
            const int KB = (u.nc + 63) / 64;
            const int buf = j & 1;
            if (j >= 2 && !mbar_wait(&ctl->b_free[buf], (unsigned)(((j >> 1) - 1) & 1), abort, wlim)) break;
            unsigned char *B = Bb + buf * bsize;
            const float sc = pscale[s];
            const float *Ps = P + (long long)s * sP;
            constexpr int nq = NB / 4;
            const int total = nq * KB * 8;
            for (int i0 = rank; i0 < total; i0 += 2 * PDENS_GATHER) {
                float4 v[2][8];
#pragma unroll
                for (int uu = 0; uu < 2; ++uu) {
                    const int idx = i0 + uu * PDENS_GATHER;
                    const int qd = idx % nq, ch = idx / nq;
                    const bool live = idx < total && qd * 4 < u.np;
                    const float *Pq = Ps + (live ? pids[u.p0 + qd * 4] : 0);
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const int a = (ch >> 3) * 64 + (ch & 7) * 8 + e;
                        v[uu][e] = (live && a < u.nc)
                                       ? __ldg(reinterpret_cast<const float4 *>(Pq + (long long)cids[u.c0 + a] * nphi))
                                       : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                    }
                }
#pragma unroll
                for (int uu = 0; uu < 2; ++uu) {
                    const int idx = i0 + uu * PDENS_GATHER;
                    if (idx >= total) continue;
                    const int qd = idx % nq, ch = idx / nq;
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        unsigned short h[8];
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const float x = r == 0 ? v[uu][e].x : r == 1 ? v[uu][e].y : r == 2 ? v[uu][e].z : v[uu][e].w;
                            h[e] = __half_as_ushort(__float2half_rn(x * sc));
                        }
                        uint4 qv;
                        qv.x = h[0] | ((unsigned)h[1] << 16);
                        qv.y = h[2] | ((unsigned)h[3] << 16);
                        qv.z = h[4] | ((unsigned)h[5] << 16);
                        qv.w = h[6] | ((unsigned)h[7] << 16);
                        *reinterpret_cast<uint4 *>(B + (size_t)(ch >> 3) * NB * 128 + sw128_offset(qd * 4 + r, ch & 7)) = qv;
                    }
                }
            }
            fence_async_smem();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&ctl->b_full[buf])) : "memory");
        }
    } else {
        // epilogue groups: warps 0-3 accumulator 0 (even point blocks), warps 8-11 accumulator 1
        const int eg = warp < 4 ? 0 : 1, quarter = warp & 3;
        long long ause = 0;
        for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
            const DUnit u = units[it / k];
            const int s = it % k;
            const int tx = u.t / (nt * nt), ty = (u.t / nt) % nt, tz = u.t % nt;
            const float inv = 1.0f / pscale[s];
            bool stop = false;
            for (int pb = eg; pb < TILE_PTS / 128; pb += 2, ++ause) {
                const bool ok = mbar_wait(&ctl->acc_full[eg], (unsigned)(ause & 1), abort, wlim) && !*abort;
                tc_fence_after();
                const int lp = pb * 128 + quarter * 32 + lane;
                float r = 0.0f;
                if (ok) {
                    for (int c = 0; c < u.np; c += 32) {
                        const uint4 *q = reinterpret_cast<const uint4 *>(
                            phi_pmc + ((long long)(u.pch + c / 32) * TILE_PTS + lp) * 32);
                        uint4 ph[4];
#pragma unroll
                        for (int w = 0; w < 4; ++w) ph[w] = __ldg(q + w);
                        float v[32];
                        tmem_ld32(tmem + eg * 128 + ((unsigned)(quarter * 32) << 16) + (unsigned)c, v);
#pragma unroll
                        for (int w = 0; w < 4; ++w) {
                            const __half2 *hh = reinterpret_cast<const __half2 *>(&ph[w]);
#pragma unroll
                            for (int e = 0; e < 4; ++e) {
                                const float2 f2 = __half22float2(hh[e]);
                                r = fmaf(v[8 * w + 2 * e], f2.x, r);
                                r = fmaf(v[8 * w + 2 * e + 1], f2.y, r);
                            }
                        }
                    }
                }
                tc_fence_before();
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&ctl->acc_empty[eg])) : "memory");
                if (!ok) {
                    stop = true;
                    break;
                }
                const int gx = tx * TILE + (lp >> 6), gy = ty * TILE + ((lp >> 3) & 7), gz = tz * TILE + (lp & 7);
                if (gx < n && gy < n && gz < n)
                    atomicAdd(rho + (long long)s * n3 + ((long long)gx * n + gy) * n + gz, r * inv);
            }
            if (stop) break;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 5) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
    }
    if (threadIdx.x == 0 && ctl->abort) atomicExch(err, 1);
}

// chunked point-major f16 copy of a tile set's tables: chunk c of tile t holds the slots
// off[t] + j*W .. + W - 1 (j = c - first[t]) as [512 points][W], zeros past the tile's count
__global__ void chunked_pm_kernel(const float *__restrict__ val, const int *__restrict__ off,
                                  const int *__restrict__ chunk_tile, const int *__restrict__ chunk_j, int W,
                                  long long nchunks, unsigned short *__restrict__ out) {
    const long long tot = nchunks * TILE_PTS * W;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const long long ch = e / ((long long)TILE_PTS * W);
        const int rem = (int)(e - ch * TILE_PTS * W), p = rem / W, a = rem - p * W;
        const int t = chunk_tile[ch], sl = chunk_j[ch] * W + a;
        const int cnt = off[t + 1] - off[t];
        out[e] = sl < cnt ? __half_as_ushort(__float2half_rn(val[(long long)(off[t] + sl) * TILE_PTS + p])) : 0;
    }
}

// per-state power-of-two scale: 2^-e with 2^(e-1) < max|P_s| <= 2^e (1 for an all-zero state)
__global__ void maxabs_kernel(const float *__restrict__ P, long long len, int k, unsigned *__restrict__ bits) {
    const int s = blockIdx.y;
    float m = 0.0f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < len; i += (long long)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(P[(long long)s * len + i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&bits[s], __float_as_uint(m));
}

__global__ void scale_kernel(const unsigned *__restrict__ bits, int k, float *__restrict__ scale) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= k) return;
    const float m = __uint_as_float(bits[s]);
    int e = 0;
    if (m > 0.0f && isfinite(m)) frexpf(m, &e);
    scale[s] = (m > 0.0f && isfinite(m)) ? ldexpf(1.0f, -e) : 1.0f;
}

}  // namespace

// point-major f16 copy of a tile set: [tile][512][CK], CK = 64 * ceil(max functions per tile / 64)
void build_point_major_f16(const int *off_h, const float *val_h_or_null, const double *vald_h_or_null,
                           int ntiles, int CK, unsigned short *out_h) {
#pragma omp parallel for schedule(dynamic, 16)
    for (int t = 0; t < ntiles; ++t)
        for (int sl = off_h[t]; sl < off_h[t + 1]; ++sl) {
            const int a = sl - off_h[t];
            for (int lp = 0; lp < TILE_PTS; ++lp) {
                const float v = val_h_or_null ? val_h_or_null[(size_t)sl * TILE_PTS + lp]
                                              : (float)vald_h_or_null[(size_t)sl * TILE_PTS + lp];
                out_h[((size_t)t * TILE_PTS + lp) * CK + a] = __half_as_ushort(__float2half_rn(v));
            }
        }
}

bool encode_map_2d(CUtensorMap *map, CUtensorMapDataType dt, const void *ptr, unsigned long long inner,
                   unsigned long long rows, unsigned long long row_bytes, unsigned box_inner, unsigned box_rows);

size_t density_tc_smem(int KBmax, int NB) {
    return 1024 + (size_t)DENS_STAGES * 16384 + (size_t)KBmax * NB * 128 + sizeof(DensShared);
}

// largest state group G (<= 16, G * NP <= 256) whose shared memory fits; 0 if none does
int density_tc_group(int KBmax, int NP, int k) {
    if (KBmax > DENS_KBMAX) return 0;
    for (int G = std::min(16, std::min(k, 256 / NP)); G >= 1; --G)
        if (density_tc_smem(KBmax, G * NP) <= 227 * 1024) return G;
    return 0;
}

void response_density_tc(cudaStream_t st, const GridShape &g, const TileSet<float> &chi,
                         const TileSet<float> &phi, const unsigned short *chi_pm, int CK, int NPmax, int nphi,
                         const float *P, long long sP, int k, float *rho, unsigned *scratch_bits,
                         float *scale, int *err, bool phi_quads, const unsigned short *phi_pm,
                         const int *live_tiles, int nlive) {
    if (k <= 0) return;
    ProfScope ps(st, ST_DENSITY, 2.0 * k * g.pair_points, 2.0 * g.table_values + 4.0 * k * g.n * g.n * g.n);
    check(cudaMemsetAsync(scratch_bits, 0, sizeof(unsigned) * k, st), "memset maxabs");
    maxabs_kernel<<<dim3(64, k), 256, 0, st>>>(P, sP, k, scratch_bits);
    check_launch("maxabs_kernel");
    scale_kernel<<<(k + 127) / 128, 128, 0, st>>>(scratch_bits, k, scale);
    check_launch("scale_kernel");
    CUtensorMap mx;
    if (!encode_map_2d(&mx, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, chi_pm, (unsigned long long)CK,
                       (unsigned long long)chi.ntiles * TILE_PTS, (unsigned long long)CK * 2, 64, 128))
        throw CudaError{cudaErrorInvalidValue, "cuTensorMapEncodeTiled (density)"};
    const int NP = NPmax, KBmax = CK / 64;
    static const bool no_persistent = [] {
        const char *e = std::getenv("TDDFT_NO_PERSISTENT_DENSITY");
        return e && e[0] == '1';
    }();
    if (!no_persistent && phi_quads && phi_pm && live_tiles && NP % 32 == 0 && NP <= 128 && KBmax <= PDENS_KB) {
        // persistent kernel over (tile, state) items; tiles without chi or phi only need zeros
        const size_t psm = 1024 + (size_t)PDENS_STAGES * 16384 + 2 * (size_t)PDENS_KB * NP * 128 + sizeof(PDensShared);
        static const bool pattr = [&]() {
            check(cudaFuncSetAttribute(density_tc_persistent_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       227 * 1024),
                  "attr density_tc_persistent");
            return true;
        }();
        (void)pattr;
        check(cudaMemsetAsync(rho, 0, sizeof(float) * (size_t)k * g.n * g.n * g.n, st), "memset rho");
        const int nitems = nlive * k;
        if (nitems > 0) {
            int dev = 0, sms = 0;
            check(cudaGetDevice(&dev), "cudaGetDevice");
            check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
            const int grid = std::min(sms, nitems);
            density_tc_persistent_kernel<<<grid, PDENS_THREADS, psm, st>>>(mx, g.n, g.nt, NP, k, live_tiles, nitems,
                                                                           chi.off, chi.ids, phi.off, phi.ids, nphi,
                                                                           phi_pm, P, sP, scale, rho, err,
                                                                           active_wait_limit());
            check_launch("density_tc_persistent_kernel");
        }
        return;
    }
    const int G = density_tc_group(KBmax, NP, k);
    if (G < 1) throw CudaError{cudaErrorInvalidValue, "density_tc: tile too large for shared memory"};
    const int ngroups = (k + G - 1) / G;
    const size_t sm = density_tc_smem(KBmax, G * NP);
    static const bool attr = [&]() {   // once per process, thread-safe
        check(cudaFuncSetAttribute(density_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024),
              "attr density_tc");
        return true;
    }();
    (void)attr;
    dim3 grid(ngroups, chi.ntiles);
    density_tc_kernel<<<grid, DENS_THREADS, sm, st>>>(mx, g.n, g.nt, KBmax, NP, G, k, chi.off, chi.ids, phi.off,
                                                      phi.ids, phi.val, nphi, P, sP, scale, rho, err,
                                                      phi_quads ? 1 : 0, NP % 32 == 0 ? phi_pm : nullptr,
                                                      active_wait_limit());
    check_launch("density_tc_kernel");
}

// chunked point-major f16 tables of a tile set (device built); returns the number of chunks
long long build_chunked_pm(cudaStream_t st, Mem &mem, const TileSet<float> &ts, const std::vector<int> &off_h, int W,
                           unsigned short **out, std::vector<int> &first) {
    const int ntl = ts.ntiles;
    first.assign(ntl + 1, 0);
    std::vector<int> ct, cj;
    for (int t = 0; t < ntl; ++t) {
        const int nch = (off_h[t + 1] - off_h[t] + W - 1) / W;
        first[t + 1] = first[t] + nch;
        for (int j = 0; j < nch; ++j) {
            ct.push_back(t);
            cj.push_back(j);
        }
    }
    const long long nchunks = first[ntl];
    *out = mem.alloc<unsigned short>(std::max<long long>(1, nchunks * TILE_PTS * W));
    if (nchunks == 0) return 0;
    int *dct = mem.alloc<int>(ct.size()), *dcj = mem.alloc<int>(cj.size());
    check(cudaMemcpy(dct, ct.data(), ct.size() * sizeof(int), cudaMemcpyHostToDevice), "upload chunk tiles");
    check(cudaMemcpy(dcj, cj.data(), cj.size() * sizeof(int), cudaMemcpyHostToDevice), "upload chunk index");
    const long long tot = nchunks * TILE_PTS * W;
    chunked_pm_kernel<<<(int)std::min<long long>((tot + 255) / 256, 8 * 1216), 256, 0, st>>>(
        ts.val, ts.off, dct, dcj, W, nchunks, *out);
    check_launch("chunked_pm_kernel");
    check(cudaStreamSynchronize(st), "sync chunked tables");
    return nchunks;
}

size_t density_units_smem() {
    return 1024 + (size_t)PDENS_STAGES * 16384 + 2 * (size_t)UD_KB * UD_NB * 128 + sizeof(PDensShared);
}

// response density of dense tiles: units of <= 320 chi and <= 128 phi of a tile, rho accumulated
void response_density_units(cudaStream_t st, const GridShape &g, const TileSet<float> &chi, const TileSet<float> &phi,
                            const unsigned short *chi_pmc, long long nchunks_chi, const unsigned short *phi_pmc,
                            const DUnit *units, int nunits, int nphi, const float *P, long long sP, int k, float *rho,
                            unsigned *scratch_bits, float *scale, int *err) {
    if (k <= 0) return;
    ProfScope ps(st, ST_DENSITY, 2.0 * k * g.pair_points, 2.0 * g.table_values + 4.0 * k * g.n * g.n * g.n);
    check(cudaMemsetAsync(scratch_bits, 0, sizeof(unsigned) * k, st), "memset maxabs");
    maxabs_kernel<<<dim3(64, k), 256, 0, st>>>(P, sP, k, scratch_bits);
    check_launch("maxabs_kernel");
    scale_kernel<<<(k + 127) / 128, 128, 0, st>>>(scratch_bits, k, scale);
    check_launch("scale_kernel");
    check(cudaMemsetAsync(rho, 0, sizeof(float) * (size_t)k * g.n * g.n * g.n, st), "memset rho");
    const long long nitems = (long long)nunits * k;
    if (nitems == 0) return;
    if (nitems > (1LL << 31) - 1) throw CudaError{cudaErrorInvalidValue, "density units: too many items"};
    CUtensorMap mx;
    if (!encode_map_2d(&mx, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, chi_pmc, 64ull, (unsigned long long)nchunks_chi * TILE_PTS,
                       128ull, 64, 128))
        throw CudaError{cudaErrorInvalidValue, "cuTensorMapEncodeTiled (density units)"};
    static const bool attr = [&]() {
        check(cudaFuncSetAttribute(density_units_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)density_units_smem()),
              "attr density_units");
        return true;
    }();
    (void)attr;
    int dev = 0, sms = 0;
    check(cudaGetDevice(&dev), "cudaGetDevice");
    check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    const int grid = (int)std::min<long long>(sms, nitems);
    density_units_kernel<<<grid, PDENS_THREADS, density_units_smem(), st>>>(
        mx, g.n, g.nt, k, units, (int)nitems, chi.ids, phi.ids, nphi, phi_pmc, P, sP, scale, rho, err,
        active_wait_limit());
    check_launch("density_units_kernel");
}

}  // namespace tddft

// ================================================================================================
// Potential integrals on the tensor cores (mixed precision): V_s,ab = dV sum_r chi_a(r) V_s(r) phi_b(r)
// (the <chi|V_SCF|phi> matrix of Eqs. operator_TDA / operator_RPA) as one tcgen05 kind::f16
// product per tile and state,
//
//   D[a][b] = sum_r X[a][r] W[b][r],   W[b][r] = V_s(r) phi_b(r)
//
// M = chi functions of the tile (up to 3 blocks of 128), N = phi functions of the tile, K = the
// 512 tile points in 8 slices of 64. Per slice the chi rows and the phi rows (float16 copies of
// both tables, function-major) come by TMA into a double-buffered, 128-byte-swizzled stage; four
// worker warps scale the phi rows in place by V_s (scaled by a power of two), and one thread
// issues the MMAs. The epilogue adds dV * D into the output matrix with vector reductions where
// four phi of one atom are contiguous. Tiles are launched by class of chi blocks (1, 2, 3) so
// that the smaller ones share an SM three or two at a time.
namespace tddft {
namespace {

struct __align__(8) IntShared {
    unsigned long long x_full[2];
    unsigned long long w_ready[2];
    unsigned long long mma_done[2];
    unsigned long long acc_done;
    unsigned long long drain;
    unsigned int tmem_base;
    int abort;
    int pid[256];      // the tile's phi indices (np <= NP <= 128)
};

__device__ __forceinline__ void red_add_v4(float *addr, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

// CTA = (state, unit of the launch's list: a tile, or a chunk of a dense tile's chi and phi
// slots); mbmax: most chi row blocks of a listed unit (sizes the X stages), tmem_cols: TMEM
// columns allocated (mbmax x acc_stride, a power of two). Per 64-point
// K slice the TMA warp loads the tile's chi rows (mX) and its phi rows (mP, float16 copies of the
// phi tables) straight into the B operand's stage; four warps then scale that stage in place by
// V at its points (shared memory only), and the MMA warp multiplies. Rows of the stage past the
// tile's np hold other tiles' phi: their accumulator columns are never read.
__global__ void __launch_bounds__(192, 3) integrals_tc_kernel(
    const __grid_constant__ CUtensorMap mX,   // function-major chi: [slot][512] f16
    const __grid_constant__ CUtensorMap mP,   // function-major phi: [slot][512] f16, box NP rows
    int n, int nt, int NP, int k, const int *__restrict__ cids, const int *__restrict__ pids, int nchi,
    int nphi, const float *__restrict__ V, const float *__restrict__ vscale, float dV, float *__restrict__ out,
    bool vec_ok, int acc_stride, const VTile *__restrict__ units, int mbmax, int tmem_cols, int *err,
    long long wlim) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<unsigned long long>(smem_raw) + 1023ull) & ~1023ull);
    const VTile u = units[blockIdx.y];
    const int t = u.t, s0 = blockIdx.x;
    const int c0 = u.c0, nc = u.nc;
    const int p0 = u.p0, np = u.np;
    if (nc == 0 || np == 0) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int MB = (nc + 127) / 128;                 // <= mbmax (the host lists tiles by M blocks)
    const int NB = NP;                               // <= acc_stride, multiple of 16
    // layout: X stages [2][mbmax x 16 KB], W stages [2][NB x 128 B], V tile [512] f32, control
    unsigned char *Xs = base;
    const int xstage = mbmax * 16384;
    unsigned char *Ws = base + 2 * xstage;
    float *Vt = reinterpret_cast<float *>(Ws + (size_t)2 * NB * 128);
    IntShared *ctl = reinterpret_cast<IntShared *>(Vt + TILE_PTS);
    volatile int *abort = &ctl->abort;
    const long long n3 = (long long)n * n * n;
    const int tx = t / (nt * nt), ty = (t / nt) % nt, tz = t % nt;

    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&ctl->x_full[i], 1);
            mbar_init(&ctl->w_ready[i], 128);
            mbar_init(&ctl->mma_done[i], 1);
        }
        mbar_init(&ctl->acc_done, 1);
        mbar_init(&ctl->drain, 1);
        ctl->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ctl->tmem_base)),
                     "r"(tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    for (int i = threadIdx.x; i < np; i += blockDim.x) ctl->pid[i] = pids[p0 + i];
    // V of the state on the tile points, scaled
    const float vs = vscale[s0];
    for (int lp = threadIdx.x; lp < TILE_PTS; lp += blockDim.x) {
        const int gx = tx * TILE + (lp >> 6), gy = ty * TILE + ((lp >> 3) & 7), gz = tz * TILE + (lp & 7);
        float v = 0.0f;
        if (gx < n && gy < n && gz < n) v = V[(long long)s0 * n3 + ((long long)gx * n + gy) * n + gz];
        Vt[lp] = v * vs;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = ctl->tmem_base;
    const unsigned idesc = idesc_f16(128, NB);
    constexpr int KS = TILE_PTS / 64;                // 8 K slices

    if (warp == 4) {
        if (lane == 0) {
            int kb = 0;
            for (; kb < KS; ++kb) {
                const int st = kb & 1, use = kb >> 1;
                if (use > 0 && !mbar_wait(&ctl->mma_done[st], (use - 1) & 1, abort, wlim)) break;
                mbar_expect_tx(&ctl->x_full[st], MB * 16384 + NB * 128);
                for (int mb = 0; mb < MB; ++mb)
                    tma_load_2d(Xs + st * xstage + mb * 16384, &mX, &ctl->x_full[st], kb * 64, c0 + mb * 128);
                tma_load_2d(Ws + (size_t)st * NB * 128, &mP, &ctl->x_full[st], kb * 64, p0);
            }
            // after an abort, the loads already issued land before the block exits
            if (*abort)
                for (int j = kb > 2 ? kb - 2 : 0; j < kb; ++j) mbar_drain(&ctl->x_full[j & 1], (unsigned)((j >> 1) & 1), wlim);
        }
    } else if (warp == 5) {
        if (lane == 0) {
            for (int kb = 0; kb < KS; ++kb) {
                const int st = kb & 1, use = kb >> 1;
                if (!mbar_wait(&ctl->x_full[st], use & 1, abort, wlim)) break;
                if (!mbar_wait(&ctl->w_ready[st], use & 1, abort, wlim)) break;
                tc_fence_after();
                const unsigned wb = smem_u32(Ws + (size_t)st * NB * 128);
                for (int mb = 0; mb < MB; ++mb) {
                    const unsigned xa = smem_u32(Xs + st * xstage + mb * 16384);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma_f16(tmem + mb * acc_stride, smem_desc(xa + kk * 32), smem_desc(wb + kk * 32), idesc,
                                (kb > 0 || kk > 0) ? 1u : 0u);
                }
                mma_commit(&ctl->mma_done[st]);
            }
            mma_commit(&ctl->acc_done);
            if (*abort) {
                mma_commit(&ctl->drain);
                mbar_drain(&ctl->drain, 0, wlim);
            }
        }
    } else {
        // workers: scale the phi rows of each landed stage by V (8 points per 16-byte chunk),
        // then the epilogue
        for (int kb = 0; kb < KS; ++kb) {
            const int st = kb & 1, use = kb >> 1;
            if (!mbar_wait(&ctl->x_full[st], use & 1, abort, wlim)) break;
            unsigned char *W = Ws + (size_t)st * NB * 128;
            for (int idx = threadIdx.x; idx < np * 8; idx += 128) {
                const int row = idx >> 3, c8 = idx & 7;
                uint4 *q = reinterpret_cast<uint4 *>(W + sw128_offset(row, c8));
                uint4 w = *q;
                const float4 *vv = reinterpret_cast<const float4 *>(Vt + kb * 64 + c8 * 8);
                const float4 v0 = vv[0], v1 = vv[1];
                __half2 *h = reinterpret_cast<__half2 *>(&w);
                float2 a;
                a = __half22float2(h[0]); h[0] = __floats2half2_rn(a.x * v0.x, a.y * v0.y);
                a = __half22float2(h[1]); h[1] = __floats2half2_rn(a.x * v0.z, a.y * v0.w);
                a = __half22float2(h[2]); h[2] = __floats2half2_rn(a.x * v1.x, a.y * v1.y);
                a = __half22float2(h[3]); h[3] = __floats2half2_rn(a.x * v1.z, a.y * v1.w);
                *q = w;
            }
            fence_async_smem();
            asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&ctl->w_ready[st])) : "memory");
        }
        const bool ok = mbar_wait(&ctl->acc_done, 0, abort, wlim) && !*abort;
        tc_fence_after();
        const float f = dV / vs;
        for (int mb = 0; mb < MB; ++mb) {
            const int a = mb * 128 + warp * 32 + lane;
            const bool arow = ok && a < nc;
            float *o = out + (long long)s0 * nchi * nphi + (arow ? (long long)cids[c0 + a] * nphi : 0);
            for (int c = 0; c < np; c += 32) {
                float v[32];
                tmem_ld32(tmem + mb * acc_stride + ((unsigned)(warp * 32) << 16) + (unsigned)c, v);
                if (!arow) continue;
#pragma unroll
                for (int j = 0; j < 32; j += 4) {
                    const int b = c + j;
                    if (b >= np) break;
                    const int B0 = ctl->pid[b];
                    // four consecutive phi of one atom land on one aligned float4
                    if (vec_ok && b + 3 < np && (B0 & 3) == 0 && ctl->pid[b + 3] == B0 + 3) {
                        red_add_v4(o + B0, f * v[j], f * v[j + 1], f * v[j + 2], f * v[j + 3]);
                    } else {
#pragma unroll
                        for (int u = 0; u < 4; ++u)
                            if (b + u < np) atomicAdd(o + ctl->pid[b + u], f * v[j + u]);
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 5) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols));
    }
    if (threadIdx.x == 0 && ctl->abort) atomicExch(err, 1);
}

__global__ void vmaxabs_kernel(const float *__restrict__ V, long long n3, unsigned *__restrict__ bits) {
    const int s = blockIdx.y;
    float m = 0.0f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n3; i += (long long)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(V[(long long)s * n3 + i]));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(&bits[s], __float_as_uint(m));
}

}  // namespace

size_t integrals_tc_smem(int NB, int G, int mbmax) {
    return 1024 + (size_t)2 * mbmax * 16384 + (size_t)2 * NB * 128 + (size_t)G * TILE_PTS * 4 + sizeof(IntShared);
}

// one state per CTA: the accumulator of each 128-row chi block takes NP <= 128 TMEM columns, and
// a tile may hold up to three such blocks
int integrals_tc_group(int NP, int k, int maxc) {
    if (maxc > 384 || NP > 128 || k < 1) return 0;
    return integrals_tc_smem(NP, 1, 3) <= 227 * 1024 ? 1 : 0;
}

void potential_integrals_tc(cudaStream_t st, const GridShape &g, const TileSet<float> &chi,
                            const TileSet<float> &phi, const unsigned short *chi_fm16, int nslots,
                            const unsigned short *phi_fm16, int nslots_phi, int NPmax,
                            int maxc, int nchi, int nphi, const float *V, int k, float *out, unsigned *scratch_bits,
                            float *scale, const VTile *unit_list, const int *units_by_blocks, int *err) {
    if (k <= 0) return;
    ProfScope ps(st, ST_INTEGRALS, 2.0 * k * g.pair_points,
                 2.0 * g.table_values + 4.0 * k * g.n * g.n * g.n + 4.0 * k * nchi * nphi);
    check(cudaMemsetAsync(out, 0, sizeof(float) * (size_t)k * nchi * nphi, st), "memset(integrals)");
    check(cudaMemsetAsync(scratch_bits, 0, sizeof(unsigned) * k, st), "memset vmaxabs");
    const long long n3 = (long long)g.n * g.n * g.n;
    vmaxabs_kernel<<<dim3(64, k), 256, 0, st>>>(V, n3, scratch_bits);
    check_launch("vmaxabs_kernel");
    scale_kernel<<<(k + 127) / 128, 128, 0, st>>>(scratch_bits, k, scale);
    check_launch("scale_kernel");
    CUtensorMap mx;
    if (!encode_map_2d(&mx, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, chi_fm16, (unsigned long long)TILE_PTS,
                       (unsigned long long)nslots, (unsigned long long)TILE_PTS * 2, 64, 128))
        throw CudaError{cudaErrorInvalidValue, "cuTensorMapEncodeTiled (integrals)"};
    if (NPmax > 128 || NPmax % 16) throw CudaError{cudaErrorInvalidValue, "integrals_tc: phi per tile"};
    CUtensorMap mp;
    if (!encode_map_2d(&mp, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, phi_fm16, (unsigned long long)TILE_PTS,
                       (unsigned long long)nslots_phi, (unsigned long long)TILE_PTS * 2, 64, NPmax))
        throw CudaError{cudaErrorInvalidValue, "cuTensorMapEncodeTiled (integrals phi)"};
    // one launch per class of units by 128-row chi blocks (1, 2, 3), one state per CTA: the
    // smaller a class's shared memory and TMEM, the more CTAs share an SM (3, 2, 1)
    if (NPmax > 128) throw CudaError{cudaErrorInvalidValue, "integrals_tc: more than 128 phi per tile"};
    static const bool attr = [&]() {   // once per process, thread-safe
        check(cudaFuncSetAttribute(integrals_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024),
              "attr integrals_tc");
        return true;
    }();
    (void)attr;
    const bool vec_ok = (nphi % 4 == 0) && ((reinterpret_cast<unsigned long long>(out) & 15ull) == 0);
    const VTile *lp = unit_list;
    for (int c = 0; c < 3; ++c) {
        const int cnt = units_by_blocks[c];
        const VTile *lst = lp;
        lp += cnt;
        if (cnt == 0) continue;
        const int mbmax = c + 1;
        const int stride = 128;                           // one state: NB = NPmax <= 128 columns
        const int tmem_cols = mbmax == 1 ? 128 : (mbmax == 2 ? 256 : 512);
        const size_t sm = integrals_tc_smem(NPmax, 1, mbmax);
        // grid.y holds at most 65535 units: launch the class in slices
        for (int u0 = 0; u0 < cnt; u0 += 65535) {
            dim3 grid(k, std::min(65535, cnt - u0));
            integrals_tc_kernel<<<grid, 192, sm, st>>>(mx, mp, g.n, g.nt, NPmax, k, chi.ids, phi.ids, nchi, nphi, V,
                                                       scale, (float)g.dV, out, vec_ok, stride, lst + u0, mbmax,
                                                       tmem_cols, err, active_wait_limit());
            check_launch("integrals_tc_kernel");
        }
    }
}

}  // namespace tddft

// ================================================================================================
// Allocation-free variant of the tensor-core response density. Some callers cannot allocate
// device memory at the point where they need a density: a process whose own pool allocator has
// already reserved the device memory, or a latency-bound loop in which cudaMalloc / cudaFree
// (which synchronise the whole device) are not allowed. For them the per-state scale words and
// the wait-expiry flag live in one fixed file-scope device array instead of context workspace,
// and the caller passes float32 device buffers for P and rho. The array is shared by every call
// on a device, so overlapping calls race and must be serialised by the caller.
namespace tddft {

constexpr int NOALLOC_MAX_STATES = 64;

struct NoallocScratch {
    unsigned bits[NOALLOC_MAX_STATES];
    float scale[NOALLOC_MAX_STATES];
    int err;
};

// one copy per device that loads the library (64 + 64 words + a flag, about 520 bytes); each call
// clears it before use, so nothing in it needs to start at zero
static __device__ __align__(256) NoallocScratch g_density_noalloc_scratch;

namespace {
std::mutex g_noalloc_mu;
NoallocScratch *g_noalloc_addr[64] = {};   // device address of the array, per device ordinal
}  // namespace

// device address of the scratch array on the current device, looked up once per device with that
// device current (the first call on a device does this set-up)
NoallocScratch *noalloc_scratch_address() {
    int dev = 0;
    check(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= 64) throw CudaError{cudaErrorInvalidDevice, "device ordinal beyond 63"};
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        check(cudaGetSymbolAddress(&p, g_density_noalloc_scratch), "cudaGetSymbolAddress(density scratch)");
        g_noalloc_addr[dev] = static_cast<NoallocScratch *>(p);
    }
    return g_noalloc_addr[dev];
}

int noalloc_max_states() { return NOALLOC_MAX_STATES; }

// rho[k][n^3] from P[k][N_chi][N_phi] (float32, device); no allocation, no context workspace.
void response_density_tc_noalloc(cudaStream_t st, const GridShape &g, const TileSet<float> &chi,
                                 const TileSet<float> &phi, const unsigned short *chi_pm, int CK, int NPmax,
                                 int nphi, const float *P, long long sP, int k, float *rho,
                                 const unsigned short *phi_pm) {
    if (k < 1 || k > NOALLOC_MAX_STATES) throw CudaError{cudaErrorInvalidValue, "k beyond the scratch maximum"};
    NoallocScratch *s = noalloc_scratch_address();
    // the scale words must start at zero for the max reduction; the flag is cleared per call
    check(cudaMemsetAsync(s, 0, sizeof(NoallocScratch), st), "clear density scratch");
    maxabs_kernel<<<dim3(64, k), 256, 0, st>>>(P, sP, k, s->bits);
    check_launch("maxabs_kernel");
    scale_kernel<<<(k + 127) / 128, 128, 0, st>>>(s->bits, k, s->scale);
    check_launch("scale_kernel");
    CUtensorMap mx;
    if (!encode_map_2d(&mx, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, chi_pm, (unsigned long long)CK,
                       (unsigned long long)chi.ntiles * TILE_PTS, (unsigned long long)CK * 2, 64, 128))
        throw CudaError{cudaErrorInvalidValue, "cuTensorMapEncodeTiled (density)"};
    const int NP = NPmax, KBmax = CK / 64;
    const int G = density_tc_group(KBmax, NP, k);
    if (G < 1) throw CudaError{cudaErrorInvalidValue, "density_tc: tile too large for shared memory"};
    const size_t sm = density_tc_smem(KBmax, G * NP);
    check(cudaFuncSetAttribute(density_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024),
          "attr density_tc");
    dim3 grid((k + G - 1) / G, chi.ntiles);
    density_tc_kernel<<<grid, DENS_THREADS, sm, st>>>(mx, g.n, g.nt, KBmax, NP, G, k, chi.off, chi.ids, phi.off,
                                                      phi.ids, phi.val, nphi, P, sP, s->scale, rho, &s->err, 0,
                                                      NP % 32 == 0 ? phi_pm : nullptr, active_wait_limit());
    check_launch("density_tc_kernel (allocation-free)");
}

// wait-expiry flag of the last call on this device (synchronises the stream)
int response_density_tc_noalloc_error(cudaStream_t st) {
    NoallocScratch *s = noalloc_scratch_address();
    int h = 0;
    check(cudaMemcpyAsync(&h, &s->err, sizeof(int), cudaMemcpyDeviceToHost, st), "D2H density flag");
    check(cudaStreamSynchronize(st), "sync density flag");
    return h;
}

}  // namespace tddft
