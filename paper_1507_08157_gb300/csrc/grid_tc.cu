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

namespace tddft {

using namespace tc;

namespace {

struct __align__(8) DensShared {
    unsigned long long a_full;
    unsigned long long mma_done;
    unsigned int tmem_base;
    int abort;
};

constexpr int DENS_TMEM_COLS = 256;

__global__ void __launch_bounds__(192, 1) density_tc_kernel(
    const __grid_constant__ CUtensorMap mX,   // point-major chi: [tile*512 + point][CK] f16
    int n, int nt, int KBmax, int NP, int G, int k, const int *__restrict__ coff, const int *__restrict__ cids,
    const int *__restrict__ poff, const int *__restrict__ pids, const float *__restrict__ pval, int nphi,
    const float *__restrict__ P, long long sP, const float *__restrict__ pscale, float *__restrict__ rho,
    int *err) {
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
    unsigned char *A = base;                             // KBmax x [128 rows x 128 B]
    unsigned char *B = base + (size_t)KBmax * 16384;     // KBmax x [NB rows x 128 B]
    DensShared *ctl = reinterpret_cast<DensShared *>(B + (size_t)KBmax * NB * 128);
    volatile int *abort = &ctl->abort;

    if (threadIdx.x == 0) {
        mbar_init(&ctl->a_full, 1);
        mbar_init(&ctl->mma_done, 1);
        ctl->abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 5) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ctl->tmem_base)),
                     "r"(DENS_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // gather the P block: row (s, b), K = a, 8 consecutive a per 16-byte chunk
    {
        const int chunks = KB * 8;                       // 16-byte chunks per row
        for (int idx = threadIdx.x; idx < NB * chunks; idx += blockDim.x) {
            const int row = idx % NB, ch = idx / NB;     // consecutive threads -> consecutive rows (b)
            const int sl = row / NP, b = row - sl * NP;
            const int kb = ch >> 3, c8 = ch & 7;
            unsigned short h[8];
            const bool live = sl < gs && b < np;
            const float sc = live ? pscale[s0 + sl] : 0.0f;
            const float *Ps = P + (long long)(s0 + (live ? sl : 0)) * sP;
            const int col = live ? pids[p0 + b] : 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int a = kb * 64 + c8 * 8 + j;
                float v = 0.0f;
                if (live && a < nc) v = Ps[(long long)cids[c0 + a] * nphi + col] * sc;
                h[j] = __half_as_ushort(__float2half_rn(v));
            }
            uint4 q;
            q.x = h[0] | ((unsigned)h[1] << 16);
            q.y = h[2] | ((unsigned)h[3] << 16);
            q.z = h[4] | ((unsigned)h[5] << 16);
            q.w = h[6] | ((unsigned)h[7] << 16);
            *reinterpret_cast<uint4 *>(B + (size_t)kb * NB * 128 + sw128_offset(row, c8)) = q;
        }
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const unsigned tmem = ctl->tmem_base;
    const unsigned idesc = idesc_f16(128, NB);

    for (int pb = 0; pb < TILE_PTS / 128; ++pb) {
        const unsigned par = pb & 1;
        if (warp == 4 && lane == 0 && !*abort) {
            mbar_expect_tx(&ctl->a_full, KB * 16384);
            for (int kb = 0; kb < KB; ++kb)
                tma_load_2d(A + kb * 16384, &mX, &ctl->a_full, kb * 64, t * TILE_PTS + pb * 128);
        } else if (warp == 5 && lane == 0) {
            if (mbar_wait(&ctl->a_full, par, abort)) {
                tc_fence_after();
                for (int kb = 0; kb < KB; ++kb) {
                    const unsigned a = smem_u32(A + kb * 16384), bb = smem_u32(B + (size_t)kb * NB * 128);
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        mma_f16(tmem, smem_desc(a + kk * 32), smem_desc(bb + kk * 32), idesc,
                                (kb > 0 || kk > 0) ? 1u : 0u);
                }
            }
            mma_commit(&ctl->mma_done);
        } else if (warp < 4) {
            const bool ok = mbar_wait(&ctl->mma_done, par, abort) && !*abort;
            tc_fence_after();
            const int lp = pb * 128 + warp * 32 + lane;      // tile point of this TMEM lane
            float acc[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[i] = 0.0f;
            for (int c = 0; c < NB; c += 32) {
                float v[32];
                tmem_ld32(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c, v);
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int col = c + j;
                    const int sl = col / NP, b = col - sl * NP;
                    if (sl < gs && b < np) {
                        const float w = v[j] * pval[(long long)(p0 + b) * TILE_PTS + lp];
#pragma unroll
                        for (int q = 0; q < 16; ++q)
                            if (q == sl) acc[q] += w;
                    }
                }
            }
            const int gx = tx * TILE + (lp >> 6), gy = ty * TILE + ((lp >> 3) & 7), gz = tz * TILE + (lp & 7);
            if (ok && gx < n && gy < n && gz < n) {
                const long long gi = ((long long)gx * n + gy) * n + gz;
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    if (q < gs) rho[(long long)(s0 + q) * n3 + gi] = acc[q] / pscale[s0 + q];
            }
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
    }
    if (warp == 5) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(DENS_TMEM_COLS));
    }
    if (threadIdx.x == 0 && ctl->abort) atomicExch(err, 1);
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
    const int s = threadIdx.x;
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
    return 1024 + (size_t)KBmax * 16384 + (size_t)KBmax * NB * 128 + sizeof(DensShared);
}

// largest state group G (<= 16, G * NP <= 256) whose shared memory fits; 0 if none does
int density_tc_group(int KBmax, int NP, int k) {
    for (int G = std::min(16, std::min(k, 256 / NP)); G >= 1; --G)
        if (density_tc_smem(KBmax, G * NP) <= 227 * 1024) return G;
    return 0;
}

void response_density_tc(cudaStream_t st, const GridShape &g, const TileSet<float> &chi,
                         const TileSet<float> &phi, const unsigned short *chi_pm, int CK, int NPmax, int nphi,
                         const float *P, long long sP, int k, float *rho, unsigned *scratch_bits,
                         float *scale, int *err) {
    if (k <= 0) return;
    ProfScope ps(st, ST_DENSITY, 2.0 * k * g.pair_points, 2.0 * g.table_values + 4.0 * k * g.n * g.n * g.n);
    check(cudaMemsetAsync(scratch_bits, 0, sizeof(unsigned) * k, st), "memset maxabs");
    maxabs_kernel<<<dim3(64, k), 256, 0, st>>>(P, sP, k, scratch_bits);
    check_launch("maxabs_kernel");
    scale_kernel<<<1, 32, 0, st>>>(scratch_bits, k, scale);
    check_launch("scale_kernel");
    CUtensorMap mx;
    if (!encode_map_2d(&mx, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, chi_pm, (unsigned long long)CK,
                       (unsigned long long)chi.ntiles * TILE_PTS, (unsigned long long)CK * 2, 64, 128))
        throw CudaError{cudaErrorInvalidValue, "cuTensorMapEncodeTiled (density)"};
    const int NP = NPmax, KBmax = CK / 64;
    const int G = density_tc_group(KBmax, NP, k);
    if (G < 1) throw CudaError{cudaErrorInvalidValue, "density_tc: tile too large for shared memory"};
    const int ngroups = (k + G - 1) / G;
    const size_t sm = density_tc_smem(KBmax, G * NP);
    static bool attr = false;
    if (!attr) {
        check(cudaFuncSetAttribute(density_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024),
              "attr density_tc");
        attr = true;
    }
    dim3 grid(ngroups, chi.ntiles);
    density_tc_kernel<<<grid, 192, sm, st>>>(mx, g.n, g.nt, KBmax, NP, G, k, chi.off, chi.ids, phi.off, phi.ids,
                                             phi.val, nphi, P, sP, scale, rho, err);
    check_launch("density_tc_kernel");
}

}  // namespace tddft
