// Real-space grid work of the response potential V_SCF (paper Secs. II A, II C, III A), SIMT path:
//
//  * response_density: rho_s(r) = sum_ab chi_a(r) P_s,ab phi_b(r), owner-computes per 8^3 tile:
//      T[r][b] = sum_a X[a][r] P[a][b] as a tile-local GEMM, then rho[r] = sum_b T[r][b] Phi[b][r]
//      reduced across the 16 lanes that hold one point's row. No atomics: every grid point
//      belongs to exactly one tile.
//  * potential_integrals: V_s,ab = dV sum_r chi_a(r) V_s(r) phi_b(r): per tile a GEMM over the
//      tile's points, X (a x r) times (V * Phi)^T (r x b), added into the output matrix.
//  * hartree_fxc: v_H = IFFT[4 pi FFT(rho) / |G|^2] (G = 0 dropped) plus f_xc * rho, with a
//      hand-written mixed-radix (2, 3, 4, 5) Stockham FFT; two real states share one complex
//      transform (rho_a + i rho_b), since the kernel is real and even.
//  * fxc_lda: f_xc = d^2(n eps_xc)/dn^2, Slater exchange + Perdew-Wang 1992 correlation.
#include "tddft_internal.h"

#include <cmath>

namespace tddft {

namespace {

__device__ __forceinline__ long long tile_point_index(int n, int nt, int t, int lp, bool &valid) {
    const int tx = t / (nt * nt), ty = (t / nt) % nt, tz = t % nt;
    const int lx = lp >> 6, ly = (lp >> 3) & 7, lz = lp & 7;
    const int gx = tx * TILE + lx, gy = ty * TILE + ly, gz = tz * TILE + lz;
    valid = gx < n && gy < n && gz < n;
    return ((long long)gx * n + gy) * n + gz;
}

// ------------------------------------------------------------------------------------------------
// response density
template <typename T>
__global__ void __launch_bounds__(256) density_kernel(int n, int nt, const int *__restrict__ coff,
                                                      const int *__restrict__ cids,
                                                      const T *__restrict__ cval,
                                                      const int *__restrict__ poff,
                                                      const int *__restrict__ pids,
                                                      const T *__restrict__ pval, int nphi,
                                                      const T *__restrict__ P, long long sP,
                                                      T *__restrict__ rho) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *Xs = reinterpret_cast<T *>(smem_raw);   // [16][64]
    T *Ps = Xs + 16 * 64;                      // [16][65]
    T *Phs = Ps + 16 * 65;                     // [64][65]
    T *rs = Phs + 64 * 65;                     // [512]
    const int t = blockIdx.x, s = blockIdx.y;
    const int c0 = coff[t], nc = coff[t + 1] - c0;
    const int p0 = poff[t], np = poff[t + 1] - p0;
    const T *Pst = P + (long long)s * sP;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    for (int i = tid; i < TILE_PTS; i += 256) rs[i] = T(0);
    __syncthreads();
    if (nc > 0 && np > 0) {
        for (int pb = 0; pb < TILE_PTS / 64; ++pb) {
            for (int bb = 0; bb < np; bb += 64) {
                T acc[4][4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
                for (int ab = 0; ab < nc; ab += 16) {
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int m = tid & 63, kk = (tid >> 6) + 4 * i;
                        const int a = ab + kk;
                        Xs[kk * 64 + m] = a < nc ? cval[(long long)(c0 + a) * TILE_PTS + pb * 64 + m] : T(0);
                        const int bj = bb + m;
                        Ps[kk * 65 + m] = (a < nc && bj < np)
                                              ? Pst[(long long)cids[c0 + a] * nphi + pids[p0 + bj]]
                                              : T(0);
                    }
                    __syncthreads();
#pragma unroll
                    for (int kk = 0; kk < 16; ++kk) {
                        T xa[4], pb4[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) xa[u] = Xs[kk * 64 + ty + 16 * u];
#pragma unroll
                        for (int v = 0; v < 4; ++v) pb4[v] = Ps[kk * 65 + tx + 16 * v];
#pragma unroll
                        for (int u = 0; u < 4; ++u)
#pragma unroll
                            for (int v = 0; v < 4; ++v) acc[u][v] = fma(xa[u], pb4[v], acc[u][v]);
                    }
                    __syncthreads();
                }
                // stage Phi[b][point] for this (point block, b block)
                for (int i = 0; i < 16; ++i) {
                    const int m = tid & 63, j = (tid >> 6) + 4 * i;
                    const int bj = bb + j;
                    Phs[j * 65 + m] = bj < np ? pval[(long long)(p0 + bj) * TILE_PTS + pb * 64 + m] : T(0);
                }
                __syncthreads();
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    T part = T(0);
#pragma unroll
                    for (int v = 0; v < 4; ++v) part = fma(acc[u][v], Phs[(tx + 16 * v) * 65 + ty + 16 * u], part);
#pragma unroll
                    for (int off = 8; off > 0; off >>= 1) part += __shfl_xor_sync(0xffffffffu, part, off);
                    if (tx == 0) rs[pb * 64 + ty + 16 * u] += part;
                }
                __syncthreads();
            }
        }
    }
    for (int lp = tid; lp < TILE_PTS; lp += 256) {
        bool valid;
        const long long gi = tile_point_index(n, nt, t, lp, valid);
        if (valid) rho[(long long)s * n * n * n + gi] = rs[lp];
    }
}

// ------------------------------------------------------------------------------------------------
// potential integrals
template <typename T>
__global__ void __launch_bounds__(256) integrals_kernel(int n, int nt, const int *__restrict__ coff,
                                                        const int *__restrict__ cids,
                                                        const T *__restrict__ cval,
                                                        const int *__restrict__ poff,
                                                        const int *__restrict__ pids,
                                                        const T *__restrict__ pval, int nchi,
                                                        int nphi, const T *__restrict__ V, T dV,
                                                        T *__restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *Xs = reinterpret_cast<T *>(smem_raw);   // [16][65]  (point, a)
    T *Ws = Xs + 16 * 65;                      // [16][65]  (point, b)
    T *Vs = Ws + 16 * 65;                      // [512]
    const int t = blockIdx.x, s = blockIdx.y;
    const int c0 = coff[t], nc = coff[t + 1] - c0;
    const int p0 = poff[t], np = poff[t + 1] - p0;
    if (nc == 0 || np == 0) return;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const long long n3 = (long long)n * n * n;
    for (int lp = tid; lp < TILE_PTS; lp += 256) {
        bool valid;
        const long long gi = tile_point_index(n, nt, t, lp, valid);
        Vs[lp] = valid ? V[(long long)s * n3 + gi] : T(0);
    }
    __syncthreads();
    T *Os = out + (long long)s * nchi * nphi;
    for (int ab = 0; ab < nc; ab += 64) {
        for (int bb = 0; bb < np; bb += 64) {
            T acc[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
            for (int pc = 0; pc < TILE_PTS; pc += 16) {
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int kk = tid & 15, m = (tid >> 4) + 16 * i;
                    const int a = ab + m, bj = bb + m;
                    Xs[kk * 65 + m] = a < nc ? cval[(long long)(c0 + a) * TILE_PTS + pc + kk] : T(0);
                    Ws[kk * 65 + m] = bj < np ? pval[(long long)(p0 + bj) * TILE_PTS + pc + kk] * Vs[pc + kk] : T(0);
                }
                __syncthreads();
#pragma unroll
                for (int kk = 0; kk < 16; ++kk) {
                    T xa[4], wb[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) xa[u] = Xs[kk * 65 + ty + 16 * u];
#pragma unroll
                    for (int v = 0; v < 4; ++v) wb[v] = Ws[kk * 65 + tx + 16 * v];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) acc[u][v] = fma(xa[u], wb[v], acc[u][v]);
                }
                __syncthreads();
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int a = ab + ty + 16 * u;
                if (a >= nc) continue;
                const long long row = (long long)cids[c0 + a] * nphi;
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const int bj = bb + tx + 16 * v;
                    if (bj < np) atomicAdd(&Os[row + pids[p0 + bj]], dV * acc[u][v]);
                }
            }
        }
    }
}

// ------------------------------------------------------------------------------------------------
// FFT: mixed-radix Stockham in shared memory
template <typename T> struct C2;
template <> struct C2<float> { using t = float2; };
template <> struct C2<double> { using t = double2; };

struct Plan {
    int n, nst;
    int radix[12];
};

bool make_plan(int n, Plan &p) {
    p.n = n;
    p.nst = 0;
    int m = n;
    while (m > 1) {
        int r;
        if (m % 4 == 0) r = 4;
        else if (m % 2 == 0) r = 2;
        else if (m % 3 == 0) r = 3;
        else if (m % 5 == 0) r = 5;
        else return false;
        if (p.nst >= 12) return false;
        p.radix[p.nst++] = r;
        m /= r;
    }
    return true;
}

template <typename T> __device__ __forceinline__ void sincospi_t(T x, T *s, T *c);
template <> __device__ __forceinline__ void sincospi_t<float>(float x, float *s, float *c) { sincospif(x, s, c); }
template <> __device__ __forceinline__ void sincospi_t<double>(double x, double *s, double *c) { sincospi(x, s, c); }

template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return {a.x + b.x, a.y + b.y}; }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return {a.x - b.x, a.y - b.y}; }
template <typename V, typename T> __device__ __forceinline__ V cmul(V a, T c, T s) {
    return {a.x * c - a.y * s, a.x * s + a.y * c};
}

// DFT of size R with sign SG (-1 forward, +1 inverse) on v[0..R)
template <typename T, int SG, typename V>
__device__ __forceinline__ void small_dft(int R, V *v) {
    if (R == 2) {
        V a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if (R == 4) {
        V a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
        V b0 = cadd(v[1], v[3]), b1 = csub(v[1], v[3]);
        // i * SG * b1
        V ib1 = {-T(SG) * b1.y, T(SG) * b1.x};
        v[0] = cadd(a0, b0);
        v[2] = csub(a0, b0);
        v[1] = cadd(a1, ib1);
        v[3] = csub(a1, ib1);
    } else if (R == 3) {
        const T h = T(0.86602540378443864676);   // sqrt(3)/2
        V t1 = cadd(v[1], v[2]), t2 = csub(v[1], v[2]);
        V m = {v[0].x - T(0.5) * t1.x, v[0].y - T(0.5) * t1.y};
        V it2 = {-T(SG) * h * t2.y, T(SG) * h * t2.x};
        v[0] = cadd(v[0], t1);
        v[1] = cadd(m, it2);
        v[2] = csub(m, it2);
    } else {  // R == 5
        const T c1 = T(0.30901699437494742410), c2 = T(-0.80901699437494742410);   // cos(2pi/5), cos(4pi/5)
        const T s1 = T(0.95105651629515357212), s2 = T(0.58778525229247312917);    // sin(2pi/5), sin(4pi/5)
        V a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
        V a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
        V x0 = v[0];
        V m1 = {x0.x + c1 * a1.x + c2 * a2.x, x0.y + c1 * a1.y + c2 * a2.y};
        V m2 = {x0.x + c2 * a1.x + c1 * a2.x, x0.y + c2 * a1.y + c1 * a2.y};
        // SG * i * (s1 b1 + s2 b2) and SG * i * (s2 b1 - s1 b2)
        V n1 = {s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y};
        V n2 = {s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y};
        V in1 = {-T(SG) * n1.y, T(SG) * n1.x};
        V in2 = {-T(SG) * n2.y, T(SG) * n2.x};
        v[0] = {x0.x + a1.x + a2.x, x0.y + a1.y + a2.y};
        v[1] = cadd(m1, in1);
        v[4] = csub(m1, in1);
        v[2] = cadd(m2, in2);
        v[3] = csub(m2, in2);
    }
}

// Per-CTA tables of a plan, built once before the transforms: the stage twiddles
// tw[off_s + kk (R - 1) + r - 1] = exp(-2 pi i kk r / (Ns R)) (forward sign; the inverse takes the
// conjugate) and kk = j mod Ns for every butterfly index j of every stage. The transforms then
// look these up instead of evaluating sines and dividing per element.
constexpr int FFT_KK_BYTES = 2048;      // sum over stages of n / R (n <= 256)

template <typename T>
__device__ void fft_tables(const Plan &pl, typename C2<T>::t *tw, unsigned char *kkt) {
    const int n = pl.n;
    int Ns = 1, toff = 0, koff = 0;
    for (int st = 0; st < pl.nst; ++st) {
        const int R = pl.radix[st], nb = n / R;
        for (int i = threadIdx.x; i < Ns * (R - 1); i += blockDim.x) {
            const int kk = i / (R - 1), r = i - kk * (R - 1) + 1;
            T sn, cs;
            sincospi_t<T>(T(-2) * T(kk * r) / T(Ns * R), &sn, &cs);
            tw[toff + i] = {cs, sn};
        }
        for (int jj = threadIdx.x; jj < nb; jj += blockDim.x) kkt[koff + jj] = (unsigned char)(jj % Ns);
        toff += Ns * (R - 1);
        koff += nb;
        Ns *= R;
    }
}

// One Stockham stage of radix R (a compile-time constant, so that the R values of a butterfly
// stay in registers) on one line: butterflies j = t0, t0 + tpl, ... < nb = n / R.
template <typename T, int SG, int R>
__device__ __forceinline__ void fft_stage(const typename C2<T>::t *src, typename C2<T>::t *dst, int nb, int Ns,
                                          int t0, int tpl, const typename C2<T>::t *tws,
                                          const unsigned char *kks) {
    using V = typename C2<T>::t;
    for (int j = t0; j < nb; j += tpl) {
        V v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[j + r * nb];
        const int kk = kks[j];
        if (Ns > 1) {
            const V *w = tws + kk * (R - 1) - 1;
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], w[r].x, SG < 0 ? w[r].y : -w[r].y);
        }
        small_dft<T, SG>(R, v);
        const int base = (j - kk) * R + kk;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[base + r * Ns] = v[r];
    }
}

// FFT of `lines` lines of length n held at buf0 (line-major, lines ld >= n apart); returns the
// buffer with the result. blockDim.x / lines threads work on each line (lines divides blockDim.x).
template <typename T, int SG>
__device__ typename C2<T>::t *fft_lines(typename C2<T>::t *buf0, typename C2<T>::t *buf1, int lines, int ld,
                                        const Plan &pl, const typename C2<T>::t *tw, const unsigned char *kkt) {
    using V = typename C2<T>::t;
    V *in = buf0, *out = buf1;
    const int n = pl.n;
    const int tpl = blockDim.x / lines;
    const int line = threadIdx.x / tpl, t0 = threadIdx.x - line * tpl;
    int Ns = 1, toff = 0, koff = 0;
    for (int st = 0; st < pl.nst; ++st) {
        const int R = pl.radix[st];
        const int nb = n / R;
        if (line < lines) {
            const V *src = in + line * ld;
            V *dst = out + line * ld;
            switch (R) {
                case 2: fft_stage<T, SG, 2>(src, dst, nb, Ns, t0, tpl, tw + toff, kkt + koff); break;
                case 3: fft_stage<T, SG, 3>(src, dst, nb, Ns, t0, tpl, tw + toff, kkt + koff); break;
                case 4: fft_stage<T, SG, 4>(src, dst, nb, Ns, t0, tpl, tw + toff, kkt + koff); break;
                default: fft_stage<T, SG, 5>(src, dst, nb, Ns, t0, tpl, tw + toff, kkt + koff); break;
            }
        }
        __syncthreads();
        V *tmp = in;
        in = out;
        out = tmp;
        toff += Ns * (R - 1);
        koff += nb;
        Ns *= R;
    }
    return in;
}

template <typename T> __host__ __device__ constexpr int lines_per_cta() { return sizeof(T) == 8 ? 8 : 16; }

// forward transform along z of (rho_a + i rho_b); lines = n*n per pair
template <typename T>
__global__ void __launch_bounds__(256) fft_z_forward_real(Plan pl, const T *__restrict__ rho, int k,
                                                          typename C2<T>::t *__restrict__ work) {
    using V = typename C2<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = pl.n, L = lines_per_cta<T>();
    V *b0 = reinterpret_cast<V *>(smem_raw), *b1 = b0 + L * n, *tw = b1 + L * n;
    unsigned char *kkt = reinterpret_cast<unsigned char *>(tw + n);
    fft_tables<T>(pl, tw, kkt);
    const long long n3 = (long long)n * n * n;
    const int pair = blockIdx.y;
    const long long line0 = (long long)blockIdx.x * L;
    const long long nlines = (long long)n * n;
    const T *ra = rho + (2LL * pair) * n3;
    const bool has_b = 2 * pair + 1 < k;
    const T *rb = rho + (2LL * pair + 1) * n3;
    for (int i = threadIdx.x; i < L * n; i += blockDim.x) {
        const int l = i / n, j = i - l * n;
        V v = {T(0), T(0)};
        if (line0 + l < nlines) {
            const long long gi = (line0 + l) * n + j;
            v.x = ra[gi];
            v.y = has_b ? rb[gi] : T(0);
        }
        b0[i] = v;
    }
    __syncthreads();
    V *res = fft_lines<T, -1>(b0, b1, L, n, pl, tw, kkt);
    V *w = work + (long long)pair * n3;
    for (int i = threadIdx.x; i < L * n; i += blockDim.x) {
        const int l = i / n, j = i - l * n;
        if (line0 + l < nlines) w[(line0 + l) * n + j] = res[i];
    }
}

// inverse transform along z, then V = Re/Im + fxc * rho
template <typename T>
__global__ void __launch_bounds__(256) fft_z_inverse_real(Plan pl, const typename C2<T>::t *__restrict__ work,
                                                          const T *__restrict__ rho,
                                                          const T *__restrict__ fxc, int k,
                                                          T *__restrict__ V) {
    using Vc = typename C2<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = pl.n, L = lines_per_cta<T>();
    Vc *b0 = reinterpret_cast<Vc *>(smem_raw), *b1 = b0 + L * n, *tw = b1 + L * n;
    unsigned char *kkt = reinterpret_cast<unsigned char *>(tw + n);
    fft_tables<T>(pl, tw, kkt);
    const long long n3 = (long long)n * n * n;
    const int pair = blockIdx.y;
    const long long line0 = (long long)blockIdx.x * L;
    const long long nlines = (long long)n * n;
    const Vc *w = work + (long long)pair * n3;
    for (int i = threadIdx.x; i < L * n; i += blockDim.x) {
        const int l = i / n, j = i - l * n;
        b0[i] = (line0 + l < nlines) ? w[(line0 + l) * n + j] : Vc{T(0), T(0)};
    }
    __syncthreads();
    Vc *res = fft_lines<T, +1>(b0, b1, L, n, pl, tw, kkt);
    const bool has_b = 2 * pair + 1 < k;
    for (int i = threadIdx.x; i < L * n; i += blockDim.x) {
        const int l = i / n, j = i - l * n;
        if (line0 + l >= nlines) continue;
        const long long gi = (line0 + l) * n + j;
        const T f = fxc ? fxc[gi] : T(0);
        const long long ia = (2LL * pair) * n3 + gi;
        V[ia] = res[i].x + f * rho[ia];
        if (has_b) {
            const long long ib = (2LL * pair + 1) * n3 + gi;
            V[ib] = res[i].y + f * rho[ib];
        }
    }
}

// transform along a strided axis (stride s: n for y, n*n for x) for a block of W consecutive
// z columns; AXIS 1 = y, 0 = x. For the x axis the forward transform, the Poisson kernel
// 4 pi / |G|^2 / n^3 (G = 0 -> 0) and the inverse transform are fused.
template <typename T, int AXIS, int SG, bool POISSON>
__global__ void __launch_bounds__(256) fft_strided(Plan pl, typename C2<T>::t *__restrict__ work,
                                                   T two_pi_over_L) {
    using V = typename C2<T>::t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = pl.n, W = lines_per_cta<T>();
    // lines n + 1 apart: the transposing loads and stores (consecutive threads, consecutive
    // lines) then hit distinct banks
    const int ld = n + 1;
    V *b0 = reinterpret_cast<V *>(smem_raw), *b1 = b0 + W * ld, *tw = b1 + W * ld;
    unsigned char *kkt = reinterpret_cast<unsigned char *>(tw + n);
    fft_tables<T>(pl, tw, kkt);
    const long long n3 = (long long)n * n * n;
    const int pair = blockIdx.z;
    const int o = blockIdx.y;            // x index (AXIS 1) or y index (AXIS 0)
    const int w0 = blockIdx.x * W;       // first z column
    const long long s = AXIS == 1 ? n : (long long)n * n;
    const long long base = (long long)pair * n3 + (AXIS == 1 ? (long long)o * n * n : (long long)o * n);
    V *data = work + base;
    for (int i = threadIdx.x; i < W * n; i += blockDim.x) {
        const int j = i / W, w = i - j * W;    // consecutive threads -> consecutive z
        V v = {T(0), T(0)};
        if (w0 + w < n) v = data[(long long)j * s + w0 + w];
        b0[w * ld + j] = v;
    }
    __syncthreads();
    V *res;
    if (!POISSON) {
        res = fft_lines<T, SG>(b0, b1, W, ld, pl, tw, kkt);
    } else {
        res = fft_lines<T, -1>(b0, b1, W, ld, pl, tw, kkt);
        const T inv_n3 = T(1) / T(n3);
        for (int i = threadIdx.x; i < W * n; i += blockDim.x) {
            const int w = i / n, j = i - w * n;
            const int mx = j <= n / 2 ? j : j - n;
            const int my = o <= n / 2 ? o : o - n;
            const int zz = w0 + w;
            const int mz = zz <= n / 2 ? zz : zz - n;
            const T g2 = two_pi_over_L * two_pi_over_L * T(mx * mx + my * my + mz * mz);
            const T kern = (mx == 0 && my == 0 && mz == 0) ? T(0) : T(4.0 * 3.14159265358979323846) / g2 * inv_n3;
            res[w * ld + j].x *= kern;
            res[w * ld + j].y *= kern;
        }
        __syncthreads();
        V *other = (res == b0) ? b1 : b0;
        res = fft_lines<T, +1>(res, other, W, ld, pl, tw, kkt);
    }
    for (int i = threadIdx.x; i < W * n; i += blockDim.x) {
        const int j = i / W, w = i - j * W;
        if (w0 + w < n) data[(long long)j * s + w0 + w] = res[w * ld + j];
    }
}

// ------------------------------------------------------------------------------------------------
// LDA kernel
// f_xc(n) = d^2(n eps_xc)/dn^2 (Slater exchange, PW92 correlation at zeta = 0), derived here in
// the variable x = rs^(1/2) = (3 / (4 pi n))^(1/6), in which PW92's denominator is the quartic
// Q(x) = 2A (b1 x + b2 x^2 + b3 x^3 + b4 x^4) and eps_c = -2A (1 + a1 x^2) ln(1 + 1/Q). With
// dx/dn = -x / (6n), d^2(n eps)/dn^2 = x (x eps'' - 5 eps') / (36 n) (primes: d/dx); exchange,
// n eps_x = -(3/4)(3/pi)^(1/3) n^(4/3), gives -(4/9)(3/4)(3/pi)^(1/3) n^(-2/3).
__global__ void fxc_kernel(const double *__restrict__ n0, double *__restrict__ out, long long npts) {
    const double A = 0.031091, a1 = 0.21370;
    const double b1 = 7.5957, b2 = 3.5876, b3 = 1.6382, b4 = 0.49294;
    const double pi = 3.14159265358979323846;
    const double cx = 0.75 * cbrt(3.0 / pi);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < npts;
         i += (long long)gridDim.x * blockDim.x) {
        const double n = n0[i];
        if (!(n >= 1e-10)) {
            out[i] = 0.0;
            continue;
        }
        const double fx = -(4.0 / 9.0) * cx / cbrt(n * n);
        const double x = sqrt(cbrt(3.0 / (4.0 * pi * n)));
        const double Q = 2.0 * A * x * (b1 + x * (b2 + x * (b3 + x * b4)));
        const double Q1 = 2.0 * A * (b1 + x * (2.0 * b2 + x * (3.0 * b3 + x * 4.0 * b4)));
        const double Q2 = 2.0 * A * (2.0 * b2 + x * (6.0 * b3 + x * 12.0 * b4));
        const double P0 = -2.0 * A * (1.0 + a1 * x * x), P1 = -4.0 * A * a1 * x, P2 = -4.0 * A * a1;
        const double qq = Q * (Q + 1.0);
        const double L0 = log1p(1.0 / Q), L1 = -Q1 / qq, L2 = -Q2 / qq + Q1 * Q1 * (2.0 * Q + 1.0) / (qq * qq);
        const double e1 = P1 * L0 + P0 * L1;
        const double e2 = P2 * L0 + 2.0 * P1 * L1 + P0 * L2;
        out[i] = fx + x * (x * e2 - 5.0 * e1) / (36.0 * n);
    }
}

size_t density_smem(size_t es) { return es * (16 * 64 + 16 * 65 + 64 * 65 + 512); }
size_t integrals_smem(size_t es) { return es * (16 * 65 * 2 + 512); }

}  // namespace

bool fft_size_ok(int n) {
    Plan p;
    return n >= 8 && n <= 256 && make_plan(n, p);
}

template <typename T>
void response_density(cudaStream_t st, const GridShape &g, const TileSet<T> &chi,
                      const TileSet<T> &phi, int nphi, const T *P, long long sP, int k, T *rho) {
    if (k <= 0) return;
    ProfScope ps(st, ST_DENSITY, 2.0 * k * g.pair_points,
                 sizeof(T) * (g.table_values + (double)k * g.n * g.n * g.n));
    const size_t sm = density_smem(sizeof(T));
    static const bool attr = [&]() {   // once per process, thread-safe
        check(cudaFuncSetAttribute(density_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm),
              "cudaFuncSetAttribute(density)");
        return true;
    }();
    (void)attr;
    dim3 grid(chi.ntiles, k);
    density_kernel<T><<<grid, 256, sm, st>>>(g.n, g.nt, chi.off, chi.ids, chi.val, phi.off, phi.ids,
                                             phi.val, nphi, P, sP, rho);
    check_launch("density_kernel");
}

template <typename T>
void potential_integrals(cudaStream_t st, const GridShape &g, const TileSet<T> &chi,
                         const TileSet<T> &phi, int nchi, int nphi, const T *V, int k, T *out) {
    if (k <= 0) return;
    ProfScope ps(st, ST_INTEGRALS, 2.0 * k * g.pair_points,
                 sizeof(T) * (g.table_values + (double)k * g.n * g.n * g.n + (double)k * nchi * nphi));
    check(cudaMemsetAsync(out, 0, sizeof(T) * (size_t)k * nchi * nphi, st), "memset(integrals)");
    const size_t sm = integrals_smem(sizeof(T));
    dim3 grid(chi.ntiles, k);
    integrals_kernel<T><<<grid, 256, sm, st>>>(g.n, g.nt, chi.off, chi.ids, chi.val, phi.off, phi.ids,
                                               phi.val, nchi, nphi, V, T(g.dV), out);
    check_launch("integrals_kernel");
}

template <typename T>
void hartree_fxc(cudaStream_t st, const GridShape &g, const T *rho, const T *fxc, int k, T *V,
                 void *work) {
    if (k <= 0) return;
    using Vc = typename C2<T>::t;
    Plan pl;
    if (!make_plan(g.n, pl)) throw CudaError{cudaErrorInvalidValue, "FFT size not 2/3/5-smooth"};
    const int n = g.n, L = lines_per_cta<T>();
    const int pairs = (k + 1) / 2;
    const double n3d = (double)n * n * n;
    ProfScope ps(st, ST_FFT, pairs * 2.0 * 5.0 * n3d * std::log2(n3d), sizeof(T) * (2.0 * k + 1.0) * n3d);
    const size_t sm = (2 * (size_t)L * (n + 1) + n) * sizeof(Vc) + FFT_KK_BYTES;
    static const bool attr = [&]() {   // once per process, thread-safe
        const int mx = (2 * L * 257 + 256) * (int)sizeof(Vc) + FFT_KK_BYTES;
        check(cudaFuncSetAttribute(fft_z_forward_real<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx), "attr fz");
        check(cudaFuncSetAttribute(fft_z_inverse_real<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx), "attr iz");
        check(cudaFuncSetAttribute(fft_strided<T, 1, -1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx), "attr fy");
        check(cudaFuncSetAttribute(fft_strided<T, 1, +1, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx), "attr iy");
        check(cudaFuncSetAttribute(fft_strided<T, 0, -1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx), "attr x");
        return true;
    }();
    (void)attr;
    Vc *w = reinterpret_cast<Vc *>(work);
    const long long nlines = (long long)n * n;
    dim3 gz((unsigned)((nlines + L - 1) / L), pairs);
    dim3 gs((n + L - 1) / L, n, pairs);
    const T tpl = T(2.0 * 3.14159265358979323846 / g.cell);
    fft_z_forward_real<T><<<gz, 256, sm, st>>>(pl, rho, k, w);
    check_launch("fft_z_forward_real");
    fft_strided<T, 1, -1, false><<<gs, 256, sm, st>>>(pl, w, tpl);
    check_launch("fft_y_forward");
    fft_strided<T, 0, -1, true><<<gs, 256, sm, st>>>(pl, w, tpl);
    check_launch("fft_x_poisson");
    fft_strided<T, 1, +1, false><<<gs, 256, sm, st>>>(pl, w, tpl);
    check_launch("fft_y_inverse");
    fft_z_inverse_real<T><<<gz, 256, sm, st>>>(pl, w, rho, fxc, k, V);
    check_launch("fft_z_inverse_real");
}

void fxc_lda(cudaStream_t st, const double *n0, double *fxc, long long npts) {
    fxc_kernel<<<304, 256, 0, st>>>(n0, fxc, npts);
    check_launch("fxc_kernel");
}

template void response_density<float>(cudaStream_t, const GridShape &, const TileSet<float> &,
                                       const TileSet<float> &, int, const float *, long long, int,
                                       float *);
template void response_density<double>(cudaStream_t, const GridShape &, const TileSet<double> &,
                                        const TileSet<double> &, int, const double *, long long, int,
                                        double *);
template void potential_integrals<float>(cudaStream_t, const GridShape &, const TileSet<float> &,
                                         const TileSet<float> &, int, int, const float *, int,
                                         float *);
template void potential_integrals<double>(cudaStream_t, const GridShape &, const TileSet<double> &,
                                          const TileSet<double> &, int, int, const double *, int,
                                          double *);
template void hartree_fxc<float>(cudaStream_t, const GridShape &, const float *, const float *, int,
                                 float *, void *);
template void hartree_fxc<double>(cudaStream_t, const GridShape &, const double *, const double *,
                                  int, double *, void *);

}  // namespace tddft
