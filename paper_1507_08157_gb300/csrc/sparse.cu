// Cluster-blocked sparse layout of the truncated (linear-scaling) form, Sec. IV of the paper:
// clusters, patterns and pair lists built on the host; block-sparse products on the CUDA cores
// (float64, and float32 where the tensor cores are off); conversions between the boundary's
// atom-blocked order, the cluster blocks and dense matrices (for the grid kernels).
#include "sparse.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <stdexcept>
#include <string>

namespace tddft {

int BlockPattern::find(int a, int b) const {
    const auto beg = col.begin() + row_ptr[a], end = col.begin() + row_ptr[a + 1];
    const auto it = std::lower_bound(beg, end, b);
    return (it != end && *it == b) ? (int)(it - col.begin()) : -1;
}

namespace {

int grid_for(long long n) {
    const long long b = (n + 255) / 256;
    return (int)std::max(1LL, std::min(b, 8LL * 152));
}

// ---- kernels -----------------------------------------------------------------------------------

// one 256-thread block per (64 x 64 sub-tile of an output block, listed output block, batch entry):
// 16-deep K slices of the A and B blocks of each pair staged in shared memory; thread (tx, ty)
// owns rows ty + 16u and columns tx + 16v of the sub-tile
template <typename T>
__global__ void __launch_bounds__(256) bsr_simt_kernel(int BR, int BK, int BC, const int *__restrict__ out,
                                                      const int *__restrict__ ptr, const int *__restrict__ pa,
                                                      const int *__restrict__ pb, const T *__restrict__ A,
                                                      long long sA, const T *__restrict__ B, long long sB,
                                                      T *__restrict__ C, long long sC, T alpha, T beta,
                                                      const T *__restrict__ mask) {
    __shared__ T As[16][65];
    __shared__ T Bs[16][65];
    const int nsub_c = BC / 64;
    const int m0 = (blockIdx.x / nsub_c) * 64, n0 = (blockIdx.x % nsub_c) * 64;
    const int oi = blockIdx.y, o = out[oi];
    const long long b = blockIdx.z;
    A += b * sA;
    B += b * sB;
    C += b * sC;
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    T acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
    for (int j = ptr[oi]; j < ptr[oi + 1]; ++j) {
        const T *Ab = A + (long long)pa[j] * BR * BK + (long long)m0 * BK;
        const T *Bb = B + (long long)pb[j] * BK * BC + n0;
        for (int k0 = 0; k0 < BK; k0 += 16) {
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int kk = t & 15, m = (t >> 4) + 16 * i;
                As[kk][m] = Ab[(long long)m * BK + k0 + kk];
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int n = t & 63, kk = (t >> 6) + 4 * i;
                Bs[kk][n] = Bb[(long long)(k0 + kk) * BC + n];
            }
            __syncthreads();
#pragma unroll
            for (int kk = 0; kk < 16; ++kk) {
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
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int r = m0 + ty + 16 * u;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int c = n0 + tx + 16 * v;
            const long long idx = (long long)o * BR * BC + (long long)r * BC + c;
            T val = alpha * acc[u][v];
            if (beta != T(0)) val = fma(beta, C[idx], val);
            if (mask) val *= mask[idx];
            C[idx] = val;
        }
    }
}

// output blocks without any pair: C = mask (beta C)
template <typename T>
__global__ void bsr_empty_kernel(int bsize, const int *__restrict__ empty, T *__restrict__ C, long long sC, T beta,
                                 const T *__restrict__ mask) {
    const int o = empty[blockIdx.x];
    T *Cb = C + (long long)blockIdx.y * sC + (long long)o * bsize;
    const T *mb = mask ? mask + (long long)o * bsize : nullptr;
    for (int i = threadIdx.x; i < bsize; i += blockDim.x) {
        T v = beta == T(0) ? T(0) : beta * Cb[i];
        if (mb) v *= mb[i];
        Cb[i] = v;
    }
}

// out[blk] = in[blk]^T, blocks R x Cc row-major in, Cc x R out; one CTA per block, 32 x 32 tiles
template <typename T>
__global__ void bsr_transpose_kernel(const T *__restrict__ in, T *__restrict__ out, int R, int Cc) {
    __shared__ T tile[32][33];
    const long long blk = blockIdx.x;
    const T *src = in + blk * R * Cc;
    T *dst = out + blk * R * Cc;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
    for (int r0 = 0; r0 < R; r0 += 32)
        for (int c0 = 0; c0 < Cc; c0 += 32) {
            for (int i = ty; i < 32; i += 8) tile[i][tx] = src[(long long)(r0 + i) * Cc + c0 + tx];
            __syncthreads();
            for (int i = ty; i < 32; i += 8) dst[(long long)(c0 + i) * R + r0 + tx] = tile[tx][i];
            __syncthreads();
        }
}

struct LayoutView {   // the device arrays a conversion kernel needs, by value
    const int *blk_row, *blk_col, *blk_of, *rowfun, *colfun, *chi_cl, *chi_row, *phi_cl, *phi_col;
    const int *chi_atom, *phi_atom, *chi_first, *phi_first, *phi_cnt;
    const long long *abi_off;
    int natoms, ncl, nc, nv;
    long long len, nnz;
};

LayoutView view(const SparseLayout &L) {
    return LayoutView{L.blk_row, L.blk_col, L.blk_of, L.rowfun, L.colfun, L.chi_cl, L.chi_row, L.phi_cl, L.phi_col,
                      L.chi_atom, L.phi_atom, L.chi_first, L.phi_first, L.phi_cnt, L.abi_off, L.natoms, L.ncl,
                      L.nc, L.nv, L.len(), L.nnz_abi};
}

// the boundary index of cluster-block entry q, or -1 (padding, or an atom pair off the pattern)
__device__ __forceinline__ long long abi_index(const LayoutView &v, long long q) {
    const long long blk = q / CB_SIZE;
    const int w = (int)(q - blk * CB_SIZE), r = w / CB_C, c = w - r * CB_C;
    const int f = v.rowfun[v.blk_row[blk] * CB_R + r], g = v.colfun[v.blk_col[blk] * CB_C + c];
    if (f < 0 || g < 0) return -1;
    const int I = v.chi_atom[f], J = v.phi_atom[g];
    const long long off = v.abi_off[(long long)I * v.natoms + J];
    if (off < 0) return -1;
    return off + (long long)(f - v.chi_first[I]) * v.phi_cnt[J] + (g - v.phi_first[J]);
}

template <typename T>
__global__ void cb_from_abi_kernel(LayoutView v, const double *__restrict__ src, T *__restrict__ dst, int k) {
    const long long tot = v.len * k;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const long long b = e / v.len, q = e - b * v.len;
        const long long i = abi_index(v, q);
        dst[e] = i >= 0 ? T(src[b * v.nnz + i]) : T(0);
    }
}

template <typename T>
__global__ void cb_to_abi_kernel(LayoutView v, const T *__restrict__ src, double *__restrict__ dst, int k) {
    const long long tot = v.len * k;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const long long b = e / v.len, q = e - b * v.len;
        const long long i = abi_index(v, q);
        if (i >= 0) dst[b * v.nnz + i] = (double)src[e];
    }
}

template <typename T>
__global__ void cb_mask_kernel(LayoutView v, T *__restrict__ mask) {
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < v.len; q += (long long)gridDim.x * blockDim.x)
        mask[q] = abi_index(v, q) >= 0 ? T(1) : T(0);
}

template <typename T>
__global__ void cb_to_dense_kernel(LayoutView v, const T *__restrict__ src, T *__restrict__ dst, int k) {
    const long long per = (long long)v.nc * v.nv, tot = per * k;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const long long b = e / per, w = e - b * per;
        const int f = (int)(w / v.nv), g = (int)(w - (long long)f * v.nv);
        const int blk = v.blk_of[v.chi_cl[f] * v.ncl + v.phi_cl[g]];
        dst[e] = blk >= 0 ? src[b * v.len + (long long)blk * CB_SIZE + v.chi_row[f] * CB_C + v.phi_col[g]] : T(0);
    }
}

template <typename T>
__global__ void cb_from_dense_kernel(LayoutView v, const T *__restrict__ src, T *__restrict__ dst,
                                     const T *__restrict__ mask, int k) {
    const long long tot = v.len * k;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const long long b = e / v.len, q = e - b * v.len;
        const long long blk = q / CB_SIZE;
        const int w = (int)(q - blk * CB_SIZE), r = w / CB_C, c = w - r * CB_C;
        const int f = v.rowfun[v.blk_row[blk] * CB_R + r], g = v.colfun[v.blk_col[blk] * CB_C + c];
        dst[e] = (f >= 0 && g >= 0) ? mask[q] * src[b * (long long)v.nc * v.nv + (long long)f * v.nv + g] : T(0);
    }
}

// ---- host set-up -------------------------------------------------------------------------------

struct Invalid : std::invalid_argument {
    using std::invalid_argument::invalid_argument;
};

double min_image(const double *a, const double *b, double cell) {
    double d2 = 0.0;
    for (int x = 0; x < 3; ++x) {
        double d = a[x] - b[x];
        d -= cell * std::nearbyint(d / cell);
        d2 += d * d;
    }
    return std::sqrt(d2);
}

// functions of a set grouped by atom: first index and count per atom
void atom_ranges(const tddft_funcs &fs, int natoms, const char *name, std::vector<int> &first, std::vector<int> &cnt) {
    first.assign(natoms, 0);
    cnt.assign(natoms, 0);
    for (int f = 0; f < fs.nfun; ++f) {
        const int a = fs.atom[f];
        if (a < 0 || a >= natoms) throw Invalid(std::string(name) + ": atom index out of range");
        if (f > 0 && a < fs.atom[f - 1]) throw Invalid(std::string(name) + ": functions must be grouped by atom");
        if (cnt[a] == 0) first[a] = f;
        cnt[a]++;
    }
}

unsigned long long morton(const double *p, double cell) {
    unsigned q[3];
    for (int x = 0; x < 3; ++x) {
        double u = p[x] / cell;
        u -= std::floor(u);
        q[x] = (unsigned)std::min(1023.0, std::floor(u * 1024.0));
    }
    unsigned long long code = 0;
    for (int b = 0; b < 10; ++b)
        for (int x = 0; x < 3; ++x) code |= (unsigned long long)((q[x] >> b) & 1u) << (3 * b + x);
    return code;
}

// pattern from a set of marked (row block, column block) pairs
BlockPattern pattern_from(int nr, int nc, const std::vector<std::vector<int>> &rows) {
    BlockPattern p;
    p.nr = nr;
    p.nc = nc;
    p.row_ptr.assign(nr + 1, 0);
    for (int a = 0; a < nr; ++a) {
        std::vector<int> r = rows[a];
        std::sort(r.begin(), r.end());
        r.erase(std::unique(r.begin(), r.end()), r.end());
        p.col.insert(p.col.end(), r.begin(), r.end());
        p.row_ptr[a + 1] = (int)p.col.size();
    }
    return p;
}

// the natural pattern of A B (a block is present when some pair of present blocks meets)
BlockPattern product_pattern(const BlockPattern &A, const BlockPattern &B) {
    std::vector<std::vector<int>> rows(A.nr);
    std::vector<int> mark(B.nc, -1);
    for (int a = 0; a < A.nr; ++a) {
        for (int i = A.row_ptr[a]; i < A.row_ptr[a + 1]; ++i) {
            const int kk = A.col[i];
            for (int j = B.row_ptr[kk]; j < B.row_ptr[kk + 1]; ++j)
                if (mark[B.col[j]] != a) {
                    mark[B.col[j]] = a;
                    rows[a].push_back(B.col[j]);
                }
        }
    }
    return pattern_from(A.nr, B.nc, rows);
}

PairList pair_list(Mem &mem, const BlockPattern &A, const BlockPattern &B, const BlockPattern &C, int BR, int BK,
                   int BC) {
    std::vector<int> out, ptr{0}, pa, pb, empty;
    for (int a = 0; a < C.nr; ++a)
        for (int o = C.row_ptr[a]; o < C.row_ptr[a + 1]; ++o) {
            const int b = C.col[o];
            const size_t before = pa.size();
            for (int i = A.row_ptr[a]; i < A.row_ptr[a + 1]; ++i) {
                const int j = B.find(A.col[i], b);
                if (j >= 0) {
                    pa.push_back(i);
                    pb.push_back(j);
                }
            }
            if (pa.size() > before) {
                out.push_back(o);
                ptr.push_back((int)pa.size());
            } else {
                empty.push_back(o);
            }
        }
    PairList pl;
    pl.nout = (int)out.size();
    pl.npairs = (int)pa.size();
    pl.nempty = (int)empty.size();
    pl.nnz_flops = 2LL * BR * BK * BC * (long long)pa.size();
    auto up = [&](const std::vector<int> &v) {
        int *d = mem.alloc<int>(std::max<size_t>(1, v.size()));
        if (!v.empty()) check(cudaMemcpy(d, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice), "upload pairs");
        return d;
    };
    pl.out = up(out);
    pl.ptr = up(ptr);
    pl.pa = up(pa);
    pl.pb = up(pb);
    pl.empty = up(empty);
    return pl;
}

struct SideMap {   // one function set's place in the cluster blocks
    std::vector<int> first, cnt;    // per atom
    std::vector<int> cl, row;       // per function: cluster, row (or column) inside its block
    int B;                          // block edge
};

// an atom-blocked input matrix as cluster blocks (float64, host), with the atom blocks beyond
// `cutoff` dropped when cutoff > 0
void cluster_blocks(const tddft_bsr &m, const SideMap &rs, const SideMap &cs, int natoms, int ncl,
                    const std::vector<int> &acl, const double *pos, double cell, double cutoff, const char *name,
                    BlockPattern &pat, std::vector<double> &val) {
    if (!m.row_ptr || !m.col_idx || !m.blk_off || !m.val) throw Invalid(std::string(name) + ": null array");
    if (m.row_ptr[0] != 0 || m.blk_off[0] != 0) throw Invalid(std::string(name) + ": row_ptr[0] and blk_off[0] must be 0");
    std::vector<std::vector<int>> rows(ncl);
    for (int I = 0; I < natoms; ++I) {
        if (m.row_ptr[I + 1] < m.row_ptr[I]) throw Invalid(std::string(name) + ": row_ptr not monotone");
        for (long long b = m.row_ptr[I]; b < m.row_ptr[I + 1]; ++b) {
            const int J = m.col_idx[b];
            if (J < 0 || J >= natoms || (b > m.row_ptr[I] && J <= m.col_idx[b - 1]))
                throw Invalid(std::string(name) + ": block columns out of range or not ascending");
            if (m.blk_off[b + 1] - m.blk_off[b] != (long long)rs.cnt[I] * cs.cnt[J])
                throw Invalid(std::string(name) + ": block size does not match the function counts");
            if (cutoff > 0.0 && min_image(pos + 3 * I, pos + 3 * J, cell) > cutoff) continue;
            rows[acl[I]].push_back(acl[J]);
        }
    }
    pat = pattern_from(ncl, ncl, rows);
    const long long bs = (long long)rs.B * cs.B;
    val.assign((size_t)pat.nnzb() * bs, 0.0);
    for (int I = 0; I < natoms; ++I)
        for (long long b = m.row_ptr[I]; b < m.row_ptr[I + 1]; ++b) {
            const int J = m.col_idx[b];
            if (cutoff > 0.0 && min_image(pos + 3 * I, pos + 3 * J, cell) > cutoff) continue;
            const int blk = pat.find(acl[I], acl[J]);
            const double *v = m.val + m.blk_off[b];
            for (int i = 0; i < rs.cnt[I]; ++i) {
                const int r = rs.row[rs.first[I] + i];
                for (int j = 0; j < cs.cnt[J]; ++j)
                    val[(size_t)blk * bs + (size_t)r * cs.B + cs.row[cs.first[J] + j]] = v[(long long)i * cs.cnt[J] + j];
            }
        }
}

// ---- atom-level patterns as bitsets (the algorithmic work of the block products) ----------------
struct Bits {
    int n = 0, W = 0;
    std::vector<unsigned long long> b;
    explicit Bits(int n_ = 0) : n(n_), W((n_ + 63) / 64), b((size_t)n_ * ((n_ + 63) / 64), 0ull) {}
    void set(int i, int j) { b[(size_t)i * W + (j >> 6)] |= 1ull << (j & 63); }
    bool get(int i, int j) const { return (b[(size_t)i * W + (j >> 6)] >> (j & 63)) & 1ull; }
    const unsigned long long *row(int i) const { return b.data() + (size_t)i * W; }
    unsigned long long *row(int i) { return b.data() + (size_t)i * W; }
};

// pattern of A B: row i is the union of the rows k of B over the k set in row i of A
Bits bool_product(const Bits &A, const Bits &B) {
    Bits C(A.n);
#pragma omp parallel for schedule(dynamic, 16)
    for (int i = 0; i < A.n; ++i) {
        unsigned long long *c = C.row(i);
        const unsigned long long *a = A.row(i);
        for (int w = 0; w < A.W; ++w)
            for (unsigned long long x = a[w]; x; x &= x - 1) {
                const int k = w * 64 + __builtin_ctzll(x);
                const unsigned long long *r = B.row(k);
                for (int q = 0; q < B.W; ++q) c[q] |= r[q];
            }
    }
    return C;
}

Bits transpose_bits(const Bits &A) {
    Bits T(A.n);
    for (int i = 0; i < A.n; ++i)
        for (int j = 0; j < A.n; ++j)
            if (A.get(i, j)) T.set(j, i);
    return T;
}

// 2 sum over (I, J) set in C of nI nJ sum over K in (row I of A) and (column J of B) of nK, with
// cols = the transpose of B's pattern and nK grouped by distinct counts
double triple_flops(const Bits &A, const Bits &colsB, const Bits &C, const std::vector<int> &nI,
                    const std::vector<int> &nK, const std::vector<int> &nJ) {
    std::vector<int> vals(nK.begin(), nK.end());
    std::sort(vals.begin(), vals.end());
    vals.erase(std::unique(vals.begin(), vals.end()), vals.end());
    std::vector<Bits> byc;
    for (int v : vals) {
        Bits m(A.n);
        for (int k = 0; k < A.n; ++k)
            if (nK[k] == v) m.b[k >> 6] |= 1ull << (k & 63);   // one row holds the mask
        byc.push_back(std::move(m));
    }
    double tot = 0.0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : tot)
    for (int I = 0; I < C.n; ++I) {
        const unsigned long long *a = A.row(I), *c = C.row(I);
        for (int w = 0; w < C.W; ++w)
            for (unsigned long long x = c[w]; x; x &= x - 1) {
                const int J = w * 64 + __builtin_ctzll(x);
                const unsigned long long *col = colsB.row(J);
                double sk = 0.0;
                for (size_t v = 0; v < vals.size(); ++v) {
                    const unsigned long long *m = byc[v].row(0);
                    long long cnt = 0;
                    for (int q = 0; q < A.W; ++q) cnt += __builtin_popcountll(a[q] & col[q] & m[q]);
                    sk += (double)cnt * vals[v];
                }
                tot += 2.0 * nI[I] * nJ[J] * sk;
            }
    }
    return tot;
}

// the atom-level pattern of an input matrix (blocks present, within `cutoff` when > 0)
Bits input_bits(const tddft_bsr &m, int natoms, const double *pos, double cell, double cutoff) {
    Bits B(natoms);
    for (int I = 0; I < natoms; ++I)
        for (long long b = m.row_ptr[I]; b < m.row_ptr[I + 1]; ++b) {
            const int J = m.col_idx[b];
            if (cutoff > 0.0 && min_image(pos + 3 * I, pos + 3 * J, cell) > cutoff) continue;
            B.set(I, J);
        }
    return B;
}

}  // namespace

// ---- products ----------------------------------------------------------------------------------
template <typename T>
void bsr_simt(cudaStream_t st, int BR, int BK, int BC, const PairList &pl, int nblk_out, const T *A, long long sA,
              const T *B, long long sB, T *C, long long sC, int nb, T alpha, T beta, const T *mask) {
    (void)nblk_out;
    if (nb <= 0) return;
    if (BR % 64 || BC % 64 || BK % 16) throw CudaError{cudaErrorInvalidValue, "bsr_simt: block sizes"};
    for (int b0 = 0; b0 < nb; b0 += 65535) {
        const int nbb = std::min(65535, nb - b0);
        if (pl.nout > 0) {
            for (int o0 = 0; o0 < pl.nout; o0 += 65535) {
                const int no = std::min(65535, pl.nout - o0);
                dim3 grid((BR / 64) * (BC / 64), no, nbb);
                bsr_simt_kernel<T><<<grid, 256, 0, st>>>(BR, BK, BC, pl.out + o0, pl.ptr + o0, pl.pa, pl.pb,
                                                         A + b0 * sA, sA, B + b0 * sB, sB, C + b0 * sC, sC, alpha,
                                                         beta, mask);
                check_launch("bsr_simt_kernel");
            }
        }
        if (pl.nempty > 0) {
            for (int o0 = 0; o0 < pl.nempty; o0 += 65535) {
                dim3 grid(std::min(65535, pl.nempty - o0), nbb);
                bsr_empty_kernel<T><<<grid, 256, 0, st>>>(BR * BC, pl.empty + o0, C + b0 * sC, sC, beta, mask);
                check_launch("bsr_empty_kernel");
            }
        }
    }
}

template <typename T>
void bsr_transpose(cudaStream_t st, const T *in, T *out, int R, int Cc, long long nblk, int nb) {
    const long long tot = nblk * nb;
    for (long long b0 = 0; b0 < tot; b0 += (1LL << 30)) {
        const long long n = std::min(tot - b0, 1LL << 30);
        bsr_transpose_kernel<T><<<(unsigned)n, 256, 0, st>>>(in + b0 * R * Cc, out + b0 * R * Cc, R, Cc);
        check_launch("bsr_transpose_kernel");
    }
}

template <typename T>
void cb_from_abi(cudaStream_t st, const SparseLayout &L, const double *src, T *dst, int k) {
    cb_from_abi_kernel<T><<<grid_for(L.len() * k), 256, 0, st>>>(view(L), src, dst, k);
    check_launch("cb_from_abi_kernel");
}
template <typename T>
void cb_to_abi(cudaStream_t st, const SparseLayout &L, const T *src, double *dst, int k) {
    cb_to_abi_kernel<T><<<grid_for(L.len() * k), 256, 0, st>>>(view(L), src, dst, k);
    check_launch("cb_to_abi_kernel");
}
template <typename T>
void cb_to_dense(cudaStream_t st, const SparseLayout &L, const T *src, T *dst, int k) {
    cb_to_dense_kernel<T><<<grid_for((long long)L.nc * L.nv * k), 256, 0, st>>>(view(L), src, dst, k);
    check_launch("cb_to_dense_kernel");
}
template <typename T>
void cb_from_dense(cudaStream_t st, const SparseLayout &L, const T *src, T *dst, const T *mask, int k) {
    cb_from_dense_kernel<T><<<grid_for(L.len() * k), 256, 0, st>>>(view(L), src, dst, mask, k);
    check_launch("cb_from_dense_kernel");
}
template <typename T>
void cb_mask(cudaStream_t st, const SparseLayout &L, T *mask) {
    cb_mask_kernel<T><<<grid_for(L.len()), 256, 0, st>>>(view(L), mask);
    check_launch("cb_mask_kernel");
}

#define INST(T)                                                                                                  \
    template void bsr_simt<T>(cudaStream_t, int, int, int, const PairList &, int, const T *, long long, const T *, \
                              long long, T *, long long, int, T, T, const T *);                                 \
    template void bsr_transpose<T>(cudaStream_t, const T *, T *, int, int, long long, int);                      \
    template void cb_from_abi<T>(cudaStream_t, const SparseLayout &, const double *, T *, int);                  \
    template void cb_to_abi<T>(cudaStream_t, const SparseLayout &, const T *, double *, int);                    \
    template void cb_to_dense<T>(cudaStream_t, const SparseLayout &, const T *, T *, int);                       \
    template void cb_from_dense<T>(cudaStream_t, const SparseLayout &, const T *, T *, const T *, int);          \
    template void cb_mask<T>(cudaStream_t, const SparseLayout &, T *);
INST(float)
INST(double)
#undef INST

// ---- the layout of a system ----------------------------------------------------------------------
std::unique_ptr<SparseLayout> sparse_build(cudaStream_t st, const tddft_sparse_system *s) {
    auto L = std::make_unique<SparseLayout>();
    const int na = s->natoms;
    L->natoms = na;
    L->nc = s->chi.nfun;
    L->nv = s->phi.nfun;
    L->cell = s->cell;
    L->r_cut = s->kernel_cutoff;
    L->r_k = s->density_kernel_cutoff;
    if (!(s->kernel_cutoff > 0.0)) throw Invalid("the truncated form needs kernel_cutoff > 0");
    SideMap chi, phi;
    chi.B = CB_R;
    phi.B = CB_C;
    atom_ranges(s->chi, na, "chi", chi.first, chi.cnt);
    atom_ranges(s->phi, na, "phi", phi.first, phi.cnt);
    for (int a = 0; a < na; ++a)
        if (chi.cnt[a] > CB_R || phi.cnt[a] > CB_C)
            throw Invalid("more than 128 chi or 64 phi functions on one atom");
    // clusters: atoms in Morton order, cut greedily at 128 chi / 64 phi functions
    std::vector<int> order(na);
    std::iota(order.begin(), order.end(), 0);
    std::vector<unsigned long long> code(na);
    for (int a = 0; a < na; ++a) code[a] = morton(s->pos + 3 * a, s->cell);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return code[a] < code[b]; });
    std::vector<int> acl(na);
    std::vector<std::vector<int>> members;
    int nch = 0, nph = 0;
    for (int a : order) {
        if (members.empty() || nch + chi.cnt[a] > CB_R || nph + phi.cnt[a] > CB_C) {
            members.emplace_back();
            nch = nph = 0;
        }
        members.back().push_back(a);
        acl[a] = (int)members.size() - 1;
        nch += chi.cnt[a];
        nph += phi.cnt[a];
    }
    const int ncl = (int)members.size();
    L->ncl = ncl;
    chi.cl.assign(L->nc, 0);
    chi.row.assign(L->nc, 0);
    phi.cl.assign(L->nv, 0);
    phi.row.assign(L->nv, 0);
    std::vector<int> rowfun((size_t)ncl * CB_R, -1), colfun((size_t)ncl * CB_C, -1);
    for (int c = 0; c < ncl; ++c) {
        int r = 0, q = 0;
        for (int a : members[c]) {
            for (int i = 0; i < chi.cnt[a]; ++i, ++r) {
                const int f = chi.first[a] + i;
                chi.cl[f] = c;
                chi.row[f] = r;
                rowfun[(size_t)c * CB_R + r] = f;
            }
            for (int i = 0; i < phi.cnt[a]; ++i, ++q) {
                const int g = phi.first[a] + i;
                phi.cl[g] = c;
                phi.row[g] = q;
                colfun[(size_t)c * CB_C + q] = g;
            }
        }
    }
    // kernel pattern: atom pairs within the cutoff, and its cluster blocks
    L->amask.assign((size_t)na * na, 0);
    std::vector<std::vector<int>> krows(ncl);
    for (int I = 0; I < na; ++I)
        for (int J = 0; J < na; ++J)
            if (min_image(s->pos + 3 * I, s->pos + 3 * J, s->cell) <= s->kernel_cutoff) {
                L->amask[(size_t)I * na + J] = 1;
                if (chi.cnt[I] && phi.cnt[J]) krows[acl[I]].push_back(acl[J]);
            }
    L->pk = pattern_from(ncl, ncl, krows);
    // the boundary's atom-blocked order of the kernel pattern
    L->abi_row_ptr.assign(na + 1, 0);
    L->abi_blk_off.assign(1, 0);
    std::vector<long long> abi_off((size_t)na * na, -1);
    for (int I = 0; I < na; ++I) {
        for (int J = 0; J < na; ++J)
            if (L->amask[(size_t)I * na + J] && chi.cnt[I] && phi.cnt[J]) {
                abi_off[(size_t)I * na + J] = L->abi_blk_off.back();
                L->abi_col.push_back(J);
                L->abi_blk_off.push_back(L->abi_blk_off.back() + (long long)chi.cnt[I] * phi.cnt[J]);
            }
        L->abi_row_ptr[I + 1] = (long long)L->abi_col.size();
    }
    L->nnz_abi = L->abi_blk_off.back();
    // device index arrays
    Mem &m = L->mem;
    auto upi = [&](const std::vector<int> &v) {
        int *d = m.alloc<int>(std::max<size_t>(1, v.size()));
        if (!v.empty()) check(cudaMemcpy(d, v.data(), v.size() * sizeof(int), cudaMemcpyHostToDevice), "upload index");
        return d;
    };
    {
        std::vector<int> br, bc, bof((size_t)ncl * ncl, -1);
        for (int a = 0; a < ncl; ++a)
            for (int i = L->pk.row_ptr[a]; i < L->pk.row_ptr[a + 1]; ++i) {
                br.push_back(a);
                bc.push_back(L->pk.col[i]);
                bof[(size_t)a * ncl + L->pk.col[i]] = i;
            }
        L->blk_row = upi(br);
        L->blk_col = upi(bc);
        L->blk_of = upi(bof);
    }
    L->rowfun = upi(rowfun);
    L->colfun = upi(colfun);
    L->chi_cl = upi(chi.cl);
    L->chi_row = upi(chi.row);
    L->phi_cl = upi(phi.cl);
    L->phi_col = upi(phi.row);
    L->chi_atom = upi(std::vector<int>(s->chi.atom, s->chi.atom + L->nc));
    L->phi_atom = upi(std::vector<int>(s->phi.atom, s->phi.atom + L->nv));
    L->chi_first = upi(chi.first);
    L->phi_first = upi(phi.first);
    L->phi_cnt = upi(phi.cnt);
    L->abi_off = m.alloc<long long>(abi_off.size());
    check(cudaMemcpy(L->abi_off, abi_off.data(), abi_off.size() * sizeof(long long), cudaMemcpyHostToDevice),
          "upload abi offsets");
    L->pos = m.alloc<double>((size_t)3 * na);
    check(cudaMemcpy(L->pos, s->pos, (size_t)3 * na * sizeof(double), cudaMemcpyHostToDevice), "upload positions");
    // ground-state matrices as cluster blocks (P^c, P^v truncated at the density-kernel cutoff)
    BlockPattern pS, pH, pP, qS, qH, qP;
    std::vector<double> v;
    Mem tmp;
    auto up = [&](Mem &mm, const std::vector<double> &h) {
        double *d = mm.alloc<double>(std::max<size_t>(1, h.size()));
        if (!h.empty()) check(cudaMemcpy(d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice), "upload blocks");
        return d;
    };
    cluster_blocks(s->S_chi, chi, chi, na, ncl, acl, s->pos, s->cell, 0.0, "S_chi", pS, v);
    double *Sc = up(m, v);
    cluster_blocks(s->H_chi, chi, chi, na, ncl, acl, s->pos, s->cell, 0.0, "H_chi", pH, v);
    double *Hc = up(tmp, v);
    cluster_blocks(s->P_c, chi, chi, na, ncl, acl, s->pos, s->cell, s->density_kernel_cutoff, "P_c", pP, v);
    double *Pc = up(m, v);
    cluster_blocks(s->S_phi, phi, phi, na, ncl, acl, s->pos, s->cell, 0.0, "S_phi", qS, v);
    double *Sv = up(m, v);
    cluster_blocks(s->H_phi, phi, phi, na, ncl, acl, s->pos, s->cell, 0.0, "H_phi", qH, v);
    double *Hv = up(tmp, v);
    cluster_blocks(s->P_v, phi, phi, na, ncl, acl, s->pos, s->cell, s->density_kernel_cutoff, "P_v", qP, v);
    double *Pv = up(m, v);
    std::vector<double>().swap(v);
    // exact constant products in float64: natural patterns, no truncation
    auto product = [&](const BlockPattern &pa_, const double *A, const BlockPattern &pb_, const double *B, int Bk,
                       BlockPattern &pc_) {
        pc_ = product_pattern(pa_, pb_);
        Mem lists;
        PairList pl = pair_list(lists, pa_, pb_, pc_, Bk, Bk, Bk);
        double *C = m.alloc<double>(std::max<size_t>(1, (size_t)pc_.nnzb() * Bk * Bk));
        bsr_simt<double>(st, Bk, Bk, Bk, pl, pc_.nnzb(), A, 0, B, 0, C, 0, 1, 1.0, 0.0, nullptr);
        check(cudaStreamSynchronize(st), "sync constant product");
        return C;
    };
    L->pcc[SP_S] = pS;
    L->cc64[SP_S] = Sc;
    L->pcc[SP_P] = pP;
    L->cc64[SP_P] = Pc;
    L->cc64[SP_M] = product(pP, Pc, pH, Hc, CB_R, L->pcc[SP_M]);
    L->cc64[SP_R] = product(pP, Pc, pS, Sc, CB_R, L->pcc[SP_R]);
    L->cc64[SP_A] = product(pS, Sc, L->pcc[SP_R], L->cc64[SP_R], CB_R, L->pcc[SP_A]);
    L->cc64[SP_T] = product(pS, Sc, pP, Pc, CB_R, L->pcc[SP_T]);
    L->pvv[SP_S] = qS;
    L->vv64[SP_S] = Sv;
    L->pvv[SP_P] = qP;
    L->vv64[SP_P] = Pv;
    L->vv64[SP_M] = product(qH, Hv, qP, Pv, CB_C, L->pvv[SP_M]);
    L->vv64[SP_R] = product(qS, Sv, qP, Pv, CB_C, L->pvv[SP_R]);
    L->vv64[SP_A] = product(L->pvv[SP_R], L->vv64[SP_R], qS, Sv, CB_C, L->pvv[SP_A]);
    L->vv64[SP_T] = product(qP, Pv, qS, Sv, CB_C, L->pvv[SP_T]);
    // pair lists of the products into the kernel pattern
    for (int x = 0; x < SP_NCONST; ++x) {
        L->left[x] = pair_list(m, L->pcc[x], L->pk, L->pk, CB_R, CB_R, CB_C);
        L->right[x] = pair_list(m, L->pk, L->pvv[x], L->pk, CB_R, CB_C, CB_C);
    }
    // algorithmic work of each product: contributing atom-block triples, without the padding and
    // the atom pairs off the pattern inside present cluster blocks
    {
        Bits pk(na);
        for (int I = 0; I < na; ++I)
            for (int J = 0; J < na; ++J)
                if (L->amask[(size_t)I * na + J] && chi.cnt[I] && phi.cnt[J]) pk.set(I, J);
        const Bits pkT = transpose_bits(pk);
        const Bits Sc_b = input_bits(s->S_chi, na, s->pos, s->cell, 0.0), Hc_b = input_bits(s->H_chi, na, s->pos, s->cell, 0.0);
        const Bits Pc_b = input_bits(s->P_c, na, s->pos, s->cell, s->density_kernel_cutoff);
        const Bits Sv_b = input_bits(s->S_phi, na, s->pos, s->cell, 0.0), Hv_b = input_bits(s->H_phi, na, s->pos, s->cell, 0.0);
        const Bits Pv_b = input_bits(s->P_v, na, s->pos, s->cell, s->density_kernel_cutoff);
        Bits cc[SP_NCONST], vv[SP_NCONST];
        cc[SP_S] = Sc_b;
        cc[SP_P] = Pc_b;
        cc[SP_M] = bool_product(Pc_b, Hc_b);
        cc[SP_R] = bool_product(Pc_b, Sc_b);
        cc[SP_A] = bool_product(Sc_b, cc[SP_R]);
        cc[SP_T] = bool_product(Sc_b, Pc_b);
        vv[SP_S] = Sv_b;
        vv[SP_P] = Pv_b;
        vv[SP_M] = bool_product(Hv_b, Pv_b);
        vv[SP_R] = bool_product(Sv_b, Pv_b);
        vv[SP_A] = bool_product(vv[SP_R], Sv_b);
        vv[SP_T] = bool_product(Pv_b, Sv_b);
        for (int x = 0; x < SP_NCONST; ++x) {
            L->left[x].alg_flops = triple_flops(cc[x], pkT, pk, chi.cnt, chi.cnt, phi.cnt);
            L->right[x].alg_flops = triple_flops(pk, transpose_bits(vv[x]), pk, chi.cnt, phi.cnt, phi.cnt);
        }
    }
    check(cudaStreamSynchronize(st), "sync sparse build");
    return L;
}

}  // namespace tddft
