// Learned atom-block preconditioner: block features of the search gradient, the model that maps
// a block's fixed features to a linear map of the block (a 3-layer perceptron: forward,
// backpropagation, Adam), and the application z_IJ = h_IJ + A_IJ h_IJ inside the PCG. It stands
// in for the inner-CG solve of Eq. precond (paper Sec. III B) inside the PCG of Sec. III C; the
// iterative solve stays as fallback and as the source of training targets.
//
// Row layout (one row per state i, chi-atom I, phi-atom J; J fastest), n_c chi and n_v phi per
// atom, s = Frobenius norm of the (h^p_IJ, h^q_IJ) pair of blocks:
//   input  x = [b, f], b = [h^p_IJ / s, h^q_IJ / s] (n_b = 2 n_c n_v),
//                      f = [M^c_II, S^chi_II, M^v_JJ, S^phi_JJ, d_IJ / 10] (n_f = 2 n_c^2 + 2 n_v^2 + 1)
//   target y = [(z^p_IJ - h^p_IJ) / s, (z^q_IJ - h^q_IJ) / s]   (correction to the identity)
//   weight w = s^2 / (sum of s^2 over the rows of the same state)
// blocks row-major, M^c = P^c H^chi, M^v = H^phi P^v, d_IJ the minimum-image atom distance (bohr).
// Model: vec(A) = H2 W3 + b3 with H1 = relu(F W1 + b1), H2 = relu(H1 W2 + b2) (row form, A an
// n_b x n_b row-major matrix per row), output y = A b; parameters W1 [n_f][w], b1, W2 [w][w], b2,
// W3 [w][n_b^2], b3 in one float32 vector. The products run through the library GEMM (tensor
// cores, float32 accumulation); inference uses the parameters rounded to bfloat16.
#include "learned.h"
#include "solver_kernels.h"

#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

namespace tddft {

namespace {

int grid_of(long long n) {
    long long b = (n + 255) / 256;
    return (int)(b < 8 * 152 ? (b > 0 ? b : 1) : 8 * 152);
}

__global__ void bias_act_kernel(float *__restrict__ H, const float *__restrict__ b, long long n, int w, int relu) {
    const long long tot = n * w;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        const float v = H[i] + b[i % w];
        H[i] = relu ? fmaxf(v, 0.0f) : v;
    }
}

// dH *= (H > 0)
__global__ void relu_back_kernel(float *__restrict__ dH, const float *__restrict__ H, long long tot) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x)
        if (!(H[i] > 0.0f)) dH[i] = 0.0f;
}

// R = Y - T (kept for the loss), dY = scale * w_row * R (w = 1 without row weights)
__global__ void residual_kernel(const float *__restrict__ Y, const float *__restrict__ T,
                                const float *__restrict__ w, int cols, float *__restrict__ R,
                                float *__restrict__ dY, long long tot, float scale) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < tot; i += (long long)gridDim.x * blockDim.x) {
        const float r = Y[i] - T[i];
        R[i] = r;
        dY[i] = scale * (w ? w[i / cols] : 1.0f) * r;
    }
}

// row weights s^2 / (sum of s^2 over the rows of the same state); one block per state
__global__ void row_weights_kernel(const float *__restrict__ s, long long per, float *__restrict__ w) {
    __shared__ double red[256];
    const float *si = s + blockIdx.x * per;
    float *wi = w + blockIdx.x * per;
    double acc = 0.0;
    for (long long r = threadIdx.x; r < per; r += blockDim.x) acc += (double)si[r] * si[r];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
    }
    const double tot = red[0];
    for (long long r = threadIdx.x; r < per; r += blockDim.x)
        wi[r] = tot > 0.0 ? (float)((double)si[r] * si[r] / tot) : 0.0f;
}

// out[j] = sum_r D[r][j] (one thread per column, rows in order, float64 accumulation)
__global__ void colsum_kernel(const float *__restrict__ D, long long n, int w, float *__restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= w) return;
    double s = 0.0;
    for (long long r = 0; r < n; ++r) s += (double)D[r * w + j];
    out[j] = (float)s;
}

__global__ void adam_kernel(float *__restrict__ W, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, long long np, float lr, float bc1, float bc2) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < np; i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        W[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
    }
}

__global__ void round_bf16_kernel(const float *__restrict__ W, float *__restrict__ out, long long np) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < np; i += (long long)gridDim.x * blockDim.x)
        out[i] = __bfloat162float(__float2bfloat16_rn(W[i]));
}

__global__ void gather_rows_kernel(const float *__restrict__ X, const long long *__restrict__ idx, int rows,
                                   int cols, float *__restrict__ out) {
    const long long tot = (long long)rows * cols;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const long long r = e / cols;
        const int c = (int)(e - r * cols);
        out[e] = X[idx[r] * cols + c];
    }
}

// per-atom fixed features: out[I] = [A_II (nb x nb, row-major), S_II] of the n x n matrices
template <typename T>
__global__ void fixed_features_kernel(const T *__restrict__ A, const T *__restrict__ S, int n, int nb, int na,
                                      float *__restrict__ out) {
    const int per = 2 * nb * nb;
    const long long tot = (long long)na * per;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const int I = (int)(e / per), r = (int)(e - (long long)I * per);
        const int which = r / (nb * nb), q = r - which * nb * nb;
        const int a = I * nb + q / nb, b = I * nb + q % nb;
        const T *M = which ? S : A;
        out[e] = (float)M[(long long)a * n + b];
    }
}

// one warp per row (i, I, J): block norm, then the row of inputs
template <typename T>
__global__ void features_kernel(const T *__restrict__ h, int k, int na, int nca, int nva, int nc, int nv,
                                const float *__restrict__ fc, const float *__restrict__ fv,
                                const float *__restrict__ dist, int n_in, float *__restrict__ X,
                                float *__restrict__ s_out) {
    const int lane = threadIdx.x & 31;
    const long long row = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long rows = (long long)k * na * na;
    if (row >= rows) return;
    const int J = (int)(row % na), I = (int)((row / na) % na), i = (int)(row / ((long long)na * na));
    const long long len = (long long)nc * nv;
    const int blk = nca * nva;
    const T *hp = h + (long long)i * len, *hq = h + (long long)(k + i) * len;
    double ss = 0.0;
    for (int e = lane; e < 2 * blk; e += 32) {
        const int q = e < blk ? e : e - blk;
        const T *src = e < blk ? hp : hq;
        const double v = (double)src[(long long)(I * nca + q / nva) * nv + J * nva + q % nva];
        ss += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    const double sc = sqrt(ss);
    const double inv = sc > 0.0 ? 1.0 / sc : 0.0;
    float *x = X + row * n_in;
    const int nfc = 2 * nca * nca, nfv = 2 * nva * nva;
    for (int e = lane; e < n_in; e += 32) {
        float v;
        if (e < 2 * blk) {
            const int q = e < blk ? e : e - blk;
            const T *src = e < blk ? hp : hq;
            v = (float)((double)src[(long long)(I * nca + q / nva) * nv + J * nva + q % nva] * inv);
        } else if (e < 2 * blk + nfc) {
            v = fc[(long long)I * nfc + (e - 2 * blk)];
        } else if (e < 2 * blk + nfc + nfv) {
            v = fv[(long long)J * nfv + (e - 2 * blk - nfc)];
        } else {
            v = dist[(long long)I * na + J];
        }
        x[e] = v;
    }
    if (lane == 0) s_out[row] = (float)sc;
}

// target rows y = (z - h) / s; one warp per row
template <typename T>
__global__ void targets_kernel(float *__restrict__ Y, const float *__restrict__ s, const T *__restrict__ h,
                               const T *__restrict__ z, int k, int na, int nca, int nva, int nc, int nv) {
    const int lane = threadIdx.x & 31;
    const long long row = blockIdx.x * (long long)(blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long rows = (long long)k * na * na;
    if (row >= rows) return;
    const int J = (int)(row % na), I = (int)((row / na) % na), i = (int)(row / ((long long)na * na));
    const long long len = (long long)nc * nv;
    const int blk = nca * nva, nb = 2 * blk;
    const float sc = s[row];
    const float inv = sc > 0.0f ? 1.0f / sc : 0.0f;
    for (int e = lane; e < nb; e += 32) {
        const int q = e < blk ? e : e - blk;
        const long long at =
            (long long)(e < blk ? i : k + i) * len + (long long)(I * nca + q / nva) * nv + J * nva + q % nva;
        Y[row * nb + e] = (float)((double)z[at] - (double)h[at]) * inv;
    }
}

// feature rows f_IJ = [fc_I, fv_J, dist_IJ] for all (I, J)
__global__ void feature_rows_kernel(const float *__restrict__ fc, const float *__restrict__ fv,
                                    const float *__restrict__ dist, int na, int nfc, int nfv, float *__restrict__ F) {
    const int nf = nfc + nfv + 1;
    const long long tot = (long long)na * na * nf;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const long long r = e / nf;
        const int c = (int)(e - r * nf);
        const int I = (int)(r / na), J = (int)(r % na);
        F[e] = c < nfc ? fc[(long long)I * nfc + c] : (c < nfc + nfv ? fv[(long long)J * nfv + c - nfc] : dist[r]);
    }
}

// z_IJ = h_IJ + A_IJ h_IJ for every state and atom block (blocks as n_b-vectors, p then q);
// one warp per (state, block), the block staged in shared memory
template <typename T>
__global__ void block_apply_kernel(const float *__restrict__ A, const T *__restrict__ h, T *__restrict__ z, int k,
                                   int na, int nca, int nva, int nc, int nv) {
    extern __shared__ float xs_raw[];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const int blk = nca * nva, nb = 2 * blk;
    float *xs = xs_raw + wib * nb;
    const long long row = blockIdx.x * (long long)(blockDim.x >> 5) + wib;
    const long long rows = (long long)k * na * na;
    const bool live = row < rows;
    const int J = live ? (int)(row % na) : 0, I = live ? (int)((row / na) % na) : 0;
    const int i = live ? (int)(row / ((long long)na * na)) : 0;
    const long long len = (long long)nc * nv;
    auto at = [&](int e) {
        const int q = e < blk ? e : e - blk;
        return (long long)(e < blk ? i : k + i) * len + (long long)(I * nca + q / nva) * nv + J * nva + q % nva;
    };
    if (live)
        for (int e = lane; e < nb; e += 32) xs[e] = (float)h[at(e)];
    __syncwarp();
    if (!live) return;
    const float *Ab = A + ((long long)I * na + J) * nb * nb;
    for (int a = lane; a < nb; a += 32) {
        float acc = 0.0f;
        for (int c = 0; c < nb; ++c) acc = fmaf(Ab[a * nb + c], xs[c], acc);
        const long long o = at(a);
        z[o] = h[o] + (T)acc;
    }
}

// y_r = A_r b_r (A rows n_b x n_b, b the first n_b entries of the input rows, ld = row stride)
__global__ void head_kernel(const float *__restrict__ A, const float *__restrict__ X, int ld, int nb, long long n,
                            float *__restrict__ Y) {
    const long long tot = n * nb;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const long long r = e / nb;
        const int a = (int)(e - r * nb);
        const float *Ar = A + r * nb * nb + (long long)a * nb;
        const float *x = X + r * ld;
        float acc = 0.0f;
        for (int c = 0; c < nb; ++c) acc = fmaf(Ar[c], x[c], acc);
        Y[e] = acc;
    }
}

// dA_r = dy_r b_r^T
__global__ void head_back_kernel(const float *__restrict__ dY, const float *__restrict__ X, int ld, int nb, long long n,
                                 float *__restrict__ dA) {
    const long long tot = n * nb * nb;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const long long r = e / ((long long)nb * nb);
        const int q = (int)(e - r * nb * nb);
        dA[e] = dY[r * nb + q / nb] * X[r * ld + q % nb];
    }
}

}  // namespace

// ---- the model object ---------------------------------------------------------------------------
struct MlpBuffers {
    Mem mem;
    long long rows = 0;
    float *H1 = nullptr, *H2 = nullptr, *A = nullptr, *dA = nullptr, *Y = nullptr, *R = nullptr, *dY = nullptr,
          *dH = nullptr, *Xb = nullptr, *Tb = nullptr, *Wb = nullptr;
    long long *idx = nullptr;
    double *scr = nullptr, *loss = nullptr;
};

}  // namespace tddft

struct tddft_mlp {
    int nb = 0, nf = 0, w = 0;        // block entries, feature entries, hidden width
    int nout = 0;                     // perceptron outputs: nb * nb
    long long np = 0;
    long long t = 0;                  // Adam steps taken
    long long version = 0;            // bumped whenever the parameters change
    tddft::Mem mem;
    float *W = nullptr, *Winf = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;
    tddft::MlpBuffers buf;
    std::string err;
};

namespace tddft {

namespace {

struct Offs {
    long long W1, b1, W2, b2, W3, b3;
};
Offs offsets(const tddft_mlp *m) {
    Offs o;
    o.W1 = 0;
    o.b1 = o.W1 + (long long)m->nf * m->w;
    o.W2 = o.b1 + m->w;
    o.b2 = o.W2 + (long long)m->w * m->w;
    o.W3 = o.b2 + m->w;
    o.b3 = o.W3 + (long long)m->w * m->nout;
    return o;
}

constexpr long long CHUNK = 8192;     // rows per inference pass over a large input

void ensure_rows(tddft_mlp *m, long long rows) {
    MlpBuffers &B = m->buf;
    if (rows <= B.rows) return;
    check(cudaDeviceSynchronize(), "sync before model buffers");
    B.mem.release();
    const int ld = m->nb + m->nf;
    B.H1 = B.mem.alloc<float>((size_t)rows * m->w);
    B.H2 = B.mem.alloc<float>((size_t)rows * m->w);
    B.dH = B.mem.alloc<float>((size_t)rows * m->w);
    B.A = B.mem.alloc<float>((size_t)rows * m->nout);
    B.dA = B.mem.alloc<float>((size_t)rows * m->nout);
    B.Y = B.mem.alloc<float>((size_t)rows * m->nb);
    B.R = B.mem.alloc<float>((size_t)rows * m->nb);
    B.dY = B.mem.alloc<float>((size_t)rows * m->nb);
    B.Xb = B.mem.alloc<float>((size_t)rows * ld);
    B.Tb = B.mem.alloc<float>((size_t)rows * m->nb);
    B.Wb = B.mem.alloc<float>((size_t)rows);
    B.idx = B.mem.alloc<long long>((size_t)rows);
    B.scr = B.mem.alloc<double>((size_t)gram_scratch_doubles(64, 32));
    B.loss = B.mem.alloc<double>(4);
    B.rows = rows;
}

// vec(A) rows [n][nb^2] of the perceptron for feature rows F (row stride ldf); keeps H1, H2
void perceptron(cudaStream_t st, tddft_mlp *m, const float *W, long long n, const float *F, int ldf, float *A) {
    const Offs o = offsets(m);
    MlpBuffers &B = m->buf;
    const int nf = m->nf, w = m->w, nout = m->nout;
    gemm<float>(st, false, false, (int)n, w, nf, 1.0f, F, ldf, 0, W + o.W1, w, 0, 0.0f, B.H1, w, 0, 1);
    bias_act_kernel<<<grid_of(n * w), 256, 0, st>>>(B.H1, W + o.b1, n, w, 1);
    check_launch("bias_act");
    gemm<float>(st, false, false, (int)n, w, w, 1.0f, B.H1, w, 0, W + o.W2, w, 0, 0.0f, B.H2, w, 0, 1);
    bias_act_kernel<<<grid_of(n * w), 256, 0, st>>>(B.H2, W + o.b2, n, w, 1);
    check_launch("bias_act");
    gemm<float>(st, false, false, (int)n, nout, w, 1.0f, B.H2, w, 0, W + o.W3, nout, 0, 0.0f, A, nout, 0, 1);
    bias_act_kernel<<<grid_of(n * nout), 256, 0, st>>>(A, W + o.b3, n, nout, 0);
    check_launch("bias_act");
}

// 2 x loss (device double) and gradient g of the weighted mean-squared loss over n rows
// X = [b, f] (n x (nb + nf)), T (n x nb) and the optional row weights rw, all on the device
void loss_grad_rows(cudaStream_t st, tddft_mlp *m, long long n, const float *X, const float *T, const float *rw,
                    double *loss2) {
    const Offs o = offsets(m);
    MlpBuffers &B = m->buf;
    const int nb = m->nb, nf = m->nf, w = m->w, nout = m->nout, ld = nb + nf;
    perceptron(st, m, m->W, n, X + nb, ld, B.A);
    head_kernel<<<grid_of(n * nb), 256, 0, st>>>(B.A, X, ld, nb, n, B.Y);
    check_launch("head");
    const long long tot = n * nb;
    residual_kernel<<<grid_of(tot), 256, 0, st>>>(B.Y, T, rw, nb, B.R, B.dY, tot, 2.0f / (float)tot);
    check_launch("residual");
    // <R, dY> = 2 sum_r w_r |R_r|^2 / (n nb) = 2 L
    dots<float>(st, B.R, tot, B.dY, tot, 1, tot, loss2, B.scr);
    head_back_kernel<<<grid_of(n * nout), 256, 0, st>>>(B.dY, X, ld, nb, n, B.dA);
    check_launch("head_back");
    float *g = m->g;
    // layer 3
    gemm<float>(st, true, false, w, nout, (int)n, 1.0f, B.H2, w, 0, B.dA, nout, 0, 0.0f, g + o.W3, nout, 0, 1);
    colsum_kernel<<<(nout + 127) / 128, 128, 0, st>>>(B.dA, n, nout, g + o.b3);
    check_launch("colsum");
    gemm<float>(st, false, true, (int)n, w, nout, 1.0f, B.dA, nout, 0, m->W + o.W3, nout, 0, 0.0f, B.dH, w, 0, 1);
    relu_back_kernel<<<grid_of(n * w), 256, 0, st>>>(B.dH, B.H2, n * w);
    check_launch("relu_back");
    // layer 2 (dH holds dL/d(pre-activation 2))
    gemm<float>(st, true, false, w, w, (int)n, 1.0f, B.H1, w, 0, B.dH, w, 0, 0.0f, g + o.W2, w, 0, 1);
    colsum_kernel<<<(w + 127) / 128, 128, 0, st>>>(B.dH, n, w, g + o.b2);
    check_launch("colsum");
    gemm<float>(st, false, true, (int)n, w, w, 1.0f, B.dH, w, 0, m->W + o.W2, w, 0, 0.0f, B.H2, w, 0, 1);
    relu_back_kernel<<<grid_of(n * w), 256, 0, st>>>(B.H2, B.H1, n * w);
    check_launch("relu_back");
    // layer 1 (H2 now holds dL/d(pre-activation 1)); F = X + nb with row stride ld
    gemm<float>(st, true, false, nf, w, (int)n, 1.0f, X + nb, ld, 0, B.H2, w, 0, 0.0f, g + o.W1, w, 0, 1);
    colsum_kernel<<<(w + 127) / 128, 128, 0, st>>>(B.H2, n, w, g + o.b1);
    check_launch("colsum");
}

void adam(cudaStream_t st, tddft_mlp *m, float lr) {
    m->t += 1;
    const float bc1 = (float)(1.0 - std::pow(0.9, (double)m->t));
    const float bc2 = (float)(1.0 - std::pow(0.999, (double)m->t));
    adam_kernel<<<grid_of(m->np), 256, 0, st>>>(m->W, m->g, m->m, m->v, m->np, lr, bc1, bc2);
    check_launch("adam");
}

void refresh_inference(cudaStream_t st, tddft_mlp *m) {
    round_bf16_kernel<<<grid_of(m->np), 256, 0, st>>>(m->W, m->Winf, m->np);
    check_launch("round_bf16");
    m->version += 1;
}

}  // namespace

int mlp_n_block(const tddft_mlp *m) { return m->nb; }
int mlp_n_feat(const tddft_mlp *m) { return m->nf; }
long long mlp_version(const tddft_mlp *m) { return m->version; }

void mlp_block_maps(cudaStream_t st, tddft_mlp *m, long long n, const float *F, float *A) {
    ensure_rows(m, std::min(n, CHUNK));
    for (long long r0 = 0; r0 < n; r0 += CHUNK) {
        const long long r = std::min(CHUNK, n - r0);
        perceptron(st, m, m->Winf, r, F + r0 * m->nf, m->nf, A + r0 * m->nout);
    }
}

template <typename T>
void learned_fixed_features(cudaStream_t st, const T *A, const T *S, int n, int nb, int na, float *out) {
    fixed_features_kernel<T><<<grid_of((long long)na * 2 * nb * nb), 256, 0, st>>>(A, S, n, nb, na, out);
    check_launch("fixed_features");
}

void learned_feature_rows(cudaStream_t st, const float *fc, const float *fv, const float *dist, int na, int nca,
                          int nva, float *F) {
    const int nfc = 2 * nca * nca, nfv = 2 * nva * nva;
    feature_rows_kernel<<<grid_of((long long)na * na * (nfc + nfv + 1)), 256, 0, st>>>(fc, fv, dist, na, nfc, nfv, F);
    check_launch("feature_rows");
}

template <typename T>
void learned_features(cudaStream_t st, const T *h, int k, int na, int nca, int nva, int nc, int nv,
                      const float *fc, const float *fv, const float *dist, float *X, float *s) {
    const long long rows = (long long)k * na * na;
    const int n_in = 2 * nca * nva + 2 * nca * nca + 2 * nva * nva + 1;
    features_kernel<T><<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(h, k, na, nca, nva, nc, nv, fc, fv, dist, n_in, X, s);
    check_launch("features");
}

template <typename T>
void learned_apply(cudaStream_t st, const float *A, const T *h, int k, int na, int nca, int nva, int nc, int nv, T *z) {
    const long long rows = (long long)k * na * na;
    const int nb = 2 * nca * nva;
    ProfScope ps(st, ST_VECTOR, 2.0 * rows * nb * nb,
                 4.0 * (double)na * na * nb * nb + 3.0 * sizeof(T) * (double)rows * nb);
    block_apply_kernel<T><<<(unsigned)((rows + 7) / 8), 256, 8 * nb * sizeof(float), st>>>(A, h, z, k, na, nca, nva, nc,
                                                                                           nv);
    check_launch("block_apply");
}

template <typename T>
void learned_targets(cudaStream_t st, const T *z, const T *h, const float *s, int k, int na, int nca, int nva, int nc,
                     int nv, float *Y, float *w) {
    const long long rows = (long long)k * na * na;
    targets_kernel<T><<<(unsigned)((rows + 7) / 8), 256, 0, st>>>(Y, s, h, z, k, na, nca, nva, nc, nv);
    check_launch("targets");
    row_weights_kernel<<<k, 256, 0, st>>>(s, (long long)na * na, w);
    check_launch("row weights");
}

#define INST_L(T)                                                                                                \
    template void learned_fixed_features<T>(cudaStream_t, const T *, const T *, int, int, int, float *);          \
    template void learned_features<T>(cudaStream_t, const T *, int, int, int, int, int, int, const float *,      \
                                      const float *, const float *, float *, float *);                         \
    template void learned_apply<T>(cudaStream_t, const float *, const T *, int, int, int, int, int, int, T *);   \
    template void learned_targets<T>(cudaStream_t, const T *, const T *, const float *, int, int, int, int, int, \
                                     int, float *, float *);
INST_L(float)
INST_L(double)
#undef INST_L

}  // namespace tddft

// ---- C ABI: the model object -------------------------------------------------------------------
using namespace tddft;

namespace {

bool dev_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <typename F>
tddft_status mlp_guard(tddft_mlp *m, F &&f) {
    try {
        return f();
    } catch (const CudaError &e) {
        m->err = std::string(e.where) + ": " + cudaGetErrorString(e.code);
        cudaGetLastError();
        return e.code == cudaErrorMemoryAllocation ? TDDFT_E_NOMEM : TDDFT_E_CUDA;
    } catch (const std::bad_alloc &) {
        m->err = "out of memory";
        return TDDFT_E_NOMEM;
    }
}

}  // namespace

extern "C" {

tddft_status tddft_mlp_create(int32_t n_block, int32_t n_feat, int32_t width, tddft_mlp **out) {
    if (!out || n_block < 1 || n_feat < 1 || width < 1 || n_block > 128 || n_feat > 4096 || width > 4096)
        return TDDFT_E_INVALID;
    auto m = new (std::nothrow) tddft_mlp();
    if (!m) return TDDFT_E_NOMEM;
    m->nb = n_block;
    m->nf = n_feat;
    m->w = width;
    m->nout = n_block * n_block;
    m->np = (long long)n_feat * width + width + (long long)width * width + width + (long long)width * m->nout + m->nout;
    tddft_status rc = mlp_guard(m, [&]() -> tddft_status {
        m->W = m->mem.alloc<float>((size_t)m->np);
        m->Winf = m->mem.alloc<float>((size_t)m->np);
        m->m = m->mem.alloc<float>((size_t)m->np);
        m->v = m->mem.alloc<float>((size_t)m->np);
        m->g = m->mem.alloc<float>((size_t)m->np);
        for (float *p : {m->W, m->Winf, m->m, m->v, m->g})
            check(cudaMemset(p, 0, (size_t)m->np * sizeof(float)), "memset model");
        return TDDFT_OK;
    });
    if (rc != TDDFT_OK) {
        delete m;
        return rc;
    }
    *out = m;
    return TDDFT_OK;
}

void tddft_mlp_destroy(tddft_mlp *m) {
    if (!m) return;
    cudaDeviceSynchronize();
    delete m;
}

const char *tddft_mlp_last_error(const tddft_mlp *m) { return m ? m->err.c_str() : "null model"; }

int64_t tddft_mlp_size(const tddft_mlp *m) { return m ? m->np : 0; }

tddft_status tddft_mlp_set(tddft_mlp *m, const float *theta) {
    if (!m || !theta) return TDDFT_E_INVALID;
    return mlp_guard(m, [&]() -> tddft_status {
        check(cudaMemcpy(m->W, theta, (size_t)m->np * sizeof(float), cudaMemcpyDefault), "set parameters");
        check(cudaMemset(m->m, 0, (size_t)m->np * sizeof(float)), "reset adam m");
        check(cudaMemset(m->v, 0, (size_t)m->np * sizeof(float)), "reset adam v");
        m->t = 0;
        refresh_inference(nullptr, m);
        check(cudaStreamSynchronize(nullptr), "sync set");
        return TDDFT_OK;
    });
}

tddft_status tddft_mlp_get(const tddft_mlp *m, float *theta) {
    if (!m || !theta) return TDDFT_E_INVALID;
    return mlp_guard(const_cast<tddft_mlp *>(m), [&]() -> tddft_status {
        check(cudaMemcpy(theta, m->W, (size_t)m->np * sizeof(float), cudaMemcpyDefault), "get parameters");
        return TDDFT_OK;
    });
}

tddft_status tddft_mlp_forward(tddft_mlp *m, int64_t n, const float *X, float *Y) {
    if (!m || n < 0 || (n > 0 && (!X || !Y))) return TDDFT_E_INVALID;
    if (n == 0) return TDDFT_OK;
    if (!dev_ptr(X) || !dev_ptr(Y)) {
        m->err = "tddft_mlp_forward: X and Y must be device pointers";
        return TDDFT_E_INVALID;
    }
    return mlp_guard(m, [&]() -> tddft_status {
        ensure_rows(m, std::min((long long)n, CHUNK));
        const int ld = m->nb + m->nf;
        for (long long r0 = 0; r0 < n; r0 += CHUNK) {
            const long long r = std::min(CHUNK, (long long)n - r0);
            perceptron(nullptr, m, m->Winf, r, X + r0 * ld + m->nb, ld, m->buf.A);
            head_kernel<<<grid_of(r * m->nb), 256>>>(m->buf.A, X + r0 * ld, ld, m->nb, r, Y + r0 * m->nb);
            check_launch("head");
        }
        check(cudaStreamSynchronize(nullptr), "sync forward");
        return TDDFT_OK;
    });
}

tddft_status tddft_mlp_loss_grad(tddft_mlp *m, int64_t n, const float *X, const float *T, const float *w,
                                 double *loss, float *grad) {
    if (!m || n <= 0 || !X || !T) return TDDFT_E_INVALID;
    if (!dev_ptr(X) || !dev_ptr(T) || (w && !dev_ptr(w))) {
        m->err = "tddft_mlp_loss_grad: X, T and w must be device pointers";
        return TDDFT_E_INVALID;
    }
    return mlp_guard(m, [&]() -> tddft_status {
        ensure_rows(m, n);
        loss_grad_rows(nullptr, m, n, X, T, w, m->buf.loss);
        double l = 0.0;
        check(cudaMemcpy(&l, m->buf.loss, sizeof(double), cudaMemcpyDeviceToHost), "D2H loss");
        if (loss) *loss = 0.5 * l;
        if (grad) check(cudaMemcpy(grad, m->g, (size_t)m->np * sizeof(float), cudaMemcpyDeviceToHost), "D2H grad");
        return TDDFT_OK;
    });
}

tddft_status tddft_mlp_train(tddft_mlp *m, int64_t n, const float *X, const float *T, const float *w, int32_t steps,
                             int32_t batch, float lr, const int64_t *order, double *loss_first, double *loss_last) {
    if (!m || n <= 0 || !X || !T || steps < 0 || batch < 1 || !order || !(lr > 0.0f)) return TDDFT_E_INVALID;
    if (!dev_ptr(X) || !dev_ptr(T) || (w && !dev_ptr(w))) {
        m->err = "tddft_mlp_train: X, T and w must be device pointers";
        return TDDFT_E_INVALID;
    }
    for (long long i = 0; i < (long long)steps * batch; ++i)
        if (order[i] < 0 || order[i] >= n) {
            m->err = "tddft_mlp_train: sample index out of range";
            return TDDFT_E_INVALID;
        }
    return mlp_guard(m, [&]() -> tddft_status {
        ensure_rows(m, batch);
        MlpBuffers &B = m->buf;
        const int ld = m->nb + m->nf;
        for (int s = 0; s < steps; ++s) {
            check(cudaMemcpyAsync(B.idx, order + (long long)s * batch, (size_t)batch * sizeof(long long),
                                  cudaMemcpyHostToDevice, nullptr),
                  "H2D minibatch");
            gather_rows_kernel<<<grid_of((long long)batch * ld), 256>>>(X, B.idx, batch, ld, B.Xb);
            check_launch("gather X");
            gather_rows_kernel<<<grid_of((long long)batch * m->nb), 256>>>(T, B.idx, batch, m->nb, B.Tb);
            check_launch("gather T");
            if (w) {
                gather_rows_kernel<<<grid_of(batch), 256>>>(w, B.idx, batch, 1, B.Wb);
                check_launch("gather w");
            }
            loss_grad_rows(nullptr, m, batch, B.Xb, B.Tb, w ? B.Wb : nullptr, B.loss + (s == 0 ? 0 : 1));
            adam(nullptr, m, lr);
        }
        refresh_inference(nullptr, m);
        double h[2] = {0.0, 0.0};
        if (steps > 0) check(cudaMemcpy(h, B.loss, 2 * sizeof(double), cudaMemcpyDeviceToHost), "D2H loss");
        check(cudaStreamSynchronize(nullptr), "sync train");
        if (loss_first) *loss_first = 0.5 * h[0];
        if (loss_last) *loss_last = 0.5 * (steps > 1 ? h[1] : h[0]);
        return TDDFT_OK;
    });
}

}  // extern "C"
