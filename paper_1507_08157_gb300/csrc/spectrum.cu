// Transition dipoles, oscillator strengths and broadened spectra of converged excitations. The
// paper reports every result as energies with oscillator strengths and as spectra broadened by
// 0.025 eV Lorentzians (Sec. IV). Standard linear-response forms: the transition dipole of
// excitation m is the dipole of its response density rho^q (Sec. II C builds rho from the q
// kernel), the pair normalised by <p, q> = 1 (Eq. Tsiper_multiple); f = (2/3) omega |mu|^2. The
// position of grid point i along an axis is i h - L/2 (measured from the cell centre).
#include "solver_kernels.h"

#include <cuda_runtime.h>

namespace tddft {
namespace {

constexpr int DIP_THREADS = 256;

// one block per (slice, state): float64 sums of x rho, y rho, z rho over a grid-stride range
template <typename T>
__global__ void __launch_bounds__(DIP_THREADS) dipole_kernel(const T *__restrict__ rho, int n, double h, double L,
                                                             int nblk, double *__restrict__ partials) {
    const int s = blockIdx.y, b = blockIdx.x;
    const long long n2 = (long long)n * n, n3 = n2 * n;
    const T *r = rho + (long long)s * n3;
    double ax = 0.0, ay = 0.0, az = 0.0;
    for (long long l = (long long)b * DIP_THREADS + threadIdx.x; l < n3; l += (long long)nblk * DIP_THREADS) {
        const int i = (int)(l / n2), j = (int)((l / n) % n), q = (int)(l % n);
        const double v = (double)r[l];
        ax += (i * h - 0.5 * L) * v;
        ay += (j * h - 0.5 * L) * v;
        az += (q * h - 0.5 * L) * v;
    }
    __shared__ double red[3][DIP_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) {
        ax += __shfl_xor_sync(0xffffffffu, ax, o);
        ay += __shfl_xor_sync(0xffffffffu, ay, o);
        az += __shfl_xor_sync(0xffffffffu, az, o);
    }
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[0][w] = ax;
        red[1][w] = ay;
        red[2][w] = az;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double t = 0.0;
        for (int q = 0; q < DIP_THREADS / 32; ++q) t += red[threadIdx.x][q];
        partials[((long long)s * nblk + b) * 3 + threadIdx.x] = t;
    }
}

// one thread: partial sums in a fixed order, rotation to the Ritz pairs, strengths
__global__ void ritz_kernel(int k, const double *omega, const double *vecs, const double *partials, int nblk,
                            double dV, double *out) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double mu[KMAX][3];
    for (int j = 0; j < k; ++j)
        for (int a = 0; a < 3; ++a) {
            double t = 0.0;
            for (int b = 0; b < nblk; ++b) t += partials[((long long)j * nblk + b) * 3 + a];
            mu[j][a] = dV * t;
        }
    for (int m = 0; m < k; ++m) {
        double r[3] = {0.0, 0.0, 0.0};
        for (int j = 0; j < k; ++j)
            for (int a = 0; a < 3; ++a) r[a] += vecs[j * k + m] * mu[j][a];
        out[m] = (2.0 / 3.0) * omega[m] * (r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
        for (int a = 0; a < 3; ++a) out[k + 3 * m + a] = r[a];
    }
}

__global__ void lorentz_kernel(int k, const double *omega, const double *f, double gamma, int n, const double *E,
                               double *S) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const double inv_pi = 0.31830988618379067154;
    double t = 0.0;
    for (int i = 0; i < k; ++i) {
        const double d = E[e] - omega[i];
        t += f[i] * (gamma * inv_pi) / (d * d + gamma * gamma);
    }
    S[e] = t;
}

}  // namespace

template <typename T>
void dipole_partials(cudaStream_t st, const T *rho, int n, double h, double L, int k, int nblk, double *partials) {
    ProfScope ps(st, ST_TRACE, 6.0 * k * (double)n * n * n, sizeof(T) * (double)k * n * n * n);
    dipole_kernel<T><<<dim3(nblk, k), DIP_THREADS, 0, st>>>(rho, n, h, L, nblk, partials);
    check_launch("dipole_kernel");
}

void ritz_strengths(cudaStream_t st, int k, const double *omega, const double *vecs, const double *partials,
                    int nblk, double dV, double *out) {
    ProfScope ps(st, ST_SMALL, 0.0, 0.0);
    ritz_kernel<<<1, 1, 0, st>>>(k, omega, vecs, partials, nblk, dV, out);
    check_launch("ritz_kernel");
}

void lorentz_spectrum(cudaStream_t st, int k, const double *omega, const double *f, double gamma, int n,
                      const double *E, double *S) {
    ProfScope ps(st, ST_SMALL, 0.0, 0.0);
    lorentz_kernel<<<(n + 255) / 256, 256, 0, st>>>(k, omega, f, gamma, n, E, S);
    check_launch("lorentz_kernel");
}

template void dipole_partials<float>(cudaStream_t, const float *, int, double, double, int, int, double *);
template void dipole_partials<double>(cudaStream_t, const double *, int, double, double, int, int, double *);

}  // namespace tddft
