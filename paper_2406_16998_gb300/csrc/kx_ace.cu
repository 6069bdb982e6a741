// ACE tail in float64 (adaptively compressed exchange, the construction Sec. 4
// builds from Vx applied to every occupied orbital):
//   M = dV Psi^T W            (W = Vx Psi, n_orb x n_orb, symmetric, negative semidefinite)
//   -M = R^T R                (Cholesky, R upper triangular)
//   xi = W R^{-1}             (so that -xi (dV xi^T Psi) = W)
#include "kx_internal.h"

#include <algorithm>

namespace kx {
namespace {

constexpr int kG = 32;  // gram tile

// part[s][a][b] = sum over slab s of grid points of psi_a(x) W_b(x)
__global__ void gram_kernel(const double *__restrict__ psi, const double *__restrict__ W, int n_orb, long long N,
                            long long slab, double *__restrict__ part) {
    __shared__ double Ps[kG][kG + 1], Ws[kG][kG + 1];
    const int a0 = blockIdx.x * kG, b0 = blockIdx.y * kG;
    const long long x0 = blockIdx.z * slab, x1 = min(N, x0 + slab);
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 rows of 32
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    for (long long xb = x0; xb < x1; xb += kG) {
        for (int r = ty; r < kG; r += 8) {
            long long x = xb + tx;
            int a = a0 + r, b = b0 + r;
            Ps[r][tx] = (a < n_orb && x < x1) ? psi[(long long)a * N + x] : 0.0;
            Ws[r][tx] = (b < n_orb && x < x1) ? W[(long long)b * N + x] : 0.0;
        }
        __syncthreads();
        for (int k = 0; k < kG; ++k) {
            double w = Ws[tx][k];
#pragma unroll
            for (int u = 0; u < 4; ++u) acc[u] = fma(Ps[ty + 8 * u][k], w, acc[u]);
        }
        __syncthreads();
    }
    for (int u = 0; u < 4; ++u) {
        int a = a0 + ty + 8 * u, b = b0 + tx;
        if (a < n_orb && b < n_orb) part[((long long)blockIdx.z * n_orb + a) * n_orb + b] = acc[u];
    }
}

__global__ void gram_reduce_kernel(const double *__restrict__ part, int n_slab, int n_orb, double dV,
                                   double *__restrict__ M, double *__restrict__ M_out, double *__restrict__ negM) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_orb * n_orb) return;
    double s = 0.0;
    for (int k = 0; k < n_slab; ++k) s += part[(long long)k * n_orb * n_orb + e];
    s *= dV;
    M[e] = s;
    if (M_out) M_out[e] = s;
    negM[e] = -s;
}

// In-place Cholesky of the symmetric positive definite A (lower triangle used):
// A = L L^T; writes R = L^T (upper) to R.  One CTA; *bad = 1 if a pivot <= 0.
__global__ void cholesky_kernel(double *__restrict__ A, int n, double *__restrict__ R, int *__restrict__ bad) {
    __shared__ double piv;
    for (int k = 0; k < n; ++k) {
        if (threadIdx.x == 0) {
            double d = A[k * n + k];
            if (!(d > 0.0)) {
                *bad = 1;
                d = 1.0;
            }
            piv = sqrt(d);
            A[k * n + k] = piv;
        }
        __syncthreads();
        for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) A[i * n + k] /= piv;
        __syncthreads();
        const int m = n - k - 1;
        for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
            int i = k + 1 + e / m, j = k + 1 + e % m;
            if (j <= i) A[i * n + j] -= A[i * n + k] * A[j * n + k];
        }
        __syncthreads();
    }
    for (int e = threadIdx.x; e < n * n; e += blockDim.x) {
        int i = e / n, j = e % n;  // R[i][j] = L[j][i] for j >= i
        R[e] = (j >= i) ? A[j * n + i] : 0.0;
    }
}

// Rinv = R^{-1} (upper triangular), one thread per column, back substitution.
__global__ void triinv_kernel(const double *__restrict__ R, int n, double *__restrict__ Rinv) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    for (int i = n - 1; i >= 0; --i) {
        double s = (i == j) ? 1.0 : 0.0;
        if (i > j) {
            Rinv[i * n + j] = 0.0;
            continue;
        }
        for (int k = i + 1; k <= j; ++k) s -= R[i * n + k] * Rinv[k * n + j];
        Rinv[i * n + j] = s / R[i * n + i];
    }
}

// xi_b(x) = sum_k W_k(x) Rinv[k][b]
__global__ void xi_kernel(const double *__restrict__ W, const double *__restrict__ Rinv, int n_orb, long long N,
                          double *__restrict__ xi) {
    __shared__ double Ws[16][128 + 1];
    __shared__ double Rs[16][32];
    const long long x0 = (long long)blockIdx.x * 128;
    const int b0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 127, ty = threadIdx.x >> 7;  // 2 groups of 16 b
    double acc[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) acc[u] = 0.0;
    for (int k0 = 0; k0 < n_orb; k0 += 16) {
        for (int e = threadIdx.x; e < 16 * 128; e += blockDim.x) {
            int kk = e / 128, xx = e % 128;
            long long x = x0 + xx;
            Ws[kk][xx] = (k0 + kk < n_orb && x < N) ? W[(long long)(k0 + kk) * N + x] : 0.0;
        }
        for (int e = threadIdx.x; e < 16 * 32; e += blockDim.x) {
            int kk = e / 32, bb = e % 32;
            Rs[kk][bb] = (k0 + kk < n_orb && b0 + bb < n_orb) ? Rinv[(k0 + kk) * n_orb + b0 + bb] : 0.0;
        }
        __syncthreads();
        for (int kk = 0; kk < 16; ++kk) {
            double w = Ws[kk][tx];
#pragma unroll
            for (int u = 0; u < 16; ++u) acc[u] = fma(w, Rs[kk][ty * 16 + u], acc[u]);
        }
        __syncthreads();
    }
    long long x = x0 + tx;
    if (x < N) {
        for (int u = 0; u < 16; ++u) {
            int b = b0 + ty * 16 + u;
            if (b < n_orb) xi[(long long)b * N + x] = acc[u];
        }
    }
}

}  // namespace

int ace_run(kx_plan *p, int n_orb, const double *psi, const double *W, double *xi, double *M_out, cudaStream_t s) {
    const long long N = (long long)p->N;
    const int tiles = (n_orb + kG - 1) / kG;
    const int n_slab = (int)std::max(1LL, std::min<long long>(128, (N + 4095) / 4096));
    const long long slab = (N + n_slab - 1) / n_slab;
    const size_t nn = (size_t)n_orb * n_orb;
    const size_t bytes = sizeof(double) * (nn * (size_t)n_slab + 4 * nn) + 256;
    int rc = ensure_workspace(p, bytes);
    if (rc) return rc;
    double *part = (double *)p->ws.ptr;
    double *M = part + nn * n_slab;
    double *A = M + nn;
    double *R = A + nn;
    double *Rinv = R + nn;
    int *bad = reinterpret_cast<int *>(Rinv + nn);
    KX_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), s));
    gram_kernel<<<dim3(tiles, tiles, n_slab), 256, 0, s>>>(psi, W, n_orb, N, slab, part);
    KX_LAUNCH_CHECK("gram_kernel launch");
    gram_reduce_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(part, n_slab, n_orb, p->dV, M, M_out, A);
    KX_LAUNCH_CHECK("gram_reduce_kernel launch");
    cholesky_kernel<<<1, 256, 0, s>>>(A, n_orb, R, bad);
    KX_LAUNCH_CHECK("cholesky_kernel launch");
    triinv_kernel<<<(n_orb + 127) / 128, 128, 0, s>>>(R, n_orb, Rinv);
    KX_LAUNCH_CHECK("triinv_kernel launch");
    xi_kernel<<<dim3((unsigned)((N + 127) / 128), (unsigned)((n_orb + 31) / 32)), 256, 0, s>>>(W, Rinv, n_orb, N, xi);
    KX_LAUNCH_CHECK("xi_kernel launch");
    int h_bad = 0;
    KX_CUDA_TRY(cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    KX_CUDA_TRY(cudaStreamSynchronize(s));
    if (h_bad) return set_error(KX_ERR_ARG, "kx_ace: -M is not positive definite");
    return KX_OK;
}

}  // namespace kx
