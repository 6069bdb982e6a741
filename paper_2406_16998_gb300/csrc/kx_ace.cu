// ACE tail (adaptively compressed exchange, the construction Sec. 4 builds
// from Vx applied to every occupied orbital) and the compressed operator's
// application:
//   M = dV Psi^T W            (W = Vx Psi, n_orb x n_orb, symmetric, negative semidefinite)
//   -M = R^T R                (Cholesky, R upper triangular)
//   xi = W R^{-1}             (so that -xi (dV xi^T Psi) = W)
//   V_ACE phi = -xi (dV xi^T phi)
// The small matrices (M, its Cholesky factor, R^{-1}, the projections
// dV xi^T phi) are float64.  The two grid-sized products, a projection
// A^T B over all grid points and a combination A C of grid vectors, run in
// float64 for KX_FP64 plans; for the tensor-core plans they take float32
// products summed in float32 over short blocks (256 grid points, or one
// combination) and in float64 across blocks, because float64 arithmetic on
// this GPU runs at a small fraction of the float32 rate and both products
// are bound by memory traffic once they run in float32.
#include "kx_internal.h"

#include <algorithm>

namespace kx {
namespace {

constexpr int kG = 32;  // gram tile

// part[s][a][b] = sum over slab s of grid points of psi_a(x) W_b(x)   (a < na, b < nb)
__global__ void gram_kernel(const double *__restrict__ psi, int na, const double *__restrict__ W, int nb, long long N,
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
            Ps[r][tx] = (a < na && x < x1) ? psi[(long long)a * N + x] : 0.0;
            Ws[r][tx] = (b < nb && x < x1) ? W[(long long)b * N + x] : 0.0;
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
        if (a < na && b < nb) part[((long long)blockIdx.z * na + a) * nb + b] = acc[u];
    }
}

// M[e] = dV sum_k part[k][e] in a fixed order (deterministic); optional copies
// of M and -M.
__global__ void gram_reduce_kernel(const double *__restrict__ part, int n_slab, int n_e, double dV,
                                   double *__restrict__ M, double *__restrict__ M_out, double *__restrict__ negM) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_e) return;
    double s = 0.0;
    for (int k = 0; k < n_slab; ++k) s += part[(long long)k * n_e + e];
    s *= dV;
    M[e] = s;
    if (M_out) M_out[e] = s;
    if (negM) negM[e] = -s;
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

// xi_b(x) = sgn sum_k W_k(x) Rinv[k][b]   (k < na, b < nb; Rinv row-major na x nb)
__global__ void xi_kernel(const double *__restrict__ W, const double *__restrict__ Rinv, int na, int nb, long long N,
                          double sgn, double *__restrict__ xi) {
    __shared__ double Ws[16][128 + 1];
    __shared__ double Rs[16][32];
    const long long x0 = (long long)blockIdx.x * 128;
    const int b0 = blockIdx.y * 32;
    const int tx = threadIdx.x & 127, ty = threadIdx.x >> 7;  // 2 groups of 16 b
    double acc[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) acc[u] = 0.0;
    for (int k0 = 0; k0 < na; k0 += 16) {
        for (int e = threadIdx.x; e < 16 * 128; e += blockDim.x) {
            int kk = e / 128, xx = e % 128;
            long long x = x0 + xx;
            Ws[kk][xx] = (k0 + kk < na && x < N) ? W[(long long)(k0 + kk) * N + x] : 0.0;
        }
        for (int e = threadIdx.x; e < 16 * 32; e += blockDim.x) {
            int kk = e / 32, bb = e % 32;
            Rs[kk][bb] = (k0 + kk < na && b0 + bb < nb) ? Rinv[(k0 + kk) * nb + b0 + bb] : 0.0;
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
            if (b < nb) xi[(long long)b * N + x] = sgn * acc[u];
        }
    }
}

// ---------------------------------------------------------------------------
// float32-product forms of the two grid-sized products
// ---------------------------------------------------------------------------
constexpr int kPT = 64;   // projection tile: 64 a x 64 b per CTA
constexpr int kPX = 64;   // grid points per shared-memory step
constexpr int kPBlk = 4;  // steps summed in float32 before the float64 accumulation (256 points)

// part[blockIdx.x][a][b] = sum over the CTA's grid points [x0, x0 + span) of
// A_a(x) B_b(x) for its 64 x 64 tile (blockIdx.y, blockIdx.z).  Thread (tx, ty)
// of a 16 x 16 layout owns a = a0 + ty + 16 i, b = b0 + tx + 16 j (i, j < 4):
// per four grid points it reads four a-rows (two distinct per warp, broadcast)
// and four b-rows as float4 and does 64 FMAs.
__global__ void __launch_bounds__(256) proj32_kernel(const double *__restrict__ A, int na,
                                                     const double *__restrict__ B, int nb, long long N,
                                                     long long span, double *__restrict__ part) {
    __shared__ __align__(16) float As[kPT][kPX + 4];
    __shared__ __align__(16) float Bs[kPT][kPX + 4];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int a0 = blockIdx.y * kPT, b0 = blockIdx.z * kPT;
    const long long x0 = (long long)blockIdx.x * span;
    const long long x1 = min(N, x0 + span);
    double acc[4][4];
    float s[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            acc[i][j] = 0.0;
            s[i][j] = 0.f;
        }
    const int lx = tid & 63, lr = tid >> 6;  // loader: one grid point, rows lr + 4k
    int steps = 0;
    for (long long xb = x0; xb < x1; xb += kPX) {
        const long long x = xb + lx;
        const bool okx = x < x1;
        float va[16], vb[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int r = lr + 4 * k;
            va[k] = (okx && a0 + r < na) ? (float)__ldg(A + (long long)(a0 + r) * N + x) : 0.f;
            vb[k] = (okx && b0 + r < nb) ? (float)__ldg(B + (long long)(b0 + r) * N + x) : 0.f;
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            As[lr + 4 * k][lx] = va[k];
            Bs[lr + 4 * k][lx] = vb[k];
        }
        __syncthreads();
#pragma unroll 2
        for (int xx = 0; xx < kPX; xx += 4) {
            float4 av[4], bv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) av[i] = *reinterpret_cast<const float4 *>(&As[ty + 16 * i][xx]);
#pragma unroll
            for (int j = 0; j < 4; ++j) bv[j] = *reinterpret_cast<const float4 *>(&Bs[tx + 16 * j][xx]);
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    s[i][j] = fmaf(av[i].x, bv[j].x, s[i][j]);
                    s[i][j] = fmaf(av[i].y, bv[j].y, s[i][j]);
                    s[i][j] = fmaf(av[i].z, bv[j].z, s[i][j]);
                    s[i][j] = fmaf(av[i].w, bv[j].w, s[i][j]);
                }
        }
        __syncthreads();
        if (++steps == kPBlk) {
            steps = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    acc[i][j] += (double)s[i][j];
                    s[i][j] = 0.f;
                }
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int a = a0 + ty + 16 * i, b = b0 + tx + 16 * j;
            if (a < na && b < nb) part[((long long)blockIdx.x * na + a) * nb + b] = acc[i][j] + (double)s[i][j];
        }
}

constexpr int kCX = 128;  // combination tile: 128 grid points x 64 output vectors per CTA
constexpr int kCB = 64;
constexpr int kCA = 32;   // input vectors per shared-memory step

// out_b(x) = sgn sum_a A_a(x) C[a][b]   (a < na, b < nb; C row-major na x nb).
// Thread (tx, ty) of a 32 x 8 layout owns x = x0 + tx + 32 k (k < 4) and
// b = b0 + 8 ty + j (j < 8): the C row piece it needs is the same for the
// whole warp (two broadcast float4 reads), the A values are consecutive
// across lanes.  Sums over a stay in float32 (na <= 256 terms).
__global__ void __launch_bounds__(256) combine32_kernel(const double *__restrict__ A, int na,
                                                        const double *__restrict__ C, int nb, long long N, double sgn,
                                                        double *__restrict__ out) {
    __shared__ __align__(16) float As[kCA][kCX];
    __shared__ __align__(16) float Cs[kCA][kCB];
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const long long x0 = (long long)blockIdx.x * kCX;
    const int b0 = blockIdx.y * kCB;
    float acc[8][4];
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[j][k] = 0.f;
    const int lx = tid & 127, lr = tid >> 7;  // loader: one grid point, rows lr + 2m
    const long long xl = x0 + lx;
    for (int a0 = 0; a0 < na; a0 += kCA) {
        float va[16];
#pragma unroll
        for (int m = 0; m < 16; ++m) {
            const int r = lr + 2 * m;
            va[m] = (xl < N && a0 + r < na) ? (float)__ldg(A + (long long)(a0 + r) * N + xl) : 0.f;
        }
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int e = tid + 256 * m, r = e >> 6, c = e & 63;
            Cs[r][c] = (a0 + r < na && b0 + c < nb) ? (float)__ldg(C + (long long)(a0 + r) * nb + b0 + c) : 0.f;
        }
#pragma unroll
        for (int m = 0; m < 16; ++m) As[lr + 2 * m][lx] = va[m];
        __syncthreads();
#pragma unroll 4
        for (int r = 0; r < kCA; ++r) {
            float av[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) av[k] = As[r][tx + 32 * k];
            const float4 c0 = *reinterpret_cast<const float4 *>(&Cs[r][8 * ty]);
            const float4 c1 = *reinterpret_cast<const float4 *>(&Cs[r][8 * ty + 4]);
            const float cv[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
            for (int j = 0; j < 8; ++j)
#pragma unroll
                for (int k = 0; k < 4; ++k) acc[j][k] = fmaf(av[k], cv[j], acc[j][k]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int b = b0 + 8 * ty + j;
        if (b >= nb) continue;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const long long x = x0 + tx + 32 * k;
            if (x < N) out[(long long)b * N + x] = sgn * (double)acc[j][k];
        }
    }
}

// part (n_split x na x nb) of A^T B over the grid, float64 or float32 products
// by plan precision; returns n_split.
int launch_projection(const kx_plan *p, const double *A, int na, const double *B, int nb, double *part,
                      int n_split, cudaStream_t s) {
    const long long N = (long long)p->N;
    const long long span = (N + n_split - 1) / n_split;
    if (p->precision == KX_FP64) {
        gram_kernel<<<dim3((na + kG - 1) / kG, (nb + kG - 1) / kG, n_split), 256, 0, s>>>(A, na, B, nb, N, span, part);
        KX_LAUNCH_CHECK("gram_kernel launch");
    } else {
        proj32_kernel<<<dim3(n_split, (na + kPT - 1) / kPT, (nb + kPT - 1) / kPT), 256, 0, s>>>(A, na, B, nb, N, span,
                                                                                               part);
        KX_LAUNCH_CHECK("proj32_kernel launch");
    }
    return KX_OK;
}

// Grid points per projection CTA: enough CTAs for a few per SM, at least 256
// points each; float64 plans keep the earlier fixed slab split.
int projection_split(const kx_plan *p, int na, int nb) {
    const long long N = (long long)p->N;
    if (p->precision == KX_FP64) return (int)std::max(1LL, std::min<long long>(128, (N + 4095) / 4096));
    const long long tiles = (long long)((na + kPT - 1) / kPT) * ((nb + kPT - 1) / kPT);
    const long long want = std::max(1LL, (3LL * p->num_sms + tiles - 1) / tiles);
    return (int)std::max(1LL, std::min<long long>(want, (N + 255) / 256));
}

// out = sgn A C (grid vectors), float64 or float32 products by plan precision.
int launch_combination(const kx_plan *p, const double *A, int na, const double *C, int nb, double sgn, double *out,
                       cudaStream_t s) {
    const long long N = (long long)p->N;
    if (p->precision == KX_FP64) {
        xi_kernel<<<dim3((unsigned)((N + 127) / 128), (unsigned)((nb + 31) / 32)), 256, 0, s>>>(A, C, na, nb, N, sgn,
                                                                                              out);
        KX_LAUNCH_CHECK("xi_kernel launch");
    } else {
        combine32_kernel<<<dim3((unsigned)((N + kCX - 1) / kCX), (unsigned)((nb + kCB - 1) / kCB)), 256, 0, s>>>(
            A, na, C, nb, N, sgn, out);
        KX_LAUNCH_CHECK("combine32_kernel launch");
    }
    return KX_OK;
}

}  // namespace

int ace_run(kx_plan *p, int n_orb, const double *psi, const double *W, double *xi, double *M_out, cudaStream_t s) {
    const int n_slab = projection_split(p, n_orb, n_orb);
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
    if ((rc = launch_projection(p, psi, n_orb, W, n_orb, part, n_slab, s))) return rc;
    gram_reduce_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(part, n_slab, (int)nn, p->dV, M, M_out, A);
    KX_LAUNCH_CHECK("gram_reduce_kernel launch");
    cholesky_kernel<<<1, 256, 0, s>>>(A, n_orb, R, bad);
    KX_LAUNCH_CHECK("cholesky_kernel launch");
    triinv_kernel<<<(n_orb + 127) / 128, 128, 0, s>>>(R, n_orb, Rinv);
    KX_LAUNCH_CHECK("triinv_kernel launch");
    if ((rc = launch_combination(p, W, n_orb, Rinv, n_orb, 1.0, xi, s))) return rc;
    int h_bad = 0;
    KX_CUDA_TRY(cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    KX_CUDA_TRY(cudaStreamSynchronize(s));
    if (h_bad) return set_error(KX_ERR_ARG, "kx_ace: -M is not positive definite");
    return KX_OK;
}

int ace_apply_run(kx_plan *p, int n_xi, const double *xi, int n_vec, const double *phi, double *out,
                  cudaStream_t s) {
    const int n_split = projection_split(p, n_xi, n_vec);
    const size_t ne = (size_t)n_xi * n_vec;
    int rc = ensure_workspace(p, sizeof(double) * ne * ((size_t)n_split + 1) + 256);
    if (rc) return rc;
    double *part = (double *)p->ws.ptr;
    double *P = part + ne * n_split;
    // P = dV xi^T phi, then out = -xi P
    if ((rc = launch_projection(p, xi, n_xi, phi, n_vec, part, n_split, s))) return rc;
    gram_reduce_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, s>>>(part, n_split, (int)ne, p->dV, P, nullptr,
                                                                    nullptr);
    KX_LAUNCH_CHECK("gram_reduce_kernel launch");
    return launch_combination(p, xi, n_xi, P, n_vec, -1.0, out, s);
}

}  // namespace kx
