// Plan set-up on the GPU (float64): 1D finite-difference Laplacians, their
// eigendecompositions, the f(Lambda) table and the split tensor-core operands.
//
// Sec. 3, Eq. 12: Lk is the centred finite-difference second-derivative matrix
// on the 1D grid of axis k with its boundary condition built in.
// Sec. 3, Eq. 13: Lk Vk = Vk Lambda_k; Vk orthogonal (Lk symmetric).
// Sec. 3, Eq. 19: the scaling diagonal holds f(l1_i + l2_j + l3_k).
#include "kx_internal.h"
#include "kx_fd.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>

namespace kx {
namespace {

constexpr int kEigThreads = 256;
constexpr int kMaxSweeps = 40;

// One CTA per axis: build Lk in shared memory, diagonalise it by cyclic Jacobi
// with a round-robin (tournament) ordering so that n/2 disjoint rotations are
// applied per step, then sort eigenpairs ascending.  All loops are bounded.
__global__ void __launch_bounds__(kEigThreads) eig1d_kernel(int n0, int n1, int n2, double h0, double h1,
                                                          double h2, int bc0, int bc1, int bc2, int order,
                                                          double *lam0, double *lam1, double *lam2,
                                                          double *V0, double *V1, double *V2) {
    extern __shared__ double A[];  // n*n
    __shared__ double cs[kMaxN / 2 + 1], sn[kMaxN / 2 + 1];
    __shared__ int pp[kMaxN / 2 + 1], qq[kMaxN / 2 + 1];
    __shared__ double red[kEigThreads / 32];
    __shared__ int perm[kMaxN];
    __shared__ double lam_s[kMaxN];
    __shared__ int done;

    const int ax = blockIdx.x;
    const int n = ax == 0 ? n0 : (ax == 1 ? n1 : n2);
    const double h = ax == 0 ? h0 : (ax == 1 ? h1 : h2);
    const int bc = ax == 0 ? bc0 : (ax == 1 ? bc1 : bc2);
    double *lam = ax == 0 ? lam0 : (ax == 1 ? lam1 : lam2);
    double *V = ax == 0 ? V0 : (ax == 1 ? V1 : V2);
    const int tid = threadIdx.x;
    const int m = order / 2;
    const double ih2 = 1.0 / (h * h);

    // Lk (one thread per row so periodic wrap-around sums stay race-free)
    for (int i = tid; i < n * n; i += blockDim.x) A[i] = 0.0;
    for (int i = tid; i < n * n; i += blockDim.x) V[i] = (i / n == i % n) ? 1.0 : 0.0;
    __syncthreads();
    for (int i = tid; i < n; i += blockDim.x) {
        for (int p = -m; p <= m; ++p) {
            int j = i + p;
            if (bc == KX_PERIODIC) {
                j %= n;
                if (j < 0) j += n;
            } else if (j < 0 || j >= n) {
                continue;
            }
            A[i * n + j] += fd_weight(m, p < 0 ? -p : p) * ih2;
        }
    }
    __syncthreads();

    const int mm = (n % 2 == 0) ? n : n + 1;  // players incl. a dummy for odd n
    const int half = mm / 2;
    for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
        // convergence: off-diagonal vs total Frobenius norm
        double off = 0.0, tot = 0.0;
        for (int i = tid; i < n * n; i += blockDim.x) {
            double a = A[i];
            tot += a * a;
            if (i / n != i % n) off += a * a;
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            tot += __shfl_xor_sync(0xffffffffu, tot, o);
        }
        if ((tid & 31) == 0) red[tid >> 5] = off;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += red[w];
            red[0] = s;
        }
        __syncthreads();
        double off_all = red[0];
        __syncthreads();
        if ((tid & 31) == 0) red[tid >> 5] = tot;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
            for (int w = 0; w < (int)(blockDim.x / 32); ++w) s += red[w];
            done = (off_all <= 1e-30 * s) ? 1 : 0;
        }
        __syncthreads();
        if (done) break;

        for (int round = 0; round < mm - 1; ++round) {
            if (tid < half) {
                int p, q;
                if (tid == 0) {
                    p = round;
                    q = mm - 1;
                } else {
                    p = (round + tid) % (mm - 1);
                    q = (round - tid + (mm - 1)) % (mm - 1);
                }
                if (p > q) { int t = p; p = q; q = t; }
                double c = 1.0, s = 0.0;
                if (q < n) {
                    double apq = A[p * n + q];
                    if (fabs(apq) > 1e-18 * (fabs(A[p * n + p]) + fabs(A[q * n + q]))) {
                        double theta = (A[q * n + q] - A[p * n + p]) / (2.0 * apq);
                        double t = 1.0 / (fabs(theta) + sqrt(theta * theta + 1.0));
                        if (theta < 0.0) t = -t;
                        c = 1.0 / sqrt(t * t + 1.0);
                        s = t * c;
                    }
                } else {
                    p = q = -1;  // pairs with the dummy player do nothing
                }
                pp[tid] = p;
                qq[tid] = q;
                cs[tid] = c;
                sn[tid] = s;
            }
            __syncthreads();
            // A <- A J  (columns p, q of every row) and V <- V J
            for (int e = tid; e < n * half; e += blockDim.x) {
                int r = e / half, t = e % half;
                int p = pp[t], q = qq[t];
                if (p < 0 || sn[t] == 0.0) continue;
                double c = cs[t], s = sn[t];
                double ap = A[r * n + p], aq = A[r * n + q];
                A[r * n + p] = c * ap - s * aq;
                A[r * n + q] = s * ap + c * aq;
                double vp = V[r * n + p], vq = V[r * n + q];
                V[r * n + p] = c * vp - s * vq;
                V[r * n + q] = s * vp + c * vq;
            }
            __syncthreads();
            // A <- J^T A  (rows p, q of every column)
            for (int e = tid; e < n * half; e += blockDim.x) {
                int col = e / half, t = e % half;
                int p = pp[t], q = qq[t];
                if (p < 0 || sn[t] == 0.0) continue;
                double c = cs[t], s = sn[t];
                double ap = A[p * n + col], aq = A[q * n + col];
                A[p * n + col] = c * ap - s * aq;
                A[q * n + col] = s * ap + c * aq;
            }
            __syncthreads();
            for (int t = tid; t < half; t += blockDim.x) {
                int p = pp[t], q = qq[t];
                if (p >= 0 && sn[t] != 0.0) {
                    A[p * n + q] = 0.0;
                    A[q * n + p] = 0.0;
                }
            }
            __syncthreads();
        }
    }

    // sort eigenpairs ascending (single thread; n <= 128)
    if (tid == 0) {
        for (int i = 0; i < n; ++i) {
            lam_s[i] = A[i * n + i];
            perm[i] = i;
        }
        for (int i = 0; i < n; ++i) {
            int best = i;
            for (int j = i + 1; j < n; ++j)
                if (lam_s[perm[j]] < lam_s[perm[best]]) best = j;
            int t = perm[i]; perm[i] = perm[best]; perm[best] = t;
        }
    }
    __syncthreads();
    for (int i = tid; i < n * n; i += blockDim.x) A[i] = V[i];
    __syncthreads();
    for (int i = tid; i < n * n; i += blockDim.x) {
        int x = i / n, k = i % n;
        V[i] = A[x * n + perm[k]];
    }
    for (int k = tid; k < n; k += blockDim.x) lam[k] = lam_s[perm[k]];
}

// f(l1_k1 + l2_k2 + l3_k3) for every spectral point, float64 and float32.
__global__ void ftable_kernel(int n1, int n2, int n3, const double *l1, const double *l2, const double *l3,
                              int kind, double omega, double *f64, float *f32) {
    size_t N = (size_t)n1 * n2 * n3;
    for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < N;
         idx += (size_t)gridDim.x * blockDim.x) {
        int k1 = (int)(idx % n1);
        int k2 = (int)((idx / n1) % n2);
        int k3 = (int)(idx / ((size_t)n1 * n2));
        double f = kernel_f_value(kind, omega, l1[k1] + l2[k2] + l3[k3]);
        f64[idx] = f;
        f32[idx] = (float)f;
    }
}

// Split the 2^14-scaled, zero-padded V into fp16 hi and lo blocks stored in 8x8
// core-matrix order: element (x, k) at (x/8)*np*8 + (k/8)*64 + (x%8)*8 + (k%8).
__global__ void split_v_kernel(int n, int np, const double *V, __half *out) {
    int total = np * np;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        int x = e / np, k = e % np;
        double v = (x < n && k < n) ? V[x * n + k] * (double)kVScale : 0.0;
        __half hi = __double2half(v);
        __half lo = __double2half(v - (double)__half2float(hi));
        size_t off = (size_t)(x >> 3) * np * 8 + (size_t)(k >> 3) * 64 + (x & 7) * 8 + (k & 7);
        out[off] = hi;
        out[(size_t)total + off] = lo;
    }
}

// max of the f table (one CTA, fixed order)
__global__ void fmax_kernel(const double *f, size_t N, double *out) {
    __shared__ double red[256];
    double m = 0.0;
    for (size_t i = threadIdx.x; i < N; i += blockDim.x) m = fmax(m, f[i]);
    red[threadIdx.x] = m;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

}  // namespace

int plan_setup(kx_plan *p) {
    KX_CUDA_TRY(cudaSetDevice(p->device));
    for (int a = 0; a < 3; ++a) {
        KX_CUDA_TRY(cudaMalloc(&p->d_lam[a], sizeof(double) * p->n[a]));
        KX_CUDA_TRY(cudaMalloc(&p->d_V[a], sizeof(double) * p->n[a] * p->n[a]));
    }
    KX_CUDA_TRY(cudaMalloc(&p->d_f64, sizeof(double) * p->N));
    KX_CUDA_TRY(cudaMalloc(&p->d_f32, sizeof(float) * p->N));
    KX_CUDA_TRY(cudaMalloc(&p->d_status, sizeof(int)));
    KX_CUDA_TRY(cudaMemset(p->d_status, 0, sizeof(int)));

    int nmax = std::max(p->n[0], std::max(p->n[1], p->n[2]));
    size_t smem = sizeof(double) * nmax * nmax;
    KX_CUDA_TRY(cudaFuncSetAttribute(eig1d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    eig1d_kernel<<<3, kEigThreads, smem>>>(p->n[0], p->n[1], p->n[2], p->h[0], p->h[1], p->h[2], p->bc[0],
                                           p->bc[1], p->bc[2], p->fd_order, p->d_lam[0], p->d_lam[1],
                                           p->d_lam[2], p->d_V[0], p->d_V[1], p->d_V[2]);
    KX_LAUNCH_CHECK("eig1d_kernel launch");
    int blocks = (int)std::min<size_t>((p->N + 255) / 256, (size_t)4 * p->num_sms);
    ftable_kernel<<<blocks, 256>>>(p->n[0], p->n[1], p->n[2], p->d_lam[0], p->d_lam[1], p->d_lam[2], p->kind,
                                   p->omega, p->d_f64, p->d_f32);
    KX_LAUNCH_CHECK("ftable_kernel launch");
    if (p->precision == KX_F16X3) {
        for (int a = 0; a < 3; ++a) {
            int np = p->np[a];
            KX_CUDA_TRY(cudaMalloc(&p->d_Vs[a], sizeof(__half) * 2 * np * np));
            split_v_kernel<<<(np * np + 255) / 256, 256>>>(p->n[a], np, p->d_V[a], p->d_Vs[a]);
            KX_LAUNCH_CHECK("split_v_kernel launch");
        }
    }
    if (p->precision == KX_FFT32)
        if (int rc = fft_setup(p)) return rc;
    double *d_fmax = nullptr;
    KX_CUDA_TRY(cudaMalloc(&d_fmax, sizeof(double)));
    fmax_kernel<<<1, 256>>>(p->d_f64, p->N, d_fmax);
    KX_LAUNCH_CHECK("fmax_kernel launch");
    cudaError_t e = cudaMemcpy(&p->fmax, d_fmax, sizeof(double), cudaMemcpyDeviceToHost);
    cudaFree(d_fmax);
    KX_CUDA_TRY(e);
    KX_CUDA_TRY(cudaDeviceSynchronize());
    return KX_OK;
}

void plan_free(kx_plan *p) {
    for (int a = 0; a < 3; ++a) {
        cudaFree(p->d_lam[a]);
        cudaFree(p->d_V[a]);
        cudaFree(p->d_Vs[a]);
    }
    cudaFree(p->d_f64);
    cudaFree(p->d_f32);
    cudaFree(p->d_fft_tw);
    cudaFree(p->d_fft_f);
    cudaFree(p->d_status);
    cudaFree(p->ws.ptr);
    cudaFree(p->ws_host.ptr);
    cudaFree(p->d_pairs);
    cudaFree(p->d_item_slot);
    cudaFree(p->d_groups);
    cudaFree(p->d_pair_mask);
    p->d_pair_mask = nullptr;
    mp_free(p);
    for (cudaEvent_t e : p->copy_events) cudaEventDestroy(e);
    p->copy_events.clear();
    if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
    p->copy_stream = nullptr;
    for (cudaEvent_t e : p->h2d_events) cudaEventDestroy(e);
    p->h2d_events.clear();
    if (p->h2d_stream) cudaStreamDestroy(p->h2d_stream);
    p->h2d_stream = nullptr;
}

}  // namespace kx
