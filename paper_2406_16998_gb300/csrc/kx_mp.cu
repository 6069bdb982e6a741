// Dirichlet values from the multipole expansion of the source (Sec. 4: the
// linear systems of isolated systems take their boundary values from the
// multipole expansion of the Coulomb kernel, imposed through the right-hand
// side).  With the exterior values phi_ext of the expansion of rho's potential
// about the box centre, moving them to the right-hand side of the
// finite-difference equation gives
//     phi = f(L) (rho + L_ext phi_ext / (4 pi)).
// The expansion is linear in rho through its moments Q_k(rho) = dV sum_x
// rho(x) R_k(x - c), so with the plan's fields
//     g_k = L_ext I_k / (4 pi)   (boundary layer of the irregular harmonic I_k)
//     h_k = f(L) g_k
// the solution is phi = f(L) rho + sum_k Q_k(rho) h_k: the existing solve plus
// a rank-K correction (K = (l_max + 1)^2).  For the exchange operator, with
// rho_ij = psi_i psi_j,
//     (Vx psi)_i -= sum_k h_k sum_j g_j Q_k(ij) psi_j,
//     E_x        -= 1/2 dV sum_ij g_i g_j <psi_i psi_j, sum_k Q_k(ij) h_k>.
// R_k and I_k are the real solid harmonics in Schmidt normalisation, for which
// sum_k R_k(v') I_k(v) = sum_l |v'|^l / |v|^(l+1) P_l(cos gamma), the Legendre
// expansion of 1 / |v - v'|.
#include "kx_internal.h"
#include "kx_tc_ptx.cuh"
#include "kx_conv.cuh"

#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

namespace kx {
namespace {

constexpr int kMpMaxL = 8;
constexpr int kMpMaxK = (kMpMaxL + 1) * (kMpMaxL + 1);
constexpr int kMaxHalf = 16;  // stencil half-width limit (order <= 32)

struct MpGeom {
    int n[3];
    double h[3], c[3];
    int m;                 // stencil half-width
    double w[kMaxHalf + 1];  // centred second-derivative weights for h = 1
    int L, K;
};

__device__ double mp_factorial(int n) {
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

// R[k] for k = l^2 + (m == 0 ? 0 : 2m - 1 + t), t = 0 (cos) / 1 (sin):
// r^l P_l^m(cos theta) (cos | sin)(m phi) sqrt((2 - delta_m0) (l-m)! / (l+m)!),
// evaluated as polynomials: (x + i y)^m times A_l^m(z, r^2), where
// A_m^m = (2m-1)!!, A_{m+1}^m = (2m+1) z A_m^m and
// (l - m) A_l^m = (2l - 1) z A_{l-1}^m - (l + m - 1) r^2 A_{l-2}^m.
__device__ void solid_harmonics(double x, double y, double z, int L, double *R) {
    const double r2 = x * x + y * y + z * z;
    double cm = 1.0, sm = 0.0, dfact = 1.0;
    for (int m = 0; m <= L; ++m) {
        double p1 = 0.0, p2 = 0.0;
        for (int l = m; l <= L; ++l) {
            double a;
            if (l == m)
                a = dfact;
            else if (l == m + 1)
                a = (2 * m + 1) * z * p1;
            else
                a = ((2 * l - 1) * z * p1 - (l + m - 1) * r2 * p2) / (l - m);
            p2 = p1;
            p1 = a;
            const double nrm = sqrt((m == 0 ? 1.0 : 2.0) * mp_factorial(l - m) / mp_factorial(l + m));
            if (m == 0) {
                R[l * l] = nrm * a;
            } else {
                R[l * l + 2 * m - 1] = nrm * a * cm;
                R[l * l + 2 * m] = nrm * a * sm;
            }
        }
        const double cn = x * cm - y * sm, sn = x * sm + y * cm;
        cm = cn;
        sm = sn;
        dfact *= (2 * m + 1);
    }
}

// One thread per grid point: R_k(x - c) and g_k(x) = (1 / 4 pi) sum over the
// exterior points e the stencil of x reaches of w_|d| / h_a^2 I_k(e - c).
__global__ void mp_fields_kernel(const MpGeom G, long long N, double *__restrict__ R, double *__restrict__ Gk) {
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N) return;
    const int i1 = (int)(idx % G.n[0]);
    const int i2 = (int)((idx / G.n[0]) % G.n[1]);
    const int i3 = (int)(idx / ((long long)G.n[0] * G.n[1]));
    const int ii[3] = {i1, i2, i3};
    double v[3];
    for (int a = 0; a < 3; ++a) v[a] = (ii[a] + 1) * G.h[a] - G.c[a];
    double Rv[kMpMaxK], g[kMpMaxK];
    solid_harmonics(v[0], v[1], v[2], G.L, Rv);
    for (int k = 0; k < G.K; ++k) {
        R[(long long)k * N + idx] = Rv[k];
        g[k] = 0.0;
    }
    for (int a = 0; a < 3; ++a) {
        for (int side = 0; side < 2; ++side) {
            // exterior indices e on this side within reach: |e - i_a| <= m
            const int e0 = side == 0 ? ii[a] - G.m : G.n[a];
            const int e1 = side == 0 ? -1 : ii[a] + G.m;
            for (int e = e0; e <= e1; ++e) {
                const int d = e > ii[a] ? e - ii[a] : ii[a] - e;
                double p[3] = {v[0], v[1], v[2]};
                p[a] = (e + 1) * G.h[a] - G.c[a];
                solid_harmonics(p[0], p[1], p[2], G.L, Rv);
                const double r = sqrt(p[0] * p[0] + p[1] * p[1] + p[2] * p[2]);
                const double wd = G.w[d] / (G.h[a] * G.h[a]);
                double inv = 1.0 / r;  // 1 / r^(2l+1), l = 0 first
                for (int l = 0; l <= G.L; ++l) {
                    for (int k = l * l; k < (l + 1) * (l + 1); ++k) g[k] += wd * Rv[k] * inv;
                    inv /= r * r;
                }
            }
        }
    }
    const double s = 1.0 / (4.0 * 3.14159265358979323846);
    for (int k = 0; k < G.K; ++k) Gk[(long long)k * N + idx] = g[k] * s;
}

__global__ void to_f32_kernel(const double *__restrict__ in, float *__restrict__ out, long long n) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

// C[k][j][i] = scale g_j mask(i, j) Q[k][i][j]   (T = float or double)
template <typename T>
__global__ void mp_coef_kernel(const double *__restrict__ Q, const unsigned char *__restrict__ mask,
                               const double *__restrict__ occ, int n, int K, double scale, T *__restrict__ C) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long nn = (long long)n * n;
    if (e >= nn * K) return;
    const int k = (int)(e / nn), i = (int)((e % nn) / n), j = (int)(e % n);
    const double gj = occ ? occ[j] : 1.0;
    C[(long long)k * nn + (long long)j * n + i] = (T)(mask[(long long)i * n + j] ? scale * gj * Q[e] : 0.0);
}

constexpr int kMcX = 128;  // correction tile: 128 grid points x 64 orbitals

// vx_i(x) -= T_i(x), T_i(x) = sum_k h_k(x) sum_j C[k][j][i] psi_j(x), float32
// products (psi converted once per tile into shared memory, C[k] staged per k);
// e_part[CTA] = sum over the tile of g_i psi_i(x) T_i(x).  Thread (tx, ty) owns
// x = x0 + tx + 32 q (q < 4) and i = i0 + 8 ty + u (u < 8); the orbitals are
// taken in pairs (u, u + 1) by packed f32x2 FMAs.
__global__ void __launch_bounds__(256) mp_combine32_kernel(const double *__restrict__ psi, int n,
                                                           const float *__restrict__ C, const float *__restrict__ H,
                                                           int K, const double *__restrict__ occ, long long N,
                                                           double *__restrict__ vx, double *__restrict__ e_part) {
    extern __shared__ __align__(16) float mp_smem[];
    float *Ps = mp_smem;                  // [n][kMcX]
    float *Cs = mp_smem + (size_t)n * kMcX;  // [n][64]
    __shared__ double red[8];
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const long long x0 = (long long)blockIdx.x * kMcX;
    const int i0 = blockIdx.y * 64;
    for (int e = tid; e < n * kMcX; e += 256) {
        const int j = e / kMcX, c = e % kMcX;
        const long long x = x0 + c;
        Ps[e] = x < N ? (float)psi[(long long)j * N + x] : 0.f;
    }
    float2 acc[4][4];  // acc[up][q]: orbitals 2 up (.x) and 2 up + 1 (.y) at point q
#pragma unroll
    for (int up = 0; up < 4; ++up)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[up][q] = make_float2(0.f, 0.f);
    for (int k = 0; k < K; ++k) {
        __syncthreads();
        const float *Ck = C + (size_t)k * n * n;
        for (int e = tid; e < n * 64; e += 256) {
            const int j = e >> 6, c = e & 63;
            Cs[e] = i0 + c < n ? Ck[(size_t)j * n + i0 + c] : 0.f;
        }
        __syncthreads();
        float2 t[4][4];
#pragma unroll
        for (int up = 0; up < 4; ++up)
#pragma unroll
            for (int q = 0; q < 4; ++q) t[up][q] = make_float2(0.f, 0.f);
#pragma unroll 2
        for (int j = 0; j < n; ++j) {
            float2 pv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float v = Ps[j * kMcX + tx + 32 * q];
                pv[q] = make_float2(v, v);
            }
            const float4 c0 = *reinterpret_cast<const float4 *>(&Cs[j * 64 + 8 * ty]);
            const float4 c1 = *reinterpret_cast<const float4 *>(&Cs[j * 64 + 8 * ty + 4]);
            const float2 cv[4] = {make_float2(c0.x, c0.y), make_float2(c0.z, c0.w), make_float2(c1.x, c1.y),
                                  make_float2(c1.z, c1.w)};
#pragma unroll
            for (int up = 0; up < 4; ++up)
#pragma unroll
                for (int q = 0; q < 4; ++q) fma2(t[up][q], cv[up], pv[q]);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const long long x = x0 + tx + 32 * q;
            const float hk = x < N ? __ldg(H + (size_t)k * N + x) : 0.f;
            const float2 h2 = make_float2(hk, hk);
#pragma unroll
            for (int up = 0; up < 4; ++up) fma2(acc[up][q], h2, t[up][q]);
        }
    }
    double e = 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int i = i0 + 8 * ty + u;
        if (i >= n) continue;
        const double gi = occ ? occ[i] : 1.0;
        float ei = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const long long x = x0 + tx + 32 * q;
            if (x >= N) continue;
            const float a = (u & 1) ? acc[u >> 1][q].y : acc[u >> 1][q].x;
            vx[(long long)i * N + x] -= (double)a;
            ei = fmaf(Ps[i * kMcX + tx + 32 * q], a, ei);
        }
        e += gi * (double)ei;
    }
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    if ((tid & 31) == 0) red[ty] = e;
    __syncthreads();
    if (tid == 0) {
        double sum = 0.0;
        for (int w = 0; w < 8; ++w) sum += red[w];
        e_part[(long long)blockIdx.y * gridDim.x + blockIdx.x] = sum;
    }
}

// float64 form: one thread per (grid point, orbital), block partials of the energy.
__global__ void mp_combine64_kernel(const double *__restrict__ psi, int n, const double *__restrict__ C,
                                    const double *__restrict__ H, int K, const double *__restrict__ occ, long long N,
                                    double *__restrict__ vx, double *__restrict__ e_part) {
    __shared__ double red[256];
    const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    double e = 0.0;
    if (x < N) {
        double T = 0.0;
        for (int k = 0; k < K; ++k) {
            const double *Ck = C + (size_t)k * n * n;
            double t = 0.0;
            for (int j = 0; j < n; ++j) t = fma(Ck[(size_t)j * n + i], psi[(long long)j * N + x], t);
            T = fma(H[(size_t)k * N + x], t, T);
        }
        vx[(long long)i * N + x] -= T;
        e = (occ ? occ[i] : 1.0) * psi[(long long)i * N + x] * T;
    }
    red[threadIdx.x] = e;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) e_part[(long long)blockIdx.y * gridDim.x + blockIdx.x] = red[0];
}

// ---------------------------------------------------------------------------
// Moments on the tensor cores (at most 64 orbitals): for the harmonic pairs
// (2p, 2p+1) of this CTA, D_p[(t, i)][j] = sum_x (psi_i R_{2p+t})(x) psi_j(x)
// over the CTA's grid points, as 128 x 64 tcgen05 products with K = grid
// points: A rows are (harmonic t, orbital i), B rows orbitals j, both K-major
// fp16 hi/lo splits of power-of-two-scaled values (|psi s_psi| < 1,
// |R_k s_k| < 2^14), three products per k-step (cross terms first, the hi*hi
// chain split over two accumulators as in the mode products).  One step = 64
// grid points: every thread stages two (orbital, 8-point) tasks of B and the
// matching rows of all A tiles, then one thread issues the step's products.
// ---------------------------------------------------------------------------
constexpr int kMtX = 64;                  // grid points per step
constexpr int kMtPairs = 4;               // harmonic pairs per CTA (two fp32 accumulators of 64 columns each)
constexpr uint32_t kMtGroup = 1024;       // bytes per 8-row group: 8 core matrices of 8 points along K
constexpr size_t kMtB = 64 * kMtX * 2;    // hi (or lo) of B: 64 orbitals x 64 points fp16
constexpr size_t kMtA = 128 * kMtX * 2;   // hi (or lo) of one A pair tile
// raw inputs of one step, copied a step ahead: psi rows (64 points, float64,
// rows padded by 16 bytes so that lanes reading different rows hit distinct
// banks) and the pass's 8 weight rows (float32)
constexpr int kMtRawRow = kMtX * 8 + 16;
constexpr size_t kMtRawPsi = 64 * (size_t)kMtRawRow;
constexpr size_t kMtRaw = kMtRawPsi + 2 * kMtPairs * kMtX * 4;
constexpr size_t kMtSmem = 2 * kMtB + (size_t)kMtPairs * 2 * kMtA + 2 * kMtRaw + 1024;

__device__ __forceinline__ void mt_split_store(uint8_t *hi, uint8_t *lo, int off, const float *w) {
    __half2 h[4], l[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const __half2 hh = __floats2half2_rn(w[2 * c], w[2 * c + 1]);
        const float2 hf = __half22float2(hh);
        h[c] = hh;
        l[c] = __floats2half2_rn(w[2 * c] - hf.x, w[2 * c + 1] - hf.y);
    }
    *reinterpret_cast<uint4 *>(hi + off) = *reinterpret_cast<uint4 *>(h);
    *reinterpret_cast<uint4 *>(lo + off) = *reinterpret_cast<uint4 *>(l);
}

// Three-product split MMA of one step into (Da, Db); accumulate = 0 starts them.
__device__ __forceinline__ void mt_issue(uint32_t da, uint32_t db, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi,
                                         uint32_t b_lo, bool accumulate) {
    const uint32_t idesc = ptx::idesc_f16(128, 64, 0, 0);  // A and B K-major
    const uint64_t ah0 = ptx::sdesc(a_hi, 128, kMtGroup), al0 = ptx::sdesc(a_lo, 128, kMtGroup);
    const uint64_t bh0 = ptx::sdesc(b_hi, 128, kMtGroup), bl0 = ptx::sdesc(b_lo, 128, kMtGroup);
    const uint64_t inc = 256 >> 4;  // one k-step = 16 points = two core matrices
    uint64_t ah = ah0, al = al0, bh = bh0, bl = bl0;
    for (int ks = 0; ks < kMtX / 16; ++ks) {
        ptx::mma_f16(da, ah, bl, idesc, (ks > 0 || accumulate) ? 1u : 0u);
        ptx::mma_f16(da, al, bh, idesc, 1u);
        ah += inc;
        al += inc;
        bh += inc;
        bl += inc;
    }
    ah = ah0;
    bh = bh0;
    for (int ks = 0; ks < kMtX / 16; ++ks) {
        if (ks & 1)
            ptx::mma_f16(db, ah, bh, idesc, (ks > 1 || accumulate) ? 1u : 0u);
        else
            ptx::mma_f16(da, ah, bh, idesc, 1u);
        ah += inc;
        bh += inc;
    }
}

__global__ void __launch_bounds__(256, 1) mp_moments_tc_kernel(const double *__restrict__ psi, int n,
                                                               const float *__restrict__ R32, int K,
                                                               const float *__restrict__ Rmax,
                                                               const float *__restrict__ psimax, long long N,
                                                               long long span, double *__restrict__ part,
                                                               int *status, long long timeout_cycles) {
    extern __shared__ uint8_t mt_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(mt_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *Bhi = smem, *Blo = smem + kMtB;
    uint8_t *A0 = smem + 2 * kMtB;  // pair p: hi at A0 + 2p kMtA, lo after it
    uint8_t *raw0 = A0 + (size_t)kMtPairs * 2 * kMtA;  // two raw stages
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int kp0 = blockIdx.y * kMtPairs;
    const int npair = min(kMtPairs, (K + 1) / 2 - kp0);
    if (warp == 0) {
        ptx::tmem_alloc(&tslot, 512);
        ptx::tmem_relinquish();
    }
    if (tid == 0) {
        ptx::mbar_init(&bar, 1);
        ptx::fence_mbar_init();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = tslot;
    int e = 0;
    frexpf(*psimax, &e);
    const float sp = ldexpf(1.f, -e);  // |psi sp| < 1
    float sk[2 * kMtPairs];
#pragma unroll
    for (int q = 0; q < 2 * kMtPairs; ++q) {
        const int k = 2 * kp0 + q;
        int ek = 0;
        if (k < K) frexpf(Rmax[k], &ek);
        sk[q] = (k < K && q < 2 * npair) ? ldexpf(1.f, 14 - ek) : 0.f;  // |R_k sk| < 2^14
    }
    const long long x0 = (long long)blockIdx.x * span;
    const long long x1 = min(N, x0 + span);
    const int nsteps = x1 > x0 ? (int)((x1 - x0 + kMtX - 1) / kMtX) : 0;
    // copies of step t's raw inputs into stage t & 1: psi rows i < n and the
    // pass's weight rows, 16-byte pieces (zero-filled past the range)
    auto issue_raw = [&](int t) {
        uint8_t *dst = raw0 + (size_t)(t & 1) * kMtRaw;
        const long long xs = x0 + (long long)t * kMtX;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int piece = tid + 256 * m, i = piece >> 5, c = piece & 31;  // row i, 2 points per piece
            const long long x = xs + 2 * c;
            const bool ok_ = i < n && x < x1;
            ptx::cp_async16(dst + i * kMtRawRow + 16 * c, ok_ ? (const void *)(psi + (long long)i * N + x) : psi,
                            ok_ ? 16u : 0u);
        }
        if (tid < 2 * kMtPairs * kMtX / 4) {
            const int q = tid >> 4, c = tid & 15;  // weight row q, 4 points per piece
            const int k = 2 * kp0 + q;
            const long long x = xs + 4 * c;
            const bool ok_ = q < 2 * npair && k < K && x < x1;
            ptx::cp_async16(dst + kMtRawPsi + q * (kMtX * 4) + 16 * c,
                            ok_ ? (const void *)(R32 + (long long)k * N + x) : R32, ok_ ? 16u : 0u);
        }
    };
    if (nsteps > 0) issue_raw(0);
    ptx::cp_async_commit();
    uint32_t phase = 0;
    bool ok = true;
    for (int s = 0; s < nsteps && ok; ++s) {
        if (s + 1 < nsteps) issue_raw(s + 1);
        ptx::cp_async_commit();
        ptx::cp_async_wait<1>();  // this thread's copies of step s have landed
        if (s > 0) {
            // the previous step's products have read the tiles
            ok = __syncthreads_and(ptx::mbar_wait_bounded(&bar, phase, timeout_cycles));
            phase ^= 1u;
            if (!ok) break;
            ptx::tc_fence_after();
        } else {
            __syncthreads();
        }
        const uint8_t *rs = raw0 + (size_t)(s & 1) * kMtRaw;
#pragma unroll 1
        for (int r = 0; r < 2; ++r) {
            const int i = tid & 63, g = (tid >> 6) + 4 * r;  // orbital, group of 8 points
            float v[8];
            {
                const double2 *src = reinterpret_cast<const double2 *>(rs + i * kMtRawRow + 64 * g);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const double2 d = src[c];
                    v[2 * c] = f64_to_f32(d.x) * sp;
                    v[2 * c + 1] = f64_to_f32(d.y) * sp;
                }
            }
            mt_split_store(Bhi, Blo, (i >> 3) * kMtGroup + g * 128 + (i & 7) * 16, v);
#pragma unroll
            for (int q = 0; q < 2 * kMtPairs; ++q) {
                if (q >= 2 * npair) break;
                const float4 *wr = reinterpret_cast<const float4 *>(rs + kMtRawPsi + q * (kMtX * 4) + 32 * g);
                const float4 a = wr[0], b = wr[1];
                const float rv[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
                float w[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) w[c] = v[c] * (rv[c] * sk[q]);
                const int row = (q & 1) * 64 + i;
                uint8_t *Ahi = A0 + (size_t)(q >> 1) * 2 * kMtA;
                mt_split_store(Ahi, Ahi + kMtA, (row >> 3) * kMtGroup + g * 128 + (row & 7) * 16, w);
            }
        }
        ptx::fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            ptx::tc_fence_after();
            for (int p = 0; p < npair; ++p) {
                const uint32_t sA = ptx::smem_u32(A0 + (size_t)p * 2 * kMtA);
                mt_issue(tmem + 128 * p, tmem + 128 * p + 64, sA, sA + (uint32_t)kMtA, ptx::smem_u32(Bhi),
                         ptx::smem_u32(Blo), s > 0);
            }
            ptx::mma_commit(&bar);
        }
    }
    ptx::cp_async_wait<0>();
    if (nsteps > 0 && ok) ok = __syncthreads_and(ptx::mbar_wait_bounded(&bar, phase, timeout_cycles));
    if (!ok && tid == 0) atomicExch(status, KX_ERR_TIMEOUT);
    ptx::tc_fence_after();
    if (warp < 4) {
        // lane r of TMEM = A row r = (harmonic 2p + r / 64, orbital r % 64)
        const int row = warp * 32 + lane, t = row >> 6, i = row & 63;
        const uint32_t tl = tmem + ((uint32_t)(32 * warp) << 16);
        const long long nn = (long long)n * n;
        for (int p = 0; p < npair; ++p) {
            const int k = 2 * (kp0 + p) + t;
            const float un = (k < K && sk[2 * p + t] > 0.f) ? 1.f / (sp * sp * sk[2 * p + t]) : 0.f;
            for (int c0 = 0; c0 < 64; c0 += 16) {
                float va[16], vb[16];
                ptx::tmem_ld16x2(tl + 128 * p + c0, tl + 128 * p + 64 + c0, va, vb);
                if (k >= K || i >= n) continue;
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const int j = c0 + c;
                    if (j < n)
                        part[((long long)blockIdx.x * K + k) * nn + (long long)i * n + j] =
                            (nsteps > 0 && ok) ? (double)(va[c] + vb[c]) * (double)un : 0.0;
                }
            }
        }
    }
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, 512);
    }
}

// ---------------------------------------------------------------------------
// Correction on the tensor cores (at most 64 orbitals):
//   T[x][i] = sum_k sum_j (h_k(x) psi_j(x)) C_k[j][i]
// is one product with inner dimension K n: per 128-point tile, for each k the
// A tile (h_k psi)[x][j] (MN-major: points contiguous) and the B tile
// C_k[j][i] (MN-major: orbitals i contiguous) are fp16 hi/lo splits, and the
// products accumulate into one TMEM pair.  Every term carries the same overall
// scale: A_k is scaled by s_psi s_h,k and B_k by t_k with s_h,k t_k = S for
// all k (t_k puts max |C_k| near 2^14, S is the largest common value that
// keeps every |A_k| < 2^14), so T = D / (s_psi S).
// ---------------------------------------------------------------------------
constexpr int kCtM = 128;                 // grid points per tile
constexpr size_t kCtA = 128 * 64 * 2;     // hi (or lo) of A_k: 128 points x 64 orbitals fp16
constexpr size_t kCtB = 64 * 64 * 2;      // hi (or lo) of B_k
constexpr size_t kCtStage = 2 * kCtA + 2 * kCtB;
constexpr int kCtStages = 3;               // B_{k+1} is copied while A_k is built and k-1's products run
constexpr size_t kCtSmem = kCtStages * kCtStage + 1024;

// scale exponents: e_psi from max|psi|, per k the exponents of max|h_k| and max|C_k|
// out: sc[k] = s_psi s_h,k (the A scale), sc[K + k] = t_k, sc[2K] = 1 / (s_psi S)
__global__ void mp_ct_scales_kernel(const float *__restrict__ hmax, const float *__restrict__ cmax,
                                    const float *__restrict__ psimax, int K, float *__restrict__ sc) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    int ep = 0;
    frexpf(*psimax, &ep);  // |psi 2^-ep| < 1
    // t_k = 2^(14 - ec_k); A_k max = hmax_k 2^-ep S / t_k < 2^14  =>  S <= 2^(14 + 14 - ec_k - eh_k)
    int eS = 1 << 20;
    for (int k = 0; k < K; ++k) {
        int eh = 0, ec = 0;
        frexpf(hmax[k], &eh);
        frexpf(cmax[k], &ec);
        if (hmax[k] > 0.f && cmax[k] > 0.f) eS = min(eS, 28 - ec - eh);
    }
    if (eS == (1 << 20)) eS = 0;
    for (int k = 0; k < K; ++k) {
        int ec = 0;
        frexpf(cmax[k], &ec);
        const int et = cmax[k] > 0.f ? 14 - ec : 0;
        sc[K + k] = ldexpf(1.f, et);
        sc[k] = ldexpf(1.f, eS - et - ep);  // s_psi s_h,k
    }
    // every product term carries 2^(eS - ep): A = psi h_k sc[k], B = C_k t_k
    sc[2 * K] = ldexpf(1.f, ep - eS);
}

// max over |C_k| per k (C float64 [K][n][n])
__global__ void mp_cmax_kernel(const double *__restrict__ C, int n, int K, float *__restrict__ cmax) {
    const long long nn = (long long)n * n;
    for (int k = blockIdx.x; k < K; k += gridDim.x) {
        float m = 0.f;
        for (long long e = threadIdx.x; e < nn; e += blockDim.x) m = fmaxf(m, fabsf(f64_to_f32(C[k * nn + e])));
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int *>(cmax + k), __float_as_int(m));
    }
}

// B_k = C_k t_k split into fp16 hi/lo, MN-major core matrices (i contiguous):
// element (j, i) at (j/8) 1024 + (i/8) 128 + (j%8) 16 + (i%8) 2, hi block then lo block per k.
__global__ void mp_ct_bsplit_kernel(const double *__restrict__ C, int n, int K, const float *__restrict__ sc,
                                    __half *__restrict__ Bs) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;  // over K x 64 x 64
    if (e >= (long long)K * 4096) return;
    const int k = (int)(e >> 12), j = (int)((e >> 6) & 63), i = (int)(e & 63);
    const float v = (i < n && j < n) ? f64_to_f32(C[((long long)k * n + j) * n + i]) * sc[K + k] : 0.f;
    const __half h = __float2half_rn(v);
    const __half l = __float2half_rn(v - __half2float(h));
    const int off = (j >> 3) * 512 + (i >> 3) * 64 + (j & 7) * 8 + (i & 7);  // in halves
    Bs[(size_t)k * 8192 + off] = h;
    Bs[(size_t)k * 8192 + 4096 + off] = l;
}

__device__ __forceinline__ void ct_issue(uint32_t da, uint32_t db, uint32_t a_hi, uint32_t a_lo, uint32_t b_hi,
                                         uint32_t b_lo, bool accumulate) {
    const uint32_t idesc = ptx::idesc_f16(128, 64, 1, 1);  // A and B MN-major
    // A: M-core (8 points) stride 128, K-group (8 orbitals) stride 16 x 128; B: N-core 128, K-group 1024
    const uint64_t ah0 = ptx::sdesc(a_hi, 2048, 128), al0 = ptx::sdesc(a_lo, 2048, 128);
    const uint64_t bh0 = ptx::sdesc(b_hi, 1024, 128), bl0 = ptx::sdesc(b_lo, 1024, 128);
    const uint64_t a_inc = 4096 >> 4, b_inc = 2048 >> 4;  // one k-step = 16 orbitals
    uint64_t ah = ah0, al = al0, bh = bh0, bl = bl0;
    for (int ks = 0; ks < 4; ++ks) {
        ptx::mma_f16(da, ah, bl, idesc, (ks > 0 || accumulate) ? 1u : 0u);
        ptx::mma_f16(da, al, bh, idesc, 1u);
        ah += a_inc;
        al += a_inc;
        bh += b_inc;
        bl += b_inc;
    }
    ah = ah0;
    bh = bh0;
    for (int ks = 0; ks < 4; ++ks) {
        if (ks & 1)
            ptx::mma_f16(db, ah, bh, idesc, (ks > 1 || accumulate) ? 1u : 0u);
        else
            ptx::mma_f16(da, ah, bh, idesc, 1u);
        ah += a_inc;
        bh += b_inc;
    }
}

// acc_i(x) = T[x][i] (the float32 accumulator of the pair loop starts from the
// correction); e_part[CTA] = sum over its tiles of g_i psi_i(x) T[x][i].
// Persistent: CTA walks the tiles blockIdx.x, + gridDim.x, ...; for each tile
// the K harmonics go through a ring of three shared stages (A_k built by all
// threads; B_k copied from the pre-split array one harmonic ahead, so that the
// copy's latency overlaps the build of A_{k-1}), one thread issuing each k's
// products; all eight warps then read T (two per TMEM lane quadrant).
__global__ void __launch_bounds__(256, 1) mp_combine_tc_kernel(const double *__restrict__ psi, int n,
                                                               const __half *__restrict__ Bs,
                                                               const float *__restrict__ H, int K,
                                                               const float *__restrict__ sc,
                                                               const double *__restrict__ occ, long long N,
                                                               float *__restrict__ acc, double *__restrict__ e_part,
                                                               int *status, long long timeout_cycles) {
    extern __shared__ uint8_t ct_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(ct_raw) + 1023) & ~uintptr_t(1023));
    __shared__ uint64_t bar[kCtStages];
    __shared__ uint32_t tslot;
    __shared__ double red[8];
    __shared__ volatile int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        ptx::tmem_alloc(&tslot, 128);
        ptx::tmem_relinquish();
    }
    if (tid == 0) {
        for (int b = 0; b < kCtStages; ++b) ptx::mbar_init(&bar[b], 1);
        ptx::fence_mbar_init();
        s_abort = 0;
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = tslot;
    const float unscale = sc[2 * K];
    const long long ntiles = (N + kCtM - 1) / kCtM;
    // producer tasks of this thread: point group mg (8 points) and orbitals
    // j = 8 (jh + 2u) + jl, u < 4: eight neighbouring lanes fill one 128-byte
    // core matrix (the eight orbitals of a K group at one point group)
    const int jl = tid & 7, mg = (tid >> 3) & 15, jh = tid >> 7;
    uint32_t uses[kCtStages] = {0u, 0u, 0u};  // commits issued per stage
    uint32_t waited[kCtStages] = {0u, 0u, 0u};
    // B_k (2 x 8 KB of the pre-split array) into stage b, one cp.async group
    auto copy_b = [&](int k, int b) {
        const uint4 *src = reinterpret_cast<const uint4 *>(Bs + (size_t)k * 8192);
        uint8_t *dst = smem + b * kCtStage + 2 * kCtA;
#pragma unroll
        for (int q = 0; q < 4; ++q) ptx::cp_async16(dst + 16 * (tid + 256 * q), src + tid + 256 * q, 16u);
        ptx::cp_async_commit();
    };
    // the products that last read stage b are done (each thread waits by itself;
    // a timeout is acted on after the next block barrier)
    auto free_stage = [&](int b) {
        if (uses[b] > waited[b]) {
            if (!ptx::mbar_wait_bounded(&bar[b], waited[b] & 1u, timeout_cycles)) s_abort = 1;
            ++waited[b];
            ptx::tc_fence_after();
        }
    };
    bool ok = true;
    double e_acc = 0.0;
    for (long long tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x) {
        const long long xb = tile * kCtM + 8 * mg;
        float pv[4][8];  // psi_j at the thread's 8 points, scaled later per k
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = 8 * (jh + 2 * u) + jl;
            if (j < n && xb < N) {
                const double2 *src = reinterpret_cast<const double2 *>(psi + (long long)j * N + xb);
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const double2 d = __ldg(src + c);
                    pv[u][2 * c] = f64_to_f32(d.x);
                    pv[u][2 * c + 1] = f64_to_f32(d.y);
                }
            } else {
#pragma unroll
                for (int c = 0; c < 8; ++c) pv[u][c] = 0.f;
            }
        }
        // h_k at the thread's 8 points, fetched one harmonic ahead
        float4 hn0 = make_float4(0.f, 0.f, 0.f, 0.f), hn1 = hn0;
        if (xb < N) {
            const float4 *hs = reinterpret_cast<const float4 *>(H + xb);
            hn0 = __ldg(hs);
            hn1 = __ldg(hs + 1);
        }
        // every stage is free at a tile's start (the previous tile's products were
        // waited for); stage k % 3 is freed before B_k is copied into it
        free_stage(0);
        copy_b(0, 0);
        for (int k = 0; k < K && ok; ++k) {
            const int b = k % kCtStages;
            uint8_t *st = smem + b * kCtStage;
            if (k + 1 < K) {
                const int bn = (k + 1) % kCtStages;
                free_stage(bn);
                copy_b(k + 1, bn);
            }
            // A_k: (h_k psi_j) at the 8 points, scaled by sc[k]
            const float sk = sc[k];
            const float hv[8] = {hn0.x * sk, hn0.y * sk, hn0.z * sk, hn0.w * sk,
                                 hn1.x * sk, hn1.y * sk, hn1.z * sk, hn1.w * sk};
            if (k + 1 < K && xb < N) {
                const float4 *hs = reinterpret_cast<const float4 *>(H + (long long)(k + 1) * N + xb);
                hn0 = __ldg(hs);
                hn1 = __ldg(hs + 1);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int j = 8 * (jh + 2 * u) + jl;
                float w[8];
#pragma unroll
                for (int c = 0; c < 8; ++c) w[c] = pv[u][c] * hv[c];
                mt_split_store(st, st + kCtA, mg * 128 + (j >> 3) * 2048 + (j & 7) * 16, w);
            }
            if (k + 1 < K)
                ptx::cp_async_wait<1>();  // B_k has landed; B_{k+1} may still be copying
            else
                ptx::cp_async_wait<0>();
            ptx::fence_proxy_async_smem();
            __syncthreads();
            if (s_abort) {
                ok = false;
                break;
            }
            if (tid == 0) {
                ptx::tc_fence_after();
                const uint32_t sa = ptx::smem_u32(st), sb = sa + 2 * (uint32_t)kCtA;
                ct_issue(tmem, tmem + 64, sa, sa + (uint32_t)kCtA, sb, sb + (uint32_t)kCtB, k > 0);
                ptx::mma_commit(&bar[b]);
            }
            ++uses[b];
        }
        // the tile's last products are done: read T, update Vx psi, energy
        for (int b = 0; b < kCtStages && ok; ++b)
            while (ok && uses[b] > waited[b]) {
                ok = __syncthreads_and(ptx::mbar_wait_bounded(&bar[b], waited[b] & 1u, timeout_cycles));
                ++waited[b];
            }
        if (!ok) break;
        ptx::tc_fence_after();
        {
            const int q = warp & 3, hcol = warp >> 2;  // lane quadrant, orbital half
            const int m = q * 32 + lane;
            const long long x = tile * kCtM + m;
            const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);
            float ef = 0.f;
            for (int c0 = 32 * hcol; c0 < 32 * hcol + 32; c0 += 16) {
                float va[16], vb[16];
                ptx::tmem_ld16x2(tl + c0, tl + 64 + c0, va, vb);
                if (x >= N) continue;
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const int i = c0 + c;
                    if (i >= n) continue;
                    const float t = (va[c] + vb[c]) * unscale;
                    acc[(long long)i * N + x] = t;
                    const float gi = occ ? f64_to_f32(occ[i]) : 1.f;
                    ef = fmaf(gi * f64_to_f32(__ldg(psi + (long long)i * N + x)), t, ef);
                }
            }
            e_acc += (double)ef;
        }
        ptx::tc_fence_before();
        __syncthreads();  // TMEM read before the next tile's first product overwrites it
        ptx::tc_fence_after();
    }
    if (!ok && tid == 0) atomicExch(status, KX_ERR_TIMEOUT);
    // products still in flight after an early exit finish before TMEM is released
    for (int b = 0; b < kCtStages; ++b)
        for (; uses[b] > waited[b]; ++waited[b]) ptx::mbar_wait_bounded(&bar[b], waited[b] & 1u, timeout_cycles);
    for (int o = 16; o > 0; o >>= 1) e_acc += __shfl_xor_sync(0xffffffffu, e_acc, o);
    if (lane == 0) red[warp] = e_acc;
    ptx::tc_fence_before();
    __syncthreads();
    if (tid == 0) {
        double sum = 0.0;
        for (int w = 0; w < 8; ++w) sum += red[w];
        e_part[blockIdx.x] = sum;
    }
    if (warp == 0) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, 128);
    }
}

// Q[e] = scale sum_c part[c][e] in a fixed order.
__global__ void mp_reduce_kernel(const double *__restrict__ part, int n_part, long long n_e, double scale,
                                 double *__restrict__ Q) {
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_e) return;
    double s = 0.0;
    for (int c = 0; c < n_part; ++c) s += part[(long long)c * n_e + e];
    Q[e] = scale * s;
}

__device__ __forceinline__ float as_f32(float v) { return v; }
__device__ __forceinline__ float as_f32(double v) { return f64_to_f32(v); }

// max |a| over n values into *out (float bits, non-negative: integer max is exact and order-free)
template <typename T>
__global__ void absmax_kernel(const T *__restrict__ a, long long n, float *__restrict__ out) {
    float m = 0.f;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(as_f32(a[i])));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(reinterpret_cast<int *>(out), __float_as_int(m));
}

// ex += scale * sum of the partials, in index order (one thread: deterministic).
__global__ void mp_energy_add_kernel(const double *__restrict__ part, long long count, double scale,
                                     double *__restrict__ ex) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    double s = 0.0;
    for (long long i = 0; i < count; ++i) s += part[i];
    *ex += scale * s;
}

// ex += -1/2 sum_{i,j} g_i g_j mask(i,j) sum_k Q_k(ij) P_k(ij); fixed-order block reduction.
__global__ void mp_energy_qp_kernel(const double *__restrict__ Q, const double *__restrict__ P,
                                    const unsigned char *__restrict__ mask, const double *__restrict__ occ, int n,
                                    int K, double *__restrict__ ex) {
    __shared__ double red[256];
    const long long nn = (long long)n * n;
    double s = 0.0;
    for (long long e = threadIdx.x; e < nn; e += blockDim.x) {
        const int i = (int)(e / n), j = (int)(e % n);
        if (!mask[e]) continue;
        double t = 0.0;
        for (int k = 0; k < K; ++k) t += Q[(long long)k * nn + e] * P[(long long)k * nn + e];
        s += (occ ? occ[i] * occ[j] : 1.0) * t;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int st = blockDim.x / 2; st > 0; st >>= 1) {
        if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
        __syncthreads();
    }
    if (threadIdx.x == 0) *ex += -0.5 * red[0];
}

std::vector<double> centred_weights(int order) {
    const int m = order / 2;
    std::vector<double> w(m + 1, 0.0);
    for (int p = 1; p <= m; ++p) w[0] -= 2.0 / (double(p) * p);
    double fm = 1.0;
    for (int i = 2; i <= m; ++i) fm *= i;
    for (int p = 1; p <= m; ++p) {
        double fmp = 1.0, fpp = 1.0;
        for (int i = 2; i <= m - p; ++i) fmp *= i;
        for (int i = 2; i <= m + p; ++i) fpp *= i;
        w[p] = 2.0 * ((p % 2) ? 1.0 : -1.0) * fm * fm / (double(p) * p * fmp * fpp);
    }
    return w;
}

// Tensor-core moments: one grid-point range per SM, each range split over the
// harmonic pairs in groups of kMtPairs.
int moments_tc_split(const kx_plan *p) { return p->num_sms; }

constexpr size_t kMpSmall = 4096;  // psimax (1 float), cmax (<= 81), scales (<= 163)

size_t mp_scratch_bytes(const kx_plan *p, int n, int K) {
    const long long N = (long long)p->N;
    const size_t kn2 = (size_t)K * n * n;
    const size_t tiles = (size_t)((N + kMcX - 1) / kMcX) * ((n + 63) / 64);
    const size_t part64 = (size_t)((N + 255) / 256) * n;
    const size_t part_tc = n <= 64 ? (size_t)moments_tc_split(p) * kn2 : 0;
    // Q and P hold up to 2K matrices (the gradient's symmetric correction), Bs 2K tiles
    return kMpSmall + sizeof(double) * (4 * kn2 + std::max(std::max(tiles, part64), part_tc)) + 256 +
           (size_t)2 * K * 16384;
}

// Layout of the plan's multipole scratch for n orbitals: small float arrays
// (max |psi|, max |C_k|, scales), Q, then P or C, the partial sums, the
// pre-split B tiles.
struct MpScratch {
    float *psimax, *cmax, *sc;
    double *Q, *P, *part;
    __half *Bs;
};

MpScratch mp_layout(const kx_plan *p, int n) {
    const size_t kn2 = (size_t)p->mp_K * n * n;
    const long long N = (long long)p->N;
    const size_t tiles = (size_t)((N + kMcX - 1) / kMcX) * ((n + 63) / 64);
    const size_t part64 = (size_t)((N + 255) / 256) * n;
    const size_t part_tc = n <= 64 ? (size_t)moments_tc_split(p) * kn2 : 0;
    uint8_t *b = (uint8_t *)p->mp_scratch.ptr;
    MpScratch m;
    m.psimax = reinterpret_cast<float *>(b);
    m.cmax = reinterpret_cast<float *>(b + 256);
    m.sc = reinterpret_cast<float *>(b + 1024);
    m.Q = reinterpret_cast<double *>(b + kMpSmall);
    m.P = m.Q + 2 * kn2;
    m.part = m.P + 2 * kn2;
    const uintptr_t bs = reinterpret_cast<uintptr_t>(m.part + std::max(std::max(tiles, part64), part_tc));
    m.Bs = reinterpret_cast<__half *>((bs + 255) & ~uintptr_t(255));  // 16-byte copies need alignment
    return m;
}

// Q[k] = dV sum_x W_k psi_i psi_j for k < K (weights W: K x N).  Tensor cores for
// up to 64 orbitals on tensor-core plans (W32 and its per-field maxima), else one
// weighted projection per k.
int weighted_moments(kx_plan *p, int n, const double *psi, const double *W64, const float *W32, const float *Wmax,
                     double *Q, double *part, float *psimax, cudaStream_t s) {
    const int K = p->mp_K;
    const long long N = (long long)p->N;
    const size_t nn = (size_t)n * n;
    // 16-byte loads of 8 grid points: N % 8 == 0 (so rows and steps stay aligned) and aligned bases
    const bool tc = p->precision != KX_FP64 && n <= 64 && N % 8 == 0 &&
                    ((reinterpret_cast<uintptr_t>(psi) | reinterpret_cast<uintptr_t>(W32)) & 15) == 0;
    if (tc) {
        if (int rc = prof_begin(p, PK_MP, s)) return rc;
        KX_CUDA_TRY(cudaMemsetAsync(psimax, 0, sizeof(float), s));
        absmax_kernel<double><<<4 * p->num_sms, 256, 0, s>>>(psi, (long long)n * N, psimax);
        KX_LAUNCH_CHECK("absmax_kernel launch");
        const int n_split = moments_tc_split(p);
        const long long span = ((N + n_split - 1) / n_split + kMtX - 1) / kMtX * kMtX;
        const dim3 grid(n_split, ((K + 1) / 2 + kMtPairs - 1) / kMtPairs);
        KX_CUDA_TRY(cudaFuncSetAttribute(mp_moments_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kMtSmem));
        mp_moments_tc_kernel<<<grid, 256, kMtSmem, s>>>(psi, n, W32, K, Wmax, psimax, N, span, part, p->d_status,
                                                         4000000000LL);
        KX_LAUNCH_CHECK("mp_moments_tc_kernel launch");
        const long long ne = (long long)K * nn;
        mp_reduce_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, s>>>(part, n_split, ne, p->dV, Q);
        KX_LAUNCH_CHECK("mp_reduce_kernel launch");
        return prof_end(p, s);
    }
    const bool f64 = p->precision == KX_FP64;
    for (int k = 0; k < K; ++k)
        if (int rc = grid_projection(p, psi, n, psi, n, f64 ? W64 + (size_t)k * N : nullptr,
                                     f64 ? nullptr : W32 + (size_t)k * N, p->dV, Q + (size_t)k * nn, s, PK_MP))
            return rc;
    return KX_OK;
}

}  // namespace

void mp_free(kx_plan *p) {
    cudaFree(p->d_mpR);    // R and h share one allocation (h = R + K N)
    cudaFree(p->d_mpR32);
    cudaFree(p->d_mpMax);
    p->d_mpMax = nullptr;
    cudaFree(p->mp_scratch.ptr);
    p->d_mpR = p->d_mpH = nullptr;
    p->d_mpR32 = p->d_mpH32 = nullptr;
    p->mp_scratch = Workspace{};
    p->mp_lmax = -1;
    p->mp_K = 0;
    ++p->config_version;
}

int mp_set(kx_plan *p, int l_max) {
    if (l_max < 0) {
        cudaError_t e = cudaDeviceSynchronize();
        mp_free(p);
        return e == cudaSuccess ? KX_OK : cuda_error(e, "kx_plan_set_multipole");
    }
    if (l_max > kMpMaxL) return set_error(KX_ERR_ARG, "kx_plan_set_multipole: l_max must be in -1..8");
    if (p->kind != 0 || p->bc[0] != 0 || p->bc[1] != 0 || p->bc[2] != 0)
        return set_error(KX_ERR_UNSUPPORTED,
                         "kx_plan_set_multipole: needs Dirichlet boundaries on all axes and the unscreened kernel");
    if (p->fd_order / 2 > kMaxHalf) return set_error(KX_ERR_UNSUPPORTED, "kx_plan_set_multipole: FD order too high");
    KX_CUDA_TRY(cudaDeviceSynchronize());
    mp_free(p);
    const int K = (l_max + 1) * (l_max + 1);
    const long long N = (long long)p->N;
    MpGeom G{};
    for (int a = 0; a < 3; ++a) {
        G.n[a] = p->n[a];
        G.h[a] = p->h[a];
        G.c[a] = (p->n[a] + 1) * p->h[a] / 2.0;
    }
    G.m = p->fd_order / 2;
    const std::vector<double> w = centred_weights(p->fd_order);
    for (int d = 0; d <= G.m; ++d) G.w[d] = w[d];
    G.L = l_max;
    G.K = K;
    const size_t fld = sizeof(double) * (size_t)K * N;
    double *Gk = nullptr;
    // [R_0 .. R_{K-1} | h_0 .. h_{K-1}] in one allocation per precision, so that
    // the gradient's correction walks all 2K fields in order
    cudaError_t e = cudaMalloc(&p->d_mpR, 2 * fld);
    if (e == cudaSuccess) e = cudaMalloc(&p->d_mpR32, fld);
    if (e == cudaSuccess) {
        p->d_mpH = p->d_mpR + (size_t)K * N;
        p->d_mpH32 = p->d_mpR32 + (size_t)K * N;
    }
    if (e == cudaSuccess) e = cudaMalloc(&p->d_mpMax, sizeof(float) * 2 * K);
    if (e == cudaSuccess) e = cudaMalloc(&Gk, fld);
    if (e != cudaSuccess) {
        cudaFree(Gk);
        mp_free(p);
        return cuda_error(e, "kx_plan_set_multipole cudaMalloc");
    }
    mp_fields_kernel<<<(unsigned)((N + 127) / 128), 128>>>(G, N, p->d_mpR, Gk);
    e = cudaGetLastError();
    int rc = e == cudaSuccess ? KX_OK : cuda_error(e, "mp_fields_kernel launch");
    // h_k = f(L) g_k with the float64 solver (set-up, once per plan)
    if (!rc) rc = fp64_apply_fL(p, K, Gk, p->d_mpH, nullptr);
    if (!rc) {
        to_f32_kernel<<<1024, 256>>>(p->d_mpR, p->d_mpR32, (long long)K * N);
        to_f32_kernel<<<1024, 256>>>(p->d_mpH, p->d_mpH32, (long long)K * N);
        // per-field maxima (R_k then h_k) for the tensor-core moments' scales
        cudaMemset(p->d_mpMax, 0, sizeof(float) * 2 * K);
        for (int k = 0; k < K; ++k) {
            absmax_kernel<float><<<256, 256>>>(p->d_mpR32 + (size_t)k * N, N, p->d_mpMax + k);
            absmax_kernel<float><<<256, 256>>>(p->d_mpH32 + (size_t)k * N, N, p->d_mpMax + K + k);
        }
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) rc = cuda_error(e, "kx_plan_set_multipole set-up");
    }
    cudaFree(Gk);
    if (rc) {
        mp_free(p);
        return rc;
    }
    p->mp_lmax = l_max;
    p->mp_K = K;
    ++p->config_version;
    return KX_OK;
}

int mp_reserve_scratch(kx_plan *p, int n_orb) {
    const size_t need = mp_scratch_bytes(p, n_orb, p->mp_K);
    if (p->mp_scratch.bytes < need) {
        cudaFree(p->mp_scratch.ptr);
        p->mp_scratch = Workspace{};
        ++p->config_version;
        cudaError_t e = cudaMalloc(&p->mp_scratch.ptr, need);
        if (e != cudaSuccess) return cuda_error(e, "multipole scratch cudaMalloc");
        p->mp_scratch.bytes = need;
    }
    return KX_OK;
}

int mp_reserve(kx_plan *p, int n_orb) {
    if (p->mp_lmax < 0) return KX_OK;
    const size_t need = mp_scratch_bytes(p, n_orb, p->mp_K);
    if (p->mp_scratch.bytes < need) {
        cudaFree(p->mp_scratch.ptr);
        p->mp_scratch = Workspace{};
        ++p->config_version;
        cudaError_t e = cudaMalloc(&p->mp_scratch.ptr, need);
        if (e != cudaSuccess) return cuda_error(e, "multipole scratch cudaMalloc");
        p->mp_scratch.bytes = need;
    }
    return ensure_workspace(p, grid_projection_bytes(p, std::max(n_orb, p->mp_K), std::max(n_orb, p->mp_K)));
}

int mp_correct_vx(kx_plan *p, int n_orb, const double *psi, const double *occ, double *vx, double *ex,
                  bool energy_only, cudaStream_t s) {
    if (p->precision != KX_FP64 && n_orb > 256)
        return set_error(KX_ERR_UNSUPPORTED, "multipole boundary values: at most 256 orbitals on tensor-core plans");
    int rc = mp_reserve(p, n_orb);
    if (rc) return rc;
    const int K = p->mp_K, n = n_orb;
    const long long N = (long long)p->N;
    const size_t nn = (size_t)n * n;
    const bool f64 = p->precision == KX_FP64;
    const MpScratch m = mp_layout(p, n);
    double *Q = m.Q;
    double *P = m.P;  // energy-only: projections on h_k; otherwise C
    double *part = m.part;
    float *psimax = m.psimax;
    const unsigned char *mask = p->d_pair_mask;
    // moments Q_k(ij) = dV sum_x R_k psi_i psi_j
    if ((rc = weighted_moments(p, n, psi, p->d_mpR, p->d_mpR32, p->d_mpMax, Q, part, psimax, s))) return rc;
    if (energy_only) {
        if ((rc = weighted_moments(p, n, psi, p->d_mpH, p->d_mpH32, p->d_mpMax + K, P, part, psimax, s))) return rc;
        if (ex) {
            if ((rc = prof_begin(p, PK_MP, s))) return rc;
            mp_energy_qp_kernel<<<1, 256, 0, s>>>(Q, P, mask, occ, n, K, ex);
            KX_LAUNCH_CHECK("mp_energy_qp_kernel launch");
            if ((rc = prof_end(p, s))) return rc;
        }
        return KX_OK;
    }
    // gradient mode: fields [R | h] with coefficients 1/2 [P | Q] (P_k = dV <h_k, rho>)
    const bool sym = p->mp_grad;
    const int Kc = sym ? 2 * K : K;
    if (sym) {
        if ((rc = weighted_moments(p, n, psi, p->d_mpH, p->d_mpH32, p->d_mpMax + K, P, part, psimax, s))) return rc;
        KX_CUDA_TRY(cudaMemcpyAsync(Q + (size_t)K * nn, Q, sizeof(double) * K * nn, cudaMemcpyDeviceToDevice, s));
        KX_CUDA_TRY(cudaMemcpyAsync(Q, P, sizeof(double) * K * nn, cudaMemcpyDeviceToDevice, s));
    }
    const double cscale = sym ? 0.5 : 1.0;
    const unsigned cb = (unsigned)((nn * Kc + 255) / 256);
    if ((rc = prof_begin(p, PK_MP, s))) return rc;
    if (f64) {
        double *C = P;
        mp_coef_kernel<double><<<cb, 256, 0, s>>>(Q, mask, occ, n, Kc, cscale, C);
        KX_LAUNCH_CHECK("mp_coef_kernel launch");
        const dim3 grid((unsigned)((N + 255) / 256), (unsigned)n);
        mp_combine64_kernel<<<grid, 256, 0, s>>>(psi, n, C, sym ? p->d_mpR : p->d_mpH, Kc, occ, N, vx, part);
        KX_LAUNCH_CHECK("mp_combine64_kernel launch");
        if (ex) {
            mp_energy_add_kernel<<<1, 1, 0, s>>>(part, (long long)grid.x * grid.y, -0.5 * p->dV, ex);
            KX_LAUNCH_CHECK("mp_energy_add_kernel launch");
        }
        return prof_end(p, s);
    }
    float *C = reinterpret_cast<float *>(P);
    mp_coef_kernel<float><<<cb, 256, 0, s>>>(Q, mask, occ, n, Kc, cscale, C);
    KX_LAUNCH_CHECK("mp_coef_kernel launch");
    const dim3 grid((unsigned)((N + kMcX - 1) / kMcX), (unsigned)((n + 63) / 64));
    const size_t smem = sizeof(float) * (size_t)n * (kMcX + 64);
    KX_CUDA_TRY(cudaFuncSetAttribute(mp_combine32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    mp_combine32_kernel<<<grid, 256, smem, s>>>(psi, n, C, sym ? p->d_mpR32 : p->d_mpH32, Kc, occ, N, vx, part);
    KX_LAUNCH_CHECK("mp_combine32_kernel launch");
    if (ex) {
        mp_energy_add_kernel<<<1, 1, 0, s>>>(part, (long long)grid.x * grid.y, -0.5 * p->dV, ex);
        KX_LAUNCH_CHECK("mp_energy_add_kernel launch");
    }
    return prof_end(p, s);
}

bool mp_tc_eligible(const kx_plan *p, int n_orb, const double *psi) {
    return p->mp_lmax >= 0 && p->precision != KX_FP64 && n_orb <= 64 && p->N % 8 == 0 &&
           (reinterpret_cast<uintptr_t>(psi) & 15) == 0;
}

int mp_correct_into_acc(kx_plan *p, int n_orb, const double *psi, const double *occ, float *acc, double *ex,
                        cudaStream_t s) {
    int rc = mp_reserve_scratch(p, n_orb);
    if (rc) return rc;
    const int K = p->mp_K, n = n_orb;
    const long long N = (long long)p->N;
    const size_t nn = (size_t)n * n;
    const MpScratch m = mp_layout(p, n);
    double *Q = m.Q, *C = m.P, *part = m.part;
    float *psimax = m.psimax, *cmax = m.cmax, *sc = m.sc;
    __half *Bs = m.Bs;
    // gradient mode: fields [R | h] with coefficients 1/2 [P | Q] (P_k = dV <h_k, rho>)
    const bool sym = p->mp_grad;
    const int Kc = sym ? 2 * K : K;
    double *Qr = sym ? Q + (size_t)K * nn : Q;
    if (sym && (rc = weighted_moments(p, n, psi, p->d_mpH, p->d_mpH32, p->d_mpMax + K, Q, part, psimax, s)))
        return rc;
    if ((rc = weighted_moments(p, n, psi, p->d_mpR, p->d_mpR32, p->d_mpMax, Qr, part, psimax, s))) return rc;
    if ((rc = prof_begin(p, PK_MP, s))) return rc;
    const unsigned cb = (unsigned)((nn * Kc + 255) / 256);
    mp_coef_kernel<double><<<cb, 256, 0, s>>>(Q, p->d_pair_mask, occ, n, Kc, sym ? 0.5 : 1.0, C);
    KX_LAUNCH_CHECK("mp_coef_kernel launch");
    KX_CUDA_TRY(cudaMemsetAsync(cmax, 0, sizeof(float) * Kc, s));
    mp_cmax_kernel<<<Kc, 256, 0, s>>>(C, n, Kc, cmax);
    KX_LAUNCH_CHECK("mp_cmax_kernel launch");
    // field maxima in the same order as the fields: [R | h] or h alone
    mp_ct_scales_kernel<<<1, 1, 0, s>>>(sym ? p->d_mpMax : p->d_mpMax + K, cmax, psimax, Kc, sc);
    KX_LAUNCH_CHECK("mp_ct_scales_kernel launch");
    mp_ct_bsplit_kernel<<<(unsigned)(((long long)Kc * 4096 + 255) / 256), 256, 0, s>>>(C, n, Kc, sc, Bs);
    KX_LAUNCH_CHECK("mp_ct_bsplit_kernel launch");
    const int grid = (int)std::min<long long>((N + kCtM - 1) / kCtM, p->num_sms);
    KX_CUDA_TRY(cudaFuncSetAttribute(mp_combine_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCtSmem));
    mp_combine_tc_kernel<<<grid, 256, kCtSmem, s>>>(psi, n, Bs, sym ? p->d_mpR32 : p->d_mpH32, Kc, sc, occ, N, acc,
                                                     part, p->d_status, 4000000000LL);
    KX_LAUNCH_CHECK("mp_combine_tc_kernel launch");
    if (ex) {
        mp_energy_add_kernel<<<1, 1, 0, s>>>(part, grid, -0.5 * p->dV, ex);
        KX_LAUNCH_CHECK("mp_energy_add_kernel launch");
    }
    p->mp_applied = true;
    return prof_end(p, s);
}

int mp_correct_apply(kx_plan *p, int n_rhs, const double *b, double *x, cudaStream_t s) {
    const int K = p->mp_K;
    const size_t need = sizeof(double) * (size_t)K * n_rhs + 256;
    if (p->mp_scratch.bytes < need) {
        cudaFree(p->mp_scratch.ptr);
        p->mp_scratch = Workspace{};
        ++p->config_version;
        cudaError_t e = cudaMalloc(&p->mp_scratch.ptr, need);
        if (e != cudaSuccess) return cuda_error(e, "multipole scratch cudaMalloc");
        p->mp_scratch.bytes = need;
    }
    double *Cb = (double *)p->mp_scratch.ptr;  // [K][n_rhs]: dV sum_x R_k b_r
    int rc = grid_projection(p, p->d_mpR, K, b, n_rhs, nullptr, nullptr, p->dV, Cb, s, PK_MP);
    if (rc) return rc;
    return grid_combination(p, p->d_mpH, K, Cb, n_rhs, 1.0, true, x, s, PK_MP);
}

}  // namespace kx
