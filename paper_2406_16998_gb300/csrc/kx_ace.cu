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
#include "kx_tc_ptx.cuh"
#include "kx_conv.cuh"

#include <algorithm>
#include <cstdint>

namespace kx {
namespace {

constexpr int kG = 32;  // gram tile

// part[s][a][b] = sum over slab s of grid points of psi_a(x) W_b(x) w(x)   (a < na, b < nb; w nullable)
__global__ void gram_kernel(const double *__restrict__ psi, int na, const double *__restrict__ W, int nb,
                            const double *__restrict__ w, long long N, long long slab, double *__restrict__ part) {
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
            Ws[r][tx] = (b < nb && x < x1) ? W[(long long)b * N + x] * (w ? w[x] : 1.0) : 0.0;
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

// xi_b(x) = (accumulate ? xi_b(x) : 0) + sgn sum_k W_k(x) Rinv[k][b]   (k < na, b < nb; Rinv row-major na x nb)
__global__ void xi_kernel(const double *__restrict__ W, const double *__restrict__ Rinv, int na, int nb, long long N,
                          double sgn, bool accumulate, double *__restrict__ xi) {
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
            if (b < nb) {
                double *o = xi + (long long)b * N + x;
                *o = (accumulate ? *o : 0.0) + sgn * acc[u];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// float32-product forms of the two grid-sized products
// ---------------------------------------------------------------------------
constexpr int kPT = 64;   // projection tile: 64 a x 64 b per CTA
constexpr int kPX = 32;   // grid points per pipeline step
constexpr int kPBlk = 8;  // steps summed in float32 before the compensated accumulation (256 points)
constexpr int kPStages = 2;
// dynamic shared memory of proj32_kernel (82 KB, two CTAs per SM): raw float64
// stages of both operands, then their float32 copies (rows padded by 4 floats
// for conflict-free float4 reads)
constexpr size_t kProjRawBytes = (size_t)kPStages * 2 * kPT * kPX * sizeof(double);
constexpr size_t kProjSmem = kProjRawBytes + 2 * (size_t)kPT * (kPX + 4) * sizeof(float);

// Issues the asynchronous copies of grid points [xb, xb + kPX) of rows
// r0..r0+63 of M (nr rows in all, stride N) into raw[64][kPX]; points at or
// past xe and rows past nr are zero-filled.  VEC2: 16-byte pieces (N even,
// xb even), else 8-byte pieces.
template <bool VEC2>
__device__ __forceinline__ void proj_issue(const double *__restrict__ M, int nr, int r0, long long N, long long xb,
                                           long long xe, double *raw, int tid) {
    constexpr int per_row = VEC2 ? kPX / 2 : kPX;
#pragma unroll
    for (int m = 0; m < kPT * per_row / 256; ++m) {
        const int piece = tid + 256 * m;
        const int r = piece / per_row, c = (piece % per_row) * (VEC2 ? 2 : 1);
        const long long x = xb + c;
        long long nbytes = (r0 + r < nr) ? (xe - x) * 8 : 0;
        nbytes = nbytes < 0 ? 0 : (nbytes > (VEC2 ? 16 : 8) ? (VEC2 ? 16 : 8) : nbytes);
        const double *src = nbytes > 0 ? M + (long long)(r0 + r) * N + x : M;
        if (VEC2)
            ptx::cp_async16(raw + r * kPX + c, src, (uint32_t)nbytes);
        else
            ptx::cp_async8(raw + r * kPX + c, src, (uint32_t)nbytes);
    }
}

// part[blockIdx.x][a][b] = sum over the CTA's grid points [x0, x0 + span) of
// A_a(x) B_b(x) for its 64 x 64 tile (blockIdx.y, blockIdx.z); two CTAs per SM.
// The float64 inputs of step k+1 are copied into shared memory (cp.async)
// while step k is converted to float32 and multiplied, so the SM always has a
// step's loads in flight.  Thread (tx, ty) of a 16 x 16 layout owns
// a = a0 + ty + 16 i, b = b0 + tx + 16 j (i, j < 4): per four grid points it
// reads four a-rows (two distinct per warp, broadcast) and four b-rows as
// float4 and does 64 FMAs.  Each block of 256 points is summed in float32 and
// added to a float32 pair (sum and rounding error), so the CTA's total keeps
// about 48 bits.  w (nullable) weights every grid point of B; a tile whose A
// and B rows are the same rows of one array copies them once.
template <bool VEC2>
__global__ void __launch_bounds__(256, 2) proj32_kernel(const double *__restrict__ A, int na,
                                                        const double *__restrict__ B, int nb,
                                                        const float *__restrict__ w, long long N, long long span,
                                                        double *__restrict__ part) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    double *raw = reinterpret_cast<double *>(smem_raw);  // [stage][A|B][64][kPX]
    float(*As)[kPX + 4] = reinterpret_cast<float(*)[kPX + 4]>(smem_raw + kProjRawBytes);
    float(*Bs)[kPX + 4] = As + kPT;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int a0 = blockIdx.y * kPT, b0 = blockIdx.z * kPT;
    const long long x0 = (long long)blockIdx.x * span;
    const long long x1 = min(N, x0 + span);
    const int nsteps = x1 > x0 ? (int)((x1 - x0 + kPX - 1) / kPX) : 0;
    float acc_hi[4][4], acc_lo[4][4];
    float2 s[4][4];  // even and odd grid points of the current block
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            acc_hi[i][j] = 0.f;
            acc_lo[i][j] = 0.f;
            s[i][j] = make_float2(0.f, 0.f);
        }
    auto stage = [&](int k) { return raw + (size_t)(k % kPStages) * 2 * kPT * kPX; };
    const bool same = A == B && a0 == b0;  // the B rows are the A rows
    if (nsteps > 0) {
        proj_issue<VEC2>(A, na, a0, N, x0, x1, stage(0), tid);
        if (!same) proj_issue<VEC2>(B, nb, b0, N, x0, x1, stage(0) + kPT * kPX, tid);
    }
    ptx::cp_async_commit();
    const int lx = tid & 31, lr = tid >> 5;  // converter: one grid point, rows lr + 8m
    int blk = 0;
    for (int k = 0; k < nsteps; ++k) {
        if (k + 1 < nsteps) {
            const long long xb = x0 + (long long)(k + 1) * kPX;
            proj_issue<VEC2>(A, na, a0, N, xb, x1, stage(k + 1), tid);
            if (!same) proj_issue<VEC2>(B, nb, b0, N, xb, x1, stage(k + 1) + kPT * kPX, tid);
        }
        ptx::cp_async_commit();
        ptx::cp_async_wait<1>();  // this thread's copies of step k have landed
        __syncthreads();          // everyone's have; the float32 tiles are free
        const double *ra = stage(k), *rb = same ? stage(k) : stage(k) + kPT * kPX;
        const long long xw = x0 + (long long)k * kPX + lx;
        const float wx = (w != nullptr && xw < x1) ? __ldg(w + xw) : 1.f;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int r = lr + 8 * m;
            As[r][lx] = f64_to_f32(ra[r * kPX + lx]);
            Bs[r][lx] = f64_to_f32(rb[r * kPX + lx]) * wx;
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
                    fma2(s[i][j], make_float2(av[i].x, av[i].y), make_float2(bv[j].x, bv[j].y));
                    fma2(s[i][j], make_float2(av[i].z, av[i].w), make_float2(bv[j].z, bv[j].w));
                }
        }
        if (++blk == kPBlk) {
            blk = 0;
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    two_sum_add(acc_hi[i][j], acc_lo[i][j], s[i][j].x + s[i][j].y);
                    s[i][j] = make_float2(0.f, 0.f);
                }
        }
    }
    ptx::cp_async_wait<0>();
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int a = a0 + ty + 16 * i, b = b0 + tx + 16 * j;
            if (a < na && b < nb) {
                two_sum_add(acc_hi[i][j], acc_lo[i][j], s[i][j].x + s[i][j].y);
                part[((long long)blockIdx.x * na + a) * nb + b] = f32_to_f64(acc_hi[i][j]) + f32_to_f64(acc_lo[i][j]);
            }
        }
}

constexpr int kCX = 128;  // combination tile: 128 grid points x 64 output vectors
constexpr int kCB = 64;
constexpr int kCA = 16;   // input vectors per pipeline step
constexpr int kCStages = 3;
constexpr size_t kCombRawBytes = (size_t)kCStages * kCA * kCX * sizeof(double);
// dynamic shared memory: raw float64 stages, the float32 step tile, then C (na rows x 64, float32);
// up to 88 KB (two CTAs per SM) for na <= 128
__host__ __device__ constexpr size_t comb_smem(int na) {
    return kCombRawBytes + (size_t)kCA * kCX * sizeof(float) + (size_t)((na + kCA - 1) / kCA) * kCA * kCB * sizeof(float);
}

// out_b(x) = (accumulate ? out_b(x) : 0) + sgn sum_a A_a(x) C[a][b]
// (a < na, b < nb; C row-major na x nb).  CTA (blockIdx.x, blockIdx.y) owns output vectors b0 = 64 blockIdx.y .. +63
// and walks the 128-point tiles blockIdx.x, + gridDim.x, ...; each tile takes
// ceil(na / 16) steps of 16 input vectors, whose float64 rows are copied into
// shared memory two steps ahead (cp.async).  Thread (tx, ty) of a 32 x 8
// layout owns x = tile + tx + 32 k (k < 4) and b = b0 + 8 ty + j (j < 8): the
// C row piece it needs is the same for the whole warp (two broadcast float4
// reads), the A values are consecutive across lanes.  Sums over a stay in
// float32 (na <= 256 terms).
template <bool VEC2>
__global__ void __launch_bounds__(256, 2) combine32_kernel(const double *__restrict__ A, int na,
                                                           const double *__restrict__ C, int nb, long long N,
                                                           float sgn, bool accumulate, double *__restrict__ out) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    double *raw = reinterpret_cast<double *>(smem_raw);  // [stage][kCA][kCX]
    float(*As)[kCX] = reinterpret_cast<float(*)[kCX]>(smem_raw + kCombRawBytes);
    float(*Cs)[kCB] = reinterpret_cast<float(*)[kCB]>(smem_raw + kCombRawBytes + (size_t)kCA * kCX * sizeof(float));
    const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
    const int b0 = blockIdx.y * kCB;
    const int nch = (na + kCA - 1) / kCA;
    const long long ntiles = (N + kCX - 1) / kCX;
    const long long my_tiles = ntiles > blockIdx.x ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
    const long long nitems = my_tiles * nch;
    for (int e = tid; e < nch * kCA * kCB; e += 256) {
        const int r = e / kCB, c = e % kCB;
        Cs[r][c] = (r < na && b0 + c < nb) ? f64_to_f32(__ldg(C + (long long)r * nb + b0 + c)) : 0.f;
    }
    // item i: tile blockIdx.x + (i / nch) gridDim.x, input vectors 16 (i % nch) ..
    auto issue = [&](long long i) {
        double *dst = raw + (size_t)(i % kCStages) * kCA * kCX;
        const long long xt = (blockIdx.x + (i / nch) * gridDim.x) * kCX;
        const int r0 = (int)(i % nch) * kCA;
        constexpr int per_row = VEC2 ? kCX / 2 : kCX;
#pragma unroll
        for (int m = 0; m < kCA * per_row / 256; ++m) {
            const int piece = tid + 256 * m;
            const int r = piece / per_row, c = (piece % per_row) * (VEC2 ? 2 : 1);
            const long long x = xt + c;
            long long nbytes = (r0 + r < na) ? (N - x) * 8 : 0;
            nbytes = nbytes < 0 ? 0 : (nbytes > (VEC2 ? 16 : 8) ? (VEC2 ? 16 : 8) : nbytes);
            const double *src = nbytes > 0 ? A + (long long)(r0 + r) * N + x : A;
            if (VEC2)
                ptx::cp_async16(dst + r * kCX + c, src, (uint32_t)nbytes);
            else
                ptx::cp_async8(dst + r * kCX + c, src, (uint32_t)nbytes);
        }
    };
#pragma unroll
    for (int i = 0; i < kCStages - 1; ++i) {
        if (i < nitems) issue(i);
        ptx::cp_async_commit();
    }
    float2 acc[4][4];  // acc[jp][k] = outputs b0 + 8 ty + 2 jp (.x) and + 1 (.y) at point k
#pragma unroll
    for (int jp = 0; jp < 4; ++jp)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[jp][k] = make_float2(0.f, 0.f);
    const int lx = tid & 127, lr = tid >> 7;  // converter: one grid point, rows lr + 2m
    for (long long i = 0; i < nitems; ++i) {
        if (i + kCStages - 1 < nitems) issue(i + kCStages - 1);
        ptx::cp_async_commit();
        ptx::cp_async_wait<kCStages - 1>();  // this thread's copies of item i have landed
        __syncthreads();                     // everyone's have; the float32 tile is free
        const double *src = raw + (size_t)(i % kCStages) * kCA * kCX;
#pragma unroll
        for (int m = 0; m < kCA / 2; ++m) As[lr + 2 * m][lx] = f64_to_f32(src[(lr + 2 * m) * kCX + lx]);
        __syncthreads();
        const int ch = (int)(i % nch);
#pragma unroll 4
        for (int r = 0; r < kCA; ++r) {
            float av[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) av[k] = As[r][tx + 32 * k];
            const float4 c0 = *reinterpret_cast<const float4 *>(&Cs[ch * kCA + r][8 * ty]);
            const float4 c1 = *reinterpret_cast<const float4 *>(&Cs[ch * kCA + r][8 * ty + 4]);
            const float2 cv[4] = {make_float2(c0.x, c0.y), make_float2(c0.z, c0.w), make_float2(c1.x, c1.y),
                                  make_float2(c1.z, c1.w)};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 ak = make_float2(av[k], av[k]);
#pragma unroll
                for (int jp = 0; jp < 4; ++jp) fma2(acc[jp][k], ak, cv[jp]);
            }
        }
        if (ch == nch - 1) {
            const long long xt = (blockIdx.x + (i / nch) * gridDim.x) * kCX;
#pragma unroll
            for (int jp = 0; jp < 4; ++jp) {
                const int b = b0 + 8 * ty + 2 * jp;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const long long x = xt + tx + 32 * k;
                    if (x < N) {
                        if (b < nb) {
                            double *o = out + (long long)b * N + x;
                            *o = (accumulate ? *o : 0.0) + f32_to_f64(sgn * acc[jp][k].x);
                        }
                        if (b + 1 < nb) {
                            double *o = out + (long long)(b + 1) * N + x;
                            *o = (accumulate ? *o : 0.0) + f32_to_f64(sgn * acc[jp][k].y);
                        }
                    }
                    acc[jp][k] = make_float2(0.f, 0.f);
                }
            }
        }
    }
    ptx::cp_async_wait<0>();
}

// part (n_split x na x nb) of A^T B over the grid, float64 or float32 products
// by plan precision; returns n_split.
int launch_projection(kx_plan *p, const double *A, int na, const double *B, int nb, const double *w64,
                      const float *w32, double *part, int n_split, cudaStream_t s, int kind = PK_ACE) {
    const long long N = (long long)p->N;
    if (int rc = prof_begin(p, kind, s)) return rc;
    if (p->precision == KX_FP64) {
        const long long span = (N + n_split - 1) / n_split;
        gram_kernel<<<dim3((na + kG - 1) / kG, (nb + kG - 1) / kG, n_split), 256, 0, s>>>(A, na, B, nb, w64, N, span,
                                                                                          part);
        KX_LAUNCH_CHECK("gram_kernel launch");
    } else {
        // whole pipeline steps per CTA, so that every step starts on an even grid point
        const long long span = ((N + n_split - 1) / n_split + kPX - 1) / kPX * kPX;
        const dim3 grid(n_split, (na + kPT - 1) / kPT, (nb + kPT - 1) / kPT);
        // 16-byte copies need even N (so every row starts 16-byte aligned) and aligned bases
        const bool vec2 = N % 2 == 0 && ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15) == 0;
        if (vec2) {
            KX_CUDA_TRY(cudaFuncSetAttribute(proj32_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kProjSmem));
            proj32_kernel<true><<<grid, 256, kProjSmem, s>>>(A, na, B, nb, w32, N, span, part);
        } else {
            KX_CUDA_TRY(cudaFuncSetAttribute(proj32_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kProjSmem));
            proj32_kernel<false><<<grid, 256, kProjSmem, s>>>(A, na, B, nb, w32, N, span, part);
        }
        KX_LAUNCH_CHECK("proj32_kernel launch");
    }
    return prof_end(p, s);
}

// Number of grid-point ranges of the projection: float32 plans put two CTAs
// on each SM with at least 256 points per CTA; float64 plans keep a fixed
// slab split.  A range that starts past the end of the grid leaves a zero
// partial.
int projection_split(const kx_plan *p, int na, int nb) {
    const long long N = (long long)p->N;
    if (p->precision == KX_FP64) return (int)std::max(1LL, std::min<long long>(128, (N + 4095) / 4096));
    const long long tiles = (long long)((na + kPT - 1) / kPT) * ((nb + kPT - 1) / kPT);
    const long long want = std::max(1LL, 2LL * p->num_sms / tiles);
    return (int)std::max(1LL, std::min<long long>(want, (N + 255) / 256));
}

// out = sgn A C (grid vectors), float64 or float32 products by plan precision.
int launch_combination(kx_plan *p, const double *A, int na, const double *C, int nb, double sgn, bool accumulate,
                       double *out, cudaStream_t s, int kind = PK_ACE_COMB) {
    const long long N = (long long)p->N;
    if (int rc = prof_begin(p, kind, s)) return rc;
    if (p->precision == KX_FP64) {
        xi_kernel<<<dim3((unsigned)((N + 127) / 128), (unsigned)((nb + 31) / 32)), 256, 0, s>>>(A, C, na, nb, N, sgn,
                                                                                              accumulate, out);
        KX_LAUNCH_CHECK("xi_kernel launch");
    } else {
        const int tiles_b = (nb + kCB - 1) / kCB;
        const long long ntiles = (N + kCX - 1) / kCX;
        const int gx = (int)std::max(1LL, std::min<long long>(ntiles, std::max(1, 2 * p->num_sms / tiles_b)));
        const size_t smem = comb_smem(na);
        const dim3 grid(gx, tiles_b);
        const float fs = sgn < 0.0 ? -1.f : 1.f;
        const bool vec2 = N % 2 == 0 && (reinterpret_cast<uintptr_t>(A) & 15) == 0;
        if (vec2) {
            KX_CUDA_TRY(cudaFuncSetAttribute(combine32_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem));
            combine32_kernel<true><<<grid, 256, smem, s>>>(A, na, C, nb, N, fs, accumulate, out);
        } else {
            KX_CUDA_TRY(cudaFuncSetAttribute(combine32_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem));
            combine32_kernel<false><<<grid, 256, smem, s>>>(A, na, C, nb, N, fs, accumulate, out);
        }
        KX_LAUNCH_CHECK("combine32_kernel launch");
    }
    return prof_end(p, s);
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
    if ((rc = launch_projection(p, psi, n_orb, W, n_orb, nullptr, nullptr, part, n_slab, s))) return rc;
    if ((rc = prof_begin(p, PK_ACE, s))) return rc;
    gram_reduce_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(part, n_slab, (int)nn, p->dV, M, M_out, A);
    KX_LAUNCH_CHECK("gram_reduce_kernel launch");
    cholesky_kernel<<<1, 256, 0, s>>>(A, n_orb, R, bad);
    KX_LAUNCH_CHECK("cholesky_kernel launch");
    triinv_kernel<<<(n_orb + 127) / 128, 128, 0, s>>>(R, n_orb, Rinv);
    KX_LAUNCH_CHECK("triinv_kernel launch");
    if ((rc = prof_end(p, s))) return rc;
    if ((rc = launch_combination(p, W, n_orb, Rinv, n_orb, 1.0, false, xi, s))) return rc;
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
    if ((rc = launch_projection(p, xi, n_xi, phi, n_vec, nullptr, nullptr, part, n_split, s))) return rc;
    if ((rc = prof_begin(p, PK_ACE, s))) return rc;
    gram_reduce_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, s>>>(part, n_split, (int)ne, p->dV, P, nullptr,
                                                                    nullptr);
    KX_LAUNCH_CHECK("gram_reduce_kernel launch");
    if ((rc = prof_end(p, s))) return rc;
    return launch_combination(p, xi, n_xi, P, n_vec, -1.0, false, out, s);
}

size_t grid_projection_bytes(const kx_plan *p, int na, int nb) {
    return sizeof(double) * (size_t)na * nb * (size_t)projection_split(p, na, nb) + 256;
}

int grid_projection(kx_plan *p, const double *A, int na, const double *B, int nb, const double *w64, const float *w32,
                    double scale, double *out, cudaStream_t s, int kind) {
    const int n_split = projection_split(p, na, nb);
    const size_t ne = (size_t)na * nb;
    int rc = ensure_workspace(p, grid_projection_bytes(p, na, nb));
    if (rc) return rc;
    double *part = (double *)p->ws.ptr;
    if ((rc = launch_projection(p, A, na, B, nb, w64, w32, part, n_split, s, kind))) return rc;
    if ((rc = prof_begin(p, kind, s))) return rc;
    gram_reduce_kernel<<<(unsigned)((ne + 255) / 256), 256, 0, s>>>(part, n_split, (int)ne, scale, out, nullptr,
                                                                    nullptr);
    KX_LAUNCH_CHECK("gram_reduce_kernel launch");
    return prof_end(p, s);
}

int grid_combination(kx_plan *p, const double *A, int na, const double *C, int nb, double sgn, bool accumulate,
                     double *out, cudaStream_t s, int kind) {
    return launch_combination(p, A, na, C, nb, sgn, accumulate, out, s, kind);
}

}  // namespace kx
