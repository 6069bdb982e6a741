// Exact exchange with Bloch-periodic boundary conditions and k-point sums
// (Sec. 2.1, Eqs. 6-9; Sec. 3, Eq. 19 with complex, wavevector-dependent Vk).
//
// For a target k-point and vectors phi_v every k-point q contributes
//   (Vx phi)_v -= w_q sum_m g_mq psi_mq f(L_{k-q}) (conj(psi_mq) phi_v),
// the Poisson problem of the pair taking the Bloch phases theta_k - theta_q
// along the periodic axes.  Along such an axis the Bloch matrix at phase theta
// has the eigenvectors e^{i kappa_m x} / sqrt(n), kappa_m = (2 pi m + theta) / n,
// with the stencil's symbol (w_0 + 2 sum_p w_p cos(p kappa_m)) / h^2 as
// eigenvalue, so the complex basis of each q is written in closed form; Dirichlet
// axes keep the plan's real eigenvectors.  The forward transform contracts with
// conj(Vk), the inverse with Vk.  The six complex mode products run on the CUDA
// cores, in float64 for KX_FP64 plans and in float32 (packed f32x2 FMAs) for the
// others; the pair density is formed inside the first product and f(Lambda) is
// applied inside the third.  For Vx psi at every k-point the block of pairs
// (k, q), q > k, is solved once: read conjugated it is the block (q, k).
#include "kx_internal.h"
#include "kx_conv.cuh"
#include "kx_fd.cuh"
#include "kx_tc_ptx.cuh"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdlib>

namespace kx {
namespace {

template <typename T> struct Cx;
template <> struct Cx<float> { using t = float2; };
template <> struct Cx<double> { using t = double2; };

constexpr int kBThreads = 256;
constexpr int kBWarps = kBThreads / 32;  // output-column groups of a CTA
template <typename T> constexpr int pencils_per_thread() { return sizeof(T) == 4 ? 2 : 1; }
template <typename T> constexpr int tile_pencils() { return 32 * pencils_per_thread<T>(); }
constexpr size_t kBSmemTarget = 110 * 1024;  // two CTAs per SM where the split allows it
constexpr size_t kBSmemPipeMax = 200 * 1024;  // pipelined products: operand + two tiles
constexpr int kBMaxPerSm = 4;                  // resident pipelined CTAs per SM used (energy partial slots)

template <typename T2> __device__ __forceinline__ T2 cmul_conj(T2 a, T2 b) {  // conj(a) b
    T2 r;
    r.x = a.x * b.x + a.y * b.y;
    r.y = a.x * b.y - a.y * b.x;
    return r;
}

// res[j][u] = sum_k Ms[k][w + 8u] Ts[k][l + 32j] for the warp w and lane l of
// the calling thread (operand padded to NCP = 8U columns).  float32: two packed
// accumulators per output, (sum a_re v, sum a_im v), combined at the end.
template <typename T, int PQ, int U>
__device__ __forceinline__ void tile_products(const typename Cx<T>::t *Ts, const typename Cx<T>::t *Ms, int ld,
                                              int n, int lane, int warp, typename Cx<T>::t (&res)[PQ][U]) {
    constexpr int NCP = 8 * U;
    if constexpr (sizeof(T) == 4) {
        float2 accA[PQ][U], accB[PQ][U];
#pragma unroll
        for (int j = 0; j < PQ; ++j)
#pragma unroll
            for (int u = 0; u < U; ++u) accA[j][u] = accB[j][u] = make_float2(0.f, 0.f);
        const float2 *mcol = Ms + warp;
        const float2 *tcol = Ts + lane;
#pragma unroll 2
        for (int k = 0; k < n; ++k) {
            float2 ar[PQ], ai[PQ];
#pragma unroll
            for (int j = 0; j < PQ; ++j) {
                const float2 a = tcol[k * ld + 32 * j];
                ar[j] = make_float2(a.x, a.x);
                ai[j] = make_float2(a.y, a.y);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const float2 v = mcol[k * NCP + 8 * u];
#pragma unroll
                for (int j = 0; j < PQ; ++j) {
                    fma2(accA[j][u], ar[j], v);
                    fma2(accB[j][u], ai[j], v);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < PQ; ++j)
#pragma unroll
            for (int u = 0; u < U; ++u)
                res[j][u] = make_float2(accA[j][u].x - accB[j][u].y, accA[j][u].y + accB[j][u].x);
    } else {
#pragma unroll
        for (int j = 0; j < PQ; ++j)
#pragma unroll
            for (int u = 0; u < U; ++u) res[j][u] = make_double2(0.0, 0.0);
        for (int k = 0; k < n; ++k) {
#pragma unroll
            for (int j = 0; j < PQ; ++j) {
                const double2 a = Ts[k * ld + lane + 32 * j];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const double2 v = Ms[k * NCP + warp + 8 * u];
                    res[j][u].x = fma(a.x, v.x, fma(-a.y, v.y, res[j][u].x));
                    res[j][u].y = fma(a.x, v.y, fma(a.y, v.x, res[j][u].y));
                }
            }
        }
    }
}

// Stage the output columns [c0, c0 + ncy) of the operand (n x n, M[k][c]) with
// zero padding up to NCP = 8U columns.
template <typename T, int U>
__device__ __forceinline__ void stage_operand(typename Cx<T>::t *Ms, const typename Cx<T>::t *__restrict__ M, int n,
                                              int c0, int ncy, int lane, int warp) {
    constexpr int NCP = 8 * U;
    for (int k = warp; k < n; k += kBWarps)
        for (int cl = lane; cl < NCP; cl += 32) {
            typename Cx<T>::t z;
            z.x = z.y = (T)0;
            Ms[k * NCP + cl] = cl < ncy ? M[(size_t)k * n + c0 + cl] : z;
        }
}

// The first product (mode 1 forward, pencils contiguous): for the R chunk
// items, out[r][x2, x3][c] = sum_k M[k][c] rho_r[x2, x3][k], where item r is the
// pair (v, m) = divmod(r0 + r, n_orb) and rho_r = conj(P_m) F_v is formed while
// the tile is loaded.  Pencils q (N / n per item), QB = 32 PQ of them per CTA;
// warp w owns the output columns c0 + w + 8u (u < U, operand zero-padded to
// 8U columns), lane l the pencils l + 32j (j < PQ).  Chunk-relative indices
// stay below 2^31 and pair indices below 2^24 (checked at launch and entry).
template <typename T, int U>
__global__ void __launch_bounds__(kBThreads) bloch_form_kernel(
    typename Cx<T>::t *__restrict__ out, int n_cols, int n, const typename Cx<T>::t *__restrict__ M, int nc,
    int n_split, const typename Cx<T>::t *__restrict__ P, const typename Cx<T>::t *__restrict__ F, int n_orb,
    long long r0, long long N) {
    using T2 = typename Cx<T>::t;
    constexpr int PQ = pencils_per_thread<T>();
    constexpr int QB = 32 * PQ;
    constexpr int NCP = 8 * U;
    extern __shared__ __align__(16) unsigned char bloch_smem[];
    T2 *Ms = reinterpret_cast<T2 *>(bloch_smem);  // n x NCP
    T2 *Ts = Ms + (size_t)n * NCP;                // n x (QB + 1): Ts[k * ld + ql]
    const int ld = QB + 1;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int split = (int)(blockIdx.x % n_split);
    const int tile = (int)(blockIdx.x / n_split);
    const int c0 = split * nc;
    const int ncy = min(nc, n - c0);
    stage_operand<T, U>(Ms, M, n, c0, ncy, lane, warp);
    const int q0 = tile * QB;
    const int nq = min(QB, n_cols - q0);
    const int ppi = (int)(N / n);  // pencils per item
#pragma unroll 4
    for (int ql = warp; ql < nq; ql += kBWarps) {
        const int q = q0 + ql;
        const int r = q / ppi;
        const long long x0 = (long long)(q - r * ppi) * n;
        const int rr = (int)r0 + r;
        const int vv = rr / n_orb, m = rr - vv * n_orb;
        const T2 *Pp = P + (long long)m * N + x0;
        const T2 *Fp = F + (long long)vv * N + x0;
        for (int k = lane; k < n; k += 32) Ts[k * ld + ql] = cmul_conj(Pp[k], Fp[k]);
    }
    __syncthreads();
    T2 res[PQ][U];
    tile_products<T, PQ, U>(Ts, Ms, ld, n, lane, warp, res);
    __syncthreads();
#pragma unroll
    for (int j = 0; j < PQ; ++j) {
        const int ql = lane + 32 * j;
        if (ql >= nq) continue;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int cl = warp + 8 * u;
            if (cl < ncy) Ts[cl * ld + ql] = res[j][u];
        }
    }
    __syncthreads();
    for (int ql = warp; ql < nq; ql += kBWarps) {
        T2 *dst = out + (size_t)(q0 + ql) * n + c0;
        for (int cl = lane; cl < ncy; cl += 32) dst[cl] = Ts[cl * ld + ql];
    }
}

// Energy-only epilogue of the third product (E_x through Parseval): item r of
// the chunk (pair (v, m) = divmod(r0 + r, n_orb)) weighs cb g_q[m] g_k[v], and
// each CTA writes sum weight f |Y|^2 over its outputs to partial[blockIdx.x].
struct EnergyArgs {
    const double *occ_q = nullptr, *occ_k = nullptr;  // nullable: occupations 1
    int n_orb = 1;
    long long r0 = 0;
    double cb = 0.0;
    double *partial = nullptr;
};

// The products that read a plain input (all but the first): persistent CTAs,
// each with a fixed column split and a strided run of tiles, the operand staged
// once, and the next tile copied in (cp.async) while the current one is
// multiplied; the current tile's buffer then stages the output.  Same mapping
// and arithmetic as bloch_form_kernel.  EPI: 0 plain, 1 output times f (third
// product), 2 no output, the energy sum instead (third product, EnergyArgs).
template <typename T, int EPI, int U>
__global__ void __launch_bounds__(kBThreads) bloch_mode_pipe_kernel(
    const typename Cx<T>::t *__restrict__ in, typename Cx<T>::t *__restrict__ out, int n_cols, int n, int inner,
    const typename Cx<T>::t *__restrict__ M, int nc, int n_split, const T *__restrict__ f, EnergyArgs ea) {
    using T2 = typename Cx<T>::t;
    constexpr int PQ = pencils_per_thread<T>();
    constexpr int QB = 32 * PQ;
    constexpr int NCP = 8 * U;
    extern __shared__ __align__(16) unsigned char bloch_smem[];
    T2 *Ms = reinterpret_cast<T2 *>(bloch_smem);  // n x NCP
    const int ld = QB + 1;
    T2 *const Tb0 = Ms + (size_t)n * NCP;  // two tile buffers of n x ld
    const int tsz = n * ld;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int split = (int)(blockIdx.x % n_split);
    const int t_first = (int)(blockIdx.x / n_split);
    const int t_stride = (int)(gridDim.x / n_split);
    const int n_tiles = (n_cols + QB - 1) / QB;
    const int c0 = split * nc;
    const int ncy = min(nc, n - c0);
    stage_operand<T, U>(Ms, M, n, c0, ncy, lane, warp);
    auto issue = [&](int t, T2 *buf) {
        const int q0 = t * QB;
        const int nq = min(QB, n_cols - q0);
        if (inner == 1) {
            for (int ql = warp; ql < nq; ql += kBWarps) {
                const T2 *src = in + (size_t)(q0 + ql) * n;
                for (int k = lane; k < n; k += 32) {
                    if constexpr (sizeof(T) == 4) ptx::cp_async8(buf + k * ld + ql, src + k, 8);
                    else ptx::cp_async16(buf + k * ld + ql, src + k, 16);
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < PQ; ++j) {
                const int ql = lane + 32 * j;
                if (ql < nq) {
                    const int q = q0 + ql;
                    const int o = q / inner;
                    const T2 *src = in + (size_t)o * n * inner + (q - o * inner);
                    for (int k = warp; k < n; k += kBWarps) {
                        if constexpr (sizeof(T) == 4) ptx::cp_async8(buf + k * ld + ql, src + (size_t)k * inner, 8);
                        else ptx::cp_async16(buf + k * ld + ql, src + (size_t)k * inner, 16);
                    }
                }
            }
        }
    };
    double e_acc = 0.0;  // EPI == 2
    if (t_first < n_tiles) issue(t_first, Tb0);
    ptx::cp_async_commit();
    int it = 0;
    for (int t = t_first; t < n_tiles; t += t_stride, ++it) {
        T2 *cur = Tb0 + (it & 1) * tsz;
        if (t + t_stride < n_tiles) issue(t + t_stride, Tb0 + ((it + 1) & 1) * tsz);
        ptx::cp_async_commit();
        ptx::cp_async_wait<1>();
        __syncthreads();
        const int q0 = t * QB;
        const int nq = min(QB, n_cols - q0);
        T2 res[PQ][U];
        tile_products<T, PQ, U>(cur, Ms, ld, n, lane, warp, res);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < PQ; ++j) {
            const int ql = lane + 32 * j;
            if (ql >= nq) continue;
            int i_in = 0;
            double wj = 0.0;
            if constexpr (EPI != 0) {
                const int item = (q0 + ql) / inner;
                i_in = (q0 + ql) - item * inner;
                if constexpr (EPI == 2) {
                    const long long rr = ea.r0 + item;
                    const long long vv = rr / ea.n_orb, mm = rr - vv * ea.n_orb;
                    wj = ea.cb * (ea.occ_q ? ea.occ_q[mm] : 1.0) * (ea.occ_k ? ea.occ_k[vv] : 1.0);
                }
            }
            T ej = 0;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int cl = warp + 8 * u;
                if (cl < ncy) {
                    T2 v = res[j][u];
                    if constexpr (EPI == 1) {
                        const T fv = f[(size_t)(c0 + cl) * inner + i_in];
                        v.x *= fv;
                        v.y *= fv;
                    }
                    if constexpr (EPI == 2) {
                        const T fv = f[(size_t)(c0 + cl) * inner + i_in];
                        ej = fma(fv, v.x * v.x + v.y * v.y, ej);
                    } else {
                        cur[cl * ld + ql] = v;
                    }
                }
            }
            if constexpr (EPI == 2) e_acc += wj * (double)ej;
        }
        __syncthreads();
        if constexpr (EPI == 2) continue;  // no output
        if (inner == 1) {
            for (int ql = warp; ql < nq; ql += kBWarps) {
                T2 *dst = out + (size_t)(q0 + ql) * n + c0;
                for (int cl = lane; cl < ncy; cl += 32) dst[cl] = cur[cl * ld + ql];
            }
        } else {
#pragma unroll
            for (int j = 0; j < PQ; ++j) {
                const int ql = lane + 32 * j;
                if (ql < nq) {
                    const int q = q0 + ql;
                    const int o = q / inner;
                    T2 *dst = out + (size_t)o * n * inner + (q - o * inner);
                    for (int cl = warp; cl < ncy; cl += kBWarps) dst[(size_t)(c0 + cl) * inner] = cur[cl * ld + ql];
                }
            }
        }
        __syncthreads();
    }
    ptx::cp_async_wait<0>();
    if constexpr (EPI == 2) {
        __shared__ double red[kBWarps];
        for (int o = 16; o > 0; o >>= 1) e_acc += __shfl_xor_sync(0xffffffffu, e_acc, o);
        if (lane == 0) red[warp] = e_acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int w = 0; w < kBWarps; ++w) t += red[w];
            ea.partial[blockIdx.x] = t;
        }
    }
}

struct BlochAxes {
    int n[3];
    double h[3];
    int bc[3];
    double theta[3];
    int order;
    const double *V[3];    // plan's real eigenvectors (Dirichlet axes), V[x][k]
    const double *lam[3];  // plan's eigenvalues (Dirichlet axes)
};

// blockIdx.x = axis, blockIdx.y shares the n x n entries: the forward operand
// Mf[k][c] = conj(V[k][c]) and the inverse operand Mi[k][c] = V[c][k] in T, and
// the eigenvalues lam_out (float64).
template <typename T>
__global__ void bloch_basis_kernel(BlochAxes ax, typename Cx<T>::t *Mf0, typename Cx<T>::t *Mf1,
                                   typename Cx<T>::t *Mf2, typename Cx<T>::t *Mi0, typename Cx<T>::t *Mi1,
                                   typename Cx<T>::t *Mi2, double *lam0, double *lam1, double *lam2) {
    using T2 = typename Cx<T>::t;
    const int a = blockIdx.x;
    const int n = ax.n[a];
    T2 *Mf = a == 0 ? Mf0 : (a == 1 ? Mf1 : Mf2);
    T2 *Mi = a == 0 ? Mi0 : (a == 1 ? Mi1 : Mi2);
    double *lam = a == 0 ? lam0 : (a == 1 ? lam1 : lam2);
    const bool bloch = ax.bc[a] == KX_PERIODIC;
    const double th = ax.theta[a];
    const double inv_sqrt_n = 1.0 / sqrt((double)n);
    for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < n * n; e += gridDim.y * blockDim.x) {
        int x = e / n, m = e - x * n;
        double vr, vi;
        if (bloch) {
            // e^{i 2 pi m x / n} with the angle reduced exactly, times e^{i theta x / n}
            int t = (int)(((long long)m * x) % n);
            double s1, c1, s2, c2;
            sincospi(2.0 * t / n, &s1, &c1);
            sincos(th * x / n, &s2, &c2);
            vr = (c1 * c2 - s1 * s2) * inv_sqrt_n;
            vi = (s1 * c2 + c1 * s2) * inv_sqrt_n;
        } else {
            vr = ax.V[a][x * n + m];
            vi = 0.0;
        }
        T2 v;
        v.x = (T)vr;
        v.y = (T)vi;
        Mi[m * n + x] = v;
        v.y = -v.y;
        Mf[x * n + m] = v;
    }
    if (blockIdx.y != 0) return;
    const int mo = ax.order / 2;
    const double ih2 = 1.0 / (ax.h[a] * ax.h[a]);
    for (int m = threadIdx.x; m < n; m += blockDim.x) {
        if (bloch) {
            double kap = (2.0 * M_PI * m + th) / n;
            double s = fd_weight(mo, 0);
            for (int p = 1; p <= mo; ++p) s += 2.0 * fd_weight(mo, p) * cos(p * kap);
            lam[m] = s * ih2;
        } else {
            lam[m] = ax.lam[a][m];
        }
    }
}

template <typename T>
__global__ void bloch_ftable_kernel(int n1, int n2, int n3, const double *l1, const double *l2, const double *l3,
                                    int kind, double omega, T *f) {
    const long long N = (long long)n1 * n2 * n3;
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < N;
         idx += (long long)gridDim.x * blockDim.x) {
        int k1 = (int)(idx % n1);
        int k2 = (int)((idx / n1) % n2);
        int k3 = (int)(idx / ((long long)n1 * n2));
        f[idx] = (T)kernel_f_value(kind, omega, l1[k1] + l2[k2] + l3[k3]);
    }
}

// complex float64 -> float32 (count complex values)
__global__ void bloch_to_f32_kernel(const double2 *__restrict__ src, float2 *__restrict__ dst, long long count) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < count;
         e += (long long)gridDim.x * blockDim.x) {
        double2 v = src[e];
        dst[e] = make_float2(f64_to_f32(v.x), f64_to_f32(v.y));
    }
}

// out_v[x] -= sum over the chunk items r = v * n_orb + m in [r0, r1) of
// w_q g_mq psi_m[x] X_{r - r0}[x] (m ascending, one thread per (v, x)).
template <typename T>
__global__ void bloch_accum_kernel(const typename Cx<T>::t *__restrict__ X, long long r0, long long r1, int n_orb,
                                   const typename Cx<T>::t *__restrict__ P, const double *__restrict__ occ_q,
                                   double wq, double2 *__restrict__ out, long long N) {
    using T2 = typename Cx<T>::t;
    const long long v_lo = r0 / n_orb, v_hi = (r1 - 1) / n_orb;
    const long long total = (v_hi - v_lo + 1) * N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        long long vl = e / N, x = e - vl * N;
        long long v = v_lo + vl;
        long long m0 = max(0LL, r0 - v * n_orb), m1 = min((long long)n_orb, r1 - v * n_orb);
        T sr = 0, si = 0;
        for (long long m = m0; m < m1; ++m) {
            T2 p = P[m * N + x];
            T2 xx = X[(v * n_orb + m - r0) * N + x];
            T c = (T)(wq * (occ_q ? occ_q[m] : 1.0));
            sr = fma(c, p.x * xx.x - p.y * xx.y, sr);
            si = fma(c, p.x * xx.y + p.y * xx.x, si);
        }
        double2 o = out[v * N + x];
        if constexpr (sizeof(T) == 4) {
            o.x -= f32_to_f64(sr);
            o.y -= f32_to_f64(si);
        } else {
            o.x -= sr;
            o.y -= si;
        }
        out[v * N + x] = o;
    }
}

// partial[k * nb + b] = w_k sum_n g_kn sum_x Re(conj(psi_kn[x]) vx_kn[x]) over a
// grid-stride share (block b of nb).
constexpr int kEThreads = 256;
__global__ void __launch_bounds__(kEThreads) bloch_energy_kernel(const double2 *__restrict__ psi,
                                                                const double2 *__restrict__ vx,
                                                                const double *__restrict__ occ_k, int n_orb,
                                                                long long N, double wk, double *partial) {
    double s = 0.0;
    const long long total = (long long)n_orb * N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        double2 a = psi[e], b = vx[e];
        double g = occ_k ? occ_k[e / N] : 1.0;
        s += g * (a.x * b.x + a.y * b.y);
    }
    __shared__ double red[kEThreads / 32];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < kEThreads / 32; ++w) t += red[w];
        partial[blockIdx.x] = wk * t;
    }
}

__global__ void bloch_energy_final_kernel(const double *partial, int count, double half_dv, double *ex) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double t = 0.0;
        for (int i = 0; i < count; ++i) t += partial[i];
        *ex = half_dv * t;
    }
}

inline size_t al256(size_t b) { return (b + 255) / 256 * 256; }

// Output columns per CTA split for an axis of n points: all n where the shared
// memory allows two CTAs per SM, else halves; the per-thread output count U
// rounds the split up to 8U columns from the instantiated set.
template <typename T> int outputs_for(int nc) {
    const int need = (nc + kBWarps - 1) / kBWarps;
    if (sizeof(T) == 8) return need <= 2 ? 2 : (need <= 4 ? 4 : 8);
    return need <= 2 ? 2 : need <= 4 ? 4 : need <= 6 ? 6 : need <= 8 ? 8 : need <= 12 ? 12 : 16;
}

template <typename T>
void choose_split(int n, int *nc, int *n_split, int *U, size_t *smem) {
    using T2 = typename Cx<T>::t;
    const int max_cols = kBWarps * (sizeof(T) == 4 ? 16 : 8);
    auto bytes = [n](int u) { return sizeof(T2) * ((size_t)n * 8 * u + (size_t)n * (tile_pencils<T>() + 1)); };
    int c = std::min(n, max_cols);
    while (bytes(outputs_for<T>(c)) > kBSmemTarget && c > kBWarps) c = (c + 1) / 2;
    *nc = c;
    *n_split = (n + c - 1) / c;
    *U = outputs_for<T>(c);
    *smem = bytes(*U);
}

template <typename T, int U>
int launch_form_u(unsigned blocks, size_t smem, cudaStream_t s, typename Cx<T>::t *out, int n_cols, int n,
                  const typename Cx<T>::t *M, int nc, int n_split, const typename Cx<T>::t *P,
                  const typename Cx<T>::t *F, int n_orb, long long r0, long long N) {
    static bool attr = false;  // once per instantiation
    if (!attr) {
        KX_CUDA_TRY(cudaFuncSetAttribute(bloch_form_kernel<T, U>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         200 * 1024));
        attr = true;
    }
    bloch_form_kernel<T, U><<<blocks, kBThreads, smem, s>>>(out, n_cols, n, M, nc, n_split, P, F, n_orb, r0, N);
    KX_LAUNCH_CHECK("bloch_form_kernel launch");
    return KX_OK;
}

// The first product of a chunk: pair densities of items [r0, r0 + R) formed
// from P (orbitals at q) and F (vectors at k), contracted along axis 0 into out.
template <typename T>
int launch_form(kx_plan *p, long long R, typename Cx<T>::t *out, const typename Cx<T>::t *M,
                const typename Cx<T>::t *P, const typename Cx<T>::t *F, int n_orb, long long r0, cudaStream_t s) {
    const int n = p->n[0];
    const long long N = (long long)p->N;
    const long long n_cols = R * (N / n);
    int nc, n_split, U;
    size_t smem;
    choose_split<T>(n, &nc, &n_split, &U, &smem);
    const long long blocks = (n_cols + tile_pencils<T>() - 1) / tile_pencils<T>() * n_split;
    if (R * N >= (1LL << 31) || blocks > 0x7fffffffLL)
        return set_error(KX_ERR_ARG, "Bloch exchange: chunk too large for one launch");
    if (int rc = prof_begin(p, PK_BLOCH, s)) return rc;
    const unsigned b = (unsigned)blocks;
    const int nco = (int)n_cols;
#define KX_BLOCH_FORM(UU) launch_form_u<T, UU>(b, smem, s, out, nco, n, M, nc, n_split, P, F, n_orb, r0, N)
    int rc;
    if (U == 2) rc = KX_BLOCH_FORM(2);
    else if (U == 4) rc = KX_BLOCH_FORM(4);
    else if (U == 8) rc = KX_BLOCH_FORM(8);
    else if constexpr (sizeof(T) == 4) {
        if (U == 6) rc = KX_BLOCH_FORM(6);
        else if (U == 12) rc = KX_BLOCH_FORM(12);
        else rc = KX_BLOCH_FORM(16);
    } else {
        rc = set_error(KX_ERR_ARG, "Bloch exchange: no kernel for this split");
    }
#undef KX_BLOCH_FORM
    if (rc) return rc;
    return prof_end(p, s);
}

// Split for the pipelined products (two tile buffers): all n columns where the
// shared memory (operand + two tiles) fits 200 KB, else halves.
template <typename T>
void choose_split_pipe(int n, int *nc, int *n_split, int *U, size_t *smem) {
    using T2 = typename Cx<T>::t;
    const int max_cols = kBWarps * (sizeof(T) == 4 ? 16 : 8);
    auto bytes = [n](int u) { return sizeof(T2) * ((size_t)n * 8 * u + 2 * (size_t)n * (tile_pencils<T>() + 1)); };
    int c = std::min(n, max_cols);
    while (bytes(outputs_for<T>(c)) > kBSmemPipeMax && c > kBWarps) c = (c + 1) / 2;
    *nc = c;
    *n_split = (n + c - 1) / c;
    *U = outputs_for<T>(c);
    *smem = bytes(*U);
}

template <typename T, int EPI, int U>
int launch_pipe_u(kx_plan *p, long long n_tiles, size_t smem, cudaStream_t s, const typename Cx<T>::t *in,
                  typename Cx<T>::t *out, int n_cols, int n, int inner, const typename Cx<T>::t *M, int nc,
                  int n_split, const T *f, const EnergyArgs &ea) {
    static int per_sm = 0;  // resident CTAs per SM at this instantiation's shared memory (set once)
    static size_t per_sm_smem = 0;
    if (per_sm == 0 || per_sm_smem != smem) {
        KX_CUDA_TRY(cudaFuncSetAttribute(bloch_mode_pipe_kernel<T, EPI, U>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBSmemPipeMax));
        KX_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bloch_mode_pipe_kernel<T, EPI, U>,
                                                                  kBThreads, smem));
        per_sm = std::max(per_sm, 1);
        per_sm_smem = smem;
    }
    const long long per_split =
        std::max(1LL, std::min(n_tiles, (long long)std::min(per_sm, kBMaxPerSm) * p->num_sms / n_split));
    const unsigned blocks = (unsigned)(per_split * n_split);
    bloch_mode_pipe_kernel<T, EPI, U><<<blocks, kBThreads, smem, s>>>(in, out, n_cols, n, inner, M, nc, n_split, f,
                                                                       ea);
    KX_LAUNCH_CHECK("bloch_mode_pipe_kernel launch");
    return KX_OK;
}

template <typename T, int EPI>
int launch_pipe(kx_plan *p, int axis, long long R, const typename Cx<T>::t *in, typename Cx<T>::t *out,
                const typename Cx<T>::t *M, const T *f, cudaStream_t s, const EnergyArgs &ea = EnergyArgs()) {
    const int n = p->n[axis];
    const long long N = (long long)p->N;
    const int inner = axis == 0 ? 1 : (axis == 1 ? p->n[0] : p->n[0] * p->n[1]);
    const long long n_cols = R * (N / n);
    int nc, n_split, U;
    size_t smem;
    choose_split_pipe<T>(n, &nc, &n_split, &U, &smem);
    const long long n_tiles = (n_cols + tile_pencils<T>() - 1) / tile_pencils<T>();
    if (R * N >= (1LL << 31)) return set_error(KX_ERR_ARG, "Bloch exchange: chunk too large for one launch");
    if (smem > kBSmemPipeMax) return set_error(KX_ERR_UNSUPPORTED, "Bloch exchange: axis too long for the tile");
    if (int rc = prof_begin(p, PK_BLOCH, s)) return rc;
    const int nco = (int)n_cols;
#define KX_BLOCH_PIPE(UU) \
    launch_pipe_u<T, EPI, UU>(p, n_tiles, smem, s, in, out, nco, n, inner, M, nc, n_split, f, ea)
    int rc;
    if (U == 2) rc = KX_BLOCH_PIPE(2);
    else if (U == 4) rc = KX_BLOCH_PIPE(4);
    else if (U == 8) rc = KX_BLOCH_PIPE(8);
    else if constexpr (sizeof(T) == 4) {
        if (U == 6) rc = KX_BLOCH_PIPE(6);
        else if (U == 12) rc = KX_BLOCH_PIPE(12);
        else rc = KX_BLOCH_PIPE(16);
    } else {
        rc = set_error(KX_ERR_ARG, "Bloch exchange: no kernel for this split");
    }
#undef KX_BLOCH_PIPE
    if (rc) return rc;
    return prof_end(p, s);
}

// Device workspace of one call: bases, eigenvalues, f table, float32 copies of
// the orbitals and vectors (float32 plans), chunk buffers A and B.
struct BlochLayout {
    size_t Mf[3], Mi[3], lam[3], f, P, F, A, B, partial, total;
    long long chunk;
};

template <typename T>
BlochLayout bloch_layout(const kx_plan *p, int n_orb, int n_vec, int n_kpt, size_t partial_doubles = 0) {
    using T2 = typename Cx<T>::t;
    BlochLayout L;
    const size_t N = p->N;
    size_t off = 0;
    for (int a = 0; a < 3; ++a) {
        L.Mf[a] = off;
        off += al256(sizeof(T2) * p->n[a] * p->n[a]);
        L.Mi[a] = off;
        off += al256(sizeof(T2) * p->n[a] * p->n[a]);
        L.lam[a] = off;
        off += al256(sizeof(double) * p->n[a]);
    }
    L.f = off;
    off += al256(sizeof(T) * N);
    const bool f32 = sizeof(T) == 4;
    L.P = off;
    off += f32 ? al256(sizeof(T2) * N * n_orb) : 0;
    L.F = off;
    off += f32 ? al256(sizeof(T2) * N * n_vec) : 0;
    L.partial = off;
    off += al256(sizeof(double) * std::max(partial_doubles, 2 * (size_t)p->num_sms * std::max(1, n_kpt)));
    const long long pairs = (long long)n_orb * n_vec;
    const size_t budget = (size_t)2 << 30;  // both chunk buffers
    long long chunk = (long long)std::max<size_t>(1, budget / (2 * sizeof(T2) * N));
    if (const char *e = std::getenv("KX_CHUNK_PAIRS"))  // tuning override (pairs per chunk)
        if (std::atoll(e) > 0) chunk = std::min(chunk, std::atoll(e));
    chunk = std::min(chunk, pairs);
    L.chunk = chunk;
    L.A = off;
    off += al256(sizeof(T2) * N * chunk);
    L.B = off;
    off += al256(sizeof(T2) * N * chunk);
    L.total = off;
    return L;
}

// The same solves read the other way (kx_vx_kpoints with k < q): the pair
// (q m, k v) has the density conj(rho) and the phase -theta, and f(L_{-theta})
// conj(rho) = conj(f(L_theta) rho) (L_{-theta} = conj(L_theta)), so
// out_m[x] -= sum over the chunk items r = v * n_orb + m in [r0, r1) of
// w_k g_vk F_v[x] conj(X_{r - r0}[x]) (v ascending, one thread per (m, x)).
template <typename T>
__global__ void bloch_accum_rev_kernel(const typename Cx<T>::t *__restrict__ X, long long r0, long long r1,
                                       int n_orb, const typename Cx<T>::t *__restrict__ F,
                                       const double *__restrict__ occ_k, double wk, double2 *__restrict__ out,
                                       long long N) {
    using T2 = typename Cx<T>::t;
    const long long v_lo = r0 / n_orb, v_hi = (r1 - 1) / n_orb;
    const long long total = (long long)n_orb * N;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        long long m = e / N, x = e - m * N;
        T sr = 0, si = 0;
        bool any = false;
        for (long long v = v_lo; v <= v_hi; ++v) {
            long long r = v * n_orb + m;
            if (r < r0 || r >= r1) continue;
            any = true;
            T2 fv = F[v * N + x];
            T2 xx = X[(r - r0) * N + x];
            T c = (T)(wk * (occ_k ? occ_k[v] : 1.0));
            sr = fma(c, fv.x * xx.x + fv.y * xx.y, sr);  // F conj(X)
            si = fma(c, fv.y * xx.x - fv.x * xx.y, si);
        }
        if (!any) continue;
        double2 o = out[m * N + x];
        if constexpr (sizeof(T) == 4) {
            o.x -= f32_to_f64(sr);
            o.y -= f32_to_f64(si);
        } else {
            o.x -= sr;
            o.y -= si;
        }
        out[m * N + x] = o;
    }
}

// Solves of the k-point pairs (k, q) for q = q_begin .. n_kpt - 1 with the
// vectors phi at k (n_vec of them): out_k -= w_q g_mq psi_mq X for every q and,
// when out_all is given, out_all[q] -= w_k g_vk phi_v conj(X) for q > k (the
// reversed pairs, phi being psi_k).  psi: n_kpt x n_orb x N complex, occ:
// n_kpt x n_orb (nullable).  Outputs are accumulated into.
template <typename T>
int bloch_sweep(kx_plan *p, int n_kpt, const double *theta, const double *wk, int n_orb, const double *psi,
                const double *occ, int k, int q_begin, int n_vec, const double *phi, double *out_k,
                double *out_all, cudaStream_t s) {
    using T2 = typename Cx<T>::t;
    const long long N = (long long)p->N;
    BlochLayout L = bloch_layout<T>(p, n_orb, n_vec, n_kpt);
    if (int rc = ensure_workspace(p, L.total)) return rc;
    char *ws = static_cast<char *>(p->ws.ptr);
    T2 *Mf[3], *Mi[3];
    double *lam[3];
    for (int a = 0; a < 3; ++a) {
        Mf[a] = reinterpret_cast<T2 *>(ws + L.Mf[a]);
        Mi[a] = reinterpret_cast<T2 *>(ws + L.Mi[a]);
        lam[a] = reinterpret_cast<double *>(ws + L.lam[a]);
    }
    T *f = reinterpret_cast<T *>(ws + L.f);
    T2 *A = reinterpret_cast<T2 *>(ws + L.A);
    T2 *B = reinterpret_cast<T2 *>(ws + L.B);
    const bool f32 = sizeof(T) == 4;
    const int blocks = 4 * p->num_sms;
    const T2 *F;
    if (f32) {
        T2 *Fw = reinterpret_cast<T2 *>(ws + L.F);
        if (int rc = prof_begin(p, PK_BLOCH_OTHER, s)) return rc;
        bloch_to_f32_kernel<<<blocks, 256, 0, s>>>(reinterpret_cast<const double2 *>(phi),
                                                   reinterpret_cast<float2 *>(Fw), N * n_vec);
        KX_LAUNCH_CHECK("bloch_to_f32_kernel launch");
        if (int rc = prof_end(p, s)) return rc;
        F = Fw;
    } else {
        F = reinterpret_cast<const T2 *>(phi);
    }
    BlochAxes ax;
    for (int a = 0; a < 3; ++a) {
        ax.n[a] = p->n[a];
        ax.h[a] = p->h[a];
        ax.bc[a] = p->bc[a];
        ax.V[a] = p->d_V[a];
        ax.lam[a] = p->d_lam[a];
    }
    ax.order = p->fd_order;
    const long long pairs = (long long)n_orb * n_vec;
    const double *occ_k = occ ? occ + (size_t)k * n_orb : nullptr;
    for (int q = q_begin; q < n_kpt; ++q) {
        for (int a = 0; a < 3; ++a) ax.theta[a] = theta[3 * k + a] - theta[3 * q + a];
        if (int rc = prof_begin(p, PK_BLOCH_OTHER, s)) return rc;
        bloch_basis_kernel<T><<<dim3(3, 16), 256, 0, s>>>(ax, Mf[0], Mf[1], Mf[2], Mi[0], Mi[1], Mi[2], lam[0], lam[1],
                                                lam[2]);
        KX_LAUNCH_CHECK("bloch_basis_kernel launch");
        bloch_ftable_kernel<T><<<blocks, 256, 0, s>>>(p->n[0], p->n[1], p->n[2], lam[0], lam[1], lam[2], p->kind,
                                                      p->omega, f);
        KX_LAUNCH_CHECK("bloch_ftable_kernel launch");
        const T2 *Pq;
        const double2 *psi_q = reinterpret_cast<const double2 *>(psi) + (size_t)q * n_orb * N;
        if (f32) {
            T2 *Pw = reinterpret_cast<T2 *>(ws + L.P);
            bloch_to_f32_kernel<<<blocks, 256, 0, s>>>(psi_q, reinterpret_cast<float2 *>(Pw), N * n_orb);
            KX_LAUNCH_CHECK("bloch_to_f32_kernel launch");
            Pq = Pw;
        } else {
            Pq = reinterpret_cast<const T2 *>(psi_q);
        }
        if (int rc = prof_end(p, s)) return rc;
        const double *occ_q = occ ? occ + (size_t)q * n_orb : nullptr;
        const bool reverse = out_all && q > k;
        for (long long r0 = 0; r0 < pairs; r0 += L.chunk) {
            const long long r1 = std::min(pairs, r0 + L.chunk);
            const long long R = r1 - r0;
            int rc;
            if ((rc = launch_form<T>(p, R, A, Mf[0], Pq, F, n_orb, r0, s))) return rc;
            if ((rc = launch_pipe<T, 0>(p, 1, R, A, B, Mf[1], nullptr, s))) return rc;
            if ((rc = launch_pipe<T, 1>(p, 2, R, B, A, Mf[2], f, s))) return rc;
            if ((rc = launch_pipe<T, 0>(p, 2, R, A, B, Mi[2], nullptr, s))) return rc;
            if ((rc = launch_pipe<T, 0>(p, 1, R, B, A, Mi[1], nullptr, s))) return rc;
            if ((rc = launch_pipe<T, 0>(p, 0, R, A, B, Mi[0], nullptr, s))) return rc;
            if ((rc = prof_begin(p, PK_BLOCH_OTHER, s))) return rc;
            const long long nv = (r1 - 1) / n_orb - r0 / n_orb + 1;
            const int ab = (int)std::min<long long>((nv * N + 255) / 256, 8LL * p->num_sms);
            bloch_accum_kernel<T><<<ab, 256, 0, s>>>(B, r0, r1, n_orb, Pq, occ_q, wk[q],
                                                     reinterpret_cast<double2 *>(out_k), N);
            KX_LAUNCH_CHECK("bloch_accum_kernel launch");
            if (reverse) {
                const int rb = (int)std::min<long long>((n_orb * N + 255) / 256, 8LL * p->num_sms);
                double2 *out_q = reinterpret_cast<double2 *>(out_all) + (size_t)q * n_orb * N;
                bloch_accum_rev_kernel<T><<<rb, 256, 0, s>>>(B, r0, r1, n_orb, F, occ_k, wk[k], out_q, N);
                KX_LAUNCH_CHECK("bloch_accum_rev_kernel launch");
            }
            if ((rc = prof_end(p, s))) return rc;
        }
    }
    return KX_OK;
}

// Vx of the vectors phi at k-point k (out overwritten): every q contributes.
template <typename T>
int bloch_run(kx_plan *p, int n_kpt, const double *theta, const double *wk, int n_orb, const double *psi,
              const double *occ, int k, int n_vec, const double *phi, double *out, cudaStream_t s) {
    KX_CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(double2) * p->N * (size_t)n_vec, s));
    return bloch_sweep<T>(p, n_kpt, theta, wk, n_orb, psi, occ, k, 0, n_vec, phi, out, nullptr, s);
}

// Vx psi at every k-point: the pair blocks (k, q) with q >= k are solved once
// and serve both Vx psi_k and, read conjugated, Vx psi_q.
template <typename T>
int bloch_all(kx_plan *p, int n_kpt, const double *theta, const double *wk, int n_orb, const double *psi,
              const double *occ, double *vx, double *ex, cudaStream_t s) {
    const size_t N = p->N;
    KX_CUDA_TRY(cudaMemsetAsync(vx, 0, sizeof(double2) * N * (size_t)n_orb * n_kpt, s));
    for (int k = 0; k < n_kpt; ++k) {
        const size_t off = (size_t)k * n_orb * N * 2;
        if (int rc = bloch_sweep<T>(p, n_kpt, theta, wk, n_orb, psi, occ, k, k, n_orb, psi + off, vx + off, vx, s))
            return rc;
    }
    if (!ex) return KX_OK;
    BlochLayout L = bloch_layout<T>(p, n_orb, n_orb, n_kpt);
    double *partial = reinterpret_cast<double *>(static_cast<char *>(p->ws.ptr) + L.partial);
    const int nb = 2 * p->num_sms;
    if (int rc = prof_begin(p, PK_BLOCH_OTHER, s)) return rc;
    for (int k = 0; k < n_kpt; ++k) {
        const size_t off = (size_t)k * n_orb * N;
        bloch_energy_kernel<<<nb, kEThreads, 0, s>>>(reinterpret_cast<const double2 *>(psi) + off,
                                                     reinterpret_cast<const double2 *>(vx) + off,
                                                     occ ? occ + (size_t)k * n_orb : nullptr, n_orb, (long long)N,
                                                     wk[k], partial + (size_t)k * nb);
        KX_LAUNCH_CHECK("bloch_energy_kernel launch");
    }
    bloch_energy_final_kernel<<<1, 32, 0, s>>>(partial, nb * n_kpt, 0.5 * p->dV, ex);
    KX_LAUNCH_CHECK("bloch_energy_final_kernel launch");
    return prof_end(p, s);
}

// E_x alone (Eq. 8 through Parseval): forward transforms of the pair blocks
// (k, q), q >= k, the block (q, k) counted by doubling (its coefficients are
// the conjugates), the energy sum taken in the third product's epilogue.
template <typename T>
int bloch_energy_only(kx_plan *p, int n_kpt, const double *theta, const double *wk, int n_orb, const double *psi,
                      const double *occ, double *ex, cudaStream_t s) {
    using T2 = typename Cx<T>::t;
    const long long N = (long long)p->N;
    const long long pairs = (long long)n_orb * n_orb;
    const long long chunk = bloch_layout<T>(p, n_orb, n_orb, n_kpt).chunk;
    const long long n_launch = (pairs + chunk - 1) / chunk * ((long long)n_kpt * (n_kpt + 1) / 2);
    const size_t slot = (size_t)kBMaxPerSm * p->num_sms;
    BlochLayout L = bloch_layout<T>(p, n_orb, n_orb, n_kpt, (size_t)n_launch * slot);
    if (int rc = ensure_workspace(p, L.total)) return rc;
    char *ws = static_cast<char *>(p->ws.ptr);
    T2 *Mf[3];
    double *lam[3];
    for (int a = 0; a < 3; ++a) {
        Mf[a] = reinterpret_cast<T2 *>(ws + L.Mf[a]);
        lam[a] = reinterpret_cast<double *>(ws + L.lam[a]);
    }
    T2 *Mi_unused = reinterpret_cast<T2 *>(ws + L.Mi[0]);
    T *f = reinterpret_cast<T *>(ws + L.f);
    T2 *A = reinterpret_cast<T2 *>(ws + L.A);
    T2 *B = reinterpret_cast<T2 *>(ws + L.B);
    double *partial = reinterpret_cast<double *>(ws + L.partial);
    KX_CUDA_TRY(cudaMemsetAsync(partial, 0, sizeof(double) * (size_t)n_launch * slot, s));
    const bool f32 = sizeof(T) == 4;
    const int blocks = 4 * p->num_sms;
    BlochAxes ax;
    for (int a = 0; a < 3; ++a) {
        ax.n[a] = p->n[a];
        ax.h[a] = p->h[a];
        ax.bc[a] = p->bc[a];
        ax.V[a] = p->d_V[a];
        ax.lam[a] = p->d_lam[a];
    }
    ax.order = p->fd_order;
    long long li = 0;
    for (int k = 0; k < n_kpt; ++k) {
        const double2 *psi_k = reinterpret_cast<const double2 *>(psi) + (size_t)k * n_orb * N;
        const T2 *F;
        if (int rc = prof_begin(p, PK_BLOCH_OTHER, s)) return rc;
        if (f32) {
            T2 *Fw = reinterpret_cast<T2 *>(ws + L.F);
            bloch_to_f32_kernel<<<blocks, 256, 0, s>>>(psi_k, reinterpret_cast<float2 *>(Fw), N * n_orb);
            KX_LAUNCH_CHECK("bloch_to_f32_kernel launch");
            F = Fw;
        } else {
            F = reinterpret_cast<const T2 *>(psi_k);
        }
        if (int rc = prof_end(p, s)) return rc;
        for (int q = k; q < n_kpt; ++q) {
            for (int a = 0; a < 3; ++a) ax.theta[a] = theta[3 * k + a] - theta[3 * q + a];
            if (int rc = prof_begin(p, PK_BLOCH_OTHER, s)) return rc;
            // the inverse operands are written but not used
            bloch_basis_kernel<T><<<dim3(3, 16), 256, 0, s>>>(ax, Mf[0], Mf[1], Mf[2], Mi_unused,
                                                              reinterpret_cast<T2 *>(ws + L.Mi[1]),
                                                              reinterpret_cast<T2 *>(ws + L.Mi[2]), lam[0], lam[1],
                                                              lam[2]);
            KX_LAUNCH_CHECK("bloch_basis_kernel launch");
            bloch_ftable_kernel<T><<<blocks, 256, 0, s>>>(p->n[0], p->n[1], p->n[2], lam[0], lam[1], lam[2],
                                                          p->kind, p->omega, f);
            KX_LAUNCH_CHECK("bloch_ftable_kernel launch");
            const T2 *Pq;
            const double2 *psi_q = reinterpret_cast<const double2 *>(psi) + (size_t)q * n_orb * N;
            if (f32) {
                T2 *Pw = reinterpret_cast<T2 *>(ws + L.P);
                bloch_to_f32_kernel<<<blocks, 256, 0, s>>>(psi_q, reinterpret_cast<float2 *>(Pw), N * n_orb);
                KX_LAUNCH_CHECK("bloch_to_f32_kernel launch");
                Pq = Pw;
            } else {
                Pq = reinterpret_cast<const T2 *>(psi_q);
            }
            if (int rc = prof_end(p, s)) return rc;
            EnergyArgs ea;
            ea.occ_q = occ ? occ + (size_t)q * n_orb : nullptr;
            ea.occ_k = occ ? occ + (size_t)k * n_orb : nullptr;
            ea.n_orb = n_orb;
            ea.cb = -0.5 * p->dV * wk[k] * wk[q] * (q > k ? 2.0 : 1.0);
            for (long long r0 = 0; r0 < pairs; r0 += chunk, ++li) {
                const long long R = std::min(pairs, r0 + chunk) - r0;
                ea.r0 = r0;
                ea.partial = partial + (size_t)li * slot;
                int rc;
                if ((rc = launch_form<T>(p, R, A, Mf[0], Pq, F, n_orb, r0, s)))
                    return rc;
                if ((rc = launch_pipe<T, 0>(p, 1, R, A, B, Mf[1], nullptr, s))) return rc;
                if ((rc = launch_pipe<T, 2>(p, 2, R, B, nullptr, Mf[2], f, s, ea))) return rc;
            }
        }
    }
    if (int rc = prof_begin(p, PK_BLOCH_OTHER, s)) return rc;
    bloch_energy_final_kernel<<<1, 32, 0, s>>>(partial, (int)(n_launch * slot), 1.0, ex);
    KX_LAUNCH_CHECK("bloch_energy_final_kernel launch");
    return prof_end(p, s);
}

}  // namespace

int bloch_vx_apply(kx_plan *p, int n_kpt, const double *theta, const double *wk, int n_orb, const double *psi,
                   const double *occ, int k, int n_vec, const double *phi, double *out, cudaStream_t s) {
    return p->precision == KX_FP64 ? bloch_run<double>(p, n_kpt, theta, wk, n_orb, psi, occ, k, n_vec, phi, out, s)
                                   : bloch_run<float>(p, n_kpt, theta, wk, n_orb, psi, occ, k, n_vec, phi, out, s);
}

int bloch_vx_all(kx_plan *p, int n_kpt, const double *theta, const double *wk, int n_orb, const double *psi,
                 const double *occ, double *vx, double *ex, cudaStream_t s) {
    return p->precision == KX_FP64 ? bloch_all<double>(p, n_kpt, theta, wk, n_orb, psi, occ, vx, ex, s)
                                   : bloch_all<float>(p, n_kpt, theta, wk, n_orb, psi, occ, vx, ex, s);
}

int bloch_energy(kx_plan *p, int n_kpt, const double *theta, const double *wk, int n_orb, const double *psi,
                 const double *occ, double *ex, cudaStream_t s) {
    return p->precision == KX_FP64 ? bloch_energy_only<double>(p, n_kpt, theta, wk, n_orb, psi, occ, ex, s)
                                   : bloch_energy_only<float>(p, n_kpt, theta, wk, n_orb, psi, occ, ex, s);
}

}  // namespace kx
