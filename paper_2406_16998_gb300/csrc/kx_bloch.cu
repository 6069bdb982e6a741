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
// conj(Vk), the inverse with Vk.  The six complex mode products run on the
// tensor cores (split fp16 products, float32 plans, axes of 32 or 64 points:
// the pass kernels with per-item scales, bloch_pass_kernel and
// bloch_pass0_kernel, when every axis qualifies, else bloch_tc_ws_kernel with
// per-tile scales) or on the CUDA cores (float64 for KX_FP64 plans, float32 with
// packed f32x2 FMAs otherwise: bloch_form_kernel, bloch_mode_pipe_kernel); the
// pair density is formed inside the first product and f(Lambda) is applied
// inside the third.  For Vx psi at every k-point the block of pairs (k, q),
// q > k, is solved once: read conjugated it is the block (q, k).
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

// ---- tensor-core form of the float32 products (axes of 32 or 64 points)
//
// A complex product D = A M (A: 128 pencils x n, M: n x n) is one real GEMM
// [A_r | A_i] (128 x 2n) times B = [[M_r, M_i], [-M_i, M_r]] (2n x 2n): columns
// [0, n) of the result are D_r, [n, 2n) are D_i.  Both operands are split into
// fp16 hi and lo (three products hi lo, lo hi into Da, hi hi into Db, fp32 in
// TMEM); A carries a per-tile power-of-two scale from the tile's maximum, B the
// fixed 2^14 (|M| <= 1).  Shared-memory layouts are the no-swizzle core-matrix
// layouts with both operands MN-major: A element (m, kk) at
// (m/8) 128 + (kk/8) 2048 + (kk%8) 16 + (m%8) 2 bytes, B element (kk, c) at
// (c/8) 128 + (kk/8) 32n + (kk%8) 16 + (c%8) 2 bytes.
constexpr int kTcMaxN = 64;  // axes of 32 or 64 points (epilogue halves of 16-column chunks)
constexpr int kTcLd = 130;  // float2 row stride of the fp32 tile (128 pencils + 2: 16-byte rows)

__host__ __device__ inline size_t tc_b_bytes(int n) { return (size_t)8 * n * n; }      // one of hi / lo
__host__ __device__ inline size_t tc_a_bytes(int n) { return (size_t)512 * n; }        // one of hi / lo
__host__ __device__ inline size_t tc_s_bytes(int n) { return (size_t)8 * n * kTcLd; }  // fp32 tile
__host__ __device__ inline size_t tc_smem_bytes(int n) {
    return 1024 + 2 * tc_b_bytes(n) + 2 * tc_a_bytes(n) + tc_s_bytes(n);
}

// B = [[M_r, M_i], [-M_i, M_r]] 2^14 split into fp16 hi (first 4n^2 halves) and lo.
__global__ void bloch_tc_bsplit_kernel(const float2 *__restrict__ M, int n, __half *__restrict__ out) {
    const int n2 = 2 * n;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n2 * n2) return;
    const int kk = e / n2, c = e - kk * n2;
    const int k = kk % n, cc = c % n;
    const float2 m = M[k * n + cc];
    float v;
    if (kk < n) v = c < n ? m.x : m.y;
    else v = c < n ? -m.y : m.x;
    v *= kVScale;
    const __half h = __float2half_rn(v);
    const __half l = __float2half_rn(v - __half2float(h));
    const size_t off = (size_t)(c >> 3) * 64 + (size_t)(kk >> 3) * (16 * n) + (kk & 7) * 8 + (c & 7);  // halves
    out[off] = h;
    out[(size_t)4 * n * n + off] = l;
}

__device__ __forceinline__ void tc_split_store(uint8_t *hi, uint8_t *lo, int off, const float *w) {
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

// Persistent, one CTA per SM, 256 threads; tiles of 128 pencils, strided.  Per
// tile: its maximum over the fp32 tile in shared memory, the split A, one
// thread issuing the 3 x 2n/16 products and, while they run, the next tile's
// fp32 values copied in (cp.async, or formed from P and F when FORM) and this
// tile's f(Lambda) values fetched (EPI 1, 2); then a bounded wait and an
// epilogue in which warp w reads TMEM lane quadrant w % 4 for complex columns
// [w / 4 * n / 2, + n / 2), unscales (times f for EPI 1, the energy sum for
// EPI 2) and stores from registers, consecutive pencils in consecutive lanes.
// For contiguous pencils at n = 64 (mode 1) it computes the transpose D^T =
// B^T A^T instead (same shared bytes, operand roles swapped), so that a lane
// holds one output column and consecutive lanes store consecutive addresses.
// A wait that runs out sets *status and ends the kernel.
template <bool FORM, int EPI>
__global__ void __launch_bounds__(256, 1) bloch_tc_kernel(const float2 *__restrict__ in, float2 *__restrict__ out,
                                                         int n_cols, int n, int inner,
                                                         const __half *__restrict__ Bs, const float *__restrict__ f,
                                                         const float2 *__restrict__ P, const float2 *__restrict__ F,
                                                         int n_orb, long long r0, long long N, EnergyArgs ea,
                                                         int *status, long long timeout_cycles) {
    extern __shared__ uint8_t tc_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(tc_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *Bh = smem, *Bl = Bh + tc_b_bytes(n);
    uint8_t *Ah = Bl + tc_b_bytes(n), *Al = Ah + tc_a_bytes(n);
    float2 *S = reinterpret_cast<float2 *>(Al + tc_a_bytes(n));  // [k][m], row stride kTcLd
    __shared__ uint64_t bar;
    __shared__ uint32_t tslot;
    __shared__ float s_wmax[8];
    __shared__ double s_red[8];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        ptx::tmem_alloc(&tslot, 256);
        ptx::tmem_relinquish();
    }
    if (tid == 0) {
        ptx::mbar_init(&bar, 1);
        ptx::fence_mbar_init();
    }
    {  // B hi and lo, once
        const uint4 *src = reinterpret_cast<const uint4 *>(Bs);
        uint4 *dst = reinterpret_cast<uint4 *>(Bh);
        const int n16 = (int)(2 * tc_b_bytes(n) / 16);
        for (int e = tid; e < n16; e += 256) ptx::cp_async16(dst + e, src + e, 16u);
        ptx::cp_async_commit();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = tslot;
    const int n2 = 2 * n;
    // contiguous pencils (inner == 1) at n = 64: the transposed product, so that
    // a TMEM lane holds one output column across pencils and stores coalesce
    const bool transposed = inner == 1 && n == 64 && EPI == 0;
    const uint32_t idesc = transposed ? ptx::idesc_f16(n2, 128, 1, 1) : ptx::idesc_f16(128, n2, 1, 1);
    const int n_tiles = (n_cols + 127) / 128;
    uint32_t phase = 0;
    bool ok = true;
    double e_acc = 0.0;
    // the fp32 tile t into S[k][m] (cp.async, or formed from P and F when FORM;
    // pencils past the end as zeros)
    auto load_tile = [&](int t) {
        const int q0 = t * 128;
        const int nq = min(128, n_cols - q0);
        if (FORM) {
            // four pencils per warp at a time, all their loads issued before use
            // (n is 32 or 64: one or two values per lane and pencil)
            const int ppi = (int)(N / n);
            for (int m = warp; m < 128; m += 32) {
                float2 pv[4][2], fv[4][2];
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const int mb = m + 8 * b;
#pragma unroll
                    for (int h = 0; h < 2; ++h) pv[b][h] = fv[b][h] = make_float2(0.f, 0.f);
                    if (mb < nq) {
                        const int q = q0 + mb;
                        const int r = q / ppi;
                        const long long x0 = (long long)(q - r * ppi) * n;
                        const int rr = (int)r0 + r;
                        const int vv = rr / n_orb, mm = rr - vv * n_orb;
                        const float2 *Pp = P + (long long)mm * N + x0;
                        const float2 *Fp = F + (long long)vv * N + x0;
#pragma unroll
                        for (int h = 0; h < 2; ++h)
                            if (lane + 32 * h < n) {
                                pv[b][h] = Pp[lane + 32 * h];
                                fv[b][h] = Fp[lane + 32 * h];
                            }
                    }
                }
#pragma unroll
                for (int b = 0; b < 4; ++b)
#pragma unroll
                    for (int h = 0; h < 2; ++h)
                        if (lane + 32 * h < n) S[(lane + 32 * h) * kTcLd + m + 8 * b] = cmul_conj(pv[b][h], fv[b][h]);
            }
        } else if (inner == 1) {
            for (int m = warp; m < 128; m += 8) {
                float2 *row = S + m;
                if (m >= nq) {
                    for (int k = lane; k < n; k += 32) row[k * kTcLd] = make_float2(0.f, 0.f);
                    continue;
                }
                const int q = q0 + m;
                {
                    const float2 *src = in + (size_t)q * n;
                    for (int k = lane; k < n; k += 32) ptx::cp_async8(row + k * kTcLd, src + k, 8u);
                }
            }
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int m = lane + 32 * j;
                if (m >= nq) {
                    for (int k = warp; k < n; k += 8) S[k * kTcLd + m] = make_float2(0.f, 0.f);
                    continue;
                }
                const int q = q0 + m;
                const int o = q / inner;
                const float2 *src = in + (size_t)o * n * inner + (q - o * inner);
                for (int k = warp; k < n; k += 8) ptx::cp_async8(S + k * kTcLd + m, src + (size_t)k * inner, 8u);
            }
        }
        ptx::cp_async_commit();
    };
    if (blockIdx.x < n_tiles) load_tile(blockIdx.x);
    for (int t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
        const int q0 = t * 128;
        const int nq = min(128, n_cols - q0);
        ptx::cp_async_wait<0>();
        __syncthreads();
        // 1. the tile's maximum and the A scale
        float mx = 0.f;
        for (int e = tid; e < n * 64; e += 256) {  // two complex values per load
            const float4 v = reinterpret_cast<const float4 *>(S + (e >> 6) * kTcLd)[e & 63];
            mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
        }
        for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if (lane == 0) s_wmax[warp] = mx;
        __syncthreads();
        mx = s_wmax[0];
#pragma unroll
        for (int w = 1; w < 8; ++w) mx = fmaxf(mx, s_wmax[w]);
        // scale 2^e with e = 14 - exponent(max), capped at 100 so that it and
        // its inverse stay finite: a tile below 2^-86 (vacuum far from the
        // orbitals) then loses at most its own values, under 2^-100 of any
        // normal tile
        int ex = 0;
        if (mx > 0.f && isfinite(mx)) frexpf(mx, &ex);
        const int eA = min(14 - ex, 100);
        const float sA = ldexpf(1.f, eA);
        const float unscale = ldexpf(1.f, -eA - kVScaleExp);
        // 2. A = [A_r | A_i] sA, split
        // consecutive threads take consecutive k: their 8-pencil reads fall on
        // distinct banks (row stride 129 float2) and their 16-byte core-matrix
        // rows fill contiguous 128-byte runs
        for (int task = tid; task < n * 16; task += 256) {
            const int k = task % n, g = task / n;
            const float4 *src = reinterpret_cast<const float4 *>(S + k * kTcLd + 8 * g);
            float wr[8], wi[8];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float4 v = src[c];
                wr[2 * c] = v.x * sA;
                wi[2 * c] = v.y * sA;
                wr[2 * c + 1] = v.z * sA;
                wi[2 * c + 1] = v.w * sA;
            }
            tc_split_store(Ah, Al, g * 128 + (k >> 3) * 2048 + (k & 7) * 16, wr);
            tc_split_store(Ah, Al, g * 128 + ((n + k) >> 3) * 2048 + ((n + k) & 7) * 16, wi);
        }
        ptx::fence_proxy_async_smem();
        __syncthreads();
        // 3. products; S is free again, so the next tile loads while they run
        if (tid == 0) {
            ptx::tc_fence_after();
            const uint32_t ah0 = ptx::smem_u32(Ah), al0 = ptx::smem_u32(Al);
            const uint32_t bh0 = ptx::smem_u32(Bh), bl0 = ptx::smem_u32(Bl);
            const uint32_t gb = 32u * (uint32_t)n;  // B K-group stride
            const uint32_t da = tmem, db = tmem + (uint32_t)n2;  // n2 = 128 columns when transposed
            for (int ks = 0; ks < n2 / 16; ++ks) {
                const uint64_t ah = ptx::sdesc(ah0 + 4096u * ks, 2048, 128), al = ptx::sdesc(al0 + 4096u * ks, 2048, 128);
                const uint64_t bh = ptx::sdesc(bh0 + 2u * gb * ks, gb, 128), bl = ptx::sdesc(bl0 + 2u * gb * ks, gb, 128);
                if (transposed) {  // D^T = B^T A^T: the same shared bytes, operand roles swapped
                    ptx::mma_f16(da, bh, al, idesc, ks > 0 ? 1u : 0u);
                    ptx::mma_f16(da, bl, ah, idesc, 1u);
                    ptx::mma_f16(db, bh, ah, idesc, ks > 0 ? 1u : 0u);
                } else {
                    ptx::mma_f16(da, ah, bl, idesc, ks > 0 ? 1u : 0u);
                    ptx::mma_f16(da, al, bh, idesc, 1u);
                    ptx::mma_f16(db, ah, bh, idesc, ks > 0 ? 1u : 0u);
                }
            }
            ptx::mma_commit(&bar);
        }
        if (t + (int)gridDim.x < n_tiles) load_tile(t + gridDim.x);
        // EPI 1 and 2: this thread's f(Lambda) values (row m, its n / 2 columns),
        // fetched while the products run
        float fpre[kTcMaxN / 2];
        if constexpr (EPI != 0) {
            const int m = 32 * (warp & 3) + lane, hh = warp >> 2;
            const int q = q0 + min(m, nq - 1);
            const int i_in = q - (q / inner) * inner;
#pragma unroll
            for (int c = 0; c < kTcMaxN / 2; ++c)
                fpre[c] = c < (n >> 1) ? f[(size_t)(hh * (n >> 1) + c) * inner + i_in] : 0.f;
        }
        ok = __syncthreads_and(ptx::mbar_wait_bounded(&bar, phase, timeout_cycles));
        phase ^= 1u;
        if (!ok) break;
        ptx::tc_fence_after();
        // 4. epilogue: TMEM -> registers -> global
        if (transposed) {
            // lane row c' of D^T: real (c' < n) or imaginary part of column c' mod n;
            // warp halves take pencils [0, 64) and [64, 128)
            const int qd = warp & 3, hh = warp >> 2;
            const int cr = 32 * qd + lane;
            const int im = cr >= n ? 1 : 0;
            const int c = cr - im * n;
            const uint32_t tl = tmem + ((uint32_t)(32 * qd) << 16);
            float *ob = reinterpret_cast<float *>(out + (size_t)q0 * n + c) + im;
            for (int m0 = 64 * hh; m0 < 64 * hh + 64; m0 += 16) {
                float va[16], vb[16];
                ptx::tmem_ld16x2(tl + (uint32_t)m0, tl + (uint32_t)(n2 + m0), va, vb);
#pragma unroll
                for (int j = 0; j < 16; ++j)
                    if (m0 + j < nq) ob[(size_t)(m0 + j) * 2 * n] = (va[j] + vb[j]) * unscale;
            }
        } else {
            // complex column c of row m
            const int qd = warp & 3, hh = warp >> 2;
            const int m = 32 * qd + lane;
            const uint32_t tl = tmem + ((uint32_t)(32 * qd) << 16);
            const int half = n >> 1;
            const bool valid = m < nq;
            const int q = q0 + min(m, nq - 1);
            const int item = q / inner;
            const int i_in = q - item * inner;
            float2 *dst = inner == 1 ? out + (size_t)q * n : out + (size_t)item * n * inner + i_in;
            double wj = 0.0;
            if constexpr (EPI == 2) {
                const long long rr = ea.r0 + item;
                const long long vv = rr / ea.n_orb, mm = rr - vv * ea.n_orb;
                wj = valid ? ea.cb * (ea.occ_q ? ea.occ_q[mm] : 1.0) * (ea.occ_k ? ea.occ_k[vv] : 1.0) : 0.0;
            }
            float ej = 0.f;
            // half is 16 or 32: one or two chunks of 16 columns (indices fixed at
            // compile time so that fpre stays in registers)
#pragma unroll
            for (int cc = 0; cc < kTcMaxN / 32; ++cc) {
                if (16 * cc >= half) break;
                const int c0 = hh * half + 16 * cc;
                float ra[16], rb[16], ia[16], ib[16];
                ptx::tmem_ld16x2(tl + (uint32_t)c0, tl + (uint32_t)(n2 + c0), ra, rb);
                ptx::tmem_ld16x2(tl + (uint32_t)(n + c0), tl + (uint32_t)(n2 + n + c0), ia, ib);
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    float2 v = make_float2((ra[c] + rb[c]) * unscale, (ia[c] + ib[c]) * unscale);
                    if constexpr (EPI == 1) {
                        const float fv = fpre[16 * cc + c];
                        v.x *= fv;
                        v.y *= fv;
                    }
                    if constexpr (EPI == 2) {
                        const float fv = fpre[16 * cc + c];
                        ej = fmaf(fv, v.x * v.x + v.y * v.y, ej);
                    } else if (valid) {
                        dst[(size_t)(c0 + c) * inner] = v;
                    }
                }
            }
            if constexpr (EPI == 2) e_acc += wj * (double)ej;
        }
        ptx::tc_fence_before();
    }
    if (!ok) {
        if (tid == 0) atomicExch(status, KX_ERR_TIMEOUT);
        // the products whose wait ran out finish before TMEM is released
        ptx::mbar_wait_bounded(&bar, phase ^ 1u, timeout_cycles);
    }
    ptx::cp_async_wait<0>();
    if constexpr (EPI == 2) {
        for (int o = 16; o > 0; o >>= 1) e_acc += __shfl_xor_sync(0xffffffffu, e_acc, o);
        if (lane == 0) s_red[warp] = e_acc;
    }
    ptx::tc_fence_before();
    __syncthreads();
    if constexpr (EPI == 2) {
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < 8; ++w) t += s_red[w];
            ea.partial[blockIdx.x] = t;
        }
    }
    if (warp == 0) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, 256);
    }
}

// Warp-specialised form of bloch_tc_kernel (same operands, layouts, scales and
// arithmetic): 8 epilogue warps (0-7, TMEM lane quadrant w % 4, complex
// columns [w / 4 * n / 2, + n / 2), or in transposed mode pencils [64 (w / 4),
// + 64)) and 4 producer warps (8-11).  Two TMEM slots of 256 columns: while the
// epilogue drains tile i from slot i & 1, the producers take tile i + 1's
// maximum, wait until tile i's products have read A, split tile i + 1 into A,
// issue its products into the other slot (once the epilogue has freed it) and
// copy tile i + 2 into the fp32 tile.  The tile's scale exponent goes to the
// epilogue through shared memory and a per-slot mbarrier.  Every wait is
// bounded; producers agree on the outcome of theirs with a barrier vote.
constexpr int kTwEpiWarps = 8, kTwProdWarps = 8;
constexpr int kTwThreads = 32 * (kTwEpiWarps + kTwProdWarps);
constexpr int kTwProd = 32 * kTwProdWarps;

template <bool FORM, int EPI>
__global__ void __launch_bounds__(kTwThreads, 1) bloch_tc_ws_kernel(
    const float2 *__restrict__ in, float2 *__restrict__ out, int n_cols, int n, int inner,
    const __half *__restrict__ Bs, const float *__restrict__ f, const float2 *__restrict__ P,
    const float2 *__restrict__ F, int n_orb, long long r0, long long N, EnergyArgs ea, int *status,
    long long timeout_cycles) {
    extern __shared__ uint8_t tc_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(tc_raw) + 1023) & ~uintptr_t(1023));
    uint8_t *Bh = smem, *Bl = Bh + tc_b_bytes(n);
    uint8_t *Ah = Bl + tc_b_bytes(n), *Al = Ah + tc_a_bytes(n);
    float2 *S = reinterpret_cast<float2 *>(Al + tc_a_bytes(n));  // [k][m], row stride kTcLd
    __shared__ uint64_t mma_done[2], epi_done[2], sc_full[2], drain;
    __shared__ int s_eA[2];
    __shared__ uint32_t tslot;
    __shared__ float s_wmax[kTwProdWarps];
    __shared__ double s_red[kTwEpiWarps];
    __shared__ volatile int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == 0) {
        ptx::tmem_alloc(&tslot, 512);
        ptx::tmem_relinquish();
    }
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            ptx::mbar_init(&mma_done[b], 1);
            ptx::mbar_init(&epi_done[b], 32 * kTwEpiWarps);
            ptx::mbar_init(&sc_full[b], 1);
        }
        ptx::mbar_init(&drain, 1);
        ptx::fence_mbar_init();
        s_abort = 0;
    }
    if (warp >= kTwEpiWarps) {  // B hi and lo, once (its copies complete before the first split)
        const uint4 *src = reinterpret_cast<const uint4 *>(Bs);
        uint4 *dst = reinterpret_cast<uint4 *>(Bh);
        const int n16 = (int)(2 * tc_b_bytes(n) / 16);
        for (int e = tid - 32 * kTwEpiWarps; e < n16; e += kTwProd) ptx::cp_async16(dst + e, src + e, 16u);
        ptx::cp_async_commit();
    }
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = tslot;
    const int n2 = 2 * n;
    const bool transposed = inner == 1 && n == 64 && EPI == 0;
    const uint32_t idesc = transposed ? ptx::idesc_f16(n2, 128, 1, 1) : ptx::idesc_f16(128, n2, 1, 1);
    const int n_tiles = (n_cols + 127) / 128;
    const int n_my = blockIdx.x < n_tiles ? (n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;
    auto timed_out = [&]() {
        s_abort = 1;
        atomicExch(status, KX_ERR_TIMEOUT);
    };
    auto wait = [&](uint64_t *bar, uint32_t parity) {
        const long long t0 = clock64();
        while (!ptx::mbar_try_wait(bar, parity)) {
            if (s_abort) return false;
            if (clock64() - t0 > timeout_cycles) {
                timed_out();
                return false;
            }
        }
        return true;
    };
    double e_acc = 0.0;

    if (warp >= kTwEpiWarps) {
        // ------------------------------------------------------------ producers
        const int pt = tid - 32 * kTwEpiWarps, pw = warp - kTwEpiWarps;
        // the fp32 tile of local tile i into S[k][m] (cp.async, or formed from P
        // and F when FORM; pencils past the end as zeros)
        auto load_tile = [&](int i) {
            const int q0 = (blockIdx.x + i * gridDim.x) * 128;
            const int nq = min(128, n_cols - q0);
            if (FORM) {
                const int ppi = (int)(N / n);
                for (int m0 = pw; m0 < 128; m0 += 4 * kTwProdWarps) {
                    float2 pv[4][2], fv[4][2];
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int mb = m0 + kTwProdWarps * b;
#pragma unroll
                        for (int h = 0; h < 2; ++h) pv[b][h] = fv[b][h] = make_float2(0.f, 0.f);
                        if (mb < nq) {
                            const int q = q0 + mb;
                            const int r = q / ppi;
                            const long long x0 = (long long)(q - r * ppi) * n;
                            const int rr = (int)r0 + r;
                            const int vv = rr / n_orb, mm = rr - vv * n_orb;
                            const float2 *Pp = P + (long long)mm * N + x0;
                            const float2 *Fp = F + (long long)vv * N + x0;
#pragma unroll
                            for (int h = 0; h < 2; ++h)
                                if (lane + 32 * h < n) {
                                    pv[b][h] = Pp[lane + 32 * h];
                                    fv[b][h] = Fp[lane + 32 * h];
                                }
                        }
                    }
#pragma unroll
                    for (int b = 0; b < 4; ++b)
#pragma unroll
                        for (int h = 0; h < 2; ++h)
                            if (lane + 32 * h < n)
                                S[(lane + 32 * h) * kTcLd + m0 + kTwProdWarps * b] = cmul_conj(pv[b][h], fv[b][h]);
                }
            } else if (inner == 1) {
                for (int m = pw; m < 128; m += kTwProdWarps) {
                    float2 *row = S + m;
                    if (m >= nq) {
                        for (int k = lane; k < n; k += 32) row[k * kTcLd] = make_float2(0.f, 0.f);
                        continue;
                    }
                    const float2 *src = in + (size_t)(q0 + m) * n;
                    for (int k = lane; k < n; k += 32) ptx::cp_async8(row + k * kTcLd, src + k, 8u);
                }
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int m = lane + 32 * j;
                    if (m >= nq) {
                        for (int k = pw; k < n; k += kTwProdWarps) S[k * kTcLd + m] = make_float2(0.f, 0.f);
                        continue;
                    }
                    const int q = q0 + m;
                    const int o = q / inner;
                    const float2 *src = in + (size_t)o * n * inner + (q - o * inner);
                    for (int k = pw; k < n; k += kTwProdWarps)
                        ptx::cp_async8(S + k * kTcLd + m, src + (size_t)k * inner, 8u);
                }
            }
            ptx::cp_async_commit();
        };
        const uint32_t ah0 = ptx::smem_u32(Ah), al0 = ptx::smem_u32(Al);
        const uint32_t bh0 = ptx::smem_u32(Bh), bl0 = ptx::smem_u32(Bl);
        const uint32_t gb = 32u * (uint32_t)n;  // B K-group stride
        if (n_my > 0) load_tile(0);
        bool ok = true;
        for (int i = 0; i < n_my && ok; ++i) {
            const int sl = i & 1;
            ptx::cp_async_wait<0>();
            ok = ptx::named_bar_and(1, kTwProd, !s_abort);
            if (!ok) break;
            // 1. the tile's maximum and the A scale (capped at 2^100, as in bloch_tc_kernel)
            float mx = 0.f;
            for (int e = pt; e < n * 64; e += kTwProd) {  // two complex values per load
                const float4 v = reinterpret_cast<const float4 *>(S + (e >> 6) * kTcLd)[e & 63];
                mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
            }
            for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if (lane == 0) s_wmax[pw] = mx;
            // A is free once tile i - 1's products have completed
            bool w_ok = i == 0 || wait(&mma_done[sl ^ 1], (uint32_t)(((i - 1) >> 1) & 1));
            ok = ptx::named_bar_and(1, kTwProd, w_ok);
            if (!ok) break;
            mx = s_wmax[0];
#pragma unroll
            for (int w = 1; w < kTwProdWarps; ++w) mx = fmaxf(mx, s_wmax[w]);
            int ex = 0;
            if (mx > 0.f && isfinite(mx)) frexpf(mx, &ex);
            const int eA = min(14 - ex, 100);
            const float sA = ldexpf(1.f, eA);
            // 2. A = [A_r | A_i] sA, split
            for (int task = pt; task < n * 16; task += kTwProd) {
                const int k = task % n, g = task / n;
                const float4 *src = reinterpret_cast<const float4 *>(S + k * kTcLd + 8 * g);
                float wr[8], wi[8];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    const float4 v = src[c];
                    wr[2 * c] = v.x * sA;
                    wi[2 * c] = v.y * sA;
                    wr[2 * c + 1] = v.z * sA;
                    wi[2 * c + 1] = v.w * sA;
                }
                tc_split_store(Ah, Al, g * 128 + (k >> 3) * 2048 + (k & 7) * 16, wr);
                tc_split_store(Ah, Al, g * 128 + ((n + k) >> 3) * 2048 + ((n + k) & 7) * 16, wi);
            }
            ptx::fence_proxy_async_smem();
            // 3. products into slot sl once the epilogue has drained it (tile i - 2)
            w_ok = i < 2 || pt != 0 || wait(&epi_done[sl], (uint32_t)(((i - 2) >> 1) & 1));
            ok = ptx::named_bar_and(1, kTwProd, w_ok);
            if (!ok) break;
            if (pt == 0) {
                s_eA[sl] = eA;
                ptx::mbar_arrive(&sc_full[sl]);
                ptx::tc_fence_after();
                const uint32_t da = tmem + 256u * (uint32_t)sl, db = da + (uint32_t)n2;
                for (int ks = 0; ks < n2 / 16; ++ks) {
                    const uint64_t ah = ptx::sdesc(ah0 + 4096u * ks, 2048, 128),
                                   al = ptx::sdesc(al0 + 4096u * ks, 2048, 128);
                    const uint64_t bh = ptx::sdesc(bh0 + 2u * gb * ks, gb, 128),
                                   bl = ptx::sdesc(bl0 + 2u * gb * ks, gb, 128);
                    if (transposed) {  // D^T = B^T A^T: the same shared bytes, operand roles swapped
                        ptx::mma_f16(da, bh, al, idesc, ks > 0 ? 1u : 0u);
                        ptx::mma_f16(da, bl, ah, idesc, 1u);
                        ptx::mma_f16(db, bh, ah, idesc, ks > 0 ? 1u : 0u);
                    } else {
                        ptx::mma_f16(da, ah, bl, idesc, ks > 0 ? 1u : 0u);
                        ptx::mma_f16(da, al, bh, idesc, 1u);
                        ptx::mma_f16(db, ah, bh, idesc, ks > 0 ? 1u : 0u);
                    }
                }
                ptx::mma_commit(&mma_done[sl]);
            }
            // 4. S is free: the next tile loads while the products and the epilogue run
            if (i + 1 < n_my) load_tile(i + 1);
        }
        ptx::cp_async_wait<0>();
        if (pt == 0 && s_abort) {
            // a wait gave up: the products already issued finish before TMEM is released
            ptx::mma_commit(&drain);
            ptx::mbar_wait_bounded(&drain, 0, timeout_cycles);
        }
    } else {
        // ------------------------------------------------------------ epilogue
        for (int i = 0; i < n_my; ++i) {
            const int sl = i & 1;
            const int q0 = (blockIdx.x + i * gridDim.x) * 128;
            const int nq = min(128, n_cols - q0);
            // EPI 1 and 2: this thread's f(Lambda) values (row m, its n / 2 columns),
            // fetched before the products are waited for
            float fpre[kTcMaxN / 2];
            if constexpr (EPI != 0) {
                const int m = 32 * (warp & 3) + lane, hh = warp >> 2;
                const int q = q0 + min(m, nq - 1);
                const int i_in = q - (q / inner) * inner;
#pragma unroll
                for (int c = 0; c < kTcMaxN / 2; ++c)
                    fpre[c] = c < (n >> 1) ? f[(size_t)(hh * (n >> 1) + c) * inner + i_in] : 0.f;
            }
            const uint32_t par = (uint32_t)((i >> 1) & 1);
            const bool ok = __all_sync(0xffffffffu, wait(&sc_full[sl], par) && wait(&mma_done[sl], par));
            if (!ok) break;
            ptx::tc_fence_after();
            const float unscale = ldexpf(1.f, -s_eA[sl] - kVScaleExp);
            const uint32_t slot = tmem + 256u * (uint32_t)sl;
            if (transposed) {
                const int qd = warp & 3, hh = warp >> 2;
                const int cr = 32 * qd + lane;
                const int im = cr >= n ? 1 : 0;
                const int c = cr - im * n;
                const uint32_t tl = slot + ((uint32_t)(32 * qd) << 16);
                float *ob = reinterpret_cast<float *>(out + (size_t)q0 * n + c) + im;
                for (int m0 = 64 * hh; m0 < 64 * hh + 64; m0 += 16) {
                    float va[16], vb[16];
                    ptx::tmem_ld16x2(tl + (uint32_t)m0, tl + (uint32_t)(n2 + m0), va, vb);
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (m0 + j < nq) ob[(size_t)(m0 + j) * 2 * n] = (va[j] + vb[j]) * unscale;
                }
            } else {
                const int qd = warp & 3, hh = warp >> 2;
                const int m = 32 * qd + lane;
                const uint32_t tl = slot + ((uint32_t)(32 * qd) << 16);
                const int half = n >> 1;
                const bool valid = m < nq;
                const int q = q0 + min(m, nq - 1);
                const int item = q / inner;
                const int i_in = q - item * inner;
                float2 *dst = inner == 1 ? out + (size_t)q * n : out + (size_t)item * n * inner + i_in;
                double wj = 0.0;
                if constexpr (EPI == 2) {
                    const long long rr = ea.r0 + item;
                    const long long vv = rr / ea.n_orb, mm = rr - vv * ea.n_orb;
                    wj = valid ? ea.cb * (ea.occ_q ? ea.occ_q[mm] : 1.0) * (ea.occ_k ? ea.occ_k[vv] : 1.0) : 0.0;
                }
                float ej = 0.f;
#pragma unroll
                for (int cc = 0; cc < kTcMaxN / 32; ++cc) {
                    if (16 * cc >= half) break;
                    const int c0 = hh * half + 16 * cc;
                    float ra[16], rb[16], ia[16], ib[16];
                    ptx::tmem_ld16x2(tl + (uint32_t)c0, tl + (uint32_t)(n2 + c0), ra, rb);
                    ptx::tmem_ld16x2(tl + (uint32_t)(n + c0), tl + (uint32_t)(n2 + n + c0), ia, ib);
#pragma unroll
                    for (int c = 0; c < 16; ++c) {
                        float2 v = make_float2((ra[c] + rb[c]) * unscale, (ia[c] + ib[c]) * unscale);
                        if constexpr (EPI == 1) {
                            const float fv = fpre[16 * cc + c];
                            v.x *= fv;
                            v.y *= fv;
                        }
                        if constexpr (EPI == 2) {
                            const float fv = fpre[16 * cc + c];
                            ej = fmaf(fv, v.x * v.x + v.y * v.y, ej);
                        } else if (valid) {
                            dst[(size_t)(c0 + c) * inner] = v;
                        }
                    }
                }
                if constexpr (EPI == 2) e_acc += wj * (double)ej;
            }
            ptx::tc_fence_before();
            ptx::mbar_arrive(&epi_done[sl]);
        }
        if constexpr (EPI == 2) {
            for (int o = 16; o > 0; o >>= 1) e_acc += __shfl_xor_sync(0xffffffffu, e_acc, o);
            if (lane == 0) s_red[warp] = e_acc;
        }
    }
    ptx::tc_fence_before();
    __syncthreads();
    if constexpr (EPI == 2) {
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < kTwEpiWarps; ++w) t += s_red[w];
            ea.partial[blockIdx.x] = t;
        }
    }
    if (warp == 0) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, 512);
    }
}

// ---- tensor-core products of strided pencils (axes 2 and 3) with per-item scales
//
// Same operands and arithmetic as bloch_tc_kernel (A = [A_r | A_i], the split B,
// three products into Da and Db), but A is written straight from registers:
// along axes 2 and 3 the 8 pencils of a group are one contiguous 64-byte run for
// each k, which a producer thread loads, scales by the power of two of its
// item's maximum, splits and stores as the real (kk = k) and imaginary
// (kk = n + k) core-matrix rows.  Item maxima come from the previous product's
// epilogue (each epilogue records the largest component it writes, per item) or,
// for the first of these products, from the bound sqrt(n1) max|psi_m| max|phi_v|
// on the mode-1 output (the Bloch bases are unitary).  Warp roles follow the
// Gamma-point pass kernels: 8 epilogue warps (TMEM lane quadrant w % 4, complex
// columns [w / 4 n / 2, + n / 2)), 8 producer warps in two groups of four that
// take alternate tiles (group g fills A stage g), one MMA warp, two TMEM slots.
// A's core matrices sit 144 bytes apart along the pencils, so that the 16-byte
// rows the producers write for one k land on distinct bank groups:
//   A element (m, kk) at (m/8) 144 + (kk/8) 2304 + (kk%8) 16 + (m%8) 2 bytes.
constexpr int kBpEpiWarps = 8, kBpProdWarps = 8, kBpGroupThreads = 128;
constexpr int kBpMmaWarp = kBpEpiWarps + kBpProdWarps;
constexpr int kBpThreads = 32 * (kBpMmaWarp + 1);
constexpr int kBpCore = 144;
constexpr int kBpU = 4;  // producer tasks (64 bytes each) in flight per thread
__host__ __device__ inline size_t bp_a_bytes(int n) { return (size_t)(n / 4) * 16 * kBpCore; }  // one of hi / lo
__host__ __device__ inline size_t bp_smem_bytes(int n) { return 1024 + 2 * tc_b_bytes(n) + 4 * bp_a_bytes(n); }

struct BpArgs {
    const float2 *in;
    float2 *out;
    int n, inner;
    long long n_cols, ppi;  // pencils, pencils per item (N / n)
    const __half *Bs;
    const float *f;
    const float *in_max;                 // per item; nullptr: the bound below
    const float *pmax, *fmax;            // bound of item r: mul pmax[m] fmax[v], r0 + r = v n_orb + m
    float bound_mul;
    long long r0;
    int n_orb;
    float *out_max;                      // per item, zeroed by the caller (nullable)
    EnergyArgs ea;
    int *status;
    long long timeout_cycles;
};

// Maximum of an item's input, and its split exponent: e with max 2^e < 2^14,
// capped at 100 (as the per-tile scale of bloch_tc_kernel) so that it and its
// inverse stay finite.  Pencil counts are below 2^31 (checked at launch), so
// the index arithmetic of this kernel uses 32-bit division.
__device__ __forceinline__ float bp_item_max(const BpArgs &a, unsigned item) {
    if (a.in_max) return a.in_max[item];
    const long long r = a.r0 + item;
    const long long v = r / a.n_orb, m = r - v * a.n_orb;
    return a.bound_mul * a.pmax[m] * a.fmax[v];
}
__device__ __forceinline__ int bp_exp(float mx) {
    int ex = 0;
    if (mx > 0.f && isfinite(mx)) frexpf(mx, &ex);
    return min(14 - ex, 100);
}

template <int EPI>
__global__ void __launch_bounds__(kBpThreads, 1) bloch_pass_kernel(const BpArgs a) {
    extern __shared__ uint8_t bp_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(bp_raw) + 1023) & ~uintptr_t(1023));
    const int n = a.n, n2 = 2 * n;
    uint8_t *Bh = smem, *Bl = Bh + tc_b_bytes(n);
    uint8_t *stage0 = Bl + tc_b_bytes(n);  // stage s: hi at stage0 + 2 s ab, lo ab further
    const size_t ab = bp_a_bytes(n);
    __shared__ uint64_t full[2], empty[2], tfull[2], tempty[2], drain;
    __shared__ uint32_t tslot;
    __shared__ volatile int s_abort;
    __shared__ double s_red[kBpEpiWarps];
    __shared__ const float2 *s_p0[2][16];
    __shared__ float s_sc[2][16];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == kBpMmaWarp) {
        ptx::tmem_alloc(&tslot, 512);
        ptx::tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            ptx::mbar_init(&full[s], kBpGroupThreads);
            ptx::mbar_init(&empty[s], 1);
            ptx::mbar_init(&tfull[s], 1);
            ptx::mbar_init(&tempty[s], 32 * kBpEpiWarps);
        }
        ptx::mbar_init(&drain, 1);
        ptx::fence_mbar_init();
        s_abort = 0;
    }
    {  // B hi and lo, once
        const uint4 *src = reinterpret_cast<const uint4 *>(a.Bs);
        uint4 *dst = reinterpret_cast<uint4 *>(Bh);
        const int n16 = (int)(2 * tc_b_bytes(n) / 16);
        for (int e = tid; e < n16; e += kBpThreads) dst[e] = __ldg(src + e);
    }
    ptx::fence_proxy_async_smem();
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = tslot;
    const long long n_tiles = (a.n_cols + 127) / 128;
    const int n_my = (int)((n_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x);
    auto wait = [&](uint64_t *bar, uint32_t parity) {
        const long long t0 = clock64();
        while (!ptx::mbar_try_wait(bar, parity)) {
            if (s_abort) return false;
            if (clock64() - t0 > a.timeout_cycles) {
                s_abort = 1;
                atomicExch(a.status, KX_ERR_TIMEOUT);
                return false;
            }
        }
        return true;
    };

    if (warp == kBpMmaWarp) {
        // ---------------------------------------------------------------- MMA issue
        if (lane == 0) {
            const uint32_t idesc = ptx::idesc_f16(128, n2, 1, 1);
            const uint32_t bh0 = ptx::smem_u32(Bh), bl0 = ptx::smem_u32(Bl);
            const uint32_t gb = 32u * (uint32_t)n;  // B K-group stride
            bool ok = true;
            for (int it = 0; it < n_my && ok; ++it) {
                const int s = it & 1;  // A stage and TMEM slot
                ok = wait(&full[s], (uint32_t)((it >> 1) & 1));
                if (ok && it >= 2) ok = wait(&tempty[s], (uint32_t)(((it >> 1) - 1) & 1));
                if (!ok) break;
                ptx::tc_fence_after();
                const uint32_t ah0 = ptx::smem_u32(stage0 + 2 * s * ab), al0 = ah0 + (uint32_t)ab;
                const uint32_t da = tmem + 256u * (uint32_t)s, db = da + (uint32_t)n2;
                for (int ks = 0; ks < n2 / 16; ++ks) {
                    const uint32_t ao = (uint32_t)(2 * 16 * kBpCore * ks);
                    const uint64_t ah = ptx::sdesc(ah0 + ao, 16 * kBpCore, kBpCore),
                                   al = ptx::sdesc(al0 + ao, 16 * kBpCore, kBpCore);
                    const uint64_t bh = ptx::sdesc(bh0 + 2u * gb * ks, gb, 128),
                                   bl = ptx::sdesc(bl0 + 2u * gb * ks, gb, 128);
                    ptx::mma_f16(da, ah, bl, idesc, ks > 0 ? 1u : 0u);
                    ptx::mma_f16(da, al, bh, idesc, 1u);
                    ptx::mma_f16(db, ah, bh, idesc, ks > 0 ? 1u : 0u);
                }
                ptx::mma_commit(&empty[s]);
                ptx::mma_commit(&tfull[s]);
            }
            if (!ok) {
                // a wait gave up: the products already issued finish before TMEM is released
                ptx::mma_commit(&drain);
                ptx::mbar_wait_bounded(&drain, 0, a.timeout_cycles);
            }
        }
        __syncwarp();
    } else if (warp >= kBpEpiWarps) {
        // ---------------------------------------------------------------- producers
        const int ptid = tid - 32 * kBpEpiWarps;
        const int grp = ptid / kBpGroupThreads, gtid = ptid % kBpGroupThreads;
        const int bar_id = 2 + grp;
        const int ntask = 16 * n;  // 16 pencil groups x n values of k
        const unsigned inner = (unsigned)a.inner, ppi = (unsigned)a.ppi;
        // first pencil of group g of local tile it (>= n_cols past the end) and its address
        auto gq = [&](int it, int g) { return (unsigned)((blockIdx.x + (long long)it * gridDim.x) * 128 + 8 * g); };
        auto addr = [&](unsigned q) {
            const unsigned o = q / inner;
            return a.in + (long long)o * n * inner + (q - o * inner);
        };
        // the descriptor of the group's first tile; later ones are written after
        // each tile, their item maxima loaded at its start (published by the vote
        // that opens the next iteration)
        if (gtid < 16 && grp < n_my) {
            const unsigned q = gq(grp, gtid);
            const bool in = q < a.n_cols;
            s_p0[grp][gtid] = in ? addr(q) : nullptr;
            s_sc[grp][gtid] = in ? ldexpf(1.f, bp_exp(bp_item_max(a, q / ppi))) : 0.f;
        }
        for (int it = grp; it < n_my; it += 2) {
            bool ok = it < 2 || wait(&empty[grp], (uint32_t)(((it >> 1) - 1) & 1));
            ok = ptx::named_bar_and(bar_id, kBpGroupThreads, ok && !s_abort);
            if (!ok) break;
            const bool more = it + 2 < n_my;
            float nxt_mx = 0.f;
            if (gtid < 16 && more) {
                const unsigned q = gq(it + 2, gtid);
                if (q < a.n_cols) nxt_mx = bp_item_max(a, q / ppi);
            }
            if (more) {  // the group's next tile into L2 (one 128-byte line per 16 pencils and k)
                for (int l = gtid; l < 8 * n; l += kBpGroupThreads) {
                    const unsigned q = gq(it + 2, 2 * (l & 7));
                    if (q < a.n_cols) ptx::prefetch_l2(addr(q) + (long long)(l >> 3) * inner);
                }
            }
            uint8_t *Ahi = stage0 + 2 * grp * ab, *Alo = Ahi + ab;
            for (int t0 = gtid; t0 < ntask; t0 += kBpGroupThreads * kBpU) {
                float4 v[kBpU][4];
#pragma unroll
                for (int r = 0; r < kBpU; ++r) {  // every load of the batch first
                    const int t = t0 + r * kBpGroupThreads;
                    const float2 *p = t < ntask ? s_p0[grp][t & 15] : nullptr;
                    if (p != nullptr) {
                        const float4 *src = reinterpret_cast<const float4 *>(p + (long long)(t >> 4) * a.inner);
#pragma unroll
                        for (int c = 0; c < 4; ++c) v[r][c] = __ldg(src + c);
                    } else {
#pragma unroll
                        for (int c = 0; c < 4; ++c) v[r][c] = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                }
#pragma unroll
                for (int r = 0; r < kBpU; ++r) {
                    const int t = t0 + r * kBpGroupThreads;
                    if (t >= ntask) continue;
                    const int g = t & 15, k = t >> 4;
                    const float sc = s_sc[grp][g];
                    float wr[8], wi[8];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        wr[2 * c] = v[r][c].x * sc;
                        wi[2 * c] = v[r][c].y * sc;
                        wr[2 * c + 1] = v[r][c].z * sc;
                        wi[2 * c + 1] = v[r][c].w * sc;
                    }
                    const int ki = n + k;
                    tc_split_store(Ahi, Alo, g * kBpCore + (k >> 3) * (16 * kBpCore) + (k & 7) * 16, wr);
                    tc_split_store(Ahi, Alo, g * kBpCore + (ki >> 3) * (16 * kBpCore) + (ki & 7) * 16, wi);
                }
            }
            ptx::fence_proxy_async_smem();
            ptx::mbar_arrive(&full[grp]);
            ptx::named_bar(bar_id, kBpGroupThreads);  // every thread is done with this descriptor
            if (gtid < 16 && more) {
                const unsigned q = gq(it + 2, gtid);
                const bool in = q < a.n_cols;
                s_p0[grp][gtid] = in ? addr(q) : nullptr;
                s_sc[grp][gtid] = in ? ldexpf(1.f, bp_exp(nxt_mx)) : 0.f;
            }
        }
    } else {
        // ---------------------------------------------------------------- epilogue
        const int qd = warp & 3, hh = warp >> 2;
        const int m = 32 * qd + lane;
        const int half = n >> 1;
        double e_acc = 0.0;
        for (int it = 0; it < n_my; ++it) {
            const int b = it & 1;
            const long long q0 = (blockIdx.x + (long long)it * gridDim.x) * 128;
            const int nq = (int)min(128LL, a.n_cols - q0);
            const bool valid = m < nq;
            const long long q = q0 + min(m, nq - 1);
            const long long item = q / a.ppi;
            const long long o = q / a.inner;
            const long long i_in = q - o * a.inner;
            const float unscale = ldexpf(1.f, -bp_exp(bp_item_max(a, (unsigned)item)) - kVScaleExp);
            float fpre[kTcMaxN / 2];
            if constexpr (EPI != 0) {
#pragma unroll
                for (int c = 0; c < kTcMaxN / 2; ++c)
                    fpre[c] = c < half ? a.f[(long long)(hh * half + c) * a.inner + i_in] : 0.f;
            }
            double wj = 0.0;
            if constexpr (EPI == 2) {
                const long long rr = a.ea.r0 + item;
                const long long vv = rr / a.ea.n_orb, mm = rr - vv * a.ea.n_orb;
                wj = valid ? a.ea.cb * (a.ea.occ_q ? a.ea.occ_q[mm] : 1.0) * (a.ea.occ_k ? a.ea.occ_k[vv] : 1.0)
                           : 0.0;
            }
            if (!__all_sync(0xffffffffu, wait(&tfull[b], (uint32_t)((it >> 1) & 1)))) break;
            ptx::tc_fence_after();
            const uint32_t tl = tmem + 256u * (uint32_t)b + ((uint32_t)(32 * qd) << 16);
            float2 *dst = a.out + o * n * a.inner + i_in;
            float my_max = 0.f, ej = 0.f;
            // 8 complex columns at a time (real and imaginary parts, Da and Db)
#pragma unroll
            for (int cc = 0; cc < kTcMaxN / 16; ++cc) {
                if (8 * cc >= half) break;
                const int c0 = hh * half + 8 * cc;
                float ra[8], rb[8], ia[8], ib[8];
                ptx::tmem_ld8x4(tl + (uint32_t)c0, tl + (uint32_t)(n2 + c0), tl + (uint32_t)(n + c0),
                                tl + (uint32_t)(n2 + n + c0), ra, rb, ia, ib);
#pragma unroll
                for (int c = 0; c < 8; ++c) {
                    float2 v = make_float2((ra[c] + rb[c]) * unscale, (ia[c] + ib[c]) * unscale);
                    if constexpr (EPI == 1) {
                        v.x *= fpre[8 * cc + c];
                        v.y *= fpre[8 * cc + c];
                    }
                    if constexpr (EPI == 2) {
                        ej = fmaf(fpre[8 * cc + c], v.x * v.x + v.y * v.y, ej);
                    } else if (valid) {
                        dst[(long long)(c0 + c) * a.inner] = v;
                        my_max = fmaxf(my_max, fmaxf(fabsf(v.x), fabsf(v.y)));
                    }
                }
            }
            if constexpr (EPI == 2) {
                e_acc += wj * (double)ej;
            } else if (a.out_max != nullptr) {
                // one atomic per warp when its 32 pencils belong to one item
                const long long item0 = __shfl_sync(0xffffffffu, item, 0);
                if (__all_sync(0xffffffffu, !valid || item == item0)) {
                    float r = my_max;
                    for (int off = 16; off > 0; off >>= 1) r = fmaxf(r, __shfl_xor_sync(0xffffffffu, r, off));
                    if (lane == 0 && r > 0.f) atomicMax(reinterpret_cast<int *>(a.out_max + item0), __float_as_int(r));
                } else if (valid && my_max > 0.f) {
                    atomicMax(reinterpret_cast<int *>(a.out_max + item), __float_as_int(my_max));
                }
            }
            ptx::tc_fence_before();
            ptx::mbar_arrive(&tempty[b]);
        }
        if constexpr (EPI == 2) {
            for (int off = 16; off > 0; off >>= 1) e_acc += __shfl_xor_sync(0xffffffffu, e_acc, off);
            if (lane == 0) s_red[warp] = e_acc;
        }
    }
    ptx::tc_fence_before();
    __syncthreads();
    if constexpr (EPI == 2) {
        if (tid == 0) {
            double t = 0.0;
            for (int w = 0; w < kBpEpiWarps; ++w) t += s_red[w];
            a.ea.partial[blockIdx.x] = t;
        }
    }
    if (warp == kBpMmaWarp) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, 512);
    }
}

// ---- the same for the contiguous axis (axis 1, n = 64), forward product with
// the pair density formed on the way (FORM) or inverse product
//
// The 128 pencils of a tile are contiguous in memory and belong to one item
// (pencils per item a multiple of 128), so a tile is one 64 KB run (two, P and
// F, when FORM) with one split scale.  A is K-major: a producer task loads 8
// complex values of one pencil (64 contiguous bytes) and writes its real and
// imaginary 16-byte core-matrix rows; core matrices sit 144 bytes apart along
// K, so that the 8 tasks of a pencil land on distinct bank groups:
//   A element (m, kk) at (m/8) (2n/8) 144 + (kk/8) 144 + (m%8) 16 + (kk%8) 2 bytes.
// The products compute the transpose D^T = B^T A^T (as bloch_tc_kernel does for
// contiguous pencils), so that a TMEM lane holds one output component across
// pencils and consecutive lanes store consecutive addresses.  The output feeds
// either the next product (whose scale comes from the bound sqrt(n1) max|rho|)
// or the accumulation, so no maximum is recorded.
template <bool FORM>
__global__ void __launch_bounds__(kBpThreads, 1) bloch_pass0_kernel(const BpArgs a, const float2 *__restrict__ P,
                                                                    const float2 *__restrict__ F, long long N) {
    extern __shared__ uint8_t bp_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(bp_raw) + 1023) & ~uintptr_t(1023));
    const int n = a.n, n2 = 2 * n, nkc = n / 8;
    const int sbo = (n2 / 8) * kBpCore;  // A: stride of 8-pencil groups
    uint8_t *Bh = smem, *Bl = Bh + tc_b_bytes(n);
    uint8_t *stage0 = Bl + tc_b_bytes(n);
    const size_t ab = bp_a_bytes(n);
    __shared__ uint64_t full[2], empty[2], tfull[2], tempty[2], drain;
    __shared__ uint32_t tslot;
    __shared__ volatile int s_abort;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (warp == kBpMmaWarp) {
        ptx::tmem_alloc(&tslot, 512);
        ptx::tmem_relinquish();
    }
    if (tid == 0) {
        for (int s = 0; s < 2; ++s) {
            ptx::mbar_init(&full[s], kBpGroupThreads);
            ptx::mbar_init(&empty[s], 1);
            ptx::mbar_init(&tfull[s], 1);
            ptx::mbar_init(&tempty[s], 32 * kBpEpiWarps);
        }
        ptx::mbar_init(&drain, 1);
        ptx::fence_mbar_init();
        s_abort = 0;
    }
    {  // B hi and lo, once
        const uint4 *src = reinterpret_cast<const uint4 *>(a.Bs);
        uint4 *dst = reinterpret_cast<uint4 *>(Bh);
        const int n16 = (int)(2 * tc_b_bytes(n) / 16);
        for (int e = tid; e < n16; e += kBpThreads) dst[e] = __ldg(src + e);
    }
    ptx::fence_proxy_async_smem();
    ptx::tc_fence_before();
    __syncthreads();
    ptx::tc_fence_after();
    const uint32_t tmem = tslot;
    const long long n_tiles = (a.n_cols + 127) / 128;
    const int n_my = (int)((n_tiles - blockIdx.x + gridDim.x - 1) / gridDim.x);
    const unsigned ppi = (unsigned)a.ppi;
    auto wait = [&](uint64_t *bar, uint32_t parity) {
        const long long t0 = clock64();
        while (!ptx::mbar_try_wait(bar, parity)) {
            if (s_abort) return false;
            if (clock64() - t0 > a.timeout_cycles) {
                s_abort = 1;
                atomicExch(a.status, KX_ERR_TIMEOUT);
                return false;
            }
        }
        return true;
    };
    auto tile_q0 = [&](int it) { return (unsigned)((blockIdx.x + (long long)it * gridDim.x) * 128); };

    if (warp == kBpMmaWarp) {
        // ---------------------------------------------------------------- MMA issue: D^T = B^T A^T
        if (lane == 0) {
            const uint32_t idesc = ptx::idesc_f16(n2, 128, 1, 0);
            const uint32_t bh0 = ptx::smem_u32(Bh), bl0 = ptx::smem_u32(Bl);
            const uint32_t gb = 32u * (uint32_t)n;
            bool ok = true;
            for (int it = 0; it < n_my && ok; ++it) {
                const int s = it & 1;
                ok = wait(&full[s], (uint32_t)((it >> 1) & 1));
                if (ok && it >= 2) ok = wait(&tempty[s], (uint32_t)(((it >> 1) - 1) & 1));
                if (!ok) break;
                ptx::tc_fence_after();
                const uint32_t ah0 = ptx::smem_u32(stage0 + 2 * s * ab), al0 = ah0 + (uint32_t)ab;
                const uint32_t da = tmem + 256u * (uint32_t)s, db = da + 128u;
                for (int ks = 0; ks < n2 / 16; ++ks) {
                    const uint32_t ao = (uint32_t)(2 * kBpCore * ks);
                    const uint64_t ah = ptx::sdesc(ah0 + ao, kBpCore, (uint32_t)sbo),
                                   al = ptx::sdesc(al0 + ao, kBpCore, (uint32_t)sbo);
                    const uint64_t bh = ptx::sdesc(bh0 + 2u * gb * ks, gb, 128),
                                   bl = ptx::sdesc(bl0 + 2u * gb * ks, gb, 128);
                    ptx::mma_f16(da, bh, al, idesc, ks > 0 ? 1u : 0u);
                    ptx::mma_f16(da, bl, ah, idesc, 1u);
                    ptx::mma_f16(db, bh, ah, idesc, ks > 0 ? 1u : 0u);
                }
                ptx::mma_commit(&empty[s]);
                ptx::mma_commit(&tfull[s]);
            }
            if (!ok) {
                ptx::mma_commit(&drain);
                ptx::mbar_wait_bounded(&drain, 0, a.timeout_cycles);
            }
        }
        __syncwarp();
    } else if (warp >= kBpEpiWarps) {
        // ---------------------------------------------------------------- producers
        const int ptid = tid - 32 * kBpEpiWarps;
        const int grp = ptid / kBpGroupThreads, gtid = ptid % kBpGroupThreads;
        const int bar_id = 2 + grp;
        const int ntask = 128 * nkc;  // 128 pencils x n / 8 chunks
        constexpr int U = FORM ? 2 : 4;
        // first value of the tile (its pencils are consecutive, of one item)
        auto base = [&](unsigned q0, const float2 *&p, const float2 *&f) {
            if (FORM) {
                const unsigned item = q0 / ppi;
                const long long rr = a.r0 + item;
                const long long vv = rr / a.n_orb, mm = rr - vv * a.n_orb;
                const long long x0 = (long long)(q0 - item * ppi) * n;
                p = P + mm * N + x0;
                f = F + vv * N + x0;
            } else {
                p = a.in + (long long)q0 * n;
                f = nullptr;
            }
        };
        // the item maximum of the group's next tile is loaded a tile ahead
        float mx_cur = grp < n_my ? bp_item_max(a, tile_q0(grp) / ppi) : 0.f;
        for (int it = grp; it < n_my; it += 2) {
            bool ok = it < 2 || wait(&empty[grp], (uint32_t)(((it >> 1) - 1) & 1));
            ok = ptx::named_bar_and(bar_id, kBpGroupThreads, ok && !s_abort);
            if (!ok) break;
            const unsigned q0 = tile_q0(it);
            const int nq = (int)min(128LL, a.n_cols - q0);
            const float sc = ldexpf(1.f, bp_exp(mx_cur));
            const bool more = it + 2 < n_my;
            if (more) {
                const unsigned qn = tile_q0(it + 2);
                mx_cur = bp_item_max(a, qn / ppi);
                const float2 *pn, *fn;  // the next tile into L2, one 128-byte line per thread and step
                base(qn, pn, fn);
                const int lines = (int)min(128LL, a.n_cols - qn) * n / 16;
                for (int l = gtid; l < lines; l += kBpGroupThreads) {
                    ptx::prefetch_l2(pn + 16 * l);
                    if (FORM) ptx::prefetch_l2(fn + 16 * l);
                }
            }
            const float2 *pb, *fb;
            base(q0, pb, fb);
            uint8_t *Ahi = stage0 + 2 * grp * ab, *Alo = Ahi + ab;
            for (int t0 = gtid; t0 < ntask; t0 += kBpGroupThreads * U) {
                float4 v[U][4], w[FORM ? U : 1][4];
#pragma unroll
                for (int r = 0; r < U; ++r) {  // every load of the batch first
                    const int t = t0 + r * kBpGroupThreads;
                    const int m = t / nkc, kc = t - m * nkc;
                    if (t < ntask && m < nq) {
                        const long long off = (long long)m * n + 8 * kc;
                        const float4 *sp = reinterpret_cast<const float4 *>(pb + off);
#pragma unroll
                        for (int c = 0; c < 4; ++c) v[r][c] = __ldg(sp + c);
                        if (FORM) {
                            const float4 *sf = reinterpret_cast<const float4 *>(fb + off);
#pragma unroll
                            for (int c = 0; c < 4; ++c) w[FORM ? r : 0][c] = __ldg(sf + c);
                        }
                    } else {
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            v[r][c] = make_float4(0.f, 0.f, 0.f, 0.f);
                            if (FORM) w[FORM ? r : 0][c] = make_float4(0.f, 0.f, 0.f, 0.f);
                        }
                    }
                }
#pragma unroll
                for (int r = 0; r < U; ++r) {
                    const int t = t0 + r * kBpGroupThreads;
                    if (t >= ntask) continue;
                    const int m = t / nkc, kc = t - m * nkc;
                    float wr[8], wi[8];
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        float2 x0 = make_float2(v[r][c].x, v[r][c].y), x1 = make_float2(v[r][c].z, v[r][c].w);
                        if (FORM) {
                            x0 = cmul_conj(x0, make_float2(w[FORM ? r : 0][c].x, w[FORM ? r : 0][c].y));
                            x1 = cmul_conj(x1, make_float2(w[FORM ? r : 0][c].z, w[FORM ? r : 0][c].w));
                        }
                        wr[2 * c] = x0.x * sc;
                        wi[2 * c] = x0.y * sc;
                        wr[2 * c + 1] = x1.x * sc;
                        wi[2 * c + 1] = x1.y * sc;
                    }
                    const int row = (m >> 3) * sbo + (m & 7) * 16;
                    tc_split_store(Ahi, Alo, row + kc * kBpCore, wr);
                    tc_split_store(Ahi, Alo, row + (nkc + kc) * kBpCore, wi);
                }
            }
            ptx::fence_proxy_async_smem();
            ptx::mbar_arrive(&full[grp]);
        }
    } else {
        // ---------------------------------------------------------------- epilogue
        // lane row c' of D^T: real (c' < n) or imaginary part of column c' mod n;
        // warps 0-3 take pencils [0, 64) of the tile, warps 4-7 pencils [64, 128)
        const int qd = warp & 3, hh = warp >> 2;
        const int cr = 32 * qd + lane;
        const int im = cr >= n ? 1 : 0;
        const int c = cr - im * n;
        for (int it = 0; it < n_my; ++it) {
            const int b = it & 1;
            const unsigned q0 = tile_q0(it);
            const int nq = (int)min(128LL, a.n_cols - q0);
            const float unscale = ldexpf(1.f, -bp_exp(bp_item_max(a, q0 / ppi)) - kVScaleExp);
            if (!__all_sync(0xffffffffu, wait(&tfull[b], (uint32_t)((it >> 1) & 1)))) break;
            ptx::tc_fence_after();
            const uint32_t tl = tmem + 256u * (uint32_t)b + ((uint32_t)(32 * qd) << 16);
            float *ob = reinterpret_cast<float *>(a.out + (long long)q0 * n + c) + im;
            for (int m0 = 64 * hh; m0 < 64 * hh + 64; m0 += 16) {
                float va[16], vb[16];
                ptx::tmem_ld16x2(tl + (uint32_t)m0, tl + (uint32_t)(128 + m0), va, vb);
                if (cr < n2) {
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (m0 + j < nq) ob[(long long)(m0 + j) * n2] = (va[j] + vb[j]) * unscale;
                }
            }
            ptx::tc_fence_before();
            ptx::mbar_arrive(&tempty[b]);
        }
    }
    ptx::tc_fence_before();
    __syncthreads();
    if (warp == kBpMmaWarp) {
        ptx::tc_fence_after();
        ptx::tmem_dealloc(tmem, 512);
    }
}

// max (|re| + |im|) of each of the vectors x[v] (N values each) into vmax[v]
// (zeroed before): an upper bound of the modulus, for the split scales above.
__global__ void bloch_vmax_kernel(const float2 *__restrict__ x, long long N, float *__restrict__ vmax) {
    const float2 *v = x + (long long)blockIdx.y * N;
    float m = 0.f;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < N; e += (long long)gridDim.x * blockDim.x) {
        const float2 a = v[e];
        m = fmaxf(m, fabsf(a.x) + fabsf(a.y));
    }
    for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
    if ((threadIdx.x & 31) == 0 && m > 0.f) atomicMax(reinterpret_cast<int *>(vmax + blockIdx.y), __float_as_int(m));
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
// (memory-latency bound: four orbitals' loads in flight per thread, four blocks per SM)
template <typename T>
__global__ void __launch_bounds__(256, 4) bloch_accum_kernel(const typename Cx<T>::t *__restrict__ X, long long r0, long long r1, int n_orb,
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
        // four orbitals' loads issued together, the sums still in ascending m
        long long m = m0;
        for (; m + 4 <= m1; m += 4) {
            T2 p[4], xx[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                p[u] = P[(m + u) * N + x];
                xx[u] = X[(v * n_orb + m + u - r0) * N + x];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const T c = (T)(wq * (occ_q ? occ_q[m + u] : 1.0));
                sr = fma(c, p[u].x * xx[u].x - p[u].y * xx[u].y, sr);
                si = fma(c, p[u].x * xx[u].y + p[u].y * xx[u].x, si);
            }
        }
        for (; m < m1; ++m) {
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

// The float32 forms of bloch_accum_kernel (forward sums, REV false) and
// bloch_accum_rev_kernel (reversed, REV true) with two neighbouring points per
// thread: 16-byte loads, so that each thread keeps 128 bytes of its four
// items' loads in flight (N even).  Same terms in the same order per point.
template <bool REV>
__global__ void __launch_bounds__(256, 3) bloch_accum2_kernel(const float2 *__restrict__ X, long long r0, long long r1,
                                                              int n_orb, const float2 *__restrict__ Y,
                                                              const double *__restrict__ occ, double w,
                                                              double2 *__restrict__ out, long long N) {
    const long long v_lo = r0 / n_orb, v_hi = (r1 - 1) / n_orb;
    const long long N2 = N / 2;
    // forward: one thread per (vector v, point pair), Y = P, sum over m;
    // reversed: one thread per (band m, point pair), Y = F, sum over v
    const long long rows = REV ? (long long)n_orb : v_hi - v_lo + 1;
    const long long total = rows * N2;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const long long rl = e / N2, x = 2 * (e - rl * N2);
        long long a, b;  // the summed index runs over [a, b]
        long long orow;  // output row
        if (REV) {
            const long long m = rl;
            if (r1 - 1 - m < 0) continue;
            a = max(v_lo, (r0 - m + n_orb - 1) / n_orb);
            b = min(v_hi, (r1 - 1 - m) / n_orb);
            if (a > b) continue;
            orow = m;
        } else {
            const long long v = v_lo + rl;
            a = max(0LL, r0 - v * n_orb);
            b = min((long long)n_orb, r1 - v * n_orb) - 1;
            orow = v;
        }
        // item of summed index t: forward r = orow n_orb + t, reversed r = t n_orb + orow
        auto item = [&](long long t) { return REV ? t * n_orb + orow - r0 : orow * n_orb + t - r0; };
        float sr0 = 0.f, si0 = 0.f, sr1 = 0.f, si1 = 0.f;
        auto term = [&](float c, float4 y, float4 xx) {
            if (REV) {  // Y conj(X)
                sr0 = fmaf(c, y.x * xx.x + y.y * xx.y, sr0);
                si0 = fmaf(c, y.y * xx.x - y.x * xx.y, si0);
                sr1 = fmaf(c, y.z * xx.z + y.w * xx.w, sr1);
                si1 = fmaf(c, y.w * xx.z - y.z * xx.w, si1);
            } else {  // Y X
                sr0 = fmaf(c, y.x * xx.x - y.y * xx.y, sr0);
                si0 = fmaf(c, y.x * xx.y + y.y * xx.x, si0);
                sr1 = fmaf(c, y.z * xx.z - y.w * xx.w, sr1);
                si1 = fmaf(c, y.z * xx.w + y.w * xx.z, si1);
            }
        };
        long long t = a;
        for (; t + 4 <= b + 1; t += 4) {
            float4 y[4], xx[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                y[u] = *reinterpret_cast<const float4 *>(Y + (t + u) * N + x);
                xx[u] = *reinterpret_cast<const float4 *>(X + item(t + u) * N + x);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) term((float)(w * (occ ? occ[t + u] : 1.0)), y[u], xx[u]);
        }
        for (; t <= b; ++t)
            term((float)(w * (occ ? occ[t] : 1.0)), *reinterpret_cast<const float4 *>(Y + t * N + x),
                 *reinterpret_cast<const float4 *>(X + item(t) * N + x));
        double2 *o = out + orow * N + x;
        double2 o0 = o[0], o1 = o[1];
        o0.x -= f32_to_f64(sr0);
        o0.y -= f32_to_f64(si0);
        o1.x -= f32_to_f64(sr1);
        o1.y -= f32_to_f64(si1);
        o[0] = o0;
        o[1] = o1;
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

// Tensor-core products: float32 plans, axes of 32 or 64 points (KX_BLOCH_TC, a
// tuning and test override, is a bit mask of the axes allowed to use them: 0
// none, 7 all).
inline bool tc_axis(const kx_plan *p, int axis) {
    if (p->precision == KX_FP64) return false;
    if (const char *e = std::getenv("KX_BLOCH_TC"))
        if (((std::atoi(e) >> axis) & 1) == 0) return false;
    const int n = p->n[axis];
    return n % 32 == 0 && n <= kTcMaxN;
}

template <bool FORM, int EPI>
int launch_tc(kx_plan *p, int axis, long long R, const float2 *in, float2 *out, const __half *Bs, const float *f,
              const float2 *P, const float2 *F, int n_orb, long long r0, cudaStream_t s,
              const EnergyArgs &ea = EnergyArgs()) {
    const int n = p->n[axis];
    const long long N = (long long)p->N;
    const int inner = axis == 0 ? 1 : (axis == 1 ? p->n[0] : p->n[0] * p->n[1]);
    const long long n_cols = R * (N / n);
    if (R * N >= (1LL << 31)) return set_error(KX_ERR_ARG, "Bloch exchange: chunk too large for one launch");
    const long long n_tiles = (n_cols + 127) / 128;
    const int grid = (int)std::min<long long>(n_tiles, p->num_sms);
    const size_t smem = tc_smem_bytes(n);
    static bool attr = false;  // once per instantiation
    if (!attr) {
        KX_CUDA_TRY(cudaFuncSetAttribute(bloch_tc_kernel<FORM, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tc_smem_bytes(kTcMaxN)));
        attr = true;
    }
    // warp-specialised form unless KX_BLOCH_WS=0 (comparison runs)
    const char *ws_env = std::getenv("KX_BLOCH_WS");
    const bool ws = !(ws_env && std::atoi(ws_env) == 0);
    static bool attr_ws = false;
    if (ws && !attr_ws) {
        KX_CUDA_TRY(cudaFuncSetAttribute(bloch_tc_ws_kernel<FORM, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tc_smem_bytes(kTcMaxN)));
        attr_ws = true;
    }
    if (int rc = prof_begin(p, PK_BLOCH, s)) return rc;
    if (ws)
        bloch_tc_ws_kernel<FORM, EPI><<<grid, kTwThreads, smem, s>>>(in, out, (int)n_cols, n, inner, Bs, f, P, F,
                                                                     n_orb, r0, N, ea, p->d_status, 2000000000LL);
    else
        bloch_tc_kernel<FORM, EPI><<<grid, 256, smem, s>>>(in, out, (int)n_cols, n, inner, Bs, f, P, F, n_orb, r0, N,
                                                           ea, p->d_status, 2000000000LL);
    KX_LAUNCH_CHECK("bloch_tc_kernel launch");
    return prof_end(p, s);
}

// Products along axes 2 and 3 through bloch_pass_kernel: both axes on the
// tensor cores with pencil groups of 8 contiguous values (n1 and n1 n2
// multiples of 8), unless KX_BLOCH_PASS=0 (comparison runs).
inline bool bp_axes(const kx_plan *p) {
    if (const char *e = std::getenv("KX_BLOCH_PASS"))
        if (std::atoi(e) == 0) return false;
    return tc_axis(p, 1) && tc_axis(p, 2) && p->n[0] % 8 == 0;
}

template <int EPI>
int launch_bp(kx_plan *p, int axis, long long R, const float2 *in, float2 *out, const __half *Bs, const float *f,
              const float *in_max, const float *pmax, const float *fmax, long long r0, int n_orb, float *out_max,
              cudaStream_t s, const EnergyArgs &ea = EnergyArgs()) {
    const int n = p->n[axis];
    const long long N = (long long)p->N;
    if (R * N >= (1LL << 31)) return set_error(KX_ERR_ARG, "Bloch exchange: chunk too large for one launch");
    BpArgs a;
    a.in = in;
    a.out = out;
    a.n = n;
    a.inner = axis == 1 ? p->n[0] : p->n[0] * p->n[1];
    a.ppi = N / n;
    a.n_cols = R * a.ppi;
    a.Bs = Bs;
    a.f = f;
    a.in_max = in_max;
    a.pmax = pmax;
    a.fmax = fmax;
    a.bound_mul = 1.001f * std::sqrt((float)p->n[0]);  // |mode-1 output| <= sqrt(n1) max|rho|
    a.r0 = r0;
    a.n_orb = n_orb;
    a.out_max = out_max;
    a.ea = ea;
    a.status = p->d_status;
    a.timeout_cycles = 2000000000LL;
    const long long n_tiles = (a.n_cols + 127) / 128;
    if (n_tiles == 0) return KX_OK;
    if (out_max) KX_CUDA_TRY(cudaMemsetAsync(out_max, 0, sizeof(float) * R, s));
    static bool attr = false;  // once per instantiation
    if (!attr) {
        KX_CUDA_TRY(cudaFuncSetAttribute(bloch_pass_kernel<EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bp_smem_bytes(kTcMaxN)));
        attr = true;
    }
    const int grid = (int)std::min<long long>(n_tiles, p->num_sms);
    if (int rc = prof_begin(p, PK_BLOCH, s)) return rc;
    bloch_pass_kernel<EPI><<<grid, kBpThreads, bp_smem_bytes(n), s>>>(a);
    KX_LAUNCH_CHECK("bloch_pass_kernel launch");
    return prof_end(p, s);
}

// Products along axis 1 through bloch_pass0_kernel: n1 = 64 on the tensor cores,
// a multiple of 128 pencils per item, axes 2 and 3 through bloch_pass_kernel
// (whose last inverse product records the maxima this one's scales need).
inline bool bp0_axis(const kx_plan *p) {
    return bp_axes(p) && tc_axis(p, 0) && p->n[0] == 64 && (p->N / 64) % 128 == 0;
}

template <bool FORM>
int launch_bp0(kx_plan *p, long long R, const float2 *in, float2 *out, const __half *Bs, const float2 *P,
               const float2 *F, const float *in_max, const float *pmax, const float *fmax, long long r0, int n_orb,
               cudaStream_t s) {
    const int n = p->n[0];
    const long long N = (long long)p->N;
    if (R * N >= (1LL << 31)) return set_error(KX_ERR_ARG, "Bloch exchange: chunk too large for one launch");
    BpArgs a;
    a.in = in;
    a.out = out;
    a.n = n;
    a.inner = 1;
    a.ppi = N / n;
    a.n_cols = R * a.ppi;
    a.Bs = Bs;
    a.f = nullptr;
    a.in_max = in_max;
    a.pmax = pmax;
    a.fmax = fmax;
    a.bound_mul = 1.001f;  // |rho| <= max|psi_m| max|phi_v|
    a.r0 = r0;
    a.n_orb = n_orb;
    a.out_max = nullptr;
    a.status = p->d_status;
    a.timeout_cycles = 2000000000LL;
    const long long n_tiles = (a.n_cols + 127) / 128;
    if (n_tiles == 0) return KX_OK;
    static bool attr = false;  // once per instantiation
    if (!attr) {
        KX_CUDA_TRY(cudaFuncSetAttribute(bloch_pass0_kernel<FORM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)bp_smem_bytes(kTcMaxN)));
        attr = true;
    }
    const int grid = (int)std::min<long long>(n_tiles, p->num_sms);
    if (int rc = prof_begin(p, PK_BLOCH, s)) return rc;
    bloch_pass0_kernel<FORM><<<grid, kBpThreads, bp_smem_bytes(n), s>>>(a, P, F, N);
    KX_LAUNCH_CHECK("bloch_pass0_kernel launch");
    return prof_end(p, s);
}

// Per-vector maxima of n_vec float32 vectors (vmax zeroed here first).
inline int vector_maxima(kx_plan *p, const float2 *x, long long N, int n_vec, float *vmax, cudaStream_t s) {
    KX_CUDA_TRY(cudaMemsetAsync(vmax, 0, sizeof(float) * n_vec, s));
    const dim3 g((unsigned)std::min<long long>((N + 255) / 256, 64), (unsigned)n_vec);
    bloch_vmax_kernel<<<g, 256, 0, s>>>(x, N, vmax);
    KX_LAUNCH_CHECK("bloch_vmax_kernel launch");
    return KX_OK;
}

// Device workspace of one call: bases, eigenvalues, f table, float32 copies of
// the orbitals and vectors and their maxima (float32 plans), chunk buffers A and
// B and two per-item maximum arrays.
struct BlochLayout {
    size_t Mf[3], Mi[3], lam[3], Bf[3], Bi[3], f, P, F, Pmax, Fmax, mx0, mx1, A, B, partial, total;
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
        // split tensor-core operands (forward, inverse) of the axes that use them
        const size_t bsz = tc_axis(p, a) ? al256(2 * tc_b_bytes(p->n[a])) : 0;
        L.Bf[a] = off;
        off += bsz;
        L.Bi[a] = off;
        off += bsz;
    }
    L.f = off;
    off += al256(sizeof(T) * N);
    const bool f32 = sizeof(T) == 4;
    L.P = off;
    off += f32 ? al256(sizeof(T2) * N * n_orb) : 0;
    L.F = off;
    off += f32 ? al256(sizeof(T2) * N * n_vec) : 0;
    L.Pmax = off;
    off += f32 ? al256(sizeof(float) * n_orb) : 0;
    L.Fmax = off;
    off += f32 ? al256(sizeof(float) * n_vec) : 0;
    L.partial = off;
    off += al256(sizeof(double) * std::max(partial_doubles, 2 * (size_t)p->num_sms * std::max(1, n_kpt)));
    const long long pairs = (long long)n_orb * n_vec;
    const size_t budget = (size_t)2 << 30;  // both chunk buffers
    long long chunk = (long long)std::max<size_t>(1, budget / (2 * sizeof(T2) * N));
    if (const char *e = std::getenv("KX_CHUNK_PAIRS"))  // tuning override (pairs per chunk)
        if (std::atoll(e) > 0) chunk = std::min(chunk, std::atoll(e));
    chunk = std::min(chunk, pairs);
    L.chunk = chunk;
    L.mx0 = off;
    off += f32 ? al256(sizeof(float) * chunk) : 0;
    L.mx1 = off;
    off += f32 ? al256(sizeof(float) * chunk) : 0;
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
__global__ void __launch_bounds__(256, 4) bloch_accum_rev_kernel(const typename Cx<T>::t *__restrict__ X, long long r0, long long r1,
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
        // the vectors v whose item v n_orb + m lies in [r0, r1): a contiguous run
        const long long va = max(v_lo, (r0 - m + n_orb - 1) / n_orb), vb = min(v_hi, (r1 - 1 - m) / n_orb);
        if (r1 - 1 - m < 0 || va > vb) continue;
        // four vectors' loads issued together, the sums still in ascending v
        long long v = va;
        for (; v + 4 <= vb + 1; v += 4) {
            T2 fv[4], xx[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                fv[u] = F[(v + u) * N + x];
                xx[u] = X[((v + u) * n_orb + m - r0) * N + x];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const T c = (T)(wk * (occ_k ? occ_k[v + u] : 1.0));
                sr = fma(c, fv[u].x * xx[u].x + fv[u].y * xx[u].y, sr);  // F conj(X)
                si = fma(c, fv[u].y * xx[u].x - fv[u].x * xx[u].y, si);
            }
        }
        for (; v <= vb; ++v) {
            T2 f1 = F[v * N + x];
            T2 x1 = X[(v * n_orb + m - r0) * N + x];
            T c = (T)(wk * (occ_k ? occ_k[v] : 1.0));
            sr = fma(c, f1.x * x1.x + f1.y * x1.y, sr);
            si = fma(c, f1.y * x1.x - f1.x * x1.y, si);
        }
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
                const double *occ, int k, int q_begin, int q_end, int n_vec, const double *phi, double *out_k,
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
        if (bp_axes(p))
            if (int rc = vector_maxima(p, reinterpret_cast<const float2 *>(Fw), N, n_vec,
                                       reinterpret_cast<float *>(ws + L.Fmax), s))
                return rc;
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
    for (int q = q_begin; q < q_end; ++q) {
        for (int a = 0; a < 3; ++a) ax.theta[a] = theta[3 * k + a] - theta[3 * q + a];
        if (int rc = prof_begin(p, PK_BLOCH_OTHER, s)) return rc;
        bloch_basis_kernel<T><<<dim3(3, 16), 256, 0, s>>>(ax, Mf[0], Mf[1], Mf[2], Mi[0], Mi[1], Mi[2], lam[0], lam[1],
                                                lam[2]);
        KX_LAUNCH_CHECK("bloch_basis_kernel launch");
        bloch_ftable_kernel<T><<<blocks, 256, 0, s>>>(p->n[0], p->n[1], p->n[2], lam[0], lam[1], lam[2], p->kind,
                                                      p->omega, f);
        KX_LAUNCH_CHECK("bloch_ftable_kernel launch");
        if constexpr (sizeof(T) == 4) {
            for (int a = 0; a < 3; ++a) {
                if (!tc_axis(p, a)) continue;
                const int nb = (4 * p->n[a] * p->n[a] + 255) / 256;
                bloch_tc_bsplit_kernel<<<nb, 256, 0, s>>>(Mf[a], p->n[a], reinterpret_cast<__half *>(ws + L.Bf[a]));
                KX_LAUNCH_CHECK("bloch_tc_bsplit_kernel launch");
                bloch_tc_bsplit_kernel<<<nb, 256, 0, s>>>(Mi[a], p->n[a], reinterpret_cast<__half *>(ws + L.Bi[a]));
                KX_LAUNCH_CHECK("bloch_tc_bsplit_kernel launch");
            }
        }
        const T2 *Pq;
        const double2 *psi_q = reinterpret_cast<const double2 *>(psi) + (size_t)q * n_orb * N;
        if (f32) {
            T2 *Pw = reinterpret_cast<T2 *>(ws + L.P);
            bloch_to_f32_kernel<<<blocks, 256, 0, s>>>(psi_q, reinterpret_cast<float2 *>(Pw), N * n_orb);
            KX_LAUNCH_CHECK("bloch_to_f32_kernel launch");
            if (bp_axes(p))
                if (int rc = vector_maxima(p, reinterpret_cast<const float2 *>(Pw), N, n_orb,
                                           reinterpret_cast<float *>(ws + L.Pmax), s))
                    return rc;
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
            if constexpr (sizeof(T) == 4) {
                auto Bf = [&](int a) { return reinterpret_cast<const __half *>(ws + L.Bf[a]); };
                auto Bi = [&](int a) { return reinterpret_cast<const __half *>(ws + L.Bi[a]); };
                if (bp0_axis(p))
                    rc = launch_bp0<true>(p, R, nullptr, A, Bf(0), Pq, F, nullptr, reinterpret_cast<const float *>(ws + L.Pmax),
                                          reinterpret_cast<const float *>(ws + L.Fmax), r0, n_orb, s);
                else
                    rc = tc_axis(p, 0) ? launch_tc<true, 0>(p, 0, R, nullptr, A, Bf(0), nullptr, Pq, F, n_orb, r0, s)
                                       : launch_form<T>(p, R, A, Mf[0], Pq, F, n_orb, r0, s);
                if (rc) return rc;
                if (bp_axes(p)) {
                    // axes 2 and 3 with per-item scales: the bound from the orbital
                    // maxima, then the maxima each product records
                    float *mx0 = reinterpret_cast<float *>(ws + L.mx0), *mx1 = reinterpret_cast<float *>(ws + L.mx1);
                    const float *pm = reinterpret_cast<const float *>(ws + L.Pmax);
                    const float *fm = reinterpret_cast<const float *>(ws + L.Fmax);
                    if ((rc = launch_bp<0>(p, 1, R, A, B, Bf(1), nullptr, nullptr, pm, fm, r0, n_orb, mx0, s))) return rc;
                    if ((rc = launch_bp<1>(p, 2, R, B, A, Bf(2), f, mx0, nullptr, nullptr, 0, n_orb, mx1, s))) return rc;
                    if ((rc = launch_bp<0>(p, 2, R, A, B, Bi(2), nullptr, mx1, nullptr, nullptr, 0, n_orb, mx0, s)))
                        return rc;
                    if ((rc = launch_bp<0>(p, 1, R, B, A, Bi(1), nullptr, mx0, nullptr, nullptr, 0, n_orb,
                                           bp0_axis(p) ? mx1 : nullptr, s)))
                        return rc;
                } else {
                    rc = tc_axis(p, 1)
                             ? launch_tc<false, 0>(p, 1, R, A, B, Bf(1), nullptr, nullptr, nullptr, n_orb, 0, s)
                             : launch_pipe<T, 0>(p, 1, R, A, B, Mf[1], nullptr, s);
                    if (rc) return rc;
                    rc = tc_axis(p, 2) ? launch_tc<false, 1>(p, 2, R, B, A, Bf(2), f, nullptr, nullptr, n_orb, 0, s)
                                       : launch_pipe<T, 1>(p, 2, R, B, A, Mf[2], f, s);
                    if (rc) return rc;
                    rc = tc_axis(p, 2)
                             ? launch_tc<false, 0>(p, 2, R, A, B, Bi(2), nullptr, nullptr, nullptr, n_orb, 0, s)
                             : launch_pipe<T, 0>(p, 2, R, A, B, Mi[2], nullptr, s);
                    if (rc) return rc;
                    rc = tc_axis(p, 1)
                             ? launch_tc<false, 0>(p, 1, R, B, A, Bi(1), nullptr, nullptr, nullptr, n_orb, 0, s)
                             : launch_pipe<T, 0>(p, 1, R, B, A, Mi[1], nullptr, s);
                    if (rc) return rc;
                }
                if (bp0_axis(p))
                    rc = launch_bp0<false>(p, R, A, B, Bi(0), nullptr, nullptr,
                                           reinterpret_cast<const float *>(ws + L.mx1), nullptr, nullptr, 0, n_orb, s);
                else
                    rc = tc_axis(p, 0)
                             ? launch_tc<false, 0>(p, 0, R, A, B, Bi(0), nullptr, nullptr, nullptr, n_orb, 0, s)
                             : launch_pipe<T, 0>(p, 0, R, A, B, Mi[0], nullptr, s);
                if (rc) return rc;
            } else {
                if ((rc = launch_form<T>(p, R, A, Mf[0], Pq, F, n_orb, r0, s))) return rc;
                if ((rc = launch_pipe<T, 0>(p, 1, R, A, B, Mf[1], nullptr, s))) return rc;
                if ((rc = launch_pipe<T, 1>(p, 2, R, B, A, Mf[2], f, s))) return rc;
                if ((rc = launch_pipe<T, 0>(p, 2, R, A, B, Mi[2], nullptr, s))) return rc;
                if ((rc = launch_pipe<T, 0>(p, 1, R, B, A, Mi[1], nullptr, s))) return rc;
                if ((rc = launch_pipe<T, 0>(p, 0, R, A, B, Mi[0], nullptr, s))) return rc;
            }
            if ((rc = prof_begin(p, PK_BLOCH_OTHER, s))) return rc;
            const long long nv = (r1 - 1) / n_orb - r0 / n_orb + 1;
            // float32 sums with an even N: two points per thread (16-byte loads)
            const bool pairs2 = sizeof(T) == 4 && N % 2 == 0;
            const long long per = pairs2 ? 2 : 1;
            const int ab = (int)std::min<long long>((nv * N / per + 255) / 256, 8LL * p->num_sms);
            if constexpr (sizeof(T) == 4) {
                if (pairs2)
                    bloch_accum2_kernel<false><<<ab, 256, 0, s>>>(B, r0, r1, n_orb, Pq, occ_q, wk[q],
                                                                  reinterpret_cast<double2 *>(out_k), N);
            }
            if (!pairs2)
                bloch_accum_kernel<T><<<ab, 256, 0, s>>>(B, r0, r1, n_orb, Pq, occ_q, wk[q],
                                                         reinterpret_cast<double2 *>(out_k), N);
            KX_LAUNCH_CHECK("bloch_accum_kernel launch");
            if (reverse) {
                const int rb = (int)std::min<long long>((n_orb * N / per + 255) / 256, 8LL * p->num_sms);
                double2 *out_q = reinterpret_cast<double2 *>(out_all) + (size_t)q * n_orb * N;
                if constexpr (sizeof(T) == 4) {
                    if (pairs2)
                        bloch_accum2_kernel<true><<<rb, 256, 0, s>>>(B, r0, r1, n_orb, F, occ_k, wk[k], out_q, N);
                }
                if (!pairs2)
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
    return bloch_sweep<T>(p, n_kpt, theta, wk, n_orb, psi, occ, k, 0, n_kpt, n_vec, phi, out, nullptr, s);
}

// Vx psi at every k-point: the pair blocks (k, q) with q >= k are solved once
// and serve both Vx psi_k and, read conjugated, Vx psi_q.
template <typename T>
int bloch_all(kx_plan *p, int n_kpt, const double *theta, const double *wk, int n_orb, const double *psi,
              const double *occ, long long b_begin, long long b_end, double *vx, double *ex, cudaStream_t s) {
    const size_t N = p->N;
    KX_CUDA_TRY(cudaMemsetAsync(vx, 0, sizeof(double2) * N * (size_t)n_orb * n_kpt, s));
    // blocks (k, q), q >= k, numbered k-major: the blocks of row k are
    // [row_start(k), row_start(k) + n_kpt - k)
    long long row_start = 0;
    for (int k = 0; k < n_kpt; ++k) {
        const long long row_end = row_start + (n_kpt - k);
        const long long lo = std::max(b_begin, row_start), hi = std::min(b_end, row_end);
        if (lo < hi) {
            const size_t off = (size_t)k * n_orb * N * 2;
            const int q0 = k + (int)(lo - row_start), q1 = k + (int)(hi - row_start);
            if (int rc = bloch_sweep<T>(p, n_kpt, theta, wk, n_orb, psi, occ, k, q0, q1, n_orb, psi + off, vx + off,
                                        vx, s))
                return rc;
        }
        row_start = row_end;
    }
    if (!ex) return KX_OK;
    // the energy partials live in the plan workspace; an empty block range ran
    // no sweep, so the workspace may still be unsized (or sized for a smaller
    // call): size it here before any kernel writes into it
    BlochLayout L = bloch_layout<T>(p, n_orb, n_orb, n_kpt);
    if (int rc = ensure_workspace(p, L.total)) return rc;
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
            if (bp_axes(p))
                if (int rc = vector_maxima(p, reinterpret_cast<const float2 *>(Fw), N, n_orb,
                                           reinterpret_cast<float *>(ws + L.Fmax), s))
                    return rc;
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
            if constexpr (sizeof(T) == 4) {
                for (int a = 0; a < 3; ++a) {
                    if (!tc_axis(p, a)) continue;
                    const int nb = (4 * p->n[a] * p->n[a] + 255) / 256;
                    bloch_tc_bsplit_kernel<<<nb, 256, 0, s>>>(Mf[a], p->n[a],
                                                              reinterpret_cast<__half *>(ws + L.Bf[a]));
                    KX_LAUNCH_CHECK("bloch_tc_bsplit_kernel launch");
                }
            }
            const T2 *Pq;
            const double2 *psi_q = reinterpret_cast<const double2 *>(psi) + (size_t)q * n_orb * N;
            if (f32) {
                T2 *Pw = reinterpret_cast<T2 *>(ws + L.P);
                bloch_to_f32_kernel<<<blocks, 256, 0, s>>>(psi_q, reinterpret_cast<float2 *>(Pw), N * n_orb);
                KX_LAUNCH_CHECK("bloch_to_f32_kernel launch");
                if (bp_axes(p))
                    if (int rc = vector_maxima(p, reinterpret_cast<const float2 *>(Pw), N, n_orb,
                                               reinterpret_cast<float *>(ws + L.Pmax), s))
                        return rc;
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
                if constexpr (sizeof(T) == 4) {
                    auto Bf = [&](int a) { return reinterpret_cast<const __half *>(ws + L.Bf[a]); };
                    if (bp0_axis(p))
                        rc = launch_bp0<true>(p, R, nullptr, A, Bf(0), Pq, F, nullptr, reinterpret_cast<const float *>(ws + L.Pmax),
                                              reinterpret_cast<const float *>(ws + L.Fmax), r0, n_orb, s);
                    else
                        rc = tc_axis(p, 0) ? launch_tc<true, 0>(p, 0, R, nullptr, A, Bf(0), nullptr, Pq, F, n_orb, r0, s)
                                           : launch_form<T>(p, R, A, Mf[0], Pq, F, n_orb, r0, s);
                    if (rc) return rc;
                    if (bp_axes(p)) {
                        float *mx0 = reinterpret_cast<float *>(ws + L.mx0);
                        const float *pm = reinterpret_cast<const float *>(ws + L.Pmax);
                        const float *fm = reinterpret_cast<const float *>(ws + L.Fmax);
                        if ((rc = launch_bp<0>(p, 1, R, A, B, Bf(1), nullptr, nullptr, pm, fm, r0, n_orb, mx0, s)))
                            return rc;
                        if ((rc = launch_bp<2>(p, 2, R, B, nullptr, Bf(2), f, mx0, nullptr, nullptr, 0, n_orb, nullptr,
                                               s, ea)))
                            return rc;
                    } else {
                        rc = tc_axis(p, 1)
                                 ? launch_tc<false, 0>(p, 1, R, A, B, Bf(1), nullptr, nullptr, nullptr, n_orb, 0, s)
                                 : launch_pipe<T, 0>(p, 1, R, A, B, Mf[1], nullptr, s);
                        if (rc) return rc;
                        rc = tc_axis(p, 2)
                                 ? launch_tc<false, 2>(p, 2, R, B, nullptr, Bf(2), f, nullptr, nullptr, n_orb, 0, s, ea)
                                 : launch_pipe<T, 2>(p, 2, R, B, nullptr, Mf[2], f, s, ea);
                        if (rc) return rc;
                    }
                } else {
                    if ((rc = launch_form<T>(p, R, A, Mf[0], Pq, F, n_orb, r0, s))) return rc;
                    if ((rc = launch_pipe<T, 0>(p, 1, R, A, B, Mf[1], nullptr, s))) return rc;
                    if ((rc = launch_pipe<T, 2>(p, 2, R, B, nullptr, Mf[2], f, s, ea))) return rc;
                }
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
                 const double *occ, long long b_begin, long long b_end, double *vx, double *ex, cudaStream_t s) {
    return p->precision == KX_FP64
               ? bloch_all<double>(p, n_kpt, theta, wk, n_orb, psi, occ, b_begin, b_end, vx, ex, s)
               : bloch_all<float>(p, n_kpt, theta, wk, n_orb, psi, occ, b_begin, b_end, vx, ex, s);
}

int bloch_energy(kx_plan *p, int n_kpt, const double *theta, const double *wk, int n_orb, const double *psi,
                 const double *occ, double *ex, cudaStream_t s) {
    return p->precision == KX_FP64 ? bloch_energy_only<double>(p, n_kpt, theta, wk, n_orb, psi, occ, ex, s)
                                   : bloch_energy_only<float>(p, n_kpt, theta, wk, n_orb, psi, occ, ex, s);
}

}  // namespace kx
